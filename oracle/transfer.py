"""Multigrid transfer operators as explicit sparse matrices (Section 3.2).

Test infrastructure: see ``oracle/__init__.py``.

Generic prolongation P = sum_e S_e P_e G_e (Section 3.2, first equation): G_e
gathers the coarse cell's values, P_e is the elementwise L2-orthogonal
projection P_e = M_e^-1 M_e^{l,l-1} computed in reference space over the fine
cell (Section 3.2, second equation), S_e scatters into the fine vector with the
weight 1/multiplicity of a shared node of a continuous space.  Restriction is
the transpose R = P^T (Section 3.2, third equation).

Here P_e is built literally from 1D mass matrices, M^-1 M^{f,c}, integrated
exactly with a Gauss rule of sufficient degree; the 3D operator is their
Kronecker product.  c-transfer (DG <- FE at equal h, p): P_e = I, shared FE
values are injected into the duplicated DG nodes and restriction sums the
duplicates (Section 3.2, c-coarsening).

Constrained (Dirichlet) FE nodes carry no unknown: prolongation reads zero
there and restriction writes zero there, so P = Z_f P_full Z_c and R = P^T
(Z = the diagonal 0/1 mask of unconstrained nodes).
"""
import numpy as np
import scipy.sparse as sp

from . import basis


def projection_1d(nodes_f, nodes_c, child=None):
    """1D L2 projection M_f^-1 M_fc from the coarse Lagrange basis to the fine one.

    ``child`` None: same interval (p-transfer).  child 0/1: the fine interval is
    the lower/upper half of the coarse one (h-transfer), xi_c = (child + xi_f)/2.
    """
    nf, nc = len(nodes_f), len(nodes_c)
    xq, wq = basis.gauss_legendre(nf + nc + 2)
    Lf = basis.lagrange_values(nodes_f, xq)
    xc = xq if child is None else 0.5 * (child + xq)
    Lc = basis.lagrange_values(nodes_c, xc)
    M = Lf.T @ (wq[:, None] * Lf)
    Mfc = Lf.T @ (wq[:, None] * Lc)
    return np.linalg.solve(M, Mfc)


def _kron3(Px, Py, Pz):
    """3D tensor operator, node index x fastest."""
    return np.kron(Pz, np.kron(Py, Px))


def c_transfer(dg_n, fe):
    """P: FE_p -> DG_p (injection), shape (N_DG, N_FE)."""
    E, n3 = fe.mesh.n_cells, dg_n ** 3
    rows = np.arange(E * n3)
    cols = fe.l2g.ravel()
    P = sp.csr_matrix((np.ones(E * n3), (rows, cols)), shape=(E * n3, fe.n_dofs))
    return P @ sp.diags((~fe.constrained).astype(np.float64))


def fe_transfer(fine, coarse):
    """P: coarse FE space -> fine FE space (p-transfer on one mesh or 2:1 h-transfer)."""
    mf, mc = fine.mesh, coarse.mesh
    if mf.m == mc.m:
        kind = "p"
    elif all(mf.m[d] == 2 * mc.m[d] for d in range(3)):
        kind = "h"
    else:
        raise ValueError("fine mesh must equal or refine the coarse mesh 2:1")
    nf3, nc3 = fine.n ** 3, coarse.n ** 3
    mult = fine.multiplicity()
    cells_f = np.arange(mf.n_cells)
    ijk = mf.cell_ijk(cells_f)
    if kind == "p":
        P1 = projection_1d(fine.nodes, coarse.nodes)
        Pe = {None: _kron3(P1, P1, P1)}
        parent = cells_f
        keys = [None] * mf.n_cells
    else:
        P1 = [projection_1d(fine.nodes, coarse.nodes, child=c) for c in (0, 1)]
        Pe = {}
        for cz in (0, 1):
            for cy in (0, 1):
                for cx in (0, 1):
                    Pe[(cx, cy, cz)] = _kron3(P1[cx], P1[cy], P1[cz])
        parent = mc.cell_index(ijk[:, 0] // 2, ijk[:, 1] // 2, ijk[:, 2] // 2)
        keys = [tuple(int(v) for v in (ijk[e, 0] % 2, ijk[e, 1] % 2, ijk[e, 2] % 2))
                for e in range(mf.n_cells)]
    rows, cols, vals = [], [], []
    for e in range(mf.n_cells):
        gf = fine.l2g[e]
        gc = coarse.l2g[parent[e]]
        blk = Pe[keys[e]] / mult[gf][:, None]
        rows.append(np.repeat(gf, nc3))
        cols.append(np.tile(gc, nf3))
        vals.append(blk.ravel())
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(fine.n_dofs, coarse.n_dofs)).tocsr()
    P.sum_duplicates()
    Zf = sp.diags((~fine.constrained).astype(np.float64))
    Zc = sp.diags((~coarse.constrained).astype(np.float64))
    return (Zf @ P @ Zc).tocsr()


def dg_transfer(fine, coarse):
    """P: coarse DG space -> fine DG space (p-transfer on one mesh or 2:1 h-transfer).

    DG spaces share no nodes, so S_e has no multiplicity weights and P is block
    diagonal over the fine cells: the block of a fine cell is the L2 projection
    of its parent cell's basis (Section 3.2).
    """
    mf, mc = fine.mesh, coarse.mesh
    if mf.m == mc.m:
        kind = "p"
    elif all(mf.m[d] == 2 * mc.m[d] for d in range(3)):
        kind = "h"
    else:
        raise ValueError("fine mesh must equal or refine the coarse mesh 2:1")
    nf3, nc3 = fine.n ** 3, coarse.n ** 3
    rows, cols, vals = [], [], []
    ijk = mf.cell_ijk(np.arange(mf.n_cells))
    if kind == "p":
        P1 = projection_1d(fine.nodes, coarse.nodes)
        blocks = {None: _kron3(P1, P1, P1)}
    else:
        P1 = [projection_1d(fine.nodes, coarse.nodes, child=c) for c in (0, 1)]
        blocks = {(cx, cy, cz): _kron3(P1[cx], P1[cy], P1[cz])
                  for cz in (0, 1) for cy in (0, 1) for cx in (0, 1)}
    for e in range(mf.n_cells):
        if kind == "p":
            parent, key = e, None
        else:
            parent = mc.cell_index(ijk[e, 0] // 2, ijk[e, 1] // 2, ijk[e, 2] // 2)
            key = tuple(int(v) for v in ijk[e] % 2)
        blk = blocks[key]
        rows.append(np.repeat(e * nf3 + np.arange(nf3), nc3))
        cols.append(np.tile(parent * nc3 + np.arange(nc3), nf3))
        vals.append(blk.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(fine.n_dofs, coarse.n_dofs))
