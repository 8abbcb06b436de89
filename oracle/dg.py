"""SIPG discretization of -lap(u) = f on hexahedra (Section 2 of the paper).

Test infrastructure: see ``oracle/__init__.py``.

What is computed (the paper's Section 2, Eqs. WeakFormDG, InteriorPenaltyFlux1/2,
BoundaryConditions and the penalty definition after them), written with [u] =
u^- - u^+, the face normal n = outward normal of the lower cell e^- and
{d_n u} = (grad u^- + grad u^+).n / 2:

    a(v,u) = sum_e int_e grad v . grad u
           + sum_{interior f} int_f ( -{d_n v}[u] - [v]{d_n u} + tau_f [v][u] )
           + sum_{Dirichlet f} int_f ( -d_n v u - v d_n u + 2 tau_e v u )
           + sum_{Neumann f} 0

The interior term is the sum of the paper's face terms -(grad v,(u-u*)n) -
(v, sigma*.n) over both sides with u* = {u}, sigma* = {grad u} - tau [[u]].  The
Dirichlet term follows from the mirror principle u^+ = -u^- (homogeneous part),
grad u^+ . n = grad u^- . n, which gives {u} = 0 and [[u]] = 2 u^- n, hence the
factor 2 tau_e.  The Neumann mirror u^+ = u^-, grad u^+.n = -grad u^-.n makes
both face terms vanish.  Penalty: tau_e = (p+1)^2 (A(dOmega_e \\ Gamma)/2 +
A(dOmega_e cap Gamma)) / V(Omega_e); tau_f = max(tau_e-, tau_e+) on interior
faces and tau_e on boundary faces; all areas and volumes by the operator's own
(p+1)-point Gauss rules.

Integrals use (p+1)-point Gauss-Legendre rules in each direction on cells and
faces, evaluated here with full (non sum-factorised) dense reference basis
tables: the plain definition, no blocking or reordering.

Two evaluation modes, checked equal in the tests:
* ``assemble()`` builds the global CSR matrix from element and face matrices;
* ``apply(u)`` evaluates A u cell by cell and face by face with the same dense
  reference tables (for meshes whose matrix would not fit in memory).
"""
import numpy as np
import scipy.sparse as sp

from . import basis
from .mesh import DIRICHLET, NEUMANN


def _face_points(d, side_upper_cell, xq):
    """Reference points (n^2, 3) of the face normal to d on one side.

    For the lower cell the face is xi_d = 1, for the upper cell xi_d = 0.
    Face point index qf = q1 + n*q2 over the tangential directions t1 < t2.
    """
    n = len(xq)
    t1, t2 = [t for t in range(3) if t != d]
    pts = np.zeros((n * n, 3))
    q2, q1 = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pts[:, t1] = xq[q1.ravel()]
    pts[:, t2] = xq[q2.ravel()]
    pts[:, d] = 0.0 if side_upper_cell else 1.0
    return pts


class SIPG:
    """DG Q_p space with GL nodal basis on a ``Mesh`` and its SIPG Laplacian."""

    def __init__(self, mesh, k, penalty_factor=1.0, chunk=4096):
        if k < 1:
            raise ValueError("degree >= 1")
        self.mesh, self.k, self.n = mesh, int(k), int(k) + 1
        self.penalty_factor = float(penalty_factor)
        self.chunk = chunk
        n = self.n
        self.nodes = basis.gauss_lobatto(n)
        self.xq, self.wq = basis.gauss_legendre(n)
        self.cpts = basis.tensor_points(self.xq)
        self.cw = basis.tensor_weights(self.wq)
        self.V, self.G = basis.tensor_basis(self.nodes, self.cpts)
        self.wf = np.outer(self.wq, self.wq).ravel()  # index q1 + n*q2 -> w[q1] w[q2]
        self.fV, self.fG = {}, {}
        for d in range(3):
            for s in (0, 1):  # 0: lower cell (xi_d=1), 1: upper cell (xi_d=0)
                self.fV[d, s], self.fG[d, s] = basis.tensor_basis(
                    self.nodes, _face_points(d, s == 1, self.xq))
        self.n_dofs = mesh.n_cells * n ** 3
        self._tau = None

    @property
    def tau(self):
        """tau_e of every cell (computed on first use)."""
        if self._tau is None:
            self._tau = self._penalty()
        return self._tau

    def tau_of(self, cells):
        """tau_e of the given cells only (each cell's value depends on that cell alone)."""
        cells = np.asarray(cells)
        if self._tau is None and len(cells) > self.mesh.n_cells // 4:
            return self.tau[cells]
        if self._tau is not None:
            return self._tau[cells]
        uniq, inv = np.unique(cells, return_inverse=True)
        return self._penalty(uniq)[inv]

    # ---------------------------------------------------------------- geometry
    def cell_geometry(self, cells):
        """JxW (C,Q) and metric M = JxW J^-1 J^-T (C,Q,3,3) at cell Gauss points."""
        _, J = self.mesh.map(cells, self.cpts)
        det = np.linalg.det(J)
        Jinv = np.linalg.inv(J)
        jxw = np.abs(det) * self.cw[None, :]
        metric = np.einsum("cq,cqab,cqdb->cqad", jxw, Jinv, Jinv)
        return jxw, metric

    def _side_geometry(self, cells, d, s):
        """|det J| and J^-1 at the face points of side s of the given cells."""
        pts = _face_points(d, s == 1, self.xq)
        _, J = self.mesh.map(cells, pts)
        return np.abs(np.linalg.det(J)), np.linalg.inv(J)

    def face_geometry(self, d, LU):
        """Canonical data of faces normal to d; LU rows are (lower, upper) cells.

        Returns dA (F,n^2) = area element times face weights, nrm (F,n^2,3) =
        unit normal pointing out of the lower cell (out of the only cell on a
        boundary face), and c[s] (F,n^2,3) = J_s^-1 nrm for each present side,
        so that the normal derivative is d_n u = sum_b c_b d u/d xi_b.  The
        geometry is taken from the lower cell when it exists.
        """
        F = len(LU)
        nq = self.n ** 2
        dA = np.zeros((F, nq))
        nrm = np.zeros((F, nq, 3))
        c = {0: np.zeros((F, nq, 3)), 1: np.zeros((F, nq, 3))}
        has_lo = LU[:, 0] >= 0
        for s, sel in ((0, has_lo), (1, ~has_lo)):
            if not np.any(sel):
                continue
            cells = LU[sel, s]
            adet, Jinv = self._side_geometry(cells, d, s)
            raw = Jinv[:, :, d, :]                      # J^-T e_d (row d of J^-1)
            norm = np.linalg.norm(raw, axis=-1)
            sign = 1.0 if s == 0 else -1.0
            nrm[sel] = sign * raw / norm[..., None]
            dA[sel] = adet * norm * self.wf[None, :]
        for s in (0, 1):
            sel = LU[:, s] >= 0
            if np.any(sel):
                _, Jinv = self._side_geometry(LU[sel, s], d, s)
                c[s][sel] = np.einsum("fqba,fqa->fqb", Jinv, nrm[sel])
        return dA, nrm, c

    def _penalty(self, which=None):
        """tau_e per cell (penalty definition in Section 2) times the factor."""
        mesh = self.mesh
        which = np.arange(mesh.n_cells) if which is None else np.asarray(which)
        E = len(which)
        vol = np.zeros(E)
        a_int = np.zeros(E)
        a_bdry = np.zeros(E)
        for c0 in range(0, E, self.chunk):
            loc = np.arange(c0, min(E, c0 + self.chunk))
            cells = which[loc]
            jxw, _ = self.cell_geometry(cells)
            vol[loc] = jxw.sum(axis=1)
            ijk = mesh.cell_ijk(cells)
            for d in range(3):
                for s in (0, 1):  # s=0: face at xi_d=1 (upper side), s=1: xi_d=0
                    adet, Jinv = self._side_geometry(cells, d, s)
                    area = (adet * np.linalg.norm(Jinv[:, :, d, :], axis=-1)
                            * self.wf[None, :]).sum(axis=1)
                    on_bdry = (ijk[:, d] == mesh.m[d] - 1) if s == 0 else (ijk[:, d] == 0)
                    a_bdry[loc] += np.where(on_bdry, area, 0.0)
                    a_int[loc] += np.where(on_bdry, 0.0, area)
        return self.penalty_factor * (self.k + 1) ** 2 * (0.5 * a_int + a_bdry) / vol

    # ------------------------------------------------------ local operators
    def _face_blocks(self, d, LU):
        """Per-face operators: values V_s (n^2,n^3) shared, and geometry data."""
        dA, nrm, c = self.face_geometry(d, LU)
        return dA, c

    def cell_matrices(self, cells):
        _, metric = self.cell_geometry(cells)
        return np.einsum("bqi,cqbe,eqj->cij", self.G, metric, self.G)

    def _dn_matrix(self, d, s, c):
        """Normal-derivative tables (F,n^2,n^3): sum_b c_b dN/dxi_b at face points."""
        return np.einsum("fqb,bqi->fqi", c, self.fG[d, s])

    # -------------------------------------------------------------- assembly
    def assemble(self):
        """Global CSR matrix A (homogeneous part only, Section 2)."""
        mesh, n3 = self.mesh, self.n ** 3
        rows, cols, vals = [], [], []
        loc = np.arange(n3)

        def add(block, rdofs, cdofs):
            rows.append(np.repeat(rdofs[:, :, None], cdofs.shape[1], axis=2).ravel())
            cols.append(np.repeat(cdofs[:, None, :], rdofs.shape[1], axis=1).ravel())
            vals.append(block.ravel())

        for c0 in range(0, mesh.n_cells, self.chunk):
            cells = np.arange(c0, min(mesh.n_cells, c0 + self.chunk))
            dofs = cells[:, None] * n3 + loc[None, :]
            add(self.cell_matrices(cells), dofs, dofs)
        for d in range(3):
            LU = mesh.faces(d)
            dA, c = self._face_blocks(d, LU)
            inner = (LU[:, 0] >= 0) & (LU[:, 1] >= 0)
            if np.any(inner):
                L, U = LU[inner, 0], LU[inner, 1]
                w = dA[inner]
                tau = np.maximum(self.tau[L], self.tau[U])[:, None] * w
                VL, VU = self.fV[d, 0], self.fV[d, 1]
                DL = self._dn_matrix(d, 0, c[0][inner])
                DU = self._dn_matrix(d, 1, c[1][inner])
                # jump operator [VL, -VU], average normal derivative (DL + DU)/2
                jmp = {0: np.broadcast_to(VL, DL.shape), 1: -np.broadcast_to(VU, DU.shape)}
                avg = {0: 0.5 * DL, 1: 0.5 * DU}
                cells = {0: L, 1: U}
                for a in (0, 1):
                    for b in (0, 1):
                        blk = (np.einsum("fqi,fq,fqj->fij", jmp[a], tau, jmp[b])
                               - np.einsum("fqi,fq,fqj->fij", avg[a], w, jmp[b])
                               - np.einsum("fqi,fq,fqj->fij", jmp[a], w, avg[b]))
                        add(blk, cells[a][:, None] * n3 + loc, cells[b][:, None] * n3 + loc)
            for s in (0, 1):
                sel = (LU[:, s] >= 0) & (LU[:, 1 - s] < 0)
                if not np.any(sel) or mesh.side_bc(d, upper=(s == 0)) != DIRICHLET:
                    continue
                cell = LU[sel, s]
                w = dA[sel]
                Vs = np.broadcast_to(self.fV[d, s], (len(cell),) + self.fV[d, s].shape)
                Ds = self._dn_matrix(d, s, c[s][sel])
                tw = 2.0 * self.tau[cell][:, None] * w
                blk = (np.einsum("fqi,fq,fqj->fij", Vs, tw, Vs)
                       - np.einsum("fqi,fq,fqj->fij", Ds, w, Vs)
                       - np.einsum("fqi,fq,fqj->fij", Vs, w, Ds))
                dofs = cell[:, None] * n3 + loc
                add(blk, dofs, dofs)
        N = self.n_dofs
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(N, N)).tocsr()
        A.sum_duplicates()
        return A

    # --------------------------------------------------- matrix-free (naive)
    def apply(self, u, cells=None):
        """v = A u with dense reference tables, cell by cell and face by face.

        With ``cells`` given, only the rows of those cells are computed (the rest
        of v is zero); u must still be the full vector.
        """
        mesh, n3 = self.mesh, self.n ** 3
        U = np.asarray(u, dtype=np.float64).reshape(mesh.n_cells, n3)
        Vout = np.zeros_like(U)
        want = np.ones(mesh.n_cells, bool) if cells is None else np.zeros(mesh.n_cells, bool)
        if cells is not None:
            want[np.asarray(cells)] = True
        todo = np.nonzero(want)[0]
        for c0 in range(0, len(todo), self.chunk):
            cs = todo[c0:c0 + self.chunk]
            _, metric = self.cell_geometry(cs)
            grad = np.einsum("bqi,ci->cqb", self.G, U[cs])
            flux = np.einsum("cqab,cqb->cqa", metric, grad)
            Vout[cs] += np.einsum("bqi,cqb->ci", self.G, flux)
        for d in range(3):
            if cells is None:
                LU = mesh.faces(d)
            else:
                LU = mesh.faces_of_cells(d, todo)
            if len(LU) == 0:
                continue
            dA, c = self._face_blocks(d, LU)
            vals, dns = {}, {}
            for s in (0, 1):
                ok = LU[:, s] >= 0
                vals[s] = np.zeros(dA.shape)
                dns[s] = np.zeros(dA.shape)
                if np.any(ok):
                    Us = U[LU[ok, s]]
                    vals[s][ok] = Us @ self.fV[d, s].T
                    gref = np.einsum("bqi,fi->fqb", self.fG[d, s], Us)
                    dns[s][ok] = np.einsum("fqb,fqb->fq", c[s][ok], gref)
            inner = (LU[:, 0] >= 0) & (LU[:, 1] >= 0)
            if np.any(inner):
                L, U_ = LU[inner, 0], LU[inner, 1]
                w = dA[inner]
                tau = np.maximum(self.tau_of(L), self.tau_of(U_))[:, None]
                jump = vals[0][inner] - vals[1][inner]
                avg = 0.5 * (dns[0][inner] + dns[1][inner])
                val_coef = w * (-avg + tau * jump)    # multiplies [v]
                dn_coef = w * (-0.5 * jump)           # multiplies d_n v (each side)
                for s, cells_s, sgn in ((0, L, 1.0), (1, U_, -1.0)):
                    m = want[cells_s]
                    if not np.any(m):
                        continue
                    contrib = sgn * val_coef[m] @ self.fV[d, s]
                    contrib += np.einsum("fq,fqb,bqi->fi", dn_coef[m], c[s][inner][m], self.fG[d, s])
                    np.add.at(Vout, cells_s[m], contrib)
            for s in (0, 1):
                sel = (LU[:, s] >= 0) & (LU[:, 1 - s] < 0)
                if not np.any(sel) or mesh.side_bc(d, upper=(s == 0)) != DIRICHLET:
                    continue
                cell = LU[sel, s]
                m = want[cell]
                w = dA[sel][m]
                uu, qq = vals[s][sel][m], dns[s][sel][m]
                tau = self.tau_of(cell[m])[:, None]
                contrib = (w * (-qq + 2.0 * tau * uu)) @ self.fV[d, s]
                contrib += np.einsum("fq,fqb,bqi->fi", w * (-uu), c[s][sel][m], self.fG[d, s])
                np.add.at(Vout, cell[m], contrib)
        return Vout.ravel()

    def diagonal(self):
        """diag(A) from the element and face self-coupling blocks."""
        return self.assemble().diagonal() if self.n_dofs <= 200000 else self._diag_blocks()

    def _diag_blocks(self):
        mesh, n3 = self.mesh, self.n ** 3
        D = np.zeros((mesh.n_cells, n3))
        for c0 in range(0, mesh.n_cells, self.chunk):
            cs = np.arange(c0, min(mesh.n_cells, c0 + self.chunk))
            _, metric = self.cell_geometry(cs)
            D[cs] += np.einsum("bqi,cqbe,eqi->ci", self.G, metric, self.G)
        for d in range(3):
            LU = mesh.faces(d)
            dA, c = self._face_blocks(d, LU)
            inner = (LU[:, 0] >= 0) & (LU[:, 1] >= 0)
            for s in (0, 1):
                has = LU[:, s] >= 0
                bd = has & (LU[:, 1 - s] < 0)
                for sel, kind in ((has & inner, 0), (bd, 1)):
                    if not np.any(sel):
                        continue
                    if kind == 1 and mesh.side_bc(d, upper=(s == 0)) != DIRICHLET:
                        continue
                    cell = LU[sel, s]
                    w = dA[sel]
                    Vs = self.fV[d, s]
                    Ds = self._dn_matrix(d, s, c[s][sel])
                    if kind == 0:
                        # c[1] is taken along the lower cell's outward normal,
                        # which points into the upper cell: flip its sign
                        sgn = -1.0 if s == 0 else 1.0
                        tau = np.maximum(self.tau[LU[sel, 0]], self.tau[LU[sel, 1]])[:, None]
                        dd = (np.einsum("fq,qi->fi", tau * w, Vs * Vs)
                              + sgn * np.einsum("fq,fqi,qi->fi", w, Ds, Vs))
                    else:
                        tau = self.tau[cell][:, None]
                        dd = (np.einsum("fq,qi->fi", 2.0 * tau * w, Vs * Vs)
                              - 2.0 * np.einsum("fq,fqi,qi->fi", w, Ds, Vs))
                    np.add.at(D, cell, dd)
        return D.ravel()

    # ------------------------------------------------------------ problem data
    def rhs(self, f, g=None, h=None):
        """b_i = int f N_i + sum_Dir int (-d_n N_i + 2 tau_e N_i) g + sum_Neu int N_i h.

        f, g, h are callables of physical points (..., 3).  The inhomogeneous
        split of Section 2 puts g and h only into the right-hand side.
        """
        mesh, n3 = self.mesh, self.n ** 3
        B = np.zeros((mesh.n_cells, n3))
        for c0 in range(0, mesh.n_cells, self.chunk):
            cs = np.arange(c0, min(mesh.n_cells, c0 + self.chunk))
            x, _ = mesh.map(cs, self.cpts)
            jxw, _ = self.cell_geometry(cs)
            B[cs] += (f(x) * jxw) @ self.V
        for d in range(3):
            LU = mesh.faces(d)
            for s in (0, 1):
                sel = (LU[:, s] >= 0) & (LU[:, 1 - s] < 0)
                if not np.any(sel):
                    continue
                kind = mesh.side_bc(d, upper=(s == 0))
                sub = LU[sel]
                dA, c = self._face_blocks(d, sub)
                cell = sub[:, s]
                x, _ = mesh.map(cell, _face_points(d, s == 1, self.xq))
                if kind == DIRICHLET and g is not None:
                    gv = g(x) * dA
                    tau = self.tau[cell][:, None]
                    contrib = (2.0 * tau * gv) @ self.fV[d, s]
                    contrib -= np.einsum("fq,fqb,bqi->fi", gv, c[s], self.fG[d, s])
                    np.add.at(B, cell, contrib)
                elif kind == NEUMANN and h is not None:
                    np.add.at(B, cell, (h(x) * dA) @ self.fV[d, s])
        return B.ravel()

    def interpolate(self, func):
        """Nodal interpolant I_h u: values of u at the mapped GL nodes."""
        mesh = self.mesh
        x, _ = mesh.map(np.arange(mesh.n_cells), basis.tensor_points(self.nodes))
        return func(x).ravel()

    def l2_error(self, u, func):
        """|| u_h - u ||_L2 with an (n+2)-point Gauss rule per direction."""
        mesh, n3 = self.mesh, self.n ** 3
        xq, wq = basis.gauss_legendre(self.n + 2)
        pts, w = basis.tensor_points(xq), basis.tensor_weights(wq)
        V, _ = basis.tensor_basis(self.nodes, pts)
        U = np.asarray(u).reshape(mesh.n_cells, n3)
        err = 0.0
        for c0 in range(0, mesh.n_cells, self.chunk):
            cs = np.arange(c0, min(mesh.n_cells, c0 + self.chunk))
            x, J = mesh.map(cs, pts)
            jxw = np.abs(np.linalg.det(J)) * w[None, :]
            diff = U[cs] @ V.T - func(x)
            err += float(np.sum(diff * diff * jxw))
        return np.sqrt(err)
