"""Continuous FE Laplacian a(v,u) = (grad v, grad u) (Section 2, Eq. WeakFormFE).

Test infrastructure: see ``oracle/__init__.py``.

Space: continuous Q_p on the same hexahedral mesh, nodes at the GL points of
each cell, global node grid of (m0 p+1) x (m1 p+1) x (m2 p+1) points numbered
lexicographically (x fastest).  Dirichlet conditions are imposed strongly: the
nodes on Dirichlet sides are constrained and kept in the system with a unit
diagonal (Section 2, "constrained degrees of freedom are kept in the system with
diagonal entries set to 1"); only the homogeneous operator is needed inside the
multigrid cycle.  Integrals use the (p+1)-point Gauss rule and the cell's own
mapping, evaluated with dense reference tables.
"""
import numpy as np
import scipy.sparse as sp

from . import basis
from .mesh import DIRICHLET


class FESpace:
    def __init__(self, mesh, p, chunk=4096):
        if p < 1:
            raise ValueError("degree >= 1")
        self.mesh, self.p, self.n = mesh, int(p), int(p) + 1
        self.chunk = chunk
        n = self.n
        self.nodes = basis.gauss_lobatto(n)
        xq, wq = basis.gauss_legendre(n)
        self.cpts = basis.tensor_points(xq)
        self.cw = basis.tensor_weights(wq)
        self.V, self.G = basis.tensor_basis(self.nodes, self.cpts)
        self.grid = tuple(mesh.m[d] * self.p + 1 for d in range(3))
        self.n_dofs = self.grid[0] * self.grid[1] * self.grid[2]
        self.l2g = self._local_to_global()
        self.constrained = self._constrained()

    def _local_to_global(self):
        """(E, n^3) global node of local node (a,b,c) of cell (i,j,k)."""
        mesh, p, n = self.mesh, self.p, self.n
        ijk = mesh.cell_ijk(np.arange(mesh.n_cells))
        c, b, a = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        a, b, c = a.ravel(), b.ravel(), c.ravel()
        gx = ijk[:, 0:1] * p + a[None, :]
        gy = ijk[:, 1:2] * p + b[None, :]
        gz = ijk[:, 2:3] * p + c[None, :]
        Nx, Ny, _ = self.grid
        return gx + Nx * (gy + Ny * gz)

    def node_coords(self):
        Nx, Ny, Nz = self.grid
        g = np.arange(self.n_dofs)
        return np.stack([g % Nx, (g // Nx) % Ny, g // (Nx * Ny)], axis=1)

    def _constrained(self):
        """Boolean mask of nodes on Dirichlet sides."""
        gi = self.node_coords()
        mask = np.zeros(self.n_dofs, bool)
        for d in range(3):
            if self.mesh.bc[2 * d] == DIRICHLET:
                mask |= gi[:, d] == 0
            if self.mesh.bc[2 * d + 1] == DIRICHLET:
                mask |= gi[:, d] == self.grid[d] - 1
        return mask

    def multiplicity(self):
        """Number of cells sharing each global node."""
        return np.bincount(self.l2g.ravel(), minlength=self.n_dofs).astype(np.float64)

    def cell_metric(self, cells):
        _, J = self.mesh.map(cells, self.cpts)
        Jinv = np.linalg.inv(J)
        jxw = np.abs(np.linalg.det(J)) * self.cw[None, :]
        return np.einsum("cq,cqab,cqdb->cqad", jxw, Jinv, Jinv)

    def cell_matrices(self, cells):
        return np.einsum("bqi,cqbe,eqj->cij", self.G, self.cell_metric(cells), self.G)

    def assemble(self, constrain=True):
        """Global CSR matrix; constrained rows/columns replaced by identity."""
        rows, cols, vals = [], [], []
        E, n3 = self.mesh.n_cells, self.n ** 3
        for c0 in range(0, E, self.chunk):
            cs = np.arange(c0, min(E, c0 + self.chunk))
            Ae = self.cell_matrices(cs)
            g = self.l2g[cs]
            rows.append(np.repeat(g[:, :, None], n3, axis=2).ravel())
            cols.append(np.repeat(g[:, None, :], n3, axis=1).ravel())
            vals.append(Ae.ravel())
        N = self.n_dofs
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(N, N)).tocsr()
        A.sum_duplicates()
        if constrain:
            keep = sp.diags((~self.constrained).astype(np.float64))
            A = (keep @ A @ keep + sp.diags(self.constrained.astype(np.float64))).tocsr()
        return A

    def apply(self, u):
        """Matrix-free v = A u with the same constraint treatment as ``assemble``."""
        u = np.asarray(u, dtype=np.float64)
        uu = np.where(self.constrained, 0.0, u)
        v = np.zeros(self.n_dofs)
        E = self.mesh.n_cells
        for c0 in range(0, E, self.chunk):
            cs = np.arange(c0, min(E, c0 + self.chunk))
            g = self.l2g[cs]
            grad = np.einsum("bqi,ci->cqb", self.G, uu[g])
            flux = np.einsum("cqab,cqb->cqa", self.cell_metric(cs), grad)
            np.add.at(v, g.ravel(), np.einsum("bqi,cqb->ci", self.G, flux).ravel())
        v[self.constrained] = u[self.constrained]
        return v

    def diagonal(self):
        d = np.zeros(self.n_dofs)
        E = self.mesh.n_cells
        for c0 in range(0, E, self.chunk):
            cs = np.arange(c0, min(E, c0 + self.chunk))
            de = np.einsum("bqi,cqbe,eqi->ci", self.G, self.cell_metric(cs), self.G)
            np.add.at(d, self.l2g[cs].ravel(), de.ravel())
        d[self.constrained] = 1.0
        return d
