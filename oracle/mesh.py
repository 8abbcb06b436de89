"""Structured hexahedral box mesh and element mapping (Section 2; Section 5.3).

Test infrastructure: see ``oracle/__init__.py``.

Cells of an m0 x m1 x m2 box [lo, hi] are numbered lexicographically,
e = i0 + m0*(i1 + m1*i2).  Each cell is the image of the reference cell [0,1]^3
under x(xi).  Cartesian: the affine map.  Curvilinear: the degree-3 tensor
Lagrange interpolant (on the degree-3 GL points of the cell) of the analytic
deformation x_i <- x_i + a * prod_j sin(pi (x_j - lo_j)/(hi_j - lo_j)); the paper
uses degree-3 element mappings for its deformed cube (Section 5.3).  The
sine factors vanish on the box boundary, so boundary faces stay planar.
"""
import numpy as np

from . import basis

# box sides in the order -x, +x, -y, +y, -z, +z
DIRICHLET, NEUMANN = 0, 1


class Mesh:
    def __init__(self, m, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), deform=0,
                 amp=0.1, mapping_degree=3, bc=(0, 0, 0, 0, 0, 0)):
        self.m = tuple(int(v) for v in (m if np.ndim(m) else (m, m, m)))
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)
        self.deform = int(deform)
        self.amp = float(amp)
        self.mapping_degree = int(mapping_degree)
        self.bc = tuple(int(b) for b in bc)
        self.n_cells = self.m[0] * self.m[1] * self.m[2]
        self.h = (self.hi - self.lo) / np.asarray(self.m, dtype=np.float64)
        if self.deform:
            q = self.mapping_degree
            self._mnodes = basis.gauss_lobatto(q + 1)
            self._mpts = basis.tensor_points(self._mnodes)

    def cell_ijk(self, e):
        e = np.asarray(e)
        m0, m1, _ = self.m
        return np.stack([e % m0, (e // m0) % m1, e // (m0 * m1)], axis=-1)

    def cell_index(self, i, j, k):
        return i + self.m[0] * (j + self.m[1] * k)

    def analytic_map(self, X):
        """The exact deformation of points X (..., 3) of the undeformed box."""
        if not self.deform:
            return np.array(X, dtype=np.float64)
        s = np.ones(X.shape[:-1])
        for j in range(3):
            s = s * np.sin(np.pi * (X[..., j] - self.lo[j]) / (self.hi[j] - self.lo[j]))
        return X + self.amp * s[..., None]

    def affine(self, cells, xi):
        """Undeformed position of reference points xi (P,3) in cells: (C,P,3)."""
        ijk = self.cell_ijk(np.asarray(cells))
        return self.lo + (ijk[:, None, :] + xi[None, :, :]) * self.h

    def map(self, cells, xi):
        """Physical points x (C,P,3) and Jacobians J[c,p,a,b] = dx_a/dxi_b."""
        cells = np.atleast_1d(np.asarray(cells))
        xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
        C, P = len(cells), len(xi)
        if not self.deform:
            x = self.affine(cells, xi)
            J = np.zeros((C, P, 3, 3))
            for a in range(3):
                J[:, :, a, a] = self.h[a]
            return x, J
        # nodal values of the analytic map at the cell's mapping-support points
        Xn = self.analytic_map(self.affine(cells, self._mpts))        # (C, (q+1)^3, 3)
        V, G = basis.tensor_basis(self._mnodes, xi)                   # (P, M), (3, P, M)
        x = np.einsum("pm,cma->cpa", V, Xn)
        J = np.einsum("bpm,cma->cpab", G, Xn)
        return x, J

    # --- face bookkeeping -------------------------------------------------
    def tangential(self, d):
        """The two tangential directions of a face normal to d, ascending."""
        return [t for t in range(3) if t != d]

    def faces_of_cells(self, d, cells):
        """(lower, upper) rows of the faces normal to d that touch the given cells."""
        m = self.m
        ijk = self.cell_ijk(np.asarray(cells))
        rows = set()
        for c, (i, j, k) in zip(np.asarray(cells), ijk):
            for up in (0, 1):
                a = [int(i), int(j), int(k)]
                if up:
                    lo_c = int(c)
                    a[d] += 1
                    up_c = self.cell_index(*a) if a[d] < m[d] else -1
                else:
                    up_c = int(c)
                    a[d] -= 1
                    lo_c = self.cell_index(*a) if a[d] >= 0 else -1
                rows.add((lo_c, up_c))
        return np.array(sorted(rows), dtype=np.int64).reshape(-1, 2)

    def faces(self, d):
        """All faces normal to direction d as (lower cell or -1, upper cell or -1).

        Planes are numbered 0..m_d; plane 0 and plane m_d are boundary faces.
        Faces are listed plane-major, then lexicographically in the tangential
        cell indices (t1 fastest).
        """
        m = self.m
        t1, t2 = self.tangential(d)
        out = []
        for p in range(m[d] + 1):
            for b in range(m[t2]):
                for a in range(m[t1]):
                    ijk_lo = [0, 0, 0]
                    ijk_lo[d], ijk_lo[t1], ijk_lo[t2] = p - 1, a, b
                    ijk_up = list(ijk_lo)
                    ijk_up[d] = p
                    lo_c = self.cell_index(*ijk_lo) if p > 0 else -1
                    up_c = self.cell_index(*ijk_up) if p < m[d] else -1
                    out.append((lo_c, up_c))
        return np.array(out, dtype=np.int64).reshape(-1, 2)

    def side_bc(self, d, upper):
        return self.bc[2 * d + (1 if upper else 0)]
