"""SIPG operator on general (unstructured) hexahedral meshes (Section 2; Section 5.3
describes the paper's nozzle and lung meshes: unstructured hexahedra with
Dirichlet and Neumann boundary parts).

Test infrastructure: see ``oracle/__init__.py``.

Mesh description: vertex coordinates V (nv, 3) and cells C (E, 8), local vertex
v = i + 2 j + 4 k sitting at the reference corner (xi_0, xi_1, xi_2) = (i, j, k)
of [0,1]^3.  The cell map is the trilinear interpolant of its 8 vertices; with
``deform`` the analytic deformation x -> x + amp prod_j sin(pi (x_j - lo_j) /
(hi_j - lo_j)) of the box [lo, hi] is applied to the trilinear image and the
result interpolated by the degree-3 tensor Lagrange polynomial on the cell's
GL(3) points, as in ``oracle.mesh``.  Local face f = 2 d + s is the face xi_d =
s; its quadrature points are the n x n Gauss points in the two remaining
reference directions t1 < t2, point index q1 + n q2.  A face whose four vertex
ids occur in no other cell is a boundary face; ``face_bc[e, f]`` gives its
condition (0 Dirichlet, 1 Neumann; ignored on interior faces).

The bilinear form is the one of ``oracle.dg`` (Eqs. WeakFormDG,
InteriorPenaltyFlux1/2, BoundaryConditions, penalty definition of Section 2)
written face by face: on an interior face the cell with the smaller index is
the minus side, n its outward unit normal, [u] = u^- - u^+, {d_n u} the average
of both sides' normal derivatives along n.  Both sides are evaluated at the
same physical points: the minus side's Gauss points, and on the plus side the
Gauss points that the cell map sends to the same positions, found by matching
the physical coordinates of all n^2 points of both faces (no orientation
bookkeeping: the correspondence is read off the geometry).  The area element
and the normal come from the minus side.  Everything is assembled into a CSR
matrix with dense reference tables (small meshes only).
"""
import numpy as np
import scipy.sparse as sp

from . import basis
from .mesh import DIRICHLET


def _face_points(f, xq):
    """Reference points (n^2, 3) of local face f = 2 d + s (xi_d = s), index q1 + n q2."""
    d, s = divmod(f, 2)
    n = len(xq)
    t1, t2 = [t for t in range(3) if t != d]
    pts = np.zeros((n * n, 3))
    q2, q1 = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pts[:, t1] = xq[q1.ravel()]
    pts[:, t2] = xq[q2.ravel()]
    pts[:, d] = float(s)
    return pts


def face_vertices(f):
    """Local vertex numbers of face f = 2 d + s: the corners with bit d equal to s."""
    d, s = divmod(f, 2)
    return [v for v in range(8) if ((v >> d) & 1) == s]


class HexMesh:
    def __init__(self, vertices, cells, face_bc=None, deform=0, amp=0.1, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
        self.V = np.asarray(vertices, dtype=np.float64)
        self.C = np.asarray(cells, dtype=np.int64)
        self.n_cells = len(self.C)
        self.face_bc = (np.zeros((self.n_cells, 6), dtype=np.int64) if face_bc is None
                        else np.asarray(face_bc, dtype=np.int64))
        self.deform, self.amp = int(deform), float(amp)
        self.lo, self.hi = np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)
        self._mnodes = basis.gauss_lobatto(4)
        self._mpts = basis.tensor_points(self._mnodes)
        self._connect()

    def _connect(self):
        """nb[e, f] = (neighbour cell, its local face) or (-1, -1) on the boundary."""
        key = {}
        for e in range(self.n_cells):
            for f in range(6):
                k = tuple(sorted(int(self.C[e, v]) for v in face_vertices(f)))
                key.setdefault(k, []).append((e, f))
        self.nb = -np.ones((self.n_cells, 6, 2), dtype=np.int64)
        for sides in key.values():
            if len(sides) == 2:
                (e1, f1), (e2, f2) = sides
                self.nb[e1, f1] = (e2, f2)
                self.nb[e2, f2] = (e1, f1)
            elif len(sides) > 2:
                raise ValueError("a face shared by more than two cells")

    def trilinear(self, cells, xi):
        """Trilinear images (C, P, 3) of reference points xi (P, 3)."""
        X = self.V[self.C[np.atleast_1d(cells)]]                      # (C, 8, 3)
        w = np.ones((len(xi), 8))
        for v in range(8):
            for a in range(3):
                b = (v >> a) & 1
                w[:, v] *= xi[:, a] if b else 1.0 - xi[:, a]
        return np.einsum("pv,cva->cpa", w, X)

    def analytic_map(self, X):
        if not self.deform:
            return X
        s = np.ones(X.shape[:-1])
        for j in range(3):
            s = s * np.sin(np.pi * (X[..., j] - self.lo[j]) / (self.hi[j] - self.lo[j]))
        return X + self.amp * s[..., None]

    def map(self, cells, xi):
        """Physical points x (C, P, 3) and Jacobians J[c, p, a, b] = dx_a / dxi_b."""
        cells = np.atleast_1d(np.asarray(cells))
        xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
        if not self.deform:
            X = self.V[self.C[cells]]
            P = len(xi)
            x = self.trilinear(cells, xi)
            J = np.zeros((len(cells), P, 3, 3))
            for v in range(8):
                for b in range(3):
                    g = np.ones(P)
                    for a in range(3):
                        bit = (v >> a) & 1
                        if a == b:
                            g = g * (1.0 if bit else -1.0)
                        else:
                            g = g * (xi[:, a] if bit else 1.0 - xi[:, a])
                    J[:, :, :, b] += g[None, :, None] * X[:, v, None, :]
            return x, J
        Xn = self.analytic_map(self.trilinear(cells, self._mpts))     # (C, 64, 3)
        Vb, Gb = basis.tensor_basis(self._mnodes, xi)
        return np.einsum("pm,cma->cpa", Vb, Xn), np.einsum("bpm,cma->cpab", Gb, Xn)


class USIPG:
    """DG Q_k space with the GL nodal basis on a ``HexMesh`` and its SIPG Laplacian."""

    def __init__(self, mesh, k, penalty_factor=1.0):
        self.mesh, self.k, self.n = mesh, int(k), int(k) + 1
        self.penalty_factor = float(penalty_factor)
        n = self.n
        self.nodes = basis.gauss_lobatto(n)
        self.xq, self.wq = basis.gauss_legendre(n)
        self.cpts = basis.tensor_points(self.xq)
        self.cw = basis.tensor_weights(self.wq)
        self.V, self.G = basis.tensor_basis(self.nodes, self.cpts)
        self.wf = np.outer(self.wq, self.wq).ravel()
        self.fpts = [_face_points(f, self.xq) for f in range(6)]
        self.fV, self.fG = [], []
        for f in range(6):
            v, g = basis.tensor_basis(self.nodes, self.fpts[f])
            self.fV.append(v)
            self.fG.append(g)
        self.n_dofs = mesh.n_cells * n ** 3
        self.tau = self._penalty()

    def side(self, e, f):
        """Physical points, area element times weights, outward unit normal and J^-1 at
        the Gauss points of local face f of cell e."""
        x, J = self.mesh.map([e], self.fpts[f])
        x, J = x[0], J[0]
        Jinv = np.linalg.inv(J)
        d, s = divmod(f, 2)
        raw = (2.0 * s - 1.0) * Jinv[:, d, :]                       # J^-T (outward reference normal)
        norm = np.linalg.norm(raw, axis=-1)
        dA = np.abs(np.linalg.det(J)) * norm * self.wf
        return x, dA, raw / norm[:, None], Jinv

    def _penalty(self):
        mesh = self.mesh
        tau = np.zeros(mesh.n_cells)
        for e in range(mesh.n_cells):
            _, J = mesh.map([e], self.cpts)
            vol = float((np.abs(np.linalg.det(J[0])) * self.cw).sum())
            a_int = a_bd = 0.0
            for f in range(6):
                area = float(self.side(e, f)[1].sum())
                if mesh.nb[e, f, 0] >= 0:
                    a_int += area
                else:
                    a_bd += area
            tau[e] = self.penalty_factor * self.n ** 2 * (0.5 * a_int + a_bd) / vol
        return tau

    def matching(self, e1, f1, e2, f2):
        """perm[q] = the plus side's face point at the physical position of the minus side's point q."""
        x1 = self.side(e1, f1)[0]
        x2 = self.side(e2, f2)[0]
        dist = np.linalg.norm(x1[:, None, :] - x2[None, :, :], axis=-1)
        perm = np.argmin(dist, axis=1)
        scale = np.linalg.norm(x1.max(axis=0) - x1.min(axis=0))
        if dist[np.arange(len(perm)), perm].max() > 1e-10 * scale or len(set(perm.tolist())) != len(perm):
            raise ValueError("face points of cells %d and %d do not match" % (e1, e2))
        return perm

    def assemble(self):
        mesh, n3 = self.mesh, self.n ** 3
        N = self.n_dofs
        A = np.zeros((N, N)) if N <= 6000 else None
        if A is None:
            raise ValueError("the unstructured oracle assembles small meshes only")
        loc = np.arange(n3)
        for e in range(mesh.n_cells):
            _, J = mesh.map([e], self.cpts)
            Jinv = np.linalg.inv(J[0])
            jxw = np.abs(np.linalg.det(J[0])) * self.cw
            metric = np.einsum("q,qab,qdb->qad", jxw, Jinv, Jinv)
            A[np.ix_(e * n3 + loc, e * n3 + loc)] += np.einsum("bqi,qbe,eqj->ij", self.G, metric, self.G)
        for e1 in range(mesh.n_cells):
            for f1 in range(6):
                e2, f2 = mesh.nb[e1, f1]
                _, dA, nrm, Ji1 = self.side(e1, f1)
                V1 = self.fV[f1]
                D1 = np.einsum("qb,bqi->qi", np.einsum("qba,qa->qb", Ji1, nrm), self.fG[f1])
                r1 = e1 * n3 + loc
                if e2 < 0:
                    if mesh.face_bc[e1, f1] != DIRICHLET:
                        continue
                    tw = 2.0 * self.tau[e1] * dA
                    A[np.ix_(r1, r1)] += (np.einsum("qi,q,qj->ij", V1, tw, V1)
                                          - np.einsum("qi,q,qj->ij", D1, dA, V1)
                                          - np.einsum("qi,q,qj->ij", V1, dA, D1))
                    continue
                if e2 < e1:
                    continue                                        # visited from the minus side
                perm = self.matching(e1, f1, e2, f2)
                _, _, _, Ji2 = self.side(e2, f2)
                V2 = self.fV[f2][perm]
                D2 = np.einsum("qb,bqi->qi", np.einsum("qba,qa->qb", Ji2[perm], nrm), self.fG[f2][:, perm, :])
                tau = max(self.tau[e1], self.tau[e2]) * dA
                jmp = {0: V1, 1: -V2}
                avg = {0: 0.5 * D1, 1: 0.5 * D2}
                rows = {0: r1, 1: e2 * n3 + loc}
                for a in (0, 1):
                    for b in (0, 1):
                        blk = (np.einsum("qi,q,qj->ij", jmp[a], tau, jmp[b])
                               - np.einsum("qi,q,qj->ij", avg[a], dA, jmp[b])
                               - np.einsum("qi,q,qj->ij", jmp[a], dA, avg[b]))
                        A[np.ix_(rows[a], rows[b])] += blk
        return sp.csr_matrix(A)

    def apply(self, u):
        return self.assemble() @ np.asarray(u, dtype=np.float64)
