"""Smoothed-aggregation algebraic multigrid and the AMG-preconditioned CG used as
the coarse-grid solver (Section 3.3, "Coarse-grid solver").

Test infrastructure: see ``oracle/__init__.py``.

The paper solves its coarsest level (the FE_1 matrix on the coarse mesh) with
CG preconditioned by one V-cycle of a smoothed-aggregation AMG (Trilinos ML)
to a relative tolerance, 1e-3 here.  This module writes that solver out from
the textbook definition of smoothed aggregation (Vanek, Mandel, Brezina,
"Algebraic multigrid by smoothed aggregation for second and fourth order
elliptic problems", Computing 56, 1996), for a symmetric positive definite CSR
matrix A_0 whose constrained rows are identity rows:

1. Strength of connection.  j != i is a strong neighbour of i when
   |a_ij| > theta sqrt(a_ii a_jj), theta = 0.02.  A node without strong
   neighbours (an identity row, for one) is isolated and joins no aggregate.
2. Aggregation, three passes over the nodes in index order:
   (1) a node that is not isolated and none of whose strong neighbours is
       aggregated yet starts an aggregate with all its strong neighbours;
   (2) every node still free joins the aggregate of its strongest aggregated
       neighbour (largest |a_ij|; among values within a relative 1e-12 of the
       largest, which are ties up to the order of summation, the smallest j),
       aggregates as they stood after pass 1;
   (3) every node still free starts an aggregate with its free strong
       neighbours.
3. Tentative prolongator P~: one column per aggregate holding 1/sqrt(size) on
   its nodes (the constant null space, orthonormal columns); isolated nodes
   have zero rows.
4. Prolongator smoothing: P = (I - omega D^-1 A) P~, omega = 4 / (3 rho) with
   rho = ||D^-1 A||_inf (the row-sum bound of the spectral radius).
5. Galerkin coarse matrix A_{l+1} = P^T A_l P.
6. Levels are added while the matrix has more than ``coarse_max`` rows and the
   aggregation still shrinks it; the last one is solved by dense Cholesky.

The V-cycle smooths every level above the last with ``smooth_deg`` = 3 steps
of Chebyshev-Jacobi (Algorithm 3, the same smoother as the geometric levels,
on [0.06, 1.2] lambda with lambda from 10 Jacobi-PCG Lanczos steps) before and
after the coarse correction: the AMG V-cycle with Chebyshev(3,3) smoothing of
the paper's lung runs (Table Lung); its other runs use one ILU(0) sweep, a
sequential smoother whose data-parallel counterpart is the polynomial one.  The coarse-grid
solve is CG (Algorithm 1) preconditioned by one such V-cycle from x = 0 until
||r|| <= rtol ||b||.
"""
import numpy as np
import scipy.sparse as sp

import sipg_inputs

from .multigrid import CoarseCholesky, chebyshev, estimate_lambda

THETA = 0.02
TIE = 1e-12
EIG_ITERS = 10


def strong_neighbours(A, theta=THETA):
    """Per row i, the columns j != i with |a_ij| > theta sqrt(a_ii a_jj) (step 1)."""
    A = sp.csr_matrix(A)
    d = A.diagonal()
    out = []
    for i in range(A.shape[0]):
        lo, hi = A.indptr[i], A.indptr[i + 1]
        js, vs = A.indices[lo:hi], A.data[lo:hi]
        keep = (js != i) & (np.abs(vs) > theta * np.sqrt(np.abs(d[i] * d[js])))
        order = np.argsort(js[keep], kind="stable")
        out.append((js[keep][order], np.abs(vs[keep][order])))
    return out


def aggregate(A, theta=THETA):
    """Aggregate number of every node (-1 = isolated) and the number of aggregates (step 2)."""
    S = strong_neighbours(A, theta)
    n = len(S)
    agg = -np.ones(n, dtype=np.int64)
    isolated = np.array([len(s[0]) == 0 for s in S])
    na = 0
    # pass 1
    for i in range(n):
        if isolated[i] or agg[i] >= 0:
            continue
        js = S[i][0]
        if np.all(agg[js] < 0):
            agg[i] = na
            agg[js] = na
            na += 1
    # pass 2 (against the pass-1 aggregates)
    after1 = agg.copy()
    for i in range(n):
        if isolated[i] or after1[i] >= 0:
            continue
        js, ws = S[i]
        cand = after1[js] >= 0
        if np.any(cand):
            top = ws[cand].max()
            best = np.flatnonzero(cand & (ws >= top * (1.0 - TIE)))[0]   # smallest j among the strongest
            agg[i] = after1[js[best]]
    # pass 3
    for i in range(n):
        if isolated[i] or agg[i] >= 0:
            continue
        js = S[i][0]
        agg[i] = na
        agg[js[agg[js] < 0]] = na
        na += 1
    return agg, na


def tentative_prolongator(agg, na):
    """P~ with 1/sqrt(|aggregate|) on the nodes of each aggregate (step 3)."""
    n = len(agg)
    rows = np.flatnonzero(agg >= 0)
    sizes = np.bincount(agg[rows], minlength=na).astype(np.float64)
    vals = 1.0 / np.sqrt(sizes[agg[rows]])
    return sp.csr_matrix((vals, (rows, agg[rows])), shape=(n, na))


def smoothed_prolongator(A, Pt):
    """P = (I - omega D^-1 A) P~ with omega = 4 / (3 ||D^-1 A||_inf) (step 4)."""
    A = sp.csr_matrix(A)
    dinv = 1.0 / A.diagonal()
    rho = float(np.max(np.abs(A).sum(axis=1).A1 * np.abs(dinv)))
    omega = 4.0 / (3.0 * rho)
    return sp.csr_matrix(Pt - omega * (sp.diags(dinv) @ (A @ Pt)))


class AMGLevel:
    def __init__(self, A):
        self.A = sp.csr_matrix(A)
        self.n = self.A.shape[0]
        self.dinv = 1.0 / self.A.diagonal()
        self.P = None
        self.lam = None


class SmoothedAggregationAMG:
    """Hierarchy of steps 1-6 and its V-cycle; levels[0] is the finest."""

    def __init__(self, A, coarse_max=500, smooth_deg=3, max_levels=10):
        self.smooth_deg = smooth_deg
        self.levels = [AMGLevel(A)]
        while self.levels[-1].n > coarse_max and len(self.levels) < max_levels:
            lev = self.levels[-1]
            agg, na = aggregate(lev.A)
            if na == 0 or na >= lev.n / 1.5:
                break
            lev.P = smoothed_prolongator(lev.A, tentative_prolongator(agg, na))
            self.levels.append(AMGLevel((lev.P.T @ lev.A @ lev.P).tocsr()))
        for lev in self.levels[:-1]:
            r0 = sipg_inputs.uniform(lev.n, sipg_inputs.SEED_EIG)
            lev.lam = estimate_lambda(lambda v, A=lev.A: A @ v, lev.dinv, r0, EIG_ITERS)
        self.coarse = CoarseCholesky(self.levels[-1].A)

    def vcycle(self, b, l=0):
        """One V-cycle from x = 0 on level l (Algorithm 2 on the AMG levels)."""
        if l == len(self.levels) - 1:
            return self.coarse.solve(b)
        lev = self.levels[l]
        mult = lambda v, A=lev.A: A @ v  # noqa: E731
        x = chebyshev(mult, lev.dinv, b, np.zeros_like(b), lev.lam, self.smooth_deg, x_is_zero=True)
        r = b - lev.A @ x
        x = x + lev.P @ self.vcycle(lev.P.T @ r, l + 1)
        return chebyshev(mult, lev.dinv, b, x, lev.lam, self.smooth_deg)


def pcg(A, b, precond, rtol=1e-3, maxit=200):
    """Algorithm 1 from x = 0 until ||r|| <= rtol ||b||: (x, iterations, residual norms)."""
    x = np.zeros_like(b)
    r = b.copy()
    nb = float(np.linalg.norm(b))
    hist = [nb]
    if nb == 0.0:
        return x, 0, hist
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while hist[-1] > rtol * nb and it < maxit:
        q = A @ p
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        hist.append(float(np.linalg.norm(r)))
        it += 1
        if hist[-1] <= rtol * nb:
            break
        z = precond(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, hist


class AMGCoarseSolver:
    """The coarse-grid solve: CG preconditioned by one smoothed-aggregation V-cycle to rtol."""

    def __init__(self, A, rtol=1e-3, coarse_max=500, smooth_deg=3):
        self.A = sp.csr_matrix(A)
        self.rtol = rtol
        self.amg = SmoothedAggregationAMG(self.A, coarse_max=coarse_max, smooth_deg=smooth_deg)
        self.last_iterations = 0

    def solve(self, b):
        x, it, _ = pcg(self.A, np.asarray(b, dtype=np.float64), self.amg.vcycle, self.rtol)
        self.last_iterations = it
        return x
