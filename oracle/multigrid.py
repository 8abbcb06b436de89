"""Hybrid cph multigrid and Krylov solvers (Section 3 of the paper).

Test infrastructure: see ``oracle/__init__.py``.

* ``chebyshev``      -- Algorithm 3, Chebyshev-accelerated Jacobi.  The paper
  gives no formulas for sigma_j, theta_j; they come from the standard
  three-term Chebyshev recurrence (Saad, Iterative Methods for Sparse Linear
  Systems, 2nd ed., Alg. 12.1) applied to D^-1 A on [0.06, 1.2] * lambda_max
  (Section 3.1).  With theta = (l_hi+l_lo)/2, delta = (l_hi-l_lo)/2:
  rho_0 = delta/theta, x_1 = x_0 + D^-1 r_0 / theta, rho_j = 1/(2 theta/delta -
  rho_{j-1}), x_{j+1} = x_j + rho_j rho_{j-1} (x_j - x_{j-1}) + (2 rho_j/delta)
  D^-1 r_j; i.e. sigma_j = rho_j rho_{j-1}, theta_j = 2 rho_j / delta.
* ``estimate_lambda`` -- lambda_max of D^-1 A from 20 Jacobi-PCG iterations
  (Section 3.1) through the Lanczos tridiagonal of the CG coefficients.
* ``vcycle``         -- Algorithm 2 with x = 0 on entry, n_s pre- and
  post-smoothing steps on every level l > 0, exact coarse solve on l = 0.
* ``cg``             -- Algorithm 1 (preconditioned CG).
* ``fcg``            -- flexible CG with one retained direction (Notay):
  beta = -z_{j+1}^T A p_j / p_j^T A p_j, alpha = r^T z / p^T A p.
* ``CoarseCholesky`` -- dense direct coarse solve in FP64.
* ``build_cph``      -- the level hierarchy of the cph strategy (Section 3.2):
  DG_k -> FE_k (c) -> FE_{floor(k/2)} -> ... -> FE_1 (p) -> FE_1 on coarser
  meshes (h, while every m is even and m/2 >= 3).
"""
import numpy as np
import scipy.sparse as sp

import sipg_inputs

from .dg import SIPG
from .fe import FESpace
from .mesh import Mesh
from .transfer import c_transfer, dg_transfer, fe_transfer


def chebyshev(apply_A, dinv, b, x, lam, ns, lo=0.06, hi=1.2, x_is_zero=False):
    """n_s steps of Algorithm 3 on A x = b starting from x; returns x_{n_s}."""
    l_hi, l_lo = hi * lam, lo * lam
    theta, delta = 0.5 * (l_hi + l_lo), 0.5 * (l_hi - l_lo)
    r = b.copy() if x_is_zero else b - apply_A(x)
    x_prev = x
    x = x + dinv * r / theta
    rho_prev = delta / theta
    for _ in range(1, ns):
        rho = 1.0 / (2.0 * theta / delta - rho_prev)
        r = b - apply_A(x)
        x_new = x + rho * rho_prev * (x - x_prev) + (2.0 * rho / delta) * dinv * r
        x_prev, x, rho_prev = x, x_new, rho
    return x


def estimate_lambda(apply_A, dinv, r0, iters=20):
    """Largest eigenvalue of D^-1 A after ``iters`` Jacobi-PCG steps on A x = r0.

    The CG coefficients alpha_j, beta_j give the Lanczos matrix T with
    T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1}, T_{j,j+1} = sqrt(beta_j)/alpha_j.
    CG stops early when r^T z falls below 1e-28 of its start value.
    """
    r = r0.copy()
    z = dinv * r
    p = z.copy()
    rz = float(r @ z)
    rz0 = rz
    alphas, betas = [], []
    for _ in range(iters):
        Ap = apply_A(p)
        alpha = rz / float(p @ Ap)
        r = r - alpha * Ap
        z = dinv * r
        rz_new = float(r @ z)
        alphas.append(alpha)
        if not (rz_new > 1e-28 * rz0):
            break
        beta = rz_new / rz
        betas.append(beta)
        p = z + beta * p
        rz = rz_new
    m = len(alphas)
    T = np.zeros((m, m))
    for j in range(m):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < m:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    return float(np.max(np.linalg.eigvalsh(T)))


class CoarseCholesky:
    """Dense FP64 Cholesky factorisation A = L L^T and the two triangular solves."""

    def __init__(self, A):
        A = A.toarray() if sp.issparse(A) else np.asarray(A)
        self.L = np.linalg.cholesky(A)

    def solve(self, b):
        import scipy.linalg as sl
        y = sl.solve_triangular(self.L, b, lower=True)
        return sl.solve_triangular(self.L.T, y, lower=False)


class Level:
    def __init__(self, kind, space, A=None):
        self.kind, self.space = kind, space
        self.A = A                      # CSR or None (matrix-free)
        self.P = None                   # prolongation from level l-1 (sparse)
        self.diag = None
        self.dinv = None
        self.lam = None

    @property
    def n(self):
        return self.space.n_dofs

    def apply(self, u):
        return self.A @ u if self.A is not None else self.space.apply(u)


def coarse_meshes(mesh):
    """Meshes of the h-levels: halve while every m is even and m/2 >= 3."""
    out = [mesh]
    m = mesh.m
    while all(v % 2 == 0 and v // 2 >= 3 for v in m):
        m = tuple(v // 2 for v in m)
        out.append(Mesh(m, mesh.lo, mesh.hi, mesh.deform, mesh.amp, mesh.mapping_degree, mesh.bc))
    return out


def p_sequence(k, rule="half"):
    """Degrees of the FE levels on the finest mesh: k, then coarsened to 1."""
    seq = [k]
    while seq[-1] > 1:
        p = seq[-1]
        seq.append(max(1, p // 2) if rule == "half" else (p - 1 if rule == "minus1" else 1))
    return seq


class CPHMultigrid:
    """Hybrid multigrid V-cycle preconditioner, levels stored coarse (0) to fine (L).

    ``order`` lists the coarsening steps from the finest level (Section 3.2,
    Table SummaryCoarseningStrategies): 'c' DG -> FE at equal h and p, 'p'
    all polynomial levels down to degree 1, 'h' all geometric levels.  The
    default 'cph' is the paper's preferred strategy.  The coarsest level is
    solved directly (its space is DG when the order has no 'c'), or with
    ``coarse="amg"`` by CG preconditioned with smoothed-aggregation AMG to
    ``amg_rtol`` (Section 3.3, ``oracle.amg``).
    """

    def __init__(self, mesh, k, penalty_factor=1.0, ns=5, cheb_lo=0.06, cheb_hi=1.2,
                 eig_iters=20, lambdas=None, assemble_limit=6e7, p_rule="half", order="cph", coarse="dense",
                 amg_rtol=1e-3):
        self.ns, self.cheb_lo, self.cheb_hi = ns, cheb_lo, cheb_hi

        def make(kind, p, msh):
            if kind == "dg":
                sp_ = SIPG(msh, p, penalty_factor)
                big = sp_.n_dofs * sp_.n ** 3 * 7 > assemble_limit
            else:
                sp_ = FESpace(msh, p)
                big = sp_.n_dofs * (2 * p + 1) ** 3 > assemble_limit
            return Level(kind, sp_, None if big else sp_.assemble())

        kind, p, msh = "dg", k, mesh
        fine = [make(kind, p, msh)]
        for step in order:
            if step == "c":
                kind = "fe"
                fine.append(make(kind, p, msh))
            elif step == "p":
                for q in p_sequence(p, p_rule)[1:]:
                    p = q
                    fine.append(make(kind, p, msh))
            elif step == "h":
                for cm in coarse_meshes(msh)[1:]:
                    msh = cm
                    fine.append(make(kind, p, msh))
            else:
                raise ValueError("order letters are c, p, h")
        self.levels = fine[::-1]
        # transfers between consecutive levels
        for l in range(1, len(self.levels)):
            lf, lc = self.levels[l], self.levels[l - 1]
            if lf.kind == "dg" and lc.kind == "fe":
                lf.P = c_transfer(lf.space.n, lc.space)
            elif lf.kind == "dg":
                lf.P = dg_transfer(lf.space, lc.space)
            else:
                lf.P = fe_transfer(lf.space, lc.space)
        # smoother data on levels l > 0, coarse factor on l = 0
        for l, lev in enumerate(self.levels):
            if l == 0:
                A0 = lev.A if lev.A is not None else lev.space.assemble()
                if coarse == "amg":
                    from .amg import AMGCoarseSolver
                    self.coarse = AMGCoarseSolver(A0, rtol=amg_rtol)
                else:
                    self.coarse = CoarseCholesky(A0)
                continue
            lev.diag = lev.space.diagonal()
            lev.dinv = 1.0 / lev.diag
            if lambdas is not None:
                lev.lam = float(lambdas[l])
            else:
                r0 = sipg_inputs.uniform(lev.n, sipg_inputs.SEED_EIG)
                if lev.kind == "fe":
                    r0[lev.space.constrained] = 0.0
                lev.lam = estimate_lambda(lev.apply, lev.dinv, r0, eig_iters)

    @property
    def L(self):
        return len(self.levels) - 1

    def smooth(self, l, b, x, x_is_zero=False):
        lev = self.levels[l]
        return chebyshev(lev.apply, lev.dinv, b, x, lev.lam, self.ns,
                         self.cheb_lo, self.cheb_hi, x_is_zero)

    def vcycle(self, b, l=None):
        """Algorithm 2 with x^(l) = 0 on entry; returns the approximation x^(l)."""
        l = self.L if l is None else l
        if l == 0:
            return self.coarse.solve(b)
        lev = self.levels[l]
        x = self.smooth(l, b, np.zeros_like(b), x_is_zero=True)
        r = b - lev.apply(x)
        bc = lev.P.T @ r
        xc = self.vcycle(bc, l - 1)
        x = x + lev.P @ xc
        return self.smooth(l, b, x)


def cg(apply_A, b, x, precond, rtol=1e-10, maxit=1000, fixed_iters=None):
    """Algorithm 1.  Returns (x, iterations, residual norms)."""
    r = b - apply_A(x)
    nr0 = float(np.linalg.norm(r))
    hist = [nr0]
    v = precond(r)
    p = v.copy()
    delta = float(r @ v)
    it = 0
    while True:
        if fixed_iters is not None:
            if it >= fixed_iters:
                break
        elif hist[-1] <= rtol * nr0 or it >= maxit:
            break
        v = apply_A(p)
        omega = delta / float(p @ v)
        x = x + omega * p
        r = r - omega * v
        hist.append(float(np.linalg.norm(r)))
        it += 1
        v = precond(r)
        delta_old, delta = delta, float(r @ v)
        p = v + (delta / delta_old) * p
    return x, it, hist


def fcg(apply_A, b, x, precond, rtol=1e-10, maxit=1000, fixed_iters=None):
    """Flexible CG (one retained direction).  Returns (x, iterations, residual norms)."""
    r = b - apply_A(x)
    nr0 = float(np.linalg.norm(r))
    hist = [nr0]
    z = precond(r)
    p = z.copy()
    gamma = float(r @ z)
    it = 0
    while True:
        if fixed_iters is not None:
            if it >= fixed_iters:
                break
        elif hist[-1] <= rtol * nr0 or it >= maxit:
            break
        v = apply_A(p)
        pv = float(p @ v)
        alpha = gamma / pv
        x = x + alpha * p
        r = r - alpha * v
        hist.append(float(np.linalg.norm(r)))
        it += 1
        if fixed_iters is None and hist[-1] <= rtol * nr0:
            break
        z = precond(r)
        gamma = float(r @ z)
        beta = -float(z @ v) / pv
        p = z + beta * p
    return x, it, hist
