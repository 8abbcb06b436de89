"""Pins of the oracle's smoothed-aggregation AMG coarse-grid solver (Section 3.3).

Closed forms on the 1D Laplacian (aggregates of three nodes, the smoothed
aggregate's hat-shaped column), the defining properties of the construction
(orthonormal tentative columns spanning the constants, a symmetric positive
definite Galerkin matrix, a symmetric V-cycle that contracts the error in the
energy norm), exactness when no coarsening happens, and convergence of the
AMG-preconditioned CG to 1e-3 on the odd and prime coarse meshes whose FE_1
level is too large for a dense solve.
"""
import numpy as np
import scipy.sparse as sp

import sipg_inputs
from oracle import amg
from oracle.fe import FESpace
from oracle.mesh import Mesh
from oracle.multigrid import CPHMultigrid, fcg


def lap1d(n):
    return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()


def test_1d_laplacian_aggregates_by_hand():
    # pass 1: root 0 takes {0, 1}; 2 has an aggregated neighbour; root 3 takes {2, 3, 4}; root 6
    # takes {5, 6, 7}; pass 2: the free node 8 joins its only strong neighbour's aggregate
    agg, na = amg.aggregate(lap1d(9))
    assert na == 3
    assert list(agg) == [0, 0, 1, 1, 1, 2, 2, 2, 2]
    # pass 2 picks the strongest aggregated neighbour, the smaller index on ties: in the graph
    # 0-1, 1-2, 2-4, 3-4, 3-5 pass 1 makes {0, 1} and {3, 4, 5} and leaves node 2 between
    # node 1 (aggregate 0) and node 4 (aggregate 1)

    def graph(w24):
        W = np.zeros((6, 6))
        for (i, j), w in {(0, 1): 1.0, (1, 2): 1.0, (2, 4): w24, (3, 4): 1.0, (3, 5): 1.0}.items():
            W[i, j] = W[j, i] = w
        return sp.csr_matrix(np.diag(W.sum(axis=1) + 1.0) - W)

    assert list(amg.aggregate(graph(1.0))[0]) == [0, 0, 0, 1, 1, 1]
    assert list(amg.aggregate(graph(1.5))[0]) == [0, 0, 1, 1, 1, 1]


def test_tentative_columns_are_orthonormal_and_span_constants():
    A = FESpace(Mesh(5, deform=1, bc=(0, 1, 1, 0, 1, 1)), 1).assemble()
    agg, na = amg.aggregate(A)
    Pt = amg.tentative_prolongator(agg, na)
    assert np.allclose((Pt.T @ Pt).toarray(), np.eye(na), atol=1e-14)
    one = np.ones(A.shape[0])
    proj = Pt @ (Pt.T @ one)
    live = agg >= 0
    assert np.allclose(proj[live], 1.0, atol=1e-14) and np.all(proj[~live] == 0.0)
    # identity rows (Dirichlet nodes) are isolated, every other node is aggregated
    d = A.diagonal()
    ident = np.array([A.indptr[i + 1] - A.indptr[i] == 1 and d[i] == 1.0 for i in range(A.shape[0])])
    assert np.array_equal(~live, ident)


def test_smoothed_aggregate_is_the_hat_of_the_textbook():
    # 1D Laplacian: rho = ||D^-1 A||_inf = 2, omega = 2/3; the middle aggregate {2,3,4} with
    # value 1/sqrt(3) becomes (1, 2, 3, 2, 1) / (3 sqrt 3) on nodes 1..5
    A = lap1d(9)
    agg, na = amg.aggregate(A)
    P = amg.smoothed_prolongator(A, amg.tentative_prolongator(agg, na)).toarray()
    col = P[:, 1]
    want = np.zeros(9)
    want[1:6] = np.array([1, 2, 3, 2, 1]) / (3 * np.sqrt(3))
    assert np.allclose(col, want, atol=1e-15)


def test_galerkin_matrix_spd_and_vcycle_symmetric_contraction():
    A = FESpace(Mesh(11, deform=1), 1).assemble()
    h = amg.SmoothedAggregationAMG(A, coarse_max=100)
    assert len(h.levels) >= 2
    for lev in h.levels[1:]:
        Ac = lev.A.toarray()
        assert np.allclose(Ac, Ac.T, atol=1e-13 * np.abs(Ac).max())
        assert np.linalg.eigvalsh(Ac).min() > 0
    n = A.shape[0]
    x, y = sipg_inputs.uniform(n, 3), sipg_inputs.uniform(n, 4)
    Mx, My = h.vcycle(x), h.vcycle(y)
    assert abs(y @ Mx - x @ My) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(My)
    e = sipg_inputs.uniform(n, 5)
    e2 = e - h.vcycle(A @ e)
    energy = lambda v: float(v @ (A @ v)) ** 0.5  # noqa: E731
    assert energy(e2) < 0.5 * energy(e)


def test_no_coarsening_is_an_exact_solve():
    A = FESpace(Mesh(3), 1).assemble()
    s = amg.AMGCoarseSolver(A, coarse_max=500)
    assert len(s.amg.levels) == 1
    b = sipg_inputs.uniform(A.shape[0], 8)
    x = s.solve(b)
    assert s.last_iterations == 1
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b)


def test_amg_cg_reaches_1e3_on_odd_and_prime_coarse_meshes():
    for m, deform in ((17, 0), (13, 1), (23, 0)):
        fs = FESpace(Mesh(m, deform=deform, bc=(0, 0, 1, 0, 0, 1)), 1)
        A = fs.assemble()
        s = amg.AMGCoarseSolver(A)
        b = sipg_inputs.uniform(A.shape[0], 6)
        b[fs.constrained] = 0.0
        x = s.solve(b)
        assert np.linalg.norm(b - A @ x) <= 1e-3 * np.linalg.norm(b)
        assert 1 <= s.last_iterations <= 10, (m, s.last_iterations)


def test_cph_solve_with_amg_coarse_matches_dense_coarse_counts():
    """m = 9 (odd: no h-level, FE_1 on 10^3 nodes as the coarse level): the flexible CG with
    the inexact AMG-CG coarse solve needs at most one iteration more than with the exact one."""
    m, k = 9, 2
    dense = CPHMultigrid(Mesh(m), k)
    with_amg = CPHMultigrid(Mesh(m), k, coarse="amg")
    fine = dense.levels[-1]
    b = sipg_inputs.uniform(fine.n, sipg_inputs.SEED_RHS)
    xd, itd, _ = fcg(fine.apply, b, np.zeros_like(b), dense.vcycle, rtol=1e-10)
    xa, ita, _ = fcg(fine.apply, b, np.zeros_like(b), with_amg.vcycle, rtol=1e-10)
    assert len(with_amg.coarse.amg.levels) == 2
    assert itd <= ita <= itd + 1, (itd, ita)
    assert np.linalg.norm(xa - xd) <= 1e-8 * np.linalg.norm(xd)
