"""Pins of the oracle's SIPG operator (Section 2) against closed forms.

Symmetry, definiteness, the Neumann null space, exact polynomial consistency,
the closed-form Cartesian penalty, the textbook Q1 stiffness matrix and the
k+1 L2 convergence rate: each catches a different plausible mistake (a sign,
a dropped flux term, the Dirichlet factor 2, a wrong penalty or metric term).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle.dg import SIPG
from oracle.mesh import Mesh


def _poly(C):
    k = C.shape[0] - 1
    E = range(k + 1)

    def u(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return sum(C[a, b, c] * X ** a * Y ** b * Z ** c for a in E for b in E for c in E)

    def grad(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        g = [0 * X, 0 * X, 0 * X]
        for a in E:
            for b in E:
                for c in E:
                    if a:
                        g[0] = g[0] + C[a, b, c] * a * X ** (a - 1) * Y ** b * Z ** c
                    if b:
                        g[1] = g[1] + C[a, b, c] * b * X ** a * Y ** (b - 1) * Z ** c
                    if c:
                        g[2] = g[2] + C[a, b, c] * c * X ** a * Y ** b * Z ** (c - 1)
        return np.stack(g, axis=-1)

    def f(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        s = 0 * X
        for a in E:
            for b in E:
                for c in E:
                    if a >= 2:
                        s = s - C[a, b, c] * a * (a - 1) * X ** (a - 2) * Y ** b * Z ** c
                    if b >= 2:
                        s = s - C[a, b, c] * b * (b - 1) * X ** a * Y ** (b - 2) * Z ** c
                    if c >= 2:
                        s = s - C[a, b, c] * c * (c - 1) * X ** a * Y ** b * Z ** (c - 2)
        return s

    return u, grad, f


@pytest.mark.parametrize("deform", [0, 1])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_symmetric_and_matrix_free_equals_assembled(k, deform):
    op = SIPG(Mesh(2, deform=deform), k)
    A = op.assemble()
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
    u = np.random.default_rng(k).standard_normal(op.n_dofs)
    ref = A @ u
    assert np.max(np.abs(op.apply(u) - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.max(np.abs(op._diag_blocks() - A.diagonal())) <= 1e-13 * np.max(A.diagonal())
    rows = op.apply(u, cells=[1, 6])
    sel = np.zeros(op.n_dofs, bool)
    n3 = op.n ** 3
    for c in (1, 6):
        sel[c * n3:(c + 1) * n3] = True
    assert np.max(np.abs(rows[sel] - ref[sel])) <= 1e-13 * np.max(np.abs(ref))
    assert np.all(rows[~sel] == 0)


@pytest.mark.parametrize("deform", [0, 1])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_positive_definite_with_dirichlet(k, deform):
    A = SIPG(Mesh(2, deform=deform), k).assemble().toarray()
    assert np.linalg.eigvalsh(A)[0] > 1e-3


@pytest.mark.parametrize("deform", [0, 1])
@pytest.mark.parametrize("k", [1, 3])
def test_pure_neumann_null_space(k, deform):
    A = SIPG(Mesh(3, deform=deform, bc=(1,) * 6), k).assemble()
    assert np.max(np.abs(A @ np.ones(A.shape[0]))) <= 1e-13 * abs(A).max()
    # but not with one Dirichlet side
    A1 = SIPG(Mesh(3, deform=deform, bc=(1, 1, 0, 1, 1, 1)), k).assemble()
    assert np.max(np.abs(A1 @ np.ones(A1.shape[0]))) > 1e-2


@pytest.mark.parametrize("k", [1, 2, 3])
def test_polynomial_consistency_mixed_bc(k):
    """A I_h u = b(f=-lap u, g=u, h=du/dn) exactly for tensor degree <= k, affine cells."""
    rng = np.random.default_rng(10 + k)
    u, grad, f = _poly(rng.standard_normal((k + 1,) * 3))
    lo, hi = np.array([0.0, -1.0, 0.5]), np.array([1.0, 1.0, 2.0])
    bc = (0, 1, 0, 0, 1, 0)
    mesh = Mesh((2, 3, 2), lo=lo, hi=hi, bc=bc)

    def h(x):
        # outward normal of the box side a boundary point lies on
        g = grad(x)
        out = np.zeros(x.shape[:-1])
        for d in range(3):
            out = np.where(np.abs(x[..., d] - hi[d]) < 1e-12, g[..., d], out)
            out = np.where(np.abs(x[..., d] - lo[d]) < 1e-12, -g[..., d], out)
        return out

    op = SIPG(mesh, k)
    A = op.assemble()
    b = op.rhs(f, g=u, h=h)
    r = A @ op.interpolate(u) - b
    assert np.max(np.abs(r)) <= 1e-12 * np.max(np.abs(b))


def test_polynomial_consistency_fails_for_wrong_degree():
    # degree k+1 in one variable is not reproduced: guards the test's power
    k = 2
    C = np.zeros((k + 2,) * 3)
    C[k + 1, 0, 0] = 1.0
    u, _, f = _poly(C)
    op = SIPG(Mesh(2), k)
    r = op.assemble() @ op.interpolate(u) - op.rhs(f, g=u)
    assert np.max(np.abs(r)) > 1e-6


@pytest.mark.parametrize("k", [1, 2, 4])
def test_cartesian_penalty_closed_form(k):
    m = (2, 3, 4)
    lo, hi = np.zeros(3), np.array([1.0, 1.5, 0.8])
    op = SIPG(Mesh(m, lo=lo, hi=hi), k, penalty_factor=1.7)
    h = (hi - lo) / np.array(m)
    V = h.prod()
    area = [h[1] * h[2], h[0] * h[2], h[0] * h[1]]
    for e in range(op.mesh.n_cells):
        ijk = op.mesh.cell_ijk(e)
        a_int = a_b = 0.0
        for d in range(3):
            for on in (ijk[d] == 0, ijk[d] == m[d] - 1):
                if on:
                    a_b += area[d]
                else:
                    a_int += area[d]
        tau = 1.7 * (k + 1) ** 2 * (0.5 * a_int + a_b) / V
        assert abs(op.tau[e] - tau) <= 1e-13 * tau


def test_cube_penalty_matches_textbook_form():
    # uniform cube cells: tau_e = (k+1)^2 (3 + b_e/2) / h with b_e boundary faces
    op = SIPG(Mesh(3), 3)
    for e in range(27):
        b = sum(int(v == 0) + int(v == 2) for v in op.mesh.cell_ijk(e))
        assert abs(op.tau[e] - 16 * (3 + b / 2) * 3) < 1e-12


def test_q1_volume_block_is_textbook_stiffness():
    # trilinear brick [0,h]^3: K_ii = h/3, K_ij = 0 (edge), -h/12 (face or body diagonal)
    h = 0.25
    op = SIPG(Mesh(4, hi=(1.0, 1.0, 1.0)), 1)
    Ke = op.cell_matrices([5])[0]
    for i in range(8):
        for j in range(8):
            ndiff = bin(i ^ j).count("1")
            exact = {0: h / 3, 1: 0.0, 2: -h / 12, 3: -h / 12}[ndiff]
            assert abs(Ke[i, j] - exact) < 1e-15


def _exact(x):
    return np.sin(np.pi * x[..., 0]) * np.sin(np.pi * x[..., 1]) * np.sin(np.pi * x[..., 2])


@pytest.mark.parametrize("deform,k,ms", [(0, 1, (2, 4, 8)), (1, 1, (2, 4, 8)),
                                         (0, 2, (2, 4, 8)), (1, 2, (2, 4, 8)),
                                         (0, 3, (2, 4)), (1, 3, (2, 4))])
def test_l2_convergence_rate_k_plus_1(deform, k, ms):
    errs = []
    for m in ms:
        op = SIPG(Mesh(m, deform=deform), k)
        b = op.rhs(lambda x: 3 * np.pi ** 2 * _exact(x))
        uh = spl.spsolve(op.assemble().tocsc(), b)
        errs.append(op.l2_error(uh, _exact))
    rate = np.log2(errs[-2] / errs[-1])
    assert abs(rate - (k + 1)) < 0.2, (errs, rate)
