"""Pins of the oracle's FE operator (Eq. WeakFormFE) and transfers (Section 3.2)."""
import numpy as np
import pytest

from oracle import basis
from oracle.dg import SIPG
from oracle.fe import FESpace
from oracle.mesh import Mesh
from oracle.transfer import c_transfer, fe_transfer, projection_1d


@pytest.mark.parametrize("deform", [0, 1])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_fe_symmetric_constants_and_constraints(p, deform):
    fe = FESpace(Mesh(3, deform=deform), p)
    A0 = fe.assemble(constrain=False)
    assert abs(A0 - A0.T).max() <= 1e-14 * abs(A0).max()
    assert np.max(np.abs(A0 @ np.ones(fe.n_dofs))) <= 1e-13 * abs(A0).max()
    A = fe.assemble()
    u = np.random.default_rng(p).standard_normal(fe.n_dofs)
    assert np.max(np.abs(fe.apply(u) - A @ u)) <= 1e-13 * np.max(np.abs(A @ u))
    assert np.max(np.abs(fe.diagonal() - A.diagonal())) <= 1e-13
    c = fe.constrained
    assert np.all(A.diagonal()[c] == 1.0)
    assert np.linalg.eigvalsh(A.toarray())[0] > 0


def test_fe_energy_of_a_polynomial():
    # u = x^2 y on [0,1]^3: int |grad u|^2 = int 4x^2y^2 + x^4 = 4/9 + 1/5
    fe = FESpace(Mesh(2, bc=(1,) * 6), 2)
    xyz = fe.node_coords() / np.array(fe.grid, dtype=float)[None, :] * 0
    # nodal coordinates of the GL grid of the affine mesh
    x1 = np.concatenate([[0.0], *[(i + fe.nodes[1:]) / 2 for i in range(2)]])
    g = fe.node_coords()
    X, Y = x1[g[:, 0]], x1[g[:, 1]]
    u = X ** 2 * Y
    A = fe.assemble()
    assert abs(u @ (A @ u) - (4 / 9 + 1 / 5)) < 1e-13
    assert xyz.shape == (fe.n_dofs, 3)


def test_q1_fe_equals_textbook_stiffness():
    fe = FESpace(Mesh(1, bc=(1,) * 6), 1)
    A = fe.assemble().toarray()
    for i in range(8):
        for j in range(8):
            nd = bin(i ^ j).count("1")
            assert abs(A[i, j] - {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}[nd]) < 1e-15


@pytest.mark.parametrize("pf,pc", [(2, 1), (3, 1), (4, 2), (5, 2), (8, 4)])
def test_p_projection_is_interpolation(pf, pc):
    # nested spaces: the L2 projection reproduces the coarse basis (Section 3.2)
    nf, nc = basis.gauss_lobatto(pf + 1), basis.gauss_lobatto(pc + 1)
    P = projection_1d(nf, nc)
    assert np.max(np.abs(P - basis.lagrange_values(nc, nf))) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3])
def test_h_projection_is_child_interpolation(p):
    nodes = basis.gauss_lobatto(p + 1)
    for child in (0, 1):
        P = projection_1d(nodes, nodes, child=child)
        assert np.max(np.abs(P - basis.lagrange_values(nodes, 0.5 * (child + nodes)))) < 1e-13


def _grid_coords(fe, mesh):
    x1 = [np.concatenate([[0.0], *[(i + fe.nodes[1:]) / mesh.m[d] for i in range(mesh.m[d])]])
          for d in range(3)]
    g = fe.node_coords()
    return np.stack([x1[d][g[:, d]] for d in range(3)], axis=1)


@pytest.mark.parametrize("pf,pc", [(2, 1), (4, 2), (5, 2), (3, 1)])
def test_p_prolongation_reproduces_coarse_polynomials(pf, pc):
    mesh = Mesh((2, 3, 2), bc=(1,) * 6)
    ff, fc = FESpace(mesh, pf), FESpace(mesh, pc)
    P = fe_transfer(ff, fc)
    rng = np.random.default_rng(pf)
    C = rng.standard_normal((pc + 1,) * 3)

    def u(x):
        return sum(C[a, b, c] * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c
                   for a in range(pc + 1) for b in range(pc + 1) for c in range(pc + 1))

    uf = u(_grid_coords(ff, mesh))
    uc = u(_grid_coords(fc, mesh))
    assert np.max(np.abs(P @ uc - uf)) < 1e-12


def test_h_prolongation_reproduces_trilinear():
    mf, mc = Mesh(6, bc=(1,) * 6), Mesh(3, bc=(1,) * 6)
    ff, fc = FESpace(mf, 1), FESpace(mc, 1)
    P = fe_transfer(ff, fc)

    def u(x):
        return 1 + 2 * x[:, 0] - x[:, 1] + 3 * x[:, 0] * x[:, 1] * x[:, 2]

    assert np.max(np.abs(P @ u(_grid_coords(fc, mc)) - u(_grid_coords(ff, mf)))) < 1e-13


def test_transfers_respect_constraints():
    mesh = Mesh(4)
    ff, fc = FESpace(mesh, 4), FESpace(mesh, 2)
    P = fe_transfer(ff, fc)
    x = np.random.default_rng(0).standard_normal(fc.n_dofs)
    assert np.all((P @ x)[ff.constrained] == 0)
    assert np.all((P.T @ np.ones(ff.n_dofs))[fc.constrained] == 0)


def test_c_restriction_sums_duplicates():
    # a continuous field written into DG (duplicated) and restricted returns mult * value
    mesh = Mesh(3)
    fe = FESpace(mesh, 3)
    Pc = c_transfer(4, fe)
    w = np.random.default_rng(1).standard_normal(fe.n_dofs)
    w[fe.constrained] = 0
    dg = Pc @ w
    assert np.all(dg.reshape(27, 64) == w[fe.l2g])
    r = Pc.T @ dg
    assert np.max(np.abs(r - fe.multiplicity() * w)) < 1e-14


def test_fe_operator_is_dg_cell_part_on_continuous_functions():
    # for continuous u, the DG face terms cancel inside and the SIPG energy of
    # a continuous field equals the FE energy plus the Dirichlet boundary terms
    mesh = Mesh(2, bc=(1,) * 6)
    dg, fe = SIPG(mesh, 2), FESpace(mesh, 2)
    Pc = c_transfer(3, fe)
    Adg = dg.assemble()
    Afe = fe.assemble(constrain=False)
    diff = (Pc.T @ Adg @ Pc - Afe)
    assert abs(diff).max() < 1e-13
