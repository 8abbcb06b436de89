"""GPU parity: libsipg (through the C ABI) against the FP64 CPU oracle.

Every comparison is element by element (parity_check.close: the largest entry
error against the largest reference entry, and the relative 2-norm, whichever
is larger).  Tolerances: FP64 <= 1e-12, FP32 <= 1e-5 for single operator
applications, transfers, diagonals and the coarse solve; whole-cycle and solve
comparisons use the bounds stated at each test (more operations, same
arithmetic up to summation order).
"""
import numpy as np
import pytest

import sipg_inputs
from oracle.dg import SIPG
from oracle.fe import FESpace
from oracle.mesh import Mesh
from oracle.multigrid import CPHMultigrid, chebyshev, fcg
from oracle.transfer import c_transfer, fe_transfer
from parity_check import close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _ctx(*a, **kw):
    from paper_1910_01900_gb300 import Context
    return Context(*a, **kw)


def gpu(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(DEV, dtype)


# meshes spanning several thread blocks with a ragged last block for every degree
SHAPES = {1: (6, 5, 5), 2: (5, 4, 3), 3: (5, 3, 3), 4: (4, 3, 3), 5: (3, 3, 3), 6: (4, 2, 2), 7: (3, 2, 2),
          8: (3, 2, 2)}


@pytest.mark.parametrize("deform", [0, 1])
@pytest.mark.parametrize("k", range(1, 9))
def test_operator_apply_fp64_fp32(k, deform):
    m = SHAPES[k]
    lo, hi = (0.0, -0.5, 0.2), (1.0, 1.0, 1.4)
    bc = (0, 1, 0, 0, 1, 0)
    ctx = _ctx(m, k, deform=deform, lo=lo, hi=hi, bc=bc, operator_only=True)
    u = sipg_inputs.uniform(ctx.num_dofs(), sipg_inputs.SEED_APPLY)
    ref = SIPG(Mesh(m, lo=lo, hi=hi, deform=deform, bc=bc), k).apply(u)
    v = torch.empty(len(u), dtype=torch.float64, device=DEV)
    ctx.apply(gpu(u), v)
    assert close(v.cpu().numpy(), ref) <= 1e-12
    v32 = torch.empty(len(u), dtype=torch.float32, device=DEV)
    ctx.apply(gpu(u, torch.float32), v32)
    assert close(v32.cpu().numpy(), ref) <= 1e-5


def test_single_cell_and_pure_neumann():
    for k in (1, 4, 8):
        ctx = _ctx(1, k, operator_only=True)
        u = sipg_inputs.uniform(ctx.num_dofs(), 7)
        v = torch.empty(len(u), dtype=torch.float64, device=DEV)
        ctx.apply(gpu(u), v)
        assert close(v.cpu().numpy(), SIPG(Mesh(1), k).apply(u)) <= 1e-12
    ctx = _ctx(3, 3, deform=1, bc=(1,) * 6, operator_only=True)
    one = torch.ones(ctx.num_dofs(), dtype=torch.float64, device=DEV)
    v = torch.empty_like(one)
    ctx.apply(one, v)
    u = sipg_inputs.uniform(ctx.num_dofs(), 3)
    w = torch.empty_like(one)
    ctx.apply(gpu(u), w)
    assert v.abs().max().item() <= 1e-12 * w.abs().max().item()


def test_invalid_arguments_are_rejected():
    from paper_1910_01900_gb300 import SipgError
    with pytest.raises(SipgError):
        _ctx(0, 3)
    with pytest.raises(SipgError):
        _ctx(2, 9)
    ctx = _ctx(2, 2, operator_only=True)
    with pytest.raises(SipgError):
        ctx.vcycle(torch.zeros(ctx.num_dofs(), dtype=torch.float64, device=DEV),
                   torch.zeros(ctx.num_dofs(), dtype=torch.float64, device=DEV))


def _hierarchy(m, k, deform, **kw):
    ctx = _ctx(m, k, deform=deform, **kw)
    mg = CPHMultigrid(Mesh(m, deform=deform), k,
                      lambdas=[kw["lambda_override"]] * 16 if kw.get("lambda_override") else None)
    return ctx, mg


@pytest.mark.parametrize("m,k,deform", [(4, 3, 0), (6, 4, 1), (4, 5, 0)])
def test_levels_diagonals_and_fe_apply(m, k, deform):
    ctx, mg = _hierarchy(m, k, deform, lambda_override=2.0)
    assert ctx.num_levels == len(mg.levels)
    for l, lev in enumerate(mg.levels):
        kind, deg, mm = ctx.level_info(l)
        assert (kind == 0) == (lev.kind == "dg") and ctx.num_dofs(l) == lev.n
        u = sipg_inputs.uniform(lev.n, 100 + l)
        if lev.kind == "fe":
            u[lev.space.constrained] *= 0.5   # identity rows are exercised too
        ref = lev.apply(u)
        for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
            v = torch.empty(lev.n, dtype=dt, device=DEV)
            ctx.level_apply(l, gpu(u, dt), v)
            assert close(v.cpu().numpy(), ref) <= tol, (l, dt)
        if l > 0:
            d = torch.empty(lev.n, dtype=torch.float64, device=DEV)
            ctx.inverse_diagonal(l, d)
            assert close(d.cpu().numpy(), lev.dinv) <= 1e-12


@pytest.mark.parametrize("k,fa", [(4, 2), (3, 3)])
@pytest.mark.parametrize("deform,bc", [(1, (0, 1, 0, 0, 1, 0)), (0, (1, 1, 0, 1, 1, 1))])
def test_assembled_low_degree_levels_match_matrix_free(deform, bc, k, fa):
    """FE levels of degree 1 (by default) and up to fa (fe_assemble=fa: 125 points at degree
    2, 343 at degree 3) apply an assembled stencil: the same operator as the matrix-free cell
    and node passes and as the oracle's FE matrix, with Dirichlet and Neumann sides mixed
    (identity rows and zero columns only on Dirichlet nodes)."""
    # k = 4: DG4, FE4, FE2 (assembled), FE1 6^3 (assembled), FE1 3^3 (coarse)
    # k = 3: DG3, FE3 (assembled), FE1 6^3 (assembled), FE1 3^3 (coarse)
    m = 6
    ctx_a = _ctx(m, k, deform=deform, bc=bc, lambda_override=2.0, fe_assemble=fa)
    ctx_f = _ctx(m, k, deform=deform, bc=bc, lambda_override=2.0, fe_assemble=0)
    mg = CPHMultigrid(Mesh(m, deform=deform, bc=bc), k, lambdas=[2.0] * 16)
    checked = 0
    for l in range(1, len(mg.levels)):
        lev = mg.levels[l]
        if lev.kind != "fe" or lev.space.p > fa:
            continue
        u = sipg_inputs.uniform(lev.n, 500 + l)
        u[lev.space.constrained] *= -3.0
        ref = lev.apply(u)
        for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
            va, vf = (torch.empty(lev.n, dtype=dt, device=DEV) for _ in range(2))
            ctx_a.level_apply(l, gpu(u, dt), va)
            ctx_f.level_apply(l, gpu(u, dt), vf)
            torch.cuda.synchronize()
            assert close(va.cpu().numpy(), ref) <= tol, (l, dt)
            assert close(vf.cpu().numpy(), ref) <= tol, (l, dt)
        checked += 1
    assert checked == 2
    r = gpu(sipg_inputs.uniform(ctx_a.num_dofs(), 77))
    za, zf = torch.empty_like(r), torch.empty_like(r)
    ctx_a.vcycle(r, za)
    ctx_f.vcycle(r, zf)
    torch.cuda.synchronize()
    zo = mg.vcycle(r.cpu().numpy())
    assert close(za.cpu().numpy(), zo) <= 1e-12 and close(zf.cpu().numpy(), zo) <= 1e-12


@pytest.mark.parametrize("m,k,deform", [(6, 4, 0), (6, 5, 1), (8, 2, 0)])
def test_transfers_match_sparse_matrices(m, k, deform):
    ctx, mg = _hierarchy(m, k, deform, lambda_override=2.0)
    for l in range(1, len(mg.levels)):
        P = mg.levels[l].P
        r = sipg_inputs.uniform(mg.levels[l].n, 200 + l)
        rc = torch.empty(mg.levels[l - 1].n, dtype=torch.float64, device=DEV)
        ctx.restrict(l, gpu(r), rc)
        assert close(rc.cpu().numpy(), P.T @ r) <= 1e-12, l
        xc = sipg_inputs.uniform(mg.levels[l - 1].n, 300 + l)
        sp = mg.levels[l - 1].space
        xc[sp.constrained] = 0.0
        x0 = sipg_inputs.uniform(mg.levels[l].n, 400 + l)
        if mg.levels[l].kind == "fe":
            x0[mg.levels[l].space.constrained] = 0.0
        x = gpu(x0)
        ctx.prolongate_add(l, gpu(xc), x)
        assert close(x.cpu().numpy(), x0 + P @ xc) <= 1e-12, l


def test_coarse_solve_and_lambda_estimates():
    m, k = 6, 4
    ctx, mg = _hierarchy(m, k, 1)
    b = sipg_inputs.uniform(mg.levels[0].n, 5)
    b[mg.levels[0].space.constrained] = 0.0
    x = torch.empty(len(b), dtype=torch.float64, device=DEV)
    ctx.coarse_solve(gpu(b), x)
    assert close(x.cpu().numpy(), mg.coarse.solve(b)) <= 1e-12
    for l in range(1, len(mg.levels)):
        assert abs(ctx.lam(l) - mg.levels[l].lam) <= 1e-10 * mg.levels[l].lam, l


@pytest.mark.parametrize("level_from_top", [0, 1])
def test_chebyshev_smoother(level_from_top):
    m, k = 4, 4
    ctx, mg = _hierarchy(m, k, 1, lambda_override=1.7)
    l = len(mg.levels) - 1 - level_from_top
    lev = mg.levels[l]
    b = sipg_inputs.uniform(lev.n, 11)
    x0 = sipg_inputs.uniform(lev.n, 12)
    if lev.kind == "fe":
        b[lev.space.constrained] = 0.0
        x0[lev.space.constrained] = 0.0
    ref = chebyshev(lev.apply, lev.dinv, b, x0, 1.7, 5)
    x = gpu(x0)
    ctx.smooth(l, gpu(b), x, 5)
    assert close(x.cpu().numpy(), ref) <= 1e-11


@pytest.mark.parametrize("m,k,deform", [(4, 3, 0), (6, 3, 1), (4, 2, 1)])
def test_vcycle_fp64_and_fp32(m, k, deform):
    ctx, mg = _hierarchy(m, k, deform, lambda_override=2.2)
    r = sipg_inputs.uniform(mg.levels[-1].n, 21)
    ref = mg.vcycle(r)
    z = torch.empty(len(r), dtype=torch.float64, device=DEV)
    ctx.vcycle(gpu(r), z)
    assert close(z.cpu().numpy(), ref) <= 1e-11
    ctx32 = _ctx(m, k, deform=deform, precision=1, lambda_override=2.2)
    ctx32.vcycle(gpu(r), z)
    assert close(z.cpu().numpy(), ref) <= 1e-5


def test_fixed_iteration_fcg_matches_oracle():
    m, k = 4, 3
    ctx, mg = _hierarchy(m, k, 0, lambda_override=2.2)
    b = sipg_inputs.uniform(mg.levels[-1].n, sipg_inputs.SEED_RHS)
    ref, _, hist = fcg(mg.levels[-1].apply, b, np.zeros_like(b), mg.vcycle, fixed_iters=3)
    x = torch.zeros(len(b), dtype=torch.float64, device=DEV)
    info = ctx.solve(gpu(b), x, fixed_iters=3)
    assert info.iterations == 3
    assert close(x.cpu().numpy(), ref) <= 1e-11
    assert abs(info.res_history[3] - hist[3]) <= 1e-9 * hist[3]


@pytest.mark.parametrize("m,k,deform", [(4, 3, 0), (4, 3, 1), (6, 2, 0)])
def test_solve_to_1e10_same_iterations_as_oracle(m, k, deform):
    ctx, mg = _hierarchy(m, k, deform)
    b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=DEV)
    ctx.rhs(b)
    bo = mg.levels[-1].space.rhs(lambda x: 3 * np.pi ** 2 * np.prod(np.sin(np.pi * x), axis=-1))
    assert close(b.cpu().numpy(), bo) <= 1e-12
    ref, it, hist = fcg(mg.levels[-1].apply, bo, np.zeros_like(bo), mg.vcycle, rtol=1e-10)
    x = torch.zeros_like(b)
    info = ctx.solve(b, x, rtol=1e-10)
    assert info.converged and info.iterations == it
    assert close(x.cpu().numpy(), ref) <= 1e-10
    # mixed precision: FP32 cycle, FP64 residual, same tolerance reached
    ctx32 = _ctx(m, k, deform=deform, precision=1)
    x32 = torch.zeros_like(b)
    info32 = ctx32.solve(b, x32, rtol=1e-10)
    assert info32.converged and abs(info32.iterations - it) <= 1
    assert close(x32.cpu().numpy(), ref) <= 1e-8


def test_solve_from_a_nonzero_start_vector():
    """x0 != 0 takes the r0 = b - A x0 branch (x0 = 0 skips that apply): same iterates as the
    oracle's flexible CG started from the same x0, and the same solution as from zero."""
    m, k = 4, 3
    ctx, mg = _hierarchy(m, k, 1)
    bo = sipg_inputs.uniform(ctx.num_dofs(), sipg_inputs.SEED_RHS)
    x0 = 0.3 * sipg_inputs.uniform(ctx.num_dofs(), 9)
    ref, it, hist = fcg(mg.levels[-1].apply, bo, x0.copy(), mg.vcycle, rtol=1e-10)
    x = gpu(x0)
    info = ctx.solve(gpu(bo), x, rtol=1e-10)
    assert info.converged and info.iterations == it
    assert abs(info.r0_norm - hist[0]) <= 1e-12 * hist[0]
    assert close(x.cpu().numpy(), ref) <= 1e-10
    xz = torch.zeros_like(x)
    ctx.solve(gpu(bo), xz, rtol=1e-12)
    assert close(x.cpu().numpy(), xz.cpu().numpy()) <= 1e-6


def test_solve_host_round_trip_and_nan_rejected():
    ctx = _ctx(4, 2)
    b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=DEV)
    ctx.rhs(b)
    x = torch.zeros_like(b)
    ctx.solve(b, x)
    bh = b.cpu().numpy().copy()
    xh = np.zeros_like(bh)
    ctx.solve_host(bh, xh)
    assert close(xh, x.cpu().numpy()) <= 1e-13
    from paper_1910_01900_gb300 import SipgError
    bh[3] = np.nan
    with pytest.raises(SipgError):
        ctx.solve_host(bh, xh)


def _sampled_apply_check(m, k, deform, cells, precision=0):
    ctx = _ctx(m, k, deform=deform, operator_only=True)
    n = ctx.num_dofs()
    u = sipg_inputs.uniform(n, sipg_inputs.SEED_APPLY)
    dt = torch.float64 if precision == 0 else torch.float32
    v = torch.empty(n, dtype=dt, device=DEV)
    ctx.apply(gpu(u, dt), v)
    vv = v.cpu().numpy().astype(np.float64)
    ref = SIPG(Mesh(m, deform=deform), k).apply(u, cells=cells)
    n3 = (k + 1) ** 3
    sel = np.concatenate([np.arange(c * n3, (c + 1) * n3) for c in cells])
    return close(vv[sel], ref[sel])


def test_full_size_curved16_k5_sampled():
    """The 16^3 curved k=5 workload at full size, checked on sampled cells."""
    m = 16
    cells = [0, 15, 255, 256 * 7 + 16 * 5 + 9, 4095, 2048 + 3]
    assert _sampled_apply_check(m, 5, 1, cells) <= 1e-12
    assert _sampled_apply_check(m, 5, 1, cells, precision=1) <= 1e-5


@pytest.mark.parametrize("k", [1, 3, 5, 8])
def test_sweep_sizes_sampled(k):
    """The ~16 MDoF apply-sweep meshes at full size, sampled cells (curved)."""
    m = sipg_inputs.SWEEP_M[k]
    E = m ** 3
    cells = [0, m - 1, m * m * (m // 2) + m * 3 + 1, E // 2 + 7, E - 1]
    assert _sampled_apply_check(m, k, 1, cells) <= 1e-12


@pytest.mark.parametrize("k,deform", [(2, 0), (5, 1), (8, 0)])
def test_autotuned_tile_shapes_keep_parity(k, deform):
    m = SHAPES[k]
    ctx = _ctx(m, k, deform=deform, operator_only=True, autotune=True)
    from sipg_inputs import uniform
    u = uniform(ctx.num_dofs(), 3)
    ref = SIPG(Mesh(m, deform=deform), k).apply(u)
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        v = torch.empty(len(u), dtype=dt, device=DEV)
        ctx.apply(gpu(u, dt), v)
        assert close(v.cpu().numpy(), ref) <= tol
    from paper_1910_01900_gb300.csrc_info import max_cells_per_block
    for prec in (0, 1):
        for p in (0, 1):
            assert 1 <= ctx.tile_shape(prec, p) <= max_cells_per_block(k + 1, 8 >> prec)


@pytest.mark.parametrize("k,deform", [(3, 1), (6, 0)])
def test_every_tile_width_gives_identical_results(k, deform):
    """A cell kernel's block width changes the launch, not the arithmetic: bitwise equal
    results on the DG level (both passes) and on every FE level (cell pass)."""
    from paper_1910_01900_gb300.csrc_info import max_cells_per_block
    m = (5, 4, 6)
    ctx = _ctx(m, k, deform=deform)
    u64 = gpu(sipg_inputs.uniform(ctx.num_dofs(), 21))
    ref64 = torch.empty_like(u64)
    ctx.apply(u64, ref64)
    torch.cuda.synchronize()
    assert close(ref64.cpu().numpy(), SIPG(Mesh(m, deform=deform), k).apply(u64.cpu().numpy())) <= 1e-12
    for level in range(1, ctx.num_levels):
        kind, deg, _ = ctx.level_info(level)
        passes = (0, 1) if kind == 0 else (2,)
        for dt, prec in ((torch.float64, 0), (torch.float32, 1)):
            u = gpu(sipg_inputs.uniform(ctx.num_dofs(level), 30 + level), dt)
            ref = torch.empty_like(u)
            ctx.level_apply(level, u, ref)
            mx = max_cells_per_block(deg + 1, 8 >> prec)
            for cb in sorted({1, 2, 3, mx // 2, mx - 1, mx}):
                for p in passes:
                    ctx.set_tile_shape(prec, p, cb, level=level)
                    assert ctx.tile_shape(prec, p, level=level) == cb
                v = torch.full_like(u, float("nan"))
                ctx.level_apply(level, u, v)
                torch.cuda.synchronize()
                assert torch.equal(v, ref), (level, prec, cb)
            for p in passes:
                ctx.set_tile_shape(prec, p, 0, level=level)
    # widths beyond the limits and passes a level does not have are refused
    from paper_1910_01900_gb300.native import SipgError
    with pytest.raises(SipgError):
        ctx.set_tile_shape(0, 0, max_cells_per_block(k + 1, 8) + 1)
    with pytest.raises(SipgError):
        ctx.set_tile_shape(0, 2, 1)


def test_apply_is_deterministic_bitwise():
    """No atomics anywhere: two applications give bit-identical results."""
    ctx = _ctx((5, 4, 3), 4, deform=1, operator_only=True)
    u = gpu(sipg_inputs.uniform(ctx.num_dofs(), 9))
    v1, v2 = torch.empty_like(u), torch.empty_like(u)
    ctx.apply(u, v1)
    ctx.apply(u, v2)
    assert torch.equal(v1, v2)


def test_maxit_reports_not_converged():
    from paper_1910_01900_gb300 import native
    ctx = _ctx(4, 3)
    b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=DEV)
    ctx.rhs(b)
    x = torch.zeros_like(b)
    info = ctx.solve(b, x, rtol=1e-10, maxit=1, allow_notconv=True)
    assert info.iterations == 1 and not info.converged
    import ctypes
    st = native.lib().sipg_solve(ctx.h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), 1e-10, 1, 0,
                                 None)
    assert st == native.ENOTCONV


def test_penalty_robustness_of_cph_on_gpu():
    """cph iteration counts barely move when the penalty grows 1000x (Table PenaltyFactor, cph rows)."""
    its = []
    for pf in (1.0, 1000.0):
        ctx = _ctx(8, 3, penalty_factor=pf)
        b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=DEV)
        ctx.rhs(b)
        x = torch.zeros_like(b)
        its.append(ctx.solve(b, x, rtol=1e-10).n10)
    assert abs(its[1] - its[0]) < 1.0, its


@pytest.mark.parametrize("m,k,deform", [(4, 2, 0), (3, 4, 1), (2, 8, 1)])
def test_l2_error_diagnostic_matches_oracle(m, k, deform):
    ctx = _ctx(m, k, deform=deform, operator_only=True)
    x = sipg_inputs.uniform(ctx.num_dofs(), 31)
    e = ctx.l2_error(gpu(x))
    exact = lambda p: np.prod(np.sin(np.pi * p), axis=-1)  # noqa: E731
    ref = SIPG(Mesh(m, deform=deform), k).l2_error(x, exact)
    assert abs(e - ref) <= 1e-12 * ref


@pytest.mark.parametrize("rule,code", [("minus1", 1), ("one", 2)])
def test_other_p_sequences_match_oracle(rule, code):
    """p_{l-1} = p_l - 1 and p_{l-1} = 1 (Section 3.2): same levels, iterations and solution as the oracle."""
    m, k = 4, 4
    ctx = _ctx(m, k, p_coarsen=code)
    mg = CPHMultigrid(Mesh(m), k, p_rule=rule)
    assert ctx.num_levels == len(mg.levels)
    b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=DEV)
    ctx.rhs(b)
    bo = b.cpu().numpy()
    ref, it, _ = fcg(mg.levels[-1].apply, bo, np.zeros_like(bo), mg.vcycle, rtol=1e-10)
    x = torch.zeros_like(b)
    info = ctx.solve(b, x, rtol=1e-10)
    assert info.iterations == it
    assert close(x.cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("order,m,k", [("chp", 6, 2), ("pch", 6, 3), ("phc", 6, 2), ("hpc", 6, 2), ("cp", 4, 3),
                                       ("pc", 4, 4)])
def test_other_coarsening_orders_match_oracle(order, m, k):
    """Orders of Table SummaryCoarseningStrategies that end on FE_1: levels, iterations, solution."""
    ctx = _ctx(m, k, coarsening=order)
    mg = CPHMultigrid(Mesh(m), k, order=order)
    assert ctx.num_levels == len(mg.levels)
    for l, lev in enumerate(mg.levels):
        kind, deg, mm = ctx.level_info(l)
        assert (kind == 0) == (lev.kind == "dg") and deg == lev.space.n - 1 and ctx.num_dofs(l) == lev.n
    b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=DEV)
    ctx.rhs(b)
    bo = b.cpu().numpy()
    ref, it, _ = fcg(mg.levels[-1].apply, bo, np.zeros_like(bo), mg.vcycle, rtol=1e-10)
    x = torch.zeros_like(b)
    info = ctx.solve(b, x, rtol=1e-10)
    assert info.iterations == it
    assert close(x.cpu().numpy(), ref) <= 1e-10


def test_coarsening_without_c_is_rejected():
    from paper_1910_01900_gb300 import SipgError
    with pytest.raises(SipgError):
        _ctx(4, 2, coarsening="ph")


def test_iterative_coarse_solve_small_mesh():
    """With coarse_solver = 1 a coarsest level above coarse_dense_max gets fixed Jacobi-PCG
    iterations instead of the dense inverse: forced here on a small mesh, where 50 iterations
    nearly solve it exactly."""
    m, k = 4, 3
    ctx = _ctx(m, k, coarse_dense_max=0, coarse_iters=50, coarse_solver=1)
    mg = CPHMultigrid(Mesh(m), k)
    n0 = ctx.num_dofs(0)
    b0 = sipg_inputs.uniform(n0, 61)
    b0[mg.levels[0].space.constrained] = 0.0
    x = torch.empty(n0, dtype=torch.float64, device=DEV)
    ctx.coarse_solve(gpu(b0), x)
    torch.cuda.synchronize()
    assert close(x.cpu().numpy(), mg.coarse.solve(b0)) <= 1e-4
    b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=DEV)
    ctx.rhs(b)
    xd = torch.zeros_like(b)
    dense = _ctx(m, k).solve(b, xd, rtol=1e-10)
    for prec in (0, 1):
        c = _ctx(m, k, precision=prec, coarse_dense_max=0, coarse_iters=50, coarse_solver=1)
        xc = torch.zeros_like(b)
        info = c.solve(b, xc, rtol=1e-10)
        assert info.converged and info.iterations <= dense.iterations + 2, (prec, info.iterations)
        assert close(xc.cpu().numpy(), xd.cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("precision,coarse_solver", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_odd_mesh_with_large_coarse_level(precision, coarse_solver):
    """m = 17 cannot be halved: the coarsest FE_1 level has 18^3 = 5832 unknowns, above the
    dense limit, and is solved by AMG-CG (coarse_solver 0) or Jacobi-PCG (1); the solve (on a
    stream, so the V-cycle with the coarse iteration is captured as a CUDA graph) still
    reaches 1e-10 and so does a block of right-hand sides."""
    s = torch.cuda.Stream()
    m, k = 17, 2
    with torch.cuda.stream(s):
        ctx = _ctx(m, k, deform=1, precision=precision, stream=s, coarse_solver=coarse_solver)
        assert ctx.num_dofs(0) == 18 ** 3
        b = torch.as_tensor(sipg_inputs.uniform(ctx.num_dofs(), sipg_inputs.SEED_RHS)).to(DEV)
        x = torch.zeros_like(b)
        for _ in range(2):   # the second solve replays the captured cycle
            x.zero_()
            info = ctx.solve(b, x, rtol=1e-10, maxit=40)
            assert info.converged and info.iterations <= 20, info.iterations
        r = torch.empty_like(b)
        ctx.apply(x, r)
        s.synchronize()
        assert (torch.linalg.norm(b - r) / torch.linalg.norm(b)).item() <= 2e-10
        B = torch.stack([b, -0.5 * b, torch.as_tensor(sipg_inputs.uniform(ctx.num_dofs(), 3)).to(DEV)])
        X = torch.zeros_like(B)
        infos = ctx.solve_multi(B, X, rtol=1e-10, maxit=40)
        s.synchronize()
        assert all(i.converged for i in infos)
        assert close(X[1].cpu().numpy(), -0.5 * x.cpu().numpy()) <= 1e-6
