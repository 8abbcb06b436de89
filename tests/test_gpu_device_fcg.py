"""Flexible CG with the iteration gated on the device (Algorithm 1 structure).

On a non-default stream the solver runs its iterations as captured chunks whose
steps are conditional graph nodes: the device decides convergence, breakdown
and the iteration limit, and the host reads the state once per chunk.  On the
legacy default stream the same kernels run from a host loop that reads the
scalars every iteration.  Both paths launch the same kernels in the same order
on the same data, so solutions, residual histories and iteration counts agree
bit for bit; the edge cases (a limit that ends the solve, a fixed iteration
count, a zero start residual, a solve that ends before its first iteration)
end alike.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pair(**kw):
    from paper_1910_01900_gb300 import Context
    s = torch.cuda.Stream()
    return Context(stream=None, **kw), Context(stream=s, **kw), s


def _solve(ctx, s, b, x, **kw):
    torch.cuda.synchronize()   # inputs written on torch's stream
    if s is None:
        return ctx.solve(b, x, **kw)
    with torch.cuda.stream(s):
        info = ctx.solve(b, x, **kw)
    s.synchronize()
    return info


def _same(ih, idv, xh, xd):
    assert ih.iterations == idv.iterations
    assert ih.r0_norm == idv.r0_norm and ih.r_norm == idv.r_norm
    n = min(ih.iterations + 1, 256)
    assert list(ih.res_history[:n]) == list(idv.res_history[:n])
    assert torch.equal(xh, xd)


@pytest.mark.parametrize("k,precision,coarse", [(3, 1, 0), (2, 0, 0), (4, 1, 1)])
def test_device_gated_solve_matches_host_loop(k, precision, coarse):
    ch, cd, s = _pair(m=6, degree=k, deform=1, precision=precision, coarse_solver=coarse)
    b = torch.empty(ch.num_dofs(), dtype=torch.float64, device="cuda:0")
    ch.rhs(b)
    torch.cuda.synchronize()
    xh, xd = torch.zeros_like(b), torch.zeros_like(b)
    ih = _solve(ch, None, b, xh, rtol=1e-10, maxit=200)
    idv = _solve(cd, s, b, xd, rtol=1e-10, maxit=200)
    assert ih.converged and idv.converged
    _same(ih, idv, xh, xd)
    # a second solve from a nonzero start vector replays the same chunk graph
    xh2, xd2 = xh * 0.5, xd * 0.5
    ih = _solve(ch, None, b, xh2, rtol=1e-12, maxit=200)
    idv = _solve(cd, s, b, xd2, rtol=1e-12, maxit=200)
    _same(ih, idv, xh2, xd2)
    ch.close()
    cd.close()


def test_device_gated_limits_and_degenerate_cases():
    ch, cd, s = _pair(m=4, degree=3, precision=1)
    b = torch.empty(ch.num_dofs(), dtype=torch.float64, device="cuda:0")
    ch.rhs(b)
    torch.cuda.synchronize()
    # the iteration limit ends the solve (9 and 17 cross a chunk boundary)
    for maxit in (1, 3, 8, 9, 17):
        xh, xd = torch.zeros_like(b), torch.zeros_like(b)
        ih = _solve(ch, None, b, xh, rtol=1e-300, maxit=maxit, allow_notconv=True)
        idv = _solve(cd, s, b, xd, rtol=1e-300, maxit=maxit, allow_notconv=True)
        assert ih.iterations == maxit and not ih.converged and not idv.converged
        _same(ih, idv, xh, xd)
    # a fixed number of iterations, past the tolerance
    for fixed in (1, 8, 12):
        xh, xd = torch.zeros_like(b), torch.zeros_like(b)
        ih = _solve(ch, None, b, xh, rtol=1e-3, maxit=100, fixed_iters=fixed)
        idv = _solve(cd, s, b, xd, rtol=1e-3, maxit=100, fixed_iters=fixed)
        assert ih.iterations == fixed
        _same(ih, idv, xh, xd)
    # a zero right-hand side with a zero start vector: nothing to do
    z = torch.zeros_like(b)
    xd = torch.zeros_like(b)
    idv = _solve(cd, s, z, xd, rtol=1e-10, maxit=50)
    assert idv.iterations == 0 and idv.converged and not xd.any()
    # a tolerance of 1 is met by the start vector
    xh, xd = torch.zeros_like(b), torch.zeros_like(b)
    ih = _solve(ch, None, b, xh, rtol=1.0, maxit=50)
    idv = _solve(cd, s, b, xd, rtol=1.0, maxit=50)
    assert ih.iterations == 0
    _same(ih, idv, xh, xd)
    ch.close()
    cd.close()


def test_device_gated_solve_long_history():
    """More than 256 iterations: the history stops at 256 entries, the final
    residual is still the last iteration's."""
    ch, cd, s = _pair(m=4, degree=2, precision=0, cheb_degree=1)
    b = torch.empty(ch.num_dofs(), dtype=torch.float64, device="cuda:0")
    ch.rhs(b)
    torch.cuda.synchronize()
    xh, xd = torch.zeros_like(b), torch.zeros_like(b)
    ih = _solve(ch, None, b, xh, rtol=1e-30, maxit=300, fixed_iters=270)
    idv = _solve(cd, s, b, xd, rtol=1e-30, maxit=300, fixed_iters=270)
    assert ih.iterations == 270
    _same(ih, idv, xh, xd)
    ch.close()
    cd.close()
