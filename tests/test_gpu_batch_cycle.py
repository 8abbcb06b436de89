"""One V-cycle for all problems of a batch, inside a device-gated lockstep FCG (GPU).

On a non-default stream a batch captures one graph for the V-cycle of all its
problems: the DG level and the FE level of the same degree of every problem
run as shared batched launches (the single-problem bodies, so each problem's
numbers do not change), the levels below as per-problem branches of the same
graph; the lockstep flexible CG runs in chunks of iterations gated on the
device.  Without a stream the batch takes the host-driven path (each
problem's own cycle graph on its own stream, one host read per iteration).
Both paths launch the same arithmetic in the same order, so the solutions,
iteration counts and residual histories agree bit for bit, and each problem
matches its single-problem solve.
"""
import pytest

import sipg_inputs
from parity_check import close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

PROBS = [dict(m=4, k=3), dict(m=6, k=2), dict(m=4, k=4), dict(m=(4, 6, 4), k=2), dict(m=3, k=6),
         dict(m=(5, 3, 4), k=5)]


def _rhs(B, i):
    return torch.as_tensor(sipg_inputs.uniform(B.num_dofs(i), sipg_inputs.SEED_RHS + 40 + i)).to(DEV)


def _pair(probs, precision):
    from paper_1910_01900_gb300 import Batch
    s = torch.cuda.Stream()
    return Batch(probs, precision=precision), Batch(probs, precision=precision, stream=s), s


def _solve(B, s, bs, **kw):
    xs = [torch.zeros_like(b) for b in bs]
    torch.cuda.synchronize()
    if s is None:
        infos = B.solve(bs, xs, **kw)
    else:
        with torch.cuda.stream(s):
            infos = B.solve(bs, xs, **kw)
        s.synchronize()
    torch.cuda.synchronize()
    return xs, infos


def _same(xa, ia, xb, ib):
    for i in range(len(xa)):
        assert ia[i].iterations == ib[i].iterations, i
        assert ia[i].r_norm == ib[i].r_norm and ia[i].converged == ib[i].converged, i
        n = min(ia[i].iterations + 1, 256)
        assert list(ia[i].res_history[:n]) == list(ib[i].res_history[:n]), i
        assert torch.equal(xa[i], xb[i]), i


@pytest.mark.parametrize("precision,deform", [(1, 0), (0, 0), (1, 1)])
def test_batched_cycle_equals_host_driven_batch_and_single_solves(precision, deform):
    from paper_1910_01900_gb300 import Context
    probs = [dict(p, deform=deform) for p in PROBS]
    Bh, Bd, s = _pair(probs, precision)
    bs = [_rhs(Bh, i) for i in range(len(probs))]
    xh, ih = _solve(Bh, None, bs, rtol=1e-10)
    xd, idv = _solve(Bd, s, bs, rtol=1e-10)
    assert all(i.converged for i in idv)
    _same(xh, ih, xd, idv)
    # a second solve replays the captured graphs
    xd2, idv2 = _solve(Bd, s, bs, rtol=1e-10)
    _same(xd, idv, xd2, idv2)
    for i, p in enumerate(probs):
        c = Context(p["m"], p["k"], deform=deform, precision=precision)
        x = torch.zeros_like(bs[i])
        info = c.solve(bs[i], x, rtol=1e-10)
        torch.cuda.synchronize()
        assert info.iterations == idv[i].iterations, i
        assert close(xd[i].cpu().numpy(), x.cpu().numpy()) <= (1e-12 if precision == 0 else 1e-9), i
        c.close()


def test_batched_cycle_limits_and_idle_problems():
    probs = PROBS[:4]
    Bh, Bd, s = _pair(probs, 1)
    bs = [_rhs(Bh, i) for i in range(len(probs))]
    bs[2] = torch.zeros_like(bs[2])   # a system with nothing to solve leaves before the first iteration
    for maxit in (1, 3, 8, 9, 17):
        xh, ih = _solve(Bh, None, bs, rtol=1e-300, maxit=maxit, allow_notconv=True)
        xd, idv = _solve(Bd, s, bs, rtol=1e-300, maxit=maxit, allow_notconv=True)
        assert [i.iterations for i in idv] == [maxit, maxit, 0, maxit]
        assert not idv[0].converged and idv[2].converged
        _same(xh, ih, xd, idv)
    xh, ih = _solve(Bh, None, bs, rtol=1e-10)
    xd, idv = _solve(Bd, s, bs, rtol=1e-10)
    _same(xh, ih, xd, idv)


def test_seeded_uneven_batch_on_a_stream():
    """The 16-problem draw (m in 8..24 even, k in 2..6) through the batched cycle: every problem
    reaches 1e-10 with the iteration count of the host-driven batch."""
    probs = sipg_inputs.batch_problems()
    Bh, Bd, s = _pair(probs, 1)
    bs = []
    for i in range(len(probs)):
        b = torch.empty(Bh.num_dofs(i), dtype=torch.float64, device=DEV)
        Bh.contexts[i].rhs(b)
        bs.append(b)
    torch.cuda.synchronize()
    xh, ih = _solve(Bh, None, bs, rtol=1e-10)
    xd, idv = _solve(Bd, s, bs, rtol=1e-10)
    assert all(i.converged for i in idv)
    _same(xh, ih, xd, idv)


@pytest.mark.parametrize("precision,deform", [(1, 0), (0, 1)])
def test_batched_cycle_equals_each_problems_cycle(precision, deform):
    """One V-cycle of every problem through the batched graph equals each context's own
    V-cycle (sipg_vcycle) bit for bit, with and without a stream."""
    probs = [dict(p, deform=deform) for p in PROBS]
    Bh, Bd, s = _pair(probs, precision)
    for B, st in ((Bd, s), (Bh, None)):
        rs = [_rhs(B, i) for i in range(len(probs))]
        zs = [torch.full_like(r, float("nan")) for r in rs]
        torch.cuda.synchronize()
        if st is None:
            B.vcycle(rs, zs)
        else:
            with torch.cuda.stream(st):
                B.vcycle(rs, zs)
        torch.cuda.synchronize()
        for i in range(len(probs)):
            z = torch.empty_like(rs[i])
            B.contexts[i].vcycle(rs[i], z)
            torch.cuda.synchronize()
            assert torch.equal(zs[i], z), i
