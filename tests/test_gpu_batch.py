"""Batched problems (persistent launch, lockstep FCG) and many right-hand sides (GPU).

The batch path must give each problem exactly what the single-problem path
gives (same sum-factorisation bodies, same cell grouping) and what the oracle
gives.
"""
import numpy as np
import pytest

import sipg_inputs
from oracle.dg import SIPG
from oracle.mesh import Mesh
from oracle.multigrid import CPHMultigrid, fcg
from parity_check import close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


PROBS = [dict(m=4, k=2), dict(m=(6, 4, 3), k=3), dict(m=4, k=5), dict(m=(2, 3, 2), k=8), dict(m=(7, 6, 5), k=1),
         dict(m=3, k=6)]


@pytest.mark.parametrize("deform", [0, 1])
def test_batched_apply_equals_single_problem_and_oracle(deform):
    from paper_1910_01900_gb300 import Batch
    probs = [dict(p, deform=deform) for p in PROBS]
    B = Batch(probs)
    us, vs, refs = [], [], []
    for i, p in enumerate(probs):
        n = B.num_dofs(i)
        u = torch.as_tensor(sipg_inputs.uniform(n, 50 + i)).to(DEV)
        ref = torch.empty_like(u)
        B.contexts[i].apply(u, ref)
        torch.cuda.synchronize()
        us.append(u)
        vs.append(torch.full_like(u, float("nan")))
        refs.append(ref)
    B.apply(us, vs)
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        assert close(vs[i].cpu().numpy(), refs[i].cpu().numpy()) <= 1e-14, i
        o = SIPG(Mesh(p["m"], deform=deform), p["k"]).apply(us[i].cpu().numpy())
        assert close(vs[i].cpu().numpy(), o) <= 1e-12, i


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_solve_equals_single_solves(precision):
    from paper_1910_01900_gb300 import Batch, Context
    probs = [dict(m=4, k=3), dict(m=6, k=2), dict(m=4, k=4), dict(m=(4, 6, 4), k=2)]
    B = Batch(probs, precision=precision)
    bs = [torch.as_tensor(sipg_inputs.uniform(B.num_dofs(i), sipg_inputs.SEED_RHS + i)).to(DEV)
          for i in range(len(probs))]
    xs = [torch.zeros_like(b) for b in bs]
    infos = B.solve(bs, xs, rtol=1e-10)
    for i, p in enumerate(probs):
        c = Context(p["m"], p["k"], precision=precision)
        x = torch.zeros_like(bs[i])
        info = c.solve(bs[i], x, rtol=1e-10)
        assert infos[i].converged and infos[i].iterations == info.iterations, i
        assert close(xs[i].cpu().numpy(), x.cpu().numpy()) <= (1e-12 if precision == 0 else 1e-9), i
    # and one of them against the oracle's solve
    mg = CPHMultigrid(Mesh(4), 3)
    bo = bs[0].cpu().numpy()
    xo, it, _ = fcg(mg.levels[-1].apply, bo, np.zeros_like(bo), mg.vcycle, rtol=1e-10)
    # the FP32 cycle is the FP64 cycle rounded: a different (nearby) preconditioner, so its
    # count may move by one where the residual crosses 1e-10 between two iterations
    assert abs(infos[0].iterations - it) <= (0 if precision == 0 else 1)
    assert close(xs[0].cpu().numpy(), xo) <= (1e-10 if precision == 0 else 1e-8)


def test_seeded_uneven_batch_converges():
    """The 16-problem draw (m in 8..24 even, k in 2..6): every problem reaches 1e-10."""
    from paper_1910_01900_gb300 import Batch
    probs = sipg_inputs.batch_problems()
    B = Batch(probs, precision=1)
    bs, xs = [], []
    for i in range(len(probs)):
        b = torch.empty(B.num_dofs(i), dtype=torch.float64, device=DEV)
        B.contexts[i].rhs(b)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    infos = B.solve(bs, xs, rtol=1e-10)
    for i in range(len(probs)):
        assert infos[i].converged, i
        r = torch.empty_like(bs[i])
        B.contexts[i].apply(xs[i], r)
        torch.cuda.synchronize()   # the problem's context works on its own stream
        res = (torch.linalg.norm(bs[i] - r) / torch.linalg.norm(bs[i])).item()
        assert res <= 2e-10, (i, res)
        assert 3 <= infos[i].iterations <= 12, (i, infos[i].iterations)


def test_32_right_hand_sides():
    """32 seeded RHS on the 16^3 k=4 mesh, FP32 V-cycle / FP64 FCG."""
    from paper_1910_01900_gb300 import Batch, Context
    nrhs = 32
    B = Batch([dict(m=16, k=4)] * nrhs, precision=1)
    n = B.num_dofs(0)
    bs = [torch.as_tensor(sipg_inputs.uniform(n, sipg_inputs.SEED_RHS + r)).to(DEV) for r in range(nrhs)]
    xs = [torch.zeros_like(b) for b in bs]
    infos = B.solve(bs, xs, rtol=1e-10)
    assert all(i.converged for i in infos)
    c = Context(16, 4, precision=1)
    for r in (0, 17, 31):
        x = torch.zeros_like(bs[r])
        info = c.solve(bs[r], x, rtol=1e-10)
        assert info.iterations == infos[r].iterations
        assert close(xs[r].cpu().numpy(), x.cpu().numpy()) <= 1e-9


@pytest.mark.parametrize("precision,deform,vec_dtype", [(0, 0, torch.float64), (1, 1, torch.float32),
                                                      (0, 1, torch.float32)])
def test_apply_multi_equals_single_applies(precision, deform, vec_dtype):
    """One launch per pass for nv vectors of one operator: each row equals the single apply
    (also FP32 vectors on a context whose cycle runs in FP64: scratch made on first use)."""
    from paper_1910_01900_gb300 import Context
    m, k, nv = (6, 4, 5), 3, 7
    ctx = Context(m, k, deform=deform, precision=precision)
    n = ctx.num_dofs()
    dt = vec_dtype
    U = torch.stack([torch.as_tensor(sipg_inputs.uniform(n, 70 + r)) for r in range(nv)]).to(DEV, dt)
    V = torch.full_like(U, float("nan"))
    ctx.apply_multi(U, V)
    torch.cuda.synchronize()
    o = SIPG(Mesh(m, deform=deform), k)
    for r in range(nv):
        ref = torch.empty_like(U[r])
        ctx.apply(U[r].contiguous(), ref)
        torch.cuda.synchronize()
        assert torch.equal(V[r], ref), r
        assert close(V[r].cpu().numpy(), o.apply(U[r].cpu().numpy().astype(np.float64))) <= \
            (1e-12 if dt == torch.float64 else 1e-5)


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_multi_equals_single_solves(precision):
    """nrhs right-hand sides in lockstep through multi-vector V-cycles: the same iteration
    counts and solutions as one solve per right-hand side, and the oracle's solve."""
    from paper_1910_01900_gb300 import Context
    m, k, nrhs = 4, 3, 6
    ctx = Context(m, k, precision=precision)
    n = ctx.num_dofs()
    B = torch.stack([torch.as_tensor(sipg_inputs.uniform(n, sipg_inputs.SEED_RHS + r)) for r in range(nrhs)]).to(DEV)
    B[3] *= 1e3                 # scaled right-hand side: same iterates up to the scale
    X = torch.zeros_like(B)
    infos = ctx.solve_multi(B, X, rtol=1e-10)
    torch.cuda.synchronize()
    single = Context(m, k, precision=precision)
    for r in range(nrhs):
        x = torch.zeros(n, dtype=torch.float64, device=DEV)
        info = single.solve(B[r].contiguous(), x, rtol=1e-10)
        assert infos[r].converged and infos[r].iterations == info.iterations, r
        assert close(X[r].cpu().numpy(), x.cpu().numpy()) <= (1e-12 if precision == 0 else 1e-9), r
    mg = CPHMultigrid(Mesh(m), k)
    bo = B[0].cpu().numpy()
    xo, it, _ = fcg(mg.levels[-1].apply, bo, np.zeros_like(bo), mg.vcycle, rtol=1e-10)
    assert close(X[0].cpu().numpy(), xo) <= (1e-10 if precision == 0 else 1e-8)
    if precision == 0:
        assert infos[0].iterations == it
    # a second call with fewer right-hand sides reuses the work set
    X2 = torch.zeros_like(B[:2])
    infos2 = ctx.solve_multi(B[:2].contiguous(), X2, rtol=1e-10)
    torch.cuda.synchronize()
    assert torch.equal(X2, X[:2]) and [i.iterations for i in infos2] == [i.iterations for i in infos[:2]]
    # more right-hand sides than before: the work set grows, the cycle graph is captured anew
    B3 = torch.cat([B, B[:3] * -2.0])
    X3 = torch.zeros_like(B3)
    infos3 = ctx.solve_multi(B3, X3, rtol=1e-10)
    torch.cuda.synchronize()
    assert torch.equal(X3[:nrhs], X) and all(i.converged for i in infos3)
    assert close(X3[nrhs:].cpu().numpy(), -2.0 * X[:3].cpu().numpy()) <= 1e-9


def test_solve_multi_zero_and_nan_rows():
    """A zero right-hand side stops at once with x = 0; a non-finite one is refused."""
    from paper_1910_01900_gb300 import Context
    from paper_1910_01900_gb300.native import SipgError
    ctx = Context(4, 2)
    n = ctx.num_dofs()
    B = torch.stack([torch.as_tensor(sipg_inputs.uniform(n, 5)), torch.zeros(n, dtype=torch.float64)]).to(DEV)
    X = torch.zeros_like(B)
    infos = ctx.solve_multi(B, X, rtol=1e-10)
    torch.cuda.synchronize()
    assert infos[0].converged and infos[1].converged and infos[1].iterations == 0
    assert float(X[1].abs().max()) == 0.0
    B[1, 17] = float("nan")
    with pytest.raises(SipgError):
        ctx.solve_multi(B, torch.zeros_like(B), rtol=1e-10)
