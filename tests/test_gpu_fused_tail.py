"""The lower end of the V-cycle as one cluster launch (GPU).

Below a few thousand nodes the degree-1 FE levels of the hierarchy (their
Chebyshev steps through the 27-point stencils, the residual, the 2:1
restriction and prolongation) and the dense coarse solve run as one launch of
one thread-block cluster, barriers between the steps (Algorithms 2 and 3 on
those levels).  The launch does the arithmetic of the per-step launches in
their order, so a V-cycle, a solve and a batch with it equal the same with
one launch per step bit for bit; the library's launch count shows which of
the two ran.
"""
import pytest

import sipg_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _ctx(fuse, s=None, **kw):
    from paper_1910_01900_gb300 import Context
    return Context(fuse_tail=fuse, stream=s, **kw)


def _cycle(ctx, s, r):
    z = torch.full_like(r, float("nan"))
    torch.cuda.synchronize()
    if s is None:
        ctx.vcycle(r, z)
    else:
        with torch.cuda.stream(s):
            ctx.vcycle(r, z)
        s.synchronize()
    torch.cuda.synchronize()
    return z


def _tail_levels(ctx):
    """FE levels of degree 1 with at most 8192 nodes above the coarsest (those the tail takes)."""
    n = 0
    for l in range(1, ctx.num_levels - 1):
        kind, deg, _ = ctx.level_info(l)
        if kind != 1 or deg != 1 or ctx.num_dofs(l) > 8192:
            break
        n += 1
    return n


CASES = [dict(m=8, degree=3, deform=0, precision=1), dict(m=8, degree=3, deform=1, precision=0),
         dict(m=16, degree=5, deform=1, precision=1), dict(m=12, degree=2, deform=0, precision=0),
         dict(m=(12, 8, 6), degree=4, deform=1, precision=1, bc=(0, 1, 1, 0, 0, 1)),
         dict(m=6, degree=2, deform=0, precision=1, cheb_degree=1),
         dict(m=16, degree=2, deform=0, precision=0, cheb_degree=2, bc=(1, 0, 0, 1, 1, 0))]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join("%s%s" % kv for kv in c.items()))
def test_fused_tail_cycle_equals_per_step_launches(case):
    from paper_1910_01900_gb300 import native
    s = torch.cuda.Stream()
    a, b = _ctx(1, **case), _ctx(0, **case)
    assert _tail_levels(a) >= 1
    r = torch.as_tensor(sipg_inputs.uniform(a.num_dofs(), sipg_inputs.SEED_RHS + 7)).to(DEV)
    za = _cycle(a, None, r)
    zb = _cycle(b, None, r)
    assert torch.isfinite(za).all()
    assert torch.equal(za, zb)
    # the per-step path launches every step of the tail's levels, the fused one a single kernel
    n0 = native.launch_count()
    _cycle(a, None, r)
    n1 = native.launch_count()
    _cycle(b, None, r)
    n2 = native.launch_count()
    t = _tail_levels(a)
    ns = case.get("cheb_degree", 5)
    # per tail level: 2 ns Chebyshev steps, residual, restriction, prolongation; plus the coarse
    # solve.  Without the tail, the top tail level's first step rides on the restriction into it
    # where that ends in a node pass (from a DG level or an FE level of degree >= 3; degrees 1 and
    # 2 restrict node by node in one launch of their own)
    kind_above, deg_above, _ = a.level_info(t + 1)
    folded = kind_above == 0 or deg_above >= 3
    assert (n2 - n1) - (n1 - n0) == t * (2 * ns + 3) - (1 if folded else 0)
    # on a stream the cycle is captured as a graph and replayed: same bits
    a2, b2 = _ctx(1, s, **case), _ctx(0, s, **case)
    for _ in range(3):
        assert torch.equal(_cycle(a2, s, r), za)
        assert torch.equal(_cycle(b2, s, r), za)
    for c in (a, b, a2, b2):
        c.close()


@pytest.mark.parametrize("precision,deform", [(1, 1), (0, 0)])
def test_fused_tail_solve_equals_per_step_solve(precision, deform):
    s = torch.cuda.Stream()
    kw = dict(m=16, degree=3, deform=deform, precision=precision)
    out = []
    for fuse in (1, 0):
        for st in (None, s):
            c = _ctx(fuse, st, **kw)
            bb = torch.empty(c.num_dofs(), dtype=torch.float64, device=DEV)
            c.rhs(bb)
            x = torch.zeros_like(bb)
            torch.cuda.synchronize()
            if st is None:
                info = c.solve(bb, x, rtol=1e-10)
            else:
                with torch.cuda.stream(st):
                    info = c.solve(bb, x, rtol=1e-10)
                st.synchronize()
            torch.cuda.synchronize()
            assert info.converged
            out.append((info.iterations, list(info.res_history[:info.iterations + 1]), x))
            c.close()
    for it, hist, x in out[1:]:
        assert it == out[0][0] and hist == out[0][1]
        assert torch.equal(x, out[0][2])


def test_fused_tail_in_the_batched_cycle():
    """The batched cycle enters each problem's cycle below its two finest levels: the fused
    tail of that level replaces the per-step launches there, with the same bits."""
    from paper_1910_01900_gb300 import Batch
    probs = [dict(m=8, k=3), dict(m=16, k=2), dict(m=12, k=4), dict(m=6, k=2)]
    s = torch.cuda.Stream()
    out = []
    for fuse in (1, 0):
        B = Batch(probs, precision=1, stream=s, fuse_tail=fuse)
        bs = [torch.as_tensor(sipg_inputs.uniform(B.num_dofs(i), sipg_inputs.SEED_RHS + 60 + i)).to(DEV)
              for i in range(len(probs))]
        xs = [torch.zeros_like(b) for b in bs]
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            infos = B.solve(bs, xs, rtol=1e-10)
        s.synchronize()
        assert all(i.converged for i in infos)
        out.append(([i.iterations for i in infos], xs))
    assert out[0][0] == out[1][0]
    for xa, xb in zip(out[0][1], out[1][1]):
        assert torch.equal(xa, xb)
