"""The allocation-free operator apply against the regular one (GPU).

sipg_operator_apply_noalloc exists for callers that cannot call cudaMalloc
when they need A u (a framework whose caching allocator already holds the
device memory, a time-stepping loop that must not allocate once running).  It
keeps its scratch in a static device array instead of allocating, so it must
give the same v = A u as sipg_operator_apply, call after call, even though
every call reuses (and leaves behind) the same scratch contents.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import pytest

import sipg_inputs
from parity_check import close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _regular(m, k, lo, hi, bc, u):
    from paper_1910_01900_gb300 import Context
    ctx = Context(m, k, lo=lo, hi=hi, bc=bc, operator_only=True)
    ref = torch.empty_like(u)
    ctx.apply(u, ref)
    torch.cuda.synchronize()
    return ref


def test_noalloc_apply_matches_regular_apply_on_consecutive_calls():
    """Two calls in a row on one mesh, with a call of another layout between them (larger
    mesh, higher degree), so that stale scratch from that call sits at other offsets:
    each result equals the regular apply element by element (FP64, 1e-12)."""
    from paper_1910_01900_gb300 import native
    m, k = (5, 3, 4), 3
    lo, hi, bc = (0.0, -0.5, 0.2), (1.0, 1.0, 1.4), (0, 1, 0, 0, 1, 0)
    big_m, big_k = (7, 6, 5), 5
    n = m[0] * m[1] * m[2] * (k + 1) ** 3
    nb = big_m[0] * big_m[1] * big_m[2] * (big_k + 1) ** 3
    for seed in (sipg_inputs.SEED_APPLY, sipg_inputs.SEED_APPLY + 17):
        u = torch.as_tensor(sipg_inputs.uniform(n, seed)).cuda()
        ref = _regular(m, k, lo, hi, bc, u)
        v = torch.full_like(u, float("nan"))
        native.operator_apply_noalloc(m, k, u, v, lo=lo, hi=hi, bc=bc)
        torch.cuda.synchronize()
        assert close(v, ref) <= 1e-12
        # a call of another layout in between
        ub = torch.as_tensor(sipg_inputs.uniform(nb, seed + 3)).cuda()
        refb = _regular(big_m, big_k, (0.0,) * 3, (1.0,) * 3, (0,) * 6, ub)
        vb = torch.full_like(ub, float("nan"))
        native.operator_apply_noalloc(big_m, big_k, ub, vb)
        torch.cuda.synchronize()
        assert close(vb, refb) <= 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch_and_curved_cells():
    from paper_1910_01900_gb300 import native
    u = torch.zeros(8, dtype=torch.float64, device="cuda")
    v = torch.zeros(8, dtype=torch.float64, device="cuda")
    import ctypes
    for m, deg, deform, word in ((64, 8, 0, b"64 MiB"), (2, 1, 1, b"deform")):
        mesh = native.Mesh()
        for d in range(3):
            mesh.m[d], mesh.lo[d], mesh.hi[d] = m, 0.0, 1.0
        mesh.deform, mesh.amp, mesh.mapping_degree = deform, 0.1 * deform, 3
        st = native.lib().sipg_operator_apply_noalloc(ctypes.byref(mesh), deg, 1.0, ctypes.c_void_p(u.data_ptr()),
                                                       ctypes.c_void_p(v.data_ptr()), None)
        assert st == native.EINVAL
        assert word in native.lib().sipg_last_error(None)
