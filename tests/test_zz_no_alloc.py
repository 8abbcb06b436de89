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
import numpy as np
import pytest

import sipg_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_apply_matches_regular_apply_on_consecutive_calls():
    from paper_1910_01900_gb300 import Context, native
    m, k = (5, 3, 4), 3
    lo, hi, bc = (0.0, -0.5, 0.2), (1.0, 1.0, 1.4), (0, 1, 0, 0, 1, 0)
    ctx = Context(m, k, lo=lo, hi=hi, bc=bc, operator_only=True)
    n = ctx.num_dofs()
    for seed in (sipg_inputs.SEED_APPLY, sipg_inputs.SEED_APPLY + 17):
        u = torch.as_tensor(sipg_inputs.uniform(n, seed)).cuda()
        ref = torch.empty_like(u)
        ctx.apply(u, ref)
        v = torch.full_like(u, float("nan"))
        native.operator_apply_noalloc(m, k, u, v, lo=lo, hi=hi, bc=bc)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(v - ref) / torch.linalg.norm(ref)).item()
        assert np.isfinite(err) and err <= 1e-12, err


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1910_01900_gb300 import native
    u = torch.zeros(8, dtype=torch.float64, device="cuda")
    v = torch.zeros(8, dtype=torch.float64, device="cuda")
    mesh = native.Mesh()
    for d in range(3):
        mesh.m[d], mesh.lo[d], mesh.hi[d] = 64, 0.0, 1.0
    import ctypes
    st = native.lib().sipg_operator_apply_noalloc(ctypes.byref(mesh), 8, 1.0, ctypes.c_void_p(u.data_ptr()),
                                                   ctypes.c_void_p(v.data_ptr()), None)
    assert st == native.EINVAL
    assert b"64 MiB" in native.lib().sipg_last_error(None)
