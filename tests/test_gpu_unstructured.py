"""The SIPG operator on unstructured hexahedral meshes: GPU against the oracle.

Meshes are boxes written as unstructured meshes with shuffled vertex and cell
numbers and every cell's local vertex order turned by a proper rotation of the
cube, so that every relative orientation of two neighbours' faces occurs, and
with interior vertices moved (general trilinear cells).  The GPU reads the
neighbour's face point through an orientation code derived from shared vertex
ids; the oracle pairs face points by physical position.  Both must give the
same operator, element by element.
"""
import numpy as np
import pytest

import sipg_inputs
from oracle.unstructured import HexMesh, USIPG
from parity_check import close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _apply(ctx, u, dtype):
    v = torch.empty(len(u), dtype=dtype, device=DEV)
    ctx.apply(torch.as_tensor(u).to(DEV, dtype), v)
    torch.cuda.synchronize()
    return v.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("k,m,distort,deform", [(1, (4, 3, 3), 0.2, 0), (2, (3, 3, 4), 0.2, 1), (3, (4, 3, 3), 0.0, 1),
                                                (4, (3, 2, 2), 0.15, 0), (5, (2, 2, 3), 0.1, 1), (8, (2, 1, 1), 0.0, 0)])
def test_unstructured_apply_matches_oracle(k, m, distort, deform):
    from paper_1910_01900_gb300 import create_unstructured
    bc = (0, 1, 0, 1, 1, 0)
    V, C, F, _, _ = sipg_inputs.scrambled_box(m, 100 + k, distort=distort, bc=bc)
    ctx = create_unstructured(V, C, k, face_bc=F, deform=deform)
    assert ctx.num_dofs() == len(C) * (k + 1) ** 3
    ref = USIPG(HexMesh(V, C, F, deform=deform), k).assemble()
    u = sipg_inputs.uniform(ref.shape[0], sipg_inputs.SEED_APPLY)
    want = ref @ u
    assert close(_apply(ctx, u, torch.float64), want) <= 1e-12
    assert close(_apply(ctx, u, torch.float32), want) <= 1e-5


def test_every_tile_width_gives_identical_results():
    from paper_1910_01900_gb300 import create_unstructured
    from paper_1910_01900_gb300.csrc_info import max_cells_per_block
    k = 3
    V, C, F, _, _ = sipg_inputs.scrambled_box((5, 4, 3), 9, distort=0.2, bc=(1, 0, 0, 1, 0, 0))
    ctx = create_unstructured(V, C, k, face_bc=F, deform=1)
    for dt, prec in ((torch.float64, 0), (torch.float32, 1)):
        u = torch.as_tensor(sipg_inputs.uniform(ctx.num_dofs(), 5)).to(DEV, dt)
        ref = torch.empty_like(u)
        ctx.apply(u, ref)
        mx = max_cells_per_block(k + 1, 8 >> prec)
        for cb in sorted({1, 2, 5, mx // 2, mx}):
            for p in (0, 1):
                ctx.set_tile_shape(prec, p, cb)
            v = torch.full_like(u, float("nan"))
            ctx.apply(u, v)
            torch.cuda.synchronize()
            assert torch.equal(v, ref), (prec, cb)
        for p in (0, 1):
            ctx.set_tile_shape(prec, p, 0)


def test_neumann_null_space_and_symmetry():
    from paper_1910_01900_gb300 import create_unstructured
    k = 2
    V, C, F, _, _ = sipg_inputs.scrambled_box((3, 3, 3), 4, distort=0.2, bc=(1,) * 6)
    ctx = create_unstructured(V, C, k, face_bc=F, deform=1)
    n = ctx.num_dofs()
    one = _apply(ctx, np.ones(n), torch.float64)
    x, y = sipg_inputs.uniform(n, 1), sipg_inputs.uniform(n, 2)
    ax, ay = _apply(ctx, x, torch.float64), _apply(ctx, y, torch.float64)
    assert np.max(np.abs(one)) <= 1e-12 * np.max(np.abs(ax))
    assert abs(y @ ax - x @ ay) <= 1e-12 * np.linalg.norm(ax) * np.linalg.norm(y)


def test_bad_meshes_are_rejected():
    from paper_1910_01900_gb300 import SipgError, create_unstructured
    V, C, F, _, _ = sipg_inputs.scrambled_box((2, 2, 1), 3)
    bad = C.copy()
    bad[1, 3] = len(V)                      # vertex id out of range
    with pytest.raises(SipgError):
        create_unstructured(V, bad, 2)
    three = np.concatenate([C, C[:1]])      # the first cell twice: its faces are shared three ways
    with pytest.raises(SipgError):
        create_unstructured(V, three, 2)
