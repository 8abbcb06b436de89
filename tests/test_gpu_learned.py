"""Learned smoother (GPU): network kernels against the CPU reference network,
training, and the flexible-CG solve with the network in place of Chebyshev."""
import numpy as np
import pytest

import sipg_inputs
from oracle import mlp
from parity_check import close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _split(flat, sh):
    Fp, H, No = sh["in_pad"], sh["hidden"], sh["out_pad"]
    o = 0
    parts = []
    for shape in ((Fp, H), (H,), (H, H), (H,), (H, No), (No,)):
        n = int(np.prod(shape))
        parts.append(flat[o:o + n].reshape(shape).astype(np.float64))
        o += n
    W1, b1, W2, b2, W3, b3 = parts
    return [W1[:sh["in_dim"]], W2, W3[:, :sh["out_dim"]]], [b1, b2, b3[:sh["out_dim"]]]


def _ctx(m, k, deform=1, precision=1):
    from paper_1910_01900_gb300 import Context
    return Context(m, k, deform=deform, precision=precision)


def test_features_match_oracle():
    m, k = (4, 3, 5), 3
    ctx = _ctx(m, k)
    sh = ctx.mlp_shape()
    n = ctx.num_dofs()
    r = sipg_inputs.uniform(n, 77)
    E = m[0] * m[1] * m[2]
    feat = torch.empty(E * sh["in_pad"], dtype=torch.float32, device=DEV)
    scale = torch.empty(E, dtype=torch.float32, device=DEV)
    ctx.mlp_features(torch.as_tensor(r).to(DEV), feat, scale)
    F = mlp.features(r, m, k + 1)
    s = np.sqrt(np.mean(F * F, axis=1))
    got = feat.cpu().numpy().reshape(E, sh["in_pad"])[:, :sh["in_dim"]]
    assert np.allclose(scale.cpu().numpy(), s, rtol=1e-6)
    assert np.max(np.abs(got - mlp.bf16_round(F / s[:, None]))) <= 2 ** -7 * np.max(np.abs(F / s[:, None]))


def test_forward_and_gradients_match_cpu_network():
    ctx = _ctx(4, 4)
    sh = ctx.mlp_shape()
    rng = np.random.default_rng(5)
    flat = ctx.mlp_params()
    flat[:] = rng.standard_normal(flat.size).astype(np.float32) * 0.05
    ctx.mlp_params(flat)
    Ws, bs = _split(flat, sh)
    B = 200
    X = rng.standard_normal((B, sh["in_dim"])).astype(np.float32)
    T = rng.standard_normal((B, sh["out_dim"])).astype(np.float32)
    Y = torch.empty(B * sh["out_pad"], dtype=torch.float32, device=DEV)
    ctx.mlp_forward(torch.as_tensor(X).to(DEV), Y)
    yref, _ = mlp.forward(X.astype(np.float64), Ws, bs, bf16=True)
    y = Y.cpu().numpy().reshape(B, sh["out_pad"])[:, :sh["out_dim"]]
    assert close(y, yref) <= 1e-2
    g, loss = ctx.mlp_gradients(torch.as_tensor(X).to(DEV), torch.as_tensor(T).to(DEV))
    # the oracle network rounds the same operands to BF16 as the GPU's products read
    L, gW, gb = mlp.loss_and_grads(X.astype(np.float64), T.astype(np.float64), Ws, bs, bf16=True)
    assert abs(loss - L) <= 1e-2 * L
    gWs, gbs = _split(g, sh)
    for a, b in zip(gWs + gbs, gW + gb):
        assert close(a, b) <= 1e-2


@pytest.mark.parametrize("k,B", [(4, 1), (4, 129), (5, 300), (6, 77)])
def test_forward_row_tails_and_widths(k, B):
    """The forward pass runs on tcgen05 tensor cores in 128-row tiles: partial last tiles,
    a single row, and an output width above one MMA tile (k = 6: 343 -> 352 columns, the
    mma.sync fallback) all match the CPU network."""
    ctx = _ctx(3, k)
    sh = ctx.mlp_shape()
    rng = np.random.default_rng(11 + B)
    flat = ctx.mlp_params()
    flat[:] = rng.standard_normal(flat.size).astype(np.float32) * 0.05
    ctx.mlp_params(flat)
    Ws, bs = _split(flat, sh)
    X = rng.standard_normal((B, sh["in_dim"])).astype(np.float32)
    Y = torch.full((B * sh["out_pad"],), float("nan"), dtype=torch.float32, device=DEV)
    ctx.mlp_forward(torch.as_tensor(X).to(DEV), Y)
    yref, _ = mlp.forward(X.astype(np.float64), Ws, bs, bf16=True)
    y = Y.cpu().numpy().reshape(B, sh["out_pad"])[:, :sh["out_dim"]]
    assert np.all(np.isfinite(y))
    assert close(y, yref) <= 1e-2


def test_training_and_learned_solve():
    """Train on pairs from the plain cycle; the FCG solve still reaches 1e-10."""
    m, k = 8, 3
    ctx = _ctx(m, k)
    info = ctx.train_smoother(npairs=40000, epochs=30, seed=7)
    assert info.loss_last < info.loss_first
    # what the network gains: one damped network step removes part of the residual the
    # post-smoother faces (after pre-smoothing and coarse-grid correction); 0.92 on this
    # small mesh, 0.75 on the 32^3 k=4 workload
    assert 0 < info.damping and info.step_reduction < 0.95, (info.damping, info.step_reduction)
    b = torch.as_tensor(sipg_inputs.uniform(ctx.num_dofs(), sipg_inputs.SEED_RHS)).to(DEV)
    x0 = torch.zeros_like(b)
    ref = ctx.solve(b, x0, rtol=1e-10)
    ctx.set_smoother(1, 2, 2)
    x1 = torch.zeros_like(b)
    got = ctx.solve(b, x1, rtol=1e-10, maxit=200)
    assert got.converged and got.learned == 1
    assert close(x1, x0) <= 1e-8
    ctx.set_smoother(1)   # default: Chebyshev pre-smoothing, one network post-step
    x2 = torch.zeros_like(b)
    got2 = ctx.solve(b, x2, rtol=1e-10, maxit=200)
    assert got2.converged and got2.learned == 1
    assert close(x2, x0) <= 1e-8
    # what the network adds to the V-cycle: the energy norm of the error left by one cycle with
    # Chebyshev pre-smoothing and no post-smoothing (the cycle without the network), and by the
    # same cycle with one network post-step
    r = torch.as_tensor(sipg_inputs.uniform(ctx.num_dofs(), 71)).to(DEV)
    xs = torch.zeros_like(r)
    ctx.set_smoother(0)
    assert ctx.solve(r, xs, rtol=1e-12).converged

    def energy(e):
        ae = torch.empty_like(e)
        ctx.apply(e, ae)
        return torch.dot(e, ae).item() ** 0.5

    def left_by_cycle():
        z = torch.empty_like(r)
        ctx.vcycle(r, z)
        return energy(xs - z) / energy(xs)
    ctx.set_smoother(1, 0, 0)
    without = left_by_cycle()
    ctx.set_smoother(1, 0, 1)
    with_net = left_by_cycle()
    assert with_net < without, (with_net, without)
    ctx.set_smoother(0)
    assert ref.converged


def test_energy_norm_finetuning():
    """Fine-tuning in the energy norm on the training snapshots lowers that loss, the
    energy-optimal damping is positive, a cycle with the tuned step leaves less energy-norm
    error than the cycle without post-smoothing, and the solve still reaches 1e-10 (with and
    without the Chebyshev fallback)."""
    m, k = 8, 3
    ctx = _ctx(m, k)
    ctx.train_smoother(npairs=40000, epochs=30, seed=7)
    info = ctx.finetune_smoother(epochs=30)
    assert info.loss_last < info.loss_first <= 1.5, (info.loss_first, info.loss_last)
    assert info.damping > 0
    r = torch.as_tensor(sipg_inputs.uniform(ctx.num_dofs(), 71)).to(DEV)
    xs = torch.zeros_like(r)
    ctx.set_smoother(0)
    assert ctx.solve(r, xs, rtol=1e-12).converged

    def left(which, pre, post):
        ctx.set_smoother(which, pre, post)
        z, az = torch.empty_like(r), torch.empty_like(r)
        ctx.vcycle(r, z)
        e = xs - z
        ctx.apply(e, az)
        ax = torch.empty_like(r)
        ctx.apply(xs, ax)
        torch.cuda.synchronize()
        return (torch.dot(e, az) / torch.dot(xs, ax)).item() ** 0.5
    assert left(1, 0, 1) < left(1, 0, 0)
    b = torch.as_tensor(sipg_inputs.uniform(ctx.num_dofs(), sipg_inputs.SEED_RHS)).to(DEV)
    x0 = torch.zeros_like(b)
    ctx.set_smoother(0)
    ctx.solve(b, x0, rtol=1e-10)
    for which in (1, 2):
        ctx.set_smoother(which, 0, 1)
        x1 = torch.zeros_like(b)
        got = ctx.solve(b, x1, rtol=1e-10, maxit=200)
        assert got.converged and close(x1, x0) <= 1e-8
        if which == 2:
            assert not got.fell_back
    ctx.set_smoother(0)
