"""Pins of the CPU reference of the learned smoother network (no paper counterpart)."""
import numpy as np

from oracle import mlp


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    sizes = [11, 7, 6, 5]
    Ws, bs = mlp.init_params(sizes, 3)
    for b in bs:
        b[:] = rng.standard_normal(b.shape) * 0.1
    X = rng.standard_normal((9, 11))
    T = rng.standard_normal((9, 5))
    L, gW, gb = mlp.loss_and_grads(X, T, Ws, bs)
    eps = 1e-6
    for i in range(3):
        for (a, c) in [(0, 0), (1, 2), (Ws[i].shape[0] - 1, Ws[i].shape[1] - 1)]:
            Wp = [w.copy() for w in Ws]
            Wp[i][a, c] += eps
            Wm = [w.copy() for w in Ws]
            Wm[i][a, c] -= eps
            fd = (mlp.loss_and_grads(X, T, Wp, bs)[0] - mlp.loss_and_grads(X, T, Wm, bs)[0]) / (2 * eps)
            assert abs(fd - gW[i][a, c]) <= 1e-6 * max(1.0, abs(fd))
        for c in (0, bs[i].shape[0] - 1):
            bp = [v.copy() for v in bs]
            bp[i][c] += eps
            bm = [v.copy() for v in bs]
            bm[i][c] -= eps
            fd = (mlp.loss_and_grads(X, T, Ws, bp)[0] - mlp.loss_and_grads(X, T, Ws, bm)[0]) / (2 * eps)
            assert abs(fd - gb[i][c]) <= 1e-6 * max(1.0, abs(fd))


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0, 1e-3])
    r = mlp.bf16_round(x)
    assert r[0] == 1.0 and r[3] == -2.5 and r[4] == 0.0
    assert r[1] == 1.0                      # exactly half an ulp: ties to even
    assert r[2] == 1.0 + 2 ** -7            # above half: rounds up
    assert abs(r[5] - 1e-3) <= 2 ** -8 * 1e-3


def test_features_layout():
    m, n = (3, 2, 2), 3
    E = 12
    R = np.arange(E * n ** 3, dtype=np.float64)
    F = mlp.features(R, m, n)
    assert F.shape == (E, n ** 3 + 6 * n * n)
    assert np.all(F[:, :n ** 3] == R.reshape(E, -1))
    # cell 1 (i=1,j=0,k=0): its -x neighbour is cell 0, whose +x face nodes (x = n-1) come first
    cell0 = R.reshape(E, n, n, n)[0]
    assert np.all(F[1, n ** 3:n ** 3 + n * n] == cell0[:, :, n - 1].ravel())
    # boundary faces are zero
    assert np.all(F[0, n ** 3:n ** 3 + n * n] == 0)


def test_bf16_gradients_stay_within_bf16_error_of_exact_ones():
    """The BF16 mode rounds operands only: its gradients differ from the exact (FP64) ones by
    a few BF16 ulps relative (2^-8 each), not by a dropped or transposed term."""
    rng = np.random.default_rng(4)
    sizes = [40, 32, 32, 20]
    Ws, bs = mlp.init_params(sizes, 5)
    for b in bs:
        b[:] = rng.standard_normal(b.shape) * 0.1
    X = rng.standard_normal((64, 40))
    T = rng.standard_normal((64, 20))
    L, gW, gb = mlp.loss_and_grads(X, T, Ws, bs)
    Lq, gWq, gbq = mlp.loss_and_grads(X, T, Ws, bs, bf16=True)
    assert abs(Lq - L) <= 2e-2 * L
    for a, b in zip(gWq + gbq, gW + gb):
        assert np.linalg.norm(a - b) <= 3e-2 * np.linalg.norm(b)
        assert np.linalg.norm(a - b) > 0          # the rounding is really applied
