"""CPU reference of the learned per-element smoother network (not in the paper).

Test infrastructure: see ``oracle/__init__.py``.

The network maps the local residual of one DG cell to a correction of that
cell's values: input = the cell's n^3 residual values followed by, for each of
its six faces (order -x,+x,-y,+y,-z,+z), the neighbour's n^2 residual values on
the shared face (the neighbour's nodes on that face, in face-point order;
zeros on the domain boundary); output = n^3 correction values.  Inputs are
scaled by their root mean square s (per cell); the correction is
c * s * y with a global scale c fixed at training time.

Layers: y = W3^T relu(W2^T relu(W1^T x + b1) + b2) + b3 with weights stored
(fan_in, fan_out).  The GPU runs the contractions with BF16 operands and FP32
accumulation and stores the hidden activations in BF16; ``forward`` can
reproduce those rounding points (``bf16=True``) so the two agree up to the
summation order.

Parity unpinned by the paper (the paper has no learned part).  Pinned here by a
finite-difference gradient check of ``loss_and_grads`` (tests).
"""
import numpy as np


def bf16_round(x):
    """Round float64/float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def features(R, m, n):
    """Inputs of every cell from a DG residual vector R (cells x n^3), shape (E, n^3 + 6 n^2)."""
    E = m[0] * m[1] * m[2]
    R = np.asarray(R, dtype=np.float64).reshape(E, n, n, n)      # [cell][z][y][x]
    out = np.zeros((E, n ** 3 + 6 * n * n))
    out[:, :n ** 3] = R.reshape(E, -1)
    e = np.arange(E)
    ijk = np.stack([e % m[0], (e // m[0]) % m[1], e // (m[0] * m[1])], axis=1)
    stride = [1, m[0], m[0] * m[1]]
    col = n ** 3
    for d in range(3):
        for s in (0, 1):
            has = ijk[:, d] < m[d] - 1 if s else ijk[:, d] > 0
            nb = e + (stride[d] if s else -stride[d])
            # neighbour's face nodes: index along d is n-1 (neighbour below, s=0) or 0 (above, s=1)
            idx = 0 if s else n - 1
            if d == 0:
                face = R[:, :, :, idx]            # [z][y] -> (t1=y fastest, t2=z)
            elif d == 1:
                face = R[:, :, idx, :]            # [z][x] -> (t1=x, t2=z)
            else:
                face = R[:, idx, :, :]            # [y][x] -> (t1=x, t2=y)
            vals = face.reshape(E, n * n)
            blk = np.zeros((E, n * n))
            blk[has] = vals[nb[has]]
            out[:, col:col + n * n] = blk
            col += n * n
    return out


def init_params(sizes, seed):
    """He-uniform weights from a seeded generator, zero biases."""
    rng = np.random.default_rng(seed)
    Ws, bs = [], []
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / fi)
        Ws.append(rng.uniform(-lim, lim, (fi, fo)))
        bs.append(np.zeros(fo))
    return Ws, bs


def forward(X, Ws, bs, bf16=False):
    """Returns the output and the list of layer inputs (for backward)."""
    q = bf16_round if bf16 else (lambda a: a)
    acts = [q(X)]
    h = acts[0]
    for i, (W, b) in enumerate(zip(Ws, bs)):
        z = h @ q(W) + b
        if i < len(Ws) - 1:
            h = q(np.maximum(z, 0.0))
            acts.append(h)
        else:
            h = z
    return h, acts


def loss_and_grads(X, T, Ws, bs, bf16=False):
    """Mean squared error L = sum ||y - t||^2 / (2 B) and its gradients.

    With ``bf16=True`` the backward contractions take BF16 operands, as the
    forward ones do: the output error D = (y - t) / B and every error passed
    back through a layer are rounded to BF16 before they enter a product (the
    last layer's bias gradient sums the unrounded D).  These are the rounding
    points of a network whose matrix products all read BF16 values.
    """
    q = bf16_round if bf16 else (lambda a: a)
    B = X.shape[0]
    Y, acts = forward(X, Ws, bs, bf16)
    D = (Y - T) / B
    L = 0.5 * float(np.sum((Y - T) ** 2)) / B
    gW, gb = [None] * len(Ws), [None] * len(Ws)
    for i in range(len(Ws) - 1, -1, -1):
        Dq = q(D)
        gW[i] = acts[i].T @ Dq
        gb[i] = (D if i == len(Ws) - 1 else Dq).sum(axis=0)
        if i > 0:
            D = q(Dq @ q(Ws[i]).T) * (acts[i] > 0)
    return L, gW, gb
