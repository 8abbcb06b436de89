"""Timing of the learned smoother's network pass (the three forward GEMMs).

    python -m paper_1910_01900_gb300.mlpbench [--m M] [--k K] [--repeats R]

Builds the network of an m^3 curved mesh of degree k (inputs n^3 + 6 n^2, two
hidden layers of 256, outputs n^3, one row per cell), fills it with seeded
random weights and inputs, and times `sipg_mlp_forward` on all cells with
CUDA events (mean of R calls after 3 warm-ups).  The call includes the input
conversion to BF16, the output copy and a stream synchronisation, so the
GEMMs alone take less; the ncu capture of `gemm_tc_kernel` gives their time.
Prints one JSON line.
"""
import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=32)
    ap.add_argument("--k", type=int, default=4)
    ap.add_argument("--repeats", type=int, default=20)
    args = ap.parse_args(argv)
    import numpy as np
    import torch

    from . import Context
    ctx = Context(args.m, args.k, deform=1, precision=1)
    sh = ctx.mlp_shape()
    rng = np.random.default_rng(2024)
    flat = ctx.mlp_params()
    flat[:] = rng.standard_normal(flat.size).astype(np.float32) * 0.05
    ctx.mlp_params(flat)
    rows = args.m ** 3
    X = torch.as_tensor(rng.standard_normal((rows, sh["in_dim"])).astype(np.float32)).cuda()
    Y = torch.empty(rows * sh["out_pad"], dtype=torch.float32, device="cuda")
    for _ in range(3):
        ctx.mlp_forward(X, Y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.repeats):
        ctx.mlp_forward(X, Y)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.repeats
    flops = 2.0 * rows * (sh["in_pad"] * sh["hidden"] + sh["hidden"] ** 2 + sh["hidden"] * sh["out_pad"])
    print(json.dumps({"m": args.m, "k": args.k, "rows": rows, "shape": sh, "ms_per_call": ms,
                      "gemm_flop": flops, "tflops_incl_call_overhead": flops / (ms * 1e-3) / 1e12}))


if __name__ == "__main__":
    main()
