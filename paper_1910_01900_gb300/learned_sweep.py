"""Time to 1e-10 with the learned smoother against Chebyshev: a sweep.

    python -m paper_1910_01900_gb300.learned_sweep [--m 32] [--k 4]

The learned-smoother workload: 32^3 curved cells, k = 4, FP32 V-cycle, FP64
flexible CG to 1e-10 from x = 0 with a seeded uniform right-hand side (seed
1911).  For each training budget (pairs x epochs, seed 2024) the network is
trained once, then the solve runs with each learned cycle (steps_pre network
pre-steps, 0 = Chebyshev pre-smoothing; steps_post network post-steps) and
reports iterations, time (CUDA events on the library stream, median of 3
after one warm-up), whether the Chebyshev rate test switched the solve back
to Chebyshev (fell_back), and what one learned cycle leaves of the energy-
norm error of x* = A^-1 r (as learned_gain); each learned cycle runs with
the fallback and without it (smoother 2: the network alone, maxit 100).
One budget's network is then fine-tuned in the energy norm (cumulative 50,
200, 500 and 1000 passes over the training snapshots, learning rate 3e-4)
and measured again after each stage.  Chebyshev(d, d) cycles for d =
1, 2, 3, 5 on the same problem give the reference: the network replaces
smoothing steps, so it has to beat the cheaper Chebyshev cycles too.  One
JSON line per row.
"""
import argparse
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import sipg_inputs  # noqa: E402  (seeded input generators)

BUDGETS = [(25000, 20), (100000, 20), (100000, 60), (300000, 20)]
CYCLES = [(0, 1), (0, 2), (0, 3), (1, 1), (2, 2)]
# energy-norm fine-tuning (sipg_smoother_finetune) of one budget's network,
# passes added at each row (cumulative 50, 200, 500, 1000)
FINETUNE_BUDGET = (100000, 20)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=32)
    ap.add_argument("--k", type=int, default=4)
    ap.add_argument("--repeats", type=int, default=3)
    ap.add_argument("--finetune-passes", type=int, nargs="*", default=[50, 150, 300, 500])
    ap.add_argument("--finetune-lr", type=float, default=3e-4)
    args = ap.parse_args(argv)
    import torch

    from . import Context
    s = torch.cuda.Stream()

    def timed_solve(ctx, b):
        x = torch.zeros_like(b)
        with torch.cuda.stream(s):
            ts, info = [], None
            for rep in range(args.repeats + 1):
                x.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                info = ctx.solve(b, x, rtol=1e-10, maxit=100, allow_notconv=True)
                e1.record(s)
                e1.synchronize()
                if rep:
                    ts.append(e0.elapsed_time(e1))
        return float(np.median(ts)), info

    def energy_left(ctx, r, xs, e0):
        z, az = torch.empty_like(r), torch.empty_like(r)
        torch.cuda.synchronize()
        ctx.vcycle(r, z)   # on the library stream
        s.synchronize()
        d = xs - z
        torch.cuda.synchronize()
        ctx.apply(d, az)
        s.synchronize()
        return torch.dot(d, az).item() ** 0.5 / e0

    with torch.cuda.stream(s):
        ref = Context(args.m, args.k, deform=1, precision=1, stream=s)
    n = ref.num_dofs()
    b = torch.as_tensor(sipg_inputs.uniform(n, sipg_inputs.SEED_RHS)).cuda()
    r = torch.as_tensor(sipg_inputs.uniform(n, 71)).cuda()
    xs = torch.zeros_like(r)
    with torch.cuda.stream(s):
        ref.solve(r, xs, rtol=1e-12, maxit=200)
    s.synchronize()
    ax = torch.empty_like(xs)
    ref.apply(xs, ax)
    s.synchronize()
    e0 = torch.dot(xs, ax).item() ** 0.5
    for d in (1, 2, 3, 5):
        with torch.cuda.stream(s):
            ctx = Context(args.m, args.k, deform=1, precision=1, stream=s, cheb_degree=d)
        ms, info = timed_solve(ctx, b)
        print(json.dumps({"cycle": "chebyshev(%d,%d)" % (d, d), "iterations": info.iterations, "ms": round(ms, 3),
                          "converged": bool(info.converged),
                          "energy_error_left": energy_left(ctx, r, xs, e0)}), flush=True)
        ctx.close()
    for npairs, epochs in BUDGETS:
        with torch.cuda.stream(s):
            ctx = Context(args.m, args.k, deform=1, precision=1, stream=s)
            t = ctx.train_smoother(npairs=npairs, epochs=epochs, seed=2024)
        tuned = 0
        for extra in ([0] + args.finetune_passes if (npairs, epochs) == FINETUNE_BUDGET else (0,)):
            if extra:   # energy-norm fine-tuning on top (cumulative passes)
                with torch.cuda.stream(s):
                    t = ctx.finetune_smoother(epochs=extra, lr=args.finetune_lr)
                s.synchronize()
                tuned += extra
            for pre, post in (CYCLES if not tuned else CYCLES[:2]):
                for which in (1, 2):   # with and without the Chebyshev fallback
                    ctx.set_smoother(which, pre, post)
                    ms, info = timed_solve(ctx, b)
                    print(json.dumps({"cycle": "learned pre %d post %d" % (pre, post), "fallback": which == 1,
                                      "pairs": npairs, "epochs": epochs, "energy_passes": tuned,
                                      "train_s": round(t.seconds, 2),
                                      "loss": [round(t.loss_first, 4), round(t.loss_last, 4)],
                                      "damping": round(t.damping, 3), "iterations": info.iterations,
                                      "ms": round(ms, 3), "converged": bool(info.converged),
                                      "fell_back": bool(info.fell_back),
                                      "energy_error_left": energy_left(ctx, r, xs, e0)}), flush=True)
        ctx.close()


if __name__ == "__main__":
    main()
