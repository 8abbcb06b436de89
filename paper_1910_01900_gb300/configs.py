"""Solve-time measurements of the named workloads (one JSON line each).

    python -m paper_1910_01900_gb300.configs [--which NAME ...] [--steps K]

cube4_k3        4^3 Cartesian, k=3, manufactured RHS: FP64 multigrid and mixed precision.
cube32_k4       32^3 Cartesian, k=4 (4.1 MDoF), manufactured RHS: mixed precision vs plain FP64 multigrid.
batch16         the 16 seeded problems (m in 8..24 even, k in 2..6), FP32 cycle / FP64 FCG:
                one batch (persistent launches, lockstep FCG) vs the 16 solves one after another.
rhs32           32 seeded right-hand sides on 16^3 k=4: batch, one N x 32 block on one
                context (sipg_solve_multi) and one after another.
curved32_k4     32^3 curved, k=4: learned smoother (trained on 10^5 pairs) vs Chebyshev,
                iterations and time to 1e-10.

Times are CUDA-event times on the library stream (b and x on the device), the
median of K repetitions after one warm-up; setup and training are reported
separately.  cube4_k3 and cube32_k4 also report the L2 error of each solution
against the exact sine solution and the mixed-precision solution's relative
difference from the FP64 one.
"""
import argparse
import json
import sys
import time

import os

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import sipg_inputs  # noqa: E402  (seeded input generators, shared with the tests)

SEED_RHS = sipg_inputs.SEED_RHS
_uniform = sipg_inputs.uniform


def _timed(fn, steps, stream):
    import torch
    fn()
    ts = []
    out = None
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts)), out


def run_single(name, m, k, deform, steps, stream, rhs="manufactured"):
    import torch

    from . import Context
    res = {"workload": name}
    for prec in (0, 1):
        t0 = time.perf_counter()
        ctx = Context(m, k, deform=deform, precision=prec, stream=stream)
        setup = time.perf_counter() - t0
        N = ctx.num_dofs()
        if rhs == "manufactured":
            b = torch.empty(N, dtype=torch.float64, device="cuda")
            ctx.rhs(b)
        else:
            b = torch.as_tensor(_uniform(N, SEED_RHS)).cuda()
        x = torch.zeros_like(b)

        def solve():
            x.zero_()
            return ctx.solve(b, x, rtol=1e-10)
        with torch.cuda.stream(stream):
            ms, info = _timed(solve, steps, stream)
        key = "fp64_mg" if prec == 0 else "mixed"
        res[key] = {"ms": ms, "s_per_mdof": ms * 1e-3 * 1e6 / N, "iterations": info.iterations,
                    "n10": info.n10, "setup_s": setup, "dofs": N}
        stream.synchronize()
        if rhs == "manufactured":   # discretisation error against the exact sine solution
            res[key]["l2_error_vs_exact"] = ctx.l2_error(x)
        if prec == 0:
            x_fp64 = x.clone()
        else:                       # what the FP32 V-cycle changes in the converged solution
            res[key]["rel_diff_vs_fp64_solution"] = (torch.linalg.norm(x - x_fp64) /
                                                     torch.linalg.norm(x_fp64)).item()
        ctx.close()
    res["speedup_mixed_vs_fp64_mg"] = res["fp64_mg"]["ms"] / res["mixed"]["ms"]
    return res


def run_batch(name, problems, steps, stream):
    import torch

    from . import Batch, Context
    t0 = time.perf_counter()
    B = Batch(problems, precision=1, stream=stream)
    setup = time.perf_counter() - t0
    bs, xs = [], []
    for i, p in enumerate(problems):
        n = B.num_dofs(i)
        if name == "rhs32":
            b = torch.as_tensor(_uniform(n, SEED_RHS + i)).cuda()
        else:
            b = torch.empty(n, dtype=torch.float64, device="cuda")
            B.contexts[i].rhs(b)
        bs.append(b)
        xs.append(torch.zeros_like(b))

    def solve_batch():
        for x in xs:
            x.zero_()
        return B.solve(bs, xs, rtol=1e-10)
    with torch.cuda.stream(stream):
        ms_b, infos = _timed(solve_batch, steps, stream)
    total = sum(B.num_dofs(i) for i in range(len(problems)))
    # the same problems solved one after another with separate contexts
    ctxs = [Context(p["m"], p["k"], deform=p.get("deform", 0), precision=1, stream=stream) for p in problems] \
        if name != "rhs32" else [Context(problems[0]["m"], problems[0]["k"], precision=1, stream=stream)]

    def solve_seq():
        its = []
        for i in range(len(problems)):
            c = ctxs[i] if len(ctxs) > 1 else ctxs[0]
            xs[i].zero_()
            its.append(c.solve(bs[i], xs[i], rtol=1e-10).iterations)
        return its
    with torch.cuda.stream(stream):
        ms_s, its = _timed(solve_seq, steps, stream)
    res = {"workload": name, "problems": len(problems), "dofs_total": total, "setup_s": setup,
           "batch_ms": ms_b, "sequential_ms": ms_s, "speedup_batch_vs_sequential": ms_s / ms_b,
           "batch_s_per_mdof": ms_b * 1e-3 * 1e6 / total,
           "iterations": [i.iterations for i in infos], "sequential_iterations": its,
           "all_converged": all(i.converged for i in infos)}
    if name == "rhs32":
        # the same right-hand sides as one N x 32 block on one context (sipg_solve_multi)
        c = ctxs[0]
        Bm = torch.stack(bs)
        Xm = torch.zeros_like(Bm)

        def solve_multi():
            Xm.zero_()
            return c.solve_multi(Bm, Xm, rtol=1e-10)
        with torch.cuda.stream(stream):
            ms_m, minfos = _timed(solve_multi, steps, stream)
        res.update({"multi_ms": ms_m, "multi_s_per_mdof": ms_m * 1e-3 * 1e6 / total,
                    "speedup_multi_vs_sequential": ms_s / ms_m,
                    "multi_iterations": [i.iterations for i in minfos],
                    "multi_all_converged": all(i.converged for i in minfos),
                    "multi_rel_diff_vs_sequential": float(torch.linalg.norm(Xm - torch.stack(xs)) /
                                                     torch.linalg.norm(torch.stack(xs)))})
    return res


def run_learned(steps, stream, npairs=100000, epochs=20):
    import torch

    from . import Context
    m, k = 32, 4
    ctx = Context(m, k, deform=1, precision=1, stream=stream)
    N = ctx.num_dofs()
    with torch.cuda.stream(stream):
        info = ctx.train_smoother(npairs=npairs, epochs=epochs, seed=2024)
    b = torch.as_tensor(_uniform(N, SEED_RHS + 99)).cuda()
    x = torch.zeros_like(b)
    out = {"workload": "curved32_k4", "dofs": N, "train": {"pairs": info.npairs, "epochs": info.epochs,
                                                           "loss_first": info.loss_first,
                                                           "loss_last": info.loss_last,
                                                           "seconds": info.seconds,
                                                           "chebyshev_rate": info.cheb_rate,
                                                           "iter_ms_chebyshev": info.iter_ms_chebyshev,
                                                           "iter_ms_learned": info.iter_ms_learned,
                                                           "damping": info.damping,
                                                           "step_reduction": info.step_reduction}}
    print(json.dumps({"workload": "curved32_k4", "train": out["train"]}), flush=True)
    for which, pre, post, label in ((0, 0, 1, "chebyshev"), (1, 0, 1, "learned"), (1, 2, 2, "learned_2_2")):
        ctx.set_smoother(which, pre, post)

        def solve():
            x.zero_()
            return ctx.solve(b, x, rtol=1e-10, maxit=300)
        with torch.cuda.stream(stream):
            ms, r = _timed(solve, steps, stream)
        out[label] = {"ms": ms, "iterations": r.iterations, "converged": bool(r.converged), "n10": r.n10,
                      "fell_back": int(r.fell_back)}
    out["learned_speedup"] = out["chebyshev"]["ms"] / out["learned"]["ms"]
    # the plain FP64 multigrid on the same problem and right-hand side
    ctx64 = Context(m, k, deform=1, precision=0, stream=stream)

    def solve64():
        x.zero_()
        return ctx64.solve(b, x, rtol=1e-10, maxit=300)
    with torch.cuda.stream(stream):
        ms, r = _timed(solve64, steps, stream)
    out["plain_fp64_mg"] = {"ms": ms, "iterations": r.iterations, "converged": bool(r.converged), "n10": r.n10}
    out["learned_speedup_vs_plain_fp64_mg"] = ms / out["learned"]["ms"]
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--which", nargs="+", default=["cube4_k3", "cube32_k4", "batch16", "rhs32", "curved32_k4"])
    ap.add_argument("--steps", type=int, default=3)
    args = ap.parse_args(argv)
    import torch
    stream = torch.cuda.Stream()
    for w in args.which:
        if w == "cube4_k3":
            r = run_single(w, 4, 3, 0, args.steps, stream)
        elif w == "cube32_k4":
            r = run_single(w, 32, 4, 0, args.steps, stream)
        elif w == "batch16":
            r = run_batch(w, sipg_inputs.batch_problems(), args.steps, stream)
        elif w == "rhs32":
            r = run_batch(w, [dict(m=16, k=4)] * 32, args.steps, stream)
        elif w == "curved32_k4":
            r = run_learned(args.steps, stream)
        else:
            raise SystemExit("unknown workload " + w)
        print(json.dumps(r), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
