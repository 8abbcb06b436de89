"""Per-level timing of a multigrid hierarchy, and the V-cycle and solve it makes.

    python -m paper_1910_01900_gb300.levels [--m M] [--k K] [--curved 0|1]
                                            [--precision 0 1] [--fe-assemble 0 1 2]
                                            [--fuse-tail 0 1] [--cycles-only]

For each V-cycle precision and each `fe_assemble` setting (FE levels of degree
<= fe_assemble apply an assembled stencil, 0 = all matrix-free): the time of
one operator application on every smoothed level, of one V-cycle and of one
solve to 1e-10 with a seeded uniform right-hand side (`--fuse-tail`: with the
lower end of the cycle in one cluster launch, 1 = the default, or one launch
per step; `--cycles-only`: the V-cycles alone).  CUDA events on the
library stream around back-to-back calls (20 for applies and V-cycles, 3 for
solves) after 3 warm-up calls; a level's time includes the host cost of the
call, so levels that run in a few microseconds show that floor.  Prints one
JSON line per setting.
"""
import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import sipg_inputs  # noqa: E402  (seeded input generators)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=16)
    ap.add_argument("--k", type=int, default=5)
    ap.add_argument("--curved", type=int, default=1)
    ap.add_argument("--precision", type=int, nargs="+", default=[0, 1])
    ap.add_argument("--fe-assemble", type=int, nargs="+", default=[0, 1, 2])
    ap.add_argument("--fuse-tail", type=int, nargs="+", default=[1])
    ap.add_argument("--cycles-only", action="store_true")
    args = ap.parse_args(argv)
    import torch

    from . import Context
    s = torch.cuda.Stream()

    def timeit(fn, reps=20):
        with torch.cuda.stream(s):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                fn()
            e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps * 1e3   # microseconds

    for prec in args.precision:
        dt = torch.float64 if prec == 0 else torch.float32
        for fa, fuse in [(fa, fuse) for fa in args.fe_assemble for fuse in args.fuse_tail]:
            ctx = Context(args.m, args.k, deform=args.curved, precision=prec, stream=s, fe_assemble=fa,
                          fuse_tail=fuse)
            levels = {}
            for level in (range(1, ctx.num_levels) if not args.cycles_only else ()):
                kind, deg, mm = ctx.level_info(level)
                u = torch.as_tensor(sipg_inputs.uniform(ctx.num_dofs(level), 5)).to("cuda", dt)
                v = torch.empty_like(u)
                levels[level] = {"kind": "DG" if kind == 0 else "FE", "degree": deg, "m": list(mm),
                                 "apply_us": round(timeit(lambda: ctx.level_apply(level, u, v)), 2)}
            r = torch.as_tensor(sipg_inputs.uniform(ctx.num_dofs(), 7)).cuda()
            z = torch.empty_like(r)
            t_v = timeit(lambda: ctx.vcycle(r, z))
            if args.cycles_only:
                print(json.dumps({"m": args.m, "k": args.k, "curved": args.curved, "precision": prec,
                                  "fe_assemble": fa, "fuse_tail": fuse, "vcycle_us": round(t_v, 1)}), flush=True)
                ctx.close()
                continue
            b = torch.as_tensor(sipg_inputs.uniform(ctx.num_dofs(), sipg_inputs.SEED_RHS)).cuda()
            x = torch.zeros_like(b)
            info = {}

            def solve():
                x.zero_()
                info["it"] = ctx.solve(b, x).iterations
            t_s = timeit(solve, reps=3)
            print(json.dumps({"m": args.m, "k": args.k, "curved": args.curved, "precision": prec,
                              "fe_assemble": fa, "fuse_tail": fuse, "levels": levels, "vcycle_us": round(t_v, 1),
                              "solve_ms": round(t_s / 1e3, 3), "iterations": info["it"]}), flush=True)
            ctx.close()


if __name__ == "__main__":
    main()
