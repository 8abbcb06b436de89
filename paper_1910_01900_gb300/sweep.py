"""Operator-apply throughput sweep (DoF/s and roofline fraction per degree).

    python -m paper_1910_01900_gb300.sweep [--k 1 2 ...] [--curved 0 1] [--precision 0 1]
                                           [--m M] [--repeats R]

Default meshes hold about 16 MDoF for k = 1..8 (m = 126, 84, 63, 50, 42, 36,
32, 28 cells per direction), vectors far larger than L2.  Times come from CUDA
events around each of the two DG passes (library stream), averaged over R
launches after 3 warm-up launches.  Prints one JSON line per case.
"""
import argparse
import json
import os
import sys

SWEEP_M = {1: 126, 2: 84, 3: 63, 4: 50, 5: 42, 6: 36, 7: 32, 8: 28}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--k", type=int, nargs="+", default=list(range(1, 9)))
    ap.add_argument("--curved", type=int, nargs="+", default=[1, 0])
    ap.add_argument("--precision", type=int, nargs="+", default=[0, 1])
    ap.add_argument("--m", type=int, default=0)
    ap.add_argument("--repeats", type=int, default=20)
    args = ap.parse_args(argv)
    import torch

    from . import Context, fma_peak
    from .roofline import bytes_alg, flops_alg
    peaks = {0: fma_peak(0), 1: fma_peak(1)}
    hbm = None
    p = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    if os.path.exists(p):
        hbm = json.load(open(p)).get("hbm_gbs")
    for curved in args.curved:
        for k in args.k:
            m = args.m or SWEEP_M[k]
            ctx = Context(m, k, deform=curved, operator_only=True)
            N = ctx.num_dofs()
            for prec in args.precision:
                dt = torch.float64 if prec == 0 else torch.float32
                g = torch.Generator(device="cuda").manual_seed(1910)
                u = torch.rand(N, dtype=dt, device="cuda", generator=g) * 2 - 1
                v = torch.empty_like(u)
                ctx.time_apply(u, v, 3)
                te, ti = ctx.time_apply(u, v, args.repeats)
                fe, fi = flops_alg(k, bool(curved))
                t = (te + ti) * 1e-3
                ach = (fe + fi) * N / t
                rec = {"k": k, "m": m, "curved": curved, "precision": "f64" if prec == 0 else "f32", "dofs": N,
                       "ms_eval": te, "ms_integrate": ti, "dof_per_s": N / t,
                       "flops_per_dof": fe + fi, "tflops": ach / 1e12, "alu_peak_tflops": peaks[prec] / 1e12,
                       "alu_frac": ach / peaks[prec]}
                if hbm:
                    gbs = bytes_alg(k, bool(curved), 8 if prec == 0 else 4) * N / t / 1e9
                    rec.update({"alg_gbs": gbs, "hbm_frac": gbs / hbm})
                print(json.dumps(rec), flush=True)
            ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
