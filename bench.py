"""Benchmark: SIPG solve to 1e-10 and operator apply on one GB300.

Workload (one "step" = one pass of the whole hot path): the 16^3 curved cube
(x_i += 0.1 prod_j sin(pi x_j), degree-3 mapping), degree k = 5 (884,736 DoF),
seeded uniform[-1,1] right-hand side, plain FP64 cph multigrid (DG5 -> FE5 ->
FE2 -> FE1 -> FE1 8^3 -> FE1 4^3 dense coarse solve), Chebyshev(5,5),
flexible CG to a relative residual of 1e-10.  Setup is excluded (Section 3.1).

value = solve time per MDoF (s/MDoF, lower is better), from CUDA events on the
library stream, inputs resident in HBM, L2 flushed (256 MB write) before
every timed step.  e2e = the same solve through sipg_solve_host (host b in,
host x out, copies inside the timed region).

Also reported: the FP64 and FP32 operator-apply throughput of the same
operator, the roofline of the dominant kernel against the measured FP64 FMA
peak, and the oracle's CPU time on a bounded sample.

--impl reference times the FP64 CPU oracle (the only reference that exists:
the paper ships no code) on a bounded sample of the same workload.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import sipg_inputs  # noqa: E402

WORKLOAD = "curved16_k5"
METRIC = "SIPG apply DoF/s & %roofline; solve s/MDoF to 1e-10 rel. res. vs plain FP64 MG"


def flops_alg(k, curved):
    """Algorithmic FLOPs per DoF of one operator apply (even-odd 1D kernels).

    One 1D sweep over n^2 lines costs n^2 (2(ceil(n/2)^2 + floor(n/2)^2) + 2n);
    a cell does 12 sweeps.  Each interior face, per side and per direction
    (forward and backward) costs one normal-derivative pass n^2 * 2n plus 4 face
    sweeps of n (2(ceil^2+floor^2)) + 2n^2 each; about 3 faces per cell, both
    sides counted.  Pointwise: 6 flops per cell point (Cartesian) or 18
    (curved), 12 per face point per side; curved faces add 2 tangential
    derivative sweeps per side and direction.  Returns (eval, integrate) parts.
    """
    n = k + 1
    h, hc = n // 2, (n + 1) // 2
    line = 2 * (hc * hc + h * h) + 2 * n
    sweep = n * n * line
    face_sweep = n * line
    n3 = n ** 3
    per_side = n * n * 2 * n + 4 * face_sweep + (2 * face_sweep if curved else 0)
    cell_half = 6 * sweep
    face_half = 3 * 2 * per_side           # 3 faces per cell, both sides, one direction
    point = (18 if curved else 6) * n3 + 3 * 2 * 12 * n * n
    ev = (cell_half + face_half) / n3
    it = (cell_half + face_half + point) / n3
    return ev, it


def clocks_sampler(stop, out):
    cmd = ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-i", "0"]
    while not stop.is_set():
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=5)
            out.append(r.stdout.strip().splitlines()[0])
        except Exception:
            pass
        stop.wait(0.2)


def summarize_clocks(samples):
    if not samples:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for s in samples:
        f = [x.strip() for x in s.split(",")]
        try:
            sm.append(float(f[0]))
            mx = float(f[1])
        except (ValueError, IndexError):
            continue
        for nm, v in zip(names, f[3:7]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def run_gb300(args):
    import torch
    import torch.distributed as dist

    from paper_1910_01900_gb300 import Context, fma_peak

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    cfg = sipg_inputs.WORKLOADS[WORKLOAD]
    m, k, deform = cfg["m"], cfg["k"], cfg["deform"]
    with torch.cuda.stream(stream):
        ctx = Context(m, k, deform=deform, precision=0, stream=stream)
        N = ctx.num_dofs()
        b = torch.as_tensor(sipg_inputs.uniform(N, sipg_inputs.SEED_RHS + rank)).to(dev)
        x = torch.zeros_like(b)
        flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    def step():
        x.zero_()
        return ctx.solve(b, x, rtol=1e-10, maxit=100)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            info = step()
    torch.cuda.synchronize()
    samples, stop = [], threading.Event()
    th = threading.Thread(target=clocks_sampler, args=(stop, samples), daemon=True)
    th.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    times, iters = [], []
    t_wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            iters.append(info.iterations)
            assert info.converged, "solve did not converge"
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    ms = float(np.mean(times))
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    # end-to-end: host b in, host x out, through the public C ABI
    bh = b.cpu().numpy().copy()
    xh = np.zeros_like(bh)
    ctx.solve_host(bh, xh)
    e2e_t = []
    for _ in range(max(1, min(args.steps, 5))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.solve_host(bh, xh)
        e2e_t.append(time.perf_counter() - t0)
    e2e_s = float(np.mean(e2e_t))
    # operator apply throughput and per-kernel times (FP64 and FP32)
    u64 = torch.as_tensor(sipg_inputs.uniform(N, sipg_inputs.SEED_APPLY)).to(dev)
    v64 = torch.empty_like(u64)
    u32, v32 = u64.float(), torch.empty(N, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        ctx.time_apply(u64, v64, 3)
        te64, ti64 = ctx.time_apply(u64, v64, 20)
        ctx.time_apply(u32, v32, 3)
        te32, ti32 = ctx.time_apply(u32, v32, 20)
    stop.set()
    th.join(timeout=2)
    clocks = summarize_clocks(samples)
    peak64 = fma_peak(0)
    fe, fi = flops_alg(k, bool(deform))
    # dominant kernel in the FP64 solve: the DG integration pass (face fluxes +
    # transposed sweeps); its algorithmic work per launch is fi * N
    ach = fi * N / (ti64 * 1e-3)
    out = {
        "metric": METRIC, "value": ms * 1e-3 * 1e6 / N, "unit": "s/MDoF", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "curved16_k5: 16^3 curved cube (amp 0.1, Q3 mapping), k=5, %d DoF, seeded "
                               "uniform RHS, plain FP64 cph MG + Chebyshev(5,5), FCG to 1e-10" % N,
                   "l2": "flushed (256 MB write) before every timed step", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "iterations": int(np.median(iters)),
        "e2e": {"value": e2e_s * 1e6 / N, "unit": "s/MDoF", "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N},
        "apply": {"fp64_dof_per_s": N / ((te64 + ti64) * 1e-3), "fp32_dof_per_s": N / ((te32 + ti32) * 1e-3),
                  "fp64_ms": [te64, ti64], "fp32_ms": [te32, ti32]},
        "roofline": {"kernel": "dg_integrate_kernel<double,6,curved>", "bound": "alu", "achieved": ach / 1e12,
                     "peak": peak64 / 1e12, "unit": "TFLOP/s", "frac": ach / peak64, "traffic": None,
                     "peak_source": "measured DFMA probe in this run (sipg_fma_peak)"},
        "gpu_launches": None,
        "clocks": clocks,
        "wall_s": wall,
    }
    if rank == 0:
        out["cpu_baseline"] = cpu_baseline(m, k, deform, N)
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(m, k, deform, N, reps=2):
    """The FP64 oracle's matrix-free operator apply on the full workload mesh."""
    from oracle.dg import SIPG
    from oracle.mesh import Mesh
    op = SIPG(Mesh(m, deform=deform), k)
    u = sipg_inputs.uniform(N, sipg_inputs.SEED_APPLY)
    op.apply(u)
    t0 = time.perf_counter()
    for _ in range(reps):
        op.apply(u)
    t = (time.perf_counter() - t0) / reps
    return {"value": N / t, "unit": "DoF/s (operator apply)", "cores": os.cpu_count(), "kind": "oracle",
            "sample": "%d FP64 oracle applies of the full %d^3 curved k=%d operator (numpy, dense reference "
                      "tables)" % (reps, m, k)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cfg = sipg_inputs.WORKLOADS[WORKLOAD]
    m, k, deform = cfg["m"], cfg["k"], cfg["deform"]
    from oracle.dg import SIPG
    from oracle.mesh import Mesh
    op = SIPG(Mesh(m, deform=deform), k)
    N = op.n_dofs
    u = sipg_inputs.uniform(N, sipg_inputs.SEED_APPLY)
    for _ in range(args.warmup):
        op.apply(u)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        op.apply(u)
        ts.append(time.perf_counter() - t0)
    t = float(np.mean(ts))
    out = {"impl": "reference", "metric": METRIC, "value": None, "unit": "s/MDoF", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": False,
           "dtype": "f64", "data": "synthetic", "config": {"workload": WORKLOAD},
           "apply_dof_per_s": N / t,
           "cpu_baseline": {"value": None, "unit": "s/MDoF", "kind": "oracle", "cores": os.cpu_count(),
                            "sample": "one oracle operator apply per step"},
           "e2e": {"value": None, "unit": "s/MDoF", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
