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
from paper_1910_01900_gb300.roofline import flops_alg  # noqa: E402

WORKLOAD = "curved16_k5"
METRIC = "SIPG apply DoF/s & %roofline; solve s/MDoF to 1e-10 rel. res. vs plain FP64 MG"


# Iterations of this workload's FP64 solve to 1e-10 (measured on the GB300; the
# GPU path and the oracle reach equal counts in the parity tests).  The oracle
# arm scales one timed fine-level operator apply by the number of fine-level
# applies the oracle's solve performs: ITERATIONS V-cycles (flexible CG
# preconditions once before its loop and once after every non-final
# iteration) with 2 n_s DG applies each (n_s - 1 pre-smoothing from x = 0, one
# residual, n_s post-smoothing), ITERATIONS outer applies and the initial
# residual: a lower bound of the oracle's solve time (FE levels, transfers and
# vector updates are left out).
ITERATIONS = 6
NS = 5
# DRAM bytes per DoF of the FP64 curved k=5 integration pass, from the ncu
# capture summarised in profiles/dg_kernels_curved32_k5_fp64.md (32^3 cells,
# scaled to this workload by the number of cells it processes).
INTEGRATE_DRAM_BYTES_PER_DOF = 126.1
DG_APPLIES_PER_SOLVE = ITERATIONS * 2 * NS + ITERATIONS + 1


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


def whole_job(seconds, units, world, device="cpu"):
    """Whole-job figures of N replicas: the slowest rank's time (max over ranks)
    and the units (DoF) all ranks processed (sum).  Every rank gets both."""
    if world == 1:
        return seconds, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(u.item()))


def s_per_mdof(seconds, dofs):
    return seconds * 1e6 / dofs


def run_gb300(args):
    import torch
    import torch.distributed as dist

    from paper_1910_01900_gb300 import Context, fma_peak, launch_count

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

    # the clock sampler runs from before the warm-up, so that starting it costs
    # the timed steps nothing; it covers the whole timed region
    samples, stop = [], threading.Event()
    th = threading.Thread(target=clocks_sampler, args=(stop, samples), daemon=True)
    th.start()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            info = step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    times, iters, launches = [], [], 0
    t_wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0 = launch_count()
            e0.record(stream)
            info = step()
            e1.record(stream)
            launches += launch_count() - l0
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            iters.append(info.iterations)
            assert info.converged, "solve did not converge"
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    # the same solve with the V-cycle in FP32 (outer FCG, residual, coarse solve in FP64)
    with torch.cuda.stream(stream):
        ctx32 = Context(m, k, deform=deform, precision=1, stream=stream)
        x32 = torch.zeros_like(b)
        for _ in range(args.warmup):
            x32.zero_()
            ctx32.solve(b, x32, rtol=1e-10, maxit=100)
        t32, it32 = [], []
        torch.cuda.nvtx.range_push("timed_mixed")
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            x32.zero_()
            e0.record(stream)
            info32 = ctx32.solve(b, x32, rtol=1e-10, maxit=100)
            e1.record(stream)
            e1.synchronize()
            t32.append(e0.elapsed_time(e1))
            it32.append(info32.iterations)
        torch.cuda.nvtx.range_pop()
        err32 = (torch.linalg.norm(x32 - x) / torch.linalg.norm(x)).item()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    # whole job: the slowest replica's mean step time over the DoF of all replicas
    ms = float(np.mean(times))
    job_s, job_dofs = whole_job(ms * 1e-3, N, world, dev)
    ms = job_s * 1e3
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
    e2e_s, _ = whole_job(float(np.mean(e2e_t)), N, world, dev)
    mixed_s, _ = whole_job(float(np.mean(t32)) * 1e-3, N, world, dev)
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
        "metric": METRIC, "value": s_per_mdof(job_s, job_dofs), "unit": "s/MDoF", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "curved16_k5: 16^3 curved cube (amp 0.1, Q3 mapping), k=5, %d DoF, seeded "
                               "uniform RHS, plain FP64 cph MG + Chebyshev(5,5), FCG to 1e-10" % N,
                   "l2": "flushed (256 MB write) before every timed step", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "iterations": int(np.median(iters)),
        "solve_mixed": {"value": s_per_mdof(mixed_s, job_dofs), "unit": "s/MDoF",
                        "iterations": int(np.median(it32)), "rel_diff_vs_fp64_solution": err32,
                        "speedup_vs_plain_fp64_mg": float(np.mean(times)) / float(np.mean(t32))},
        "e2e": {"value": s_per_mdof(e2e_s, job_dofs), "unit": "s/MDoF", "h2d_bytes_per_step": 8 * job_dofs,
                "d2h_bytes_per_step": 8 * job_dofs},
        "apply": {"fp64_dof_per_s": N / ((te64 + ti64) * 1e-3), "fp32_dof_per_s": N / ((te32 + ti32) * 1e-3),
                  "fp64_ms": [te64, ti64], "fp32_ms": [te32, ti32]},
        "roofline": {"kernel": "dg_integrate_kernel<double,6,curved>", "bound": "alu", "achieved": ach / 1e12,
                     "peak": peak64 / 1e12, "unit": "TFLOP/s", "frac": ach / peak64, "traffic": INTEGRATE_DRAM_BYTES_PER_DOF * N,
                     "traffic_source": "ncu dram__bytes_read+write of a 32^3 capture scaled by cells",
                     "peak_source": "measured DFMA probe in this run (sipg_fma_peak)"},
        "gpu_launches": int(launches),
        "gpu_launches_per_step": launches / max(1, args.steps),
        "clocks": clocks,
        "wall_s": wall,
    }
    if rank == 0:
        out["cpu_baseline"] = cpu_baseline(m, k, deform, N)
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def oracle_apply_time(m, k, deform, N, reps):
    from oracle.dg import SIPG
    from oracle.mesh import Mesh
    op = SIPG(Mesh(m, deform=deform), k)
    u = sipg_inputs.uniform(N, sipg_inputs.SEED_APPLY)
    op.apply(u)
    t0 = time.perf_counter()
    for _ in range(reps):
        op.apply(u)
    return (time.perf_counter() - t0) / reps


def host_cpu():
    """The host CPU as the OS names it: the model name (x86), else the Arm implementer and part
    codes (Grace: 0x41 / 0xd4f), else the machine type."""
    import platform
    import re
    try:
        info = open("/proc/cpuinfo").read()
        m = re.search(r"^model name\s*:\s*(.+)$", info, re.M)
        if m:
            return m.group(1).strip()
        imp = re.search(r"^CPU implementer\s*:\s*(\S+)", info, re.M)
        part = re.search(r"^CPU part\s*:\s*(\S+)", info, re.M)
        if imp and part:
            return "%s, implementer %s, part %s" % (platform.machine(), imp.group(1), part.group(1))
    except OSError:
        pass
    return platform.machine() or "unknown"


def cpu_baseline(m, k, deform, N, reps=2):
    """The FP64 oracle on a bounded sample: full-mesh operator applies, scaled to one solve."""
    t = oracle_apply_time(m, k, deform, N, reps)
    return {"value": t * DG_APPLIES_PER_SOLVE * 1e6 / N, "unit": "s/MDoF", "cores": os.cpu_count(),
            "cpu": host_cpu(), "kind": "oracle",
            "sample": "%d FP64 oracle applies of the full %d^3 curved k=%d operator (numpy), %.2f s each, "
                      "scaled by the %d fine-level applies of a %d-iteration solve (lower bound: FE levels, "
                      "transfers and vector updates not counted)" % (reps, m, k, t, DG_APPLIES_PER_SOLVE,
                                                                     ITERATIONS),
            "apply_dof_per_s": N / t}


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
    value = t * DG_APPLIES_PER_SOLVE * 1e6 / N
    sample = ("each step: one FP64 oracle apply of the full %d^3 curved k=%d operator (numpy), scaled by the "
              "%d fine-level applies of a %d-iteration solve (lower bound)" % (m, k, DG_APPLIES_PER_SOLVE,
                                                                              ITERATIONS))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s/MDoF", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "curved16_k5: 16^3 curved cube, k=5, %d DoF, FP64" % N},
           "cpu_baseline": {"value": value, "unit": "s/MDoF", "kind": "oracle", "cores": os.cpu_count(),
                            "cpu": host_cpu(), "sample": sample},
           "e2e": {"value": value, "unit": "s/MDoF", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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
