"""Benchmark: SIPG solve to 1e-10 and operator apply on one GB300.

Workload (one "step" = one pass of the whole hot path): the 32^3 Cartesian
unit cube, degree k = 4 (4,096,000 DoF), manufactured right-hand side
(u = prod sin(pi x_j), f = 3 pi^2 u, homogeneous Dirichlet), plain FP64 cph
multigrid (DG4 -> FE4 -> FE2 -> FE1 -> FE1 16^3 -> 8^3 -> 4^3 dense coarse
solve), Chebyshev(5,5), flexible CG to a relative residual of 1e-10.  Setup is
excluded (Section 3.1).

value = solve time per MDoF (s/MDoF, lower is better), from CUDA events on the
library stream, inputs resident in HBM, L2 flushed (256 MB write) before
every timed step.  e2e = the same solve through sipg_solve_host (host b in,
host x out, copies inside the timed region).  solve_mixed = the same solve with
the V-cycle in FP32 (outer FCG, residual and coarse solve in FP64).

Also reported: the operator-apply throughput at the 16 MDoF point of the
degree sweep (42^3 curved cells, k = 5), FP64 and FP32; the roofline of the
solve's dominant kernel; the 16^3 curved k = 5 solve (884,736 DoF) as an
extra; and the FP64 CPU oracle timed on a bounded sample of the workload.

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
from paper_1910_01900_gb300.roofline import bytes_alg, flops_alg  # noqa: E402

WORKLOAD = "cube32_k4"
EXTRA = "curved16_k5"
APPLY_K = 5          # apply throughput: the degree-5 point of the ~16 MDoF sweep, curved cells
METRIC = "SIPG apply DoF/s & %roofline; solve s/MDoF to 1e-10 rel. res. vs plain FP64 MG"

# DRAM bytes per launch of the solve's dominant kernel, per DoF: ncu
# dram__bytes_read.sum + dram__bytes_write.sum of dg_integrate_kernel<double,5,
# Cartesian> on this workload's mesh (111,714,048 + 13,050,368 bytes over
# 4,096,000 DoF in one captured launch; the command is in traffic_source).
DOMINANT_DRAM_BYTES_PER_DOF = (111714048 + 13050368) / 4096000
DOMINANT_NCU_COMMAND = ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                        "--clock-control none -k regex:dg_integrate -s 4 -c 1 python -m "
                        "paper_1910_01900_gb300.sweep --k 4 --curved 0 --precision 0 --m 32 --repeats 2 "
                        "(dram bytes of one launch on the workload's 32^3 k=4 mesh)")

# The oracle's bounded samples: the workload's degree and geometry on a cube
# with fewer cells per axis (one oracle V-cycle on the full 32^3 mesh takes
# minutes).  Both samples keep the DG and FE_k levels matrix-free, as they
# are at full size.
CPU_SAMPLE_M = 16        # cpu_baseline of the GPU arm: 1/8 of the workload's cells
REF_SAMPLE_M = 8         # each step of the reference arm: 1/64 of its cells
ORACLE_ASSEMBLE_LIMIT = 5e6


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


def timed_solves(ctx, b, x, steps, warmup, stream, flush, launch_count=None):
    """warmup untimed then `steps` timed solves of ctx from x = 0 (CUDA events on the
    library stream, L2 flushed before each); returns (ms list, iterations list, launches, info)."""
    import torch
    info = None
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            x.zero_()
            info = ctx.solve(b, x, rtol=1e-10, maxit=100)
    torch.cuda.synchronize()
    times, iters, launches = [], [], 0
    with torch.cuda.stream(stream):
        for _ in range(steps):
            flush.fill_(1.0)
            x.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            l0 = launch_count() if launch_count else 0
            e0.record(stream)
            info = ctx.solve(b, x, rtol=1e-10, maxit=100)
            e1.record(stream)
            if launch_count:
                launches += launch_count() - l0
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            iters.append(info.iterations)
            assert info.converged, "solve did not converge"
    torch.cuda.synchronize()
    return times, iters, launches, info


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
        b = torch.empty(N, dtype=torch.float64, device=dev)
        ctx.rhs(b)                      # manufactured right-hand side
        x = torch.zeros_like(b)
        flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    # the clock sampler runs from before the warm-up, so that starting it costs
    # the timed steps nothing; it covers every timed region
    samples, stop = [], threading.Event()
    th = threading.Thread(target=clocks_sampler, args=(stop, samples), daemon=True)
    th.start()
    if world > 1:
        dist.barrier()
    t_wall0 = time.perf_counter()
    times, iters, launches, _ = timed_solves(ctx, b, x, args.steps, args.warmup, stream, flush, launch_count)
    wall = time.perf_counter() - t_wall0
    l2_fp64 = ctx.l2_error(x)
    # the same solve with the V-cycle in FP32 (outer FCG, residual, coarse solve in FP64)
    with torch.cuda.stream(stream):
        ctx32 = Context(m, k, deform=deform, precision=1, stream=stream)
    x32 = torch.zeros_like(b)
    t32, it32, _, _ = timed_solves(ctx32, b, x32, args.steps, args.warmup, stream, flush)
    with torch.cuda.stream(stream):
        err32 = (torch.linalg.norm(x32 - x) / torch.linalg.norm(x)).item()
        l2_mixed = ctx32.l2_error(x32)
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
    # per-pass times of the workload's own DG operator (the solve's dominant kernel)
    u64 = torch.as_tensor(sipg_inputs.uniform(N, sipg_inputs.SEED_APPLY)).to(dev)
    v64 = torch.empty_like(u64)
    with torch.cuda.stream(stream):
        ctx.time_apply(u64, v64, 3)
        te_w, ti_w = ctx.time_apply(u64, v64, 20)
    del u64, v64
    ctx32.close()
    # the extra workload: 16^3 curved k = 5 solves, FP64 and mixed
    ecfg = sipg_inputs.WORKLOADS[EXTRA]
    with torch.cuda.stream(stream):
        cx = Context(ecfg["m"], ecfg["k"], deform=ecfg["deform"], precision=0, stream=stream)
        cx32 = Context(ecfg["m"], ecfg["k"], deform=ecfg["deform"], precision=1, stream=stream)
        Ne = cx.num_dofs()
        be = torch.as_tensor(sipg_inputs.uniform(Ne, sipg_inputs.SEED_RHS + rank)).to(dev)
        xe, xe32 = torch.zeros_like(be), torch.zeros_like(be)
    te, ite, _, _ = timed_solves(cx, be, xe, args.steps, args.warmup, stream, flush)
    te32, ite32, _, _ = timed_solves(cx32, be, xe32, args.steps, args.warmup, stream, flush)
    cx.close()
    cx32.close()
    # operator apply at the 16 MDoF point of the degree sweep (curved, k = 5)
    ma = sipg_inputs.SWEEP_M[APPLY_K]
    with torch.cuda.stream(stream):
        ca = Context(ma, APPLY_K, deform=1, operator_only=True, stream=stream)
        Na = ca.num_dofs()
        ua = torch.as_tensor(sipg_inputs.uniform(Na, sipg_inputs.SEED_APPLY)).to(dev)
        va = torch.empty_like(ua)
        ca.time_apply(ua, va, 3)
        ta_e64, ta_i64 = ca.time_apply(ua, va, 20)
        ua32, va32 = ua.float(), torch.empty(Na, dtype=torch.float32, device=dev)
        ca.time_apply(ua32, va32, 3)
        ta_e32, ta_i32 = ca.time_apply(ua32, va32, 20)
    torch.cuda.synchronize()
    ca.close()
    stop.set()
    th.join(timeout=2)
    clocks = summarize_clocks(samples)
    peak64 = fma_peak(0)
    hbm = measured_peaks().get("hbm_gbs")
    fe_w, fi_w = flops_alg(k, bool(deform))
    # dominant kernel of the FP64 solve: the DG integration pass (face fluxes +
    # transposed sweeps) of the finest level; its algorithmic work per launch is fi_w * N
    ach = fi_w * N / (ti_w * 1e-3)
    fa_e, fa_i = flops_alg(APPLY_K, True)
    apply64 = Na / ((ta_e64 + ta_i64) * 1e-3)
    apply32 = Na / ((ta_e32 + ta_i32) * 1e-3)
    out = {
        "metric": METRIC, "value": s_per_mdof(job_s, job_dofs), "unit": "s/MDoF", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "cube32_k4: 32^3 Cartesian unit cube, k=4, %d DoF, manufactured RHS "
                               "(sin product), plain FP64 cph MG + Chebyshev(5,5), FCG to 1e-10" % N,
                   "l2": "flushed (256 MB write) before every timed step", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "iterations": int(np.median(iters)),
        "l2_error_vs_exact": l2_fp64,
        "solve_mixed": {"value": s_per_mdof(mixed_s, job_dofs), "unit": "s/MDoF", "ms": float(np.mean(t32)),
                        "iterations": int(np.median(it32)), "rel_diff_vs_fp64_solution": err32,
                        "l2_error_vs_exact": l2_mixed,
                        "speedup_vs_plain_fp64_mg": float(np.mean(times)) / float(np.mean(t32))},
        "e2e": {"value": s_per_mdof(e2e_s, job_dofs), "unit": "s/MDoF", "h2d_bytes_per_step": 8 * job_dofs,
                "d2h_bytes_per_step": 8 * job_dofs},
        "apply": {"workload": "%d^3 curved cells (amp 0.1, Q3 mapping), k=%d, %d DoF, seeded uniform u"
                              % (ma, APPLY_K, Na),
                  "fp64_dof_per_s": apply64, "fp32_dof_per_s": apply32,
                  "fp64_ms": [ta_e64, ta_i64], "fp32_ms": [ta_e32, ta_i32],
                  "fp64_alu_frac": (fa_e + fa_i) * apply64 / peak64,
                  "fp32_hbm_frac_paper_bytes": (bytes_alg(APPLY_K, True, 4) * apply32 / (hbm * 1e9)) if hbm else None,
                  "fp64_ops_per_dof": fa_e + fa_i, "fp32_paper_bytes_per_dof": bytes_alg(APPLY_K, True, 4)},
        "extra_solve": {"workload": "curved16_k5: 16^3 curved cube (amp 0.1, Q3 mapping), k=5, %d DoF, seeded "
                                    "uniform RHS" % Ne,
                        "fp64": {"value": s_per_mdof(float(np.mean(te)) * 1e-3, Ne), "unit": "s/MDoF",
                                 "ms": float(np.mean(te)), "iterations": int(np.median(ite))},
                        "mixed": {"value": s_per_mdof(float(np.mean(te32)) * 1e-3, Ne), "unit": "s/MDoF",
                                  "ms": float(np.mean(te32)), "iterations": int(np.median(ite32))}},
        "roofline": {"kernel": "dg_integrate_kernel<double,5,Cartesian> (finest level of the workload)",
                     "bound": "alu", "achieved": ach / 1e12, "peak": peak64 / 1e12, "unit": "TFLOP/s",
                     "frac": ach / peak64,
                     "traffic": DOMINANT_DRAM_BYTES_PER_DOF * N if DOMINANT_DRAM_BYTES_PER_DOF else None,
                     "traffic_source": DOMINANT_NCU_COMMAND,
                     "ms_per_launch": ti_w, "eval_pass_ms_per_launch": te_w,
                     "ops_per_dof": fi_w,
                     "peak_source": "FP64 FMA rate measured in this run (sipg_fma_peak, all SMs); "
                                    "152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz = 1.259 TFLOP/s by unit count"},
        "gpu_launches": int(launches),
        "gpu_launches_per_step": launches / max(1, args.steps),
        "clocks": clocks,
        "wall_s": wall,
    }
    if rank == 0:
        out["cpu_baseline"] = cpu_baseline(k, int(np.median(iters)))
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


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


class CpuClock:
    """Wall time and the process's CPU time over a region: CPU / wall = the cores it kept
    busy on average (numpy's and scipy's own threads included)."""

    def __enter__(self):
        self.t, self.c = time.perf_counter(), os.times()
        return self

    def __exit__(self, *exc):
        c = os.times()
        self.wall = time.perf_counter() - self.t
        self.cpu = (c.user - self.c.user) + (c.system - self.c.system)
        self.cores = self.cpu / max(self.wall, 1e-9)


def oracle_sample(m, k, estimate=False):
    """The oracle's cph hierarchy on the m^3 Cartesian cube at degree k.  Without
    ``estimate`` every level gets a fixed Chebyshev bound instead of the eigenvalue
    estimate (setup work that changes no operation count of a V-cycle)."""
    from oracle.mesh import Mesh
    from oracle.multigrid import CPHMultigrid
    return CPHMultigrid(Mesh(m), k, lambdas=None if estimate else [2.0] * 16, assemble_limit=ORACLE_ASSEMBLE_LIMIT)


def oracle_iteration(mg, r):
    """One outer iteration of the oracle's flexible CG: one V-cycle and one fine-level apply."""
    with CpuClock() as c:
        z = mg.vcycle(r)
        mg.levels[-1].apply(z)
    return c


def cpu_baseline(k, iterations):
    """The FP64 oracle on a bounded sample: one full V-cycle (every level, transfer and the
    coarse solve) plus one fine-level apply on the workload's cube at 1/8 of its cells,
    per MDoF, times the iterations the GPU solve took; and one complete oracle solve of
    the 4^3 k = 3 cube (the oracle's own flexible CG to 1e-10)."""
    from oracle.mesh import Mesh
    from oracle.multigrid import CPHMultigrid, fcg
    mg = oracle_sample(CPU_SAMPLE_M, k)
    n = mg.levels[-1].n
    c = oracle_iteration(mg, sipg_inputs.uniform(n, sipg_inputs.SEED_RHS))
    per_mdof = c.wall * 1e6 / n
    small = CPHMultigrid(Mesh(4), 3)
    bo = small.levels[-1].space.rhs(lambda p: 3 * np.pi ** 2 * np.prod(np.sin(np.pi * p), axis=-1))
    with CpuClock() as cs:
        _, it_small, _ = fcg(small.levels[-1].apply, bo, np.zeros_like(bo), small.vcycle, rtol=1e-10)
    return {"value": per_mdof * iterations, "unit": "s/MDoF", "cores": round(c.cores, 2),
            "cores_available": os.cpu_count(), "cpu": host_cpu(), "kind": "oracle",
            "sample": "one FP64 oracle V-cycle (all %d levels, transfers, dense coarse solve) plus one fine-level "
                      "apply on the %d^3 Cartesian k=%d cube (%d DoF, 1/8 of the workload's cells), %.2f s, "
                      "per MDoF times the %d iterations of the GPU solve; cores = process CPU time / wall "
                      "time of the sample" % (len(mg.levels), CPU_SAMPLE_M, k, n, c.wall, iterations),
            "small_solve": {"workload": "cube4_k3: 4^3 Cartesian, k=3, 4096 DoF, manufactured RHS",
                            "seconds": cs.wall, "iterations": it_small, "s_per_mdof": cs.wall * 1e6 / 4096,
                            "cores": round(cs.cores, 2)}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle.multigrid import fcg
    k = sipg_inputs.WORKLOADS[WORKLOAD]["k"]
    mg = oracle_sample(REF_SAMPLE_M, k, estimate=True)
    n = mg.levels[-1].n
    # the oracle's own iteration count: one complete (untimed) solve of the sample with
    # the workload's manufactured right-hand side
    fine = mg.levels[-1]
    bo = fine.space.rhs(lambda p: 3 * np.pi ** 2 * np.prod(np.sin(np.pi * p), axis=-1))
    _, iterations, _ = fcg(fine.apply, bo, np.zeros_like(bo), mg.vcycle, rtol=1e-10)
    r = sipg_inputs.uniform(n, sipg_inputs.SEED_RHS)
    for _ in range(args.warmup):
        oracle_iteration(mg, r)
    ts, cores = [], []
    for _ in range(args.steps):
        c = oracle_iteration(mg, r)
        ts.append(c.wall)
        cores.append(c.cores)
    t = float(np.mean(ts))
    value = t * 1e6 / n * iterations
    sample = ("each step: one FP64 oracle V-cycle (all %d levels, transfers, dense coarse solve) plus one "
              "fine-level apply on the %d^3 Cartesian k=%d cube (%d DoF, 1/64 of the workload's cells); value = "
              "mean step time per MDoF times the %d iterations of the oracle's own solve of the sample to 1e-10 "
              "(manufactured right-hand side)"
              % (len(mg.levels), REF_SAMPLE_M, k, n, iterations))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s/MDoF", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "cube32_k4: 32^3 Cartesian unit cube, k=4, 4096000 DoF, FP64 (sampled)"},
           "cpu_baseline": {"value": value, "unit": "s/MDoF", "kind": "oracle", "cores": round(float(np.mean(cores)), 2),
                            "cores_available": os.cpu_count(), "cpu": host_cpu(), "sample": sample},
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
