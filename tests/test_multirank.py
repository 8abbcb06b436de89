"""The N > 1 path of bench.py on the CPU: world_size 2 over gloo.

The path does not shard a single problem: `bench.py --gpus N` runs N independent
replicas (one problem per rank, no data-path collective).  What the ranks share
is the timing contract: the whole job takes as long as the slowest replica and
processes the DoF of all replicas, so value = max time / summed MDoF.  The
reference arm runs on rank 0 only; the other ranks exit at once.
"""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    seconds = 0.010 + 0.005 * rank          # rank 1 is the slow replica
    dofs = 1000 + rank                       # replicas may differ in size
    t, n = bench.whole_job(seconds, dofs, world)
    q.put((rank, t, n, bench.s_per_mdof(t, n)))
    dist.destroy_process_group()


def test_whole_job_is_max_time_over_summed_dofs():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, t, n, v in res:
        assert t == pytest.approx(0.015) and n == 2001
        assert v == pytest.approx(0.015 * 1e6 / 2001)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(0.02, 500, 1) == (0.02, 500)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_host_cpu_is_named():
    sys.path.insert(0, ROOT)
    import bench
    name = bench.host_cpu()
    assert isinstance(name, str) and name and name != "unknown"
