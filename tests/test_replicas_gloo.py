"""Multi-rank host logic of bench.py on CPU: two gloo ranks (world size 2).

Replicas sweep independent grids, so the only cross-rank step is the timing
reduction: the job's time is the slowest rank's, and the job's throughput is
the units of all ranks over that time.  The reference (oracle) arm runs on
rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = bench.rank_env()
        elapsed = [0.75, 1.25][rank]            # rank 1 is the slower one
        slow = bench.reduce_max(elapsed, dist, "cpu")
        units = 1000.0 * (rank + 1)             # rank-local count, only rank 0's is used below
        dist.barrier()
        q.put((r, w, lr, slow, bench.job_rate(units, w, slow)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    assert all(g[1] == 2 and g[2] == g[0] for g in got)
    assert all(g[3] == 1.25 for g in got)                 # max over ranks, on every rank
    assert got[0][4] == pytest.approx(1000.0 * 2 / 1.25)  # units x world / slowest time


def test_single_process_defaults():
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    out = subprocess.run([sys.executable, "-c", "import bench; print(bench.rank_env())"], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "(1, 0, 0)"
    assert bench.reduce_max(2.5) == 2.5
    assert bench.job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2"], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=120)
    assert out.returncode == 0
    assert out.stdout.strip() == ""


def test_gpu_local_cpus_from_topology(monkeypatch):
    """CPU affinity column of nvidia-smi's topology matrix, intersected with the allowed CPUs."""
    topo = ("\tGPU0\tGPU1\tNIC0\tCPU Affinity\tNUMA Affinity\tGPU NUMA ID\n"
            "GPU0\t X \tNV18\tSYS\t0-3,8\t0\t2\n"
            "GPU1\tNV18\t X \tSYS\t4-7\t1\t3\n")

    class Out:
        stdout = topo

    monkeypatch.setattr(bench.subprocess, "run", lambda *a, **k: Out())
    monkeypatch.setattr(bench.os, "sched_getaffinity", lambda pid: set(range(6)))
    assert bench.gpu_local_cpus(0) == {0, 1, 2, 3}
    assert bench.gpu_local_cpus(1) == {4, 5}
    assert bench.gpu_local_cpus(2) is None
    assert bench.parse_cpulist("0-2,5") == {0, 1, 2, 5} and bench.parse_cpulist("N/A") is None


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference (the oracle on the host cores) prints one JSON line with the
    base contract's keys, its own cpu_baseline and an e2e without host/device copies."""
    import json
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "GCell/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
