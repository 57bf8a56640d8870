"""Slab decomposition of a sweep (multi-GPU path) on CPU: row-range plans, the in-process
halo exchange and the point-to-point exchange between gloo ranks (world sizes 2 and 3).
The local sweep is the FP32 oracle here, so the decomposed result must equal the oracle's
single-grid result bit for bit: only the partition and the exchange are under test."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import stencil_inputs as gen  # noqa: E402
from paper_2002_05983_gb300 import slabs  # noqa: E402


def oracle_sweep(dim, r, c):
    import oracle
    oracle.build()

    def run(block, steps):
        return torch.from_numpy(oracle.sweep_f32(block.numpy(), dim, r, c, steps))
    return run


def test_plan_covers_the_axis_and_sizes_the_halos():
    ps = slabs.plan(103, 4, 6)
    assert [p.own for p in ps] == [(0, 26), (26, 52), (52, 78), (78, 103)]
    assert [p.local for p in ps] == [(0, 32), (20, 58), (46, 84), (72, 103)]
    assert ps[0].recv_lo == (0, 0) and ps[0].recv_hi == (26, 32) and ps[0].send_lo == (0, 0)
    assert ps[1].recv_lo == (20, 26) and ps[1].send_lo == (26, 32) and ps[1].send_hi == (46, 52)
    assert ps[3].recv_hi == (103, 103) and ps[3].send_hi == (103, 103)
    # what rank k sends up is exactly what rank k+1 receives below, and vice versa
    for a, b in zip(ps, ps[1:]):
        assert a.send_hi == b.recv_lo and b.send_lo == a.recv_hi
    assert slabs.plan(10, 1, 50)[0].local == (0, 10)
    with pytest.raises(ValueError):
        slabs.plan(10, 4, 3)            # slabs of 2-3 rows are lower than the halo
    with pytest.raises(ValueError):
        slabs.plan(3, 4, 0)


def test_passes_split_the_steps():
    assert slabs.passes(7, 3) == [3, 3, 1]
    assert slabs.passes(6, 3) == [3, 3]
    assert slabs.passes(2, 5) == [2]


@pytest.mark.parametrize("dim,r,shape,iters,t,ranks", [
    (2, 1, (61, 40), 7, 3, 3), (2, 4, (96, 24), 5, 2, 4), (2, 2, (50, 33), 9, 4, 2),
    (3, 1, (30, 10, 12), 5, 2, 3), (3, 3, (40, 6, 8), 4, 2, 2), (2, 3, (17, 20), 3, 1, 1)])
def test_in_process_slabs_equal_the_single_grid_sweep(dim, r, shape, iters, t, ranks):
    import oracle
    oracle.build()
    c = gen.coefficients(dim, r)
    f = gen.workload_grid(dim, *shape[::-1], seed=41)
    got = slabs.sweep_slabs_local(torch.from_numpy(f), r, iters, t, ranks, oracle_sweep(dim, r, c))
    assert np.array_equal(got.numpy(), oracle.sweep_f32(f, dim, r, c, iters))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, case, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dim, r, shape, iters, t = case
        c = gen.coefficients(dim, r)
        f = gen.workload_grid(dim, *shape[::-1], seed=43)
        s = slabs.plan(shape[0], world, r * t)[rank]
        block = torch.from_numpy(np.ascontiguousarray(f[s.local[0]:s.local[1]]))
        own = slabs.sweep_slabs_dist(block, shape[0], r, iters, t, rank, world, dist, oracle_sweep(dim, r, c))
        parts = [None] * world
        dist.all_gather_object(parts, (rank, own.numpy()))
        q.put(np.concatenate([p for _, p in sorted(parts, key=lambda x: x[0])]) if rank == 0 else None)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,case", [(2, (2, 2, (64, 40), 7, 3)), (3, (3, 1, (36, 12, 16), 5, 2))])
def test_gloo_ranks_exchange_halos(world, case):
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(k, world, port, case, q)) for k in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = next(g for g in got if g is not None)
    dim, r, shape, iters, t = case
    f = gen.workload_grid(dim, *shape[::-1], seed=43)
    assert np.array_equal(got, oracle.sweep_f32(f, dim, r, gen.coefficients(dim, r), iters))
