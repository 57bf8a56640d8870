"""Domain decomposition of a sweep over several GPUs: slabs along the streaming axis.

The grid is cut into slabs of whole rows (2D: y) or planes (3D: z), one per
rank.  A pass of t steps needs, around a slab, the r*t rows the stencil's
dependency cone reaches (Eq. 1 applied t times): every rank holds its slab
plus up to H = r*t halo rows on each side that are not at the grid's border,
receives those halo rows from its neighbours before every pass (point-to-point
send/recv of the slab faces, the only exchange of the method), and sweeps the
whole local block with the library (stencil_run, t steps).  Values next to a
cut are computed with the clamp of the local block, which is wrong there, but
a wrong value spreads by r rows per step, so after t steps it has reached only
the halo: the owned rows are exact, bit for bit equal to the single-grid sweep
(the arithmetic of every cell is the same).  At the grid's own border the
local block ends where the grid does, so the clamp is the real one.

A rank's slab must be at least H rows high (halos come from the adjacent slab
only).  The exchange goes through ``torch.distributed`` (NCCL between GPUs,
gloo on CPU); ``exchange_local`` does the same copies between slabs held by one
process (several slabs swept one after another on one device).

This module computes row ranges and moves rows; every cell update runs in the
library's kernels (or, in CPU tests, in the function the caller passes).
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Slab:
    """Row ranges of one rank, in global stream-axis indices (half-open)."""
    own: tuple       # rows this rank owns and returns
    local: tuple     # rows of its local block: own plus the halos inside the grid
    recv_lo: tuple   # halo rows below the slab (received from rank - 1), may be empty
    recv_hi: tuple   # halo rows above the slab (received from rank + 1), may be empty
    send_lo: tuple   # own rows sent to rank - 1 (its upper halo)
    send_hi: tuple   # own rows sent to rank + 1 (its lower halo)


def plan(n: int, ranks: int, halo: int):
    """Slabs of an axis of n rows over `ranks` ranks with halos of `halo` rows.

    Rows are split as evenly as possible (the first n % ranks slabs one row
    higher).  Raises ValueError when a slab is lower than the halo."""
    if ranks < 1 or n < ranks:
        raise ValueError(f"cannot cut {n} rows into {ranks} slabs")
    if halo < 0:
        raise ValueError("halo must be >= 0")
    base, extra = divmod(n, ranks)
    bounds = [0]
    for k in range(ranks):
        bounds.append(bounds[-1] + base + (1 if k < extra else 0))
    out = []
    for k in range(ranks):
        a, b = bounds[k], bounds[k + 1]
        if ranks > 1 and b - a < halo:
            raise ValueError(f"slab {k} has {b - a} rows, fewer than the halo of {halo}")
        lo, hi = max(0, a - halo), min(n, b + halo)
        out.append(Slab(own=(a, b), local=(lo, hi), recv_lo=(lo, a), recv_hi=(b, hi),
                        send_lo=(a, min(b, a + halo)) if k > 0 else (a, a),
                        send_hi=(max(a, b - halo), b) if k < ranks - 1 else (b, b)))
    return out


def _rows(block, slab: Slab, rows: tuple):
    """View of global rows [rows) inside the local block (stream axis first)."""
    o = slab.local[0]
    return block[rows[0] - o:rows[1] - o]


def exchange_local(blocks, slabs):
    """Fill every block's halo rows from the adjacent slabs' owned rows (one process)."""
    for k, s in enumerate(slabs):
        if k > 0 and s.recv_lo[1] > s.recv_lo[0]:
            _rows(blocks[k], s, s.recv_lo).copy_(_rows(blocks[k - 1], slabs[k - 1], s.recv_lo))
        if k < len(slabs) - 1 and s.recv_hi[1] > s.recv_hi[0]:
            _rows(blocks[k], s, s.recv_hi).copy_(_rows(blocks[k + 1], slabs[k + 1], s.recv_hi))


def exchange_dist(block, slabs, rank: int, dist, group=None):
    """Point-to-point halo exchange of this rank's block with ranks rank-1 and rank+1."""
    s = slabs[rank]
    if not block.is_contiguous():
        raise ValueError("the local block must be contiguous (rows of the stream axis are then contiguous)")
    ops = []
    if rank > 0:
        ops += [dist.P2POp(dist.isend, _rows(block, s, s.send_lo), rank - 1, group),
                dist.P2POp(dist.irecv, _rows(block, s, s.recv_lo), rank - 1, group)]
    if rank < len(slabs) - 1:
        ops += [dist.P2POp(dist.isend, _rows(block, s, s.send_hi), rank + 1, group),
                dist.P2POp(dist.irecv, _rows(block, s, s.recv_hi), rank + 1, group)]
    if ops:
        for w in dist.batch_isend_irecv(ops):
            w.wait()


def passes(iters: int, t: int):
    """Degrees of the passes of a sweep: t, t, ..., then iters mod t."""
    t = max(1, min(t, iters)) if iters > 0 else 1
    return [t] * (iters // t) + ([iters % t] if iters % t else [])


def sweep_slabs_local(grid, radius: int, iters: int, t: int, ranks: int, sweep):
    """Sweep `grid` (stream axis first: (ny, nx) or (nz, ny, nx)) cut into `ranks` slabs held
    by one process: per pass, exchange the halos, then call sweep(block, steps) -> new block
    on every slab.  Returns the owned rows put back together (a new tensor)."""
    import torch
    n = grid.shape[0]
    slabs = plan(n, ranks, radius * t)
    blocks = [grid[s.local[0]:s.local[1]].clone() for s in slabs]
    for steps in passes(iters, t):
        exchange_local(blocks, slabs)
        blocks = [sweep(b, steps) for b in blocks]
    return torch.cat([_rows(b, s, s.own) for b, s in zip(blocks, slabs)], dim=0)


def sweep_slabs_dist(block, n: int, radius: int, iters: int, t: int, rank: int, world: int, dist, sweep,
                     group=None):
    """This rank's part of a distributed sweep: `block` holds rows slabs[rank].local of the
    grid on entry; returns this rank's owned rows after `iters` steps."""
    slabs = plan(n, world, radius * t)
    for steps in passes(iters, t):
        exchange_dist(block, slabs, rank, dist, group)
        block = sweep(block, steps)
    return _rows(block, slabs[rank], slabs[rank].own)


def library_sweep(stencil):
    """sweep(block, steps) through the library for a Stencil bound to CUDA tensors."""
    def run(block, steps):
        return stencil.run(block.contiguous(), steps)
    return run
