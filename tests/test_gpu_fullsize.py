"""Full-size configurations, in the launch configuration bench.py times (library default
schedules), checked on sampled outputs.

After n steps a cell depends only on the input within r*n cells of it (per axis, clamped
at the grid's border), so the oracle run on that window -- cut from the same input, with
the grid's own border where the window reaches it -- gives the sampled cell exactly.
Samples: the corners, points next to every edge, points straddling strip/tile and block
boundaries, and seeded random interior points."""
import functools

import numpy as np
import pytest
import torch

import oracle
import paper_2002_05983_gb300 as st
import stencil_inputs as gen
from gpu_util import to_storage

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=2)
def grid(dim, n):
    f = gen.workload_grid(dim, *(n,) * dim)
    return f


def samples(shape, h, extra, seed):
    """Sample coordinates (tuples in array order) for a grid of `shape`."""
    rng = np.random.default_rng(seed)
    pts = set()
    for corner in np.ndindex(*(2,) * len(shape)):
        pts.add(tuple((n - 1) * c for n, c in zip(shape, corner)))
    for axis, n in enumerate(shape):
        for v in (1, 3, n - 2, n // 2):
            p = [m // 3 for m in shape]
            p[axis] = v
            pts.add(tuple(p))
    for v in extra:                    # x positions at tile / block boundaries
        p = [m // 2 for m in shape]
        p[-1] = min(max(v, 0), shape[-1] - 1)
        pts.add(tuple(p))
    for _ in range(12):
        pts.add(tuple(int(rng.integers(0, n)) for n in shape))
    return sorted(pts)


def window_value(f, dim, r, c, iters, p, passes=None, dt=None):
    h = r * iters
    lo = [max(0, v - h) for v in p]
    hi = [min(n, v + h + 1) for n, v in zip(f.shape, p)]
    win = np.ascontiguousarray(f[tuple(slice(a, b) for a, b in zip(lo, hi))])
    if passes is None:
        out = oracle.sweep_f32(win, dim, r, c, iters)
    else:   # 16-bit storage: FP32 passes of the schedule's degrees, rounded in between
        out = to_storage(win, dt).float().numpy()
        for k in passes:
            out = to_storage(oracle.sweep_f32(out, dim, r, c, k), dt).float().numpy()
    return out[tuple(v - a for v, a in zip(p, lo))]


def pass_degrees(iters, t):
    return [t] * (iters // t) + ([iters % t] if iters % t else [])


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_2d_16384_samples_bit_exact(r):
    n, iters = 16384, 20
    f = grid(2, n)
    c = gen.coefficients(2, r)
    s = st.Stencil(2, r, c)
    got = s.run(torch.from_numpy(f).cuda(), iters).cpu().numpy()
    assert st.stencil_get_device_status() == 0
    cx = 512 - 2 * (-(-(s.default_schedule((n, n)).t - 1) * r // 4) * 4)   # compute width of a strip
    extra = [k * cx + d for k in (1, 2, 17, 32) for d in (-1, 0, 1)]
    for p in samples(f.shape, r * iters, extra, seed=r):
        assert got[p] == window_value(f, 2, r, c, iters, p), (r, p)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_3d_512_samples_bit_exact(r):
    n, iters = 512, 8
    f = grid(3, n)
    c = gen.coefficients(3, r)
    s = st.Stencil(3, r, c)
    got = s.run(torch.from_numpy(f).cuda(), iters).cpu().numpy()
    assert st.stencil_get_device_status() == 0
    extra = [k * 64 + d for k in (1, 4) for d in (-1, 0)]
    for p in samples(f.shape, r * iters, extra, seed=10 + r):
        assert got[p] == window_value(f, 3, r, c, iters, p), (r, p)


def test_2d_32768_bf16_samples_bit_exact():
    n, r, iters, dt = 32768, 4, 10, "bf16"
    f = grid(2, n)
    c = gen.coefficients(2, r)
    s = st.Stencil(2, r, c)
    x = to_storage(f, dt).cuda()
    t = s.default_schedule((n, n), st.STENCIL_BF16).t
    got = s.run(x, iters).float().cpu().numpy()
    del x
    torch.cuda.empty_cache()
    assert st.stencil_get_device_status() == 0
    for p in samples(f.shape, r * iters, [496, 497, 16 * 496], seed=30):
        assert got[p] == window_value(f, 2, r, c, iters, p, pass_degrees(iters, t), dt), p
