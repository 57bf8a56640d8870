"""Full-size configurations checked element by element against the oracle.

Each grid runs at the library's default schedule (the launch configuration the
benchmark times) for 3 full passes plus a remainder pass, and the whole output
is compared with the oracle run on the whole grid: bit for bit with the FP32
oracle for FP32 storage, and with the FP32 oracle run pass by pass (rounded to
the storage type between passes) for BF16/FP16 storage.  Sizes are the
benchmark workloads: 2D 16384^2 and 3D 512^3 FP32, radius 1..4 (Eq. 1, clamp
to edge); 3D 768^3 and 2D 32768^2 radius 4 in BF16 and FP16.
"""
import functools

import numpy as np
import pytest
import torch

import oracle
import paper_2002_05983_gb300 as st
import stencil_inputs as gen
from gpu_util import CODE, TORCH_DT, assert_bits_equal, oracle_passes, to_storage

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=2)
def grid(dim, n):
    return gen.workload_grid(dim, *(n,) * dim)


def _default_t(s, shape, dt):
    return s.default_schedule(shape, CODE[dt]).t


def _run(s, f, iters, dt):
    x = to_storage(f, dt).cuda() if dt != "f32" else torch.from_numpy(f).cuda()
    out = s.run(x, iters)
    del x
    torch.cuda.synchronize()
    assert st.stencil_get_device_status() == 0
    got = out.cpu()
    del out
    torch.cuda.empty_cache()
    return got


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_2d_16384_fp32_whole_grid(r):
    n = 16384
    f = grid(2, n)
    c = gen.coefficients(2, r)
    s = st.Stencil(2, r, c)
    iters = 3 * _default_t(s, (n, n), "f32") + 1
    got = _run(s, f, iters, "f32")
    assert_bits_equal(got, oracle.sweep_f32(f, 2, r, c, iters), f"2D 16384^2 r={r} iters={iters}")


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_3d_512_fp32_whole_grid(r):
    n = 512
    f = grid(3, n)
    c = gen.coefficients(3, r)
    s = st.Stencil(3, r, c)
    iters = 3 * _default_t(s, (n, n, n), "f32") + 1
    got = _run(s, f, iters, "f32")
    assert_bits_equal(got, oracle.sweep_f32(f, 3, r, c, iters), f"3D 512^3 r={r} iters={iters}")


@pytest.mark.parametrize("dt", ["bf16", "f16"])
@pytest.mark.parametrize("dim,n", [(3, 768), (2, 32768)])
def test_precision_configs_whole_grid(dim, n, dt):
    """The 16-bit storage configurations, radius 4: one rounding per pass of t steps."""
    r = 4
    f = grid(dim, n)
    c = gen.coefficients(dim, r)
    s = st.Stencil(dim, r, c)
    t = _default_t(s, (n,) * dim, dt)
    iters = 3 * t + 1
    got = _run(s, f, iters, dt)
    want = oracle_passes(f, dim, r, c, iters, t, dt)
    assert got.dtype == TORCH_DT[dt]
    assert_bits_equal(got, want, f"{dim}D {n} {dt} r=4 iters={iters}")
    assert np.isfinite(want).all()
