"""Shared-coefficient stencils (one coefficient per distance) on the GPU, through the C ABI.

The FP32 path sums the 2*dim neighbours at each distance left to right and
applies one FMA per distance, exactly as the FP32 shared oracle does, so every
schedule must match it bit for bit; 16-bit storage runs the one-step kernel
and must match the FP32 oracle step by step with rounding in between."""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_05983_gb300 as st
import stencil_inputs as gen
from gpu_util import assert_bits_equal, make_input, run_gpu, to_storage

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("r,t", [(1, 1), (1, 3), (1, 5), (2, 1), (2, 3), (3, 2), (4, 1), (4, 2)])
def test_shared_2d_stream_bit_exact(r, t):
    nx, ny = 1000, 777
    c = gen.shared_coefficients(2, r)
    f = make_input(2, nx, ny)
    iters = 2 * t + 1
    s = st.Stencil(2, r, c, shared=True)
    want = oracle.sweep_shared_f32(f, 2, r, c, iters)
    for seg in (0, 97):
        got = run_gpu(s, torch.from_numpy(f), iters, kernel=st.KERNEL_STREAM, t=t, seg=seg)
        assert_bits_equal(got, want, f"shared 2D r={r} t={t} seg={seg}")
    w64 = oracle.sweep_shared_f64(f.astype(np.float64), 2, r, c.astype(np.float64), iters)
    assert np.max(np.abs(got.numpy() - w64)) <= 2e-6 * iters


@pytest.mark.parametrize("r,t", [(1, 1), (1, 2), (2, 1), (3, 1), (4, 1)])
def test_shared_3d_stream_bit_exact(r, t):
    nx, ny, nz = 100, 70, 53
    c = gen.shared_coefficients(3, r)
    f = make_input(3, nx, ny, nz)
    iters = 2 * t + 1
    s = st.Stencil(3, r, c, shared=True)
    got = run_gpu(s, torch.from_numpy(f), iters, kernel=st.KERNEL_STREAM, t=t, seg=19)
    assert_bits_equal(got, oracle.sweep_shared_f32(f, 3, r, c, iters), f"shared 3D r={r} t={t}")


@pytest.mark.parametrize("dim,shape,r", [(2, (300, 260), 3), (3, (40, 36, 44), 2), (2, (7, 12), 6), (3, (4, 9, 16), 5)])
def test_shared_naive_and_default_schedules(dim, shape, r):
    """The one-step kernel (also radius 5, 6, which have no shared streaming kernel) and the
    library's default schedule equal the oracle bit for bit."""
    c = gen.shared_coefficients(dim, r)
    f = gen.uniform_grid(shape, seed=21)
    s = st.Stencil(dim, r, c, shared=True)
    want = oracle.sweep_shared_f32(f, dim, r, c, 6)
    assert_bits_equal(run_gpu(s, torch.from_numpy(f), 6, kernel=st.KERNEL_NAIVE), want, "shared naive")
    assert_bits_equal(run_gpu(s, torch.from_numpy(f), 6), want, "shared default")


@pytest.mark.parametrize("dt", ["bf16", "f16"])
def test_shared_16bit_storage_step_by_step(dt):
    dim, r, iters = 2, 2, 4
    c = gen.shared_coefficients(dim, r)
    f = gen.uniform_grid((64, 96), seed=22)
    s = st.Stencil(dim, r, c, shared=True)
    got = run_gpu(s, to_storage(f, dt), iters).float().numpy()
    cur = to_storage(f, dt).float().numpy()
    for _ in range(iters):
        cur = to_storage(oracle.sweep_shared_f32(cur, dim, r, c, 1), dt).float().numpy()
    assert np.array_equal(got, cur)


def test_shared_and_full_handles_batch_together():
    """A batch mixing shared and full handles of the same radius keeps them apart."""
    f = make_input(2, 256, 130)
    cs, cf = gen.shared_coefficients(2, 2), gen.coefficients(2, 2)
    hs, hf = st.Stencil(2, 2, cs, shared=True), st.Stencil(2, 2, cf)
    xs, xf = torch.from_numpy(f).cuda(), torch.from_numpy(f).cuda()
    ys, yf = torch.empty_like(xs), torch.empty_like(xf)
    items = [(hs.handle, xs.data_ptr(), ys.data_ptr(), 256, 130, 1, 6, 0),
             (hf.handle, xf.data_ptr(), yf.data_ptr(), 256, 130, 1, 6, 0)]
    st.stencil_run_batched(items, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st.stencil_get_device_status() == 0
    assert np.array_equal(ys.cpu().numpy(), oracle.sweep_shared_f32(f, 2, 2, cs, 6))
    assert np.array_equal(yf.cpu().numpy(), oracle.sweep_f32(f, 2, 2, cf, 6))
