"""Parity of the CUDA path with the CPU oracle, through the C ABI.

FP32: the library evaluates every cell as the same multiply-then-FMA chain as
the FP32 oracle, so results must be bit-identical for every schedule, and
within 2e-6 * iters of the FP64 oracle.  16-bit storage: bit-identical to the
FP32 oracle run pass by pass with rounding to the storage type in between.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_05983_gb300 as st
import stencil_inputs as gen
from gpu_util import (assert_bits_equal, make_input, oracle_passes, run_gpu, shape_of,
                      to_storage)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    st.library()
    yield


def test_smoke_config_2d_r1_256():
    """2D r=1, 256^2, 10 iterations, t=1: bit-exact vs fp32 oracle, <= 2e-5 vs fp64."""
    c = gen.coefficients(2, 1)
    f = gen.uniform_grid((256, 256), seed=0)
    s = st.Stencil(2, 1, c)
    want32 = oracle.sweep_f32(f, 2, 1, c, 10)
    want64 = oracle.sweep_f64(f, 2, 1, c, 10)
    for sched in ({"kernel": st.KERNEL_NAIVE}, {"kernel": st.KERNEL_STREAM, "t": 1}, {}):
        got = run_gpu(s, torch.from_numpy(f), 10, **sched)
        assert_bits_equal(got, want32, f"smoke {sched}")
        assert np.max(np.abs(got.numpy() - want64)) <= 2e-6 * 10


CASES_2D = [(r, t) for r in (1, 2, 3, 4, 5, 6) for t in sorted({1, 2, 3, st.stencil_max_t(2, r, 0)})]


@pytest.mark.parametrize("r,t", CASES_2D)
def test_2d_stream_bit_exact(r, t):
    """Several x tiles and y segments with ragged tails; iters = 2t+1 (remainder pass)."""
    nx, ny = 1000, 777
    c = gen.coefficients(2, r)
    f = make_input(2, nx, ny)
    iters = 2 * t + 1
    want = oracle.sweep_f32(f, 2, r, c, iters)
    s = st.Stencil(2, r, c)
    got = run_gpu(s, torch.from_numpy(f), iters, kernel=st.KERNEL_STREAM, t=t, seg=97)
    assert_bits_equal(got, want, f"2D r={r} t={t}")
    w64 = oracle.sweep_f64(f.astype(np.float64), 2, r, c.astype(np.float64), iters)
    assert np.max(np.abs(got.numpy() - w64)) <= 2e-6 * iters


CASES_3D = [(r, t, vy) for r in (1, 2, 3, 4, 5, 6) for vy in (2, 4)
            for t in sorted({1, st.stencil_max_t(3, r, 0, vy)})]


@pytest.mark.parametrize("r,t,vy", CASES_3D)
def test_3d_stream_bit_exact(r, t, vy):
    nx, ny, nz = 100, 70, 53
    c = gen.coefficients(3, r)
    f = make_input(3, nx, ny, nz)
    iters = 2 * t + 1
    want = oracle.sweep_f32(f, 3, r, c, iters)
    s = st.Stencil(3, r, c)
    got = run_gpu(s, torch.from_numpy(f), iters, kernel=st.KERNEL_STREAM, t=t, rows_per_thread=vy, seg=19)
    assert_bits_equal(got, want, f"3D r={r} t={t} vy={vy}")


@pytest.mark.parametrize("t", [1, 2, 3, 4])
@pytest.mark.parametrize("seg", [7, 19, 0])
def test_3d_r1_ring_phases(t, seg):
    """3D radius 1 at every degree whose input ring is not a whole number of chunks
    (t = 2: 5 slots, t = 3: 4 slots, chunks of 3 steps) and its neighbours: segments of 7
    and 19 planes start the blocks at every offset in the ring and the chunk, so each
    slot is reused in both phases of its mbarrier on several laps."""
    nx, ny, nz = 100, 70, 53
    c = gen.coefficients(3, 1)
    f = make_input(3, nx, ny, nz)
    iters = 2 * t + 1
    s = st.Stencil(3, 1, c)
    got = run_gpu(s, torch.from_numpy(f), iters, kernel=st.KERNEL_STREAM, t=t, rows_per_thread=2, seg=seg)
    assert_bits_equal(got, oracle.sweep_f32(f, 3, 1, c, iters), f"3D r=1 t={t} seg={seg}")


@pytest.mark.parametrize("dim,r", [(2, 1), (2, 4), (2, 6), (3, 1), (3, 3), (3, 5)])
def test_schedules_bit_identical_to_naive(dim, r):
    """Every FP32 schedule equals the one-thread-per-cell t=1 schedule bit for bit."""
    shape = (300, 260) if dim == 2 else (40, 36, 44)
    f = make_input(dim, *shape[::-1])
    c = gen.coefficients(dim, r)
    s = st.Stencil(dim, r, c)
    x = torch.from_numpy(f)
    iters = 7
    ref = run_gpu(s, x, iters, kernel=st.KERNEL_NAIVE)
    scheds = []
    for vy in ((1,) if dim == 2 else (2, 4)):
        for t in range(1, st.stencil_max_t(dim, r, 0, vy) + 1):
            for seg in (0, 1, 7, 61, 5000):   # 5000: one block sweeps several strips/tiles
                scheds.append(dict(kernel=st.KERNEL_STREAM, t=t, seg=seg, rows_per_thread=vy))
    for sc in scheds:
        try:
            got = run_gpu(s, x, iters, **sc)
        except st.StencilError as e:
            assert e.code == st.STENCIL_ERR_UNSUPPORTED, sc   # halo wider than the tile
            continue
        assert torch.equal(got, ref), sc


@pytest.mark.parametrize("dim,shape,r", [
    (2, (1, 4), 1), (2, (3, 8), 4), (2, (64, 4), 3), (2, (5, 1000), 2),
    (3, (1, 1, 4), 2), (3, (3, 5, 8), 4), (3, (9, 2, 12), 1), (3, (2, 40, 8), 3),
    (2, (7, 12), 6), (3, (4, 9, 16), 5)])
def test_tiny_and_degenerate_grids(dim, shape, r):
    """Sides smaller than the radius, single rows/planes: clamp everywhere."""
    f = gen.uniform_grid(shape, seed=5)
    c = gen.coefficients(dim, r)
    s = st.Stencil(dim, r, c)
    for t in sorted({1, min(2, st.stencil_max_t(dim, r, 0))}):
        want = oracle.sweep_f32(f, dim, r, c, 5)
        got = run_gpu(s, torch.from_numpy(f), 5, kernel=st.KERNEL_STREAM, t=t)
        assert_bits_equal(got, want, f"tiny {shape} t={t}")
        got = run_gpu(s, torch.from_numpy(f), 5, kernel=st.KERNEL_NAIVE)
        assert_bits_equal(got, want, f"tiny naive {shape}")


def test_unaligned_rows_use_naive_path():
    f = gen.uniform_grid((33, 1001), seed=6)
    c = gen.coefficients(2, 2)
    s = st.Stencil(2, 2, c)
    want = oracle.sweep_f32(f, 2, 2, c, 4)
    assert_bits_equal(run_gpu(s, torch.from_numpy(f), 4), want, "auto on unaligned nx")
    with pytest.raises(st.StencilError) as e:
        run_gpu(s, torch.from_numpy(f), 4, kernel=st.KERNEL_STREAM)
    assert e.value.code == st.STENCIL_ERR_UNSUPPORTED


def test_iters_zero_copies_and_input_untouched():
    f = gen.uniform_grid((40, 64), seed=7)
    s = st.Stencil(2, 1, gen.coefficients(2, 1))
    x = torch.from_numpy(f).cuda()
    keep = x.clone()
    out = s.run(x, 0)
    assert torch.equal(out, x)
    out = s.run(x, 9)
    torch.cuda.synchronize()
    assert torch.equal(x, keep)
    with pytest.raises(st.StencilError) as e:
        s.run(x, 3, out=x)
    assert e.value.code == st.STENCIL_ERR_ALIAS


@pytest.mark.parametrize("dt", ["bf16", "f16"])
@pytest.mark.parametrize("dim,r,t", [(2, 1, 1), (2, 1, 6), (2, 4, 3), (3, 2, 1), (3, 1, 3), (3, 4, 2)])
def test_low_precision_storage_bit_exact(dt, dim, r, t):
    """16-bit grids: FP32 arithmetic inside a pass, one rounding per pass."""
    shape = (190, 264) if dim == 2 else (29, 34, 40)
    f = make_input(dim, *shape[::-1])
    c = gen.coefficients(dim, r)
    iters = 2 * t + 1
    want = oracle_passes(f, dim, r, c, iters, t, dt)
    s = st.Stencil(dim, r, c)
    sched = dict(kernel=st.KERNEL_STREAM, t=t)
    if dim == 3:
        sched.update(rows_per_thread=2 if t > 1 else 4)
    got = run_gpu(s, to_storage(f, dt), iters, **sched)
    assert_bits_equal(got, want, f"{dt} {dim}D r={r} t={t}")
    # naive path = one rounding per step
    got = run_gpu(s, to_storage(f, dt), iters, kernel=st.KERNEL_NAIVE)
    assert_bits_equal(got, oracle_passes(f, dim, r, c, iters, 1, dt), f"{dt} naive")


def test_run_host_end_to_end():
    f = make_input(3, 64, 48, 40)
    c = gen.coefficients(3, 2)
    s = st.Stencil(3, 2, c)
    x = torch.from_numpy(f).pin_memory()
    out = torch.empty_like(x).pin_memory()
    s.run_host(x, out, 6)
    assert_bits_equal(out, oracle.sweep_f32(f, 3, 2, c, 6), "run_host")


@pytest.mark.parametrize("dim,shape,r,t,dt", [
    (2, (64, 128), 1, 3, "f32"),
    (2, (96, 256), 4, 2, "bf16"),    # 16-bit 2D, two rows per step: the producer rotates over the warps
    (3, (24, 40, 72), 1, 2, "f32"),  # input ring of 5 slots that wraps inside a 3-step chunk
    (3, (24, 40, 72), 1, 3, "f32"),  # 4 slots
    (3, (24, 40, 72), 4, 1, "f32"),  # shifting queue
])
def test_fault_injection_times_out_and_context_survives(dim, shape, r, t, dt):
    """A copy that is never issued makes the bounded wait expire: the kernel records
    TIMEOUT, lets its copies in flight land and returns; the same context keeps working
    afterwards."""
    f = gen.uniform_grid(shape, seed=8)
    c = gen.coefficients(dim, r)
    s = st.Stencil(dim, r, c)
    x = to_storage(f, dt).cuda() if dt != "f32" else torch.from_numpy(f).cuda()
    assert st.stencil_get_device_status(clear=True) == 0
    st.stencil_set_fault_injection(s.handle, 10, 50)
    s.run(x, t, sched=st.schedule(kernel=st.KERNEL_STREAM, t=t))
    assert st.stencil_get_device_status(clear=True) == st.STENCIL_ERR_TIMEOUT
    assert st.stencil_get_device_status() == 0
    st.stencil_set_fault_injection(s.handle, -1, 0)
    got = run_gpu(s, x.cpu(), t, kernel=st.KERNEL_STREAM, t=t)
    want = oracle.sweep_f32(f, dim, r, c, t) if dt == "f32" else oracle_passes(f, dim, r, c, t, t, dt)
    assert_bits_equal(got, want, f"after fault {dim}D r={r} t={t} {dt}")

