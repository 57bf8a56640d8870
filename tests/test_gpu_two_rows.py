"""2D sweeps that advance two rows per step (planes_per_step = 2), against the oracle.

With two rows per step every level trails the one below by 2 + max(r, 2) rows and
its register queue spans 2r + 2 rows (2 + max(r, 2) + r, rounded up to whole steps);
a pass whose degree has no two-row kernel (a remainder pass) runs with one row per
step.  Results must equal the FP32 oracle bit for bit, like every other schedule.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_05983_gb300 as st
import stencil_inputs as gen
from gpu_util import assert_bits_equal, make_input, oracle_passes, run_gpu, to_storage

pytestmark = pytest.mark.gpu

# degrees compiled with two rows per step (FP32)
TWO_ROW = {1: (2, 3, 4, 5), 2: (2, 3, 4), 3: (2, 3), 4: (2, 3)}
CASES = [(r, t) for r, ts in TWO_ROW.items() for t in ts]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    st.library()
    yield


@pytest.mark.parametrize("r,t", CASES)
@pytest.mark.parametrize("seg", [97, 0])
def test_two_rows_bit_exact(r, t, seg):
    """Several strips and segments with ragged tails; iters = 2t+1 (remainder pass)."""
    nx, ny = 1000, 777
    c = gen.coefficients(2, r)
    f = make_input(2, nx, ny)
    iters = 2 * t + 1
    want = oracle.sweep_f32(f, 2, r, c, iters)
    s = st.Stencil(2, r, c)
    got = run_gpu(s, torch.from_numpy(f), iters, kernel=st.KERNEL_STREAM, t=t, seg=seg, planes_per_step=2)
    assert_bits_equal(got, want, f"2D r={r} t={t} seg={seg} two rows")


@pytest.mark.parametrize("r", sorted(TWO_ROW))
def test_two_rows_every_segment_parity(r):
    """Segments of 1, 2, 3, 5 and 61 rows start on odd and even rows, some shorter
    than the pipeline's lag; a segment longer than the grid sweeps several strips."""
    nx, ny = 300, 131
    c = gen.coefficients(2, r)
    f = make_input(2, nx, ny)
    s = st.Stencil(2, r, c)
    x = torch.from_numpy(f)
    for t in TWO_ROW[r]:
        iters = 3 * t
        want = oracle.sweep_f32(f, 2, r, c, iters)
        for seg in (1, 2, 3, 5, 61, 5000):
            got = run_gpu(s, x, iters, kernel=st.KERNEL_STREAM, t=t, seg=seg, planes_per_step=2)
            assert_bits_equal(got, want, f"r={r} t={t} seg={seg}")


@pytest.mark.parametrize("shape,r", [((1, 8), 1), ((2, 8), 4), ((3, 16), 2), ((5, 12), 3), ((4, 1000), 4),
                                     ((7, 40), 1)])
def test_two_rows_tiny_grids(shape, r):
    """Fewer rows than the lags and the radius: clamp at both ends of every level."""
    f = gen.uniform_grid(shape, seed=15)
    c = gen.coefficients(2, r)
    s = st.Stencil(2, r, c)
    for t in TWO_ROW[r]:
        want = oracle.sweep_f32(f, 2, r, c, 2 * t)
        got = run_gpu(s, torch.from_numpy(f), 2 * t, kernel=st.KERNEL_STREAM, t=t, planes_per_step=2)
        assert_bits_equal(got, want, f"tiny {shape} r={r} t={t}")


def test_two_rows_fault_injection_times_out():
    f = gen.uniform_grid((64, 128), seed=8)
    c = gen.coefficients(2, 2)
    s = st.Stencil(2, 2, c)
    x = torch.from_numpy(f).cuda()
    assert st.stencil_get_device_status(clear=True) == 0
    st.stencil_set_fault_injection(s.handle, 11, 50)
    s.run(x, 3, sched=st.schedule(kernel=st.KERNEL_STREAM, t=3, planes_per_step=2))
    assert st.stencil_get_device_status(clear=True) == st.STENCIL_ERR_TIMEOUT
    st.stencil_set_fault_injection(s.handle, -1, 0)
    got = run_gpu(s, x.cpu(), 3, kernel=st.KERNEL_STREAM, t=3, planes_per_step=2)
    assert_bits_equal(got, oracle.sweep_f32(f, 2, 2, c, 3), "after fault")


@pytest.mark.parametrize("dt", ["bf16", "f16"])
@pytest.mark.parametrize("r,t", [(1, 1), (1, 4), (2, 3), (3, 2), (4, 1), (4, 3)])
def test_two_rows_low_precision_storage(dt, r, t):
    """16-bit grids with two rows per step: FP32 arithmetic in a pass, one rounding per pass."""
    nx, ny = 264, 190
    f = make_input(2, nx, ny)
    c = gen.coefficients(2, r)
    iters = 2 * t + 1
    s = st.Stencil(2, r, c)
    got = run_gpu(s, to_storage(f, dt), iters, kernel=st.KERNEL_STREAM, t=t, planes_per_step=2, seg=37)
    assert_bits_equal(got, oracle_passes(f, 2, r, c, iters, t, dt), f"{dt} r={r} t={t} two rows")


def test_default_schedules_use_two_rows_for_radius_2_to_4():
    """The library's 2D rule: radius 1 at t = 4 with one row per step, radii 2-4 two rows."""
    for r, t, p in ((1, 4, 1), (2, 3, 2), (3, 2, 2), (4, 2, 2)):
        s = st.Stencil(2, r, gen.coefficients(2, r))
        d = s.default_schedule((16384, 16384))
        assert (d.t, d.planes_per_step) == (t, p), r


@pytest.mark.parametrize("dt", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_four_rows_one_level_bit_exact(dt, r):
    """t = 1 passes with four rows per step: segments of 1, 3, 6 and 97 rows (starting on
    every row residue mod 4), a ragged grid, a remainder-free multi-pass run."""
    nx, ny = 264, 203
    f = make_input(2, nx, ny)
    c = gen.coefficients(2, r)
    s = st.Stencil(2, r, c)
    x = to_storage(f, dt) if dt != "f32" else torch.from_numpy(f)
    want = oracle_passes(f, 2, r, c, 3, 1, dt) if dt != "f32" else oracle.sweep_f32(f, 2, r, c, 3)
    for seg in (1, 3, 6, 97, 0):
        got = run_gpu(s, x, 3, kernel=st.KERNEL_STREAM, t=1, seg=seg, planes_per_step=4)
        assert_bits_equal(got, want, f"{dt} r={r} seg={seg} four rows")


@pytest.mark.parametrize("shape,r", [((1, 8), 1), ((3, 16), 4), ((5, 16), 2), ((9, 8), 3)])
def test_four_rows_tiny_grids(shape, r):
    f = gen.uniform_grid(shape, seed=16)
    c = gen.coefficients(2, r)
    s = st.Stencil(2, r, c)
    got = run_gpu(s, torch.from_numpy(f), 4, kernel=st.KERNEL_STREAM, t=1, planes_per_step=4)
    assert_bits_equal(got, oracle.sweep_f32(f, 2, r, c, 4), f"tiny {shape} r={r} four rows")


def test_resolved_rows_per_step_fall_back_to_compiled_counts():
    """A pass runs with the requested rows per step where that count is compiled for its
    degree, else with the next smaller compiled count (4 -> 2 -> 1)."""
    n = 1024
    for r, t, asked, want in ((4, 1, 4, 4), (4, 2, 4, 2), (4, 2, 2, 2), (1, 7, 2, 1), (1, 3, 4, 2), (2, 6, 2, 1)):
        s = st.Stencil(2, r, gen.coefficients(2, r))
        res = st.stencil_resolve_schedule(s.handle, n, n, 1, st.STENCIL_F32,
                                          st.schedule(kernel=st.KERNEL_STREAM, t=t, planes_per_step=asked))
        assert (res.t, res.planes_per_step) == (t, want), (r, t, asked)
        feats = st.stencil_schedule_features(s.handle, n, n, 1, st.STENCIL_F32,
                                             st.schedule(kernel=st.KERNEL_STREAM, t=t, planes_per_step=asked))
        assert int(feats[14]) == want
