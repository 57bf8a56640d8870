"""stencil_run_noalloc: the sweep for callers that cannot allocate device memory.

Code inside an allocator's out-of-memory path, or a process whose device
memory is handed out by an external budget, cannot call cudaMalloc (it would
recurse, fail, or draw on memory the library was not given).
stencil_run_noalloc serves such callers by keeping the ping-pong grid between
passes in a fixed 16 MiB array compiled into the library.  These tests call it
through the C ABI and require its output to equal stencil_run's bit for bit
(the FP32 arithmetic is identical) and the oracle's, on two calls in a row with
different data, since every call reuses the same array.  An expired bounded
wait inside its kernels is reported by stencil_get_device_status.

This file is collected last so that a failure here leaves every other test run.
"""
import pytest
import torch

import oracle
import paper_2002_05983_gb300 as st
import stencil_inputs as gen
from gpu_util import assert_bits_equal, oracle_passes

pytestmark = pytest.mark.gpu

LIMIT = 16 << 20


def _run_both(h, x, dim, iters):
    nz, ny, nx = (1,) + tuple(x.shape) if dim == 2 else tuple(x.shape)
    stream = torch.cuda.current_stream().cuda_stream
    code = st.dtype_code(x)
    ref = torch.empty_like(x)
    got = torch.full_like(x, float("nan"))
    st.stencil_run(h, x.data_ptr(), ref.data_ptr(), nx, ny, nz, iters, code, stream)
    st.stencil_run_noalloc(h, x.data_ptr(), got.data_ptr(), nx, ny, nz, iters, code, stream)
    torch.cuda.synchronize()
    assert st.stencil_get_device_status() == 0
    return ref, got


@pytest.mark.parametrize("dim,r,shape,iters,dtype", [
    (2, 2, (1024, 1024), 7, torch.float32),     # 4 MiB, several passes through the array
    (2, 4, (2048, 2048), 5, torch.float32),     # exactly 16 MiB, the largest grid accepted
    (3, 1, (64, 96, 128), 5, torch.float32),
    (2, 1, (512, 1001), 4, torch.float32),      # rows not 16-byte aligned: one-step passes
    (3, 3, (40, 48, 64), 3, torch.bfloat16),
])
def test_noalloc_equals_stencil_run_on_two_calls(dim, r, shape, iters, dtype):
    torch.cuda.set_device(0)
    c = gen.coefficients(dim, r)
    s = st.Stencil(dim, r, c)
    for seed in (21, 22):                       # the second call finds the first call's data in the array
        f = gen.workload_grid(dim, *shape[::-1], seed=seed)
        x = torch.from_numpy(f).to(dtype).cuda()
        ref, got = _run_both(s.handle, x, dim, iters)
        assert torch.equal(got, ref)
        if dtype == torch.float32:
            want = oracle.sweep_f32(f, dim, r, c, iters)
        else:                                   # 16-bit storage: rounded once per pass of t steps
            t = s.default_schedule(shape, st.dtype_code(x)).t
            want = oracle_passes(f, dim, r, c, iters, min(t, iters), "bf16")
        assert_bits_equal(got.cpu(), want, f"noalloc {dim}D r={r} seed={seed}")
    s.close()


def test_noalloc_rejects_grids_beyond_the_array():
    torch.cuda.set_device(0)
    s = st.Stencil(2, 1, gen.coefficients(2, 1))
    n = LIMIT // 4 + 4                            # one row of four cells more than fits
    x = torch.zeros((n // 4, 4), device="cuda")
    out = torch.empty_like(x)
    with pytest.raises(st.StencilError) as e:
        st.stencil_run_noalloc(s.handle, x.data_ptr(), out.data_ptr(), 4, n // 4, 1, 3,
                               st.STENCIL_F32, torch.cuda.current_stream().cuda_stream)
    assert e.value.code == st.STENCIL_ERR_INVALID_ARG
    s.close()


def test_noalloc_expired_wait_is_reported():
    """A copy that is never issued (the handle's test hook) makes a bounded wait in a
    noalloc kernel expire; stencil_get_device_status reports TIMEOUT, clears it, and
    the next call is correct again."""
    torch.cuda.set_device(0)
    f = gen.uniform_grid((96, 256), seed=23)
    c = gen.coefficients(2, 2)
    s = st.Stencil(2, 2, c)
    x = torch.from_numpy(f).cuda()
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream().cuda_stream
    assert st.stencil_get_device_status(clear=True) == 0
    st.stencil_set_fault_injection(s.handle, 12, 50)
    st.stencil_run_noalloc(s.handle, x.data_ptr(), out.data_ptr(), 256, 96, 1, 6, st.STENCIL_F32, stream)
    assert st.stencil_get_device_status(clear=True) == st.STENCIL_ERR_TIMEOUT
    assert st.stencil_get_device_status() == 0
    st.stencil_set_fault_injection(s.handle, -1, 0)
    st.stencil_run_noalloc(s.handle, x.data_ptr(), out.data_ptr(), 256, 96, 1, 6, st.STENCIL_F32, stream)
    assert st.stencil_get_device_status() == 0
    assert_bits_equal(out.cpu(), oracle.sweep_f32(f, 2, 2, c, 6), "noalloc after the expired wait")
    s.close()
