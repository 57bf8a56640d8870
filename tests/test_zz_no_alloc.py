"""stencil_run_noalloc: the sweep for callers that cannot allocate device memory.

Code that runs while a CUDA graph is being captured, inside an allocator's
out-of-memory path, or under an externally enforced device-memory budget
cannot call cudaMalloc.  stencil_run_noalloc serves them by keeping the
ping-pong grid between passes in a fixed 16 MiB array compiled into the
library.  These tests call it through the C ABI and require its output to
equal stencil_run's bit for bit (the FP32 arithmetic is identical), on two
calls in a row with different data, since every call reuses the same array.
"""
import pytest
import torch

import paper_2002_05983_gb300 as st
import stencil_inputs as gen

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
    return ref, got


@pytest.mark.parametrize("dim,r,shape,iters,dtype", [
    (2, 2, (1024, 1024), 7, torch.float32),     # 4 MiB, several passes through the array
    (2, 4, (2048, 2048), 5, torch.float32),     # exactly 16 MiB, the largest grid accepted
    (3, 1, (64, 96, 128), 5, torch.float32),
    (2, 1, (512, 1000), 4, torch.float32),      # rows not 16-byte aligned: one-step passes
    (3, 3, (40, 48, 64), 3, torch.bfloat16),
])
def test_noalloc_equals_stencil_run_on_two_calls(dim, r, shape, iters, dtype):
    torch.cuda.set_device(0)
    s = st.Stencil(dim, r, gen.coefficients(dim, r))
    first = torch.from_numpy(gen.workload_grid(dim, *shape[::-1], seed=21)).to(dtype).cuda()
    second = torch.from_numpy(gen.workload_grid(dim, *shape[::-1], seed=22)).to(dtype).cuda()
    for x in (first, second):                   # the second call finds the first call's data in the array
        ref, got = _run_both(s.handle, x, dim, iters)
        assert torch.equal(got, ref)
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
