"""Sanitizer substitutes on the GPU (compute-sanitizer is not available): canary-padded
output buffers must come back with their guards untouched and the input unchanged, for
ragged shapes and many schedules; and a sweep split into two calls equals one call
(a sweep is a pure function of its input, so this is the checkpoint/resume property)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_05983_gb300 as st
import stencil_inputs as gen
from gpu_util import make_input, to_storage

pytestmark = pytest.mark.gpu

GUARD = 4096          # elements of canary before and after the output
CANARY = -7.25        # exactly representable in FP32, BF16 and FP16


CASES = [  # dim, (nx, ny, nz), r, schedule fields
    (2, (1000, 77, 1), 4, dict(kernel=st.KERNEL_STREAM, t=2, seg=13)),
    (2, (1000, 77, 1), 1, dict(kernel=st.KERNEL_STREAM, t=5, seg=0)),
    (2, (516, 300, 1), 6, dict(kernel=st.KERNEL_STREAM, t=3, seg=0)),
    (2, (1001, 9, 1), 2, dict()),                                  # unaligned rows: one-step kernel
    (3, (100, 37, 23), 3, dict(kernel=st.KERNEL_STREAM, t=1, rows_per_thread=4, seg=5)),
    (3, (68, 70, 19), 1, dict(kernel=st.KERNEL_STREAM, t=2, rows_per_thread=2, seg=0)),
    (3, (36, 9, 7), 5, dict(kernel=st.KERNEL_STREAM, t=1, rows_per_thread=2, seg=3)),
]


@pytest.mark.parametrize("dt", ["f32", "bf16"])
@pytest.mark.parametrize("dim,size,r,sched", CASES)
def test_output_guards_and_input_untouched(dim, size, r, sched, dt):
    nx, ny, nz = size
    if dt != "f32" and nx % 8:
        pytest.skip("16-bit rows need 16-byte alignment for the streaming kernel")
    f = make_input(dim, nx, ny, nz)
    x = to_storage(f, dt).cuda()
    x0 = x.clone()
    n = x.numel()
    buf = torch.full((GUARD + n + GUARD,), CANARY, dtype=x.dtype, device="cuda")
    out = buf[GUARD:GUARD + n].view(x.shape)
    s = st.Stencil(dim, r, gen.coefficients(dim, r))
    s.run(x, 5, out=out, sched=st.schedule(**sched) if sched else None)
    torch.cuda.synchronize()
    assert st.stencil_get_device_status() == 0
    assert torch.all(buf[:GUARD] == CANARY) and torch.all(buf[GUARD + n:] == CANARY)
    assert torch.equal(x, x0)
    if dt == "f32":
        assert np.array_equal(out.cpu().numpy(), oracle.sweep_f32(f, dim, r, gen.coefficients(dim, r), 5))


@pytest.mark.parametrize("dim,shape,r,a,b", [(2, (300, 1024), 3, 4, 7), (2, (260, 512), 1, 10, 5),
                                            (3, (30, 40, 64), 2, 3, 2), (3, (20, 24, 32), 4, 1, 1)])
def test_split_sweep_equals_one_sweep(dim, shape, r, a, b):
    """run(a) then run(b) from its output == run(a + b), bit for bit, at every split (the FP32
    arithmetic per cell does not depend on the temporal degree of the passes)."""
    f = gen.uniform_grid(shape, seed=50)
    s = st.Stencil(dim, r, gen.coefficients(dim, r))
    x = torch.from_numpy(f).cuda()
    whole = s.run(x, a + b)
    part = s.run(s.run(x, a), b)
    torch.cuda.synchronize()
    assert torch.equal(whole, part)
