"""Bounds-checked kernels (memory-checker substitute; compute-sanitizer is not available).

With stencil_set_checked the streaming sweeps use instantiations that test every
shared-memory access, global store and TMA copy against its buffer.  Ragged shapes
that exercise edge tiles, clamp frames, short and long segments, both block orders and
both register-queue forms must run with no access reported and match the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_05983_gb300 as st
import stencil_inputs as gen
from gpu_util import make_input, oracle_passes, to_storage

pytestmark = pytest.mark.gpu

CASES = [  # dim, r, t, rows, dtype, shapes (ny, nx) / (nz, ny, nx)
    (2, 1, 1, 1, "f32", [(37, 1000), (5, 4)]),
    (2, 1, 5, 1, "f32", [(777, 1000), (16, 516)]),
    (2, 4, 2, 1, "f32", [(301, 1000), (3, 8)]),
    (2, 6, 2, 1, "f32", [(90, 1036), (7, 12)]),
    (2, 2, 3, 1, "bf16", [(65, 1032), (9, 16)]),
    (3, 1, 2, 2, "f32", [(23, 37, 100), (3, 5, 8)]),
    (3, 3, 1, 4, "f32", [(19, 70, 68), (2, 40, 8)]),
    (3, 5, 1, 2, "f32", [(11, 21, 36), (4, 9, 16)]),
    (3, 2, 1, 2, "f16", [(13, 30, 48)]),
]


@pytest.mark.parametrize("dim,r,t,rows,dt,shapes", CASES)
def test_checked_kernels_report_no_access_out_of_range(dim, r, t, rows, dt, shapes):
    c = gen.coefficients(dim, r)
    s = st.Stencil(dim, r, c)
    st.stencil_set_checked(s.handle, True)
    assert st.stencil_get_device_status(clear=True) == 0
    iters = 2 * t   # whole passes: only these degrees are compiled checked
    for shape in shapes:
        f = make_input(dim, *shape[::-1])
        x = to_storage(f, dt).cuda()
        for seg in (0, 3, 41):
            out = s.run(x, iters, sched=st.schedule(kernel=st.KERNEL_STREAM, t=t, rows_per_thread=rows, seg=seg))
            torch.cuda.synchronize()
            assert st.stencil_get_device_status(clear=True) == 0, (shape, seg)
            got = out.float().cpu().numpy()
            want = (oracle.sweep_f32(f, dim, r, c, iters) if dt == "f32"
                    else oracle_passes(f, dim, r, c, iters, t, dt))
            assert np.array_equal(got, want), (shape, seg)
    # a schedule without a checked instantiation is refused, not run unchecked
    with pytest.raises(st.StencilError) as e:
        s.run(x, 3, sched=st.schedule(kernel=st.KERNEL_STREAM, t=3 if t != 3 else 1, rows_per_thread=rows))
    assert e.value.code == st.STENCIL_ERR_UNSUPPORTED
    st.stencil_set_checked(s.handle, False)
