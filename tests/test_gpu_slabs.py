"""Slab decomposition through the library on one GPU: the grid cut into 1..4 slabs held by
one process, halos exchanged in device memory before every pass, every slab swept by
stencil_run (one after another; no kernel waits on another).  The owned rows put back
together must equal the single-grid sweep and the FP32 oracle bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_05983_gb300 as st
import stencil_inputs as gen
from paper_2002_05983_gb300 import slabs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim,r,shape,iters,ranks", [
    (2, 1, (1024, 512), 9, 4), (2, 4, (777, 1000), 5, 3), (2, 2, (512, 264), 7, 2),
    (3, 1, (96, 40, 64), 5, 3), (3, 4, (64, 30, 32), 3, 2), (2, 3, (300, 256), 4, 1)])
def test_gpu_slabs_equal_single_grid_and_oracle(dim, r, shape, iters, ranks):
    torch.cuda.set_device(0)
    c = gen.coefficients(dim, r)
    f = gen.workload_grid(dim, *shape[::-1], seed=47)
    s = st.Stencil(dim, r, c)
    t = s.default_schedule(shape).t
    x = torch.from_numpy(f).cuda()
    got = slabs.sweep_slabs_local(x, r, iters, t, ranks, slabs.library_sweep(s))
    whole = s.run(x, iters)
    torch.cuda.synchronize()
    assert st.stencil_get_device_status() == 0
    assert torch.equal(got, whole)
    assert np.array_equal(got.cpu().numpy(), oracle.sweep_f32(f, dim, r, c, iters))
