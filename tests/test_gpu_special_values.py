"""Special values through the streaming kernels: subnormals, signed zeros, the largest finite
values, infinities and NaN, in FP32, BF16 and FP16 storage.

Eq. 1 is a chain of IEEE multiplies and fused multiply-adds, so every finite or infinite result,
the sign of a zero and the position of every NaN are fixed by the inputs: the kernels must match
the oracle (run pass by pass with rounding to the storage type between passes for 16-bit
storage) bit for bit on every cell that is not NaN, and be NaN exactly where the oracle is.  This
pins the widening of 16-bit cells and the packing of results on the values the random-input
parity tests never produce (a BF16 cell is widened by moving its bits into the upper half of a
binary32, which must keep subnormals, -0, inf and NaN intact).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_05983_gb300 as st
import stencil_inputs as gen
from gpu_util import CODE, oracle_passes, to_storage

pytestmark = pytest.mark.gpu

SPECIAL = {   # finite values that exercise the ends of each storage type's range
    "f32": [0.0, -0.0, 1e-45, -1e-45, 3e-39, -2.5e-38, 1.2e-38, 3.0e38, -3.0e38],
    "bf16": [0.0, -0.0, 9.2e-41, -9.2e-41, 3e-39, -2.5e-38, 1.2e-38, 3.0e38, -3.0e38],
    "f16": [0.0, -0.0, 6e-8, -6e-8, 3e-6, -4e-5, 6.1e-5, 65504.0, -65504.0],
}


def _grid(dim, shape, dt, nonfinite, seed):
    rng = np.random.default_rng(seed)
    f = gen.uniform_grid(shape, seed=seed).astype(np.float32)
    flat = f.reshape(-1)
    idx = rng.choice(flat.size, size=flat.size // 6, replace=False)
    vals = SPECIAL[dt] + ([np.inf, -np.inf, np.nan] if nonfinite else [])
    flat[idx] = rng.choice(np.array(vals, np.float32), size=idx.size)
    return f


def _want(f, dim, r, c, iters, t, dt):
    if dt == "f32":
        return oracle.sweep_f32(f, dim, r, c, iters)
    return oracle_passes(f, dim, r, c, iters, t, dt)


def _assert_same(got, want, what):
    g = got.float().numpy() if got.dtype != torch.float32 else got.numpy()
    gn, wn = np.isnan(g), np.isnan(want)
    assert np.array_equal(gn, wn), f"{what}: NaN at {int((gn != wn).sum())} cells where the oracle has none or the reverse"
    gb, wb = g.view(np.uint32)[~gn], want.astype(np.float32).view(np.uint32)[~wn]
    if not np.array_equal(gb, wb):
        k = int(np.argmax(gb != wb))
        raise AssertionError(f"{what}: {int((gb != wb).sum())} cells differ, e.g. got {g[~gn][k]!r} "
                             f"want {want[~wn][k]!r}")


@pytest.mark.parametrize("dt", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("dim,shape,r", [(2, (40, 136), 1), (2, (40, 136), 4), (3, (14, 20, 72), 1),
                                         (3, (14, 20, 72), 4)])
@pytest.mark.parametrize("nonfinite", [False, True])
def test_special_values_match_the_oracle(dt, dim, shape, r, nonfinite):
    c = gen.coefficients(dim, r)
    s = st.Stencil(dim, r, c)
    f = _grid(dim, shape, dt, nonfinite, seed=31 + r)
    x = (to_storage(f, dt) if dt != "f32" else torch.from_numpy(f)).cuda()
    t_def = s.default_schedule(shape, CODE[dt]).t
    for t in sorted({1, t_def}):
        iters = 2 * t + 1
        out = s.run(x, iters, sched=st.schedule(kernel=st.KERNEL_STREAM, t=t))
        torch.cuda.synchronize()
        assert st.stencil_get_device_status() == 0
        src = to_storage(f, dt).float().numpy() if dt != "f32" else f
        _assert_same(out.cpu(), _want(src, dim, r, c, iters, t, dt),
                     f"{dt} {dim}D r={r} t={t} nonfinite={nonfinite}")
    s.close()
