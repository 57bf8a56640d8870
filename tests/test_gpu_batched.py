"""Batched persistent sweeps (stencil_run_batched) against the oracle, through the C ABI.

A mixed batch (2D and 3D, radius 1..4, FP32 and BF16, different step counts)
must give every grid the oracle's result: FP32 bit for bit; BF16 bit for bit
against the FP32 oracle run pass by pass with rounding between passes, at the
temporal degree the batch uses for that grid (its default degree, passes of t
steps then a remainder pass, exactly like stencil_run)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_05983_gb300 as st
import stencil_inputs as gen
from gpu_util import oracle_passes, to_storage

pytestmark = pytest.mark.gpu

MIX = [  # dim, r, (ny, nx) or (nz, ny, nx), iters, dtype
    (2, 1, (300, 520), 10, "f32"), (2, 2, (130, 264), 9, "f32"), (2, 3, (96, 1024), 6, "bf16"),
    (2, 4, (257, 512), 8, "f32"), (2, 1, (64, 64), 7, "bf16"), (3, 1, (40, 36, 64), 6, "f32"),
    (3, 2, (17, 30, 48), 4, "bf16"), (3, 3, (24, 40, 40), 3, "f32"), (3, 4, (20, 26, 32), 2, "f32"),
    (2, 4, (70, 136), 12, "f32"), (3, 1, (9, 12, 16), 5, "f32"),
]


def batch_degree(s, shape, dim, iters, code):
    return min(s.default_schedule(shape, code).t, iters)


def make_batch(mix, seed=30):
    out = []
    for k, (dim, r, shape, iters, dt) in enumerate(mix):
        c = gen.coefficients(dim, r)
        f = gen.workload_grid(dim, *shape[::-1], seed=seed + k)
        s = st.Stencil(dim, r, c)
        x = to_storage(f, dt).cuda()
        y = torch.full_like(x, float("nan"))
        out.append(dict(dim=dim, r=r, shape=shape, iters=iters, dt=dt, c=c, f=f, s=s, x=x, y=y))
    return out


def items_of(batch):
    items = []
    for b in batch:
        shape = b["shape"]
        nx, ny, nz = (shape[1], shape[0], 1) if b["dim"] == 2 else shape[::-1]
        items.append((b["s"].handle, b["x"].data_ptr(), b["y"].data_ptr(), nx, ny, nz, b["iters"],
                      st.dtype_code(b["x"])))
    return items


def check(batch):
    for b in batch:
        got = b["y"].float().cpu().numpy()
        if b["dt"] == "f32":
            want = oracle.sweep_f32(b["f"], b["dim"], b["r"], b["c"], b["iters"])
        else:
            t = batch_degree(b["s"], b["shape"], b["dim"], b["iters"], st.STENCIL_BF16)
            want = oracle_passes(b["f"], b["dim"], b["r"], b["c"], b["iters"], t, b["dt"])
        assert np.array_equal(got, want), (b["dim"], b["r"], b["shape"], b["dt"])


def test_mixed_batch_matches_oracle_and_replays():
    torch.cuda.set_device(0)
    batch = make_batch(MIX)
    stream = torch.cuda.current_stream().cuda_stream
    assert st.stencil_get_device_status(clear=True) == 0
    st.stencil_run_batched(items_of(batch), stream)
    torch.cuda.synchronize()
    assert st.stencil_get_device_status() == 0
    check(batch)
    # second call replays the cached graph; new input data, same buffers
    for k, b in enumerate(batch):
        b["f"] = gen.workload_grid(b["dim"], *b["shape"][::-1], seed=90 + k)
        b["x"].copy_(to_storage(b["f"], b["dt"]).cuda())
        b["y"].fill_(float("nan"))
    st.stencil_run_batched(items_of(batch), stream)
    torch.cuda.synchronize()
    check(batch)


def test_batch_rejects_overlapping_outputs_and_unaligned_rows():
    torch.cuda.set_device(0)
    batch = make_batch(MIX[:2])
    items = items_of(batch)
    bad = [items[0], (items[1][0], items[1][1], items[0][2]) + items[1][3:]]   # two outputs alias
    with pytest.raises(st.StencilError) as e:
        st.stencil_run_batched(bad, torch.cuda.current_stream().cuda_stream)
    assert e.value.code == st.STENCIL_ERR_ALIAS
    s = st.Stencil(2, 1, gen.coefficients(2, 1))
    x = torch.zeros((8, 1001), device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(st.StencilError) as e:
        st.stencil_run_batched([(s.handle, x.data_ptr(), y.data_ptr(), 1001, 8, 1, 3, 0)],
                               torch.cuda.current_stream().cuda_stream)
    assert e.value.code == st.STENCIL_ERR_UNSUPPORTED


def test_batch_dependency_wait_times_out_without_hanging():
    """Pass 0 of one grid never reports completion: its next pass's bounded waits expire,
    the status records it and the context keeps working."""
    torch.cuda.set_device(0)
    mix = [(2, 1, (256, 512), 12, "f32"), (2, 1, (128, 264), 12, "f32")]   # three passes of t = 4
    batch = make_batch(mix)
    st.stencil_set_fault_injection(batch[0]["s"].handle, 0, 50)
    assert st.stencil_get_device_status(clear=True) == 0
    st.stencil_run_batched(items_of(batch), torch.cuda.current_stream().cuda_stream)
    assert st.stencil_get_device_status(clear=True) == st.STENCIL_ERR_TIMEOUT
    st.stencil_set_fault_injection(batch[0]["s"].handle, -1, 0)
    st.stencil_run_batched(items_of(batch), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st.stencil_get_device_status() == 0
    check(batch)


def test_remainder_passes_and_single_pass_grids():
    """Step counts that are not multiples of the degree get a remainder pass (its own kernel
    class, after every full pass); grids with fewer steps than the degree run one pass."""
    torch.cuda.set_device(0)
    mix = [(2, 1, (200, 512), 9, "f32"), (2, 2, (120, 256), 7, "bf16"), (2, 4, (90, 264), 5, "f32"),
           (3, 1, (30, 20, 48), 5, "bf16"), (2, 1, (64, 128), 3, "f32"), (3, 2, (16, 16, 16), 1, "f32")]
    batch = make_batch(mix, seed=60)
    st.stencil_run_batched(items_of(batch), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st.stencil_get_device_status() == 0
    check(batch)


def test_batched_workload_96_grids_matches_oracle():
    """The batched workload: 96 seeded grids (64 2D sides 512-8192, 32 3D sides 64-384, radius
    1-4, FP32 and BF16, rows rounded down to 8 cells), 100 steps each, in one call; every
    grid against the oracle."""
    torch.cuda.set_device(0)
    mix = []
    for it in gen.batch_list():
        nx = it["nx"] - it["nx"] % 8
        shape = (it["ny"], nx) if it["dim"] == 2 else (it["nz"], it["ny"], nx)
        mix.append((it["dim"], it["r"], shape, 100, it["dtype"]))
    batch = make_batch(mix, seed=100)
    st.stencil_run_batched(items_of(batch), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert st.stencil_get_device_status() == 0
    check(batch)
