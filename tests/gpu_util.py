"""Shared helpers of the GPU tests: seeded inputs, oracle references, comparisons."""
import numpy as np
import torch

import oracle
import paper_2002_05983_gb300 as st
import stencil_inputs as gen

TORCH_DT = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}
CODE = {"f32": st.STENCIL_F32, "bf16": st.STENCIL_BF16, "f16": st.STENCIL_F16}


def shape_of(dim, nx, ny, nz=1):
    return (ny, nx) if dim == 2 else (nz, ny, nx)


def make_input(dim, nx, ny, nz=1, seed=0):
    return gen.workload_grid(dim, nx, ny, nz, seed=seed)


def to_storage(a: np.ndarray, dt: str) -> torch.Tensor:
    """fp32 array -> CPU tensor of the storage type (round to nearest even)."""
    return torch.from_numpy(np.ascontiguousarray(a)).to(TORCH_DT[dt])


def run_gpu(stencil, x: torch.Tensor, iters, **sched):
    xd = x.cuda()
    out = stencil.run(xd, iters, sched=st.schedule(**sched) if sched else None)
    torch.cuda.synchronize()
    assert st.stencil_get_device_status() == 0
    return out.cpu()


def oracle_passes(a32: np.ndarray, dim, r, c, iters, t, dt):
    """Reference for 16-bit storage: fp32 oracle for each pass of t steps, the grid
    rounded to the storage type between passes (input rounded first)."""
    cur = to_storage(a32, dt).float().numpy()
    done = 0
    while done < iters:
        k = min(t, iters - done)
        cur = oracle.sweep_f32(cur, dim, r, c, k)
        cur = to_storage(cur, dt).float().numpy()
        done += k
    return cur


def assert_bits_equal(got: torch.Tensor, want: np.ndarray, what=""):
    g = got.float().numpy() if got.dtype != torch.float32 else got.numpy()
    if not np.array_equal(g, want):
        bad = np.argwhere(g != want)
        i = tuple(bad[0])
        raise AssertionError(f"{what}: {len(bad)} cells differ, first at {i}: got {g[i]!r} want {want[i]!r}")
