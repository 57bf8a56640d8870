"""Work, traffic and roofline arithmetic for star-stencil sweeps (host logic).

Definitions follow Section IV of the paper:
  * FLOP per cell update (Table I, Section IV.A): 4*D*r + 1, i.e. 8r+1 in 2D
    and 12r+1 in 3D -- 2*D*r + 1 multiplies and 2*D*r adds, no coefficient
    shared.
  * Bytes per cell update with full spatial reuse (Table I): one read and
    one write of the stored element, 2*s (8 for FP32).  With temporal
    blocking of degree t the grid crosses memory once per t updates: 2*s/t.
  * GCell/s (Eq. 3, printed upside down in the paper; the run times quoted in
    Section IV.C fix the orientation): cells * iterations / time / 1e9.
    GFLOP/s and GB/s are GCell/s times the per-cell FLOP and byte counts;
    redundant (halo) work is not counted.
  * Compute-block size (Eq. 2): csize = bsize - 2 * par_time * rad.
  * Roofline ratio (Tables IV/V): achieved GB/s over the device's memory
    bandwidth.
The roofline used for GB300 is R(t) = min(P_fp32 / F, BW * t / (2 s)) cells/s.
"""
from __future__ import annotations

# GB300: 152 SMs, 128 FP32 lanes per SM, an FMA counts 2 FLOP, 2070 MHz max SM clock.
GB300_SMS = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
FP32_PEAK_NOMINAL = GB300_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6  # FLOP/s


def num_coeffs(dim: int, radius: int) -> int:
    return 2 * dim * radius + 1


def flop_per_cell(dim: int, radius: int) -> int:
    return 4 * dim * radius + 1


def fp32_instr_per_cell(dim: int, radius: int) -> int:
    """Issue slots of arithmetic per cell update: one FMUL plus 2*D*r FFMA."""
    return 2 * dim * radius + 1


def bytes_per_cell(elem_bytes: int = 4, t: int = 1) -> float:
    return 2.0 * elem_bytes / t


def gcells(cells: int, iters: int, seconds: float) -> float:
    return cells * iters / seconds / 1e9


def gflops(gcell_s: float, dim: int, radius: int) -> float:
    return gcell_s * flop_per_cell(dim, radius)


def gbs(gcell_s: float, elem_bytes: int = 4) -> float:
    return gcell_s * bytes_per_cell(elem_bytes)


def csize(bsize: int, par_time: int, radius: int) -> int:
    return bsize - 2 * par_time * radius


def roofline_ratio(gcell_s: float, peak_gbs: float, elem_bytes: int = 4) -> float:
    return gbs(gcell_s, elem_bytes) / peak_gbs


def roofline_cells(dim: int, radius: int, t: int, elem_bytes: int, peak_flops: float,
                   peak_bw: float) -> float:
    """R(t) in cells/s: the lower of the FP32 and the HBM roof at temporal degree t."""
    return min(peak_flops / flop_per_cell(dim, radius), peak_bw * t / (2.0 * elem_bytes))


def roofline_bound(dim: int, radius: int, t: int, elem_bytes: int, peak_flops: float,
                   peak_bw: float) -> str:
    hbm = peak_bw * t / (2.0 * elem_bytes)
    alu = peak_flops / flop_per_cell(dim, radius)
    return "hbm" if hbm <= alu else "alu"


def model_accuracy(measured: float, estimated: float) -> float:
    return measured / estimated
