"""Tile geometry of the streaming kernel, compiled on the host from the header the kernels use.

Pins the layout decisions that set how many blocks an SM holds and where TMA boxes start:
  * 3D radius 1 FP32: an input ring of 5 slots at t = 2 (43.0 KB, 5 blocks per SM instead of
    the 4 that a 6-slot ring of whole 3-step chunks allows) and 4 slots at t = 3, slot index
    wrapping inside a chunk;
  * every compiled shape keeps tile origins, the input box origin and its width on 16-byte
    boundaries, with the x halo in whole 4-cell vectors (16-bit storage too);
  * the rows-per-step ring geometry (lags, queue depth, chunk length) of the 2D kernels.
Shared memory per SM: 228 KB, 1 KB of it reserved per resident block.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CFG = os.path.join(ROOT, "paper_2002_05983_gb300", "csrc", "sweep_cfg.h")

# (D, R, T, VY, ES, TX, TY, P): the benchmark defaults and the shapes whose geometry changed
SHAPES = [(3, 1, 1, 2, 4, 16, 8, 1), (3, 1, 2, 2, 4, 16, 8, 1), (3, 1, 3, 2, 4, 16, 8, 1),
          (3, 1, 2, 2, 2, 16, 8, 1), (3, 2, 1, 2, 4, 16, 8, 1), (3, 3, 1, 4, 4, 16, 8, 1),
          (3, 4, 1, 4, 4, 16, 8, 1), (3, 4, 1, 2, 2, 16, 8, 1), (3, 2, 2, 2, 2, 16, 8, 1),
          (3, 2, 2, 2, 4, 16, 8, 1),
          (2, 1, 4, 1, 4, 128, 1, 1), (2, 2, 3, 1, 4, 128, 1, 2), (2, 3, 2, 1, 4, 128, 1, 2),
          (2, 4, 2, 1, 4, 128, 1, 2), (2, 4, 2, 1, 2, 128, 1, 2), (2, 4, 1, 1, 2, 128, 1, 4),
          (2, 5, 2, 1, 2, 128, 1, 1), (2, 6, 3, 1, 4, 128, 1, 1)]
FIELDS = ["BX", "BY", "CX", "CY", "HTX", "PADIN", "PWIN", "PH", "QP", "U", "ROT", "KS", "DS", "WRAP", "PFS",
          "SMEM", "OK", "ALIGN", "L1", "GAP"]


@pytest.fixture(scope="module")
def geo(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("geo")
    lines = ["#define __host__", "#define __device__", f'#include "{CFG}"', "#include <cstdio>",
             "using namespace stn;", "template <class G> void show() {",
             '  std::printf("' + " ".join(["%lld"] * len(FIELDS)) + '\\n", ' +
             ", ".join(f"(long long)G::{f}" for f in FIELDS) + ");", "}", "int main() {"]
    lines += [f"  show<Geo<{', '.join(map(str, s))}>>();" for s in SHAPES]
    lines += ["  return 0;", "}"]
    src = d / "geo.cpp"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "geo"
    subprocess.run([cxx, "-std=c++17", "-O0", str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    return {s: dict(zip(FIELDS, map(int, ln.split()))) for s, ln in zip(SHAPES, out)}


def blocks_by_smem(smem):
    return (228 * 1024) // (smem + 1024)


def test_every_shape_is_valid_and_aligned(geo):
    for s, g in geo.items():
        es = s[4]
        assert g["OK"] == 1, s
        assert g["HTX"] % 4 == 0 and g["CX"] % g["ALIGN"] == 0, s        # whole vectors, 16-byte tile origins
        assert (g["HTX"] + g["PADIN"]) % g["ALIGN"] == 0, s               # 16-byte input box origin
        assert (g["PWIN"] * es) % 16 == 0 and g["PADIN"] >= 4 * ((s[1] + 3) // 4), s
        assert g["U"] <= g["DS"] and (g["WRAP"] == 1) == (g["DS"] % g["U"] != 0), s
        assert g["HTX"] == -(-((s[2] - 1) * s[1]) // 4) * 4, s             # r (t - 1) rounded up to 4 cells
        assert g["L1"] == max(s[1], s[7]) and g["GAP"] == s[7] + g["L1"], s


def test_3d_radius1_ring_keeps_blocks_resident(geo):
    t2 = geo[(3, 1, 2, 2, 4, 16, 8, 1)]
    assert (t2["DS"], t2["PFS"], t2["WRAP"], t2["SMEM"]) == (5, 3, 1, 43008)
    assert blocks_by_smem(t2["SMEM"]) == 5
    assert blocks_by_smem(t2["SMEM"] + 1 * 5248) == 4           # one more slot (a 6-slot ring): 4 blocks
    t3 = geo[(3, 1, 3, 2, 4, 16, 8, 1)]
    assert (t3["DS"], t3["WRAP"], t3["SMEM"]) == (4, 1, 53504) and blocks_by_smem(t3["SMEM"]) == 4
    t1 = geo[(3, 1, 1, 2, 4, 16, 8, 1)]
    assert (t1["DS"], t1["WRAP"]) == (6, 0)                     # one level: 4 steps ahead, whole chunks
    h = geo[(3, 1, 2, 2, 2, 16, 8, 1)]
    assert (h["DS"], h["WRAP"]) == (6, 0)                       # 16-bit rings are small enough


def test_16bit_tiles_compute_as_wide_as_fp32(geo):
    for a, b in (((3, 1, 2, 2, 4, 16, 8, 1), (3, 1, 2, 2, 2, 16, 8, 1)),
                 ((3, 2, 2, 2, 4, 16, 8, 1), (3, 2, 2, 2, 2, 16, 8, 1)),
                 ((2, 4, 2, 1, 4, 128, 1, 2), (2, 4, 2, 1, 2, 128, 1, 2))):
        assert geo[a]["CX"] == geo[b]["CX"], (a, b)
    assert geo[(2, 4, 2, 1, 2, 128, 1, 2)]["CX"] == 504          # 512 - 2 * 4
    assert geo[(3, 1, 2, 2, 2, 16, 8, 1)]["CX"] == 56


def test_rows_per_step_geometry(geo):
    g = geo[(2, 4, 2, 1, 4, 128, 1, 2)]                           # the headline radius-4 kernel
    assert (g["L1"], g["GAP"], g["QP"], g["U"], g["ROT"]) == (4, 6, 10, 5, 1)
    g = geo[(2, 4, 1, 1, 2, 128, 1, 4)]
    assert (g["L1"], g["GAP"], g["QP"], g["U"]) == (4, 8, 12, 3)
    g = geo[(2, 1, 4, 1, 4, 128, 1, 1)]
    assert (g["QP"], g["U"], g["ROT"]) == (3, 3, 1)
