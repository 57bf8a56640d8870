"""Host logic pinned to the paper's printed numbers (Tables I, III, IV, V; Eqs. 2, 3)
and the seeded input generators pinned to SplitMix64's published definition."""
import csv
import os

import numpy as np
import pytest

import stencil_inputs as gen
from paper_2002_05983_gb300 import metrics as M

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as fh:
        lines = [ln for ln in fh if not ln.startswith("#")]
    return list(csv.DictReader(lines)) if lines[0][0].isalpha() else list(csv.reader(lines))


def test_table_i_flop_and_bytes():
    for row in _rows("table_i.csv"):
        d, r = int(row["dim"]), int(row["radius"])
        assert M.flop_per_cell(d, r) == int(row["flop_per_cell"])
        assert M.bytes_per_cell(4) == float(row["byte_per_cell"])
        assert M.flop_per_cell(d, r) / M.bytes_per_cell(4) == pytest.approx(float(row["flop_per_byte"]))
        # one multiply + 2Dr FMAs (Section V.A: 4r+1 / 6r+1 DSPs per cell update)
        assert M.fp32_instr_per_cell(d, r) == (4 * r + 1 if d == 2 else 6 * r + 1)


def test_table_iii_eq2_and_metric_identities():
    for row in _rows("table_iii.csv"):
        d, r, t = int(row["dim"]), int(row["radius"]), int(row["par_time"])
        cx = M.csize(int(row["bsize_x"]), t, r)
        assert int(row["nx"]) % cx == 0                      # input is a multiple of csize (Sec. IV.C)
        if d == 3:
            cy = M.csize(int(row["bsize_y"]), t, r)
            assert int(row["ny"]) % cy == 0
        gc = float(row["gcells"])
        # GCell/s is printed to 3 decimals, so the identities hold to 0.0005 * factor
        assert M.gflops(gc, d, r) == pytest.approx(float(row["gflops"]),
                                                   abs=5e-4 * M.flop_per_cell(d, r) + 1e-3)
        assert M.gbs(gc, 4) == pytest.approx(float(row["gbs"]), abs=5e-4 * 8 + 1e-3)
        acc = 100 * M.model_accuracy(float(row["gbs"]), float(row["est_gbs"]))
        assert acc == pytest.approx(float(row["accuracy_pct"]), abs=0.06)
        # Eq. 3 orientation: 1000 iterations take >= 3 s (2D) / >= 11 s (3D) (Section IV.C)
        cells = int(row["nx"]) * int(row["ny"]) * int(row["nz"])
        seconds = cells * 1000 / (gc * 1e9)
        assert seconds >= (3.0 if d == 2 else 11.0) - 0.1
        assert M.gcells(cells, 1000, seconds) == pytest.approx(gc)


def test_roofline_ratio_tables_iv_v():
    for dev, peak, d, r, gc, ratio in _rows("roofline_ratio.csv"):
        assert M.roofline_ratio(float(gc), float(peak)) == pytest.approx(float(ratio), abs=6e-3)


def test_gb300_roofline_shape():
    bw, p = 6792e9, M.FP32_PEAK_NOMINAL
    assert p == pytest.approx(80.55e12, rel=1e-3)
    # t = 1 is HBM-bound for every radius; large t is FP32-bound
    for d in (2, 3):
        for r in (1, 2, 3, 4):
            assert M.roofline_bound(d, r, 1, 4, p, bw) == "hbm"
            assert M.roofline_bound(d, r, 64, 4, p, bw) == "alu"
            assert M.roofline_cells(d, r, 1, 4, p, bw) == pytest.approx(bw / 8)
    # bf16 storage doubles the HBM roof
    assert M.roofline_cells(2, 1, 1, 2, p, bw) == pytest.approx(bw / 4)


def test_splitmix64_reference_values():
    # SplitMix64 seeded with 1234567 (Vigna's splitmix64.c, state += GAMMA then mix):
    # first outputs as listed in the widely used test vector of that reference implementation.
    got = gen.splitmix64(1234567, np.arange(5, dtype=np.uint64))
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [int(v) for v in got] == want


def test_uniform_counter_based_and_in_range():
    a = gen.uniform(0, 1000)
    b = gen.uniform(0, 400, offset=600)
    assert np.array_equal(a[600:], b)
    assert a.dtype == np.float32 and a.min() >= 0 and a.max() < 1
    # 24-bit grid: every value times 2^24 is an integer
    assert np.all(np.floor(a.astype(np.float64) * 2 ** 24) == a.astype(np.float64) * 2 ** 24)
    assert abs(float(a.mean()) - 0.5) < 0.03


def test_coefficients_normalised_and_distinct():
    for d in (2, 3):
        for r in (1, 2, 3, 4):
            c = gen.coefficients(d, r)
            assert c.size == 2 * d * r + 1
            assert np.all(c > 0)
            assert len(np.unique(c)) == c.size
            assert abs(float(c.astype(np.float64).sum()) - 1.0) < c.size * 2 ** -24


def test_bump_input():
    g = gen.uniform_plus_bump((8, 40, 36))
    u = gen.uniform_grid((8, 40, 36))
    d = g.astype(np.float64) - u
    assert d.max() == pytest.approx(1.0, abs=1e-6)           # amplitude 1 at the centre plane
    assert np.unravel_index(np.argmax(d), d.shape) == (4, 20, 18)
    assert g.min() >= 0 and g.max() < 2


def test_batch_list_shape():
    items = gen.batch_list()
    assert len(items) == 96
    assert sum(1 for it in items if it["dim"] == 2) == 64
    for it in items:
        lo, hi = (512, 8192) if it["dim"] == 2 else (64, 384)
        assert lo <= it["nx"] <= hi and lo <= it["ny"] <= hi
        assert it["dim"] == 2 or lo <= it["nz"] <= hi
        assert 1 <= it["r"] <= 4 and it["dtype"] in ("f32", "bf16")
    assert {it["dtype"] for it in items} == {"f32", "bf16"}
