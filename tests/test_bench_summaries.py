"""The committed ncu summaries that bench.py attaches to its line: DRAM traffic per launch and the
limiter of each benchmark kernel are used only while the kernel sources keep the hash they were
captured with, and the limiter's classification follows its stated thresholds."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _lines(name):
    with open(os.path.join(ROOT, "profiles", name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def test_summaries_match_the_current_kernel_sources():
    h = bench.kernel_source_hash(os.path.join(ROOT, "paper_2002_05983_gb300", "csrc"))
    for name in ("dram_traffic.txt", "ncu_limits.txt"):
        rows = _lines(name)
        assert rows and all(r[0] == h for r in rows), name
    # every benchmark kernel of the headline (2D) and of the 3D key has both lines
    for dim, r, t in ((2, 1, 4), (2, 2, 3), (2, 3, 2), (2, 4, 2)):
        assert bench.traffic_for(dim, r, t) is not None
        assert bench.limiter_for(dim, r, t, 0.5)["kind"] is not None


def test_dram_traffic_is_close_to_the_algorithmic_bytes():
    for f in _lines("dram_traffic.txt"):
        dim, n = int(f[1]), (16384 ** 2 if f[1] == "2" else 512 ** 3)
        assert 0.9 <= int(f[5]) / (2 * 4 * n) <= 1.02   # no re-reads (the 3D capture leaves writes in L2)


def test_limiter_classification():
    lim = bench.limiter_for(2, 4, 2, 0.67)
    assert lim["kind"] == "issue" and lim["dram_pct"] < 80 and lim["fma_pipe_pct"] < 80
    assert bench.limiter_for(2, 4, 2, 0.9)["kind"] == "hbm"       # the live bandwidth decides first
    assert bench.limiter_for(2, 4, 9, 0.5)["kind"] is None         # no counters for this kernel
