"""Host-side logic of the tuning driver (no GPU): the seeded problem set, the timing
database built from stencil_timing rows, and the analytic model's accuracy ratio."""
import math

import numpy as np

import paper_2002_05983_gb300 as st
from paper_2002_05983_gb300 import tune


def timing(t, seg, ns, analytic, feats):
    row = st.Timing()
    row.sched.t, row.sched.seg = t, seg
    row.ns_per_cell, row.analytic_ns_per_cell, row.model_ns_per_cell = ns, analytic, -1.0
    for i, v in enumerate(feats):
        row.features[i] = v
    return row


def test_problem_set_is_seeded_and_streamable():
    a, b = tune.tuning_problems(30), tune.tuning_problems(30)
    assert a == b
    assert tune.tuning_problems(30, seed=4) != a
    for p in a:
        assert p["nx"] % 8 == 0 and p["ny"] % 8 == 0 and p["nx"] >= 64
        assert p["dim"] in (2, 3) and 1 <= p["r"] <= 4 and (p["nz"] == 1) == (p["dim"] == 2)
        assert p["dtype"] in (st.STENCIL_F32, st.STENCIL_BF16)


def test_database_and_accuracy_from_rows():
    f = list(range(st.NFEAT))
    meas = [({"dim": 2}, [timing(1, 128, 0.004, 0.005, f), timing(2, 256, 0.002, 0.004, f),
                          timing(3, 512, -1.0, 0.003, f)]),          # an unmeasured row is skipped
            ({"dim": 3}, [timing(1, 64, 0.008, 0.004, f)])]
    X, y, g = tune.database(meas)
    assert X.shape == (3, st.NFEAT) and X.dtype == np.float32
    # target: log of measured over analytic time (the analytic model's error)
    np.testing.assert_allclose(y, np.log([0.8, 0.5, 2.0]).astype(np.float32), rtol=1e-6)
    assert list(g) == [0, 0, 1]
    ratio = tune.analytic_accuracy(meas)
    np.testing.assert_allclose(sorted(ratio), sorted([0.8, 0.5, 2.0]), rtol=1e-6)  # float32 fields
    assert math.isclose(float(np.median(ratio)), 0.8, rel_tol=1e-6)


def test_regret_arithmetic_on_a_timing_table():
    """Regret T(pick)/T(best) - 1 over a problem's measured candidates, and the schedule
    match that maps a pick back to its measured row (t, segment, rows, rows per step)."""
    times = [0.010, 0.008, 0.0125, 0.0096]
    assert tune.regret_of(times, 1) == 0.0
    assert abs(tune.regret_of(times, 3) - 0.2) < 1e-12
    assert abs(tune.regret_of(times, 0) - 0.25) < 1e-12
    a, b = st.Schedule(), st.Schedule()
    a.t, a.seg, a.rows_per_thread, a.planes_per_step = 2, 256, 1, 2
    b.t, b.seg, b.rows_per_thread, b.planes_per_step = 2, 256, 1, 2
    assert tune.same_schedule(a, b)
    b.planes_per_step = 1
    assert not tune.same_schedule(a, b)
