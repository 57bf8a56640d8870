"""Schedule tuning driver: measured timing database, cost-model training, regret.

The paper picks FPGA parameters with a performance model and places and
routes the top few (Sections V.A and VI.A).  Here the choice of temporal
degree, rows per step (2D), stream-segment length and (3D) rows per thread is
made by ``stencil_tune``: exhaustively on the GPU, from the analytic
bandwidth/issue model, or from a learned cost model (a 2x64 ReLU MLP whose
forward/backward/Adam kernels are in csrc/mlp.cu) that predicts the log of
measured over analytic time, i.e. learns the analytic model's error.  This
module only loops over problems and marshals arrays; all timing and training
runs in the library.
"""
from __future__ import annotations

import math

import numpy as np

from . import (STENCIL_BF16, STENCIL_F32, Stencil, TUNE_ANALYTIC, TUNE_EXHAUSTIVE, TUNE_MODEL,
               stencil_model_create, stencil_model_destroy, stencil_model_train, stencil_tune)


def tuning_problems(n: int, seed: int = 3):
    """Seeded problems shaped like the batched workload (2D sides 512..8192, 3D 64..384,
    radius 1..4, FP32/BF16), sides rounded to multiples of 8 so that every candidate of the
    streaming kernel applies."""
    import stencil_inputs as gen
    u = gen.uniform(seed, 8 * n)
    out = []
    for i in range(n):
        a = u[8 * i:8 * i + 8]
        dim = 2 if a[0] < 2 / 3 else 3
        lo, hi = (512, 8192) if dim == 2 else (64, 384)
        side = [int(lo + a[k] * (hi - lo)) // 8 * 8 for k in (1, 2, 3)]
        r = 1 + min(int(a[4] * 4), 3)
        dtype = STENCIL_BF16 if a[5] < 0.5 else STENCIL_F32
        nz = side[2] if dim == 3 else 1
        out.append(dict(dim=dim, r=r, nx=side[0], ny=side[1], nz=nz, dtype=dtype))
    return out


def coeffs_for(dim, r):
    import stencil_inputs as gen
    return gen.coefficients(dim, r)


def measure(problems):
    """Exhaustive timing of every candidate schedule of every problem.
    Returns a list of (problem, rows) with rows = list of Timing."""
    out = []
    for p in problems:
        s = Stencil(p["dim"], p["r"], coeffs_for(p["dim"], p["r"]))
        _, rows = stencil_tune(s.handle, p["nx"], p["ny"], p["nz"], p["dtype"], TUNE_EXHAUSTIVE, store=False)
        out.append((p, rows))
        s.close()
    return out


def database(measured):
    """Feature matrix X, target y = log(measured / analytic ns per cell update) (the
    analytic model's error, which stencil_tune's MODEL mode multiplies back in), problem
    index per row."""
    X, y, g = [], [], []
    for i, (_, rows) in enumerate(measured):
        for t in rows:
            if t.ns_per_cell > 0 and t.analytic_ns_per_cell > 0:
                X.append(list(t.features))
                y.append(math.log(t.ns_per_cell / t.analytic_ns_per_cell))
                g.append(i)
    return np.asarray(X, np.float32), np.asarray(y, np.float32), np.asarray(g)


def same_schedule(a, b) -> bool:
    return (a.t == b.t and a.seg == b.seg and a.rows_per_thread == b.rows_per_thread
            and a.planes_per_step == b.planes_per_step)


def regret_of(times, pick: int) -> float:
    """T(pick) / T(best) - 1 over a problem's measured candidate times."""
    times = np.asarray(times, np.float64)
    return float(times[pick] / times.min() - 1.0)


def train(X, y, epochs=3000, lr=3e-3, seed=0, hidden=64):
    m = stencil_model_create(X.shape[1], hidden, seed)
    loss = stencil_model_train(m, X, y, epochs=epochs, lr=lr)
    return m, loss


def regret(model, measured):
    """Per problem: T(pick)/T(best) - 1 for the model's pick and the analytic pick, the
    times being the exhaustive measurements of those schedules."""
    res = []
    for p, rows in measured:
        times = np.array([t.ns_per_cell for t in rows], np.float64)
        best = times.min()
        s = Stencil(p["dim"], p["r"], coeffs_for(p["dim"], p["r"]))
        picks = {}
        for name, mode in (("model", TUNE_MODEL), ("analytic", TUNE_ANALYTIC)):
            ch, _ = stencil_tune(s.handle, p["nx"], p["ny"], p["nz"], p["dtype"], mode,
                                 model=model if mode == TUNE_MODEL else None, store=False)
            k = [i for i, t in enumerate(rows) if same_schedule(t.sched, ch)]
            picks[name] = regret_of(times, k[0]) if k else float("nan")
        s.close()
        res.append(dict(problem=p, best_ns=best, **{f"regret_{k}": v for k, v in picks.items()}))
    return res


def analytic_accuracy(measured):
    """Measured / analytic-predicted time per cell update, every timed schedule (the
    model-accuracy ratio the paper reports per configuration)."""
    return np.array([t.ns_per_cell / t.analytic_ns_per_cell for _, rows in measured for t in rows
                     if t.ns_per_cell > 0 and t.analytic_ns_per_cell > 0], np.float64)


def evaluate(n_train=48, n_test=16, seed=3, epochs=3000):
    """Measure, train on the first n_train problems, report regret on the rest."""
    probs = tuning_problems(n_train + n_test, seed)
    meas = measure(probs)
    X, y, _ = database(meas[:n_train])
    model, loss = train(X, y, epochs=epochs)
    try:
        test = regret(model, meas[n_train:])
        train_r = regret(model, meas[:n_train])
    finally:
        stencil_model_destroy(model)
    return dict(rows_train=int(len(y)), rows_total=int(sum(len(r) for _, r in meas)), train_loss=loss,
                test=test, train=train_r, analytic_ratio=analytic_accuracy(meas))
