"""Schedule tuner and cost model on the GPU.

The MLP's CUDA forward and backward kernels are checked against a float64
NumPy evaluation of the same network, which is itself pinned by finite
differences; the tuner's choices must be valid schedules whose results stay
bit-identical to the oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2002_05983_gb300 as st
import stencil_inputs as gen
from paper_2002_05983_gb300 import tune

pytestmark = pytest.mark.gpu
H = 16
NF = 5


def unpack(p, nf=NF, h=H):
    i = 0
    W1 = p[i:i + nf * h].reshape(nf, h); i += nf * h
    b1 = p[i:i + h]; i += h
    W2 = p[i:i + h * h].reshape(h, h); i += h * h
    b2 = p[i:i + h]; i += h
    w3 = p[i:i + h]; i += h
    b3 = p[i]
    return W1, b1, W2, b2, w3, b3


def np_loss(p, X, y):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    a1 = np.maximum(X @ W1 + b1, 0)
    a2 = np.maximum(a1 @ W2 + b2, 0)
    out = a2 @ w3 + b3
    return np.mean((out - y) ** 2), out


def np_grad(p, X, y):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    z1 = X @ W1 + b1; a1 = np.maximum(z1, 0)
    z2 = a1 @ W2 + b2; a2 = np.maximum(z2, 0)
    out = a2 @ w3 + b3
    d3 = 2 * (out - y) / len(y)
    gw3 = a2.T @ d3; gb3 = d3.sum()
    d2 = np.outer(d3, w3) * (z2 > 0)
    gW2 = a1.T @ d2; gb2 = d2.sum(0)
    d1 = d2 @ W2.T * (z1 > 0)
    gW1 = X.T @ d1; gb1 = d1.sum(0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])


@pytest.fixture
def model_and_data():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(40, NF)).astype(np.float32)
    y = (X[:, 0] - 0.5 * X[:, 1] + 0.3 * X[:, 2] ** 2).astype(np.float32)
    m = st.stencil_model_create(NF, H, seed=7)
    st.stencil_model_normalization(m, np.zeros(NF), np.ones(NF), 0.0, 1.0)
    yield m, X, y
    st.stencil_model_destroy(m)


def test_numpy_gradient_pinned_by_finite_differences(model_and_data):
    m, X, y = model_and_data
    p = st.stencil_model_params(m).astype(np.float64)
    g = np_grad(p, X.astype(np.float64), y.astype(np.float64))
    rng = np.random.default_rng(1)
    for k in rng.choice(len(p), 25, replace=False):
        e = np.zeros_like(p); e[k] = 1e-6
        fd = (np_loss(p + e, X, y)[0] - np_loss(p - e, X, y)[0]) / 2e-6
        assert fd == pytest.approx(g[k], rel=1e-4, abs=1e-7)


def test_cuda_forward_and_backward_match_float64(model_and_data):
    m, X, y = model_and_data
    p = st.stencil_model_params(m).astype(np.float64)
    loss_ref, out_ref = np_loss(p, X.astype(np.float64), y.astype(np.float64))
    pred = st.stencil_model_predict(m, X)
    np.testing.assert_allclose(pred, out_ref, rtol=1e-4, atol=1e-5)
    loss, g = st.stencil_model_grad(m, X, y)
    assert loss == pytest.approx(loss_ref, rel=1e-4)
    np.testing.assert_allclose(g, np_grad(p, X.astype(np.float64), y.astype(np.float64)), rtol=2e-3, atol=1e-5)


def test_training_fits_a_smooth_function(model_and_data):
    m, X, y = model_and_data
    before, _ = st.stencil_model_grad(m, X, y)
    after = st.stencil_model_train(m, X, y, epochs=1500, lr=1e-2)
    assert after < 0.05 * before


@pytest.mark.parametrize("dim,r,shape,dt", [(2, 2, (520, 1024), st.STENCIL_F32), (3, 1, (48, 40, 64), st.STENCIL_F32),
                                          (2, 4, (256, 512), st.STENCIL_BF16)])
def test_tune_modes_pick_valid_schedules(dim, r, shape, dt):
    c = gen.coefficients(dim, r)
    s = st.Stencil(dim, r, c)
    nx, ny, nz = (shape[1], shape[0], 1) if dim == 2 else shape[::-1]
    chosen, rows = st.stencil_tune(s.handle, nx, ny, nz, dt, st.TUNE_EXHAUSTIVE, store=False)
    assert len(rows) >= 3
    times = [t.ns_per_cell for t in rows]
    assert min(times) > 0
    k = int(np.argmin(times))
    assert tune.same_schedule(chosen, rows[k].sched)
    feats = np.array([list(t.features) for t in rows], np.float32)
    assert np.all(np.isfinite(feats))
    # analytic mode stores its pick; stencil_run then uses it and stays bit-exact
    a, _ = st.stencil_tune(s.handle, nx, ny, nz, dt, st.TUNE_ANALYTIC, store=True)
    assert a.t >= 1 and a.seg >= 1
    if dt == st.STENCIL_F32:
        f = gen.workload_grid(dim, nx, ny, nz)
        got = s.run(torch.from_numpy(f).cuda(), 2 * a.t + 1).cpu().numpy()
        assert np.array_equal(got, oracle.sweep_f32(f, dim, r, c, 2 * a.t + 1))
    # model mode with a model trained on these rows: it predicts log(measured / analytic)
    X = feats
    yv = np.log([t.ns_per_cell / t.analytic_ns_per_cell for t in rows]).astype(np.float32)
    m = st.stencil_model_create(st.NFEAT, 64, 0)
    st.stencil_model_train(m, X, yv, epochs=800, lr=3e-3)
    mc, mrows = st.stencil_tune(s.handle, nx, ny, nz, dt, st.TUNE_MODEL, model=m, store=False)
    assert all(t.model_ns_per_cell > 0 for t in mrows)
    pred = np.array([t.model_ns_per_cell for t in mrows])
    # the lowest prediction, unless it is less than 5 % below the analytic pick's (trust region)
    im = int(np.argmin(pred))
    ia = int(np.argmin([t.analytic_ns_per_cell for t in mrows]))
    want = im if pred[im] < (1 - 0.05) * pred[ia] else ia
    assert tune.same_schedule(mc, mrows[want].sched)
    np.testing.assert_allclose(pred, [t.analytic_ns_per_cell for t in mrows] *
                               np.exp(st.stencil_model_predict(m, X)), rtol=1e-5)
    st.stencil_model_destroy(m)
    s.close()


def test_active_cost_model_proposes_default_schedules():
    """With stencil_use_cost_model set, a problem without a stored pick runs the model's pick
    (stays bit-exact); a stored pick still wins; None restores the library's rule."""
    dim, r, nx, ny = 2, 3, 1024, 520
    c = gen.coefficients(dim, r)
    s = st.Stencil(dim, r, c)
    rule = s.default_schedule((ny, nx))
    _, rows = st.stencil_tune(s.handle, nx, ny, 1, st.STENCIL_F32, st.TUNE_ANALYTIC, store=False)
    X = np.array([list(t.features) for t in rows], np.float32)
    # a model that prefers one temporal degree: predicted error grows away from t = 1
    yv = np.array([0.5 * (t.sched.t - 1) for t in rows], np.float32)
    m = st.stencil_model_create(st.NFEAT, 64, 1)
    st.stencil_model_train(m, X, yv, epochs=1500, lr=3e-3)
    want, _ = st.stencil_tune(s.handle, nx, ny, 1, st.STENCIL_F32, st.TUNE_MODEL, model=m, store=False)
    try:
        st.stencil_use_cost_model(m)
        fresh = st.Stencil(dim, r, c)
        got = fresh.default_schedule((ny, nx))
        assert tune.same_schedule(got, want)
        f = gen.workload_grid(dim, nx, ny)
        out = fresh.run(torch.from_numpy(f).cuda(), 5).cpu().numpy()
        assert np.array_equal(out, oracle.sweep_f32(f, dim, r, c, 5))
        stored, _ = st.stencil_tune(fresh.handle, nx, ny, 1, st.STENCIL_F32, st.TUNE_ANALYTIC, store=True)
        assert tune.same_schedule(fresh.default_schedule((ny, nx)), stored)
    finally:
        st.stencil_use_cost_model(None)
    other = st.Stencil(dim, r, c)
    d = other.default_schedule((ny, nx))
    assert (d.t, d.planes_per_step, d.seg) == (rule.t, rule.planes_per_step, rule.seg)
    st.stencil_model_destroy(m)


def test_tuning_problem_set_is_streamable():
    for p in tune.tuning_problems(20):
        assert p["nx"] % 8 == 0 and p["nx"] >= 64
        assert 1 <= p["r"] <= 4 and p["dim"] in (2, 3)


def test_tuning_cache_file_is_shared_between_handles(tmp_path, monkeypatch):
    """A pick stored with STENCIL_TUNE_CACHE set is appended to that file and becomes the
    schedule of a fresh handle of the same problem; a bit-exact run follows it."""
    path = tmp_path / "tune.cache"
    monkeypatch.setenv("STENCIL_TUNE_CACHE", str(path))
    dim, r, nx, ny = 2, 3, 1024, 520
    c = gen.coefficients(dim, r)
    a = st.Stencil(dim, r, c)
    base = a.default_schedule((ny, nx))
    chosen, _ = st.stencil_tune(a.handle, nx, ny, 1, st.STENCIL_F32, st.TUNE_ANALYTIC, store=True)
    line = path.read_text().strip().splitlines()[-1].split()
    assert line[0] == "v2" and [int(v) for v in line[2:9]] == [dim, r, 0, 0, nx, ny, 1]
    assert int(line[-1]) == chosen.planes_per_step
    b = st.Stencil(dim, r, c)
    got = b.default_schedule((ny, nx))
    assert (got.t, got.seg, got.kernel, got.planes_per_step) == (chosen.t, chosen.seg, chosen.kernel,
                                                                 chosen.planes_per_step)
    f = gen.workload_grid(dim, nx, ny)
    out = b.run(torch.from_numpy(f).cuda(), 7).cpu().numpy()
    assert np.array_equal(out, oracle.sweep_f32(f, dim, r, c, 7))
    # another shape is not affected; without the variable the file is ignored
    assert b.default_schedule((ny, nx + 8)).t == base.t
    monkeypatch.delenv("STENCIL_TUNE_CACHE")
    b2 = st.Stencil(dim, r, c)
    assert (b2.default_schedule((ny, nx)).t, b2.default_schedule((ny, nx)).seg) == (base.t, base.seg)
