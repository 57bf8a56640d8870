"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test is built so that a plausible slip in oracle.c (a dropped term, a
swapped direction, a transposed coefficient layout, a wrap instead of a
clamp, a sum starting at i = 0, a fused first multiply, a missing clamp at
intermediate steps) fails at least one of them.
"""
from fractions import Fraction
import math

import numpy as np
import pytest

import stencil_inputs as gen

DIRS = {2: [(-1, 0), (1, 0), (0, -1), (0, 1)],
        3: [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]}


# ---------------------------------------------------------------- helpers
def shape_of(dim, nx, ny, nz=1):
    return (ny, nx) if dim == 2 else (nz, ny, nx)


def dense_operator(dim, r, c, nx, ny, nz=1):
    """One step as an N x N matrix: row p gets c_k at the clamped neighbour column.

    Written from the problem statement (Eq. 1 + clamp-to-border), independent
    of the oracle's loops: clamping is folded in by summing coefficients that
    land on the same border cell.
    """
    n = nx * ny * nz
    a = np.zeros((n, n))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                p = x + nx * (y + ny * z)
                a[p, p] += c[0]
                for i in range(1, r + 1):
                    for d, e in enumerate(DIRS[dim]):
                        q = [x + i * e[0], y + i * e[1]] + ([z + i * e[2]] if dim == 3 else [z])
                        qx = min(max(q[0], 0), nx - 1)
                        qy = min(max(q[1], 0), ny - 1)
                        qz = min(max(q[2], 0), nz - 1)
                        a[p, qx + nx * (qy + ny * qz)] += c[1 + (i - 1) * 2 * dim + d]
    return a


def rne_f32(q: Fraction) -> Fraction:
    """Round an exact rational to the nearest binary32 (ties to even), normal range."""
    if q == 0:
        return Fraction(0)
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length() - 24
    while a >= Fraction(2) ** (e + 24):
        e += 1
    while a < Fraction(2) ** (e + 23):
        e -= 1
    assert e >= -149 - 23, "subnormal range not needed by these tests"
    m = a / Fraction(2) ** e                      # in [2^23, 2^24)
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return sign * Fraction(fl) * Fraction(2) ** e


def exact_fp32_sweep(f, dim, r, c, iters):
    """Brute force with exact rationals: each fp32 FMA is exact product + sum, rounded once."""
    cq = [Fraction(float(v)) for v in c]
    cur = np.vectorize(lambda v: Fraction(float(v)), otypes=[object])(f)
    shp = cur.shape
    for _ in range(iters):
        nxt = np.empty(shp, dtype=object)
        for idx in np.ndindex(*shp):
            pos = list(idx[::-1])                 # (x, y[, z])
            acc = rne_f32(cq[0] * cur[idx])
            for i in range(1, r + 1):
                for d, e in enumerate(DIRS[dim]):
                    q = [min(max(pos[a] + i * e[a], 0), shp[::-1][a] - 1) for a in range(dim)]
                    acc = rne_f32(cq[1 + (i - 1) * 2 * dim + d] * cur[tuple(q[::-1])] + acc)
            nxt[idx] = acc
        cur = nxt
    return np.vectorize(float, otypes=[np.float64])(cur)


def run_f64(oracle_mod, f, dim, r, c, iters):
    return oracle_mod.sweep_f64(f, dim, r, c, iters)


# ---------------------------------------------------------------- pins
@pytest.mark.parametrize("dim,nx,ny,nz,r", [
    (2, 5, 7, 1, 1), (2, 5, 7, 1, 2), (2, 5, 7, 1, 4), (2, 3, 2, 1, 3),
    (3, 3, 4, 5, 1), (3, 3, 4, 5, 2), (3, 4, 3, 2, 4), (3, 1, 2, 3, 2),
    (2, 9, 8, 1, 6), (3, 4, 5, 3, 5)])
def test_dense_operator_power(oracle_mod, dim, nx, ny, nz, r):
    """A^iters x (dense operator, clamp folded in) equals the FP64 oracle."""
    rng = np.random.default_rng(100 + dim * 10 + r)
    c = gen.coefficients(dim, r, seed=7 + r).astype(np.float64)
    f = rng.random(shape_of(dim, nx, ny, nz))
    iters = 4
    a = dense_operator(dim, r, c, nx, ny, nz)
    ref = (np.linalg.matrix_power(a, iters) @ f.reshape(-1)).reshape(f.shape)
    got = run_f64(oracle_mod, f, dim, r, c, iters)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("dim,r", [(2, 1), (2, 3), (3, 2), (3, 4)])
def test_dense_operator_random_signed_coeffs(oracle_mod, dim, r):
    """Signed, non-normalised coefficients: catches sign or scale slips that convex weights hide."""
    rng = np.random.default_rng(5 + r)
    c = rng.normal(size=2 * dim * r + 1) * 0.3
    nx, ny, nz = (6, 5, 1) if dim == 2 else (4, 3, 5)
    f = rng.normal(size=shape_of(dim, nx, ny, nz))
    a = dense_operator(dim, r, c, nx, ny, nz)
    ref = (np.linalg.matrix_power(a, 3) @ f.reshape(-1)).reshape(f.shape)
    np.testing.assert_allclose(run_f64(oracle_mod, f, dim, r, c, 3), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dim,r", [(2, 1), (2, 2), (2, 4), (3, 1), (3, 3), (3, 4), (2, 6), (3, 5)])
def test_shift_stencil_exact(oracle_mod, dim, r):
    """A single unit coefficient at (distance i, direction d) moves the field by
    i*iters cells against that direction, clamped: out[p] = in[clamp(p + i*iters*e_d)].
    Pins the direction order W,E,S,N,B,A, the coefficient layout and the clamp."""
    nx, ny, nz = (11, 9, 1) if dim == 2 else (7, 6, 5)
    rng = np.random.default_rng(3)
    f = rng.random(shape_of(dim, nx, ny, nz)).astype(np.float32)
    iters = 2
    for i in range(1, r + 1):
        for d, e in enumerate(DIRS[dim]):
            c = np.zeros(2 * dim * r + 1, dtype=np.float32)
            c[1 + (i - 1) * 2 * dim + d] = 1.0
            ref = np.empty_like(f)
            for idx in np.ndindex(*f.shape):
                pos = list(idx[::-1])
                ext = f.shape[::-1]
                q = [min(max(pos[a] + i * iters * e[a], 0), ext[a] - 1) for a in range(dim)]
                ref[idx] = f[tuple(q[::-1])]
            assert np.array_equal(oracle_mod.sweep_f32(f, dim, r, c, iters), ref)
            assert np.array_equal(oracle_mod.sweep_f64(f, dim, r, c, iters), ref.astype(np.float64))


@pytest.mark.parametrize("dim,r", [(2, 1), (2, 4), (3, 2), (3, 4)])
def test_constant_field_exact_with_dyadic_coeffs(oracle_mod, dim, r):
    """Dyadic coefficients summing to exactly 1 keep a dyadic constant exactly, in fp32 and fp64."""
    k = 2 * dim * r + 1
    c = np.full(k, 0.5 / (k - 1) if ((k - 1) & (k - 2)) == 0 else 0.0)
    # build exact dyadic weights: centre 1/2, the rest sums to 1/2 in powers of two
    rest = np.zeros(k - 1)
    remaining = 0.5
    for j in range(k - 2):
        rest[j] = remaining / 2
        remaining -= rest[j]
    rest[k - 2] = remaining
    c = np.concatenate([[0.5], rest])
    assert c.sum() == 1.0
    nx, ny, nz = (9, 7, 1) if dim == 2 else (5, 6, 4)
    f = np.full(shape_of(dim, nx, ny, nz), 0.375)
    assert np.all(oracle_mod.sweep_f64(f, dim, r, c, 7) == 0.375)
    assert np.all(oracle_mod.sweep_f32(f, dim, r, c.astype(np.float32), 7) == np.float32(0.375))


@pytest.mark.parametrize("dim,r", [(2, 2), (3, 3)])
def test_constant_field_normalised_coeffs(oracle_mod, dim, r):
    """Seeded normalised coefficients: a constant drifts by at most |sum c - 1| * iters + rounding."""
    c = gen.coefficients(dim, r)
    s = float(np.sum(c.astype(np.float64)))
    nx, ny, nz = (8, 8, 1) if dim == 2 else (5, 5, 5)
    f = np.full(shape_of(dim, nx, ny, nz), 0.7)
    iters = 50
    out = oracle_mod.sweep_f64(f, dim, r, c.astype(np.float64), iters)
    bound = 0.7 * (abs(s ** iters - 1.0)) + 1e-13 * iters
    assert np.max(np.abs(out - 0.7)) <= bound + 1e-15
    assert np.ptp(out) <= 1e-13 * iters      # every cell sees the same weights


@pytest.mark.parametrize("dim,r", [(2, 1), (2, 4), (3, 1), (3, 4)])
def test_max_principle(oracle_mod, dim, r):
    """Nonnegative weights with sum ~1 keep [0,1] data within [0, 1 + K u] at every step count."""
    c = gen.coefficients(dim, r)
    nx, ny, nz = (13, 11, 1) if dim == 2 else (7, 6, 5)
    f = gen.uniform_grid(shape_of(dim, nx, ny, nz), seed=4)
    k = c.size
    for iters in (1, 3, 10):
        o32 = oracle_mod.sweep_f32(f, dim, r, c, iters)
        o64 = oracle_mod.sweep_f64(f, dim, r, c, iters)
        tol = iters * k * 2.0 ** -24 + abs(float(np.sum(c, dtype=np.float64)) - 1) * iters
        for o in (o32, o64):
            assert o.min() >= 0.0
            assert o.max() <= 1.0 + tol
            # also never above the input's max / below its min (averaging)
            assert o.max() <= f.max() + tol and o.min() >= f.min() - tol


@pytest.mark.parametrize("dim,nx,ny,nz,r,iters", [
    (2, 6, 5, 1, 2, 2), (2, 4, 3, 1, 4, 1), (3, 3, 4, 3, 1, 2), (3, 2, 3, 2, 2, 1)])
def test_fp32_exact_rational_bruteforce(oracle_mod, dim, nx, ny, nz, r, iters):
    """The fp32 oracle equals an exact-rational evaluation of the same FMA chain, bit for bit."""
    c = gen.coefficients(dim, r)
    f = gen.uniform_grid(shape_of(dim, nx, ny, nz), seed=11)
    ref = exact_fp32_sweep(f, dim, r, c, iters).astype(np.float32)
    got = oracle_mod.sweep_f32(f, dim, r, c, iters)
    assert np.array_equal(got, ref)


def test_fp32_first_operation_is_rounded_multiply(oracle_mod):
    """K=5 stencil whose centre product is inexact: a fused first step would differ."""
    c = np.array([1.0 + 2 ** -12, 0, 0, 0, 0], dtype=np.float32)
    f = np.array([[1.0 + 2 ** -13]], dtype=np.float32)
    want = rne_f32(Fraction(float(c[0])) * Fraction(float(f[0, 0])))
    assert oracle_mod.sweep_f32(f, 2, 1, c, 1)[0, 0] == np.float32(float(want))


@pytest.mark.parametrize("dim,r,iters", [(2, 1, 40), (2, 4, 40), (3, 1, 20), (3, 4, 20)])
def test_fp32_within_bound_of_fp64(oracle_mod, dim, r, iters):
    """Max-abs(fp32 - fp64) <= 2e-6 * iters (the operator is nonexpansive in max norm)."""
    c = gen.coefficients(dim, r)
    shape = shape_of(dim, 40, 33) if dim == 2 else shape_of(dim, 20, 17, 15)
    f = gen.workload_grid(dim, *shape[::-1])
    o32 = oracle_mod.sweep_f32(f, dim, r, c, iters)
    o64 = oracle_mod.sweep_f64(f.astype(np.float64), dim, r, c.astype(np.float64), iters)
    assert np.max(np.abs(o32 - o64)) <= 2e-6 * iters


def _np_step_f64(f, dim, r, c):
    """Test-side vectorised step (np.pad edge mode = clamp) in Eq. 1 order."""
    pad = [(r, r)] * f.ndim
    g = np.pad(f, pad, mode="edge")
    core = tuple(slice(r, r + n) for n in f.shape)

    def shifted(axis_from_x, off):
        sl = list(core)
        ax = f.ndim - 1 - axis_from_x
        sl[ax] = slice(r + off, r + off + f.shape[ax])
        return g[tuple(sl)]

    acc = c[0] * f
    for i in range(1, r + 1):
        for d in range(2 * dim):
            acc = acc + c[1 + (i - 1) * 2 * dim + d] * shifted(d // 2, -i if d % 2 == 0 else i)
    return acc


@pytest.mark.parametrize("dim,r,t", [(2, 1, 3), (2, 2, 4), (3, 1, 2), (3, 2, 3)])
def test_overlapped_temporal_blocking_equals_naive(oracle_mod, dim, r, t):
    """Overlapped blocking (Section III.A, Eq. 2): tiles with an r*t halo, t steps each,
    clamp applied at the grid edge of every step, reproduce t plain sweeps exactly."""
    c = gen.coefficients(dim, r).astype(np.float64)
    shape = (23, 29) if dim == 2 else (9, 11, 13)
    f = gen.uniform_grid(shape, seed=9).astype(np.float64)
    ref = oracle_mod.sweep_f64(f, dim, r, c, t)
    h = r * t
    bsize = 2 * h + 5                             # block along x (and y in 3D)
    csz = bsize - 2 * h
    assert csz > 0
    out = np.empty_like(f)
    nx = shape[-1]
    ny = shape[-2]
    ys = range(0, ny, csz) if dim == 3 else [0]
    for y0 in ys:
        for x0 in range(0, nx, csz):
            xa, xb = max(x0 - h, 0), min(x0 + csz + h, nx)
            if dim == 3:
                ya, yb = max(y0 - h, 0), min(y0 + csz + h, ny)
                blk = f[:, ya:yb, xa:xb]
            else:
                blk = f[:, xa:xb]
            # the block's own clamp is the global clamp only where the block touches the edge;
            # elsewhere the halo is wide enough that its invalid rim never reaches the centre
            for _ in range(t):
                blk = _np_step_f64(blk, dim, r, c)
            xe = min(x0 + csz, nx)
            if dim == 3:
                ye = min(y0 + csz, ny)
                out[:, y0:ye, x0:xe] = blk[:, y0 - ya:ye - ya, x0 - xa:xe - xa]
            else:
                out[:, x0:xe] = blk[:, x0 - xa:xe - xa]
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("dim,r", [(2, 3), (3, 2)])
def test_mirror_symmetry(oracle_mod, dim, r):
    """Reversing x and swapping the W/E coefficients mirrors the result."""
    c = gen.coefficients(dim, r)
    shape = (7, 10) if dim == 2 else (4, 5, 6)
    f = gen.uniform_grid(shape, seed=12)
    cm = c.copy()
    for i in range(r):
        b = 1 + i * 2 * dim
        cm[b], cm[b + 1] = c[b + 1], c[b]
    a = oracle_mod.sweep_f64(f, dim, r, c, 3)
    b = oracle_mod.sweep_f64(np.ascontiguousarray(f[..., ::-1]), dim, r, cm, 3)
    # the W and E terms swap places in the sum, so equality holds up to rounding only
    np.testing.assert_allclose(a, b[..., ::-1], rtol=0, atol=1e-14)
    assert not np.allclose(a, oracle_mod.sweep_f64(f, dim, r, cm, 3), rtol=0, atol=1e-6)


def test_iters_zero_is_copy(oracle_mod):
    f = gen.uniform_grid((5, 4), seed=3)
    c = gen.coefficients(2, 1)
    assert np.array_equal(oracle_mod.sweep_f32(f, 2, 1, c, 0), f)


def test_rejects_bad_arguments(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.sweep_f32(np.zeros((3, 3), np.float32), 2, 1, np.zeros(4), 1)
    with pytest.raises(ValueError):
        oracle_mod.sweep_f64(np.zeros((3, 3, 3)), 2, 1, np.zeros(5), 1)


# ---------------------------------------------------------------- shared-coefficient form
def expand_shared(dim, r, cs):
    """Per-(distance, direction) coefficients of a shared-coefficient stencil: c_{i,d} = c_i."""
    c = np.zeros(2 * dim * r + 1, dtype=np.float64)
    c[0] = cs[0]
    for i in range(1, r + 1):
        c[1 + (i - 1) * 2 * dim:1 + i * 2 * dim] = cs[i]
    return c


def shared_coeffs(dim, r):
    return gen.shared_coefficients(dim, r, seed=4)


@pytest.mark.parametrize("dim,nx,ny,nz,r", [(2, 6, 7, 1, 1), (2, 5, 9, 1, 3), (3, 4, 3, 5, 2), (3, 3, 4, 2, 4)])
def test_shared_form_is_the_dense_operator_with_equal_coefficients(oracle_mod, dim, nx, ny, nz, r):
    """Sharing one coefficient per distance is Eq. 1 with c_{i,d} = c_i: the FP64 shared
    oracle equals the dense operator built from the expanded coefficients."""
    cs = shared_coeffs(dim, r).astype(np.float64)
    rng = np.random.default_rng(40 + r)
    f = rng.random(shape_of(dim, nx, ny, nz))
    a = dense_operator(dim, r, expand_shared(dim, r, cs), nx, ny, nz)
    ref = (np.linalg.matrix_power(a, 3) @ f.reshape(-1)).reshape(f.shape)
    np.testing.assert_allclose(oracle_mod.sweep_shared_f64(f, dim, r, cs, 3), ref, rtol=1e-13, atol=1e-15)


def exact_shared_fp32_sweep(f, dim, r, cs, iters):
    """Brute force of the FP32 shared form with exact rationals: every add of the left-to-right
    neighbour sum rounded once, then one FMA (exact product + sum, rounded once) per distance."""
    cq = [Fraction(float(v)) for v in cs]
    cur = np.vectorize(lambda v: Fraction(float(v)), otypes=[object])(f)
    shp = cur.shape
    for _ in range(iters):
        nxt = np.empty(shp, dtype=object)
        for idx in np.ndindex(*shp):
            pos = list(idx[::-1])
            acc = rne_f32(cq[0] * cur[idx])
            for i in range(1, r + 1):
                vals = []
                for e in DIRS[dim]:
                    q = [min(max(pos[a] + i * e[a], 0), shp[::-1][a] - 1) for a in range(dim)]
                    vals.append(cur[tuple(q[::-1])])
                s = vals[0]
                for v in vals[1:]:
                    s = rne_f32(s + v)
                acc = rne_f32(cq[i] * s + acc)
            nxt[idx] = acc
        cur = nxt
    return np.vectorize(float, otypes=[np.float64])(cur)


@pytest.mark.parametrize("dim,nx,ny,nz,r,iters", [(2, 6, 5, 1, 2, 2), (2, 4, 3, 1, 4, 1), (3, 3, 4, 3, 1, 2),
                                                  (3, 2, 3, 2, 3, 1)])
def test_shared_fp32_exact_rational_bruteforce(oracle_mod, dim, nx, ny, nz, r, iters):
    cs = shared_coeffs(dim, r)
    f = gen.uniform_grid(shape_of(dim, nx, ny, nz), seed=12)
    ref = exact_shared_fp32_sweep(f, dim, r, cs, iters).astype(np.float32)
    assert np.array_equal(oracle_mod.sweep_shared_f32(f, dim, r, cs, iters), ref)


def test_shared_fp32_differs_from_full_chain_but_agrees_with_fp64():
    """The shared FP32 order is its own rounding sequence (not the full form's FMA chain
    with equal coefficients), and within 2e-6 * iters of FP64."""
    import oracle
    dim, r, iters = 2, 4, 10
    cs = shared_coeffs(dim, r)
    f = gen.uniform_grid((40, 48), seed=13)
    got = oracle.sweep_shared_f32(f, dim, r, cs, iters)
    full = oracle.sweep_f32(f, dim, r, expand_shared(dim, r, cs).astype(np.float32), iters)
    assert not np.array_equal(got, full)
    w64 = oracle.sweep_shared_f64(f.astype(np.float64), dim, r, cs.astype(np.float64), iters)
    assert np.max(np.abs(got - w64)) <= 2e-6 * iters
