"""Seeded synthetic inputs for the star-stencil workloads.

This module is shared by the CPU oracle tests, the GPU parity tests and the
benchmark.  It holds no stencil arithmetic: only the counter-based random
numbers, the coefficient draw and the Gaussian bump that define the inputs.

Random numbers are SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; constants as published by
Vigna): the generator seeded with ``s`` returns ``mix(s + k*GAMMA)`` as its
k-th output (k = 1, 2, ...), so element ``i`` of a stream is available
without running the stream, which lets huge grids be generated in chunks.

uniform(seed, n)[i] = top 24 bits of output i+1, times 2**-24  ->  [0, 1) in fp32 exactly.

Workload recipe (the paper's inputs are unspecified grids of the sizes it
lists in Section IV.C; these stand in for them):
  * grid values: uniform [0, 1) from seed 0, x fastest;
  * coefficients: K = 2*D*r + 1 weights u_k + 2**-25 from seed 1, divided by
    their sum in fp64 and rounded to fp32 (nonnegative, sum ~1, distinct);
    the one-per-distance form draws r + 1 weights the same way and divides by
    w_0 + 2*D*(w_1 + ... + w_r) (operator row sum ~1);
  * 3D workloads add a Gaussian bump exp(-|p - c|^2 / (2 sigma^2)),
    sigma = 16 cells, c = (nx//2, ny//2, nz//2), amplitude 1, summed in fp64
    and rounded once to fp32.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22

GRID_SEED = 0
COEFF_SEED = 1
BUMP_SIGMA = 16.0


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """Output idx+1 of SplitMix64 seeded with ``seed`` (idx: uint64 array)."""
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        z = s + (idx.astype(np.uint64) + np.uint64(1)) * GAMMA
        return _mix(z)


def uniform(seed: int, n: int, offset: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    """n fp32 values in [0, 1): element i uses counter offset + i."""
    if out is None:
        out = np.empty(n, dtype=np.float32)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        idx = np.arange(offset + a, offset + b, dtype=np.uint64)
        top = (splitmix64(seed, idx) >> np.uint64(40)).astype(np.float32)
        out[a:b] = top * np.float32(2.0 ** -24)
    return out


def num_coeffs(dim: int, radius: int) -> int:
    return 2 * dim * radius + 1


def coefficients(dim: int, radius: int, seed: int = COEFF_SEED) -> np.ndarray:
    """Nonnegative fp32 coefficients summing to ~1, all distinct.

    Layout: c[0] is the centre; c[1 + (i-1)*2*dim + d] is distance i in
    direction d = W(-x), E(+x), S(-y), N(+y), B(-z), A(+z).
    """
    k = num_coeffs(dim, radius)
    w = uniform(seed, k).astype(np.float64) + 2.0 ** -25
    c = (w / w.sum()).astype(np.float32)
    if len(np.unique(c)) != k:
        raise ValueError("coefficient draw is not distinct; choose another seed")
    return c


def shared_coefficients(dim: int, radius: int, seed: int = COEFF_SEED) -> np.ndarray:
    """Nonnegative fp32 coefficients of the one-per-distance form: c[0] the centre,
    c[i] every neighbour at distance i; normalised so that c[0] + 2*dim*sum(c[1:]) ~ 1."""
    w = uniform(seed, radius + 1).astype(np.float64) + 2.0 ** -25
    return (w / (w[0] + 2 * dim * w[1:].sum())).astype(np.float32)


def grid_shape(dim: int, nx: int, ny: int, nz: int = 1) -> tuple:
    return (ny, nx) if dim == 2 else (nz, ny, nx)


def uniform_grid(shape, seed: int = GRID_SEED, out: np.ndarray | None = None) -> np.ndarray:
    """Uniform [0,1) grid, row-major with x fastest (shape (ny,nx) or (nz,ny,nx))."""
    n = int(np.prod(shape))
    flat = None if out is None else out.reshape(-1)
    return uniform(seed, n, out=flat).reshape(shape)


def gaussian_bump(shape, sigma: float = BUMP_SIGMA) -> list:
    """Separable factors of exp(-|p-c|^2/(2 sigma^2)) per axis (fp64), centre at n//2."""
    return [np.exp(-((np.arange(n, dtype=np.float64) - n // 2) ** 2) / (2.0 * sigma * sigma))
            for n in shape]


def uniform_plus_bump(shape, seed: int = GRID_SEED, sigma: float = BUMP_SIGMA,
                      out: np.ndarray | None = None) -> np.ndarray:
    """3D workload input: uniform [0,1) plus a centred Gaussian bump, rounded once to fp32."""
    g = uniform_grid(shape, seed, out=out)
    fz, fy, fx = gaussian_bump(shape, sigma)
    for z in range(shape[0]):
        plane = g[z].astype(np.float64) + fz[z] * np.outer(fy, fx)
        g[z] = plane.astype(np.float32)
    return g


def workload_grid(dim: int, nx: int, ny: int, nz: int = 1, seed: int = GRID_SEED,
                  out: np.ndarray | None = None) -> np.ndarray:
    """The input of the 2D workloads (uniform) or the 3D workloads (uniform + bump)."""
    shape = grid_shape(dim, nx, ny, nz)
    if dim == 2:
        return uniform_grid(shape, seed, out=out)
    return uniform_plus_bump(shape, seed, out=out)


def batch_list(n2d: int = 64, n3d: int = 32, seed: int = 2):
    """Seeded list of mixed problems: 2D sides U[512, 8192], 3D sides U[64, 384],
    radius U{1..4}, dtype 'f32' or 'bf16'.  Returns dicts (dim, r, nx, ny, nz, dtype)."""
    out = []
    ctr = 0

    def draw(lo, hi):
        nonlocal ctr
        u = float(uniform(seed, 1, offset=ctr)[0])
        ctr += 1
        return lo + min(int(u * (hi - lo + 1)), hi - lo)

    for i in range(n2d + n3d):
        dim = 2 if i < n2d else 3
        lo, hi = (512, 8192) if dim == 2 else (64, 384)
        nx, ny = draw(lo, hi), draw(lo, hi)
        nz = draw(lo, hi) if dim == 3 else 1
        r = draw(1, 4)
        dt = "bf16" if draw(0, 1) else "f32"
        out.append(dict(dim=dim, r=r, nx=nx, ny=ny, nz=nz, dtype=dt))
    return out
