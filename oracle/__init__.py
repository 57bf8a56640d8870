"""CPU oracle for repeated star-stencil sweeps -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the cpu_baseline / reference
legs of ``bench.py`` may import this package.  The product path
(``paper_2002_05983_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, compiled here with gcc):
``sweep_f64`` is Eq. 1 of the paper in double precision, ``sweep_f32`` the
same sweep as an fp32 multiply-then-FMA chain in the same operand order.
Both clamp out-of-bound neighbours to the border cell at every step.

Parity status: both functions are pinned by tests/test_oracle_pins.py
(dense-operator brute force, exact constant field, max principle, exact
shift stencils, exact-rational fp32 brute force, fp32-vs-fp64 bound, and
Table I/III arithmetic for the metric helpers).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
          "-fno-fast-math", "-fno-unsafe-math-optimizations"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64, i32 = ctypes.c_int64, ctypes.c_int
            vp = ctypes.c_void_p
            for name in ("oracle_sweep_f64", "oracle_sweep_f32", "oracle_sweep_shared_f64", "oracle_sweep_shared_f32"):
                fn = getattr(lib, name)
                fn.argtypes = [vp, vp, i64, i64, i64, i32, i32, vp, i32, i32]
                fn.restype = i32
            lib.oracle_max_threads.restype = i32
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _dims(grid: np.ndarray, dim: int):
    if grid.ndim != dim:
        raise ValueError(f"grid must have {dim} axes, got shape {grid.shape}")
    if dim == 2:
        ny, nx = grid.shape
        return nx, ny, 1
    nz, ny, nx = grid.shape
    return nx, ny, nz


def sweep_f64(grid, dim: int, radius: int, coeffs, iters: int, threads: int = 0) -> np.ndarray:
    """`iters` FP64 Jacobi steps of Eq. 1 (clamp to edge); returns a new float64 array."""
    lib = _load()
    f = np.ascontiguousarray(grid, dtype=np.float64)
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    if c.size != 2 * dim * radius + 1:
        raise ValueError("need 2*dim*radius+1 coefficients")
    out = np.empty_like(f)
    nx, ny, nz = _dims(f, dim)
    rc = lib.oracle_sweep_f64(f.ctypes.data, out.ctypes.data, nx, ny, nz, dim, radius,
                              c.ctypes.data, iters, threads)
    if rc:
        raise RuntimeError(f"oracle_sweep_f64 failed ({rc})")
    return out


def sweep_f32(grid, dim: int, radius: int, coeffs, iters: int, threads: int = 0) -> np.ndarray:
    """`iters` FP32 steps: centre multiply then one fmaf per neighbour in Eq. 1 order."""
    lib = _load()
    f = np.ascontiguousarray(grid, dtype=np.float32)
    c = np.ascontiguousarray(coeffs, dtype=np.float32)
    if c.size != 2 * dim * radius + 1:
        raise ValueError("need 2*dim*radius+1 coefficients")
    out = np.empty_like(f)
    nx, ny, nz = _dims(f, dim)
    rc = lib.oracle_sweep_f32(f.ctypes.data, out.ctypes.data, nx, ny, nz, dim, radius,
                              c.ctypes.data, iters, threads)
    if rc:
        raise RuntimeError(f"oracle_sweep_f32 failed ({rc})")
    return out


def _sweep(fn: str, grid, dim: int, radius: int, coeffs, iters: int, threads: int, dtype, k: int):
    lib = _load()
    f = np.ascontiguousarray(grid, dtype=dtype)
    c = np.ascontiguousarray(coeffs, dtype=dtype)
    if c.size != k:
        raise ValueError(f"need {k} coefficients")
    out = np.empty_like(f)
    nx, ny, nz = _dims(f, dim)
    rc = getattr(lib, fn)(f.ctypes.data, out.ctypes.data, nx, ny, nz, dim, radius, c.ctypes.data, iters, threads)
    if rc:
        raise RuntimeError(f"{fn} failed ({rc})")
    return out


def sweep_shared_f64(grid, dim: int, radius: int, coeffs, iters: int, threads: int = 0) -> np.ndarray:
    """`iters` FP64 steps of the shared-coefficient form (c[0..r], one per distance)."""
    return _sweep("oracle_sweep_shared_f64", grid, dim, radius, coeffs, iters, threads, np.float64, radius + 1)


def sweep_shared_f32(grid, dim: int, radius: int, coeffs, iters: int, threads: int = 0) -> np.ndarray:
    """FP32 shared-coefficient steps: left-to-right neighbour sum, one fmaf per distance."""
    return _sweep("oracle_sweep_shared_f32", grid, dim, radius, coeffs, iters, threads, np.float32, radius + 1)
