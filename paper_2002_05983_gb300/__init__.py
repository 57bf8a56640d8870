"""GB300-native repeated star-stencil sweeps (2D/3D, radius 1..6, per-direction or shared coefficients, clamp to edge).

A thin ctypes binding over libstencil.so (the C ABI declared in
include/stencil.h).  The functions below carry the C names and only marshal
arguments; every step of a sweep runs in the library's CUDA kernels.  PyTorch
is used for device memory and streams only.  If the library has not been
built, every call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libstencil.so")

STENCIL_OK = 0
STENCIL_ERR_INVALID_ARG = -1
STENCIL_ERR_ALIAS = -2
STENCIL_ERR_UNSUPPORTED = -3
STENCIL_ERR_OOM = -4
STENCIL_ERR_CUDA = -5
STENCIL_ERR_TIMEOUT = -6
STENCIL_ERR_NO_DEVICE = -7
STENCIL_ERR_BOUNDS = -8

STENCIL_F32, STENCIL_BF16, STENCIL_F16 = 0, 1, 2
KERNEL_AUTO, KERNEL_STREAM, KERNEL_NAIVE = 0, 1, 2

# every symbol include/stencil.h declares
EXPORTS = ("stencil_create", "stencil_create_shared", "stencil_destroy", "stencil_run", "stencil_run_ex", "stencil_run_host",
           "stencil_default_schedule", "stencil_max_t", "stencil_get_device_status",
           "stencil_set_fault_injection", "stencil_set_checked", "stencil_run_noalloc", "stencil_run_batched", "stencil_tune",
           "stencil_resolve_schedule", "stencil_schedule_features", "stencil_model_create", "stencil_model_destroy",
           "stencil_model_train", "stencil_model_predict", "stencil_model_normalization",
           "stencil_model_params", "stencil_model_grad", "stencil_use_cost_model", "stencil_measure_peaks", "stencil_last_cuda_error",
           "stencil_strerror")

NFEAT = 18
TUNE_ANALYTIC, TUNE_EXHAUSTIVE, TUNE_MODEL = 0, 1, 2


class StencilError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})"
                         + (f", cuda error {_lib().stencil_last_cuda_error()}" if code == STENCIL_ERR_CUDA else ""))


class Schedule(ctypes.Structure):
    """stencil_schedule: 0 in any field = chosen by the library."""
    _fields_ = [("kernel", ctypes.c_int), ("t", ctypes.c_int), ("threads_x", ctypes.c_int),
                ("threads_y", ctypes.c_int), ("rows_per_thread", ctypes.c_int), ("seg", ctypes.c_int),
                ("prefetch", ctypes.c_int), ("planes_per_step", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchItem(ctypes.Structure):
    """stencil_batch_item."""
    _fields_ = [("h", ctypes.c_void_p), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("nx", ctypes.c_int64),
                ("ny", ctypes.c_int64), ("nz", ctypes.c_int64), ("iters", ctypes.c_int), ("dtype", ctypes.c_int)]


class Peaks(ctypes.Structure):
    """stencil_peaks: measured FP32 FMA throughput and copy bandwidth of the device."""
    _fields_ = [("fp32_flops", ctypes.c_double), ("copy_bytes_per_s", ctypes.c_double), ("sms", ctypes.c_int),
                ("sm_clock_khz", ctypes.c_int)]


class Timing(ctypes.Structure):
    """stencil_timing: one candidate schedule with its features and times."""
    _fields_ = [("sched", Schedule), ("features", ctypes.c_float * NFEAT), ("ns_per_cell", ctypes.c_float),
                ("analytic_ns_per_cell", ctypes.c_float), ("model_ns_per_cell", ctypes.c_float)]


_lock = threading.Lock()
_L = None


def _lib():
    global _L
    if _L is None:
        with _lock:
            if _L is None:
                if not os.path.exists(LIB_PATH):
                    raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                       "`python -c 'import __graft_entry__ as g; g.build()'`")
                lib = ctypes.CDLL(LIB_PATH)
                vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
                sp = ctypes.POINTER(Schedule)
                lib.stencil_create.argtypes = [ctypes.POINTER(vp), i32, i32, ctypes.POINTER(ctypes.c_float)]
                lib.stencil_destroy.argtypes = [vp]
                lib.stencil_run.argtypes = [vp, vp, vp, i64, i64, i64, i32, i32, vp]
                lib.stencil_run_ex.argtypes = [vp, vp, vp, i64, i64, i64, i32, i32, vp, sp]
                lib.stencil_run_host.argtypes = [vp, vp, vp, i64, i64, i64, i32, i32, vp, sp]
                lib.stencil_default_schedule.argtypes = [vp, i64, i64, i64, i32, sp]
                lib.stencil_max_t.argtypes = [i32, i32, i32, i32]
                lib.stencil_get_device_status.argtypes = [vp, i32]
                lib.stencil_set_fault_injection.argtypes = [vp, i32, i32]
                lib.stencil_set_checked.argtypes = [vp, i32]
                lib.stencil_run_noalloc.argtypes = [vp, vp, vp, i64, i64, i64, i32, i32, vp]
                lib.stencil_run_batched.argtypes = [ctypes.POINTER(BatchItem), i32, vp]
                fp = ctypes.POINTER(ctypes.c_float)
                lib.stencil_tune.argtypes = [vp, i64, i64, i64, i32, i32, vp, i32, sp,
                                             ctypes.POINTER(Timing), i32, ctypes.POINTER(i32)]
                lib.stencil_schedule_features.argtypes = [vp, i64, i64, i64, i32, sp, fp]
                lib.stencil_resolve_schedule.argtypes = [vp, i64, i64, i64, i32, sp, sp]
                lib.stencil_model_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32]
                lib.stencil_model_destroy.argtypes = [vp]
                lib.stencil_model_train.argtypes = [vp, fp, fp, i32, i32, ctypes.c_float, fp]
                lib.stencil_model_predict.argtypes = [vp, fp, fp, i32]
                lib.stencil_model_normalization.argtypes = [vp, fp, fp, ctypes.c_float, ctypes.c_float]
                lib.stencil_model_params.argtypes = [vp, fp, i32, i32]
                lib.stencil_model_grad.argtypes = [vp, fp, fp, i32, fp, fp]
                lib.stencil_measure_peaks.argtypes = [vp, ctypes.POINTER(Peaks)]
                lib.stencil_use_cost_model.argtypes = [vp]
                lib.stencil_last_cuda_error.argtypes = []
                lib.stencil_strerror.argtypes = [i32]
                lib.stencil_strerror.restype = ctypes.c_char_p
                for name in EXPORTS:
                    if name != "stencil_strerror":
                        getattr(lib, name).restype = i32
                _L = lib
    return _L


def library():
    """The loaded ctypes library (raises if it was not built)."""
    return _lib()


def strerror(code: int) -> str:
    return _lib().stencil_strerror(code).decode()


def _check(rc: int, what: str) -> int:
    if rc != STENCIL_OK:
        raise StencilError(rc, what)
    return rc


# ------------------------------------------------------------ C-named calls
def _create(fn: str, dim: int, radius: int, coeffs, k: int) -> int:
    import numpy as np
    c = np.ascontiguousarray(coeffs, dtype=np.float32).reshape(-1)
    if c.size < max(k, 1):   # the library reads k floats
        raise ValueError(f"{fn}: need {k} coefficients, got {c.size}")
    h = ctypes.c_void_p()
    _check(getattr(_lib(), fn)(ctypes.byref(h), dim, radius, c.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), fn)
    return h.value


def stencil_create(dim: int, radius: int, coeffs) -> int:
    """K = 2*dim*radius + 1 coefficients, one per (distance, direction)."""
    ok = dim in (2, 3) and 1 <= radius <= 6
    return _create("stencil_create", dim, radius, coeffs, 2 * dim * radius + 1 if ok else 0)


def stencil_create_shared(dim: int, radius: int, coeffs) -> int:
    """K = radius + 1 coefficients, one per distance."""
    ok = dim in (2, 3) and 1 <= radius <= 6
    return _create("stencil_create_shared", dim, radius, coeffs, radius + 1 if ok else 0)


def stencil_destroy(h: int) -> int:
    return _check(_lib().stencil_destroy(h), "stencil_destroy")


def stencil_run(h, in_ptr, out_ptr, nx, ny, nz, iters, dtype, stream) -> int:
    return _check(_lib().stencil_run(h, in_ptr, out_ptr, nx, ny, nz, iters, dtype, stream), "stencil_run")


def stencil_run_ex(h, in_ptr, out_ptr, nx, ny, nz, iters, dtype, stream, sched: Schedule | None) -> int:
    return _check(_lib().stencil_run_ex(h, in_ptr, out_ptr, nx, ny, nz, iters, dtype, stream,
                                        ctypes.byref(sched) if sched is not None else None), "stencil_run_ex")


def stencil_run_host(h, in_ptr, out_ptr, nx, ny, nz, iters, dtype, stream, sched: Schedule | None) -> int:
    return _check(_lib().stencil_run_host(h, in_ptr, out_ptr, nx, ny, nz, iters, dtype, stream,
                                          ctypes.byref(sched) if sched is not None else None),
                  "stencil_run_host")


def stencil_default_schedule(h, nx, ny, nz, dtype) -> Schedule:
    s = Schedule()
    _check(_lib().stencil_default_schedule(h, nx, ny, nz, dtype, ctypes.byref(s)), "stencil_default_schedule")
    return s


def stencil_max_t(dim, radius, dtype, rows_per_thread=2) -> int:
    return int(_lib().stencil_max_t(dim, radius, dtype, rows_per_thread))


def stencil_get_device_status(stream=None, clear: bool = False) -> int:
    """Raw status code (0 or STENCIL_ERR_TIMEOUT); does not raise on TIMEOUT."""
    return int(_lib().stencil_get_device_status(stream, 1 if clear else 0))


def stencil_set_checked(h, on: bool = True) -> int:
    """Use the bounds-checked kernel instantiations on this handle (see stencil.h)."""
    return _check(_lib().stencil_set_checked(h, 1 if on else 0), "stencil_set_checked")


def stencil_set_fault_injection(h, plane: int, timeout_ms: int = 50) -> int:
    return _check(_lib().stencil_set_fault_injection(h, plane, timeout_ms), "stencil_set_fault_injection")


def stencil_run_noalloc(h, in_ptr, out_ptr, nx, ny, nz, iters, dtype, stream) -> int:
    """stencil_run without device allocation (grids up to 16 MiB); see include/stencil.h."""
    return _check(_lib().stencil_run_noalloc(h, in_ptr, out_ptr, nx, ny, nz, iters, dtype, stream),
                  "stencil_run_noalloc")


def stencil_run_batched(items, stream) -> int:
    """items: sequence of BatchItem (or tuples h, in_ptr, out_ptr, nx, ny, nz, iters, dtype)."""
    arr = (BatchItem * len(items))(*[it if isinstance(it, BatchItem) else BatchItem(*it) for it in items])
    return _check(_lib().stencil_run_batched(arr, len(items), stream), "stencil_run_batched")


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def stencil_tune(h, nx, ny, nz, dtype, mode, model=None, store=True, cap=256):
    """Returns (chosen Schedule, list of Timing rows)."""
    chosen = Schedule()
    rows = (Timing * cap)()
    n = ctypes.c_int(0)
    _check(_lib().stencil_tune(h, nx, ny, nz, dtype, mode, model, 1 if store else 0, ctypes.byref(chosen),
                               rows, cap, ctypes.byref(n)), "stencil_tune")
    return chosen, [rows[i] for i in range(min(n.value, cap))]


def stencil_resolve_schedule(h, nx, ny, nz, dtype, sched: Schedule | None = None) -> Schedule:
    """The schedule a pass would run with (block shape, segment, prefetch, rows per step)."""
    out = Schedule()
    _check(_lib().stencil_resolve_schedule(h, nx, ny, nz, dtype, ctypes.byref(sched) if sched is not None else None,
                                           ctypes.byref(out)), "stencil_resolve_schedule")
    return out


def stencil_schedule_features(h, nx, ny, nz, dtype, sched: Schedule | None = None):
    import numpy as np
    f = np.zeros(NFEAT, np.float32)
    _check(_lib().stencil_schedule_features(h, nx, ny, nz, dtype,
                                            ctypes.byref(sched) if sched is not None else None, _fptr(f)),
           "stencil_schedule_features")
    return f


def stencil_model_create(n_features=NFEAT, hidden=64, seed=0) -> int:
    m = ctypes.c_void_p()
    _check(_lib().stencil_model_create(ctypes.byref(m), n_features, hidden, seed), "stencil_model_create")
    return m.value


def stencil_model_destroy(m) -> int:
    return _check(_lib().stencil_model_destroy(m), "stencil_model_destroy")


def stencil_model_train(m, X, y, epochs=2000, lr=3e-3) -> float:
    import numpy as np
    X = np.ascontiguousarray(X, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    loss = np.zeros(1, np.float32)
    _check(_lib().stencil_model_train(m, _fptr(X), _fptr(y), len(y), epochs, lr, _fptr(loss)),
           "stencil_model_train")
    return float(loss[0])


def stencil_model_predict(m, X):
    import numpy as np
    X = np.ascontiguousarray(X, np.float32)
    y = np.zeros(X.shape[0], np.float32)
    _check(_lib().stencil_model_predict(m, _fptr(X), _fptr(y), X.shape[0]), "stencil_model_predict")
    return y


def stencil_model_normalization(m, fmean, fstd, ymean, ystd) -> int:
    import numpy as np
    a = np.ascontiguousarray(fmean, np.float32)
    b = np.ascontiguousarray(fstd, np.float32)
    return _check(_lib().stencil_model_normalization(m, _fptr(a), _fptr(b), ymean, ystd),
                  "stencil_model_normalization")


def stencil_model_params(m, values=None):
    """Get (values None) or set the flat parameter vector."""
    import numpy as np
    n = _lib().stencil_model_params(m, _fptr(np.zeros(1, np.float32)), -1, 0)
    if values is None:
        p = np.zeros(n, np.float32)
        _check(_lib().stencil_model_params(m, _fptr(p), n, 0), "stencil_model_params")
        return p
    p = np.ascontiguousarray(values, np.float32)
    return _check(_lib().stencil_model_params(m, _fptr(p), p.size, 1), "stencil_model_params")


def stencil_model_grad(m, X, y):
    import numpy as np
    X = np.ascontiguousarray(X, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    n = _lib().stencil_model_params(m, _fptr(np.zeros(1, np.float32)), -1, 0)
    g = np.zeros(n, np.float32)
    loss = np.zeros(1, np.float32)
    _check(_lib().stencil_model_grad(m, _fptr(X), _fptr(y), len(y), _fptr(loss), _fptr(g)), "stencil_model_grad")
    return float(loss[0]), g


def stencil_use_cost_model(m) -> int:
    """Let model `m` (None: the built-in rule) propose the default schedules."""
    return _check(_lib().stencil_use_cost_model(m), "stencil_use_cost_model")


def stencil_measure_peaks(stream=None) -> Peaks:
    """Measured FP32 FMA throughput (FLOP/s) and copy bandwidth (bytes/s) of the current device."""
    p = Peaks()
    _check(_lib().stencil_measure_peaks(stream, ctypes.byref(p)), "stencil_measure_peaks")
    return p


def stencil_last_cuda_error() -> int:
    return int(_lib().stencil_last_cuda_error())


def stencil_strerror(code: int) -> str:
    return strerror(code)


# --------------------------------------------------------- torch convenience
_DT = {"float32": STENCIL_F32, "bfloat16": STENCIL_BF16, "float16": STENCIL_F16}


def dtype_code(t) -> int:
    return _DT[str(t.dtype).replace("torch.", "")]


def schedule(**kw) -> Schedule:
    s = Schedule()
    for k, v in kw.items():
        setattr(s, k, int(v))
    return s


def _dims(x, dim):
    if x.dim() != dim:
        raise ValueError(f"expected a {dim}-D tensor, got shape {tuple(x.shape)}")
    if dim == 2:
        ny, nx = x.shape
        return nx, ny, 1
    nz, ny, nx = x.shape
    return nx, ny, nz


class Stencil:
    """A star stencil (dim, radius, K coefficients) bound to a library handle;
    shared=True: one coefficient per distance (K = radius + 1)."""

    def __init__(self, dim: int, radius: int, coeffs, shared: bool = False):
        self.dim, self.radius, self.shared = dim, radius, shared
        self.handle = (stencil_create_shared if shared else stencil_create)(dim, radius, coeffs)

    def close(self):
        if self.handle:
            stencil_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, x, iters: int, out=None, sched: Schedule | None = None, stream=None):
        """`iters` sweeps of CUDA tensor x (shape (ny,nx) or (nz,ny,nx), fp32/bf16/fp16)."""
        import torch
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous CUDA tensor")
        if out is None:
            out = torch.empty_like(x)
        if out.shape != x.shape or out.dtype != x.dtype or not out.is_contiguous():
            raise ValueError("out must match x")
        nx, ny, nz = _dims(x, self.dim)
        st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        stencil_run_ex(self.handle, x.data_ptr(), out.data_ptr(), nx, ny, nz, iters, dtype_code(x), st, sched)
        return out

    def run_host(self, x_host, out_host, iters: int, sched: Schedule | None = None, stream=None):
        """End-to-end: host (ideally pinned) CPU tensors in and out, copies included."""
        import torch
        nx, ny, nz = _dims(x_host, self.dim)
        st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        stencil_run_host(self.handle, x_host.data_ptr(), out_host.data_ptr(), nx, ny, nz, iters,
                         dtype_code(x_host), st, sched)
        return out_host

    def default_schedule(self, shape, dtype=STENCIL_F32) -> Schedule:
        nx, ny, nz = (shape[1], shape[0], 1) if self.dim == 2 else (shape[2], shape[1], shape[0])
        return stencil_default_schedule(self.handle, nx, ny, nz, dtype)
