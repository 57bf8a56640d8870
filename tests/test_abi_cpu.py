"""CPU-side checks of the C ABI: the library loads without a GPU, exports every
symbol include/stencil.h declares, and validates arguments on the host."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2002_05983_gb300 as st

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "stencil.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stencil_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(st.LIB_PATH):
        pytest.fail("libstencil.so not built (run __graft_entry__.build())")
    return st.library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(st.EXPORTS) == names
    # the Python binding offers every entry point under the same name
    assert [n for n in names if not callable(getattr(st, n, None))] == []


def test_strerror_and_codes(lib):
    assert st.strerror(0) == "ok"
    assert "overlap" in st.strerror(st.STENCIL_ERR_ALIAS)
    assert st.strerror(-99) == "unknown status"


def test_create_validates_on_host(lib):
    c = np.ones(5, np.float32)
    for dim, r in ((1, 1), (4, 1), (2, 0), (2, 7), (3, 7)):
        with pytest.raises(st.StencilError) as e:
            st.stencil_create(dim, r, c)
        assert e.value.code == st.STENCIL_ERR_INVALID_ARG
    h = st.stencil_create(2, 1, c)
    assert st.stencil_destroy(h) == 0
    # one coefficient per distance: K = r + 1
    for dim, r in ((1, 1), (2, 0), (3, 7)):
        with pytest.raises(st.StencilError) as e:
            st.stencil_create_shared(dim, r, c)
        assert e.value.code == st.STENCIL_ERR_INVALID_ARG
    h = st.stencil_create_shared(3, 4, c)
    assert st.stencil_destroy(h) == 0
    with pytest.raises(ValueError):   # fewer coefficients than the library would read
        st.stencil_create(2, 4, c)


def test_run_rejects_bad_problems_before_touching_cuda(lib):
    h = st.stencil_create(3, 2, np.ones(13, np.float32))
    try:
        bad = [  # (in, out, nx, ny, nz, iters, dtype) -> expected code
            ((0, 64, 4, 4, 4, 1, 0), st.STENCIL_ERR_INVALID_ARG),
            ((64, 128, 0, 4, 4, 1, 0), st.STENCIL_ERR_INVALID_ARG),
            ((64, 128, 4, 4, 4, -1, 0), st.STENCIL_ERR_INVALID_ARG),
            ((64, 128, 4, 4, 4, 1, 7), st.STENCIL_ERR_INVALID_ARG),
            ((4096, 4096 + 64, 4, 4, 4, 1, 0), st.STENCIL_ERR_ALIAS),     # 256 B grids overlap
        ]
        for args, want in bad:
            assert lib.stencil_run(h, *args, None) == want
        h2 = st.stencil_create(2, 1, np.ones(5, np.float32))
        assert lib.stencil_run(h2, 64, 1 << 20, 8, 8, 2, 1, 0, None) == st.STENCIL_ERR_INVALID_ARG  # 2D, nz=2
        st.stencil_destroy(h2)
    finally:
        st.stencil_destroy(h)


def test_fault_injection_arguments(lib):
    h = st.stencil_create(2, 1, np.ones(5, np.float32))
    assert lib.stencil_set_fault_injection(h, 3, 0) == st.STENCIL_ERR_INVALID_ARG
    assert lib.stencil_set_fault_injection(h, 3, 20000) == st.STENCIL_ERR_INVALID_ARG
    assert lib.stencil_set_fault_injection(h, 3, 50) == 0
    assert lib.stencil_set_fault_injection(h, -1, 0) == 0
    st.stencil_destroy(h)


def test_compiled_temporal_degrees(lib):
    # 2D: radius 1 sweeps t = 1..16; larger radii up to the register-queue limit
    assert st.stencil_max_t(2, 1, 0) == 16
    assert [st.stencil_max_t(2, r, 0) for r in (2, 3, 4)] == [8, 6, 4]
    assert [st.stencil_max_t(3, r, 0, 2) for r in (1, 2, 3, 4)] == [6, 4, 2, 2]
    # radius 5 and 6 (beyond the paper's 1..4): 2D t = 1..3, 3D t = 1 with 2 or 4 rows
    assert [st.stencil_max_t(2, r, dt) for r in (5, 6) for dt in (0, 1, 2)] == [3] * 6
    assert [st.stencil_max_t(3, r, 0, vy) for r in (5, 6) for vy in (2, 4)] == [1] * 4
    for dt in (1, 2):
        assert st.stencil_max_t(2, 1, dt) == 16


def test_default_schedule_is_host_only(lib):
    h = st.stencil_create(2, 4, np.ones(17, np.float32))
    s = st.stencil_default_schedule(h, 16384, 16384, 1, 0)
    assert s.kernel == st.KERNEL_STREAM and 1 <= s.t <= 4 and s.threads_x > 0
    s = st.stencil_default_schedule(h, 1001, 64, 1, 0)      # rows not 16-byte aligned
    assert s.kernel == st.KERNEL_NAIVE
    st.stencil_destroy(h)
