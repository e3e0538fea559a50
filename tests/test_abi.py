"""The C-ABI library loads, exports every entry point include/*.h declares, and rejects
bad arguments before touching a device (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2502_17683_gb300 import _lib
    return _lib.load()


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(thc_cpd_\w+)\s*\(", txt))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("thc_cpd_mttkrp", "thc_cpd_loss", "thc_cpd_als_sweep", "thc_cpd_als"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2502_17683_gb300 import _lib
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(_lib.EXPORTS) == set(declared_symbols())


def test_version(lib):
    assert b"sm_103a" in lib.thc_cpd_version()


def _call_mttkrp(lib, o, v, Rt, R, mode, ptr=1, Aptrs=(1, 1, 1, 1), M=1, prec=0, ldl=0):
    from paper_2502_17683_gb300._lib import PTR4, Opts
    opts = Opts()
    opts.precision = prec
    opts.ldl = ldl
    return lib.thc_cpd_mttkrp(o, v, Rt, R, ptr, ptr, ptr, PTR4(*Aptrs), mode, M, ctypes.byref(opts))


def test_argument_validation_happens_before_device_work(lib):
    from paper_2502_17683_gb300 import _lib
    # invalid shapes / modes / null pointers / precision are reported without any CUDA call
    assert _call_mttkrp(lib, 0, 5, 5, 5, 0) == _lib.ERR_SHAPE
    assert _call_mttkrp(lib, 5, 5, -1, 5, 0) == _lib.ERR_SHAPE
    assert _call_mttkrp(lib, 5, 5, 5, 1 << 20, 0) == _lib.ERR_SHAPE
    assert _call_mttkrp(lib, 5, 5, 5, 5, 4) == _lib.ERR_ARG
    assert _call_mttkrp(lib, 5, 5, 5, 5, 0, ptr=None) == _lib.ERR_ARG
    assert _call_mttkrp(lib, 5, 5, 5, 5, 0, Aptrs=(1, None, 1, 1)) == _lib.ERR_ARG
    assert _call_mttkrp(lib, 5, 5, 5, 5, 0, M=None) == _lib.ERR_ARG
    assert _call_mttkrp(lib, 5, 5, 5, 5, 0, prec=9) == _lib.ERR_ARG
    assert b"mode" in lib.thc_cpd_last_error() or b"precision" in lib.thc_cpd_last_error()
    assert _call_mttkrp(lib, 5, 5, 5, 5, 0, ldl=4) == _lib.ERR_ARG
    assert b"ldl" in lib.thc_cpd_last_error()
    out = ctypes.c_double()
    assert lib.thc_cpd_thc_norm2(3, 4, 5, None, 1, 1, ctypes.byref(out), None) == _lib.ERR_ARG
    assert lib.thc_cpd_thc_norm2(3, 4, 5, 1, 1, 1, None, None) == _lib.ERR_ARG


def test_ldl_solve_checks_its_arguments_before_device_work(lib):
    import numpy as np
    from paper_2502_17683_gb300 import _lib
    sp = ctypes.POINTER(ctypes.c_short)
    f = lib.thc_cpd_ldl_solve
    assert f(0, 5, 1, 1, 1, None, 0, None, None) == _lib.ERR_SHAPE
    assert f(4096, 5, 1, 1, 1, None, 0, None, None) == _lib.ERR_SHAPE
    assert f(64, 0, 1, 1, 1, None, 0, None, None) == _lib.ERR_SHAPE
    assert f(64, 5, None, 1, 1, None, 0, None, None) == _lib.ERR_ARG
    # a task list with an out-of-range tile index (R = 64: 4 column tiles, n = 5: 1 row tile)
    bad = np.array([[1, 2, 1, 0], [1, 3, 2, 7]], dtype=np.int16)
    assert f(64, 5, 1, 1, 1, bad.ctypes.data_as(sp), 2, None, None) == _lib.ERR_ARG
    assert b"task 1" in lib.thc_cpd_last_error()
    bad = np.array([[2, 2, 1, 0]], dtype=np.int16)  # unknown task type
    assert f(64, 5, 1, 1, 1, bad.ctypes.data_as(sp), 1, None, None) == _lib.ERR_ARG


def test_no_cpu_fallback_when_library_missing(tmp_path):
    from paper_2502_17683_gb300 import _lib
    with pytest.raises(_lib.ThcCpdError):
        saved = _lib._lib
        _lib._lib = None
        try:
            _lib.load(str(tmp_path / "missing.so"))
        finally:
            _lib._lib = saved


def test_rows_beyond_the_hot_path_check_their_arguments_before_device_work(lib):
    from paper_2502_17683_gb300 import _lib
    from paper_2502_17683_gb300._lib import PTR4, Opts
    # core fit: shapes, R_thc limit, null pointers
    f = lib.thc_cpd_core_fit
    assert f(0, 3, 4, 5, 1, 1, 1, 1, None, None, None) == _lib.ERR_SHAPE
    assert f(2, 3, 2049, 5, 1, 1, 1, 1, None, None, None) == _lib.ERR_SHAPE
    assert f(2, 3, 4, 5, 1, None, 1, 1, None, None, None) == _lib.ERR_ARG
    assert f(2, 3, 4, 5, 1, 1, 1, None, None, None, None) == _lib.ERR_ARG
    # DF-driven ALS: shapes, null factors, split precision refused, sweeps
    g = lib.thc_cpd_df_als
    A = PTR4(1, 1, 1, 1)
    assert g(2, 3, 4, 0, 1, A, 1, 1, 0.0, None, None, None) == _lib.ERR_SHAPE
    assert g(2, 3, 4, 2049, 1, A, 1, 1, 0.0, None, None, None) == _lib.ERR_SHAPE
    assert g(2, 3, 4, 5, 1, PTR4(1, None, 1, 1), 1, 1, 0.0, None, None, None) == _lib.ERR_ARG
    assert g(2, 3, 4, 5, 1, A, 1, 0, 0.0, None, None, None) == _lib.ERR_ARG
    opts = Opts()
    opts.precision = 1
    assert g(2, 3, 4, 5, 1, A, 1, 1, 0.0, None, None, ctypes.byref(opts)) == _lib.ERR_ARG
    assert b"FP64" in lib.thc_cpd_last_error()
    # order d: d and dL ranges, mode range, mode sizes
    dims = (ctypes.c_int * 3)(3, 4, 5)
    ptrs = (ctypes.c_void_p * 3)(1, 1, 1)
    h = lib.thc_cpd_nd_mttkrp
    assert h(3, 3, dims, 6, 2, ptrs, 1, ptrs, 0, 1, None) == _lib.ERR_SHAPE  # dL = d
    assert h(9, 1, dims, 6, 2, ptrs, 1, ptrs, 0, 1, None) == _lib.ERR_SHAPE  # d > 8
    assert h(3, 1, dims, 6, 2, ptrs, 1, ptrs, 3, 1, None) == _lib.ERR_ARG    # mode = d
    bad = (ctypes.c_int * 3)(3, 0, 5)
    assert h(3, 1, bad, 6, 2, ptrs, 1, ptrs, 0, 1, None) == _lib.ERR_SHAPE
    assert lib.thc_cpd_nd_als(3, 1, dims, 6, 2, ptrs, 1, ptrs, None, 1, 0.0, None, None, None) == _lib.ERR_ARG
    # exchange energy: quadrature size, null quadrature factors
    e = lib.thc_cpd_exchange
    d1 = ctypes.c_double()
    assert e(2, 3, 4, 5, 0, 1, 1, 1, A, 1, 1, 1, ctypes.byref(d1), None, None, None) == _lib.ERR_SHAPE
    assert e(2, 3, 4, 5, 2, 1, 1, 1, A, 1, None, 1, ctypes.byref(d1), None, None, None) == _lib.ERR_ARG
