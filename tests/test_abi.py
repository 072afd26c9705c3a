"""The C ABI library builds, loads without a GPU and exports every function the header
declares; host-only calls behave (CPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "azint.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(az_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1412_6367_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("az_geometry_create", "az_csr_build", "az_integrate1d", "az_integrate2d",
                 "az_integrate_backward", "az_integrate_batch", "az_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_covers_the_header():
    from paper_1412_6367_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_host_only_calls():
    import oracle as O
    from paper_1412_6367_gb300 import api
    g = api.Geometry(0.2, 1e-3, 2e-3, 0.1, -0.2, 0.3)
    assert np.allclose(g.rotation(), O.rotation(0.1, -0.2, 0.3), atol=1e-15, rtol=0)
    with pytest.raises(api.AzError) as e:
        api.Geometry(0.1, 0, 0, wavelength=0.0)
    assert e.value.code == -1
    from paper_1412_6367_gb300 import _lib
    L = _lib.load()
    assert L.az_integrate1d(None, None, 0, None, None, None, None, 1, None, None, None, None, None) == -1
    assert b"NULL" in L.az_last_error()


def test_host_only_lut_calls():
    """The look-up-table entry points refuse NULL handles (and bad arguments) before touching
    a device."""
    from paper_1412_6367_gb300 import _lib
    L = _lib.load()
    assert L.az_lut_build(None, 1, None) == -1
    assert L.az_lut_export(None, None, None, None, None) == -1
    assert L.az_integrate_lut(None, None, 0, None, None, None, None, 1, None, None, None, None, None) == -1
    assert L.az_set_layout(None, 1) == -1
    assert b"az_set_layout" in L.az_last_error()


def test_selftest_wait_rejects_bad_arguments_on_host():
    """The bounded-wait self-test checks its arguments before any launch."""
    import ctypes as C
    from paper_1412_6367_gb300 import _lib
    L = _lib.load()
    st = C.c_int(5)
    assert L.az_selftest_wait(0, 1000, None, None) == -1
    assert L.az_selftest_wait(0, 0, C.byref(st), None) == -1
    assert L.az_selftest_wait(0, 3_000_000_000, C.byref(st), None) == -1
    assert st.value == 5


def test_csr_import_checks_the_matrix_on_host():
    """az_csr_import refuses malformed matrices before any device work."""
    import ctypes as C
    from paper_1412_6367_gb300 import _lib
    L = _lib.load()

    def call(indptr, indices, data, ny=2, nx=3, npt=2, lo=0.0, hi=1.0):
        ip = np.ascontiguousarray(indptr, dtype=np.int32)
        ix = np.ascontiguousarray(indices, dtype=np.int32)
        dv = np.ascontiguousarray(data, dtype=np.float64)
        h = C.c_void_p()
        return L.az_csr_import(ny, nx, npt, 0, 0, 2, C.c_void_p(ip.ctypes.data), C.c_void_p(ix.ctypes.data),
                               C.c_void_p(dv.ctypes.data), lo, hi, None, C.byref(h))

    good = ([0, 2, 3], [0, 4, 5], [0.5, 0.5, 1.0])
    assert call([1, 2, 3], good[1], good[2]) == -1           # indptr[0] != 0
    assert call([0, 3, 2], good[1], good[2]) == -1           # decreasing indptr
    assert call(good[0], [0, 6, 5], good[2]) == -1           # pixel outside the detector
    assert call(good[0], [4, 0, 5], good[2]) == -1           # not ascending within a row
    assert call(good[0], [0, 0, 5], good[2]) == -1           # duplicate pixel in a row
    assert call(good[0], good[1], [0.5, np.nan, 1.0]) == -1  # non-finite weight
    assert call(good[0], good[1], good[2], lo=1.0, hi=1.0) == -1  # empty radial range
    assert call([0, 0, 0], [0], [1.0]) == -8                 # no entries (AZ_ERANGE)
    assert call(good[0], good[1], good[2], ny=0) == -2       # bad shape
    assert b"az_csr_import" in L.az_last_error() or b"csr_build" in L.az_last_error()


def test_bound_corrections_reject_bad_arguments_on_host():
    """az_set_corrections and az_integrate_batch_bound refuse a NULL integrator and a
    negative frame count before touching a device."""
    from paper_1412_6367_gb300 import _lib
    L = _lib.load()
    assert L.az_set_corrections(None, None, None, None, None, None) == -1
    assert b"az_set_corrections" in L.az_last_error()
    assert L.az_integrate_batch_bound(None, None, 0, 1, None, None, None, None, None) == -1
    assert L.az_integrate_batch_bound(None, None, -1, 1, None, None, None, None, None) == -2

