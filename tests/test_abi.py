"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every function include/stag.h declares, and rejects bad arguments with
error codes before touching the device."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stag.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \t\*]*?\b(stag_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_2502_03249_gb300 as stag
    return stag.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("stag_create", "stag_destroy", "stag_upload_gauge", "stag_dslash_eo", "stag_dslash_oe",
                     "stag_apply_M", "stag_cg_solve", "stag_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared in stag.h but not exported: {missing}"


def test_abi_version_and_strerror(lib):
    assert lib.stag_abi_version() == 3
    for code in (0, 1, 2, -1, -2, -3, -4, -5, -6):
        assert len(lib.stag_strerror(code)) > 0
    assert lib.stag_strerror(12345) == b"unknown status"


def test_create_rejects_bad_geometry_without_device(lib):
    h = ctypes.c_void_p()
    for dims in ((3, 4, 4, 4), (4, 4, 4, 0), (4, 4, 4, 5), (1, 2, 2, 2)):
        d = (ctypes.c_int * 4)(*dims)
        assert lib.stag_create(ctypes.byref(h), d, None) == -2
        assert h.value is None
    d = (ctypes.c_int * 4)(4, 4, 4, 4)
    assert lib.stag_create(None, d, None) == -1
    assert lib.stag_create(ctypes.byref(h), None, None) == -1
    big = (ctypes.c_int * 4)(2048, 2048, 1024, 2)
    assert lib.stag_create(ctypes.byref(h), big, None) == -2


def test_null_context_is_rejected(lib):
    assert lib.stag_destroy(None) == 0
    assert lib.stag_dslash_eo(None, None, None, 0, 18) == -1
    assert lib.stag_apply_M(None, None, None, ctypes.c_double(0.1)) == -1
    assert lib.stag_cg_solve(None, None, None, ctypes.c_double(0.1), None, None) == -1


def test_solver_param_defaults(lib):
    import paper_2502_03249_gb300 as stag
    p = stag.SolverParams()
    lib.stag_solver_params_default(ctypes.byref(p))
    assert p.tol == 1e-10 and p.maxiter == 100000 and p.use_graph == 1
    assert p.inner_prec == stag.F32 and p.inner_recon == 12 and p.delta == 0.01
    assert p.f64_arith == stag.F64X and p.temporal_gauge == 0


def test_noalloc_rejects_bad_geometry_without_device(lib):
    """The allocation-free operator checks extents and its static limit before
    any CUDA call."""
    import paper_2502_03249_gb300 as stag
    d = (ctypes.c_int * 4)(4, 4, 3, 4)
    assert lib.stag_apply_M_noalloc(d, None, None, None, 0.1, None) == -2
    d = (ctypes.c_int * 4)(64, 64, 64, 16)   # V/2 = 2^21
    assert lib.stag_apply_M_noalloc(d, None, None, None, 0.1, None) == -1
    assert b"static scratch limit" in lib.stag_last_error()
    assert lib.stag_apply_M_noalloc(None, None, None, None, 0.1, None) == -1
    # extents whose product overflows a 64-bit integer are refused, not wrapped
    huge = (ctypes.c_int * 4)(1 << 16, 1 << 16, 1 << 16, (1 << 15) + 2)
    assert lib.stag_apply_M_noalloc(huge, None, None, None, 0.1, None) == -1
    assert b"static scratch limit" in lib.stag_last_error()
    huge = (ctypes.c_int * 4)(2147483646, 2147483646, 2147483646, 2147483646)
    assert lib.stag_apply_M_noalloc(huge, None, None, None, 0.1, None) == -1
    assert stag.NOALLOC_MAX_VH == 1 << 17
    hdr = open(HEADER).read()
    assert "#define STAG_NOALLOC_MAX_VH (1 << 17)" in hdr
