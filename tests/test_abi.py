"""CPU checks of the C ABI: the library builds, loads without a GPU and
exports every entry point that include/kop.h declares."""
import os
import re

from paper_2609_08136_b300 import _ffi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kop.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("kop_create", "kop_matvec", "nys_build", "pcg_solve", "pcg_adjoint", "kop_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = _ffi.lib()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_ctypes_table_matches_header():
    assert set(_ffi.SIGNATURES) == set(_declared())


def test_invalid_arguments_rejected_without_gpu():
    import ctypes
    lib = _ffi.lib()
    h = ctypes.c_void_p()
    # NULL X, bad d, bad bandwidth: rejected before any CUDA call
    assert lib.kop_create(None, 10, 4, 0, 1.0, None, ctypes.byref(h)) == -1
    assert lib.kop_create(ctypes.c_void_p(16), 10, 0, 0, 1.0, None, ctypes.byref(h)) == -1
    assert lib.kop_create(ctypes.c_void_p(16), 10, 4, 0, -1.0, None, ctypes.byref(h)) == -1
    assert lib.kop_create(ctypes.c_void_p(16), 10, 4, 7, 1.0, None, ctypes.byref(h)) == -1
    assert b"kernel" in lib.kop_last_error()


def test_adaptive_build_rejects_bad_arguments_without_gpu():
    import ctypes
    lib = _ffi.lib()
    out = ctypes.c_void_p()
    r = ctypes.c_int32()
    e = ctypes.c_double()
    # NULL out, NULL operator: rejected before any CUDA call
    assert lib.nys_build_adaptive(None, None, 8, 4, 8, 10, 1e-2, None, 0.0, 0, None, None, None, None,
                                  None, None, 0) == -1
    assert lib.nys_build_adaptive(None, ctypes.c_void_p(16), 8, 4, 8, 10, 1e-2, ctypes.c_void_p(16), 0.0, 0,
                                  None, ctypes.byref(out), ctypes.byref(r), ctypes.byref(e), None, None, 0) == -1
    assert b"NULL" in lib.kop_last_error()


def test_ridge_and_gradient_entry_points_reject_bad_arguments_without_gpu():
    import ctypes
    lib = _ffi.lib()
    h = ctypes.c_void_p()
    assert lib.kop_create_ridge(None, 10, 4, None, ctypes.byref(h)) == -1
    assert lib.kop_create_ridge(ctypes.c_void_p(16), 0, 4, None, ctypes.byref(h)) == -1
    assert lib.kop_create_ridge(ctypes.c_void_p(16), 10, 0, None, ctypes.byref(h)) == -1
    assert lib.kop_grad_points(None, ctypes.c_void_p(16), ctypes.c_void_p(16), 0, ctypes.c_void_p(16), None) == -1
    assert b"NULL" in lib.kop_last_error()


def test_check_cache_rejects_null_handle_without_gpu():
    lib = _ffi.lib()
    assert lib.kop_set_check_cache(None, 1, None, 0) == -1
    assert b"NULL" in lib.kop_last_error()


def test_adjoint_val_and_admm_reject_bad_arguments_without_gpu():
    import ctypes
    lib = _ffi.lib()
    d = ctypes.c_double()
    assert lib.pcg_adjoint_val(None, None, 1.0, 1, None, None, 10, None, 1e-6, 10, 0, 0, 2, 2, None, None,
                               ctypes.byref(d), ctypes.byref(d), ctypes.byref(d), None) == -1
    assert b"NULL" in lib.kop_last_error()
    h = ctypes.c_void_p()
    assert lib.admm_create(None, None, 8, 1, 0.0, 1.0, 1e-8, 10, 0, 0, 0, 2, 2, None, ctypes.byref(h)) == -1
    assert lib.admm_solve(None, None, 1.0, None, None, None, None, None, None) == -1
    assert lib.admm_destroy(None) == 0
