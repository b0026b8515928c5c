"""ctypes declarations of the C ABI in include/kop.h (argument marshalling only).

The library is the in-tree libkop.so built by ``paper_2609_08136_b300.build``.
There is no fallback: if it is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkop.so")

c_int, c_i32, c_i64, c_dbl, c_vp = ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
P = ctypes.POINTER

# name: (restype, argtypes)
SIGNATURES = {
    "kop_last_error": (ctypes.c_char_p, []),
    "kop_launch_count": (c_i64, []),
    "kop_sfu_rates": (c_int, [P(c_dbl), c_vp]),
    "kop_set_autotune": (c_int, [c_i32]),
    "kop_autotune_shapes": (c_i32, []),
    "kop_create": (c_int, [c_vp, c_i64, c_i32, c_i32, c_dbl, c_vp, P(c_vp)]),
    "kop_destroy": (c_int, [c_vp]),
    "kop_set_bandwidth": (c_int, [c_vp, c_dbl]),
    "kop_set_check_cache": (c_int, [c_vp, c_i32, c_vp, c_i64]),
    "kop_matvec": (c_int, [c_vp, c_vp, c_i32, c_vp, c_i32, c_vp]),
    "kop_cross_matvec": (c_int, [c_vp, c_vp, c_i64, c_vp, c_i32, c_vp, c_i32, c_i32, c_i32, c_vp]),
    "kop_dbw_matvec": (c_int, [c_vp, c_vp, c_i32, c_vp, c_i32, c_vp]),
    "kop_matvec_f64": (c_int, [c_vp, c_vp, c_i32, c_vp, c_i32, c_vp]),
    "kop_sync": (c_int, [c_vp, c_vp]),
    "nys_build": (c_int, [c_vp, c_vp, c_i32, c_dbl, c_i32, c_vp, P(c_vp)]),
    "nys_destroy": (c_int, [c_vp]),
    "kop_create_ridge": (c_int, [c_vp, c_i64, c_i32, c_vp, P(c_vp)]),
    "kop_grad_points": (c_int, [c_vp, c_vp, c_vp, c_i32, c_vp, c_vp]),
    "nys_build_adaptive": (c_int, [c_vp, c_vp, c_i32, c_i32, c_i32, c_i32, c_dbl, c_vp, c_dbl, c_i32, c_vp,
                                   P(c_vp), P(c_i32), P(c_dbl), P(c_i32), P(c_dbl), c_i32]),
    "nys_apply": (c_int, [c_vp, P(c_dbl), c_i32, c_vp, c_i32, c_vp, c_vp]),
    "nys_apply_noalloc": (c_int, [c_vp, P(c_dbl), c_i32, c_vp, c_i32, c_vp, c_vp]),
    "nys_eigs": (c_int, [c_vp, P(c_dbl), P(c_dbl), P(c_i32)]),
    "nys_factor": (c_int, [c_vp, c_vp, c_vp]),
    "pcg_solve": (c_int, [c_vp, c_vp, P(c_dbl), c_i32, P(c_dbl), c_i32, c_vp, c_i32, c_vp, c_dbl, c_i32, c_i32,
                          c_i32, c_i32, c_i32, c_vp, P(c_i32), P(c_dbl), P(c_dbl), c_vp]),
    "pcg_adjoint": (c_int, [c_vp, c_vp, c_dbl, c_i32, c_vp, c_vp, c_dbl, c_i32, c_i32, c_i32, c_i32, c_i32, c_vp,
                            P(c_i32), P(c_dbl), P(c_dbl), c_vp]),
    "admm_create": (c_int, [c_vp, c_vp, c_i32, c_i32, c_dbl, c_dbl, c_dbl, c_i32, c_i32, c_i32, c_i32, c_i32, c_i32,
                            c_vp, P(c_vp)]),
    "admm_solve": (c_int, [c_vp, c_vp, c_dbl, c_vp, P(c_i32), P(c_dbl), P(c_dbl), P(c_i32), c_vp]),
    "admm_destroy": (c_int, [c_vp]),
    "pcg_adjoint_val": (c_int, [c_vp, c_vp, c_dbl, c_i32, c_vp, c_vp, c_i64, c_vp, c_dbl, c_i32, c_i32, c_i32, c_i32,
                                c_i32, c_vp, P(c_i32), P(c_dbl), P(c_dbl), P(c_dbl), c_vp]),
}

_lib = None


def lib():
    """Load libkop.so (once) and declare every entry point."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2609_08136_b300.build`")
        h = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(h, name, None)
            if f is None:
                continue
            f.restype = res
            f.argtypes = args
        _lib = h
    return _lib


def exported(name: str) -> bool:
    return hasattr(lib(), name)


class KopError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


STATUS = {0: "KOP_OK", 1: "KOP_NOT_CONVERGED", -1: "KOP_EINVAL", -2: "KOP_ENOMEM", -3: "KOP_ECUDA",
          -4: "KOP_ENOTPD", -5: "KOP_ETIMEOUT"}


def check(rc: int, where: str) -> int:
    if rc < 0:
        msg = lib().kop_last_error()
        raise KopError(rc, f"{where}: {STATUS.get(rc, rc)}: {msg.decode() if msg else ''}")
    return rc
