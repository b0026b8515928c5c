"""Build and load the FP64 OpenMP host matvec (kop_oracle_c.c).  Test
infrastructure only, like the rest of this package."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kop_oracle_c.c")
_LIB = os.path.join(_HERE, "libkop_oracle.so")
_handle = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"])
    return _LIB


def _lib():
    global _handle
    if _handle is None:
        _handle = ctypes.CDLL(build())
        f = _handle.oracle_kernel_matvec
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int,
                      ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                      ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
        _handle.oracle_max_threads.restype = ctypes.c_int
    return _handle


def max_threads() -> int:
    return int(_lib().oracle_max_threads())


def kernel_matvec(kind, X, V, bw, Z=None, deriv=False, nthreads=0):
    """O = K(Z, X) V (or dK/d bw V) in FP64 on the host cores."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    Z = X if Z is None else np.ascontiguousarray(Z, dtype=np.float32)
    V = np.asarray(V, dtype=np.float64)
    vec = V.ndim == 1
    V2 = np.ascontiguousarray(V[:, None] if vec else V)
    assert Z.shape[1] == X.shape[1] and V2.shape[0] == X.shape[0]
    O = np.empty((Z.shape[0], V2.shape[1]), dtype=np.float64)
    _lib().oracle_kernel_matvec(int(kind), float(bw), int(bool(deriv)),
                                Z.ctypes.data, Z.shape[0], X.ctypes.data, X.shape[0],
                                X.shape[1], V2.ctypes.data, V2.shape[1], O.ctypes.data,
                                int(nthreads))
    return O[:, 0] if vec else O
