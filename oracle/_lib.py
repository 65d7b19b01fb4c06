"""Loader for the oracle's C core (``oracle/csrc/psf_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The library is compiled
with gcc on first use (and by ``__graft_entry__.build()``) with floating-point
contraction disabled, so that every fused multiply-add in it is an explicit
``fma()`` call.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "psf_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libpsf_oracle.so")
_lock = threading.Lock()
_handle = None

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle's C core if it is missing or older than its source."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _handle
    with _lock:
        if _handle is None:
            _handle = ctypes.CDLL(build())
            _declare(_handle)
    return _handle


_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32pp = ctypes.POINTER(_i32p)
_f64pp = ctypes.POINTER(_f64p)
_i64p = ctypes.POINTER(ctypes.c_int64)


def _declare(h: ctypes.CDLL) -> None:
    h.or_free.argtypes = [ctypes.c_void_p]
    h.or_free.restype = None
    h.or_exact_abs_sum.argtypes = [_f64p, ctypes.c_int64]
    h.or_exact_abs_sum.restype = ctypes.c_double
    h.or_norm1.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p]
    h.or_norm1.restype = ctypes.c_int
    h.or_matmul_add.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p,
                                _i32p, _i32p, _f64p, _i32pp, _i32pp, _f64pp, _i64p]
    h.or_matmul_add.restype = ctypes.c_int
    h.or_axpy.argtypes = [ctypes.c_int32, ctypes.c_double, _i32p, _i32p, _f64p, _i32p, _i32p,
                          _f64p, _i32pp, _i32pp, _f64pp, _i64p]
    h.or_axpy.restype = ctypes.c_int
    h.or_alg1.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, ctypes.c_double, ctypes.c_double,
                          ctypes.c_int32, _i32pp, _i32pp, _f64pp, _i64p, _f64p,
                          ctypes.POINTER(ctypes.c_int32), _f64p]
    h.or_alg1.restype = ctypes.c_int
    h.or_horner_dense.argtypes = [ctypes.c_int32, _f64p, _f64p, ctypes.c_int32, _f64p]
    h.or_horner_dense.restype = ctypes.c_int
    h.or_spmv.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p]
    h.or_spmv.restype = None
