"""ctypes declarations mirroring ``include/psf.h``."""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

PSF_OK, PSF_EINVAL, PSF_ENOMEM, PSF_ECUDA, PSF_ENOTCONV, PSF_ETIMEOUT, PSF_ETOOBIG, PSF_ECANCELED = range(8)
PSF_SERIES, PSF_POLY, PSF_NOFILTER, PSF_Z_SUBMULT, PSF_Z_ESTIMATE, PSF_Z_SQUARE = 0, 1, 2, 4, 8, 16
PSF_PARAM_ER, PSF_PARAM_ALG1_MAXIT, PSF_PARAM_POOL_ENTRIES = 1, 2, 3
PSF_PARAM_KERNEL, PSF_PARAM_CHUNK_COLS, PSF_PARAM_CHUNK_SLOTS = 4, 5, 6
PSF_PARAM_DENSE_XOVER = 7
PSF_MAX_Q = 23
PSF_NORM1_NOALLOC_MAX_N = 65536
PSF_TUNE_TABLE_CROSSOVER = 1
PSF_TUNE_BATCH_GRAPH = 2
PSF_TUNE_BATCH_REUSE = 3
PSF_TUNE_ALG1_FAR_SHIFT = 4
PSF_TUNE_BARRIER_BUDGET_NS = 5
PSF_TUNE_FAIL_ADMISSION = 6
PSF_TUNE_DENSE_XOVER = 7
PSF_TUNE_ROW_BITMAPS = 8

ERROR_NAMES = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONV", 5: "ETIMEOUT", 6: "ETOOBIG", 7: "ECANCELED"}

# Every function the header declares (checked by the tests).
EXPORTS = [
    "psf_version", "psf_last_error", "psf_series_create", "psf_series_set_param",
    "psf_series_destroy", "psf_eval", "psf_eval_from_host", "psf_eval_batch", "psf_product_filter", "psf_norm1",
    "psf_norm1_noalloc", "psf_server_create", "psf_server_submit", "psf_server_poll", "psf_server_stats",
    "psf_server_destroy", "psf_server_cancel", "psf_tune_set", "psf_tune_get", "psf_autotune",
    "psf_plan", "psf_result_csr", "psf_result_copy", "psf_result_info", "psf_result_step",
    "psf_result_destroy", "psf_launch_count", "psf_profile", "psf_profile_read", "psf_fp64_peak",
    "psf_autotune_batch",
]


class PsfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"psf {ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class CSRStruct(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("hbm_budget", ctypes.c_int64)]


class Completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int32), ("batch_size", ctypes.c_int32),
                ("result", ctypes.c_void_p), ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("max_concurrent", ctypes.c_int32), ("pending", ctypes.c_int32),
                ("budget_peak", ctypes.c_int64), ("cancelled", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchTune(ctypes.Structure):
    _fields_ = [("table_crossover", ctypes.c_double), ("row_bitmaps", ctypes.c_int32),
                ("batch_reuse", ctypes.c_int32), ("configs", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("ms_before", ctypes.c_double), ("ms_after", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class InfoStruct(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("q", ctypes.c_int32), ("b", ctypes.c_int32),
                ("g", ctypes.c_int32), ("products", ctypes.c_int32), ("nsteps", ctypes.c_int32),
                ("z", ctypes.c_double * 11), ("alpha10", ctypes.c_double), ("trunc", ctypes.c_double),
                ("budget", ctypes.c_double), ("nnz", ctypes.c_int64), ("fma", ctypes.c_int64)]

    def as_dict(self):
        return {"N": self.N, "q": self.q, "b": self.b, "g": self.g, "products": self.products,
                "nsteps": self.nsteps, "z": list(self.z), "alpha10": self.alpha10,
                "trunc": self.trunc, "budget": self.budget, "nnz": self.nnz, "fma": self.fma}


class StepStruct(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("index", ctypes.c_int32), ("threshold", ctypes.c_double),
                ("nnz_pre", ctypes.c_int64), ("nnz_post", ctypes.c_int64), ("eps_f", ctypes.c_double),
                ("iters", ctypes.c_int32), ("dropped", ctypes.c_double), ("fma", ctypes.c_int64)]

    def as_dict(self):
        return {"kind": ("baby", "giant", "add", "odd")[self.kind], "index": self.index,
                "threshold": self.threshold, "nnz_pre": self.nnz_pre, "nnz_post": self.nnz_post,
                "eps_f": self.eps_f, "iters": self.iters, "dropped": self.dropped, "fma": self.fma}


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Load libpsf.so (building it first if needed).  Raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if not os.path.exists(path):
                raise PsfError(PSF_ECUDA, f"{path} missing")
            h = ctypes.CDLL(path)
            _declare(h)
            _lib = h
    return _lib


def check(rc: int) -> None:
    if rc != PSF_OK:
        msg = lib().psf_last_error().decode(errors="replace")
        raise PsfError(rc, msg)


def _declare(h: ctypes.CDLL) -> None:
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    csrp = ctypes.POINTER(CSRStruct)
    h.psf_version.restype = ctypes.c_int
    h.psf_version.argtypes = []
    h.psf_last_error.restype = ctypes.c_char_p
    h.psf_last_error.argtypes = []
    h.psf_series_create.argtypes = [ctypes.POINTER(f64), i64, i32, f64, ctypes.c_uint32, ctypes.POINTER(vp)]
    h.psf_series_set_param.argtypes = [vp, i32, f64]
    h.psf_series_destroy.argtypes = [vp]
    h.psf_eval.argtypes = [vp, csrp, vp, ctypes.POINTER(vp)]
    h.psf_eval_from_host.argtypes = [vp, csrp, vp, ctypes.POINTER(vp)]
    h.psf_eval_batch.argtypes = [ctypes.POINTER(vp), csrp, i32, vp, ctypes.POINTER(vp)]
    h.psf_product_filter.argtypes = [csrp, csrp, i32, ctypes.POINTER(f64), ctypes.POINTER(csrp), f64, f64,
                                     i32, vp, ctypes.POINTER(vp)]
    h.psf_norm1.argtypes = [csrp, vp, ctypes.POINTER(f64)]
    h.psf_norm1_noalloc.argtypes = [csrp, vp, ctypes.POINTER(f64)]
    h.psf_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    h.psf_server_submit.argtypes = [vp, vp, csrp, ctypes.c_uint64]
    h.psf_server_poll.argtypes = [vp, ctypes.POINTER(Completion), i32, i32, ctypes.POINTER(i32)]
    h.psf_server_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    h.psf_server_destroy.argtypes = [vp]
    h.psf_server_cancel.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(i32)]
    h.psf_tune_set.argtypes = [i32, f64]
    h.psf_tune_get.argtypes = [i32, ctypes.POINTER(f64)]
    h.psf_autotune.argtypes = [vp, csrp, vp, ctypes.POINTER(f64), ctypes.POINTER(f64)]
    h.psf_plan.argtypes = [ctypes.POINTER(f64), i64, i32, f64, ctypes.c_uint32, ctypes.POINTER(f64),
                           ctypes.POINTER(InfoStruct), ctypes.POINTER(f64), ctypes.POINTER(f64)]
    h.psf_result_csr.argtypes = [vp, csrp]
    h.psf_result_copy.argtypes = [vp, vp, vp, vp, vp]
    h.psf_result_info.argtypes = [vp, ctypes.POINTER(InfoStruct)]
    h.psf_result_step.argtypes = [vp, i32, ctypes.POINTER(StepStruct)]
    h.psf_result_destroy.argtypes = [vp]
    h.psf_launch_count.argtypes = [ctypes.POINTER(i64)]
    h.psf_profile.argtypes = [i32]
    h.psf_profile_read.argtypes = [ctypes.POINTER(i64), ctypes.POINTER(f64), ctypes.POINTER(f64), i32]
    h.psf_fp64_peak.argtypes = [vp, ctypes.POINTER(f64)]
    h.psf_autotune_batch.argtypes = [ctypes.POINTER(vp), csrp, i32, vp, ctypes.POINTER(BatchTune)]
    for name in EXPORTS:
        if name not in ("psf_last_error",):
            getattr(h, name).restype = ctypes.c_int
