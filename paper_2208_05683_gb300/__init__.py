"""GB300 evaluator for near-sparse matrix power series f(Z) = sum_i a_i Z^i by
the Paterson-Stockmeyer scheme combined with filtering (PSSCF).

Thin Python binding over the C ABI of ``libpsf.so`` (``include/psf.h``):
argument marshalling only, every step of the computation runs in the CUDA
library.  Matrices are square CSR on the GPU (``DeviceCSR``: int32 row
pointers and columns, float64 values, torch tensors on a CUDA device).

    Series(coeffs, tol, ...).eval(Z)        Algorithm 2 (filtered PS)
    eval_batch([...series], [...Z])         many instances at once (one block-diagonal batch)
    Server(...).submit / poll               serving loop with continuous batching
    product_filter(A, B, addends, thr)      one filtered product (Eq. 11/14 + Alg. 1)
    norm1(M)                                exact ||M||_1
    norm1_noalloc(M)                        the same, without allocating device memory
    plan(coeffs, tol, norms, ...)           the a-priori analysis (host only)

The library is loaded from ``paper_2208_05683_gb300/_build/libpsf.so``; if it
is missing it is built with nvcc, and if that is impossible every call fails
with an error -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

from . import _build
from ._abi import (PSF_NOFILTER, PSF_OK, PSF_POLY, PSF_SERIES, PSF_Z_ESTIMATE, PSF_Z_SQUARE, PSF_Z_SUBMULT,
                   PSF_PARAM_ALG1_MAXIT,
                   PSF_PARAM_ER, PSF_PARAM_POOL_ENTRIES, PSF_PARAM_KERNEL, PSF_PARAM_CHUNK_COLS,
                   PSF_PARAM_CHUNK_SLOTS, PSF_PARAM_DENSE_XOVER, PSF_MAX_Q, PSF_NORM1_NOALLOC_MAX_N,
                   PsfError, CSRStruct, InfoStruct, StepStruct, ServerConfig, Completion, ServerStats, BatchTune,
                   lib, check)

__all__ = [
    "DeviceCSR", "Series", "Result", "eval_batch", "product_filter", "norm1", "norm1_noalloc", "plan",
    "Server", "autotune", "autotune_batch", "tune_get", "tune_set", "PsfError",
    "PSF_SERIES", "PSF_POLY", "PSF_NOFILTER", "PSF_Z_SUBMULT", "PSF_Z_ESTIMATE", "PSF_Z_SQUARE", "PSF_MAX_Q",
    "build", "lib",
]


def build(force: bool = False) -> str:
    """Compile libpsf.so for sm_103a (in-tree) and return its path."""
    return _build.build(force=force)


def _torch():
    import torch
    return torch


@dataclass
class DeviceCSR:
    """Square CSR matrix on a CUDA device (torch tensors)."""

    n: int
    rowptr: "object"  # torch.int32, n + 1
    col: "object"  # torch.int32, nnz
    val: "object"  # torch.float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    @staticmethod
    def from_host(rowptr, col, val, device="cuda") -> "DeviceCSR":
        torch = _torch()
        rp = torch.as_tensor(rowptr, dtype=torch.int32).to(device)
        c = torch.as_tensor(col, dtype=torch.int32).to(device)
        v = torch.as_tensor(val, dtype=torch.float64).to(device)
        return DeviceCSR(int(rp.numel()) - 1, rp.contiguous(), c.contiguous(), v.contiguous())

    def to_host(self):
        return (self.rowptr.cpu().numpy(), self.col.cpu().numpy(), self.val.cpu().numpy())

    @staticmethod
    def from_torch(t, device=None) -> "DeviceCSR":
        """From a square torch sparse CSR tensor (any index and value dtype;
        converted to int32 / float64 on ``device``, default the tensor's own
        device).  Columns must be sorted within each row; the library checks."""
        torch = _torch()
        if t.layout != torch.sparse_csr:
            raise PsfError(1, "expected a torch sparse CSR tensor (torch.sparse_csr layout)")
        if t.dim() != 2 or t.shape[0] != t.shape[1]:
            raise PsfError(1, f"expected a square matrix, got shape {tuple(t.shape)}")
        dev = t.device if device is None else torch.device(device)
        rp = t.crow_indices().to(device=dev, dtype=torch.int32).contiguous()
        c = t.col_indices().to(device=dev, dtype=torch.int32).contiguous()
        v = t.values().to(device=dev, dtype=torch.float64).contiguous()
        return DeviceCSR(int(t.shape[0]), rp, c, v)

    def to_torch(self):
        """A torch sparse CSR tensor sharing this matrix's storage."""
        torch = _torch()
        return torch.sparse_csr_tensor(self.rowptr, self.col, self.val, size=(self.n, self.n),
                                       check_invariants=False)

    def _struct(self) -> CSRStruct:
        for t in (self.rowptr, self.col, self.val):
            if not t.is_cuda or not t.is_contiguous():
                raise PsfError(1, "DeviceCSR tensors must be contiguous CUDA tensors")
        return CSRStruct(self.n, self.nnz, self.rowptr.data_ptr(), self.col.data_ptr(),
                         self.val.data_ptr())


def _as_device_csr(Z) -> "DeviceCSR":
    """DeviceCSR as given, or converted from a torch sparse CSR tensor."""
    if isinstance(Z, DeviceCSR):
        return Z
    return DeviceCSR.from_torch(Z)


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


@dataclass
class Result:
    """Result of an evaluation; ``csr`` is a DeviceCSR copy owned by torch."""

    csr: DeviceCSR
    info: dict = field(default_factory=dict)
    steps: list = field(default_factory=list)


def _take_result(handle, stream, copy: bool = True, keep: bool = False):
    torch = _torch()
    L = lib()
    view = CSRStruct()
    check(L.psf_result_csr(handle, ctypes.byref(view)))
    info = InfoStruct()
    check(L.psf_result_info(handle, ctypes.byref(info)))
    steps = []
    for i in range(info.nsteps):
        s = StepStruct()
        check(L.psf_result_step(handle, i, ctypes.byref(s)))
        steps.append(s.as_dict())
    n, nnz = view.n, view.nnz
    dev = torch.device("cuda", torch.cuda.current_device())
    rp = torch.empty(n + 1, dtype=torch.int32, device=dev)
    col = torch.empty(nnz, dtype=torch.int32, device=dev)
    val = torch.empty(nnz, dtype=torch.float64, device=dev)
    check(L.psf_result_copy(handle, ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(col.data_ptr()),
                            ctypes.c_void_p(val.data_ptr()), stream))
    if not keep:
        check(L.psf_result_destroy(handle))
    return Result(DeviceCSR(n, rp, col, val), info.as_dict(), steps)


class Series:
    """A matrix power series (or polynomial) with its evaluation options.

    coeffs   a_0..a_{m-1}
    tol      eps_tol of Algorithm 2 (series) or eps of Eq. (27) (poly=True)
    poly     evaluate the polynomial of exactly these coefficients
    filtered False gives the unfiltered PS scheme (same N, q, b)
    submult  z_i = ||Z||^i instead of exact ||Z^i||_1 for i <= 10
    estimate z_i, i = 2..10, from the deterministic 1-norm estimator (PSF_Z_ESTIMATE)
    square   run the scheme on W = Z^2 for a series of only even or only odd
             powers (PSF_Z_SQUARE)
    s        override of the PS block size q (0 = Eq. 6)
    kernel   slot map of the product kernel: "auto", "table", "bitmap", "window" or
             "cta" (one output row per block of four warps)
             (the bitmap with its wide column window, for every product)
    chunk_cols, chunk_slots  > 0: smaller row chunks (to exercise row chunking)
    dense_xover  dense-tile crossover in multiply-adds per n^3 (0: every product
             step as dense tiles, 1e300: none, None: the process-wide value)
    """

    def __init__(self, coeffs, tol: float, *, poly: bool = False, filtered: bool = True,
                 submult: bool = False, estimate: bool = False, square: bool = False, s: int = 0,
                 e_r: float | None = None,
                 maxit: int | None = None, pool_entries: int | None = None,
                 kernel: str = "auto", chunk_cols: int = 0, chunk_slots: int = 0,
                 dense_xover: float | None = None):
        L = lib()
        a = (ctypes.c_double * len(coeffs))(*[float(x) for x in coeffs])
        flags = (PSF_POLY if poly else PSF_SERIES) | (0 if filtered else PSF_NOFILTER) | \
            (PSF_Z_SUBMULT if submult else 0) | (PSF_Z_ESTIMATE if estimate else 0) | \
            (PSF_Z_SQUARE if square else 0)
        h = ctypes.c_void_p()
        check(L.psf_series_create(a, len(coeffs), int(s), float(tol), flags, ctypes.byref(h)))
        self._h = h
        self.coeffs = [float(x) for x in coeffs]
        self.tol = float(tol)
        self.flags = flags
        if e_r is not None:
            check(L.psf_series_set_param(h, PSF_PARAM_ER, float(e_r)))
        if maxit is not None:
            check(L.psf_series_set_param(h, PSF_PARAM_ALG1_MAXIT, float(maxit)))
        if pool_entries is not None:
            check(L.psf_series_set_param(h, PSF_PARAM_POOL_ENTRIES, float(pool_entries)))
        kid = {"auto": 0, "table": 1, "bitmap": 2, "window": 3, "cta": 4}[kernel]
        if kid:
            check(L.psf_series_set_param(h, PSF_PARAM_KERNEL, float(kid)))
        if chunk_cols:
            check(L.psf_series_set_param(h, PSF_PARAM_CHUNK_COLS, float(chunk_cols)))
        if chunk_slots:
            check(L.psf_series_set_param(h, PSF_PARAM_CHUNK_SLOTS, float(chunk_slots)))
        if dense_xover is not None:
            check(L.psf_series_set_param(h, PSF_PARAM_DENSE_XOVER, float(dense_xover)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().psf_series_destroy(h)
            except Exception:
                pass
            self._h = None

    def eval_handle(self, Z: DeviceCSR, stream=None):
        """psf_eval; returns the raw result handle (caller destroys it)."""
        zs = _as_device_csr(Z)._struct()
        out = ctypes.c_void_p()
        check(lib().psf_eval(self._h, ctypes.byref(zs), _stream_ptr(stream), ctypes.byref(out)))
        return out

    def eval(self, Z: DeviceCSR, stream=None) -> Result:
        """psf_eval on a DeviceCSR or a torch sparse CSR tensor on the GPU;
        ``Result.csr.to_torch()`` gives the result as a torch sparse CSR tensor."""
        st = _stream_ptr(stream)
        Z = _as_device_csr(Z)
        zs = Z._struct()
        out = ctypes.c_void_p()
        check(lib().psf_eval(self._h, ctypes.byref(zs), st, ctypes.byref(out)))
        return _take_result(out, st)

    def eval_host(self, rowptr, col, val, stream=None):
        """psf_eval_from_host on host arrays; returns ((rowptr, col, val) as
        host numpy arrays, info, steps).  The copies in both directions are
        the library's (psf_eval_from_host, psf_result_copy into host arrays)."""
        import numpy as np
        L = lib()
        rp = np.ascontiguousarray(rowptr, dtype=np.int32)
        ci = np.ascontiguousarray(col, dtype=np.int32)
        v = np.ascontiguousarray(val, dtype=np.float64)
        zs = CSRStruct(len(rp) - 1, len(ci), rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
        st = _stream_ptr(stream)
        out = ctypes.c_void_p()
        check(L.psf_eval_from_host(self._h, ctypes.byref(zs), st, ctypes.byref(out)))
        try:
            info = InfoStruct()
            check(L.psf_result_info(out, ctypes.byref(info)))
            steps = []
            for i in range(info.nsteps):
                s = StepStruct()
                check(L.psf_result_step(out, i, ctypes.byref(s)))
                steps.append(s.as_dict())
            view = CSRStruct()
            check(L.psf_result_csr(out, ctypes.byref(view)))
            orp = np.empty(view.n + 1, np.int32)
            ocol = np.empty(max(view.nnz, 1), np.int32)
            oval = np.empty(max(view.nnz, 1), np.float64)
            check(L.psf_result_copy(out, orp.ctypes.data, ocol.ctypes.data, oval.ctypes.data, st))
            (stream if stream is not None else _torch().cuda.current_stream()).synchronize()
        finally:
            L.psf_result_destroy(out)
        return (orp, ocol[: view.nnz], oval[: view.nnz]), info.as_dict(), steps


def eval_batch(series, Zs, stream=None):
    """psf_eval_batch over instances (series[i], Zs[i]); list of Results."""
    L = lib()
    count = len(Zs)
    st = _stream_ptr(stream)
    sh = (ctypes.c_void_p * count)(*[s._h.value for s in series])
    Zs = [_as_device_csr(z) for z in Zs]
    zs = (CSRStruct * count)(*[z._struct() for z in Zs])
    outs = (ctypes.c_void_p * count)()
    check(L.psf_eval_batch(sh, zs, count, st, outs))
    return [_take_result(ctypes.c_void_p(outs[i]), st) for i in range(count)]


class Server:
    """Serving loop of the library (psf_server_*): requests are admitted by
    worker threads as workers and device memory free up, evaluated in
    batches, and overlap on the GPU.  ``submit`` keeps the series and Z
    alive until the request's completion has been polled."""

    def __init__(self, workers: int = 4, max_batch: int = 64, hbm_budget: int = 0):
        cfg = ServerConfig(int(workers), int(max_batch), int(hbm_budget))
        h = ctypes.c_void_p()
        check(lib().psf_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, series: Series, Z: DeviceCSR, tag: int) -> None:
        Z = _as_device_csr(Z)
        zs = Z._struct()
        check(lib().psf_server_submit(self._h, series._h, ctypes.byref(zs), ctypes.c_uint64(int(tag))))
        self._keep[int(tag)] = (series, Z)

    def poll(self, max_items: int = 64, wait_ms: int = -1, take: bool = True):
        """Completed requests: dicts with tag, status, batch_size, queue_ms,
        latency_ms and result (a Result, or None if the request failed or
        ``take`` is False, in which case the result is released unread)."""
        torch = _torch()
        buf = (Completion * max(1, max_items))()
        got = ctypes.c_int32()
        check(lib().psf_server_poll(self._h, buf, int(max_items), int(wait_ms), ctypes.byref(got)))
        out = []
        for i in range(got.value):
            c = buf[i]
            res = None
            if c.status == PSF_OK and c.result and not take:
                check(lib().psf_result_destroy(ctypes.c_void_p(c.result)))
            elif c.status == PSF_OK and c.result:
                st = torch.cuda.current_stream()
                res = _take_result(ctypes.c_void_p(c.result), _stream_ptr(st), keep=True)
                st.synchronize()  # the copy is done before the result is freed on its own stream
                check(lib().psf_result_destroy(ctypes.c_void_p(c.result)))
            self._keep.pop(int(c.tag), None)
            out.append({"tag": int(c.tag), "status": int(c.status), "batch_size": int(c.batch_size),
                        "queue_ms": c.queue_ms, "latency_ms": c.latency_ms, "result": res})
        return out

    def cancel(self, tag: int) -> bool:
        """Withdraw the oldest request with this tag still waiting for
        admission; True if one was (it completes with PSF_ECANCELED)."""
        got = ctypes.c_int32()
        check(lib().psf_server_cancel(self._h, ctypes.c_uint64(int(tag)), ctypes.byref(got)))
        return bool(got.value)

    def stats(self) -> dict:
        s = ServerStats()
        check(lib().psf_server_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def close(self) -> None:
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().psf_server_destroy(h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def product_filter(A: DeviceCSR | None, B: DeviceCSR | None, addends=(), threshold: float = 0.0,
                   e_r: float = 0.1, maxit: int = 1000, stream=None) -> Result:
    """C = sum_t alpha_t M_t + A B, then Algorithm 1 with ||dropped||_1 <= threshold.

    ``addends`` is a sequence of (alpha, M) with M a DeviceCSR or None for I.
    """
    L = lib()
    st = _stream_ptr(stream)
    nadd = len(addends)
    alphas = (ctypes.c_double * max(nadd, 1))(*[float(a) for a, _ in addends])
    structs = [m._struct() if m is not None else None for _, m in addends]
    ptrs = (ctypes.POINTER(CSRStruct) * max(nadd, 1))()
    for i, s in enumerate(structs):
        ptrs[i] = ctypes.pointer(s) if s is not None else ctypes.POINTER(CSRStruct)()
    a_s = A._struct() if A is not None else None
    b_s = B._struct() if B is not None else None
    out = ctypes.c_void_p()
    check(L.psf_product_filter(ctypes.byref(a_s) if a_s else None, ctypes.byref(b_s) if b_s else None,
                               nadd, alphas, ptrs, float(threshold), float(e_r), int(maxit), st,
                               ctypes.byref(out)))
    return _take_result(out, st)


def norm1(M: DeviceCSR, stream=None) -> float:
    """||M||_1 with exactly rounded column sums."""
    out = ctypes.c_double()
    ms = M._struct()
    check(lib().psf_norm1(ctypes.byref(ms), _stream_ptr(stream), ctypes.byref(out)))
    return out.value


def norm1_noalloc(M: DeviceCSR, stream=None) -> float:
    """||M||_1 as norm1, in the library's static scratch region (no device
    allocation; n <= PSF_NORM1_NOALLOC_MAX_N; overlapping calls race)."""
    out = ctypes.c_double()
    ms = M._struct()
    check(lib().psf_norm1_noalloc(ctypes.byref(ms), _stream_ptr(stream), ctypes.byref(out)))
    return out.value


def autotune(series: "Series", Z: DeviceCSR, stream=None):
    """psf_autotune: time both slot maps on this evaluation and keep the
    faster crossover; returns (crossover, ms saved per evaluation)."""
    c, saved = ctypes.c_double(), ctypes.c_double()
    zs = Z._struct()
    check(lib().psf_autotune(series._h, ctypes.byref(zs), _stream_ptr(stream), ctypes.byref(c), ctypes.byref(saved)))
    return c.value, saved.value


def autotune_batch(series, Zs, stream=None) -> dict:
    """psf_autotune_batch: tune the slot-map crossover, row bitmaps and
    baby-step reuse on this batch of instances (series[i], Zs[i]) and keep
    the fastest; returns the chosen settings and the batch's time before
    and after (ms)."""
    count = len(Zs)
    sh = (ctypes.c_void_p * count)(*[s._h.value for s in series])
    Zs = [_as_device_csr(z) for z in Zs]
    zs = (CSRStruct * count)(*[z._struct() for z in Zs])
    out = BatchTune()
    check(lib().psf_autotune_batch(sh, zs, count, _stream_ptr(stream), ctypes.byref(out)))
    return out.as_dict()


def tune_get(key: int = 1) -> float:
    v = ctypes.c_double()
    check(lib().psf_tune_get(int(key), ctypes.byref(v)))
    return v.value


def tune_set(key: int, value: float) -> None:
    check(lib().psf_tune_set(int(key), float(value)))


def plan(coeffs, tol: float, norms, *, poly: bool = False, submult: bool = False, s: int = 0,
         square: bool = False, thresholds: bool = True):
    """The host planner: N, q, b, g, z, truncation bound, budget, and with
    ``thresholds`` zeta and sigma (PsfError PSF_ETOOBIG when q or b is past
    their PSF_MAX_Q + 2 entries; thresholds=False plans without them)."""
    L = lib()
    a = (ctypes.c_double * len(coeffs))(*[float(x) for x in coeffs])
    nz = list(norms) + [0.0] * (11 - len(norms))
    nrm = (ctypes.c_double * 11)(*[float(x) for x in nz[:11]])
    info = InfoStruct()
    zeta = (ctypes.c_double * (PSF_MAX_Q + 2))() if thresholds else None
    sigma = (ctypes.c_double * (PSF_MAX_Q + 2))() if thresholds else None
    flags = (PSF_POLY if poly else 0) | (PSF_Z_SUBMULT if submult else 0) | (PSF_Z_SQUARE if square else 0)
    check(L.psf_plan(a, len(coeffs), int(s), float(tol), flags, nrm, ctypes.byref(info), zeta, sigma))
    d = info.as_dict()
    if thresholds:
        d["zeta"] = {k: zeta[k] for k in range(2, d["q"] + 1)}
        d["sigma"] = {j: sigma[j] for j in range(1 + d["g"], d["b"])}
    return d
