"""Sparse building blocks of the oracle: CSR container, product, scaled add,
exact 1-norm and Algorithm 1.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The arithmetic lives
in ``csrc/psf_oracle.c``; this module only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from ._lib import lib, _i32p, _f64p

OR_OK, OR_ENOMEM, OR_ENOTCONV = 0, 2, 4


class OracleNotConverged(RuntimeError):
    """Algorithm 1 hit its pass cap, or Theta found no truncation length."""


@dataclass
class CSR:
    """Square CSR matrix, 0-based, sorted unique columns, nonzero values only."""

    n: int
    rowptr: np.ndarray  # int32, n + 1
    col: np.ndarray  # int32, nnz
    val: np.ndarray  # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @staticmethod
    def identity(n: int, alpha: float = 1.0) -> "CSR":
        return CSR(n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
                   np.full(n, alpha, dtype=np.float64))

    @staticmethod
    def empty(n: int) -> "CSR":
        return CSR(n, np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float64))

    @staticmethod
    def from_scipy(m) -> "CSR":
        m = m.tocsr().copy()
        m.sum_duplicates()
        m.eliminate_zeros()
        m.sort_indices()
        return CSR(m.shape[0], m.indptr.astype(np.int32), m.indices.astype(np.int32),
                   m.data.astype(np.float64))

    @staticmethod
    def from_dense(a: np.ndarray) -> "CSR":
        a = np.asarray(a, dtype=np.float64)
        n = a.shape[0]
        rows, cols = np.nonzero(a)
        rowptr = np.zeros(n + 1, np.int32)
        np.add.at(rowptr, rows + 1, 1)
        return CSR(n, np.cumsum(rowptr).astype(np.int32), cols.astype(np.int32),
                   a[rows, cols].astype(np.float64))

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        out[rows, self.col] = self.val
        return out


def _ptrs(m: CSR):
    rp = np.ascontiguousarray(m.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(m.col, dtype=np.int32)
    v = np.ascontiguousarray(m.val, dtype=np.float64)
    keep = (rp, ci, v)
    return keep, (rp.ctypes.data_as(_i32p), ci.ctypes.data_as(_i32p), v.ctypes.data_as(_f64p))


def _null3():
    return (ctypes.cast(None, _i32p), ctypes.cast(None, _i32p), ctypes.cast(None, _f64p))


def _take(n: int, orp, oci, ov, onnz) -> CSR:
    h = lib()
    nnz = onnz.value
    rp = np.ctypeslib.as_array(orp, shape=(n + 1,)).copy()
    ci = np.ctypeslib.as_array(oci, shape=(nnz,)).copy() if nnz else np.zeros(0, np.int32)
    v = np.ctypeslib.as_array(ov, shape=(nnz,)).copy() if nnz else np.zeros(0, np.float64)
    for p in (orp, oci, ov):
        h.or_free(ctypes.cast(p, ctypes.c_void_p))
    return CSR(n, rp.astype(np.int32), ci.astype(np.int32), v.astype(np.float64))


def _outs():
    return (_i32p(), _i32p(), _f64p(), ctypes.c_int64())


def matmul_add(A: CSR, B: CSR, init: CSR | None = None) -> CSR:
    """C = init + A B with the fixed Gustavson rounding order (see the C file)."""
    assert A.n == B.n and (init is None or init.n == A.n)
    ka, pa = _ptrs(A)
    kb, pb = _ptrs(B)
    if init is not None:
        ki, pi = _ptrs(init)
    else:
        ki, pi = None, _null3()
    orp, oci, ov, onnz = _outs()
    rc = lib().or_matmul_add(A.n, *pa, *pb, *pi, ctypes.byref(orp), ctypes.byref(oci),
                             ctypes.byref(ov), ctypes.byref(onnz))
    if rc != OR_OK:
        raise MemoryError("oracle matmul_add failed")
    del ka, kb, ki
    return _take(A.n, orp, oci, ov, onnz)


def axpy(alpha: float, M: CSR | None, X: CSR | None, n: int) -> CSR:
    """Y = alpha M + X (M = I when None; X may be None), y = fma(alpha, m, x)."""
    if M is not None:
        km, pm = _ptrs(M)
    else:
        km, pm = None, _null3()
    if X is not None:
        kx, px = _ptrs(X)
    else:
        kx, px = None, _null3()
    orp, oci, ov, onnz = _outs()
    rc = lib().or_axpy(n, float(alpha), *pm, *px, ctypes.byref(orp), ctypes.byref(oci),
                       ctypes.byref(ov), ctypes.byref(onnz))
    if rc != OR_OK:
        raise MemoryError("oracle axpy failed")
    del km, kx
    return _take(n, orp, oci, ov, onnz)


def norm1(M: CSR) -> float:
    """||M||_1 with exactly rounded column sums."""
    k, p = _ptrs(M)
    out = ctypes.c_double()
    rc = lib().or_norm1(M.n, *p, ctypes.byref(out))
    if rc != OR_OK:
        raise MemoryError("oracle norm1 failed")
    return out.value


def exact_abs_sum(x: np.ndarray) -> float:
    """Correctly rounded sum of |x| (the accumulator behind every 1-norm)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().or_exact_abs_sum(x.ctypes.data_as(_f64p), x.size)


@dataclass
class Alg1Result:
    kept: CSR
    eps_f: float
    iters: int
    c: float  # 1-norm of the dropped entries


def alg1(C: CSR, eps_g: float, e_r: float, maxit: int = 1000) -> Alg1Result:
    """Algorithm 1 (Sec. 3.1.1), see ``or_alg1`` for the step-by-step form."""
    k, p = _ptrs(C)
    orp, oci, ov, onnz = _outs()
    eps_f = ctypes.c_double()
    iters = ctypes.c_int32()
    c = ctypes.c_double()
    rc = lib().or_alg1(C.n, *p, float(eps_g), float(e_r), int(maxit), ctypes.byref(orp),
                       ctypes.byref(oci), ctypes.byref(ov), ctypes.byref(onnz),
                       ctypes.byref(eps_f), ctypes.byref(iters), ctypes.byref(c))
    if rc not in (OR_OK, OR_ENOTCONV):
        raise MemoryError("oracle alg1 failed")
    kept = _take(C.n, orp, oci, ov, onnz)
    if rc == OR_ENOTCONV:
        raise OracleNotConverged(f"Algorithm 1 did not converge in {maxit} passes")
    return Alg1Result(kept, eps_f.value, iters.value, c.value)


def horner_dense(Z: np.ndarray, a, N: int) -> np.ndarray:
    """P_N(Z) = sum_{i<N} a_i Z^i by dense Horner (Eq. 1), for small n."""
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64)[:N])
    n = Z.shape[0]
    out = np.zeros((n, n))
    rc = lib().or_horner_dense(n, Z.ctypes.data_as(_f64p), a.ctypes.data_as(_f64p), N,
                               out.ctypes.data_as(_f64p))
    if rc != OR_OK:
        raise MemoryError("oracle horner failed")
    return out
