"""Deterministic estimates of ||Z^k||_1, k = 2..10 (Sec. 3.2.2, Eq. 37).

TEST INFRASTRUCTURE ONLY: like the rest of ``oracle/`` it is imported by the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU legs alone.

The paper takes ||Z^i||, i <= 10, from Higham's normest1, a randomized block
estimator.  This is its deterministic single-vector core: Hager's 1-norm
power iteration with Higham's stopping rules and alternating test vector,
written out in the order of the steps below.  The library's optional
estimator (series flag PSF_Z_ESTIMATE) must return the same values bit for
bit, so every floating-point operation is fixed:

  * A = Z^k is applied to a vector as k products with Z, and A^T as k
    products with Z^T; a product y = M x forms each y_r as a chain of fma()
    over row r's entries in stored order, starting from +0 (or_spmv).  The
    rows of Z^T hold their entries in ascending row order of Z.
  * ||v||_1 is the exactly rounded sum of |v_i| (exact_abs_sum).
  * sgn(t) = -1 for t < 0 and +1 otherwise (+0 and -0 included).

Estimate of ||A||_1 (A = Z^k, n x n):
  1. x = (1/n, ..., 1/n) (1/n rounded once); v = A x; best = ||v||_1.
     If n = 1, best is the norm.
  2. s = sgn(v); w = A^T s; no previous index; one product with A so far.
  3. Repeat:
       j = the smallest index with |w_j| = max_i |w_i|;
       stop if a previous index p exists and |w_p| = |w_j| (e_p maximises);
       stop if five products with A were made;
       v = A e_j; e = ||v||_1; s' = sgn(v);
       if e <= best or s' = s: best = max(best, e), stop;
       best = e; s = s'; w = A^T s; p = j.
  4. b_i = (-1)^i (1 + i/(n-1)), i = 0..n-1 (the quotient, then the sum,
     each rounded); alt = (2 ||A b||_1) / (3n); the estimate is max(best, alt).

The estimate is ||A x||_1 / ||x||_1 for some x: a lower bound of ||A||_1
(up to the rounding of the products).  ||Z||_1 itself is exact (norm1).
When a column of Z holds more than MAX_COLUMN entries the estimator is not
used and the exact norms of every power are returned (power_norms): the
library's transposition orders a column's entries with one warp and bounds
that work the same way.
"""
from __future__ import annotations

import numpy as np

from ._lib import lib
from .sparse import CSR, _f64p, _ptrs, exact_abs_sum, norm1

MAX_COLUMN = 4096  # longest column of Z the estimator takes
MAX_PRODUCTS = 5   # products with A in the power iteration (the alternating vector aside)


def transpose(Z: CSR) -> CSR:
    """Z^T in CSR; each row's entries in ascending row order of Z (a stable
    sort of Z's entries by column)."""
    rows = np.repeat(np.arange(Z.n, dtype=np.int64), np.diff(Z.rowptr))
    order = np.argsort(np.asarray(Z.col, dtype=np.int64), kind="stable")
    counts = np.bincount(np.asarray(Z.col, dtype=np.int64), minlength=Z.n)
    rp = np.zeros(Z.n + 1, np.int64)
    np.cumsum(counts, out=rp[1:])
    return CSR(Z.n, rp.astype(np.int32), rows[order].astype(np.int32), np.asarray(Z.val, np.float64)[order])


def spmv(M: CSR, x: np.ndarray) -> np.ndarray:
    """y = M x, each y_r a chain of fma() over row r in stored order."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(M.n, dtype=np.float64)
    _, p = _ptrs(M)
    lib().or_spmv(M.n, *p, x.ctypes.data_as(_f64p), y.ctypes.data_as(_f64p))
    return y


def _power(M: CSR, k: int, x: np.ndarray) -> np.ndarray:
    for _ in range(k):
        x = spmv(M, x)
    return x


def _sgn(v: np.ndarray) -> np.ndarray:
    return np.where(v < 0.0, -1.0, 1.0)


def estimate_power_norm(Z: CSR, ZT: CSR, k: int) -> float:
    """The estimate of ||Z^k||_1 defined above (ZT = transpose(Z))."""
    n = Z.n
    if n == 0:
        return 0.0
    x = np.full(n, 1.0 / n)
    v = _power(Z, k, x)
    best = exact_abs_sum(v)
    if n == 1:
        return best
    s = _sgn(v)
    w = _power(ZT, k, s)
    prev = -1
    products = 1
    while True:
        aw = np.abs(w)
        j = int(np.argmax(aw))  # the first maximiser
        if prev >= 0 and aw[prev] == aw[j]:
            break
        if products == MAX_PRODUCTS:
            break
        e_j = np.zeros(n)
        e_j[j] = 1.0
        v = _power(Z, k, e_j)
        products += 1
        e = exact_abs_sum(v)
        s_new = _sgn(v)
        if e <= best or np.array_equal(s_new, s):
            best = max(best, e)
            break
        best = e
        s = s_new
        w = _power(ZT, k, s)
        prev = j
    i = np.arange(n, dtype=np.float64)
    b = 1.0 + i / float(n - 1)
    b[1::2] = -b[1::2]
    alt = (2.0 * exact_abs_sum(_power(Z, k, b))) / (3.0 * n)
    return max(best, alt)


def power_norm_estimates(Z: CSR, kmax: int = 10) -> list[float]:
    """[1, ||Z||_1, est ||Z^2||_1, ..., est ||Z^kmax||_1]; the exact norms of
    every power when a column of Z is longer than MAX_COLUMN."""
    counts = np.bincount(np.asarray(Z.col, dtype=np.int64), minlength=max(Z.n, 1))
    if Z.n > 0 and counts.max() > MAX_COLUMN:
        from .psscf import power_norms
        return power_norms(Z)
    ZT = transpose(Z)
    return [1.0, norm1(Z)] + [estimate_power_norm(Z, ZT, k) for k in range(2, kmax + 1)]
