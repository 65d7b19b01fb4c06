"""Seeded synthetic inputs shared by the tests, the benchmark, the CUDA path's
callers and the oracle.

This module holds input construction only -- test matrices, their scaling and
Taylor coefficients -- and none of the filtered-PS arithmetic.  Matrices are
returned as plain numpy CSR triples (rowptr int32, col int32, val float64),
square, 0-based, columns sorted, no stored zeros.

The shapes stand in for the paper's workloads (Sec. 4): its first set (ten
10000 x 10000 network adjacency matrices, not available here) and its second
set (random banded matrices).  Workloads:
  laplacian_1d      Z = -0.5 tridiag(-1, 2, -1)                    (||Z||_1 = 2)
  laplacian_2d      Z = -0.5 (5-point Dirichlet Laplacian, m x m)  (||Z||_1 = 4)
  banded_random     symmetric, half-bandwidth w, off-diagonals U[-1, 1],
                    diagonal_j = -sum_{i != j} |z_ij|, scaled to a target 1-norm
  banded_normal     the paper's second set: lower = upper bandwidth w,
                    N(0, 1) entries (Sec. 4, item 2)
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def _csr_from_coo(n, rows, cols, vals):
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    keep = vals != 0.0
    rows, cols, vals = rows[keep], cols[keep], vals[keep]
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return (np.cumsum(rowptr).astype(np.int32), cols.astype(np.int32), vals.astype(np.float64))


def norm1(csr) -> float:
    """Largest column sum of |z_ij| (used only to scale generated inputs)."""
    rowptr, col, val = csr
    n = len(rowptr) - 1
    return float(np.bincount(col, weights=np.abs(val), minlength=n).max()) if len(val) else 0.0


def scale(csr, factor: float):
    rowptr, col, val = csr
    return (rowptr, col, val * factor)


def laplacian_1d(n: int, alpha: float = -0.5):
    """alpha * tridiag(-1, 2, -1), n x n."""
    i = np.arange(n)
    rows = np.concatenate([i, i[1:], i[:-1]])
    cols = np.concatenate([i, i[1:] - 1, i[:-1] + 1])
    vals = np.concatenate([np.full(n, 2.0 * alpha), np.full(n - 1, -alpha), np.full(n - 1, -alpha)])
    return _csr_from_coo(n, rows, cols, vals)


def laplacian_2d(m: int, alpha: float = -0.5):
    """alpha * (5-point Dirichlet Laplacian on an m x m grid), n = m^2,
    natural (row-major) ordering."""
    n = m * m
    idx = np.arange(n)
    gi, gj = idx // m, idx % m
    rows, cols, vals = [idx], [idx], [np.full(n, 4.0 * alpha)]
    for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        ok = (gi + di >= 0) & (gi + di < m) & (gj + dj >= 0) & (gj + dj < m)
        rows.append(idx[ok])
        cols.append(idx[ok] + di * m + dj)
        vals.append(np.full(ok.sum(), -alpha))
    return _csr_from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def banded_random(n: int, hbw: int, seed: int, target_norm1: float = 2.0):
    """Symmetric banded matrix: off-diagonals U[-1, 1] from ``seed``,
    diagonal_j = -sum_{i != j} |z_ij|, then scaled to ||Z||_1 = target_norm1."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for d in range(1, hbw + 1):
        v = rng.uniform(-1.0, 1.0, n - d)
        i = np.arange(n - d)
        rows += [i, i + d]
        cols += [i + d, i]
        vals += [v, v]
    rows = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    cols = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    vals = np.concatenate(vals) if vals else np.zeros(0)
    diag = -np.bincount(cols, weights=np.abs(vals), minlength=n)
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    vals = np.concatenate([vals, diag])
    csr = _csr_from_coo(n, rows, cols, vals)
    nrm = norm1(csr)
    return scale(csr, target_norm1 / nrm) if nrm > 0 else csr


def banded_normal(n: int, w: int, seed: int):
    """Random banded matrix with lower = upper bandwidth w and N(0, 1)
    entries (the paper's second test set, Sec. 4)."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for d in range(-w, w + 1):
        i = np.arange(max(0, -d), min(n, n - d))
        rows.append(i)
        cols.append(i + d)
        vals.append(rng.standard_normal(len(i)))
    return _csr_from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def random_sparse(n: int, density: float, seed: int, target_norm1: float = 1.0):
    """Unstructured random sparse matrix (values U[-1, 1]) scaled to a 1-norm."""
    rng = np.random.default_rng(seed)
    nnz = max(1, int(round(density * n * n)))
    rows = rng.integers(0, n, nnz)
    cols = rng.integers(0, n, nnz)
    key = np.unique(rows.astype(np.int64) * n + cols)
    rows, cols = key // n, key % n
    vals = rng.uniform(-1.0, 1.0, len(key))
    csr = _csr_from_coo(n, rows, cols, vals)
    nrm = norm1(csr)
    return scale(csr, target_norm1 / nrm) if nrm > 0 else csr


# ---------------------------------------------------------------- coefficients
MAX_TERMS = 200


def _trim(a):
    while a and a[-1] == 0.0:
        a.pop()
    return a


def coeffs(kind: str, terms: int = MAX_TERMS):
    """Taylor coefficients a_0..a_{terms-1}, each the double nearest the exact
    rational value; trailing zeros (underflow) removed.

    exp: 1/i!   cos: (-1)^j/(2j)! at i = 2j (Eq. 40)   cosh: 1/(2j)! at i = 2j
    sinh: 1/(2j+1)! at i = 2j+1
    """
    a = []
    for i in range(terms):
        if kind == "exp":
            a.append(float(Fraction(1, math.factorial(i))))
        elif kind == "cos":
            a.append(float(Fraction((-1) ** (i // 2), math.factorial(i))) if i % 2 == 0 else 0.0)
        elif kind == "cosh":
            a.append(float(Fraction(1, math.factorial(i))) if i % 2 == 0 else 0.0)
        elif kind == "sinh":
            a.append(float(Fraction(1, math.factorial(i))) if i % 2 == 1 else 0.0)
        else:
            raise ValueError(kind)
    return _trim(a)


# ---------------------------------------------------------- named workloads
def workload(name: str):
    """(Z, coefficient kind, tol) of a named single-matrix workload."""
    if name == "lap1d_n256":
        return laplacian_1d(256), "exp", 1e-12
    if name == "lap2d_128x128":
        return laplacian_2d(128), "exp", 1e-12
    if name == "banded_n65536_hbw5":
        return banded_random(65536, 5, seed=0, target_norm1=2.0), "exp", 1e-12
    if name == "random_n2000":  # unstructured: the powers fill in (dense-tile steps)
        return random_sparse(2000, 0.01, seed=3, target_norm1=2.0), "exp", 1e-12
    raise KeyError(name)


# ------------------------------------------------------- instance mixtures
def _scaled(csr, target):
    nrm = norm1(csr)
    return scale(csr, target / nrm) if nrm > 0 else csr


def mixed_instance(seed: int, n_lo: int, n_hi: int, kinds=("exp", "cosh"), tols=(1e-12,)):
    """One instance of a size mixture: (Z, coefficient kind, tol).

    n = round(exp(U[ln n_lo, ln n_hi])); the type is uniform over the 1D
    Laplacian, the 2D Laplacian (n rounded to a square m^2) and the banded
    random matrix of half-bandwidth 5; ||Z||_1 ~ U[1, 4]; the series kind and
    the tolerance are drawn uniformly from ``kinds`` and ``tols``.  Everything
    follows from ``seed``.
    """
    rng = np.random.default_rng([seed, 2208])
    n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
    typ = int(rng.integers(0, 3))
    target = float(rng.uniform(1.0, 4.0))
    kind = kinds[int(rng.integers(0, len(kinds)))]
    tol = tols[int(rng.integers(0, len(tols)))]
    if typ == 0:
        Z = _scaled(laplacian_1d(max(n, 2)), target)
    elif typ == 1:
        m = max(2, int(round(math.sqrt(n))))
        Z = _scaled(laplacian_2d(m), target)
    else:
        Z = banded_random(max(n, 6), 5, seed=seed, target_norm1=target)
    return Z, kind, tol


def batch_instances(count: int = 512, seed0: int = 0):
    """The batched workload: ``count`` instances (seeds seed0..), n
    log-uniform in [64, 4096], exp or cosh, tol 1e-12."""
    return [mixed_instance(seed0 + i, 64, 4096) for i in range(count)]


def serving_requests(count: int, seed0: int = 0, n_lo: int = 256, n_hi: int = 65536):
    """Serving mixture: n log-uniform in [n_lo, n_hi], exp/cos/sinh, tol from
    {1e-8, 1e-10, 1e-12}."""
    return [mixed_instance(seed0 + i, n_lo, n_hi, kinds=("exp", "cos", "sinh"), tols=(1e-8, 1e-10, 1e-12))
            for i in range(count)]
