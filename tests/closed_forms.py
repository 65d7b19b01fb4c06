"""Closed forms and exact references used to pin the oracle.  Independent of
both the oracle and the CUDA library: plain numpy / scipy / fractions."""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def dst_basis(n: int):
    """Orthonormal eigenvectors of tridiag(-1, 2, -1): the DST-I matrix
    V_jk = sqrt(2/(n+1)) sin(jk pi/(n+1)), eigenvalues 2 - 2 cos(k pi/(n+1))."""
    j = np.arange(1, n + 1)
    V = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(j, j) * np.pi / (n + 1))
    lam = 2.0 - 2.0 * np.cos(j * np.pi / (n + 1))
    return V, lam


def fun_lap1d(n: int, alpha: float, fn) -> np.ndarray:
    """fn(alpha * tridiag(-1, 2, -1)) through the eigenbasis."""
    V, lam = dst_basis(n)
    return (V * fn(alpha * lam)) @ V.T


def exp_lap2d_column(E1: np.ndarray, c: int) -> np.ndarray:
    """Column c of exp(Z1 (+) Z1) = E1 (x) E1 (Kronecker sum identity), with
    E1 = exp(Z1) for an m x m Z1; c = c1 m + c2."""
    m = E1.shape[0]
    c1, c2 = divmod(c, m)
    return np.kron(E1[:, c1], E1[:, c2])


def cos_lap2d_column(C1: np.ndarray, S1: np.ndarray, c: int) -> np.ndarray:
    """Column c of cos(Z1 (+) Z1) = C1 (x) C1 - S1 (x) S1."""
    m = C1.shape[0]
    c1, c2 = divmod(c, m)
    return np.kron(C1[:, c1], C1[:, c2]) - np.kron(S1[:, c1], S1[:, c2])


def frac_matmul(A, B):
    n = len(A)
    return [[sum((A[i][k] * B[k][j] for k in range(n)), Fraction(0)) for j in range(n)]
            for i in range(n)]


def frac_horner(Z, a):
    """sum_i a_i Z^i in exact rational arithmetic (Horner form)."""
    n = len(Z)
    Zf = [[Fraction(x) for x in row] for row in Z]
    S = [[Fraction(a[-1]) if i == j else Fraction(0) for j in range(n)] for i in range(n)]
    for c in reversed(a[:-1]):
        S = frac_matmul(Zf, S)
        for i in range(n):
            S[i][i] += Fraction(c)
    return S


def fma_exact(a: float, b: float, c: float) -> float:
    """Correctly rounded a*b + c via exact rationals (float(Fraction) rounds
    to nearest, ties to even)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def norm1_dense(M: np.ndarray) -> float:
    return float(np.abs(M).sum(axis=0).max())
