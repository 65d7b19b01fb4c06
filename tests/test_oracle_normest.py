"""Pins of the oracle's deterministic ||Z^k||_1 estimator (Sec. 3.2.2).

The estimate is a lower bound of the exact norm, and it is exact where the
power iteration provably lands on the largest column: for nonnegative
matrices (with integer entries every sum is exact, so the comparison is
exact too) and for diagonal ones.  One small case is traced by hand.
"""
import numpy as np
import pytest

from oracle import CSR, matmul_add, norm1
from oracle.normest import MAX_COLUMN, estimate_power_norm, power_norm_estimates, spmv, transpose


def exact_power_norm(Z: CSR, k: int) -> float:
    P = Z
    for _ in range(k - 1):
        P = matmul_add(Z, P)
    return norm1(P)


def test_hand_traced_2x2():
    # Z = [[1, -2], [3, 4]], k = 1, traced by hand:
    #   x = (1/2, 1/2): v = (-1/2, 7/2), best = 4; s = (-1, +1);
    #   w = Z^T s = (2, 6): j = 1; v = Z e_1 = (-2, 4), e = 6, sgn(v) = s: stop
    #   with best = 6; b = (1, -2): Z b = (5, -5), alt = 20/6 < 6.
    Z = CSR.from_dense(np.array([[1.0, -2.0], [3.0, 4.0]]))
    assert estimate_power_norm(Z, transpose(Z), 1) == 6.0
    # k = 2: Z^2 = [[-5, -10], [15, 10]], columns 20 and 20; traced:
    #   v = Z^2 x = (-7.5, 12.5), best = 20; s = (-1, +1); w = (Z^T)^2 s = (20, 20):
    #   j = 0; v = Z^2 e_0 = (-5, 15), e = 20 <= best: stop at 20; alt = 2*|Z^2 b|/6
    #   with Z^2 b = (15, -5): 40/6 < 20.
    assert estimate_power_norm(Z, transpose(Z), 2) == 20.0


def test_transpose_and_spmv():
    rng = np.random.default_rng(3)
    a = np.where(rng.random((40, 40)) < 0.2, rng.standard_normal((40, 40)), 0.0)
    Z = CSR.from_dense(a)
    ZT = transpose(Z)
    assert np.array_equal(ZT.to_dense(), a.T)
    # rows of Z^T in ascending row order of Z
    for r in range(40):
        cols = ZT.col[ZT.rowptr[r]:ZT.rowptr[r + 1]]
        assert np.all(np.diff(cols) > 0)
    x = rng.standard_normal(40)
    assert np.allclose(spmv(Z, x), a @ x, rtol=1e-14, atol=1e-14)
    # integer data: the fma chain is exact
    b = rng.integers(-3, 4, (30, 30)).astype(float)
    b[rng.random((30, 30)) < 0.5] = 0.0
    xi = rng.integers(-5, 6, 30).astype(float)
    assert np.array_equal(spmv(CSR.from_dense(b), xi), b @ xi)


@pytest.mark.parametrize("seed", range(5))
def test_exact_for_nonnegative_integer_matrices(seed):
    rng = np.random.default_rng(seed)
    n = 25
    a = rng.integers(0, 4, (n, n)).astype(float)
    a[rng.random((n, n)) < 0.7] = 0.0
    Z = CSR.from_dense(a)
    est = power_norm_estimates(Z)
    for k in range(2, 11):
        exact = np.abs(np.linalg.matrix_power(a, k)).sum(axis=0).max()
        assert est[k] == exact == exact_power_norm(Z, k)


def test_exact_for_diagonal_and_n1():
    d = np.array([1.0, -3.0, 2.0, 0.5])
    Z = CSR.from_dense(np.diag(d))
    est = power_norm_estimates(Z)
    for k in range(2, 11):
        assert est[k] == 3.0 ** k
    one = CSR.from_dense(np.array([[-1.5]]))
    assert power_norm_estimates(one)[2:] == [1.5 ** k for k in range(2, 11)]
    assert power_norm_estimates(CSR.empty(5))[2:] == [0.0] * 9


@pytest.mark.parametrize("seed", range(6))
def test_lower_bound_of_the_exact_norm(seed):
    # signed entries: the estimate never exceeds the exact norm (beyond the
    # rounding of the products), and is usually close to it
    rng = np.random.default_rng(100 + seed)
    n = 60
    a = np.where(rng.random((n, n)) < 0.08, rng.standard_normal((n, n)), 0.0)
    Z = CSR.from_dense(a)
    est = power_norm_estimates(Z)
    ratios = []
    for k in range(2, 11):
        exact = exact_power_norm(Z, k)
        assert est[k] <= exact * (1 + 1e-12)
        ratios.append(est[k] / exact)
    assert np.median(ratios) > 0.5


def test_long_column_falls_back_to_exact_norms():
    n = MAX_COLUMN + 2
    rows = np.arange(n)
    # column 0 full (n > MAX_COLUMN entries), plus the diagonal
    a_rows = np.concatenate([rows, rows[1:]])
    a_cols = np.concatenate([np.zeros(n, int), rows[1:]])
    vals = np.concatenate([np.full(n, 0.5), np.full(n - 1, -0.25)])
    import scipy.sparse as sp
    Z = CSR.from_scipy(sp.coo_matrix((vals, (a_rows, a_cols)), shape=(n, n)))
    from oracle import power_norms
    assert power_norm_estimates(Z) == power_norms(Z)
