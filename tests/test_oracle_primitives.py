"""Pins for the oracle's sparse building blocks (CPU only).

Each check ties the oracle to something outside itself: Python's correctly
rounded math.fsum, exact rational arithmetic, scipy's sparse product, or an
Algorithm 1 example worked by hand.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from closed_forms import fma_exact
from oracle import CSR, alg1, axpy, exact_abs_sum, matmul_add, norm1


def rand_csr(n, density, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    m = sp.random(n, n, density=density, random_state=rng, format="csr",
                  data_rvs=lambda k: rng.uniform(-1, 1, k) * scale)
    return CSR.from_scipy(m)


# ------------------------------------------------------------- exact sums
@pytest.mark.parametrize("seed", range(6))
def test_exact_sum_matches_fsum_wide_range(seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, 500) * 2.0 ** rng.integers(-1100, 1000, 500)
    x = np.concatenate([x, [5e-324, 2.2250738585072014e-308, 1.7976931348623157e308 / 1e6]])
    assert exact_abs_sum(x) == math.fsum(np.abs(x))


def test_exact_sum_ties_to_even_and_sticky():
    # 1 + 2^-53 is a tie: rounds to even (1.0); a further tiny term breaks it
    assert exact_abs_sum(np.array([1.0, 2.0 ** -53])) == 1.0
    assert exact_abs_sum(np.array([1.0, 2.0 ** -53, 2.0 ** -1000])) == 1.0 + 2.0 ** -52
    assert exact_abs_sum(np.array([1.0 + 2.0 ** -52, 2.0 ** -53])) == 1.0 + 2.0 ** -51
    # subnormals add exactly
    assert exact_abs_sum(np.array([5e-324] * 7)) == 7 * 5e-324
    assert exact_abs_sum(np.array([-3.0, 4.0])) == 7.0
    assert exact_abs_sum(np.zeros(3)) == 0.0


def test_exact_sum_is_order_free():
    rng = np.random.default_rng(7)
    x = rng.standard_normal(2000) * 10.0 ** rng.integers(-20, 20, 2000)
    s = exact_abs_sum(x)
    for _ in range(3):
        assert exact_abs_sum(rng.permutation(x)) == s


def test_norm1_is_max_exact_column_sum():
    for seed in range(4):
        A = rand_csr(60, 0.1, seed, scale=10.0 ** seed)
        D = A.to_dense()
        ref = max(math.fsum(np.abs(D[:, j])) for j in range(A.n))
        assert norm1(A) == ref


# ------------------------------------------------------------- products
@pytest.mark.parametrize("seed", range(4))
def test_matmul_add_matches_scipy(seed):
    A = rand_csr(80, 0.08, seed)
    B = rand_csr(80, 0.08, seed + 100)
    I0 = rand_csr(80, 0.05, seed + 200)
    C = matmul_add(A, B, I0)
    ref = (A.to_scipy() @ B.to_scipy() + I0.to_scipy()).toarray()
    np.testing.assert_allclose(C.to_dense(), ref, rtol=1e-13, atol=1e-15)
    # structural sanity: sorted unique columns, no stored zeros
    for r in range(C.n):
        cols = C.col[C.rowptr[r]:C.rowptr[r + 1]]
        assert np.all(np.diff(cols) > 0)
    assert np.all(C.val != 0.0)


def test_matmul_integer_exact_and_cancellation_dropped():
    rng = np.random.default_rng(3)
    A = rng.integers(-3, 4, (12, 12)).astype(float)
    B = rng.integers(-3, 4, (12, 12)).astype(float)
    C = matmul_add(CSR.from_dense(A), CSR.from_dense(B))
    assert np.array_equal(C.to_dense(), A @ B)
    assert C.nnz == np.count_nonzero(A @ B)


def test_matmul_rounding_order_is_init_then_ascending_k_fma():
    # one output entry with four terms; the expected value is the chain of
    # correctly rounded fused multiply-adds, init first, then k ascending
    a = [0.1, 1e16, -1e16, 0.3]
    b = [0.7, 1.0 / 3.0, 1.0 / 3.0, 0.9]
    init = 1e-3
    A = CSR(4, np.array([0, 4, 4, 4, 4], np.int32), np.arange(4, dtype=np.int32), np.array(a))
    B = CSR(4, np.array([0, 1, 2, 3, 4], np.int32), np.zeros(4, np.int32), np.array(b))
    I0 = CSR(4, np.array([0, 1, 1, 1, 1], np.int32), np.zeros(1, np.int32), np.array([init]))
    acc = init
    for x, y in zip(a, b):
        acc = fma_exact(x, y, acc)
    C = matmul_add(A, B, I0)
    assert C.nnz == 1 and C.val[0] == acc
    # a plain left-to-right sum without fusion gives a different double here
    plain = init
    for x, y in zip(a, b):
        plain = plain + x * y
    assert plain != acc


def test_axpy_identity_and_matrix():
    M = rand_csr(30, 0.1, 1)
    X = rand_csr(30, 0.1, 2)
    Y = axpy(0.37, M, X, 30)
    np.testing.assert_array_equal(
        Y.to_dense(),
        np.vectorize(fma_exact)(0.37, M.to_dense(), X.to_dense()) * (M.to_dense() != 0)
        + X.to_dense() * (M.to_dense() == 0))
    Yi = axpy(2.5, None, None, 5)
    np.testing.assert_array_equal(Yi.to_dense(), 2.5 * np.eye(5))


# ------------------------------------------------------------- Algorithm 1
def test_alg1_hand_worked_two_passes():
    # eps_g = 1, e_r = 0.1 (bound 1.1).
    # pass 1: eps_f = 1; candidates |x| <= 1 -> column sums 1.7, 1.0, 0.05;
    #         c_1 = 1.7 > 1.1, m_1 = 1.7
    # pass 2: eps_f = 1/1.7; candidates -> column sums 0, 0.5+0.3+0.2 = 1.0, 0.05
    #         c_2 = 1.0 <= 1.1: stop.  Kept: 0.9, 0.8, 5, 2.
    C = CSR.from_dense(np.array([[0.9, 0.5, 2.0], [0.8, 0.3, 0.0], [5.0, 0.2, 0.05]]))
    r = alg1(C, 1.0, 0.1)
    assert r.iters == 2
    c1 = math.fsum([0.9, 0.8])  # correctly rounded column sum of pass 1
    assert r.eps_f == 1.0 / (c1 / 1.0)
    assert r.c == 1.0
    np.testing.assert_array_equal(r.kept.to_dense(),
                                  np.array([[0.9, 0.0, 2.0], [0.8, 0.0, 0.0], [5.0, 0.0, 0.0]]))


def test_alg1_single_pass_and_degenerate_thresholds():
    C = CSR.from_dense(np.array([[3.0, 0.01], [0.02, 4.0]]))
    r = alg1(C, 1.0, 0.1)  # candidates 0.01, 0.02: c = 0.02 <= 1.1
    assert r.iters == 1 and r.eps_f == 1.0 and r.c == 0.02
    assert r.kept.nnz == 2
    # eps_g = 0: nothing is a candidate, every nonzero stays (unfiltered PS)
    r0 = alg1(C, 0.0, 0.1)
    assert r0.kept.nnz == 4 and r0.c == 0.0
    # eps_g >= 1 still runs the first pass (reading: c_0 = +inf)
    rb = alg1(C, 100.0, 0.1)
    assert rb.iters == 1 and rb.kept.nnz == 0 and rb.c == math.fsum([0.01, 4.0])  # column 1
    # ties at eps_f are dropped: keep means |x| > eps_f strictly, and the
    # dropped tie counts in c (c is the norm of every entry not kept)
    rt = alg1(CSR.from_dense(np.array([[1.0, 0.0], [0.0, 0.5]])), 1.0, 10.0)
    assert rt.kept.nnz == 0
    assert rt.iters == 1 and rt.c == 1.0


# Hand traces with more passes.  Every value below is a multiple of 1/20 or a
# power of two, so the column sums are exact and the trace can be done on
# paper; several entries sit exactly on a later eps_f, so the ties decide the
# column sums (and with them the whole trajectory) at every pass.
#
#   column 0: 1.0, 0.5, 0.5     column 2: 0.25, 0.25, 0.25
#   column 1: 0.5, 0.5, 0.5     column 3: 0.3, 0.3, 0.3, 0.3 (4 x 4 case only)
#
# eps_g = 1, e_r = 0.1, loop while c > 1.1:
#   pass 1: eps_f = 1        candidates: every entry (1.0 is a tie)
#           sums 2.0, 1.5, 0.75 (, 1.2)  -> c_1 = 2.0, m_1 = 2
#   pass 2: eps_f = 1/2      candidates: the 0.5 ties, 0.25, 0.3
#           sums 1.0, 1.5, 0.75 (, 1.2)  -> c_2 = 1.5, m_2 = 3
#   pass 3: eps_f = fl(1/3)  candidates: 0.25 (, 0.3)
#           sums 0, 0, 0.75 (, 1.2)      -> 3 x 3: c_3 = 0.75, stop
#                                           4 x 4: c_3 = 1.2, m_3 = 1.2 / fl(1/3)
#   pass 4: eps_f = 1 / m_3  (0.2777...) candidates: 0.25 only
#           sums 0, 0, 0.75, 0           -> c_4 = 0.75, stop
# Keeping the ties in c_1 and c_2 matters: without the tie 1.0 in pass 1 the
# trace would take c_1 = 1.5 and eps_f = 2/3 next.
COLS3 = [[1.0, 0.5, 0.25], [0.5, 0.5, 0.25], [0.5, 0.5, 0.25]]


def test_alg1_hand_worked_three_passes_with_ties():
    r = alg1(CSR.from_dense(np.array(COLS3)), 1.0, 0.1)
    assert r.iters == 3
    assert r.eps_f == 1.0 / 3.0  # eps_g / m_2 with m_2 = c_2 / eps_f = 1.5 / 0.5 = 3
    assert r.c == 0.75
    np.testing.assert_array_equal(
        r.kept.to_dense(), np.array([[1.0, 0.5, 0.0], [0.5, 0.5, 0.0], [0.5, 0.5, 0.0]]))


def test_alg1_hand_worked_four_passes_with_ties():
    D = np.zeros((5, 5))
    D[:3, :3] = COLS3
    D[:4, 3] = 0.3
    D[0, 4], D[4, 4] = 4.0, 3.0  # never candidates
    r = alg1(CSR.from_dense(D), 1.0, 0.1)
    assert r.iters == 4
    eps_f3 = 1.0 / 3.0
    m_3 = 1.2 / eps_f3  # c_3 = 0.3 * 4 exactly rounded = fl(1.2); m_3 rounds to fl(3.6)
    assert m_3 == 3.6
    assert r.eps_f == 1.0 / 3.6
    assert 0.25 < r.eps_f < 0.3
    assert r.c == 0.75
    K = D.copy()
    K[:3, 2] = 0.0
    np.testing.assert_array_equal(r.kept.to_dense(), K)


@pytest.mark.parametrize("seed", range(8))
def test_alg1_invariants(seed):
    rng = np.random.default_rng(seed)
    n = 40
    D = rng.standard_normal((n, n)) * 10.0 ** rng.uniform(-16, 0, (n, n))
    D[rng.uniform(size=(n, n)) < 0.5] = 0.0
    C = CSR.from_dense(D)
    eps_g = 10.0 ** rng.uniform(-12, -4)
    e_r = 0.1
    r = alg1(C, eps_g, e_r)
    K = r.kept.to_dense()
    drop = D - K
    # kept = entries strictly above the final eps_f, values untouched
    assert np.array_equal(K != 0, np.abs(D) > r.eps_f)
    assert np.array_equal(K[K != 0], D[K != 0])
    # the guarantee of Alg. 1: ||C - C_hat||_1 <= eps_g (1 + e_r)
    cn = max(math.fsum(np.abs(drop[:, j])) for j in range(n))
    assert cn == r.c
    assert r.c <= eps_g * (1 + e_r)
    # eps_f follows the paper's sequence eps_g / m_i: it never exceeds eps_g
    assert r.eps_f <= eps_g
    if r.iters == 1:
        assert r.eps_f == eps_g
