"""GPU parity of the building blocks through the C ABI: one fused product
(weighted sum + A B) and Algorithm 1 against the oracle, bit for bit; exact
1-norms; chunked rows; malformed input and bounded failure statuses."""
import numpy as np
import pytest
import scipy.sparse as sp

import synthetic as syn
from gpu_helpers import assert_csr_bitwise, dev, ocsr
from oracle import CSR, alg1, axpy, matmul_add, norm1

pytestmark = pytest.mark.gpu

psf = pytest.importorskip("paper_2208_05683_gb300")


def rand_csr(n, density, seed, scale=1.0, mag_spread=0.0):
    rng = np.random.default_rng(seed)
    m = sp.random(n, n, density=density, random_state=rng, format="csr",
                  data_rvs=lambda k: rng.uniform(-1, 1, k) * scale * 10.0 ** (-mag_spread * rng.uniform(0, 1, k)))
    return CSR.from_scipy(m)


def oracle_product(A, B, addends, n):
    X = None
    for alpha, M in addends:
        X = axpy(alpha, M, X, n)
    if A is None:
        return X if X is not None else CSR.empty(n)
    return matmul_add(A, B, X)


@pytest.mark.parametrize("n,density,seed", [(1, 1.0, 0), (37, 0.2, 1), (100, 0.05, 2), (1000, 0.01, 3),
                                            (3001, 0.002, 4)])
def test_product_bitwise(n, density, seed):
    A = rand_csr(n, density, seed)
    B = rand_csr(n, density, seed + 10)
    M1 = rand_csr(n, density, seed + 20)
    add = [(0.5, None), (-1.25, M1), (3.0, B)]
    ref = oracle_product(A, B, add, n)
    got = psf.product_filter(dev(A), dev(B), [(a, dev(M) if M is not None else None) for a, M in add], 0.0)
    assert_csr_bitwise(got.csr, ref, f"n={n}")
    assert got.steps[0]["nnz_pre"] == ref.nnz


def test_pure_weighted_sum_and_empty():
    n = 50
    M = rand_csr(n, 0.1, 5)
    ref = oracle_product(None, None, [(2.0, None), (0.75, M)], n)
    got = psf.product_filter(None, None, [(2.0, None), (0.75, dev(M))], 0.0)
    assert_csr_bitwise(got.csr, ref)
    E = CSR.empty(n)
    got = psf.product_filter(dev(E), dev(M), [], 0.0)
    assert got.csr.nnz == 0


@pytest.mark.parametrize("seed", range(4))
def test_product_then_alg1_bitwise(seed):
    n = 400
    A = rand_csr(n, 0.03, seed, mag_spread=12)
    B = rand_csr(n, 0.03, seed + 50, mag_spread=12)
    C = matmul_add(A, B)
    rng = np.random.default_rng(seed)
    thr = 10.0 ** rng.uniform(-14, -8)
    e_r = 0.1
    ref = alg1(C, thr / (1.0 + e_r), e_r)
    got = psf.product_filter(dev(A), dev(B), [], thr, e_r)
    assert_csr_bitwise(got.csr, ref.kept, f"seed {seed}")
    st = got.steps[0]
    assert st["eps_f"] == ref.eps_f and st["iters"] == ref.iters and st["dropped"] == ref.c
    assert st["nnz_pre"] == C.nnz and st["nnz_post"] == ref.kept.nnz
    assert st["dropped"] <= thr


def test_alg1_many_passes_bitwise():
    # entries spread over many decades with a tight threshold force several passes
    n = 300
    A = rand_csr(n, 0.05, 11, mag_spread=20)
    B = rand_csr(n, 0.05, 12, mag_spread=20)
    C = matmul_add(A, B)
    ref = alg1(C, 1e-6 / 1.1, 0.1)
    assert ref.iters >= 2
    got = psf.product_filter(dev(A), dev(B), [], 1e-6, 0.1)
    assert_csr_bitwise(got.csr, ref.kept)
    assert got.steps[0]["iters"] == ref.iters and got.steps[0]["eps_f"] == ref.eps_f


def test_alg1_pass_cap_returns_enotconv():
    n = 300
    A = rand_csr(n, 0.05, 11, mag_spread=20)
    B = rand_csr(n, 0.05, 12, mag_spread=20)
    with pytest.raises(psf.PsfError) as e:
        psf.product_filter(dev(A), dev(B), [], 1e-6, 0.1, maxit=1)
    assert e.value.code == 4  # ENOTCONV, from the device status word


def test_wide_rows_take_several_chunks():
    # rows spanning more than one 8192-column bitmap chunk and rows with more
    # than 1024 entries (several accumulator chunks)
    n = 20000
    rng = np.random.default_rng(3)
    rows, cols = [], []
    for r in range(0, n, 7):
        c = rng.choice(n, size=rng.integers(1, 40), replace=False)
        rows += [r] * len(c)
        cols += list(c)
    A = CSR.from_scipy(sp.csr_matrix((rng.uniform(-1, 1, len(rows)), (rows, cols)), shape=(n, n)))
    B = rand_csr(n, 0.0015, 9)  # ~30 entries per row spread over all columns
    ref = matmul_add(A, B)
    assert max(np.diff(ref.rowptr)) > 1024
    got = psf.product_filter(dev(A), dev(B), [(1.0, None)], 0.0)
    ref2 = matmul_add(A, B, axpy(1.0, None, None, n))
    assert_csr_bitwise(got.csr, ref2, "wide")


@pytest.mark.parametrize("seed", range(3))
def test_norm1_bitwise(seed):
    M = rand_csr(2000, 0.005, seed, scale=10.0 ** (seed * 50), mag_spread=30)
    assert psf.norm1(dev(M)) == norm1(M)
    Z = ocsr(syn.laplacian_2d(64))
    assert psf.norm1(dev(Z)) == 4.0


def test_malformed_input_is_rejected():
    n = 5
    good = CSR.from_dense(np.eye(n))
    bad_order = (np.array([0, 2, 2, 2, 2, 2], np.int32), np.array([3, 1], np.int32), np.array([1.0, 2.0]))
    bad_range = (np.array([0, 1, 1, 1, 1, 1], np.int32), np.array([7], np.int32), np.array([1.0]))
    bad_val = (np.array([0, 1, 1, 1, 1, 1], np.int32), np.array([0], np.int32), np.array([np.nan]))
    # every case below is caught by the validation pass before any kernel
    # indexes with the input: row pointers first, then the row's columns
    i32 = lambda *x: np.array(x, np.int32)
    bad_dup = (i32(0, 2, 2, 2, 2, 2), i32(1, 1), np.array([1.0, 2.0]))          # repeated column
    bad_neg = (i32(0, 1, 1, 1, 1, 1), i32(-1), np.array([1.0]))                # negative column
    bad_inf = (i32(0, 1, 1, 1, 1, 1), i32(0), np.array([np.inf]))              # non-finite value
    bad_dec = (i32(0, 2, 1, 2, 2, 2), i32(0, 1), np.array([1.0, 2.0]))         # decreasing row pointers
    bad_first = (i32(1, 1, 1, 1, 1, 1), i32(0), np.array([1.0]))               # rowptr[0] != 0
    bad_last = (i32(0, 1, 1, 1, 1, 0), i32(0), np.array([1.0]))                # rowptr[n] != nnz
    cases = (bad_order, bad_range, bad_val, bad_dup, bad_neg, bad_inf, bad_dec, bad_first, bad_last)
    for i, bad in enumerate(cases):
        with pytest.raises(psf.PsfError) as e:
            psf.product_filter(dev(bad), dev(good), [], 0.0)
        assert e.value.code == 1, i
        with pytest.raises(psf.PsfError) as e:
            psf.Series(syn.coeffs("exp"), 1e-12).eval(dev(bad))
        assert e.value.code == 1, i
        with pytest.raises(psf.PsfError) as e:
            psf.Series(syn.coeffs("exp"), 1e-12).eval_host(*bad)
        assert e.value.code == 1, i


def test_rows_of_609_to_640_entries_take_every_slot():
    # banded factors whose product rows have 600..640 entries: the narrow
    # accumulator keeps a_rk in its last 32 slots (608 left), so such a row
    # takes all 640 slots with a_rk read from A's row instead of two column
    # chunks; with and without the filter, against the oracle bit for bit
    rng = np.random.default_rng(21)
    n = 2000

    def band(h):
        rows, cols = [], []
        for d in range(-h, h + 1):
            r = np.arange(max(0, -d), min(n, n - d))
            rows.append(r)
            cols.append(r + d)
        rows, cols = np.concatenate(rows), np.concatenate(cols)
        vals = rng.uniform(-1, 1, len(rows)) * 10.0 ** (-12 * rng.uniform(0, 1, len(rows)))
        return CSR.from_scipy(sp.csr_matrix((vals, (rows, cols)), shape=(n, n)))

    A, B = band(150), band(160)
    C = matmul_add(A, B, axpy(0.5, None, None, n))
    lens = np.diff(C.rowptr)
    assert ((lens > 608) & (lens <= 640)).sum() > n // 2
    got = psf.product_filter(dev(A), dev(B), [(0.5, None)], 0.0)
    assert_csr_bitwise(got.csr, C, "unfiltered")
    ref = alg1(C, 1e-14 / 1.1, 0.1)
    got = psf.product_filter(dev(A), dev(B), [(0.5, None)], 1e-14, 0.1)
    assert_csr_bitwise(got.csr, ref.kept, "filtered")
    assert got.steps[0]["iters"] == ref.iters and got.steps[0]["eps_f"] == ref.eps_f
