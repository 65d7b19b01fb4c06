"""End-to-end pins for the oracle's Algorithm 2: closed forms, exact special
cases, exact rational PS = Horner, library routines and invariants."""
import math

import numpy as np
import pytest
import scipy.linalg

import synthetic as syn
from closed_forms import (cos_lap2d_column, exp_lap2d_column, frac_horner, fun_lap1d,
                          norm1_dense)
from oracle import CSR, horner_dense, planner, psscf


def csr(t):
    return CSR(len(t[0]) - 1, *t)


def test_exp_lap1d_n256_within_tol_of_dst_closed_form():
    Z = csr(syn.laplacian_1d(256))
    r = psscf(Z, syn.coeffs("exp"), 1e-12)
    ref = fun_lap1d(256, -0.5, np.exp)
    err = norm1_dense(r.F.to_dense() - ref)
    assert err <= 1e-12
    # every filter respected its bound (Algorithm 2, Eqs. 11 and 14)
    for s in r.steps:
        assert s.c <= s.threshold
        assert s.nnz_post <= s.nnz_pre
    # the filter actually removed entries in the giant steps
    assert any(s.nnz_post < s.nnz_pre for s in r.steps if s.kind == "giant")


def test_filtered_close_to_unfiltered_within_budget():
    # Eq. (27)/(35): the filtering error is bounded by the budget (first order)
    Z = csr(syn.laplacian_1d(256))
    a = syn.coeffs("exp")
    rf = psscf(Z, a, 1e-12)
    ru = psscf(Z, a, 1e-12, filtered=False)
    assert (ru.plan.N, ru.plan.q) == (rf.plan.N, rf.plan.q)
    assert ru.F.nnz > rf.F.nnz
    assert norm1_dense(rf.F.to_dense() - ru.F.to_dense()) <= rf.plan.budget


@pytest.mark.parametrize("m", [16, 32])
def test_exp_and_cos_lap2d_kronecker(m):
    n = m * m
    Z = csr(syn.laplacian_2d(m))
    Z1 = fun_lap1d(m, -0.5, lambda x: x)  # the 1D factor, Z = Z1 (+) Z1
    E1 = scipy.linalg.expm(Z1)
    C1, S1 = scipy.linalg.cosm(Z1), scipy.linalg.sinm(Z1)
    for kind in ("exp", "cos"):
        r = psscf(Z, syn.coeffs(kind), 1e-12)
        F = r.F.to_dense()
        col = exp_lap2d_column if kind == "exp" else (lambda _, c: cos_lap2d_column(C1, S1, c))
        ref = np.stack([col(E1, c) for c in range(n)], axis=1)
        assert norm1_dense(F - ref) <= 1e-12, kind


@pytest.mark.parametrize("seed", range(3))
def test_banded_random_against_scipy_expm(seed):
    Z = csr(syn.banded_random(300, 4, seed, 2.0))
    r = psscf(Z, syn.coeffs("exp"), 1e-12)
    ref = scipy.linalg.expm(Z.to_dense())
    # scipy's own error is a few ulps of ||exp(Z)||
    assert norm1_dense(r.F.to_dense() - ref) <= 1e-12 + 1e-14 * norm1_dense(ref)


@pytest.mark.parametrize("seed", [0, 3])
def test_banded_random_cos_against_scipy_cosm(seed):
    # cos uses the literal series with zero odd coefficients (Eq. 40)
    Z = csr(syn.banded_random(300, 4, seed, 2.0))
    r = psscf(Z, syn.coeffs("cos"), 1e-12)
    ref = scipy.linalg.cosm(Z.to_dense())
    assert norm1_dense(r.F.to_dense() - ref) <= 1e-12 + 1e-14 * norm1_dense(ref)


def test_exp_times_exp_minus_is_identity():
    Z = csr(syn.banded_random(200, 3, 11, 2.0))
    Zm = CSR(Z.n, Z.rowptr, Z.col, -Z.val)
    E = psscf(Z, syn.coeffs("exp"), 1e-12).F.to_dense()
    Em = psscf(Zm, syn.coeffs("exp"), 1e-12).F.to_dense()
    # ||E Em - I|| <= ||E - e^Z|| ||Em|| + ||e^Z|| ||Em - e^-Z|| <= tol (||Em|| + ||e^Z||)
    bound = 1e-12 * (norm1_dense(Em) + norm1_dense(E) + 1e-12)
    assert norm1_dense(E @ Em - np.eye(Z.n)) <= bound * 1.01


def test_diagonal_matrix_gives_scalar_series():
    d = np.linspace(-3.0, 2.0, 50)
    Z = CSR.from_dense(np.diag(d))
    for kind, fn in (("exp", np.exp), ("cos", np.cos), ("sinh", np.sinh), ("cosh", np.cosh)):
        F = psscf(Z, syn.coeffs(kind), 1e-12).F.to_dense()
        assert np.count_nonzero(F - np.diag(np.diag(F))) == 0
        assert np.max(np.abs(np.diag(F) - fn(d))) <= 1e-12, kind


def test_nilpotent_shift_exact_entries():
    # Z = c J (J the upper shift): exp(Z)_{i,i+k} = c^k / k!, zero for k >= n
    n, c = 12, 0.75
    J = np.diag(np.full(n - 1, c), 1)
    Z = CSR.from_dense(J)
    ru = psscf(Z, syn.coeffs("exp"), 1e-14, filtered=False)
    ref = sum(np.linalg.matrix_power(J, k) / math.factorial(k) for k in range(n))
    Fu = ru.F.to_dense()
    np.testing.assert_allclose(Fu, ref, rtol=4e-16, atol=0)
    rf = psscf(Z, syn.coeffs("exp"), 1e-14)
    Ff = rf.F.to_dense()
    assert norm1_dense(Ff - ref) <= 1e-14
    # kept entries are the exact values; only diagonals below the threshold go
    kept = Ff != 0
    np.testing.assert_allclose(Ff[kept], ref[kept], rtol=4e-16)


@pytest.mark.parametrize("N", list(range(3, 31)))
def test_unfiltered_ps_equals_exact_horner(N):
    # integer Z and coefficients: FP64 arithmetic is exact, so the PS result
    # must equal the exact rational Horner value bit for bit
    rng = np.random.default_rng(N)
    n = 5
    Zd = np.eye(n) + np.diag(np.ones(n - 1), 1)  # (I + J)^k: binomial entries
    if N % 3 == 0:
        Zd = rng.integers(-1, 2, (n, n)).astype(float) * (np.abs(np.subtract.outer(
            np.arange(n), np.arange(n))) <= 1)
        if N > 16:
            Zd = np.triu(Zd)
            np.fill_diagonal(Zd, rng.integers(-1, 2, n))
    a = [float(x) for x in rng.integers(-4, 5, N)]
    a[-1] = a[-1] or 3.0
    Z = CSR.from_dense(Zd)
    r = psscf(Z, a, 1.0, poly=True, filtered=False)
    ref = np.array(frac_horner(Zd.tolist(), a), dtype=float)
    assert np.array_equal(r.F.to_dense(), ref)
    assert r.products == planner.mult_count(N)


def test_dense_horner_matches_expm():
    Z = syn.banded_random(40, 3, 2, 1.5)
    Zd = csr(Z).to_dense()
    H = horner_dense(Zd, syn.coeffs("exp"), 30)
    np.testing.assert_allclose(H, scipy.linalg.expm(Zd), rtol=0, atol=1e-14)


def test_poly_mode_uses_all_coefficients_and_eq28():
    Z = csr(syn.laplacian_1d(64))
    a = syn.coeffs("exp")[:15]
    r = psscf(Z, a, 1e-10, poly=True)
    p = r.plan
    assert p.N == 15 and p.trunc == 0.0 and p.budget == 1e-10
    H = horner_dense(Z.to_dense(), a, 15)
    assert norm1_dense(r.F.to_dense() - H) <= 1e-10


def test_n1_and_n2_need_no_products():
    Z = csr(syn.laplacian_1d(8))
    r1 = psscf(Z, [2.5], 1.0, poly=True)
    np.testing.assert_array_equal(r1.F.to_dense(), 2.5 * np.eye(8))
    r2 = psscf(Z, [2.5, -1.0], 1.0, poly=True)
    assert r2.products == 0
    np.testing.assert_array_equal(r2.F.to_dense(), 2.5 * np.eye(8) - Z.to_dense())


def test_zero_matrix():
    Z = CSR.empty(6)
    r = psscf(Z, syn.coeffs("cos"), 1e-12)
    assert r.plan.N == 1
    np.testing.assert_array_equal(r.F.to_dense(), np.eye(6))


def test_s_override():
    Z = csr(syn.laplacian_1d(256))
    a = syn.coeffs("exp")
    r = psscf(Z, a, 1e-12, s=5)
    assert (r.plan.q, r.plan.b) == (5, 4) and r.products == 7
    ref = fun_lap1d(256, -0.5, np.exp)
    assert norm1_dense(r.F.to_dense() - ref) <= 1e-12


@pytest.mark.parametrize("w,kind", [(1, "exp"), (2, "exp"), (4, "exp"), (1, "cos"), (3, "cos")])
def test_banded_normal_against_40_digit_reference(w, kind):
    # the paper's second matrix family (banded, N(0, 1) entries), eps_tol =
    # 1e-14, n = 40: within the tolerance (plus a few ulps of ||f(|Z|)||_1 for
    # the rounding the first-order bound leaves out) of f(Z) computed in
    # 40-digit arithmetic.  (At n = 60, w = 1 and 2, scipy's expm was off by
    # 1e-12..1e-11 on these non-normal matrices, the filtered scheme by 3e-15
    # and 2e-14: a library routine is not a tight enough pin here.)
    mpmath = pytest.importorskip("mpmath")
    n = 40
    Z = csr(syn.banded_normal(n, w, 1000 * w + 3))
    Zd = Z.to_dense()
    r = psscf(Z, syn.coeffs(kind), 1e-14)
    with mpmath.workdps(40):
        M = mpmath.matrix(Zd.tolist())
        E = mpmath.expm(M, method="taylor") if kind == "exp" else mpmath.cosm(M)
        ref = np.array([[float(E[i, j]) for j in range(n)] for i in range(n)])
    fa = scipy.linalg.expm(np.abs(Zd)) if kind == "exp" else scipy.linalg.coshm(np.abs(Zd))
    margin = 8 * 2.0 ** -53 * norm1_dense(fa)
    assert norm1_dense(r.F.to_dense() - ref) <= 1e-14 + margin, (w, kind)
