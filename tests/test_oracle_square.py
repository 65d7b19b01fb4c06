"""Pins of the oracle's W = Z^2 substitution for even and odd series.

Even series: f(Z) = g(Z^2) with c_k = a_{2k}; odd series: f(Z) = Z g(Z^2)
with c_k = a_{2k+1}.  Algorithm 2 then runs on W = Z^2, with the norms of W
bounded by z_{2i} of Z (Eq. 37 and Lemma 1 applied to Z).  Pinned by exact
integer arithmetic, library routines (scipy's cosm, coshm, sinhm), f(Z) in
40-digit arithmetic on non-normal matrices, the Kronecker closed form of the
2D Laplacian, and the relation between the truncation of the two plans.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import synthetic as syn
from closed_forms import cos_lap2d_column, frac_horner, fun_lap1d, norm1_dense
from oracle import CSR, planner, power_norms, psscf


def csr(t):
    return CSR(len(t[0]) - 1, *t)


def test_split_even_odd():
    c, odd = planner.split_even_odd(syn.coeffs("cos"))
    assert not odd
    assert c[:4] == [1.0, -0.5, 1.0 / 24.0, -1.0 / 720.0]
    c, odd = planner.split_even_odd(syn.coeffs("sinh"))
    assert odd
    assert c[:3] == [1.0, 1.0 / 6.0, 1.0 / 120.0]
    assert planner.split_even_odd(syn.coeffs("cosh"))[1] is False
    assert planner.split_even_odd([0.0, 0.0, 0.0]) == ([0.0, 0.0], False)
    with pytest.raises(ValueError):
        planner.split_even_odd(syn.coeffs("exp"))


@pytest.mark.parametrize("N", list(range(3, 31)))
@pytest.mark.parametrize("odd", [False, True])
def test_unfiltered_square_equals_exact_polynomial(N, odd):
    # integer Z and coefficients: every FP64 operation is exact, so the
    # substituted scheme must equal the exact rational polynomial bit for bit
    rng = np.random.default_rng(100 * N + odd)
    n = 5
    Zd = np.eye(n) + np.diag(np.ones(n - 1), 1)  # (I + J)^k: binomial entries
    if N % 3 == 0:
        Zd = np.triu(rng.integers(-1, 2, (n, n)).astype(float)) * (
            np.abs(np.subtract.outer(np.arange(n), np.arange(n))) <= 1)
    a = [0.0] * N
    for i in range(1 if odd else 0, N, 2):
        a[i] = float(rng.integers(-4, 5))
    last = N - 1 if (N - 1) % 2 == int(odd) else N - 2
    a[last] = a[last] or 3.0
    Z = CSR.from_dense(Zd)
    r = psscf(Z, a, 1.0, poly=True, filtered=False, square=True)
    ref = np.array(frac_horner(Zd.tolist(), a), dtype=float)
    assert np.array_equal(r.F.to_dense(), ref)
    NW = len(a[1 if odd else 0::2])
    assert r.plan.N == NW
    # W = Z Z, then Eq. (5) in W, then F = Z G for an odd series
    assert r.products == 1 + planner.mult_count(NW) + int(odd)


@pytest.mark.parametrize("kind", ["cos", "cosh"])
def test_even_plan_truncates_where_the_direct_plan_does(kind):
    # With z^W_i = z_{2i}, the tail of g at m sums the same terms in the same
    # order as the tail of f at 2m - 1 and 2m, so Eq. (34) gives
    # N_W = (N + 1) / 2 and the same truncation bound, bit for bit.
    a = syn.coeffs(kind)
    c, _ = planner.split_even_odd(a)
    for seed in range(4):
        Z = csr(syn.banded_random(120, 3, seed, 1.0 + seed))
        norms = power_norms(Z)
        for tol in (1e-8, 1e-12, 1e-14):
            p = planner.plan(a, tol, norms)
            pw = planner.plan(c, tol, norms, stride=2)
            assert p.N % 2 == 1
            assert pw.N == (p.N + 1) // 2
            assert pw.trunc == p.trunc
            assert pw.z[:6] == [norms[2 * i] for i in range(6)]


def test_lap2d_cos_plan_by_hand():
    # -0.5 L2D of a 128 x 128 grid: ||Z^i||_1 = 4^i, so z^W_i = 16^i and
    # alpha_10 = 4; cos needs N = 27 directly, hence N_W = 14:
    # q = floor(sqrt(13)) = 3, b = ceil(14/3) = 5, 14 - 3*4 = 2 so g = 0, and
    # 3 + 5 - 2 = 6 products in W (Eq. 5) plus W = Z Z: 7 against 9.
    norms = [4.0 ** i for i in range(11)]
    a = syn.coeffs("cos")
    p = planner.plan(a, 1e-12, norms)
    c, _ = planner.split_even_odd(a)
    pw = planner.plan(c, 1e-12, norms, stride=2)
    assert (p.N, p.q, p.b, p.g) == (27, 5, 6, 0)
    assert (pw.N, pw.q, pw.b, pw.g) == (14, 3, 5, 0)
    assert pw.z[:12] == [16.0 ** i for i in range(12)]
    assert planner.mult_count(p.N) == 9 and planner.mult_count(pw.N) + 1 == 7


@pytest.mark.parametrize("seed", [0, 5])
def test_banded_random_against_scipy(seed):
    Z = csr(syn.banded_random(300, 4, seed, 2.5))
    Zd = Z.to_dense()
    for kind, fn in (("cos", scipy.linalg.cosm), ("cosh", scipy.linalg.coshm), ("sinh", scipy.linalg.sinhm)):
        r = psscf(Z, syn.coeffs(kind), 1e-12, square=True)
        ref = fn(Zd)
        assert norm1_dense(r.F.to_dense() - ref) <= 1e-12 + 1e-14 * norm1_dense(ref), kind
        for s in r.steps:
            assert s.c <= s.threshold or s.threshold == 0.0
            assert s.nnz_post <= s.nnz_pre


def test_sinh_tolerance_is_scaled_by_the_norm_of_z():
    Z = csr(syn.banded_random(200, 3, 2, 3.0))
    r = psscf(Z, syn.coeffs("sinh"), 1e-10, square=True)
    c, odd = planner.split_even_odd(syn.coeffs("sinh"))
    assert odd
    pw = planner.plan(c, 1e-10 / r.norms[1], r.norms, stride=2)
    assert (r.plan.N, r.plan.budget) == (pw.N, pw.budget)
    assert r.steps[-1].kind == "odd"
    ref = scipy.linalg.sinhm(Z.to_dense())
    assert norm1_dense(r.F.to_dense() - ref) <= 1e-10


def test_lap2d_cos_kronecker():
    m = 16
    n = m * m
    Z = csr(syn.laplacian_2d(m))
    Z1 = fun_lap1d(m, -0.5, lambda x: x)
    C1, S1 = scipy.linalg.cosm(Z1), scipy.linalg.sinm(Z1)
    r = psscf(Z, syn.coeffs("cos"), 1e-12, square=True)
    ref = np.stack([cos_lap2d_column(C1, S1, c) for c in range(n)], axis=1)
    assert norm1_dense(r.F.to_dense() - ref) <= 1e-12
    direct = psscf(Z, syn.coeffs("cos"), 1e-12)
    assert r.products < direct.products


def test_diagonal_and_zero_matrices():
    d = np.linspace(-3.0, 2.0, 40)
    Z = CSR.from_dense(np.diag(d))
    for kind, fn in (("cos", np.cos), ("sinh", np.sinh), ("cosh", np.cosh)):
        F = psscf(Z, syn.coeffs(kind), 1e-12, square=True).F.to_dense()
        assert np.count_nonzero(F - np.diag(np.diag(F))) == 0
        assert np.max(np.abs(np.diag(F) - fn(d))) <= 1e-12, kind
    zero = CSR.empty(7)
    assert np.array_equal(psscf(zero, syn.coeffs("cos"), 1e-12, square=True).F.to_dense(), np.eye(7))
    r = psscf(zero, syn.coeffs("sinh"), 1e-12, square=True)
    assert r.F.nnz == 0 and r.plan.N == 1 and math.isinf(r.plan.budget)


def test_odd_single_term_is_a_scaled_copy_of_z():
    # a tolerance far above every term truncates g to c_0: F = Z (c_0 I) = a_1 Z
    Z = csr(syn.banded_random(60, 2, 4, 0.5))
    r = psscf(Z, syn.coeffs("sinh"), 10.0, square=True)
    assert r.plan.N == 1
    assert np.array_equal(r.F.to_dense(), Z.to_dense())


@pytest.mark.parametrize("kind", ["cos", "cosh", "sinh"])
def test_square_mode_on_banded_normal_against_40_digit_reference(kind):
    # non-normal banded N(0, 1) matrices (the paper's second family), eps_tol =
    # 1e-12: the substituted scheme is within the tolerance (plus a few ulps of
    # ||f(|Z|)||_1 of rounding) of f(Z) in 40-digit arithmetic; sinh and cosh
    # from (e^Z -/+ e^-Z) / 2
    mpmath = pytest.importorskip("mpmath")
    n = 30
    Z = csr(syn.banded_normal(n, 2, 77))
    Zd = Z.to_dense()
    r = psscf(Z, syn.coeffs(kind), 1e-12, square=True)
    with mpmath.workdps(40):
        M = mpmath.matrix(Zd.tolist())
        if kind == "cos":
            E = mpmath.cosm(M)
        else:
            Ep, Em = mpmath.expm(M, method="taylor"), mpmath.expm(-M, method="taylor")
            E = (Ep - Em) / 2 if kind == "sinh" else (Ep + Em) / 2
        ref = np.array([[float(E[i, j]) for j in range(n)] for i in range(n)])
    margin = 8 * 2.0 ** -53 * norm1_dense(scipy.linalg.coshm(np.abs(Zd)) + scipy.linalg.sinhm(np.abs(Zd)))
    assert norm1_dense(r.F.to_dense() - ref) <= 1e-12 + margin, kind
