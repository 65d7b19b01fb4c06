"""Pins for the oracle's a-priori analysis (Eqs. 5, 6, 24-28, 34-37)."""
import math
from fractions import Fraction

import numpy as np
import pytest

import synthetic as syn
from oracle import CSR, planner, power_norms, psscf


def test_ps_split_hand_values():
    # Eq. (6) worked by hand
    assert planner.ps_split(20) == (4, 5, 0)   # 4*4 = 16 < 20
    assert planner.ps_split(28) == (5, 6, 0)   # 28 - 25 = 3
    assert planner.ps_split(10) == (3, 4, 1)   # 10 - 3*3 = 1
    assert planner.ps_split(17) == (4, 5, 1)   # 17 - 16 = 1
    assert planner.ps_split(5) == (2, 3, 1)
    assert planner.ps_split(2) == (1, 2, 1)
    assert planner.ps_split(1)[0] == 0
    assert planner.ps_split(20, s=5) == (5, 4, 0)


def test_mult_count_eq5():
    for N in range(3, 61):
        q, b, g = planner.ps_split(N)
        assert q == math.isqrt(N - 1) and b == math.ceil(N / q)
        assert g == (1 if N - q * (b - 1) == 1 else 0)
        assert planner.mult_count(N) == q + b - 2 - g
    assert planner.mult_count(1) == planner.mult_count(2) == 0
    # PS beats Horner's N-1 products for N >= 5
    assert all(planner.mult_count(N) < N - 1 for N in range(5, 61))


@pytest.mark.parametrize("N", [3, 4, 5, 6, 9, 10, 17, 20, 26, 28, 37])
def test_oracle_product_count_matches_eq5(N):
    Z = CSR(*((lambda t: (len(t[0]) - 1, *t))(syn.laplacian_1d(12))))
    a = [1.0 / math.factorial(i) for i in range(N)]
    r = psscf(Z, a, 1e-12, poly=True)
    assert r.plan.N == N
    assert r.products == planner.mult_count(N)


def test_power_norms_lap1d_closed_form():
    # D Z D = -(I + S/2) with D = diag((-1)^k), S = shift up + down, so
    # |Z^i| = (I + S/2)^i entrywise; an interior column sums to exactly 2^i
    # for i < n/2 (boundary columns sum to less).
    Z = CSR(256, *syn.laplacian_1d(256))
    assert power_norms(Z) == [2.0 ** i for i in range(11)]


def test_power_norms_lap2d_closed_form():
    Z = CSR(32 * 32, *syn.laplacian_2d(32))
    assert power_norms(Z) == [4.0 ** i for i in range(11)]


def test_z_sequence_lemma1():
    norms = [1.0, 3.0, 5.0, 7.0, 8.0, 9.0, 9.5, 9.9, 10.0, 10.1, 10.2]
    z = planner.z_sequence(norms, 15)
    alpha = max(norms[k] ** (1.0 / k) for k in (5, 6, 7, 8, 9, 10))
    assert alpha == 9.0 ** (1.0 / 5)  # the k = 5 root dominates here
    assert z[:11] == norms and z[11:] == [alpha ** i for i in range(11, 16)]
    zs = planner.z_sequence(norms, 4, submult=True)
    assert zs == [1.0, 3.0, 9.0, 27.0, 81.0]


@pytest.mark.parametrize("tol", [1e-6, 1e-8, 1e-10, 1e-12, 1e-14])
@pytest.mark.parametrize("r", [1, 2, 4])
def test_theta_is_minimal_in_exact_arithmetic(tol, r):
    # exp with z_i = r^i: the exact tail sum_{i>=m} r^i/i! decides N.
    a = syn.coeffs("exp")
    z = [float(r) ** i for i in range(len(a))]
    N = planner.theta(tol, a, z)
    exact_tail = lambda m: sum(Fraction(r) ** i / math.factorial(i) for i in range(m, 200))
    half = Fraction(tol) / 2
    assert exact_tail(N) <= half < exact_tail(N - 1)


def test_theta_not_converged():
    a = syn.coeffs("exp", 8)
    z = [10.0 ** i for i in range(8)]
    assert planner.theta(1e-12, a, z) is None


def test_filter_bounds_hand_expansion_q2_b3():
    # N = 6: q = 2, b = 3, g = 0, M' = 3.  With q = 2 only d_2 exists and
    # beta_{i,2} = 0, so d_2 = z_4*0 + z_2 ||S_0|| + z_0 ||S_1|| (Eq. 24).
    a = [0.5, -1.5, 0.25, 2.0, -0.75, 1.25]
    z = [1.0, 3.0, 7.0, 20.0, 50.0, 140.0, 400.0]
    budget = 1e-9
    d, zeta, sigma = planner.filter_bounds(a, 6, 2, 3, 0, z, budget)
    B = [abs(a[2 * i]) * z[0] + abs(a[2 * i + 1]) * z[1] for i in range(3)]
    S0 = B[2]
    S1 = B[1] + z[2] * S0
    d2 = z[2] * S0 + z[0] * S1
    assert d[2] == pytest.approx(d2, rel=1e-15)
    assert zeta[2] == pytest.approx(budget / (d2 * 3), rel=1e-15)
    assert sigma == pytest.approx({1: budget / (z[2] * 3), 2: budget / (z[0] * 3)}, rel=1e-15)


def test_filter_bounds_hand_expansion_q3_b3():
    # N = 9 with q = 3: b = 3, g = 0, M' = 4.
    # beta_{i,2} = |a_{3i+2}| z_0 ; beta_{i,3} = 0
    # d_2 = sum_j z_{3(2-j)} (beta_{2-j,2} + z_1 ||S_{j-1}||)
    # d_3 = sum_j z_{3(2-j)} (z_0 ||S_{j-1}||)
    a = [1.0, 0.9, -0.8, 0.7, 0.6, -0.5, 0.4, 0.3, 0.2]
    z = [1.0, 2.0, 3.5, 6.0, 11.0, 19.0, 33.0]
    E = 2e-10
    d, zeta, sigma = planner.filter_bounds(a, 9, 3, 3, 0, z, E)
    B = [sum(abs(a[3 * i + j]) * z[j] for j in range(3)) for i in range(3)]
    S = [B[2], B[1] + z[3] * B[2]]
    S.append(B[0] + z[3] * S[1])
    beta2 = [abs(a[3 * i + 2]) * z[0] for i in range(3)]
    d2 = (z[6] * (beta2[2] + 0.0) + z[3] * (beta2[1] + z[1] * S[0])
          + z[0] * (beta2[0] + z[1] * S[1]))
    d3 = z[6] * 0.0 + z[3] * S[0] + z[0] * S[1]
    assert d[2] == pytest.approx(d2, rel=1e-15) and d[3] == pytest.approx(d3, rel=1e-15)
    assert zeta == pytest.approx({2: E / (d2 * 4), 3: E / (d3 * 4)}, rel=1e-15)
    assert sigma == pytest.approx({1: E / (z[3] * 4), 2: E / (z[0] * 4)}, rel=1e-15)


def test_filter_bounds_g1_skips_sigma_1():
    # N = 10: q = 3, b = 4, g = 1 -> M' = 4, sigma_j for j = 2, 3 only
    a = syn.coeffs("exp")[:10]
    z = [2.0 ** i for i in range(12)]
    p = planner.plan(a, 1e-10, z[:11], poly=True)
    assert (p.N, p.q, p.b, p.g) == (10, 3, 4, 1)
    assert sorted(p.sigma) == [2, 3] and sorted(p.zeta) == [2, 3]
    assert p.sigma[3] == 1e-10 / (1.0 * 4)


def test_plan_lap1d_values():
    # n = 256, exp, tol 1e-12, z_i = 2^i: the truncation length from Eq. (34)
    Z = CSR(256, *syn.laplacian_1d(256))
    p = planner.plan(syn.coeffs("exp"), 1e-12, power_norms(Z))
    assert (p.N, p.q, p.b, p.g) == (20, 4, 5, 0)
    exact = sum(Fraction(2) ** i / math.factorial(i) for i in range(20, 200))
    assert p.trunc == pytest.approx(float(exact), rel=1e-14)
    assert p.budget == 1e-12 - p.trunc


def sig2(x):
    return float(f"{x:.1e}")


def test_plan_workload_thresholds_hand_derived():
    # Thresholds of the two Laplacian workloads, derived by hand from
    # Eqs. (24)-(26), (34) and (36) with the closed-form norms z_i = 2^i
    # (1D, n = 256) and z_i = 4^i (2D, 128 x 128), eps_tol = 1e-12, in a
    # calculation independent of this planner; kept to 2 significant digits.
    Z1 = CSR(256, *syn.laplacian_1d(256))
    p = planner.plan(syn.coeffs("exp"), 1e-12, power_norms(Z1))
    assert (p.N, p.q, p.b, p.g) == (20, 4, 5, 0)
    assert sig2(p.trunc) == 4.8e-13
    assert {k: sig2(v) for k, v in p.zeta.items()} == {2: 6.6e-14, 3: 2.5e-13, 4: 1.1e-12}
    assert {j: sig2(v) for j, v in p.sigma.items()} == {1: 1.8e-17, 2: 2.9e-16, 3: 4.7e-15, 4: 7.5e-14}
    Z2 = CSR(128 * 128, *syn.laplacian_2d(128))
    n2 = power_norms(Z2)
    pe = planner.plan(syn.coeffs("exp"), 1e-12, n2)
    assert (pe.N, pe.q, pe.b, pe.g) == (28, 5, 6, 0)
    assert sig2(pe.sigma[1]) == 7.3e-26 and sig2(pe.sigma[5]) == 8.1e-14
    pc = planner.plan(syn.coeffs("cos"), 1e-12, n2)
    assert (pc.N, pc.q, pc.b, pc.g) == (27, 5, 6, 0)
