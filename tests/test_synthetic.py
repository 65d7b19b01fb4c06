"""The seeded input generators against the recipes they implement: shapes,
canonical CSR form, norms, symmetry and bandwidths, the size mixtures, the
Taylor coefficients, and determinism in the seed."""
import math
from fractions import Fraction

import numpy as np
import pytest

import synthetic as syn


def dense(t):
    rp, col, val = t
    n = len(rp) - 1
    d = np.zeros((n, n))
    for r in range(n):
        d[r, col[rp[r]:rp[r + 1]]] = val[rp[r]:rp[r + 1]]
    return d


def canonical(t):
    rp, col, val = t
    n = len(rp) - 1
    assert rp.dtype == np.int32 and col.dtype == np.int32 and val.dtype == np.float64
    assert rp[0] == 0 and rp[-1] == len(col) == len(val)
    assert np.all(np.diff(rp) >= 0)
    for r in range(n):
        c = col[rp[r]:rp[r + 1]]
        assert np.all(np.diff(c) > 0) and (len(c) == 0 or (c[0] >= 0 and c[-1] < n))
    assert np.all(val != 0.0) and np.all(np.isfinite(val))


def test_laplacians():
    L1 = syn.laplacian_1d(50)
    canonical(L1)
    d = dense(L1)
    assert np.array_equal(d, -0.5 * (2 * np.eye(50) - np.eye(50, k=1) - np.eye(50, k=-1)))
    assert syn.norm1(L1) == 2.0
    L2 = syn.laplacian_2d(9)
    canonical(L2)
    d2 = dense(L2)
    T = 2 * np.eye(9) - np.eye(9, k=1) - np.eye(9, k=-1)
    assert np.array_equal(d2, -0.5 * (np.kron(T, np.eye(9)) + np.kron(np.eye(9), T)))
    assert syn.norm1(L2) == 4.0


@pytest.mark.parametrize("seed", [0, 3])
def test_banded_random_recipe(seed):
    t = syn.banded_random(300, 5, seed, 2.0)
    canonical(t)
    d = dense(t)
    assert np.array_equal(d, d.T)  # symmetric
    i, j = np.nonzero(d)
    assert np.max(np.abs(i - j)) == 5  # half-bandwidth
    # before scaling, the diagonal was minus the column's off-diagonal 1-norm
    off = np.abs(d - np.diag(np.diag(d))).sum(axis=0)
    assert np.allclose(-np.diag(d), off, rtol=1e-14)
    assert abs(syn.norm1(t) - 2.0) <= 4e-16 * 2.0
    assert all(np.array_equal(x, y) for x, y in zip(t, syn.banded_random(300, 5, seed, 2.0)))


@pytest.mark.parametrize("w", [1, 4, 15])
def test_banded_normal_recipe(w):
    t = syn.banded_normal(1000, w, 1000 * w + 2)
    canonical(t)
    rp, col, _ = t
    rows = np.repeat(np.arange(1000), np.diff(rp))
    assert np.max(np.abs(rows - col)) == w
    assert len(col) == 1000 * (2 * w + 1) - w * (w + 1)  # the full band (no exact zeros drawn)
    v = t[2]
    assert abs(v.mean()) < 0.1 and abs(v.std() - 1.0) < 0.05  # N(0, 1)
    assert all(np.array_equal(x, y) for x, y in zip(t, syn.banded_normal(1000, w, 1000 * w + 2)))


def test_taylor_coefficients_are_the_nearest_doubles():
    e, c, ch, sh = (syn.coeffs(k) for k in ("exp", "cos", "cosh", "sinh"))
    for i in range(25):
        assert e[i] == float(Fraction(1, math.factorial(i)))
    assert c[:7] == [1.0, 0.0, -0.5, 0.0, 1.0 / 24, 0.0, -1.0 / 720]
    assert ch[:5] == [1.0, 0.0, 0.5, 0.0, 1.0 / 24]
    assert sh[:6] == [0.0, 1.0, 0.0, 1.0 / 6, 0.0, 1.0 / 120]
    for a in (e, c, ch, sh):
        assert a[-1] != 0.0 and len(a) <= syn.MAX_TERMS  # trailing underflow trimmed


def test_mixtures():
    inst = syn.batch_instances(64)
    assert len(inst) == 64
    ns = [len(Z[0]) - 1 for Z, _, _ in inst]
    assert min(ns) >= 6 and max(ns) <= 4096 + 2 * 64 + 1
    assert {k for _, k, _ in inst} == {"exp", "cosh"} and {t for _, _, t in inst} == {1e-12}
    for Z, _, _ in inst[:10]:
        canonical(Z)
        assert 1.0 - 1e-12 <= syn.norm1(Z) <= 4.0 + 1e-12
    req = syn.serving_requests(60, seed0=5)
    assert {k for _, k, _ in req} <= {"exp", "cos", "sinh"}
    assert {t for _, _, t in req} <= {1e-8, 1e-10, 1e-12}
    a, b = syn.serving_requests(3, seed0=9), syn.serving_requests(3, seed0=9)
    for (Za, ka, ta), (Zb, kb, tb) in zip(a, b):
        assert (ka, ta) == (kb, tb) and all(np.array_equal(x, y) for x, y in zip(Za, Zb))
