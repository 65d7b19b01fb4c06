"""The product kernel's one-row-per-block form (PSF_PARAM_KERNEL = 4,
k_product_cta): four warps share one output row's bitmap map and 2560
accumulator slots, fold each B row's entries together with a block barrier
between B rows, and fall back to the warp-per-row code for rows wider than
4608 columns or with more than 2560 entries.  Every case is the oracle's
result bit for bit, with the same step records as the default kernel.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synthetic as syn
from gpu_helpers import check_same, dev, ocsr
from oracle import CSR, psscf

pytestmark = pytest.mark.gpu

psf = pytest.importorskip("paper_2208_05683_gb300")


def rand_csr(n, density, seed):
    rng = np.random.default_rng(seed)
    m = sp.random(n, n, density=density, random_state=rng, format="csr", data_rvs=lambda k: rng.uniform(-1, 1, k))
    m = m / sp.linalg.norm(m, 1) * 1.5
    return CSR.from_scipy(m.tocsr())


def both(Z, a, tol, **kw):
    out = [psf.Series(a, tol, kernel=k, **kw).eval(dev(Z)) for k in ("cta", "auto")]
    assert out[0].steps == out[1].steps
    return out[0]


@pytest.mark.parametrize("kind", ["exp", "cos"])
def test_cta_lap2d_and_banded_bitwise(kind):
    for Z in (ocsr(syn.laplacian_2d(24)), ocsr(syn.laplacian_2d(70)), ocsr(syn.banded_random(700, 6, 3, 2.0))):
        a = syn.coeffs(kind)
        check_same(both(Z, a, 1e-12), psscf(Z, a, 1e-12), f"{kind} n={Z.n}")


@pytest.mark.parametrize("w", [1, 8, 15])
def test_cta_banded_normal_n1000_bitwise(w):
    # the paper's banded N(0, 1) family (Sec. 4): B rows of up to 1000 entries
    Z = ocsr(syn.banded_normal(1000, w, 5 + w))
    for kind in ("exp", "cos"):
        a = syn.coeffs(kind)
        check_same(both(Z, a, 1e-14), psscf(Z, a, 1e-14), f"w={w} {kind}")


def test_cta_fallbacks_bitwise():
    # rows with more than 2560 entries inside one 4608-column window, and
    # rows wider than the window: the block's first warp takes them
    a = [1.0, 0.5, 0.25, 0.125, 0.0625]
    for Z, what in ((rand_csr(3000, 0.05, 1), "dense rows"), (rand_csr(6000, 0.001, 2), "wide rows")):
        check_same(both(Z, a, 1e-10, poly=True, submult=True), psscf(Z, a, 1e-10, poly=True, submult=True), what)


def test_cta_twice_and_square_mode_bitwise():
    Z = ocsr(syn.laplacian_2d(40))
    s = psf.Series(syn.coeffs("cosh"), 1e-12, kernel="cta", square=True)
    ref = psscf(Z, syn.coeffs("cosh"), 1e-12, square=True)
    for rep in range(2):
        check_same(s.eval(dev(Z)), ref, f"evaluation {rep}")


def test_cta_repeated_runs_are_identical():
    # the block's warps share the row's map and accumulator: repeated runs
    # (different warp timings) give the same bits, equal to the warp-per-row
    # kernel's and the oracle's
    Z = ocsr(syn.laplacian_2d(70))
    a = syn.coeffs("exp")
    ref = psscf(Z, a, 1e-12)
    base = psf.Series(a, 1e-12, kernel="bitmap").eval(dev(Z))
    check_same(base, ref, "warp per row")
    s = psf.Series(a, 1e-12, kernel="cta")
    for rep in range(6):
        got = s.eval(dev(Z))
        check_same(got, ref, f"run {rep}")
        assert got.steps == base.steps, f"run {rep}"
