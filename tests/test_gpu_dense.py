"""The dense-tile form of a product step (PSF_PARAM_DENSE_XOVER,
PSF_TUNE_DENSE_XOVER): forced for every product step, it gives the oracle's
result bit for bit and the same step statistics as the sparse kernel; the
automatic choice picks it where the multiply-adds per n^3 pass the crossover.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synthetic as syn
from gpu_helpers import assert_csr_bitwise, check_same, dev, ocsr
from oracle import CSR, alg1, axpy, matmul_add, psscf

pytestmark = pytest.mark.gpu

psf = pytest.importorskip("paper_2208_05683_gb300")
from paper_2208_05683_gb300 import _abi  # noqa: E402

ALWAYS, NEVER = 0.0, 1e300


@pytest.fixture
def dense_xover():
    old = psf.tune_get(_abi.PSF_TUNE_DENSE_XOVER)
    yield lambda v: psf.tune_set(_abi.PSF_TUNE_DENSE_XOVER, v)
    psf.tune_set(_abi.PSF_TUNE_DENSE_XOVER, old)


def rand_csr(n, density, seed, mag_spread=0.0):
    rng = np.random.default_rng(seed)
    m = sp.random(n, n, density=density, random_state=rng, format="csr",
                  data_rvs=lambda k: rng.uniform(-1, 1, k) * 10.0 ** (-mag_spread * rng.uniform(0, 1, k)))
    return CSR.from_scipy(m)


@pytest.mark.parametrize("n,density,seed", [(1, 1.0, 0), (37, 0.2, 1), (100, 0.05, 2), (257, 0.3, 3),
                                            (1000, 0.01, 4)])
def test_dense_product_bitwise(n, density, seed, dense_xover):
    # sizes not multiples of the 64 x 64 tiles or the 16-deep k slices
    A = rand_csr(n, density, seed)
    B = rand_csr(n, density, seed + 10)
    M1 = rand_csr(n, density, seed + 20)
    add = [(0.5, None), (-1.25, M1), (3.0, B)]
    X = None
    for alpha, M in add:
        X = axpy(alpha, M, X, n)
    ref = matmul_add(A, B, X)
    dadd = [(a, dev(M) if M is not None else None) for a, M in add]
    stats = []
    for v in (ALWAYS, NEVER):
        dense_xover(v)
        got = psf.product_filter(dev(A), dev(B), dadd, 0.0)
        assert_csr_bitwise(got.csr, ref, f"n={n}, crossover {v}")
        stats.append((got.steps[0]["nnz_pre"], got.steps[0]["fma"]))
    assert stats[0] == stats[1]


@pytest.mark.parametrize("seed", range(3))
def test_dense_product_then_alg1_bitwise(seed, dense_xover):
    n = 300
    A = rand_csr(n, 0.05, seed, mag_spread=20)
    B = rand_csr(n, 0.05, seed + 50, mag_spread=20)
    C = matmul_add(A, B)
    ref = alg1(C, 1e-6 / 1.1, 0.1)
    dense_xover(ALWAYS)
    got = psf.product_filter(dev(A), dev(B), [], 1e-6, 0.1)
    assert_csr_bitwise(got.csr, ref.kept, f"seed {seed}")
    st = got.steps[0]
    assert st["eps_f"] == ref.eps_f and st["iters"] == ref.iters and st["dropped"] == ref.c
    assert st["nnz_pre"] == C.nnz and st["nnz_post"] == ref.kept.nnz


@pytest.mark.parametrize("w", [11, 15])
@pytest.mark.parametrize("kind", ["exp", "cos"])
def test_dense_steps_banded_normal_n1000_bitwise(w, kind):
    # the paper's banded N(0, 1) family (Sec. 4) where near-sparsity fades
    # (results 40 % dense at w = 11, 55 % at w = 15): every product step as
    # dense tiles, twice (the second evaluation uses the first's counts)
    Z = ocsr(syn.banded_normal(1000, w, 11 + w))
    a = syn.coeffs(kind)
    ref = psscf(Z, a, 1e-14)
    s = psf.Series(a, 1e-14, dense_xover=ALWAYS)
    for rep in range(2):
        check_same(s.eval(dev(Z)), ref, f"w={w} {kind} evaluation {rep}")


def test_dense_steps_lap2d_and_square_mode_bitwise():
    Z = ocsr(syn.laplacian_2d(30))
    for kind, opts in (("exp", {}), ("cos", {"square": True}), ("sinh", {"square": True})):
        a = syn.coeffs(kind)
        ref = psscf(Z, a, 1e-12, square=bool(opts))
        check_same(psf.Series(a, 1e-12, dense_xover=ALWAYS, **opts).eval(dev(Z)), ref, kind)


def test_automatic_choice_uses_dense_tiles_for_filled_in_products(dense_xover):
    # a random matrix whose powers fill in: at the default crossover the giant
    # steps run as dense tiles (more launches per step), the results unchanged
    Z = ocsr(syn.random_sparse(600, 0.02, 5, 2.0))
    a = syn.coeffs("exp")
    ref = psscf(Z, a, 1e-12)
    L = psf.lib()
    counts = {}
    for name, v in (("sparse", NEVER), ("auto", psf.tune_get(_abi.PSF_TUNE_DENSE_XOVER))):
        dense_xover(v)
        s = psf.Series(a, 1e-12)
        s.eval(dev(Z))  # the second evaluation knows each step's multiply-adds
        c0 = _launches(L)
        check_same(s.eval(dev(Z)), ref, name)
        counts[name] = _launches(L) - c0
    assert counts["auto"] > counts["sparse"]


def _launches(L):
    import ctypes
    v = ctypes.c_int64()
    L.psf_launch_count(ctypes.byref(v))
    return v.value


def test_dense_xover_keys_check_values():
    with pytest.raises(psf.PsfError):
        psf.tune_set(_abi.PSF_TUNE_DENSE_XOVER, -0.5)
    with pytest.raises(psf.PsfError):
        psf.Series(syn.coeffs("exp"), 1e-12, dense_xover=-2.0)
