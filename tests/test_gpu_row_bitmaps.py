"""Column bitmaps of B's rows in the product's symbolic pass
(PSF_TUNE_ROW_BITMAPS): the output pattern of a row is marked a bitmap word
at a time for B rows that have one (no more words than entries) and column
by column for the others.  With them on every product (2) and on none (0)
the results are the
oracle's bit for bit and the step statistics are the same, on matrices whose
B rows all have bitmaps (bands), none (scattered entries), or a mix, with
rows that take one column chunk and rows that take several.
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


@pytest.fixture
def row_bitmaps():
    old = psf.tune_get(_abi.PSF_TUNE_ROW_BITMAPS)
    assert old == 1.0  # the default
    yield lambda v: psf.tune_set(_abi.PSF_TUNE_ROW_BITMAPS, v)
    psf.tune_set(_abi.PSF_TUNE_ROW_BITMAPS, old)


def rand_csr(n, density, seed, mag_spread=0.0):
    rng = np.random.default_rng(seed)
    m = sp.random(n, n, density=density, random_state=rng, format="csr",
                  data_rvs=lambda k: rng.uniform(-1, 1, k) * 10.0 ** (-mag_spread * rng.uniform(0, 1, k)))
    return CSR.from_scipy(m)


def band_csr(n, lower, upper, seed, holes=0.0):
    """Entries at offsets -lower..upper of the diagonal, a fraction `holes`
    of them left out."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for d in range(-lower, upper + 1):
        r = np.arange(max(0, -d), min(n, n - d))
        keep = rng.uniform(size=len(r)) >= holes
        rows.append(r[keep])
        cols.append(r[keep] + d)
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    return CSR.from_scipy(sp.csr_matrix((rng.uniform(-1, 1, len(rows)), (rows, cols)), shape=(n, n)))


def mixed_rows(n, seed):
    """Rows of four kinds in turn: a few entries near the diagonal (more
    bitmap words than entries), a few anywhere (windows wider than one
    chunk when n is large), a dense run (a bitmap; products of more than
    640 entries) and a run with every other column (a bitmap, half full)."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for r in range(n):
        kind = r % 4
        if kind == 0:
            c = np.unique(np.clip(r + rng.integers(-40, 41, 6), 0, n - 1))
        elif kind == 1:
            c = rng.choice(n, size=5, replace=False)
        elif kind == 2:
            c0 = int(rng.integers(0, max(1, n - 300)))
            c = np.arange(c0, min(n, c0 + 60))
        else:
            c0 = int(rng.integers(0, max(1, n - 300)))
            c = np.arange(c0, min(n, c0 + 90), 2)
        rows += [r] * len(c)
        cols += list(c)
    return CSR.from_scipy(sp.csr_matrix((rng.uniform(-1, 1, len(rows)), (rows, cols)), shape=(n, n)))


def both(row_bitmaps, fn):
    out = []
    for v in (2.0, 0.0):  # every product with bitmaps, none
        row_bitmaps(v)
        out.append(fn())
    return out


def product_case(A, B, add, n, row_bitmaps, what):
    X = None
    for alpha, M in add:
        X = axpy(alpha, M, X, n)
    ref = matmul_add(A, B, X)
    dadd = [(a, dev(M) if M is not None else None) for a, M in add]
    got = both(row_bitmaps, lambda: psf.product_filter(dev(A), dev(B), dadd, 0.0))
    for g in got:
        assert_csr_bitwise(g.csr, ref, what)
    assert got[0].steps == got[1].steps, what
    return ref


@pytest.mark.parametrize("n,lower,upper,holes", [(1, 0, 0, 0.0), (33, 3, 5, 0.0), (500, 20, 7, 0.3),
                                                 (4608, 40, 40, 0.5), (4650, 64, 0, 0.1),
                                                 (12000, 90, 90, 0.6)])
def test_banded_products_bitwise(n, lower, upper, holes, row_bitmaps):
    # every B row has a bitmap; n <= 4608 is every row's window, above each
    # row's own window, aligned down to a multiple of 32 columns
    A = band_csr(n, upper, lower, 1, holes)
    B = band_csr(n, lower, upper, 2, holes)
    M = band_csr(n, 2, 2, 3)
    product_case(A, B, [(0.5, None), (-2.0, M)], n, row_bitmaps, f"band n={n}")


@pytest.mark.parametrize("n,density,seed", [(37, 0.2, 1), (1000, 0.01, 3), (3001, 0.002, 4), (9000, 0.0005, 7)])
def test_scattered_products_bitwise(n, density, seed, row_bitmaps):
    # few B rows have a bitmap (more words than entries)
    A = rand_csr(n, density, seed)
    B = rand_csr(n, density, seed + 10)
    M1 = rand_csr(n, density, seed + 20)
    product_case(A, B, [(0.5, None), (-1.25, M1), (3.0, B)], n, row_bitmaps, f"random n={n}")


@pytest.mark.parametrize("n", [3000, 12000])
def test_mixed_rows_bitwise(n, row_bitmaps):
    A = mixed_rows(n, 1)
    B = mixed_rows(n, 2)
    ref = product_case(A, B, [(2.0, None)], n, row_bitmaps, f"mixed n={n}")
    lens = np.diff(ref.rowptr)
    assert lens.max() > 640 and (lens < 200).sum() > n // 4


@pytest.mark.parametrize("seed", range(2))
def test_banded_product_then_alg1_bitwise(seed, row_bitmaps):
    n = 2000
    A = band_csr(n, 30, 30, seed, 0.2)
    B = band_csr(n, 30, 30, seed + 7, 0.2)
    rng = np.random.default_rng(seed)
    B.val[:] *= 10.0 ** (-16 * rng.uniform(0, 1, B.nnz))
    C = matmul_add(A, B)
    ref = alg1(C, 1e-9 / 1.1, 0.1)
    assert ref.iters >= 2
    got = both(row_bitmaps, lambda: psf.product_filter(dev(A), dev(B), [], 1e-9, 0.1))
    for g in got:
        assert_csr_bitwise(g.csr, ref.kept, f"seed {seed}")
        st = g.steps[0]
        assert st["eps_f"] == ref.eps_f and st["iters"] == ref.iters and st["dropped"] == ref.c
        assert st["nnz_pre"] == C.nnz and st["nnz_post"] == ref.kept.nnz


@pytest.mark.parametrize("name,Z,kind,opts", [
    ("lap2d 40 exp", syn.laplacian_2d(40), "exp", {}),
    ("lap2d 80 cos", syn.laplacian_2d(80), "cos", {}),
    ("lap2d 160 exp", syn.laplacian_2d(160), "exp", {}),
    ("banded N(0,1) w=11", syn.banded_normal(1000, 11, 22), "exp", {}),
    ("lap2d 60 cosh Z^2", syn.laplacian_2d(60), "cosh", {"square": True}),
])
def test_series_with_and_without_bitmaps_bitwise(name, Z, kind, opts, row_bitmaps):
    Z = ocsr(Z)
    a = syn.coeffs(kind)
    ref = psscf(Z, a, 1e-12, square=bool(opts))
    got = both(row_bitmaps, lambda: psf.Series(a, 1e-12, **opts).eval(dev(Z)))
    for g in got:
        check_same(g, ref, name)
    assert got[0].steps == got[1].steps


def test_row_bitmaps_key_checks():
    for bad in (-1, 0.5, 3):
        with pytest.raises(psf.PsfError):
            psf.tune_set(_abi.PSF_TUNE_ROW_BITMAPS, bad)


def test_batch_with_and_without_bitmaps_bitwise(row_bitmaps):
    # the giant stages of a block-diagonal batch: instance windows start
    # anywhere, aligned down to 32 columns for the bitmaps
    cases = [(ocsr(syn.laplacian_2d(17 + 5 * (i % 4))), ("exp", "cos", "sinh")[i % 3]) for i in range(9)]
    cases.append((ocsr(syn.banded_random(700, 6, 3, 2.0)), "exp"))
    cases.append((ocsr(syn.banded_normal(300, 11, 5)), "cosh"))
    refs = [psscf(Z, syn.coeffs(k), 1e-12) for Z, k in cases]
    series = [psf.Series(syn.coeffs(k), 1e-12) for _, k in cases]
    runs = []
    for v in (2.0, 0.0):
        row_bitmaps(v)
        for rep in range(2):  # the second batch knows every stage's sizes
            got = psf.eval_batch(series, [dev(Z) for Z, _ in cases])
            for i, (g, ref) in enumerate(zip(got, refs)):
                check_same(g, ref, f"instance {i}, bitmaps {v}, batch {rep}")
        runs.append([g.steps for g in got])
    assert runs[0] == runs[1]
