"""End-to-end GPU parity of Algorithm 2 through the C ABI against the oracle.

The bar is bitwise equality of the result CSR (row pointers, columns and
FP64 values), of the plan and of every step's Algorithm 1 decisions; it
implies the floating-point tolerance of 1e-12 relative Frobenius error, which
is asserted as well.  The GPU result is also checked against closed forms.
"""
import math

import numpy as np
import pytest

import synthetic as syn
from closed_forms import fun_lap1d, norm1_dense
from gpu_helpers import assert_csr_bitwise, check_same, dev, ocsr, rel_fro
from oracle import CSR, psscf

pytestmark = pytest.mark.gpu

psf = pytest.importorskip("paper_2208_05683_gb300")


def run_both(Z, a, tol, kernel="auto", chunk_cols=0, chunk_slots=0, **kw):
    got = psf.Series(a, tol, poly=kw.get("poly", False), filtered=kw.get("filtered", True),
                     submult=kw.get("submult", False), s=kw.get("s", 0), kernel=kernel,
                     chunk_cols=chunk_cols, chunk_slots=chunk_slots).eval(dev(Z))
    ref = psscf(Z, a, tol, **kw)
    return got, ref


def test_exp_lap1d_n256_bitwise_and_closed_form():
    Z = ocsr(syn.laplacian_1d(256))
    got, ref = run_both(Z, syn.coeffs("exp"), 1e-12)
    check_same(got, ref, "lap1d exp")
    rp, col, val = got.csr.to_host()
    F = CSR(256, rp, col, val).to_dense()
    assert norm1_dense(F - fun_lap1d(256, -0.5, np.exp)) <= 1e-12


@pytest.mark.parametrize("kind", ["exp", "cos", "cosh", "sinh"])
def test_lap2d_32_bitwise(kind):
    Z = ocsr(syn.laplacian_2d(32))
    got, ref = run_both(Z, syn.coeffs(kind), 1e-12)
    check_same(got, ref, kind)


@pytest.mark.parametrize("kernel,cols,slots", [("table", 0, 0), ("bitmap", 0, 0), ("table", 96, 0),
                                               ("bitmap", 64, 0), ("table", 0, 40), ("bitmap", 0, 33),
                                               ("table", 40, 37), ("window", 0, 0), ("window", 64, 0),
                                               ("window", 0, 33), ("window", 5000, 0)])
def test_slot_maps_and_row_chunking_bitwise(kernel, cols, slots):
    # both slot maps of the product kernel (the bitmap also with its wide
    # column window), and rows split into several column chunks (by width or
    # by accumulator slots), give the oracle's result bit for bit
    Z = ocsr(syn.laplacian_2d(24))
    for kind in ("exp", "cos"):
        got, ref = run_both(Z, syn.coeffs(kind), 1e-12, kernel=kernel, chunk_cols=cols, chunk_slots=slots)
        check_same(got, ref, f"{kernel} {cols}/{slots} {kind}")
    Zb = ocsr(syn.banded_random(700, 6, 3, 2.0))
    got, ref = run_both(Zb, syn.coeffs("exp"), 1e-12, kernel=kernel, chunk_cols=cols, chunk_slots=slots)
    check_same(got, ref, f"{kernel} {cols}/{slots} banded")


def test_second_evaluation_uses_first_as_hints():
    # the second evaluation of a series sizes its pool and picks its slot maps
    # from the first one's statistics; the result must not change
    Z = ocsr(syn.laplacian_2d(40))
    s = psf.Series(syn.coeffs("exp"), 1e-12)
    r1 = s.eval(dev(Z))
    r2 = s.eval(dev(Z))
    ref = psscf(Z, syn.coeffs("exp"), 1e-12)
    assert_csr_bitwise(r1.csr, ref.F, "first")
    assert_csr_bitwise(r2.csr, ref.F, "second")


@pytest.mark.parametrize("case", ["lap2d_exp", "lap2d_cos", "banded_drop", "banded_1e-12", "unfiltered", "poly"])
def test_repeated_evaluation_reuses_powers_bitwise(case):
    # from its second evaluation on, a series keeps the norm phase's powers
    # and uses them as baby steps until an entry is dropped; the results and
    # step records must equal the oracle's either way (the loose tolerance
    # makes baby steps drop entries)
    Z, a, tol, kw = {
        "lap2d_exp": (syn.laplacian_2d(40), syn.coeffs("exp"), 1e-12, {}),
        "lap2d_cos": (syn.laplacian_2d(40), syn.coeffs("cos"), 1e-12, {}),
        # baby step 3 drops entries: baby step 4 is a product again
        "banded_drop": (syn.banded_random(3000, 5, 7, 4.0), syn.coeffs("exp"), 1e-6, {}),
        "banded_1e-12": (syn.banded_random(3000, 5, 7, 2.0), syn.coeffs("exp"), 1e-12, {}),
        "unfiltered": (syn.laplacian_1d(300), syn.coeffs("exp"), 1e-12, {"filtered": False}),
        "poly": (syn.banded_random(500, 2, 5, 1.5), [(-1.0) ** i / math.factorial(i) for i in range(17)], 1e-11,
                 {"poly": True}),
    }[case]
    Z = ocsr(Z)
    s = psf.Series(a, tol, poly=kw.get("poly", False), filtered=kw.get("filtered", True))
    ref = psscf(Z, a, tol, **kw)
    first = s.eval(dev(Z))
    for _ in range(2):
        again = s.eval(dev(Z))
        check_same(again, ref, case)
        assert again.steps == first.steps, case


@pytest.mark.parametrize("shift", [0, 1, 2047])
def test_far_candidate_split_bitwise(shift):
    # Algorithm 1 sets candidates at or below eps_g / 2^shift apart after its
    # first pass.  Shift 1 makes later passes reach the set-apart candidates
    # (eps_f falls 6-27x on these steps), shift 0 sets every candidate apart,
    # 2047 none; the results and step records are the oracle's in every case.
    from paper_2208_05683_gb300 import _abi
    cases = [
        ("lap2d exp", ocsr(syn.laplacian_2d(48)), syn.coeffs("exp"), 1e-12),
        ("lap2d cos", ocsr(syn.laplacian_2d(48)), syn.coeffs("cos"), 1e-12),
        ("banded drop", ocsr(syn.banded_random(3000, 5, 7, 4.0)), syn.coeffs("exp"), 1e-6),
    ]
    old = psf.tune_get(_abi.PSF_TUNE_ALG1_FAR_SHIFT)
    try:
        psf.tune_set(_abi.PSF_TUNE_ALG1_FAR_SHIFT, float(shift))
        for name, Z, a, tol in cases:
            ref = psscf(Z, a, tol)
            s = psf.Series(a, tol)
            for _ in range(2):
                check_same(s.eval(dev(Z)), ref, f"{name} shift {shift}")
    finally:
        psf.tune_set(_abi.PSF_TUNE_ALG1_FAR_SHIFT, old)
    if shift == 1:
        assert any(st.iters >= 3 and (st.threshold / 1.1) / st.eps_f > 4.0 for st in ref.steps)


def test_candidates_far_below_threshold_bitwise():
    # 150 Taylor terms of exp(-x): q = 12, and the early giant steps only hold
    # entries near 1e-200 against a threshold near 1e3, far below the column
    # sums' fixed-point window.  Algorithm 1 must still drop them all and
    # report the exactly rounded column-sum maximum c, as the oracle does.
    a = [(-1.0) ** i / math.factorial(i) for i in range(150)]
    Z = ocsr(syn.banded_random(300, 2, 11, 1.0))
    ref = psscf(Z, a, 1e-11, poly=True)
    s = psf.Series(a, 1e-11, poly=True)
    for _ in range(2):  # the second evaluation takes its baby steps from the norm phase
        got = s.eval(dev(Z))
        check_same(got, ref, "poly q=12")
    assert got.info["q"] == 12
    assert any(st.c > 0.0 and st.c < 1e-150 for st in ref.steps)


@pytest.mark.parametrize("seed,n,hbw", [(0, 1000, 5), (1, 777, 3), (2, 4099, 2)])
def test_banded_random_bitwise(seed, n, hbw):
    Z = ocsr(syn.banded_random(n, hbw, seed, 2.0))
    got, ref = run_both(Z, syn.coeffs("exp"), 1e-12)
    check_same(got, ref, f"banded {n}")


@pytest.mark.parametrize("tol", [1e-8, 1e-10, 1e-14])
def test_tolerance_sweep_bitwise(tol):
    Z = ocsr(syn.banded_random(3000, 5, 7, 2.0))
    got, ref = run_both(Z, syn.coeffs("exp"), tol)
    check_same(got, ref, f"tol {tol}")


def test_unfiltered_submult_and_override():
    Z = ocsr(syn.laplacian_1d(300))
    a = syn.coeffs("exp")
    for kw in ({"filtered": False}, {"submult": True}, {"s": 5}, {"s": 2}):
        got, ref = run_both(Z, a, 1e-12, **kw)
        check_same(got, ref, str(kw))


@pytest.mark.parametrize("N", [2, 3, 5, 10, 17, 26, 30])
def test_poly_mode_g0_and_g1(N):
    Z = ocsr(syn.banded_random(500, 2, N, 1.5))
    a = [(-1.0) ** i / math.factorial(i) for i in range(N)]
    got, ref = run_both(Z, a, 1e-11, poly=True)
    check_same(got, ref, f"N={N}")


def test_degenerate_cases():
    a = syn.coeffs("exp")
    # n = 1
    Z1 = CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([0.5]))
    got, ref = run_both(Z1, a, 1e-12)
    check_same(got, ref, "n=1")
    assert abs(got.csr.to_host()[2][0] - math.exp(0.5)) <= 1e-12
    # zero matrix: N = 1, F = I
    Z0 = CSR.empty(64)
    got, ref = run_both(Z0, syn.coeffs("cos"), 1e-12)
    check_same(got, ref, "zero")
    # empty rows and a diagonal block
    d = np.zeros((40, 40))
    d[np.arange(0, 40, 3), np.arange(0, 40, 3)] = np.linspace(-2, 1, 14)
    got, ref = run_both(CSR.from_dense(d), a, 1e-12)
    check_same(got, ref, "diag")
    # nilpotent shift
    J = np.diag(np.full(20, 0.75), 1)
    got, ref = run_both(CSR.from_dense(J), a, 1e-14)
    check_same(got, ref, "nilpotent")


def test_not_converged_series():
    Z = ocsr(syn.laplacian_1d(64))
    with pytest.raises(psf.PsfError) as e:
        psf.Series(syn.coeffs("exp", 5), 1e-12).eval(dev(Z))
    assert e.value.code == 4


@pytest.mark.slow
@pytest.mark.parametrize("kind", ["exp", "cos"])
def test_lap2d_128x128_full_size_bitwise(kind):
    # the 2D Laplacian workload at full size (n = 16384)
    Z = ocsr(syn.laplacian_2d(128))
    got, ref = run_both(Z, syn.coeffs(kind), 1e-12)
    check_same(got, ref, kind)


@pytest.mark.slow
@pytest.mark.parametrize("tol", [1e-8, 1e-12, 1e-14])
def test_banded_n65536_full_size_bitwise(tol):
    # the banded workload at full size, across its tolerance sweep
    Z = ocsr(syn.banded_random(65536, 5, 0, 2.0))
    got, ref = run_both(Z, syn.coeffs("exp"), tol)
    check_same(got, ref, f"banded 65536 tol {tol}")


@pytest.mark.slow
@pytest.mark.parametrize("kind", ["exp", "cos"])
def test_lap2d_full_size_unfiltered_vs_filtered(kind):
    Z = ocsr(syn.laplacian_2d(128))
    a = syn.coeffs(kind)
    gf = psf.Series(a, 1e-12).eval(dev(Z))
    gu = psf.Series(a, 1e-12, filtered=False).eval(dev(Z))
    ru = psscf(Z, a, 1e-12, filtered=False)
    assert_csr_bitwise(gu.csr, ru.F, "unfiltered")
    assert gf.csr.nnz < gu.csr.nnz
    # filtered and unfiltered agree to the filtering budget (Eq. 35)
    import scipy.sparse as sp
    rp, col, val = gf.csr.to_host()
    Ff = sp.csr_matrix((val, col, rp), shape=(Z.n, Z.n))
    rp, col, val = gu.csr.to_host()
    Fu = sp.csr_matrix((val, col, rp), shape=(Z.n, Z.n))
    diff = abs(Ff - Fu).sum(axis=0).max()
    assert diff <= gf.info["budget"]


@pytest.mark.parametrize("w", [1, 4, 8, 15])
@pytest.mark.parametrize("kind", ["exp", "cos"])
def test_banded_normal_n1000_tol_1e14_bitwise(w, kind):
    # the paper's second test set (Sec. 4): 1000 x 1000, lower = upper
    # bandwidth w, N(0, 1) entries, eps_tol = 1e-14.  At w = 15 the result is
    # about half dense and the products' rows exceed one accumulator chunk.
    Z = ocsr(syn.banded_normal(1000, w, 11 + w))
    a = syn.coeffs(kind)
    check_same(psf.Series(a, 1e-14).eval(dev(Z)), psscf(Z, a, 1e-14), f"w={w} {kind}")


def estimate_cases():
    import scipy.sparse as sp
    n = 5000  # column 0 holds every row: longer than the estimator takes
    rows = np.concatenate([np.arange(n), np.arange(1, n)])
    cols = np.concatenate([np.zeros(n, int), np.arange(1, n)])
    vals = np.concatenate([np.full(n, 1e-4), np.full(n - 1, -0.5)])
    long_col = CSR.from_scipy(sp.coo_matrix((vals, (rows, cols)), shape=(n, n)))
    return {
        "lap2d exp": (ocsr(syn.laplacian_2d(40)), syn.coeffs("exp"), 1e-12),
        "lap2d cos": (ocsr(syn.laplacian_2d(40)), syn.coeffs("cos"), 1e-12),
        "banded": (ocsr(syn.banded_random(3000, 5, 7, 2.0)), syn.coeffs("exp"), 1e-12),
        "banded normal": (ocsr(syn.banded_normal(1000, 4, 5)), syn.coeffs("exp"), 1e-14),
        "random sparse": (ocsr(syn.random_sparse(700, 0.01, 3, 1.5)), syn.coeffs("cosh"), 1e-10),
        "n=2": (CSR.from_dense(np.array([[0.5, -1.0], [0.25, 0.75]])), syn.coeffs("exp"), 1e-12),
        "n=1": (CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([-0.5])),
                syn.coeffs("exp"), 1e-12),
        "zero": (CSR.empty(30), syn.coeffs("cos"), 1e-12),
        "long column": (long_col, syn.coeffs("exp"), 1e-12),
    }


@pytest.mark.parametrize("name", list(estimate_cases()))
def test_estimated_power_norms_bitwise(name):
    # PSF_Z_ESTIMATE: z_2..z_10 from the deterministic estimator; the plan and
    # the result must be the oracle's run with the oracle's estimates (the
    # long-column case falls back to the exact norms on both sides)
    from oracle import normest
    Z, a, tol = estimate_cases()[name]
    norms = normest.power_norm_estimates(Z)
    ref = psscf(Z, a, tol, norms=norms)
    s = psf.Series(a, tol, estimate=True)
    for _ in range(2):
        got = s.eval(dev(Z))
        check_same(got, ref, name)
        assert got.info["z"][:11] == norms[:11] or got.info["z"][:11] == ref.plan.z[:11], name


def test_extreme_fill_in_fails_cleanly():
    # an unstructured matrix (n = 200000, about 4 entries per row) whose
    # powers fill in to dense rows: the pools grow past 2^30 entries, and the
    # column-chunked rows of the products binary-search positions there,
    # before the evaluation gives up with PSF_ETOOBIG (a pool is at most
    # 2^31 - 2^20 entries).  Both norm modes end with the error, not a fault.
    Z = dev(syn.random_sparse(200000, 2e-5, 1, 2.0))
    for est in (False, True):
        with pytest.raises(psf.PsfError) as e:
            psf.Series(syn.coeffs("exp"), 1e-12, estimate=est).eval(Z)
        assert e.value.code == 6


@pytest.mark.parametrize("case", ["lap2d128 exp", "lap2d128 cos", "banded normal w15"])
def test_wide_accumulator_rows_bitwise(case):
    # From the second evaluation on, a giant step whose rows averaged more than
    # about 550 entries before the filter runs the product kernel's wide
    # accumulator (every slot to the row, a_rk read from A): the largest giant
    # step of the 128 x 128 Laplacian has rows of 625-637 entries, the dense
    # banded matrix rows of up to ~900 (column chunks inside the wide kernel).
    Z, a, tol = {
        "lap2d128 exp": (syn.laplacian_2d(128), syn.coeffs("exp"), 1e-12),
        "lap2d128 cos": (syn.laplacian_2d(128), syn.coeffs("cos"), 1e-12),
        "banded normal w15": (syn.banded_normal(1000, 15, 4), syn.coeffs("exp"), 1e-14),
    }[case]
    Z = ocsr(Z)
    ref = psscf(Z, a, tol)
    s = psf.Series(a, tol)
    for _ in range(3):
        check_same(s.eval(dev(Z)), ref, case)


def test_host_to_host_path_bitwise():
    # psf_eval_from_host (Z in host memory) and psf_result_copy into host
    # arrays: the same result as the device path, and as the oracle
    Z = syn.laplacian_2d(48)
    s = psf.Series(syn.coeffs("exp"), 1e-12)
    (rp, col, val), info, steps = s.eval_host(*Z)
    ref = psscf(ocsr(Z), syn.coeffs("exp"), 1e-12)
    assert np.array_equal(rp, ref.F.rowptr) and np.array_equal(col, ref.F.col)
    assert np.array_equal(val.view(np.uint64), np.asarray(ref.F.val).view(np.uint64))
    dev_res = s.eval(dev(ocsr(Z)))
    assert dev_res.steps == steps and dev_res.info["nnz"] == info["nnz"]
    # the zero 5 x 5 matrix through the host path: cos(0) = I
    (rp0, col0, val0), info0, _ = psf.Series(syn.coeffs("cos"), 1e-12).eval_host(
        np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0))
    assert list(rp0) == [0, 1, 2, 3, 4, 5] and list(col0) == [0, 1, 2, 3, 4] and list(val0) == [1.0] * 5
    assert info0["nnz"] == 5


def test_result_copied_out_while_the_next_evaluation_runs_bitwise():
    # psf_result_copy of one result into pinned host arrays on a second
    # stream, in flight while the next psf_eval runs on the first (its
    # read-backs go through the mapped mailbox, not behind that copy): both
    # results are the oracle's bit for bit, three times over
    import ctypes
    import torch
    from paper_2208_05683_gb300 import _abi
    L = _abi.lib()
    Z = ocsr(syn.laplacian_2d(64))
    refs = {k: psscf(Z, syn.coeffs(k), 1e-12) for k in ("exp", "cos")}
    series = {k: psf.Series(syn.coeffs(k), 1e-12) for k in refs}
    main = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    nnz = refs["exp"].F.nnz
    hr = torch.empty(Z.n + 1, dtype=torch.int32, pin_memory=True)
    hc = torch.empty(nnz, dtype=torch.int32, pin_memory=True)
    hv = torch.empty(nnz, dtype=torch.float64, pin_memory=True)
    for rep in range(3):
        h = series["exp"].eval_handle(dev(Z), main)
        done = torch.cuda.Event()
        done.record(main)
        side.wait_event(done)
        _abi.check(L.psf_result_copy(h, ctypes.c_void_p(hr.data_ptr()), ctypes.c_void_p(hc.data_ptr()),
                                     ctypes.c_void_p(hv.data_ptr()), ctypes.c_void_p(side.cuda_stream)))
        got_cos = series["cos"].eval(dev(Z), main)
        side.synchronize()
        _abi.check(L.psf_result_destroy(h))
        F = refs["exp"].F
        assert np.array_equal(hr.numpy(), F.rowptr) and np.array_equal(hc.numpy(), F.col), rep
        assert np.array_equal(hv.numpy().view(np.uint64), np.asarray(F.val).view(np.uint64)), rep
        check_same(got_cos, refs["cos"], f"cos, copy in flight, run {rep}")


def square_cases():
    return {
        "lap2d": (ocsr(syn.laplacian_2d(40)), 1e-12),
        "banded": (ocsr(syn.banded_random(3000, 5, 7, 2.0)), 1e-12),
        # baby steps in W drop entries
        "banded loose": (ocsr(syn.banded_random(3000, 5, 7, 4.0)), 1e-6),
        "random sparse": (ocsr(syn.random_sparse(700, 0.01, 3, 1.5)), 1e-10),
    }


@pytest.mark.parametrize("kind", ["cos", "cosh", "sinh"])
@pytest.mark.parametrize("mat", list(square_cases()))
def test_square_mode_bitwise(kind, mat):
    # PSF_Z_SQUARE: Algorithm 2 on W = Z Z; the second and third evaluations
    # take W from the norm phase's pool (the same bits as a fresh product)
    Z, tol = square_cases()[mat]
    a = syn.coeffs(kind)
    ref = psscf(Z, a, tol, square=True)
    s = psf.Series(a, tol, square=True)
    first = s.eval(dev(Z))
    check_same(first, ref, f"{kind} {mat}")
    assert first.info["products"] == ref.products
    assert first.info["z"] == ref.norms[:11]
    if kind == "sinh":
        assert first.steps[-1]["kind"] == "odd"
    for _ in range(2):
        again = s.eval(dev(Z))
        check_same(again, ref, f"{kind} {mat} again")
        assert again.steps == first.steps


@pytest.mark.parametrize("variant", ["unfiltered", "submult", "estimate", "s=2", "poly even", "poly odd"])
def test_square_mode_variants_bitwise(variant):
    Z = ocsr(syn.banded_random(1500, 4, 9, 2.5))
    a, kw, opts = syn.coeffs("cosh"), {}, {}
    if variant == "unfiltered":
        kw = opts = {"filtered": False}
    elif variant == "submult":
        kw = opts = {"submult": True}
    elif variant == "estimate":
        from oracle import normest
        a = syn.coeffs("sinh")
        kw, opts = {"norms": normest.power_norm_estimates(Z)}, {"estimate": True}
    elif variant == "s=2":
        kw = opts = {"s": 2}
    elif variant == "poly even":
        a = [(-1.0) ** (i // 2) / math.factorial(i) if i % 2 == 0 else 0.0 for i in range(23)]
        kw = opts = {"poly": True}
    else:
        a = [1.0 / math.factorial(i) if i % 2 else 0.0 for i in range(20)]
        kw = opts = {"poly": True}
    ref = psscf(Z, a, 1e-11, square=True, **kw)
    got = psf.Series(a, 1e-11, square=True, **opts).eval(dev(Z))
    check_same(got, ref, variant)
    assert got.info["products"] == ref.products


def test_square_mode_degenerate_cases():
    cos, sinh = syn.coeffs("cos"), syn.coeffs("sinh")
    # zero matrix: cos(0) = I, sinh(0) = 0 (g gets an infinite tolerance)
    Z0 = CSR.empty(50)
    for a in (cos, sinh):
        got = psf.Series(a, 1e-12, square=True).eval(dev(Z0))
        check_same(got, psscf(Z0, a, 1e-12, square=True), "zero")
    # n = 1
    Z1 = CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([-0.75]))
    for a, fn in ((cos, math.cos), (sinh, math.sinh)):
        got = psf.Series(a, 1e-12, square=True).eval(dev(Z1))
        check_same(got, psscf(Z1, a, 1e-12, square=True), "n=1")
        assert abs(got.csr.to_host()[2][0] - fn(-0.75)) <= 1e-12
    # g truncated to c_0: F = Z (c_0 I), a copy of Z
    Z = ocsr(syn.banded_random(60, 2, 4, 0.5))
    got = psf.Series(sinh, 10.0, square=True).eval(dev(Z))
    ref = psscf(Z, sinh, 10.0, square=True)
    assert ref.plan.N == 1
    check_same(got, ref, "N_W = 1")
    assert_csr_bitwise(got.csr, Z, "copy of Z")
    # a diagonal with empty rows, and a nilpotent shift (W = Z^2 is a shift by 2)
    d = np.zeros((40, 40))
    d[np.arange(0, 40, 3), np.arange(0, 40, 3)] = np.linspace(-2, 1, 14)
    J = np.diag(np.full(25, 0.75), 1)
    for M in (d, J):
        for a in (cos, sinh):
            got = psf.Series(a, 1e-14, square=True).eval(dev(CSR.from_dense(M)))
            check_same(got, psscf(CSR.from_dense(M), a, 1e-14, square=True), "structured")


@pytest.mark.slow
@pytest.mark.parametrize("kind", ["cos", "sinh"])
def test_square_mode_lap2d_128x128_bitwise(kind):
    Z = ocsr(syn.laplacian_2d(128))
    ref = psscf(Z, syn.coeffs(kind), 1e-12, square=True)
    s = psf.Series(syn.coeffs(kind), 1e-12, square=True)
    for _ in range(2):
        check_same(s.eval(dev(Z)), ref, kind)


def test_torch_sparse_csr_in_and_out():
    # the binding takes a torch sparse CSR tensor on the GPU (int64 indices
    # here) and returns one
    import torch
    rp, col, val = syn.laplacian_2d(24)
    t = torch.sparse_csr_tensor(torch.tensor(rp, dtype=torch.int64), torch.tensor(col, dtype=torch.int64),
                                torch.tensor(val), size=(576, 576)).to("cuda")
    got = psf.Series(syn.coeffs("exp"), 1e-12).eval(t)
    ref = psscf(ocsr((rp, col, val)), syn.coeffs("exp"), 1e-12)
    check_same(got, ref, "torch in")
    F = got.csr.to_torch()
    assert F.layout == torch.sparse_csr and F.is_cuda
    assert np.array_equal(F.to_dense().cpu().numpy(), ref.F.to_dense())


@pytest.mark.slow
@pytest.mark.parametrize("nb", [1 << 22, 1 << 23])
def test_lap1d_4m_rows_are_the_small_oracle_rows_shifted(nb):
    # Z = -0.5 tridiag(-1, 2, -1) is Toeplitz.  Each row of a product of its
    # powers depends only on the row's distance to the ends, so every row of
    # the result more than N from both ends is a shift of one interior row,
    # and the rows near the ends are those of any size >= 2N.  The norms
    # ||Z^i||_1 = 2^i, the plan and Algorithm 1's column-sum maxima are the
    # same for n = 256 and n = 2^22, so the large result must equal the
    # oracle's n = 256 result row by row (shifted), bit for bit: rows, pool
    # and column sums at 4.2 M and 8.4 M rows checked without running the
    # oracle there.  At 8.4 M rows the PS phase fills about 1.7e9 of the
    # 2^31 - 2^20 entries a pool can hold.
    ns = 256
    h = ns // 2
    a = syn.coeffs("exp")
    ref = psscf(ocsr(syn.laplacian_1d(ns)), a, 1e-12)
    got = psf.Series(a, 1e-12).eval(dev(syn.laplacian_1d(nb)))
    p = ref.plan
    assert (got.info["N"], got.info["q"], got.info["b"], got.info["g"]) == (p.N, p.q, p.b, p.g)
    assert got.info["z"] == ref.norms[:11]
    gsteps = [s for s in got.steps if s["kind"] != "add"]
    osteps = [s for s in ref.steps if not (s.kind == "giant" and s.threshold == 0.0 and p.g == 1 and s.index == 1)]
    for g, o in zip(gsteps, osteps):
        if o.threshold > 0:
            assert g["eps_f"] == o.eps_f and g["iters"] == o.iters and g["dropped"] == o.c, (g, o)
    srp, scol, sval = ref.F.rowptr, ref.F.col, np.asarray(ref.F.val)
    len_h = int(srp[h + 1] - srp[h])
    assert got.csr.nnz == ref.F.nnz + (nb - ns) * len_h
    rp, col, val = got.csr.to_host()
    rng = np.random.default_rng(5)
    rows = list(range(64)) + list(range(nb - 64, nb)) + list(rng.integers(h, nb - h, 3000))
    for r in rows:
        if r < h:
            rs, shift = r, 0
        elif r >= nb - h:
            rs, shift = r - (nb - ns), nb - ns
        else:
            rs, shift = h, r - h
        gc, gv = col[rp[r]:rp[r + 1]], val[rp[r]:rp[r + 1]]
        oc, ov = scol[srp[rs]:srp[rs + 1]] + shift, sval[srp[rs]:srp[rs + 1]]
        assert np.array_equal(gc, oc), r
        assert np.array_equal(gv.view(np.uint64), ov.view(np.uint64)), r


@pytest.mark.slow
@pytest.mark.parametrize("kind", ["exp", "cos"])
def test_lap2d_768x768_rows_are_the_128x128_oracle_rows_shifted(kind):
    # The 2D Laplacian is translation invariant away from the grid's edges:
    # a row's pattern and values depend only on the point's distance to each
    # edge, counted up to the pattern's reach (< 64 here), and the fold order
    # (row-major order of the 2D offsets) is the same on both grids.  So each
    # row (i, j) of the 768 x 768 result (n = 589824, 36 times the 128 x 128
    # workload) is row (is, js) of the 128 x 128 oracle result, its columns
    # moved by the 2D offset (i - is, j - js); the plan and Algorithm 1's
    # column-sum maxima agree, since both grids have the same column profiles.
    M, m = 768, 128
    a = syn.coeffs(kind)
    ref = psscf(ocsr(syn.laplacian_2d(m)), a, 1e-12)
    series = psf.Series(a, 1e-12)
    Zd = dev(syn.laplacian_2d(M))
    series.eval(Zd)
    # the second evaluation runs the steps whose rows spanned more than 4608
    # columns (about 2 x 25 grid rows of 768 here) with the wide column window
    got = series.eval(Zd)
    p = ref.plan
    assert (got.info["N"], got.info["q"], got.info["b"], got.info["g"]) == (p.N, p.q, p.b, p.g)
    assert got.info["z"] == ref.norms[:11]
    gsteps = [s for s in got.steps if s["kind"] != "add"]
    osteps = [s for s in ref.steps if not (s.kind == "giant" and s.threshold == 0.0 and p.g == 1 and s.index == 1)]
    for g, o in zip(gsteps, osteps):
        if o.threshold > 0:
            assert g["eps_f"] == o.eps_f and g["iters"] == o.iters and g["dropped"] == o.c, (g, o)

    def small(i):  # the small-grid index with the same distances to the edges
        return i if i < m // 2 else (i - (M - m) if i >= M - m // 2 else m // 2)

    srp, scol, sval = ref.F.rowptr, ref.F.col, np.asarray(ref.F.val)
    lens = np.diff(srp).reshape(m, m)
    cnt = np.ones(m, np.int64)
    cnt[m // 2] = M - m + 1
    assert got.csr.nnz == int((cnt[:, None] * cnt[None, :] * lens).sum())
    rp, col, val = got.csr.to_host()
    rng = np.random.default_rng(9)
    pts = [(i, j) for i in (0, 1, 63, 64, 700, M - 1) for j in (0, 2, 64, 383, M - 64, M - 1)]
    pts += [tuple(x) for x in rng.integers(0, M, (2000, 2))]
    for i, j in pts:
        r, i_s, j_s = i * M + j, small(i), small(j)
        rs = i_s * m + j_s
        oc = scol[srp[rs]:srp[rs + 1]]
        want = (oc // m + (i - i_s)) * M + (oc % m + (j - j_s))
        assert np.array_equal(col[rp[r]:rp[r + 1]], want), (i, j)
        assert np.array_equal(val[rp[r]:rp[r + 1]].view(np.uint64), sval[srp[rs]:srp[rs + 1]].view(np.uint64)), (i, j)
