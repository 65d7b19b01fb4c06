"""psf_eval_batch through the C ABI: many (series, Z) instances evaluated as
one block-diagonal batch.

Every instance's result must be bit for bit the oracle's filtered PS result
(and the result of evaluating it alone with psf_eval), with the same plan and
the same per-step Algorithm 1 decisions, whatever else is in the batch.
"""
import math

import numpy as np
import pytest

import synthetic as syn
from gpu_helpers import assert_csr_bitwise, check_same, dev, ocsr
from oracle import CSR, psscf

pytestmark = pytest.mark.gpu

psf = pytest.importorskip("paper_2208_05683_gb300")
_abi = psf._abi


def series_of(a, tol, **kw):
    return psf.Series(a, tol, poly=kw.get("poly", False), filtered=kw.get("filtered", True),
                      submult=kw.get("submult", False), s=kw.get("s", 0), square=kw.get("square", False))


def mixed_cases():
    """(name, oracle CSR, coefficients, tol, options) covering the modes."""
    poly_a = [(-1.0) ** i / math.factorial(i) for i in range(5)]
    diag = np.zeros((40, 40))
    diag[np.arange(0, 40, 3), np.arange(0, 40, 3)] = np.linspace(-2, 1, 14)
    return [
        ("lap1d exp", ocsr(syn.laplacian_1d(256)), syn.coeffs("exp"), 1e-12, {}),
        ("lap2d cos", ocsr(syn.laplacian_2d(24)), syn.coeffs("cos"), 1e-12, {}),
        ("banded sinh", ocsr(syn.banded_random(700, 6, 3, 2.0)), syn.coeffs("sinh"), 1e-10, {}),
        ("lap2d cosh", ocsr(syn.laplacian_2d(20)), syn.coeffs("cosh"), 1e-12, {}),
        ("poly N=5", ocsr(syn.banded_random(500, 2, 5, 1.5)), poly_a, 1e-11, {"poly": True}),
        ("submult", ocsr(syn.laplacian_1d(300)), syn.coeffs("exp"), 1e-12, {"submult": True}),
        ("unfiltered", ocsr(syn.laplacian_1d(128)), syn.coeffs("exp"), 1e-12, {"filtered": False}),
        ("s=2", ocsr(syn.laplacian_1d(200)), syn.coeffs("exp"), 1e-12, {"s": 2}),
        ("zero matrix", CSR.empty(64), syn.coeffs("cos"), 1e-12, {}),
        ("n=1", CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([0.5])),
         syn.coeffs("exp"), 1e-12, {}),
        ("diag", CSR.from_dense(diag), syn.coeffs("exp"), 1e-12, {}),
        ("nilpotent", CSR.from_dense(np.diag(np.full(20, 0.75), 1)), syn.coeffs("exp"), 1e-14, {}),
        ("tol 1e-8", ocsr(syn.banded_random(900, 5, 7, 2.0)), syn.coeffs("exp"), 1e-8, {}),
    ]


def test_mixed_batch_bitwise_vs_oracle_and_single():
    cases = mixed_cases()
    series = [series_of(a, tol, **kw) for _, _, a, tol, kw in cases]
    got = psf.eval_batch(series, [dev(Z) for _, Z, _, _, _ in cases])
    assert len(got) == len(cases)
    for (name, Z, a, tol, kw), g in zip(cases, got):
        ref = psscf(Z, a, tol, **kw)
        check_same(g, ref, name)
        alone = series_of(a, tol, **kw).eval(dev(Z))
        assert alone.steps == g.steps, name
        for key in ("N", "q", "b", "g", "products", "z", "trunc", "budget", "nnz"):
            assert alone.info[key] == g.info[key], (name, key)


def test_batch_order_does_not_matter():
    # the same instances in reverse order give the same results
    cases = mixed_cases()[:8]
    series = [series_of(a, tol, **kw) for _, _, a, tol, kw in cases]
    Zs = [dev(Z) for _, Z, _, _, _ in cases]
    fwd = psf.eval_batch(series, Zs)
    rev = psf.eval_batch(series[::-1], Zs[::-1])[::-1]
    for (name, *_), f, r in zip(cases, fwd, rev):
        for x, y in zip(f.csr.to_host(), r.csr.to_host()):
            assert np.array_equal(x, y), name
        assert f.steps == r.steps, name


def test_batched_workload_512_instances_sampled_against_oracle():
    # the batched workload at full size (512 instances, n in [64, 4096]);
    # a seeded sample of instances is checked against the oracle one by one
    inst = syn.batch_instances(512)
    series = [psf.Series(syn.coeffs(k), tol) for _, k, tol in inst]
    got = psf.eval_batch(series, [dev(Z) for Z, _, _ in inst])
    rng = np.random.default_rng(5)
    sample = sorted(set(rng.choice(512, 20, replace=False).tolist()) | {int(np.argmax([len(Z[0]) for Z, _, _ in inst]))})
    for i in sample:
        Z, k, tol = inst[i]
        check_same(got[i], psscf(ocsr(Z), syn.coeffs(k), tol), f"instance {i}")
    # every instance: the result's row count and a valid CSR
    for (Z, _, _), g in zip(inst, got):
        rp, col, val = g.csr.to_host()
        assert len(rp) == len(Z[0]) and rp[0] == 0 and rp[-1] == len(col)


def test_more_instances_than_one_launch_holds():
    # 1100 tiny instances: split into several launch groups
    inst = [syn.mixed_instance(9000 + i, 2, 12) for i in range(1100)]
    series = [psf.Series(syn.coeffs(k), tol) for _, k, tol in inst]
    got = psf.eval_batch(series, [dev(Z) for Z, _, _ in inst])
    for i in (0, 1, 511, 1023, 1024, 1025, 1099):
        Z, k, tol = inst[i]
        check_same(got[i], psscf(ocsr(Z), syn.coeffs(k), tol), f"instance {i}")


def test_batch_edge_cases():
    # a single instance, an empty (n = 0) instance, and an all-trivial batch
    Z = ocsr(syn.laplacian_1d(100))
    one = psf.eval_batch([psf.Series(syn.coeffs("exp"), 1e-12)], [dev(Z)])
    assert_csr_bitwise(one[0].csr, psscf(Z, syn.coeffs("exp"), 1e-12).F, "single")
    empty = dev((np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0)))
    res = psf.eval_batch([psf.Series(syn.coeffs("exp"), 1e-12)] * 3, [dev(Z), empty, dev(Z)])
    assert res[1].csr.n == 0 and res[1].csr.nnz == 0
    assert_csr_bitwise(res[2].csr, psscf(Z, syn.coeffs("exp"), 1e-12).F, "after empty")
    zeros = [CSR.empty(n) for n in (5, 17, 64)]
    res = psf.eval_batch([psf.Series(syn.coeffs("cos"), 1e-12) for _ in zeros], [dev(z) for z in zeros])
    for z, r in zip(zeros, res):
        check_same(r, psscf(z, syn.coeffs("cos"), 1e-12), "zero")
    assert psf.eval_batch([], []) == []


def test_batch_errors_fail_the_whole_batch():
    good = dev(ocsr(syn.laplacian_1d(50)))
    bad = dev((np.array([0, 1, 1, 1, 1, 1], np.int32), np.array([7], np.int32), np.array([1.0])))
    with pytest.raises(psf.PsfError) as e:
        psf.eval_batch([psf.Series(syn.coeffs("exp"), 1e-12)] * 2, [good, bad])
    assert e.value.code == 1
    # a series too short for its tolerance: Eq. (34) finds no truncation length
    with pytest.raises(psf.PsfError) as e:
        psf.eval_batch([psf.Series(syn.coeffs("exp"), 1e-12), psf.Series(syn.coeffs("exp", 5), 1e-12)],
                       [good, good])
    assert e.value.code == 4


def test_graph_and_direct_launches_agree():
    # the PS phase of a batch runs as one captured CUDA graph by default;
    # launching its kernels directly gives the same bits
    from paper_2208_05683_gb300 import _abi
    cases = mixed_cases()
    Zs = [dev(Z) for _, Z, _, _, _ in cases]
    old = psf.tune_get(_abi.PSF_TUNE_BATCH_GRAPH)
    try:
        out = {}
        for g in (1.0, 0.0):
            psf.tune_set(_abi.PSF_TUNE_BATCH_GRAPH, g)
            series = [series_of(a, tol, **kw) for _, _, a, tol, kw in cases]
            out[g] = psf.eval_batch(series, Zs)
        for (name, *_), a, b in zip(cases, out[1.0], out[0.0]):
            for x, y in zip(a.csr.to_host(), b.csr.to_host()):
                assert np.array_equal(x, y), name
            assert a.steps == b.steps, name
    finally:
        psf.tune_set(_abi.PSF_TUNE_BATCH_GRAPH, old)


def test_baby_steps_from_norm_phase_powers_bitwise():
    # while an instance has dropped no entry, its batched baby step k <= 10 is
    # copied from the power Z^k of the norm phase; an instance that drops
    # entries (loose tolerance), one with q = 12 > 10, a submultiplicative one
    # (no powers) and an unfiltered one share the batch.  Every result and
    # step record equals the oracle's and the product-only run's.
    from paper_2208_05683_gb300 import _abi
    poly150 = [(-1.0) ** i / math.factorial(i) for i in range(150)]
    cases = [
        ("lap2d exp", ocsr(syn.laplacian_2d(40)), syn.coeffs("exp"), 1e-12, {}),
        ("banded drop", ocsr(syn.banded_random(3000, 5, 7, 4.0)), syn.coeffs("exp"), 1e-6, {}),
        ("poly q=12", ocsr(syn.banded_random(300, 2, 11, 1.0)), poly150, 1e-11, {"poly": True}),
        ("submult", ocsr(syn.laplacian_1d(300)), syn.coeffs("exp"), 1e-12, {"submult": True}),
        ("unfiltered", ocsr(syn.laplacian_1d(200)), syn.coeffs("cos"), 1e-12, {"filtered": False}),
        ("banded 1e-12", ocsr(syn.banded_random(2000, 5, 8, 2.0)), syn.coeffs("cosh"), 1e-12, {}),
    ]
    Zs = [dev(Z) for _, Z, _, _, _ in cases]
    old = psf.tune_get(_abi.PSF_TUNE_BATCH_REUSE)
    try:
        out = {}
        for reuse in (1.0, 0.0):
            psf.tune_set(_abi.PSF_TUNE_BATCH_REUSE, reuse)
            series = [series_of(a, tol, **kw) for _, _, a, tol, kw in cases]
            out[reuse] = psf.eval_batch(series, Zs)
    finally:
        psf.tune_set(_abi.PSF_TUNE_BATCH_REUSE, old)
    for (name, Z, a, tol, kw), r, p in zip(cases, out[1.0], out[0.0]):
        ref = psscf(Z, a, tol, **kw)
        check_same(r, ref, name)
        for x, y in zip(r.csr.to_host(), p.csr.to_host()):
            assert np.array_equal(x, y), name
        assert r.steps == p.steps, name
    # the poly case really has q > 10, the drop case drops in a baby step
    assert out[1.0][2].info["q"] == 12
    assert any(s["kind"] == "baby" and s["nnz_post"] < s["nnz_pre"] for s in out[1.0][1].steps)


@pytest.mark.parametrize("shift", [0, 1])
def test_batch_far_candidate_split_bitwise(shift):
    # batched Algorithm 1 with the far candidates set apart per instance at
    # eps_g / 2^shift: the same bits as the default
    from paper_2208_05683_gb300 import _abi
    cases = mixed_cases()
    Zs = [dev(Z) for _, Z, _, _, _ in cases]
    old = psf.tune_get(_abi.PSF_TUNE_ALG1_FAR_SHIFT)
    try:
        psf.tune_set(_abi.PSF_TUNE_ALG1_FAR_SHIFT, float(shift))
        got = psf.eval_batch([series_of(a, tol, **kw) for _, _, a, tol, kw in cases], Zs)
    finally:
        psf.tune_set(_abi.PSF_TUNE_ALG1_FAR_SHIFT, old)
    for (name, Z, a, tol, kw), g in zip(cases, got):
        check_same(g, psscf(Z, a, tol, **kw), f"{name} shift {shift}")


def test_batch_rejects_estimated_norms():
    Z = dev(ocsr(syn.laplacian_1d(50)))
    with pytest.raises(psf.PsfError) as e:
        psf.eval_batch([psf.Series(syn.coeffs("exp"), 1e-12, estimate=True)], [Z])
    assert e.value.code == 1


def square_cases():
    """Instances with the W = Z^2 substitution (PSF_Z_SQUARE)."""
    cos, cosh, sinh = syn.coeffs("cos"), syn.coeffs("cosh"), syn.coeffs("sinh")
    odd_poly = [1.0 / math.factorial(i) if i % 2 else 0.0 for i in range(20)]
    return [
        ("sq lap2d cos", ocsr(syn.laplacian_2d(24)), cos, 1e-12, {}),
        ("sq banded sinh", ocsr(syn.banded_random(700, 6, 3, 2.0)), sinh, 1e-10, {}),
        # baby steps in W drop entries
        ("sq banded loose cosh", ocsr(syn.banded_random(900, 5, 7, 4.0)), cosh, 1e-6, {}),
        # g truncated to c_0: F = Z (c_0 I)
        ("sq sinh N_W=1", ocsr(syn.banded_random(60, 2, 4, 0.5)), sinh, 10.0, {}),
        ("sq zero sinh", CSR.empty(30), sinh, 1e-12, {}),
        ("sq zero cos", CSR.empty(12), cos, 1e-12, {}),
        ("sq n=1 sinh", CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([-0.75])), sinh,
         1e-12, {}),
        ("sq s=2 cos", ocsr(syn.laplacian_2d(20)), cos, 1e-12, {"s": 2}),
        ("sq poly odd", ocsr(syn.banded_random(500, 2, 5, 1.5)), odd_poly, 1e-11, {"poly": True}),
        ("sq unfiltered", ocsr(syn.laplacian_1d(128)), cosh, 1e-12, {"filtered": False}),
        ("sq submult", ocsr(syn.laplacian_1d(300)), sinh, 1e-12, {"submult": True}),
    ]


@pytest.mark.parametrize("graph", [1, 0])
def test_square_instances_in_a_mixed_batch(graph):
    # square instances (even, odd, trivial, empty) batched with plain ones:
    # each result is the oracle's and the single evaluation's, bit for bit
    cases = [(n, Z, a, tol, dict(kw, square=True)) for n, Z, a, tol, kw in square_cases()] + mixed_cases()[:7]
    series = [series_of(a, tol, **kw) for _, _, a, tol, kw in cases]
    old = psf.tune_get(_abi.PSF_TUNE_BATCH_GRAPH)
    psf.tune_set(_abi.PSF_TUNE_BATCH_GRAPH, graph)
    try:
        got = psf.eval_batch(series, [dev(Z) for _, Z, _, _, _ in cases])
    finally:
        psf.tune_set(_abi.PSF_TUNE_BATCH_GRAPH, old)
    for (name, Z, a, tol, kw), g in zip(cases, got):
        ref = psscf(Z, a, tol, **kw)
        check_same(g, ref, name)
        alone = series_of(a, tol, **kw).eval(dev(Z))
        assert alone.steps == g.steps, name
        for key in ("N", "q", "b", "g", "products", "z", "trunc", "budget", "nnz"):
            assert alone.info[key] == g.info[key], (name, key)


def test_wide_column_window_in_a_repeated_batch():
    # the 160 x 160 Laplacian's giant-step rows span about 6400 columns: the
    # second batch of the same series runs those stages with the bitmap's
    # wide column window; both batches give the oracle's results bit for bit
    big = ocsr(syn.laplacian_2d(160))
    small = ocsr(syn.banded_random(700, 6, 3, 2.0))
    a = syn.coeffs("exp")
    series = [psf.Series(a, 1e-12), psf.Series(a, 1e-12)]
    refs = [psscf(big, a, 1e-12), psscf(small, a, 1e-12)]
    for run in range(2):
        got = psf.eval_batch(series, [dev(big), dev(small)])
        for g, ref, name in zip(got, refs, ("lap2d 160", "banded")):
            check_same(g, ref, f"{name} run {run}")
