"""psf_autotune through the C ABI: it times both slot maps of the product
kernel on an evaluation and sets the crossover; the results do not depend on
the setting (bitwise)."""
import pytest

import synthetic as syn
from gpu_helpers import assert_csr_bitwise, check_same, dev, ocsr
from oracle import psscf

pytestmark = pytest.mark.gpu

psf = pytest.importorskip("paper_2208_05683_gb300")
from paper_2208_05683_gb300 import _abi  # noqa: E402


def test_autotune_sets_a_crossover_and_keeps_results():
    old = psf.tune_get(_abi.PSF_TUNE_TABLE_CROSSOVER)
    try:
        Z = ocsr(syn.laplacian_2d(48))
        s = psf.Series(syn.coeffs("exp"), 1e-12)
        c, saved = psf.autotune(s, dev(Z))
        assert c >= 0.0 and saved >= 0.0
        assert psf.tune_get(_abi.PSF_TUNE_TABLE_CROSSOVER) == c
        ref = psscf(Z, syn.coeffs("exp"), 1e-12)
        for crossover in (c, 0.0, 1e300):
            psf.tune_set(_abi.PSF_TUNE_TABLE_CROSSOVER, crossover)
            assert_csr_bitwise(s.eval(dev(Z)).csr, ref.F, f"crossover {crossover}")
    finally:
        psf.tune_set(_abi.PSF_TUNE_TABLE_CROSSOVER, old)


def test_autotune_batch_picks_settings_and_keeps_results():
    keys = (_abi.PSF_TUNE_TABLE_CROSSOVER, _abi.PSF_TUNE_ROW_BITMAPS, _abi.PSF_TUNE_BATCH_REUSE)
    old = [psf.tune_get(k) for k in keys]
    try:
        cases = [(ocsr(syn.laplacian_2d(16 + 4 * (i % 5))), ("exp", "cos", "sinh")[i % 3]) for i in range(12)]
        cases.append((ocsr(syn.banded_random(900, 5, 7, 2.0)), "exp"))
        series = [psf.Series(syn.coeffs(k), 1e-12) for _, k in cases]
        Zs = [dev(Z) for Z, _ in cases]
        t = psf.autotune_batch(series, Zs)
        assert t["configs"] == 4 and t["launches"] > 0
        assert t["row_bitmaps"] in (0, 1) and t["batch_reuse"] in (0, 1) and t["table_crossover"] >= 0.0
        assert 0.0 < t["ms_after"] and 0.0 < t["ms_before"]
        assert psf.tune_get(_abi.PSF_TUNE_TABLE_CROSSOVER) == t["table_crossover"]
        assert psf.tune_get(_abi.PSF_TUNE_ROW_BITMAPS) == t["row_bitmaps"]
        assert psf.tune_get(_abi.PSF_TUNE_BATCH_REUSE) == t["batch_reuse"]
        got = psf.eval_batch(series, Zs)
        for (Z, k), g in zip(cases, got):
            check_same(g, psscf(Z, syn.coeffs(k), 1e-12), k)
    finally:
        for k, v in zip(keys, old):
            psf.tune_set(k, v)
