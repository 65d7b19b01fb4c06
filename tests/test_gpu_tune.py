"""psf_autotune through the C ABI: it times both slot maps of the product
kernel on an evaluation and sets the crossover; the results do not depend on
the setting (bitwise)."""
import pytest

import synthetic as syn
from gpu_helpers import assert_csr_bitwise, dev, ocsr
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
