"""Failure paths, driven without faulting or hanging the GPU.

- A grid-barrier wait that runs out: with the wait limit set to 0, every
  block of a cooperative kernel that reaches an incomplete barrier gives up at
  once, records a device status and returns; the call reports PSF_ETIMEOUT.
- An allocation failure injected at serving admission: that request alone
  completes with PSF_ENOMEM.
- A request cancelled while it waits for admission completes with
  PSF_ECANCELED and frees its place.

After each, results are bitwise the oracle's (the control block of every
call is its own, so nothing carries over).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synthetic as syn
from gpu_helpers import assert_csr_bitwise, check_same, dev, ocsr
from oracle import CSR, alg1, matmul_add, norm1, psscf

pytestmark = pytest.mark.gpu

psf = pytest.importorskip("paper_2208_05683_gb300")
from paper_2208_05683_gb300 import _abi  # noqa: E402


def rand_csr(n, density, seed, mag_spread=0.0):
    rng = np.random.default_rng(seed)
    m = sp.random(n, n, density=density, random_state=rng, format="csr",
                  data_rvs=lambda k: rng.uniform(-1, 1, k) * 10.0 ** (-mag_spread * rng.uniform(0, 1, k)))
    return CSR.from_scipy(m)


def test_barrier_wait_runs_out_then_everything_recovers():
    A = rand_csr(300, 0.05, 11, mag_spread=20)
    B = rand_csr(300, 0.05, 12, mag_spread=20)
    Z = ocsr(syn.laplacian_2d(32))
    old = psf.tune_get(_abi.PSF_TUNE_BARRIER_BUDGET_NS)
    assert old == 2e9
    psf.tune_set(_abi.PSF_TUNE_BARRIER_BUDGET_NS, 0)
    try:
        # Algorithm 1's passes (k_alg1), the exact norm (k_norms) and a whole
        # evaluation each stop at their first grid barrier
        with pytest.raises(psf.PsfError) as e:
            psf.product_filter(dev(A), dev(B), [], 1e-6, 0.1)
        assert e.value.code == _abi.PSF_ETIMEOUT
        with pytest.raises(psf.PsfError) as e:
            psf.norm1(dev(A))
        assert e.value.code == _abi.PSF_ETIMEOUT
        with pytest.raises(psf.PsfError) as e:
            psf.Series(syn.coeffs("exp"), 1e-12).eval(dev(Z))
        assert e.value.code == _abi.PSF_ETIMEOUT
    finally:
        psf.tune_set(_abi.PSF_TUNE_BARRIER_BUDGET_NS, old)
    C = matmul_add(A, B)
    ref = alg1(C, 1e-6 / 1.1, 0.1)
    got = psf.product_filter(dev(A), dev(B), [], 1e-6, 0.1)
    assert_csr_bitwise(got.csr, ref.kept)
    assert got.steps[0]["iters"] == ref.iters and ref.iters >= 2
    assert psf.norm1(dev(A)) == norm1(A)
    check_same(psf.Series(syn.coeffs("exp"), 1e-12).eval(dev(Z)), psscf(Z, syn.coeffs("exp"), 1e-12))


def test_barrier_budget_key_checks():
    for bad in (-1, 0.5, 7e10):
        with pytest.raises(psf.PsfError):
            psf.tune_set(_abi.PSF_TUNE_BARRIER_BUDGET_NS, bad)
    with pytest.raises(psf.PsfError):
        psf.tune_set(_abi.PSF_TUNE_FAIL_ADMISSION, -1)


def requests(count):
    out = []
    for i in range(count):
        m = 16 + 4 * (i % 5)
        kind = ("exp", "cos", "sinh")[i % 3]
        out.append((ocsr(syn.laplacian_2d(m)), kind))
    return out


def test_admission_failure_fails_that_request_alone():
    reqs = requests(6)
    refs = [psscf(Z, syn.coeffs(k), 1e-12) for Z, k in reqs]
    series = [psf.Series(syn.coeffs(k), 1e-12) for _, k in reqs]
    Zs = [dev(Z) for Z, _ in reqs]
    srv = psf.Server(workers=1, max_batch=8)
    try:
        psf.tune_set(_abi.PSF_TUNE_FAIL_ADMISSION, 3)
        for i in range(len(reqs)):
            srv.submit(series[i], Zs[i], i)
        done = []
        while len(done) < len(reqs):
            done += srv.poll(16, 1000)
        assert psf.tune_get(_abi.PSF_TUNE_FAIL_ADMISSION) == 0  # used once
        # one worker admits in submission order: the third request fails
        failed = [c for c in done if c["status"] != _abi.PSF_OK]
        assert [(c["tag"], c["status"]) for c in failed] == [(2, _abi.PSF_ENOMEM)]
        assert failed[0]["result"] is None
        for c in done:
            if c["tag"] != 2:
                check_same(c["result"], refs[c["tag"]], f"request {c['tag']}")
        st = srv.stats()
        assert st["completed"] == 6 and st["failed"] == 1
    finally:
        psf.tune_set(_abi.PSF_TUNE_FAIL_ADMISSION, 0)
        srv.close()


def test_cancel_a_waiting_request():
    reqs = [(ocsr(syn.laplacian_2d(48)), "exp")] * 29 + [(ocsr(syn.laplacian_2d(20)), "cos")]
    series = [psf.Series(syn.coeffs(k), 1e-12) for _, k in reqs]
    Zs = [dev(Z) for Z, _ in reqs]
    srv = psf.Server(workers=1, max_batch=1)
    try:
        for i in range(len(reqs)):
            srv.submit(series[i], Zs[i], i)
        # 29 requests of about a millisecond each are ahead of the last one
        assert srv.cancel(29) is True
        assert srv.cancel(29) is False  # no longer waiting
        assert srv.cancel(12345) is False  # never submitted
        done = []
        while len(done) < len(reqs):
            done += srv.poll(64, 1000)
        by_tag = {c["tag"]: c for c in done}
        assert by_tag[29]["status"] == _abi.PSF_ECANCELED and by_tag[29]["result"] is None
        ref = psscf(reqs[0][0], syn.coeffs("exp"), 1e-12)
        for t in (0, 13, 28):
            assert by_tag[t]["status"] == _abi.PSF_OK
            check_same(by_tag[t]["result"], ref, f"request {t}")
        assert all(by_tag[t]["status"] == _abi.PSF_OK for t in range(29))
        st = srv.stats()
        assert st["cancelled"] == 1 and st["completed"] == 30 and st["failed"] == 0
        assert srv.cancel(5) is False  # finished requests cannot be cancelled
    finally:
        srv.close()
