"""The serving loop (psf_server_*) through the C ABI: continuous batching of
a mixed request stream.

Each request's result must be bitwise the result of evaluating it alone
(psf_eval), and a sample is checked against the oracle, while requests are
batched together and batches overlap on the device.
"""
import time

import numpy as np
import pytest

import synthetic as syn
from gpu_helpers import assert_csr_bitwise, check_same, dev, ocsr
from oracle import psscf

pytestmark = pytest.mark.gpu

psf = pytest.importorskip("paper_2208_05683_gb300")


def same_csr(a, b, what):
    for x, y in zip(a.to_host(), b.to_host()):
        assert np.array_equal(x.view(np.int64) if x.dtype == np.float64 else x,
                              y.view(np.int64) if y.dtype == np.float64 else y), what


def drain(srv, count, timeout_s=120.0):
    done = {}
    t0 = time.time()
    while len(done) < count:
        for c in srv.poll(64, 200):
            done[c["tag"]] = c
        assert time.time() - t0 < timeout_s, "requests did not complete"
    return done


def test_results_identical_alone_and_in_the_mix():
    reqs = syn.serving_requests(40, seed0=100, n_lo=64, n_hi=4096)
    series = [psf.Series(syn.coeffs(k), tol) for _, k, tol in reqs]
    Zs = [dev(Z) for Z, _, _ in reqs]
    srv = psf.Server(workers=3, max_batch=8)
    try:
        # a burst (fills two workers with batches), then Poisson arrivals
        rng = np.random.default_rng(7)
        for i in range(12):
            srv.submit(series[i], Zs[i], i)
        done = {}
        for i in range(12, len(reqs)):
            time.sleep(float(rng.exponential(0.002)))
            srv.submit(series[i], Zs[i], i)
            for c in srv.poll(64, 0):
                done[c["tag"]] = c
        done.update(drain(srv, len(reqs) - len(done)))
        stats = srv.stats()
    finally:
        srv.close()
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["max_concurrent"] >= 2, stats  # batches overlapped on the device
    assert max(c["batch_size"] for c in done.values()) > 1  # arrivals were batched
    for i, (Z, kind, tol) in enumerate(reqs):
        c = done[i]
        assert c["status"] == 0 and c["latency_ms"] >= c["queue_ms"] >= 0.0
        alone = series[i].eval(Zs[i])
        same_csr(c["result"].csr, alone.csr, f"request {i}")
        assert c["result"].steps == alone.steps
    for i in (0, 5, 17, 33):
        Z, kind, tol = reqs[i]
        check_same(done[i]["result"], psscf(ocsr(Z), syn.coeffs(kind), tol), f"request {i}")


def test_small_memory_budget_serializes_without_deadlock():
    reqs = syn.serving_requests(10, seed0=300, n_lo=64, n_hi=1024)
    series = [psf.Series(syn.coeffs(k), tol) for _, k, tol in reqs]
    Zs = [dev(Z) for Z, _, _ in reqs]
    srv = psf.Server(workers=4, max_batch=8, hbm_budget=1)  # every request alone
    try:
        for i in range(len(reqs)):
            srv.submit(series[i], Zs[i], i)
        done = drain(srv, len(reqs))
        stats = srv.stats()
    finally:
        srv.close()
    assert stats["max_concurrent"] == 1 and stats["batches"] == len(reqs)
    for i in range(len(reqs)):
        assert done[i]["batch_size"] == 1
        same_csr(done[i]["result"].csr, series[i].eval(Zs[i]).csr, f"request {i}")


def test_a_bad_request_fails_alone():
    good = [ocsr(syn.laplacian_1d(n)) for n in (50, 80, 120)]
    bad = dev((np.array([0, 1, 1, 1, 1, 1], np.int32), np.array([7], np.int32), np.array([1.0])))
    s = psf.Series(syn.coeffs("exp"), 1e-12)
    Zs = [dev(g) for g in good]
    srv = psf.Server(workers=1, max_batch=8)
    try:
        srv.submit(s, Zs[0], 0)
        srv.submit(s, bad, 1)
        srv.submit(s, Zs[1], 2)
        srv.submit(s, Zs[2], 3)
        done = drain(srv, 4)
    finally:
        srv.close()
    assert done[1]["status"] == 1 and done[1]["result"] is None
    for tag, Z in ((0, good[0]), (2, good[1]), (3, good[2])):
        assert done[tag]["status"] == 0
        assert_csr_bitwise(done[tag]["result"].csr, psscf(Z, syn.coeffs("exp"), 1e-12).F, f"request {tag}")


def test_submit_rejects_estimated_norms():
    Z = dev(ocsr(syn.laplacian_1d(50)))
    srv = psf.Server(workers=1, max_batch=4)
    try:
        with pytest.raises(psf.PsfError) as e:
            srv.submit(psf.Series(syn.coeffs("exp"), 1e-12, estimate=True), Z, 7)
        assert e.value.code == 1
    finally:
        srv.close()


def test_square_requests_in_the_mix():
    # requests with the W = Z^2 substitution batched with plain ones: each
    # result is the one it gets alone
    reqs = syn.serving_requests(24, seed0=300, n_lo=64, n_hi=2048)
    series = []
    for i, (_, kind, tol) in enumerate(reqs):
        sq = kind in ("cos", "sinh") and i % 2 == 0
        series.append(psf.Series(syn.coeffs(kind), tol, square=sq))
    assert any(s.flags & 16 for s in series)
    Zs = [dev(Z) for Z, _, _ in reqs]
    srv = psf.Server(workers=2, max_batch=8)
    try:
        for i in range(len(reqs)):
            srv.submit(series[i], Zs[i], i)
        done = drain(srv, len(reqs))
    finally:
        srv.close()
    for i in range(len(reqs)):
        c = done[i]
        assert c["status"] == 0, i
        alone = series[i].eval(Zs[i])
        same_csr(c["result"].csr, alone.csr, f"request {i}")
        assert c["result"].steps == alone.steps
