"""bench.py's reference arm (the oracle timed on the host) and its JSON line,
on the CPU: the keys the benchmark contract fixes, and a rank other than 0
exiting without work."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env_extra=None, timeout=600):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                          timeout=timeout, env=env, cwd=ROOT)


@pytest.mark.slow
def test_reference_arm_prints_one_contract_line():
    out = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "evals/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["config"]["workload"].startswith("lap2d_128x128")
    assert set(d["cpu_baseline"]) >= {"value", "unit", "cores", "kind", "sample"}
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    out = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"],
                    {"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}, timeout=120)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""


def test_clock_summary_keeps_the_timed_window():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    #        index, sm, max, power, active, hw_slow, hw_therm, sw_therm, sw_power_cap
    idle = ["0", "1400", "2070", "300", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]
    busy = ["0", "2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]
    capped = ["0", "1900", "2070", "1400", "0x4", "Not Active", "Not Active", "Not Active", "Active"]
    c.rows = [(0.0, idle), (1.0, busy), (1.05, capped), (1.1, busy), (5.0, idle)]
    c.mark(0.9, 1.08)
    s = c.summary()
    # samples up to one period after the window's end belong to it
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    c.mark(2.0, 3.0)
    assert c.summary()["reasons"] == ["unsampled"]


def test_reference_and_repo_arms_share_the_config():
    sys.path.insert(0, ROOT)
    import bench
    cfg = bench.config_dict(128 * 128, 81408, 1)
    assert cfg["workload"] == "lap2d_128x128 exp+cos tol 1e-12" and cfg["parallelism"] == "replicas x1"
    # both arms build their config with this one function
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert src.count("config_dict(") == 3  # the definition and the two arms


def test_dense_ps_baseline_matches_closed_form_and_oracle():
    # the dense baseline on the CPU (torch float64): same plan as the sparse
    # scheme, unfiltered, against the 1D Laplacian's closed form and the
    # oracle's unfiltered PS
    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synthetic as syn
    m = 40
    rp, col, val = syn.laplacian_1d(m)
    Z = oracle.CSR(m, rp, col, val)
    a = syn.coeffs("exp")
    ref = oracle.psscf(Z, a, 1e-12, filtered=False)
    p = ref.plan
    D = bench.dense_ps(torch.as_tensor(Z.to_dense()), a, p.N, p.q, p.b).numpy()
    F = bench.lap1d_closed_form(m, "exp")
    err = np.abs(D - F).sum(axis=0).max() / np.abs(F).sum(axis=0).max()
    assert err <= 1e-12
    U = ref.F.to_dense()
    assert np.abs(D - U).max() <= 1e-14 * np.abs(U).max()
    # cos through the Kronecker closed form of a small 2D Laplacian
    c, s = bench.lap1d_closed_form(6, "cos"), bench.lap1d_closed_form(6, "sin")
    Z2 = oracle.CSR(36, *syn.laplacian_2d(6))
    a = syn.coeffs("cos")
    p = oracle.psscf(Z2, a, 1e-12).plan
    D2 = bench.dense_ps(torch.as_tensor(Z2.to_dense()), a, p.N, p.q, p.b).numpy()
    F2 = np.kron(c, c) - np.kron(s, s)
    assert np.abs(D2 - F2).sum(axis=0).max() <= 1e-12 * np.abs(F2).sum(axis=0).max()
