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
