"""The bench's reference arm (the FP64 oracle on the host cores) keeps the JSON-line contract:
one line from rank 0 with the metric, the timing fields, the warm-up it actually ran, a
`cpu_baseline` that describes the run and an `e2e` object without host-device copies; any other
rank prints nothing and exits 0. Also the clocks record that every GPU line carries, from
nvidia-smi rows given as text. Runs on the CPU (the reference arm launches no GPU work)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env, *argv):
    env = dict(os.environ)
    env.update(extra_env)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", *argv], cwd=ROOT,
                          env=env, capture_output=True, text=True, timeout=600)


def test_reference_line(oracle_mod):
    r = _run({"RANK": "0", "WORLD_SIZE": "1"}, "--steps", "2", "--warmup", "5")
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "MLUPS" and d["unit"] == "MLUPS"
    assert d["higher_is_better"] is True and d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["n_gpus"] == 1 and d["steps"] == 2
    # the warm-up is floored at 3 steps and capped at 3 for the slow oracle: 3 ran
    assert d["warmup"] == 3
    assert d["value"] > 0 and d["ms_per_step"] > 0
    # value = nodes x steps / time
    nodes = d["config"]["nx"] * d["config"]["ny"]
    assert d["value"] == pytest.approx(nodes / (d["ms_per_step"] * 1e3), rel=1e-9)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "2 FP64 oracle steps" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_other_ranks_are_silent(oracle_mod):
    r = _run({"RANK": "1", "WORLD_SIZE": "2"}, "--steps", "2", "--warmup", "3")
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_clock_summary_from_nvidia_smi_rows():
    """The clocks record of a bench line from nvidia-smi's CSV rows (sm, max sm, then the four
    throttle reasons): the median SM clock, the maximum, and each reason seen Active at least
    once; malformed rows are skipped, and no rows at all read as unsampled."""
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.out = "\n".join([
        "2070, 2070, Not Active, Not Active, Not Active, Not Active",
        "1980, 2070, Not Active, Not Active, Not Active, Active",
        "2070, 2070, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "[N/A], 2070, Not Active, Not Active, Not Active, Not Active",
    ])
    s = c.summary()
    assert s["samples"] == 4 and s["sm_max_mhz"] == 2070.0
    assert s["sm_mhz"] == 2070.0            # median of 2070, 1980, 2070 (N/A skipped)
    assert s["reasons"] == ["sw_power_cap"]
    c.out = "1500, 2070, Active, Not Active, Active, Not Active"
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.out = ""
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                           "samples": 0}
