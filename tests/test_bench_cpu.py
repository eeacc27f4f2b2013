"""Host logic of bench.py that needs no GPU: the clock sampler keeps the
samples taken inside the timed region (a stand-in nvidia-smi on PATH)."""
import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FAKE = """#!/usr/bin/env python3
import datetime, time
while True:
    t = datetime.datetime.now().strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    print(t + ", 0, 2070, 2070, 900.5, 0x4, Not Active, Not Active, Not Active, Active",
          flush=True)
    time.sleep(0.02)
"""


@pytest.fixture
def fake_smi(tmp_path, monkeypatch):
    p = tmp_path / "nvidia-smi"
    p.write_text(FAKE)
    p.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_clock_samples_inside_the_region(fake_smi):
    c = fake_smi.Clocks(0)
    c.start()
    time.sleep(0.25)
    r = c.stop()
    assert r["in_region"] and r["samples"] >= 5
    assert r["sm_mhz"] == 2070 and r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["sw_power_cap"]
    assert r["region_ms"] >= 250


def test_short_region_falls_back_to_the_nearest_sample(fake_smi):
    c = fake_smi.Clocks(0, interval_ms=200)
    c.start()
    r = c.stop()                   # a region of a few microseconds
    assert r["samples"] >= 1 and r["sm_mhz"] == 2070


def test_reference_arm_prints_the_contract_line():
    # bench.py --impl reference times the FP64 oracle on the host cores (no
    # GPU): one JSON line with the contract's keys, its e2e without copies and
    # a cpu_baseline that describes this run
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    import bench
    assert j["impl"] == "reference" and j["metric"] == bench.METRIC and j["unit"] == bench.UNIT
    assert j["value"] > 0 and j["ms_per_step"] > 0 and j["higher_is_better"] is True
    assert (j["n_gpus"], j["steps"], j["warmup"]) == (1, 1, 0)
    assert j["config"]["workload"] == bench.WORKLOAD and j["data"] == "synthetic"
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == j["value"]
    assert isinstance(cb["sample"], str) and cb["sample"]
    assert j["e2e"] == {"value": j["value"], "unit": j["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
