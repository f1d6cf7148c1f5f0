"""Host logic of bench.py on the CPU: the reference arm's JSON line and the
clock-sample summary (no GPU needed)."""
import datetime
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import bench  # noqa: E402

KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config"}


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-budget", "2"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d) and d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    cb = d["cpu_baseline"]
    assert {"value", "unit", "cores", "kind", "sample"} <= set(cb) and cb["kind"] == "oracle"
    assert cb["value"] == d["value"] and cb["cores"] >= 1
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("uniform batch")


def _line(ts, sm, smax, reasons=("Not Active",) * 4):
    stamp = datetime.datetime.fromtimestamp(ts).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([stamp, "0", str(sm), str(smax), "900.0", "0x0"] + list(reasons))


def test_clock_summary_keeps_the_timed_window_and_reasons():
    t = 1_800_000_000.0
    out = "\n".join([_line(t - 1.0, 345, 2070),           # before the window: idle
                     _line(t + 0.1, 2070, 2070),
                     _line(t + 0.2, 2055, 2070, ("Not Active", "Not Active", "Not Active", "Active")),
                     _line(t + 0.3, 2070, 2070),
                     _line(t + 5.0, 500, 2070, ("Active", "Not Active", "Not Active", "Not Active"))])  # after
    c = bench.ClockSampler.summarise(out, t, t + 1.0)
    assert c["samples"] == 3 and c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]  # the hw_slowdown sample lies outside the window
    assert bench.ClockSampler.summarise("", t, t + 1)["sm_mhz"] is None
