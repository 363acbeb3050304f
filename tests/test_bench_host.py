"""Host logic of bench.py on CPU: the clock record keeps only the samples taken
inside the timed windows and reports every throttle reason seen there, and the
reference arm prints one JSON line with the keys of the benchmark line."""
import datetime
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(ts: float, sm: float, reasons=("Not Active",) * 4) -> str:
    stamp = datetime.datetime.fromtimestamp(ts).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([stamp, f"{sm:.0f}", "2070", "900.00", "0x0000000000000000", *reasons])


def test_clock_summary_keeps_timed_windows_and_reasons():
    cs = bench.ClockSampler(0)
    t0 = 1_800_000_000.0
    cs.lines = [_line(t0 - 1.0, 900.0),                                  # before the window: dropped
                _line(t0 + 0.10, 2070.0),
                _line(t0 + 0.12, 2055.0, ("Not Active", "Not Active", "Not Active", "Active")),
                _line(t0 + 0.14, 2070.0),
                _line(t0 + 5.0, 1000.0, ("Active", "Not Active", "Not Active", "Not Active")),  # after: dropped
                "garbage, line"]
    cs.mark(t0 + 0.09, t0 + 0.15)
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 3


def test_clock_summary_without_samples():
    cs = bench.ClockSampler(0)
    cs.mark(1.0, 2.0)
    s = cs.summary()
    assert s["sm_mhz"] is None and s["reasons"] == [] and s["samples"] == 0


def test_reference_arm_line_has_the_benchmark_keys():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--sample-clusters", "2"], capture_output=True, text=True, timeout=600,
                       env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]
