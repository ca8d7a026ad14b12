"""The benchmark's reference arm (the oracle on a bounded sample) prints one
JSON line with the contract's keys, on the timed workload's config; it needs
no GPU.  Tiny sample, one step."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--ref-sample-n", "3000"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "pairs/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1
    assert d["config"]["n"] == 1_000_000 and d["config"]["sample_n"] == 3000
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_clock_summary_keeps_only_the_timed_region():
    """The clock record takes the nvidia-smi rows stamped inside the timed
    region (20 ms slack) and reports the throttle reasons active there."""
    import datetime

    sys.path.insert(0, ROOT)
    import bench

    base = datetime.datetime(2026, 1, 2, 3, 4, 5)

    def row(ms, mhz, thermal="Not Active", power="Not Active"):
        ts = (base + datetime.timedelta(milliseconds=ms)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {mhz}, 2070, 900.5, 0x0, Not Active, Not Active, {thermal}, {power}"

    lines = [row(0, 900, thermal="Active"), row(100, 2070), row(120, 2055, power="Active"), row(140, 2070),
             row(400, 1200, thermal="Active")]
    t0 = (base + datetime.timedelta(milliseconds=90)).timestamp()
    t1 = (base + datetime.timedelta(milliseconds=150)).timestamp()
    got = bench.ClockSampler.summarise(lines, t0, t1)
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3,
                   "timed_region_only": True}
    assert bench.ClockSampler.summarise(lines, t1 + 1.0, t1 + 2.0) is None
    whole = bench.ClockSampler.summarise(lines, None, None)
    assert whole["samples"] == 5 and not whole["timed_region_only"]
    assert whole["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]
