"""bench.py's reference arm (the FP64 oracle timed on the host cores) prints the JSON line
of the benchmark contract; checked on a small grid so that it runs in seconds on CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
        "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
        "cpu_baseline", "e2e")


def test_reference_arm_prints_the_contract_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
           "--warmup", "1", "--shape", "16", "16", "16", "--nt", "8"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in KEYS:
        assert k in line, k
    assert line["impl"] == "reference" and line["unit"] == "gradients/hour"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1
    assert abs(line["ms_per_step"] - 3600e3 / line["value"]) < 1e-6 * line["ms_per_step"]
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["value"] == line["value"] and cpu["cores"] >= 1
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["grid"] == [16, 16, 16] and line["config"]["nt"] == 8


def test_clock_summary_reads_nvidia_smi_rows():
    """The sampler's summary: median SM clock under load, the maximum clock, and every
    throttle reason seen Active in any sample; malformed or unavailable rows are skipped
    (nvidia-smi prints "[N/A]" or "Not Active" in these columns)."""
    sys.path.insert(0, ROOT)
    import bench
    s = bench.ClockSampler(0)
    s.rows = [
        ["0", "2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["0", "2055", "2070", "1390.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
        ["0", "[N/A]", "2070", "1390.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["0", "1980", "2070", "1400.2", "0x20", "Not Active", "Not Active", "Active", "Not Active"],
        ["garbage"],
    ]
    out = s.summary()
    assert out["samples"] == 3 and out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]
    s.rows = []
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
