"""Host logic of bench.py that needs no GPU: the clock record keeps only the
nvidia-smi samples taken inside the timed region and reports the throttle
reasons seen there."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

NA = "Not Active"


def _line(mhz, hw="Not Active", cap="Not Active"):
    return f"0, {mhz}, 2070, 700.0, 0x0, {hw}, {NA}, {NA}, {cap}"


def test_clock_summary_keeps_samples_inside_the_timed_region():
    c = bench.ClockSampler(0)
    c.lines = [(0.2, _line(345)), (1.00, _line(2070)), (1.04, _line(2055, cap="Active")),
               (1.06, _line(2070)), (5.0, _line(300, hw="Active"))]
    c.t_start, c.t_end = 0.9, 1.03
    s = c.summary()
    # the idle sample before and the one long after the region are left out;
    # the one that arrived within an interval of the end is kept
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_without_samples_says_so():
    c = bench.ClockSampler(0)
    c.t_start, c.t_end = 1.0, 2.0
    c.lines = [(0.1, _line(2070)), (9.0, "garbled")]
    assert c.summary()["reasons"] == ["unsampled"]


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) prints
    one JSON line with the benchmark's metric and unit, impl = reference, its
    CPU baseline and a zero-copy end-to-end figure."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "evals/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
