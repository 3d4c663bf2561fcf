"""Host logic of bench.py that needs no GPU: the clock record keeps only the
nvidia-smi samples taken inside the timed region and reports the throttle
reasons seen there; the committed DRAM-traffic record is of the current
kernel sources; the per-function roofline takes the largest unit bound."""
import os
import sys

import numpy as np

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


def test_traffic_record_is_of_the_current_kernel_sources():
    """roofline.traffic comes from profiles/traffic_per_call.txt only while the
    tensor-core kernel sources hash to the value recorded there; the
    committed record is of the sources as they are."""
    table, sha = bench._profile_traffic()
    assert table is not None, f"traffic record is stale (sources hash to {sha})"
    assert set(table) == {"tf32x3", "exact", "mixed"}
    # a light call moves at least its input once; the mixed group more
    assert table["tf32x3"] >= 4 * bench.D * bench.N
    assert table["mixed"] > table["exact"] > table["tf32x3"]


class _FakeInstance:
    """Two functions at D = 1000: fid 0 one rotated Sphere component (blocks
    500 + 500) on TF32X3; fid 1 one rotated Weierstrass component in ten
    blocks of 100 on EXACT."""

    def curob_num_components(self, f):
        return 1

    def curob_component_layout(self, f, c):
        return ([500, 500], True) if f == 0 else ([100] * 10, True)

    def curob_component_kinds(self, f, c):
        return [0, 0] if f == 0 else [8] * 10

    def curob_query_component_precision(self, f, c):
        return 1 if f == 0 else 4


def test_roofline_takes_the_largest_unit_bound(monkeypatch):
    N = 1 << 20
    monkeypatch.setattr(bench, "NFUN", 2)
    monkeypatch.setattr(bench, "D", 1000)
    monkeypatch.setattr(bench, "N", N)
    pk = {"bf16_tflops": 2000.0, "hbm_gbs": 8000.0, "sm_max_mhz": 2000.0}

    class Args:
        precision = "exact"  # no traffic figure for a forced precision

    launch_ms = np.array([5.0, 10.0])
    roof, per_fn = bench.roofline(_FakeInstance(), pk, "measured", [1, 4], launch_ms, [2, 3],
                                  Args())
    f0, f1 = per_fn
    # Sphere: 2 (500^2 + 500^2) flop per candidate at TF32X3's algorithmic
    # rate (2000 x 1.1/2.25 / 3 TFLOP/s) binds, above x read once (4004 B per
    # candidate at 8 TB/s); it needs no SFU work
    t_tensor0 = 2 * 500000 * N / (2000e12 * (1.1 / 2.25) / 3) * 1e3
    assert t_tensor0 > 4004 * N / 8e12 * 1e3
    assert f0["binding"] == "tensor" and f0["bound_ms"]["sfu"] == 0.0
    assert abs(f0["bound_ms"]["tensor"] - round(t_tensor0, 4)) < 1e-4
    # Weierstrass: 21 cosines per variable on 152 x 16 SFU lanes at 2 GHz
    # outweigh ten 100-wide blocks' contraction on EXACT (2000 / 10 TFLOP/s)
    t_sfu1 = 21 * 1000 * N / (152 * 16 * 2e9) * 1e3
    t_tensor1 = 2 * 10 * 100 * 100 * N / (2000e12 / 10) * 1e3
    assert t_sfu1 > t_tensor1
    assert f1["binding"] == "sfu"
    assert abs(f1["bound_ms"]["sfu"] - round(t_sfu1, 4)) < 1e-4
    assert abs(f1["bound_ms"]["tensor"] - round(t_tensor1, 4)) < 1e-4
    # every function's fraction is its largest bound over its time
    for r, ms in zip(per_fn, launch_ms):
        assert abs(r["frac_of_binding"] - round(max(r["bound_ms"].values()) / ms, 4)) < 1e-3
    # the dominant group is the precision with the most time (EXACT, 10 ms):
    # achieved = its algorithmic flops over its time, peak = EXACT's rate
    assert roof["kernel"].startswith("mma_eval_kernel<EXACT>")
    assert abs(roof["achieved"] - round(2 * 10 * 100 * 100 * N / 10e-3 / 1e12, 2)) < 1e-2
    assert abs(roof["peak"] - 200.0) < 0.1
    assert roof["traffic"] is None
