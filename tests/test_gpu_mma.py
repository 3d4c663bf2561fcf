"""Tensor-core path (tcgen05, TF32x3 / BF16x3 split products, FP32 accumulation
in TMEM) against the FP64 oracle at the FP32-rounded inputs, through the C
ABI.  D = 50 and 100 span several 16/32-column K stages and a ragged tail of
the 128-candidate tile; D = 1000, N = 16384 is the benchmarked launch, checked
on sampled rows."""
import json
import os

import numpy as np
import pytest

import gpu_util as gu
from paper_1407_7737_gb300 import inputs

pytestmark = pytest.mark.gpu
ALL = list(range(37))
# per-function error reports go to $CUROB_TEST_REPORTS when it names a directory
OUT = os.environ.get("CUROB_TEST_REPORTS")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    gu.invalidate()


def _sweep(orc, D, N, mode, rows=None, seed=0):
    import torch
    cu = gu.ensure(D, N, seed)
    cu.curob_set_precision(mode)
    report = {}
    try:
        for fid in ALL:
            try:
                cu.curob_query_precision(fid)
            except cu.CurobError:  # a forced tensor-core mode this function's blocks cannot use
                continue
            o = orc.generate(fid, D, seed)[0].o
            x32 = inputs.mixed(N, D, 700 + fid, center=o, frac_near=0.1,
                               sigma=1e-3).astype(np.float32)
            got = gu.gpu_eval(fid, x32, torch.float32)
            ok, worst, excused, raw = gu.fp32_check(orc, fid, D, seed, x32, got, rows)
            report[fid] = {"ok": ok, "ratio": raw, "excused": excused}
            if excused:
                # each excused row: the variable at the jump and the oracle on
                # both sides of it (printed with -s, saved with the report)
                from oracle import parity
                ex = parity.explain_excused(fid, D, seed, x32, got, rows)
                report[fid]["excused_rows"] = ex
                for e in ex:
                    print(f"fid {fid} D {D} mode {mode} excused row {e}")
    finally:
        cu.curob_set_precision(cu.PRECISION_AUTO)
    return report


def _save(name, rep):
    if not OUT:
        return
    os.makedirs(OUT, exist_ok=True)
    with open(os.path.join(OUT, name), "w") as f:
        json.dump(rep, f, indent=1)


@pytest.mark.parametrize("D,N", [(50, 4096), (100, 1000)])
def test_auto_precision_parity(orc, D, N):
    rep = _sweep(orc, D, N, 0)
    _save(f"mma_auto_D{D}.json", rep)
    bad = {f: r for f, r in rep.items() if not r["ok"]}
    assert not bad, bad


def test_auto_precision_parity_full_size(orc):
    """The benchmarked launch (D = 1000, N = 16384, AUTO), every row of every
    function against the oracle."""
    D, N = 1000, 16384
    rep = _sweep(orc, D, N, 0, None)
    _save("mma_auto_D1000.json", rep)
    bad = {f: r for f, r in rep.items() if not r["ok"]}
    assert not bad, bad
    # every excused row is a jump the FP32 rounding of z crossed: the value
    # matches the oracle on the other side of that jump
    crossed = {f: [e for e in r.get("excused_rows", []) if not e["gpu_on_other_side"]]
               for f, r in rep.items()}
    assert not any(crossed.values()), crossed


@pytest.mark.parametrize("mode", [1, 2, 6])
def test_forced_precisions_report(orc, mode):
    """TF32x3, BF16x3 and FP16x3 forced on every function at D = 1000 (sampled rows):
    the per-function error ratio is recorded (AUTO routes the functions that
    magnify contraction error elsewhere); every value is finite."""
    D, N = 1000, 16384
    rows = np.unique(np.r_[0, N - 1, np.random.default_rng(2).integers(0, N, 62)])
    rep = _sweep(orc, D, N, mode, rows)
    _save(f"mma_mode{mode}_D1000.json", rep)
    assert all(np.isfinite(r["ratio"]) for r in rep.values())


@pytest.mark.parametrize("D,N", [(50, 2048), (100, 1000), (1000, 16384)])
def test_exact_precision_every_function(orc, D, N):
    """EXACT (integer BF16 slices, exact accumulation) forced on every
    function meets the FP32 tolerance."""
    rows = None
    if N > 4096:
        rows = np.unique(np.r_[0, 127, 128, N - 1, np.random.default_rng(3).integers(0, N, 60)])
    rep = _sweep(orc, D, N, 4, rows)
    _save(f"mma_mode4_D{D}.json", rep)
    bad = {f: r for f, r in rep.items() if not r["ok"]}
    assert not bad, bad


def test_ragged_tails(orc):
    """N not a multiple of the 128-row tile, single candidates (the
    small-population kernels turned off, so the tensor-core kernel runs)."""
    import torch
    D = 96
    cu = gu.ensure(D, 512)
    cu.curob_set_small_batch(0)
    try:
        for N in (1, 127, 129, 300):
            for fid in (0, 8, 16, 29, 35):
                o = orc.generate(fid, D, 0)[0].o
                x32 = inputs.mixed(N, D, N, center=o, frac_near=0.2, sigma=1e-3).astype(np.float32)
                got = gu.gpu_eval(fid, x32, torch.float32)
                ok, *_ = gu.fp32_check(orc, fid, D, 0, x32, got)
                assert ok, (N, fid)
    finally:
        cu.curob_set_small_batch(512)


def test_mixed_compositions_choose_member_precisions():
    """AUTO runs a composition whose members differ in sensitivity as MIXED:
    members with Discus, Weierstrass, expanded Griewank-Rosenbrock or
    Katsuura on EXACT, the others on TF32X3 (their parity is covered by the
    AUTO sweeps above)."""
    cu = gu.ensure(100, 256)
    cu.curob_set_precision(cu.PRECISION_AUTO)
    # CF4 (ID 32): Schwefel, HappyCat, Elliptic, Weierstrass, Griewank
    assert cu.curob_query_precision(32) == cu.PRECISION_MIXED
    assert [cu.curob_query_component_precision(32, c) for c in range(5)] == \
        [cu.PRECISION_TF32X3] * 3 + [cu.PRECISION_EXACT, cu.PRECISION_TF32X3]
    # a plain sensitive function and a plain insensitive one
    assert cu.curob_query_precision(8) == cu.PRECISION_EXACT
    assert cu.curob_query_precision(0) == cu.PRECISION_TF32X3
    # forced modes stay whole-function
    cu.curob_set_precision(cu.PRECISION_EXACT)
    try:
        assert cu.curob_query_precision(32) == cu.PRECISION_EXACT
        assert cu.curob_query_component_precision(32, 0) == cu.PRECISION_EXACT
    finally:
        cu.curob_set_precision(cu.PRECISION_AUTO)
    with pytest.raises(cu.CurobError):
        cu.curob_set_precision(cu.PRECISION_MIXED)


def test_launch_counts_follow_the_split():
    """The transpose of x, then one launch for a function whose blocks the
    epilogue closes; one per precision group plus the finish kernel when a
    block has a heavy kind or a composition mixes precisions."""
    cu = gu.ensure(100, 256)
    cu.curob_set_precision(cu.PRECISION_AUTO)
    cu.curob_set_small_batch(0)  # the batched kernels at every N
    assert cu.curob_query_launches(0, 256) == 2    # Sphere, TF32X3
    assert cu.curob_query_launches(3, 256) == 2    # Discus, EXACT, light
    assert cu.curob_query_launches(8, 256) == 3    # Weierstrass: heavy
    assert cu.curob_query_launches(16, 256) == 3   # rotated Modified Schwefel
    assert cu.curob_query_launches(29, 256) == 4   # CF1: MIXED, no heavy member
    assert cu.curob_query_launches(32, 256) == 4   # CF4: MIXED with heavy members
    assert cu.curob_query_launches(8, 0) == 0
    cu.curob_set_precision(3)  # SIMT: one kernel whatever the kinds
    try:
        assert cu.curob_query_launches(32, 256) == 1
    finally:
        cu.curob_set_precision(cu.PRECISION_AUTO)
    with pytest.raises(cu.CurobError):
        cu.curob_query_launches(8, -1)
    cu.curob_set_small_batch(512)
    assert cu.curob_query_launches(32, 256) == 1   # small population: one kernel


def test_heavy_scratch_slices(orc):
    """A call whose heavy-kind scratch exceeds one slice (CF4 at D = 1000:
    3000 heavy columns per candidate) runs in two candidate slices; rows on
    both sides of the slice boundary match the oracle."""
    import torch
    D = 1000
    per_row = 4 * 3000 + 2 * 8 * 5
    rows_per_slice = (256 * 2**20 // per_row) // 128 * 128
    N = rows_per_slice + 300
    cu = gu.ensure(D, N)
    cu.curob_set_precision(cu.PRECISION_AUTO)
    assert cu.curob_query_launches(32, N) == 8
    assert cu.curob_query_launches(32, rows_per_slice) == 4
    o = orc.generate(32, D, 0)[0].o
    x32 = inputs.mixed(N, D, 4242, center=o, frac_near=0.1, sigma=1e-3).astype(np.float32)
    got = gu.gpu_eval(32, x32, torch.float32)
    rows = np.unique(np.r_[0, 127, rows_per_slice - 1, rows_per_slice, rows_per_slice + 1, N - 1,
                           np.random.default_rng(5).integers(0, N, 26)])
    ok, worst, excused, raw = gu.fp32_check(orc, 32, D, 0, x32, got, rows)
    assert ok, (worst, raw)
