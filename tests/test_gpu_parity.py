"""GPU parity: libcurob against the FP64 oracle, element by element, through
the C ABI.  Sizes span several CTA tiles and a ragged tail; the full-size case
(D = 1000, N = 16384, the launch the benchmark times) is checked on sampled
rows."""
import numpy as np
import pytest

import gpu_util as gu
from paper_1407_7737_gb300 import inputs

pytestmark = pytest.mark.gpu

ALL = list(range(37))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield
    gu.invalidate()


# --------------------------------------------------------------- instance a1
@pytest.mark.parametrize("D", [10, 31, 100, 1000])
def test_instance_generation_matches_oracle(orc, D):
    """o and the permutation bit for bit; rotations orthogonal to 1e-13 and
    equal to the oracle's up to Gram-Schmidt rounding."""
    cu = gu.ensure(D, 64)
    fids = ALL if D < 1000 else [0, 8, 16, 24, 27, 29, 36]
    for fid in fids:
        ref = orc.generate(fid, D, 0)
        for c, rc in enumerate(ref):
            o, S, R = cu.curob_get_component(fid, c)
            assert np.array_equal(o, rc.o), (fid, c)
            assert np.array_equal(S, rc.S), (fid, c)
            assert len(R) == len(rc.R)
            for Rg, Ro in zip(R, rc.R):
                n = Rg.shape[0]
                assert np.abs(Rg @ Rg.T - np.eye(n)).max() <= 1e-13
                assert np.abs(Rg - Ro).max() <= 1e-11, (fid, c, np.abs(Rg - Ro).max())


# ------------------------------------------------------------------ FP64 path
@pytest.mark.parametrize("D,N", [(10, 64), (30, 4096), (50, 4096), (100, 4096)])
def test_fp64_parity_generated_instance(orc, D, N):
    cu = gu.ensure(D, N)
    worst = {}
    for fid in ALL:
        o = orc.generate(fid, D, 0)[0].o
        x = inputs.mixed(N, D, 100 + fid, center=o, frac_near=0.1, sigma=1e-3)
        ref = orc.evaluate(fid, D, 0, x, nthreads=16)
        got = gu.gpu_eval(fid, x, _torch().float64)
        err = gu.rel_err(got, ref)
        worst[fid] = err.max()
    bad = {f: e for f, e in worst.items() if not e <= 1e-12}
    assert not bad, bad


@pytest.mark.parametrize("D,N", [(10, 61), (100, 333), (1000, 16384)])
def test_fp64_parity_oracle_instance(orc, D, N):
    """The oracle's own instance loaded through curob_set_component: the FP64
    path reproduces z bit for bit, so only the transforms' libm and the
    reduction order differ."""
    cu = gu.ensure(D, N)
    rows = np.arange(N) if N <= 4096 else np.unique(np.r_[0, 1, N - 1, np.random.default_rng(0).integers(0, N, 96)])
    try:
        for fid in ALL:
            gu.load_oracle_instance(orc, fid, D, 7)
            o = orc.generate(fid, D, 7)[0].o
            x = inputs.mixed(N, D, 200 + fid, center=o, frac_near=0.1, sigma=1e-3)
            got = gu.gpu_eval(fid, x, _torch().float64)
            comps = orc.generate(fid, D, 7)
            ref = orc.evaluate_given(fid, D, comps, x[rows], nthreads=16)
            err = gu.rel_err(got[rows], ref)
            assert err.max() <= 1e-12, (fid, err.max())
    finally:
        gu.invalidate()


def test_fp64_at_optimum(orc):
    D = 50
    cu = gu.ensure(D, 16)
    for fid in ALL:
        ref_opt = orc.generate(fid, D, 0)
        for c, comp in enumerate(ref_opt):
            x = comp.o[None, :]
            got = gu.gpu_eval(fid, x, _torch().float64)[0]
            ref = orc.evaluate(fid, D, 0, x)[0]
            assert abs(got - ref) <= 1e-12 * abs(ref), (fid, c, got, ref)


# -------------------------------------------------------------- FP32 (SIMT)
@pytest.mark.parametrize("D,N", [(10, 64), (50, 4096), (100, 4096)])
def test_fp32_simt_parity(orc, D, N):
    torch = _torch()
    cu = gu.ensure(D, N)
    cu.curob_set_precision(cu.PRECISION_SIMT)
    try:
        bad = {}
        for fid in ALL:
            o = orc.generate(fid, D, 0)[0].o
            x = inputs.mixed(N, D, 300 + fid, center=o, frac_near=0.1, sigma=1e-3)
            x32 = x.astype(np.float32)
            got = gu.gpu_eval(fid, x32, torch.float32)
            ok, worst, excused, raw = gu.fp32_check(orc, fid, D, 0, x32, got)
            if not ok:
                bad[fid] = raw
        assert not bad, bad
    finally:
        cu.curob_set_precision(cu.PRECISION_AUTO)


# ------------------------------------------------------------ edges / errors
def test_edge_sizes(orc):
    torch = _torch()
    for D in (2, 3, 11):
        cu = gu.ensure(D, 70)
        fids = [f for f in ALL if D >= 10 or not (23 <= f <= 28 or f >= 35)]
        for fid in fids:
            for N in (1, 33, 70):
                x = inputs.uniform(N, D, N + fid)
                ref = orc.evaluate(fid, D, 0, x)
                got = gu.gpu_eval(fid, x, torch.float64)
                assert np.all(gu.rel_err(got, ref) <= 1e-12), (D, fid, N)


def test_errors_and_empty():
    torch = _torch()
    cu = gu.ensure(10, 8)
    x = torch.zeros(8, 10, dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    C = cu.CODES
    assert cu.curob_evaluate(0, x, 0, out, None, check=False) == 0
    assert cu.curob_evaluate(0, x, 9, out, None, check=False) == C["CUROB_ERR_CAPACITY"]
    assert cu.curob_evaluate(37, x, 1, out, None, check=False) == C["CUROB_ERR_INVALID_FID"]
    assert cu.curob_evaluate(-1, x, 1, out, None, check=False) == C["CUROB_ERR_INVALID_FID"]
    assert cu.curob_evaluate(0, x, -1, out, None, check=False) == C["CUROB_ERR_INVALID_ARGUMENT"]
    assert cu.curob_evaluate(0, None, 1, out, None, check=False) == C["CUROB_ERR_NULL_POINTER"]
    host = np.zeros((8, 10))
    assert cu.curob_evaluate(0, host, 1, out, None, check=False) == C["CUROB_ERR_INVALID_ARGUMENT"]
    assert cu.curob_initialize(10, 8, 0, check=False) == C["CUROB_ERR_ALREADY_INITIALIZED"]
    gu.invalidate()
    cu = gu.ensure(5, 8)
    assert cu.curob_evaluate(23, x, 1, out, None, check=False) == C["CUROB_ERR_INVALID_DIM"]
    assert cu.curob_evaluate(35, x, 1, out, None, check=False) == C["CUROB_ERR_INVALID_DIM"]
    gu.invalidate()
    assert cu.curob_initialize(1, 8, 0, check=False) == C["CUROB_ERR_INVALID_DIM"]
    assert cu.curob_initialize(10, 0, 0, check=False) == C["CUROB_ERR_INVALID_ARGUMENT"]


def test_nan_propagates():
    torch = _torch()
    cu = gu.ensure(10, 4)
    x = torch.zeros(4, 10, dtype=torch.float64, device="cuda")
    x[1, 3] = float("nan")
    for fid in (0, 11, 29):
        out = cu.evaluate(fid, x)
        torch.cuda.synchronize()
        assert torch.isnan(out[1]).item() and not torch.isnan(out[0]).item()


def test_host_wrappers(orc):
    cu = gu.ensure(30, 100)
    x = inputs.uniform(100, 30, 5)
    out = np.zeros(100)
    cu.curob_h_evaluate(11, x, 100, out)
    ref = orc.evaluate(11, 30, 0, x)
    assert np.all(gu.rel_err(out, ref) <= 1e-12)
    x32 = x.astype(np.float32)
    out32 = np.zeros(100, dtype=np.float32)
    cu.curob_h_evaluatef(11, x32, 100, out32)
    ref32 = orc.evaluate(11, 30, 0, x32.astype(np.float64))
    assert np.all(gu.rel_err(out32.astype(np.float64), ref32) <= 1e-5)


def _torch():
    import torch
    return torch


def test_composition_far_outside_the_box(orc):
    """Candidates so far from every member optimum that each composition
    weight underflows in FP64: the library's log-domain normalisation
    matches the oracle's (FP64 path to 1e-12, FP32 path to 1e-5)."""
    torch = _torch()
    D = 4
    comps = orc.generate(30, D, 0)
    comps[0].o = np.array([-3.0, 0, 0, 0])
    comps[1].o = np.array([3.0, 0, 0, 0])
    comps[2].o = np.array([60.0, 60, 60, 60])
    for c in comps:
        if c.rotated:
            c.S = np.arange(D, dtype=np.int32)
            c.R = [np.eye(n) for n in c.blocks]
    cu = gu.ensure(D, 8)
    try:
        for k, c in enumerate(comps):
            cu.curob_set_component(30, k, c.o, c.S, c.R)
        x = np.array([[2000.0, 0, 0, 0], [-5000.0, 100, 0, 7], [0, 0, 0, 3000.0]])
        ref = orc.evaluate_given(30, D, comps, x)
        got = gu.gpu_eval(30, x, torch.float64)
        assert np.all(np.isfinite(got))
        assert np.all(gu.rel_err(got, ref) <= 1e-12), (got, ref)
        x32 = x.astype(np.float32)
        got32 = gu.gpu_eval(30, x32, torch.float32)
        ref32 = orc.evaluate_given(30, D, comps, x32.astype(np.float64))
        assert np.all(gu.rel_err(got32, ref32) <= 1e-5), (got32, ref32)
    finally:
        gu.invalidate()
