"""The tensor-core FP64 path of curob_evaluate (error-free split product of
BF16 integer digits) against the FP64 oracle: every function at several D,
ragged and multi-slice populations, the library's own instance at D = 1000
with f from correctly rounded z beside the oracle, extreme scales, NaN, and
the path and launch queries.  Tolerance: |df| <= 1e-12 |f| (the FP64 bar)."""
import numpy as np
import pytest

from paper_1407_7737_gb300 import inputs
import gpu_util as gu

pytestmark = pytest.mark.gpu

ALL = list(range(37))
TOL = 1e-12


def _torch():
    import torch
    return torch


def _fids(D):
    return [f for f in ALL if D >= 10 or not (23 <= f <= 28 or f >= 35)]


def _tensor(cu):
    cu.curob_set_precision64(cu.PRECISION64_TENSOR)
    cu.curob_set_small_batch(0)


def _restore(cu):
    cu.curob_set_precision64(cu.PRECISION64_AUTO)
    cu.curob_set_small_batch(512)


@pytest.mark.parametrize("D,N", [(2, 200), (10, 1000), (30, 2000), (50, 4096), (100, 4096)])
def test_f64tc_parity_generated_instance(orc, D, N):
    cu = gu.ensure(D, N)
    _tensor(cu)
    try:
        bad = {}
        for fid in _fids(D):
            assert cu.curob_query_precision64(fid) == cu.PRECISION64_TENSOR
            o = orc.generate(fid, D, 0)[0].o
            x = inputs.mixed(N, D, 700 + fid, center=o, frac_near=0.1, sigma=1e-3)
            ref = orc.evaluate(fid, D, 0, x, nthreads=16)
            got = gu.gpu_eval(fid, x, _torch().float64)
            err = gu.rel_err(got, ref).max()
            if not err <= TOL:
                bad[fid] = float(err)
        assert not bad, bad
    finally:
        _restore(cu)


@pytest.mark.parametrize("D", [50, 100])
def test_f64tc_against_simt_path(orc, D):
    """The two FP64 paths agree to the FP64 bar on the same instance."""
    N = 2048
    cu = gu.ensure(D, N)
    try:
        for fid in ALL:
            x = inputs.uniform(N, D, 900 + fid)
            _tensor(cu)
            a = gu.gpu_eval(fid, x, _torch().float64)
            cu.curob_set_precision64(cu.PRECISION64_SIMT)
            b = gu.gpu_eval(fid, x, _torch().float64)
            assert gu.rel_err(a, b).max() <= TOL, fid
    finally:
        _restore(cu)


def test_f64tc_full_size_own_instance(orc):
    """D = 1000, N = 16384, the library's own instance: sampled rows against
    the oracle on that instance's data and a few rows against f from
    correctly rounded z (no rounding order shared with either side)."""
    from oracle import exact
    D, N = 1000, 16384
    cu = gu.ensure(D, N)
    rows = np.unique(np.r_[0, 1, 127, 128, N - 1, np.random.default_rng(5).integers(0, N, 59)])
    _tensor(cu)
    try:
        report, bad = {}, {}
        for fid in ALL:
            comps = _library_instance(cu, orc, fid, D)
            o = comps[0].o
            x = inputs.mixed(N, D, 800 + fid, center=o, frac_near=0.1, sigma=1e-3)
            got = gu.gpu_eval(fid, x, _torch().float64)
            ref = orc.evaluate_given(fid, D, comps, x[rows], nthreads=16)
            err = gu.rel_err(got[rows], ref)
            xr = np.r_[rows[:2], [int(np.argmin(np.abs(x - o[None, :]).max(axis=1)))]]
            ex = exact.evaluate(fid, D, comps, x[xr])
            err_x = gu.rel_err(got[xr], ex)
            report[fid] = (float(err.max()), float(err_x.max()))
            if not (err.max() <= TOL and err_x.max() <= TOL):
                bad[fid] = report[fid]
        assert not bad, bad
    finally:
        _restore(cu)


def _library_instance(cu, orc, fid, D):
    """The library's instance of fid as oracle Components (o, S, R read back)."""
    comps = []
    for c in range(cu.curob_num_components(fid)):
        sizes, rot = cu.curob_component_layout(fid, c)
        o, S, R = cu.curob_get_component(fid, c)
        comps.append(orc.Component(o=np.asarray(o), S=np.asarray(S, dtype=np.int32),
                                   blocks=list(sizes) if rot else [D], R=list(R) if rot else [],
                                   rotated=bool(rot)))
    return comps


def test_f64tc_oracle_instance_full_size(orc):
    """The oracle's own instance loaded through curob_set_component (digit
    images rebuilt), D = 1000, N = 16384, sampled rows."""
    D, N = 1000, 16384
    cu = gu.ensure(D, N)
    rows = np.unique(np.r_[0, N - 1, np.random.default_rng(1).integers(0, N, 62)])
    _tensor(cu)
    try:
        bad = {}
        for fid in ALL:
            comps = gu.load_oracle_instance(orc, fid, D, 7)
            x = inputs.mixed(N, D, 300 + fid, center=comps[0].o, frac_near=0.1, sigma=1e-3)
            got = gu.gpu_eval(fid, x, _torch().float64)
            ref = orc.evaluate_given(fid, D, comps, x[rows], nthreads=16)
            err = gu.rel_err(got[rows], ref).max()
            if not err <= TOL:
                bad[fid] = float(err)
        assert not bad, bad
    finally:
        _restore(cu)
        gu.invalidate()


@pytest.mark.parametrize("N", [129, 513, 1000, 4097])
def test_f64tc_ragged_tails(orc, N):
    """Populations that end inside a tile of 128: every row."""
    D = 50
    cu = gu.ensure(D, 4097)
    _tensor(cu)
    try:
        for fid in (0, 8, 13, 23, 29, 32, 36):
            x = inputs.uniform(N, D, N + fid)
            ref = orc.evaluate(fid, D, 0, x, nthreads=16)
            got = gu.gpu_eval(fid, x, _torch().float64)
            assert gu.rel_err(got, ref).max() <= TOL, (fid, N)
    finally:
        _restore(cu)


def test_f64tc_slices_and_launches(orc):
    """A population whose scratch exceeds one slice: rows on both sides of
    the slice boundaries, and the launch count the query reports."""
    D, N = 1000, 40000
    cu = gu.ensure(D, N)
    _tensor(cu)
    try:
        assert cu.curob_query_launches64(0, 16384) == 3
        assert cu.curob_query_launches64(10, 16384) == 2  # unrotated: no tensor-core launch
        fid = 32  # five rotated members
        L = cu.curob_query_launches64(fid, N)
        assert L % 3 == 0 and L >= 6, L
        x = inputs.uniform(N, D, 4242)
        got = gu.gpu_eval(fid, x, _torch().float64)
        slice_n = N // (L // 3)
        edges = [k * 128 for k in range(1, N // 128)]
        rows = np.unique(np.r_[0, N - 1, [e for e in edges if abs(e - slice_n) < 300][:6],
                               np.random.default_rng(3).integers(0, N, 24)])
        rows = rows[rows < N]
        ref = orc.evaluate(fid, D, 0, x[rows], nthreads=16)
        assert gu.rel_err(got[rows], ref).max() <= TOL
    finally:
        _restore(cu)


PHASE_KINDS = (8, 15)  # Weierstrass (3^k z phases), Katsuura (2^j z phases)


def test_f64tc_scales_and_optimum(orc):
    """Candidates ten times outside the box (|x| <= 1e3), at 1e-9 from o, and
    at o itself (y = 0: every digit zero).  Outside the box, functions with a
    Weierstrass or Katsuura member are left out of the comparison: the 3^20 z
    (2^32 z) phases turn one ulp of z into a different f there, so no two
    evaluations that do not share z's rounding agree (the FP64 CUDA-core
    path agrees with the oracle only because it repeats its fma order); far
    larger |x| does the same to every cosine term (2 pi |z| ulps of phase)."""
    D, N = 100, 512
    cu = gu.ensure(D, N)
    _tensor(cu)
    try:
        for fid in ALL:
            kinds = {k for c in range(cu.curob_num_components(fid))
                     for k in cu.curob_component_kinds(fid, c)}
            lo = 128 if kinds & set(PHASE_KINDS) else 0
            comps = orc.generate(fid, D, 0)
            o = comps[0].o
            rng = np.random.default_rng(fid)
            x = np.empty((N, D))
            x[:128] = rng.uniform(-1e3, 1e3, (128, D))
            x[128:256] = o[None, :] + rng.normal(0, 1e-9, (128, D))
            x[256:384] = inputs.uniform(128, D, 60 + fid)
            x[384:] = o[None, :]
            ref = orc.evaluate(fid, D, 0, x, nthreads=16)
            got = gu.gpu_eval(fid, x, _torch().float64)
            err = (np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300))[lo:]
            assert err.max() <= TOL, (fid, float(err.max()), int(np.argmax(err)) + lo)
    finally:
        _restore(cu)


def test_f64tc_nan_propagates():
    torch = _torch()
    cu = gu.ensure(50, 256)
    _tensor(cu)
    try:
        x = torch.zeros(256, 50, dtype=torch.float64, device="cuda")
        x[1, 3] = float("nan")
        x[2, 7] = float("inf")
        for fid in (0, 10, 11, 29):
            out = cu.evaluate(fid, x)
            torch.cuda.synchronize()
            assert torch.isnan(out[1]).item() and not torch.isnan(out[0]).item(), fid
            assert not torch.isfinite(out[2]).item(), fid
    finally:
        _restore(cu)


def test_f64tc_precision_setting():
    cu = gu.ensure(10, 8)
    C = cu.CODES
    assert cu.curob_set_precision64(3, check=False) == C["CUROB_ERR_INVALID_ARGUMENT"]
    assert cu.curob_set_precision64(-1, check=False) == C["CUROB_ERR_INVALID_ARGUMENT"]
    assert cu.curob_query_precision64(0) == cu.PRECISION64_TENSOR  # AUTO on a GB300
    cu.curob_set_precision64(cu.PRECISION64_SIMT)
    assert cu.curob_query_precision64(0) == cu.PRECISION64_SIMT
    assert cu.curob_query_launches64(0, 100) == 1
    cu.curob_set_precision64(cu.PRECISION64_AUTO)
