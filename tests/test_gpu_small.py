"""Small populations (the paper's timing setting, Sec. 2: 50 candidates per
call at D = 10, 32, 64, 96): the small-population kernels (one warp per
candidate and component) against the FP64 oracle through the C ABI, FP64 to
1e-12 and the FP32 path to the FP32 tolerance, and against the batched
kernels they stand in for (the FP64 path bit for bit: the same arithmetic in
the same order)."""
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


def _fids(D):
    return [f for f in ALL if D >= 10 or not (23 <= f <= 28 or f >= 35)]


@pytest.mark.parametrize("D", [10, 32, 64, 96])
def test_paper_protocol_calls_match_oracle(orc, D):
    """The calls `bench.py --paper-protocol` times (N = 50, AUTO), every
    function, FP64 and FP32, with 10 % of the rows near x_opt."""
    import torch
    N = 50
    cu = gu.ensure(D, N)
    bad = {}
    for fid in _fids(D):
        assert cu.curob_query_small(fid, N)
        o = orc.generate(fid, D, 0)[0].o
        x = inputs.mixed(N, D, 60 + fid, center=o, frac_near=0.1, sigma=1e-3)
        ref = orc.evaluate(fid, D, 0, x, nthreads=8)
        got = gu.gpu_eval(fid, x, torch.float64)
        e64 = gu.rel_err(got, ref).max()
        x32 = x.astype(np.float32)
        got32 = gu.gpu_eval(fid, x32, torch.float32)
        ok, worst, excused, raw = gu.fp32_check(orc, fid, D, 0, x32, got32)
        if not (e64 <= 1e-12 and ok):
            bad[fid] = (float(e64), raw)
    assert not bad, bad


@pytest.mark.parametrize("D,N", [(2, 7), (11, 1), (32, 200), (96, 512), (120, 33)])
def test_small_equals_batched_kernels(orc, D, N):
    """The same calls with the small kernels turned off: the FP64 values are
    identical bit for bit to the batched FP64-pipe kernel (same fma order and
    index-order sums) and within the FP64 bar of the tensor-core FP64 path,
    the FP32 ones within the FP32 tolerance of each other and of the
    oracle."""
    import torch
    cu = gu.ensure(D, N)
    try:
        for fid in _fids(D):
            x = inputs.uniform(N, D, 3 * fid + N)
            xt = torch.from_numpy(x).cuda()
            x32 = xt.float()
            cu.curob_set_small_batch(N)
            assert cu.curob_query_small(fid, N)
            a64 = cu.evaluate(fid, xt)
            a32 = cu.evaluate(fid, x32)
            cu.curob_set_small_batch(0)
            assert not cu.curob_query_small(fid, N)
            cu.curob_set_precision64(cu.PRECISION64_SIMT)
            b64 = cu.evaluate(fid, xt)
            cu.curob_set_precision64(cu.PRECISION64_AUTO)
            t64 = cu.evaluate(fid, xt)  # tensor-core FP64 path
            b32 = cu.evaluate(fid, x32)
            torch.cuda.synchronize()
            assert torch.equal(a64, b64), (fid, (a64 - b64).abs().max().item())
            assert ((t64 - a64).abs() <= 1e-12 * a64.abs()).all(), fid
            got = a32.cpu().numpy().astype(np.float64)
            ok, worst, excused, raw = gu.fp32_check(orc, fid, D, 0, x32.cpu().numpy(), got)
            assert ok, (fid, raw)
            fs = gu.f_scale(orc, fid, D, 0)
            ok2, _ = gu.fp32_ok(got, b32.cpu().numpy().astype(np.float64), fs)
            assert ok2.all() or fid in (7, 15, 16), fid
    finally:
        cu.curob_set_small_batch(512)
        cu.curob_set_precision64(cu.PRECISION64_AUTO)


def test_small_limit_and_queries():
    cu = gu.ensure(96, 2048)
    assert cu.curob_query_small(0, 50) and cu.curob_query_small(0, 512)
    assert not cu.curob_query_small(0, 513) and not cu.curob_query_small(0, 0)
    assert cu.curob_query_launches(32, 50) == 1
    cu.curob_set_small_batch(2048)
    assert cu.curob_query_small(0, 2048)
    cu.curob_set_small_batch(0)
    assert not cu.curob_query_small(0, 1)
    assert cu.curob_set_small_batch(-1, check=False) == cu.CODES["CUROB_ERR_INVALID_ARGUMENT"]
    cu.curob_set_small_batch(512)
    gu.invalidate()
    cu = gu.ensure(400, 64)  # blocks of 133 > 128: the batched kernels take every call
    assert not cu.curob_query_small(0, 50)
    gu.invalidate()
