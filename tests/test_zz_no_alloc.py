"""curob_evaluatef_multi_noalloc: the allocation-free entry point.

Some callers must not allocate device memory once they are running (an
optimizer that reserves its whole GPU budget at start-up, a plugin whose host
framework owns every device allocation).  This entry point keeps its scratch
in a static device array; here its results are checked, through the C ABI,
against the ordinary curob_evaluatef on two calls in a row with different
work, so the second call cannot lean on what the first left in the array,
and against the FP64 oracle directly.
"""
import numpy as np
import pytest

import gpu_util as gu
from paper_1407_7737_gb300 import inputs

pytestmark = pytest.mark.gpu

D = 100


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _case(torch, fids, Ns, seed):
    xs = [torch.from_numpy(inputs.uniform(n, D, seed + i).astype(np.float32)).cuda()
          for i, n in enumerate(Ns)]
    outs = [torch.full((n,), float("nan"), device="cuda") for n in Ns]
    return xs, outs


def _reference(cu, torch, fids, xs, mode):
    cu.curob_set_precision(mode)
    try:
        refs = []
        for fid, x in zip(fids, xs):
            o = torch.empty(x.shape[0], device="cuda")
            cu.curob_evaluatef(fid, x, x.shape[0], o, None)
            refs.append(o)
        torch.cuda.synchronize()
        return refs
    finally:
        cu.curob_set_precision(cu.PRECISION_AUTO)


def test_noalloc_matches_evaluatef_twice(orc, torch_cuda):
    torch = torch_cuda
    cu = gu.ensure(D, 4096)
    calls = [
        ([0, 8, 16, 29, 36, 11], [1000, 3000, 129, 1, 700, 4096]),
        ([3, 13, 21, 33], [257, 2000, 64, 1500]),
    ]
    for k, (fids, Ns) in enumerate(calls):
        xs, outs = _case(torch, fids, Ns, 300 * (k + 1))
        cu.curob_evaluatef_multi_noalloc(fids, xs, Ns, outs)
        torch.cuda.synchronize()
        cu.curob_get_device_status(None)
        auto = _reference(cu, torch, fids, xs, cu.PRECISION_AUTO)
        exact = _reference(cu, torch, fids, xs, cu.PRECISION_EXACT)
        cu.curob_set_precision(cu.PRECISION_EXACT)
        # one tensor-core launch (after the transpose of x), no finish kernel
        fused = [cu.curob_query_launches(fid, n) <= 2 for fid, n in zip(fids, Ns)]
        cu.curob_set_precision(cu.PRECISION_AUTO)
        assert not all(fused) and any(fused)  # both kinds of item are covered
        for fid, x, o, a, e, one in zip(fids, xs, outs, auto, exact, fused):
            got = o.cpu().numpy().astype(np.float64)
            fs = gu.f_scale(orc, fid, D, 0)
            for ref_t in (a, e):
                ref = ref_t.cpu().numpy().astype(np.float64)
                ok, tol = gu.fp32_ok(got, ref, fs)
                assert ok.all(), (k, fid, float((np.abs(got - ref) / tol).max()))
            if one:  # EXACT in one launch: the same tile arithmetic, bit for bit
                assert torch.equal(o, e), (k, fid)
            # and directly against the FP64 oracle at the FP32 inputs
            ok, worst, excused, raw = gu.fp32_check(orc, fid, D, 0, x.cpu().numpy(), got)
            assert ok, (k, fid, raw)


def test_noalloc_limits(torch_cuda):
    torch = torch_cuda
    cu = gu.ensure(D, 4096)
    x = torch.zeros(4, D, device="cuda")
    o = torch.zeros(4, device="cuda")
    C = cu.CODES
    assert cu.curob_evaluatef_multi_noalloc([0] * 65, [x] * 65, [4] * 65, [o] * 65,
                                            check=False) == C["CUROB_ERR_CAPACITY"]
    assert cu.curob_evaluatef_multi_noalloc([0], [x], [4097], [o],
                                            check=False) == C["CUROB_ERR_CAPACITY"]
    assert cu.curob_evaluatef_multi_noalloc([37], [x], [4], [o],
                                            check=False) == C["CUROB_ERR_INVALID_FID"]
    host = np.zeros((4, D), dtype=np.float32)
    assert cu.curob_evaluatef_multi_noalloc([0], [host], [4], [o],
                                            check=False) == C["CUROB_ERR_INVALID_ARGUMENT"]
    assert cu.curob_evaluatef_multi_noalloc([0], [x], [0], [o], check=False) == 0
