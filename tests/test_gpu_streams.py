"""Calls on several streams at once: the split launches' stream-ordered
scratch and the library's per-call state must not leak between calls, so
results are bit-identical to the same calls issued on one stream."""
import numpy as np
import pytest

import gpu_util as gu
from paper_1407_7737_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_concurrent_calls_match_one_stream():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    D, N = 100, 1500
    cu = gu.ensure(D, N)
    cu.curob_set_precision(cu.PRECISION_AUTO)
    # light, heavy, MIXED and MIXED-with-heavy functions, each twice
    fids = [0, 8, 16, 29, 32, 13, 34, 36] * 2
    xs = [torch.from_numpy(inputs.uniform(N, D, 900 + i).astype(np.float32)).cuda()
          for i in range(len(fids))]
    main = torch.cuda.current_stream()
    ref = [torch.empty(N, device="cuda") for _ in fids]
    for f, x, o in zip(fids, xs, ref):
        cu.curob_evaluatef(f, x, N, o, main)
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(4)]
    got = [torch.full((N,), float("nan"), device="cuda") for _ in fids]
    fork = torch.cuda.Event()
    fork.record(main)
    for s in streams:
        s.wait_event(fork)
    for k, (f, x, o) in enumerate(zip(fids, xs, got)):
        cu.curob_evaluatef(f, x, N, o, streams[k % len(streams)])
    torch.cuda.synchronize()
    cu.curob_get_device_status(main)
    for f, a, b in zip(fids, ref, got):
        assert torch.equal(a, b), f
