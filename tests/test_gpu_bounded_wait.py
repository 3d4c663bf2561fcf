"""A device-side wait that nothing completes gives up after its limit and
reports through a status word: no hang, no trap, and the context stays
usable for the next evaluation."""
import time

import numpy as np
import pytest

import gpu_util as gu
from paper_1407_7737_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_wait_runs_out_and_context_survives(orc):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cu = gu.cu()
    t0 = time.perf_counter()
    rc = cu.curob_selftest_bounded_wait()
    dt = time.perf_counter() - t0
    assert rc == cu.CODES["CUROB_ERR_DEVICE_TIMEOUT"]
    assert 1.5 < dt < 30.0
    # the same process keeps evaluating correctly
    gu.ensure(10, 64)
    x = inputs.uniform(64, 10, 5).astype(np.float32)
    got = gu.gpu_eval(0, x, torch.float32)
    ref = orc.evaluate(0, 10, 0, x.astype(np.float64))
    assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(ref))
