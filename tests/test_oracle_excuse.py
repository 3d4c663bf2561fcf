"""The discontinuity excuse of the FP32 checks (oracle.parity): a row is
excused only where a Step or Modified Schwefel variable sits at a jump, and
explain_excused shows that a value which differs from the oracle lies on the
other side of that jump (the FP32 rounding of z crossed it).  CPU only."""
import numpy as np

import oracle
from oracle import parity
from paper_1407_7737_gb300 import inputs


def _move_z0(comps, x, target):
    """x with z_0 of component 0's first block set to `target`, every other z
    unchanged (rows of R are orthonormal: y += (t - z_0) R[0, :])."""
    c = comps[0]
    z = oracle.component_z(7, x.size, comps, 0, x)
    y_shift = (target - z[0]) * c.R[0][0, :]
    x2 = x.copy()
    n0 = c.blocks[0]
    x2[c.S[:n0]] += y_shift  # scale 1 for Step
    return x2


def test_excused_row_lies_across_the_jump():
    D = 10
    comps = oracle.generate(7, D, 0)
    x = inputs.uniform(4, D, 3)
    x[1] = _move_z0(comps, x[1], 0.5 - 1e-7)  # floor(z + 1/2) jumps at z = 1/2
    x32 = x.astype(np.float32)
    ref = oracle.evaluate(7, D, 0, x32.astype(np.float64))
    got = ref.copy()
    # the value an evaluation lands on when its z_0 crossed 1/2: one more unit of floor^2
    zs = [oracle.component_z(7, D, comps, 0, x32[1].astype(np.float64))]
    z0 = zs[0][0]
    assert abs(z0 + 0.5 - 1.0) < 2e-5  # still next to the jump after FP32 rounding of x
    zo = [zs[0].copy()]
    zo[0][0] = parity._mirror("step", z0)
    got[1] = oracle.evaluate_from_z(7, D, zo)
    assert abs(got[1] - ref[1]) > 0.5  # a jump, far beyond the FP32 tolerance
    ok, worst, excused, raw = parity.fp32_check(7, D, 0, x32, got)
    assert ok and excused == 1 and raw > 1
    rep = parity.explain_excused(7, D, 0, x32, got)
    assert len(rep) == 1 and rep[0]["row"] == 1
    assert rep[0]["gpu_on_other_side"]
    assert [(c["member"], c["z_index"]) for c in rep[0]["crossed"]] == [(0, 0)]
    # a value that is simply wrong is not on the other side
    got[1] = ref[1] + 7.0
    rep = parity.explain_excused(7, D, 0, x32, got)
    assert len(rep) == 1 and not rep[0]["gpu_on_other_side"]


def test_mirror_reflects_across_the_jump():
    assert abs(parity._mirror("step", 1.4999999) - 1.5000001) < 1e-12
    c = 420.9687462275036
    z = 1000.0 - c + 1e-9
    zm = parity._mirror("schwefel", z)
    assert abs((zm + c) - (1000.0 - 1e-9)) < 1e-9
    z = -1500.0 - c - 2e-9
    zm = parity._mirror("schwefel", z)
    assert abs((zm + c) + (1500.0 - 2e-9)) < 1e-9


def test_two_crossed_jumps():
    """Two Step variables at their jumps, the GPU value on the other side of
    both: the explanation names both."""
    D = 10
    comps = oracle.generate(7, D, 0)
    c = comps[0]
    x = inputs.uniform(2, D, 5)
    z = oracle.component_z(7, D, comps, 0, x[0])
    n0 = c.blocks[0]
    y = (0.5 - 2e-7 - z[0]) * c.R[0][0, :] + (-1.5 + 3e-7 - z[1]) * c.R[0][1, :]
    x[0, c.S[:n0]] += y
    x32 = x.astype(np.float32)
    ref = oracle.evaluate(7, D, 0, x32.astype(np.float64))
    zs = oracle.component_z(7, D, comps, 0, x32[0].astype(np.float64))
    zo = zs.copy()
    zo[0] = parity._mirror("step", zs[0])
    zo[1] = parity._mirror("step", zs[1])
    got = ref.copy()
    got[0] = oracle.evaluate_from_z(7, D, [zo])
    rep = parity.explain_excused(7, D, 0, x32, got)
    assert len(rep) == 1 and rep[0]["gpu_on_other_side"]
    assert sorted(v["z_index"] for v in rep[0]["crossed"]) == [0, 1]
