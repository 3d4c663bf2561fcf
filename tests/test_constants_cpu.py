"""Constants the CUDA library writes as literals, pinned to their definitions
with high-precision arithmetic (CPU only)."""
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _literal(name, path):
    src = open(os.path.join(ROOT, path)).read()
    m = re.search(rf"\b{name}\s*=\s*([-+0-9.eE]+)\s*;", src)
    assert m, name
    return float(m.group(1))


def test_weierstrass_reduction_constant_eta():
    """kEta = 2 pi - 2 fl(pi): the gap between 2 pi and the double the FP64
    Weierstrass argument is built from, to double precision."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    eta = 2 * (mpmath.pi - mpmath.mpf(math.pi))
    got = _literal("kEta", "paper_1407_7737_gb300/csrc/curob_f64tc.cu")
    assert got == float(eta)
    assert abs(mpmath.mpf(got) - eta) <= 2.0 ** -53 * eta
