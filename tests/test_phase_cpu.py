"""The FP32 Weierstrass term carries the phase frac(3^k (z + 1/2)) in integer
arithmetic (Sec. 4.2: the b^k = 3^k frequencies).  Where z 2^32 is an integer
(2^-9 <= |z| <= 2^30) it takes 32 bits, elsewhere 40; this checks, on the
CPU and with Python's exact integers, that the two forms give the same
23-bit rounded phase for every k <= 20 on values where both apply, and that
both equal the exactly rounded fraction of 3^k (z + 1/2)."""
from fractions import Fraction

import numpy as np

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1


def _phases40(z):
    """The 40-bit form: P = round(z 2^40) + 2^39 in a 64-bit word, times 3
    per term; bits 17..39, rounded at bit 16."""
    P = (int(Fraction(float(z)) * 2 ** 40) + (1 << 39)) & M64
    out = []
    for _ in range(21):
        out.append(((((P >> 16) & M32) + 1) & M32) >> 1 & 0x7FFFFF)
        P = (P * 3) & M64
    return out


def _phases32(z):
    """The 32-bit form: P = z 2^32 + 2^31 modulo 2^32, times 3 per term; the
    top 23 bits rounded at bit 8 (a carry out of 32 bits wraps to 0)."""
    P = (int(Fraction(float(z)) * 2 ** 32) + (1 << 31)) & M32
    out = []
    for _ in range(21):
        out.append(((P + 256) & M32) >> 9)
        P = (P * 3) & M32
    return out


def _exact(z):
    """round(frac(3^k (z + 1/2)) 2^23) mod 2^23, ties up, from exact rationals."""
    w = Fraction(float(z)) + Fraction(1, 2)
    out = []
    for k in range(21):
        f = (3 ** k * w) % 1
        out.append(int(f * 2 ** 23 + Fraction(1, 2)) % (1 << 23))
    return out


def test_weierstrass_phase_forms_agree():
    rng = np.random.default_rng(11)
    zs = []
    for e in range(-9, 23):  # |z| in [2^-9, 2^23): both forms exact
        m = rng.uniform(1.0, 2.0, 60) * 2.0 ** e
        zs.extend(np.float32(m))
        zs.extend(np.float32(-m))
    zs.extend(np.float32([2.0 ** -9, -(2.0 ** -9), 0.5, -0.5, 1.0, 2.0 ** 22, 0.37, -41.25]))
    for z in zs:
        assert abs(float(z)) >= 2.0 ** -9
        p32 = _phases32(z)
        assert p32 == _phases40(z), z
        assert p32 == _exact(z), z


def test_weierstrass_phase_32_bit_form_needs_its_bound():
    """Below 2^-9 the 32-bit form drops bits of z (the library takes the
    40-bit form there): a value with bits below 2^-32 shows the difference."""
    z = np.float32(2.0 ** -12 * 1.2345678)
    assert _phases40(z) == _exact(z)
    assert _phases32(z) != _exact(z)
