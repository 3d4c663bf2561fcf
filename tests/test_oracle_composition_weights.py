"""Pins for the oracle's composition weights (Sec. 6, Eq. composition and
Eq. weight), on the branch every candidate inside the box takes:

  w_i = (1 / sqrt(d_i^2)) exp(-d_i^2 / (2 D sigma_i^2)),  omega_i = w_i / sum w,
  F = sum_i omega_i (lambda_i G_i + bias_i) + f_opt.

The cases use unequal sigma_i and unequal distances, chosen so that every
exponent is a small integer: d_i^2 = k_i (2 D sigma_i^2).  The expected
weights are then closed forms in e and square roots, written out below by
hand, and each plausible slip in the formula (dropping D, sigma in place of
sigma^2, dropping the 1/d factor, d in place of d^2) moves F by far more than
the tolerance: the test asserts that too, so it is known to discriminate.
"""
import math

import numpy as np

FOPT = 100.0

# Composition Function 3 (Table 1 ID 31): sigma = (20, 50, 40),
# lambda = (0.25, 1, 1e-7), bias = (0, 100, 200) (Sec. 6).
SIG = (20.0, 50.0, 40.0)
LAM = (0.25, 1.0, 1e-7)
BIAS = (0.0, 100.0, 200.0)


def _F(w, G):
    W = sum(w)
    return sum(wi / W * (l * g + b) for wi, l, g, b in zip(w, LAM, G, BIAS)) + FOPT


def test_weights_hand_worked_closed_form(orc):
    """D = 2, so 2 D sigma_i^2 = (1600, 10000, 6400).  With d^2 = (1600,
    10000, 12800) the exponents are (-1, -1, -2) and d = (40, 100, 80 sqrt 2):
    w ~ (e^-1 / 40, e^-1 / 100, e^-2 / (80 sqrt 2)); scaling by e,
    omega ~ (1/40, 1/100, 1/(80 sqrt(2) e))."""
    D = 2
    d2 = [1600.0, 10000.0, 12800.0]
    G = [4.0, 3.0, 5.0e6]                      # lambda G = (1, 3, 0.5)
    w = [1 / 40, 1 / 100, 1 / (80 * math.sqrt(2) * math.e)]
    expect = _F(w, G)
    # the weights themselves, normalised: 0.6535..., 0.2614..., 0.0850...
    W = sum(w)
    assert abs(w[0] / W - 0.65357) < 1e-4 and abs(w[2] / W - 0.08500) < 1e-4
    got = orc.compose(31, D, G, d2)
    assert abs(got - expect) <= 1e-14 * abs(expect), (got, expect)
    # plausible slips, each far outside the tolerance
    d = [math.sqrt(v) for v in d2]
    slips = {
        "no D": [math.exp(-v / (2 * s * s)) / di for v, s, di in zip(d2, SIG, d)],
        "sigma for sigma^2": [math.exp(-v / (2 * D * s)) / di for v, s, di in zip(d2, SIG, d)],
        "no 1/d": [math.exp(-v / (2 * D * s * s)) for v, s in zip(d2, SIG)],
        "d for d^2": [math.exp(-di / (2 * D * s * s)) / di for di, s in zip(d, SIG)],
        "1/d^2": [math.exp(-v / (2 * D * s * s)) / v for v, s in zip(d2, SIG)],
    }
    for name, ws in slips.items():
        assert abs(_F(ws, G) - expect) > 1e-3 * abs(expect), name


def test_weights_depend_on_D(orc):
    """The same d^2 and G at D = 4 halve every exponent: (-1/2, -1/2, -1),
    omega ~ (e^-1/2 / 40, e^-1/2 / 100, e^-1 / (80 sqrt 2)) ~ (1/40, 1/100,
    e^-1/2 / (80 sqrt 2))."""
    D = 4
    d2 = [1600.0, 10000.0, 12800.0]
    G = [4.0, 3.0, 5.0e6]
    w = [1 / 40, 1 / 100, math.exp(-0.5) / (80 * math.sqrt(2))]
    expect = _F(w, G)
    got = orc.compose(31, D, G, d2)
    assert abs(got - expect) <= 1e-14 * abs(expect), (got, expect)
    assert abs(got - orc.compose(31, 2, G, d2)) > 1.0


def test_weights_end_to_end_geometry(orc):
    """Through the evaluation itself: D = 2, identity rotations and
    permutations, x = 0, o_1 = (40, 0), o_2 = (0, 100), o_3 = (80, 80) give
    d^2 = (1600, 10000, 12800) as above.  The members are Rotated Modified
    Schwefel (z = 10 (x - o_1) = (-400, 0)), Rotated Rastrigin (z = 0.0512
    (x - o_2) = (0, -5.12)) and Rotated Elliptic (z = x - o_3 = (-80, -80):
    6400 + 1e6 * 6400)."""
    D = 2
    comps = orc.generate(31, D, 0)
    for c, o in zip(comps, ([40.0, 0.0], [0.0, 100.0], [80.0, 80.0])):
        c.o = np.array(o)
        c.S = np.arange(D, dtype=np.int32)
        c.R = [np.eye(n) for n in c.blocks]
    # Schwefel: 418.9829 D - sum g1(z_i + 420.9687462275036); z = (-400, 0)
    c = 420.9687462275036
    g1 = lambda w: w * math.sin(math.sqrt(abs(w)))  # |w| <= 500 branch
    G1 = 418.9829 * 2 - (g1(-400 + c) + g1(c))
    # Rastrigin at (0, -5.12): 0 + (5.12^2 - 10 cos(2 pi 5.12) + 10)
    G2 = 5.12 ** 2 - 10 * math.cos(2 * math.pi * 5.12) + 10
    G3 = 6400.0 + 1.0e6 * 6400.0
    w = [1 / 40, 1 / 100, 1 / (80 * math.sqrt(2) * math.e)]
    expect = _F(w, [G1, G2, G3])
    got = orc.evaluate_given(31, D, comps, np.zeros((1, D)))[0]
    assert abs(got - expect) <= 1e-13 * abs(expect), (got, expect)


def test_one_hot_at_member_optimum(orc):
    """d_i^2 = 0: omega is one-hot at the first such member (the limit the
    paper states for w_i = 1/0)."""
    G = [4.0, 3.0, 5.0e6]
    assert orc.compose(31, 2, G, [1600.0, 0.0, 0.0]) == 1.0 * 3.0 + 100.0 + FOPT
