"""Correctly rounded z and squared distances for the FP64 oracle.

TEST INFRASTRUCTURE ONLY (tests may import it; the product path never does).

The oracle and the FP64 GPU path both round while they form z = R(s(x - o)) + c
(General Setup): x - o, the scaling by s and every term of the rotation's dot
products.  To see how far those roundings move f, this module forms z from
the same double data without any intermediate rounding: x - o as an exact
TwoSum pair, s times each part as an exact TwoProduct pair (Dekker's
splitting), R_ij times each of those four parts again as exact pairs, and the
8 n terms of each dot product plus c summed by math.fsum, which returns the
correctly rounded sum of its arguments (Shewchuk's exact partial sums).  So z
here is exactly the real z of the given doubles, rounded once.  The same is
done for d^2 = ||x - o||^2 (Eq. weight).  f then comes from
``oracle.evaluate_from_z``, the oracle's own assembly.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

_SPLIT = 134217729.0  # 2^27 + 1 (Dekker / Veltkamp)


def two_sum(a, b):
    """s + e = a + b exactly (Knuth's TwoSum)."""
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def _split(a):
    c = _SPLIT * a
    hi = c - (c - a)
    return hi, a - hi


def two_prod(a, b):
    """p + e = a * b exactly (Dekker's TwoProduct; no overflow here)."""
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def _y_parts(x, o, s):
    """Four vectors whose exact sum is s (x - o)."""
    a, b = two_sum(np.asarray(x, dtype=np.float64), -np.asarray(o, dtype=np.float64))
    p1, e1 = two_prod(s, a)
    p2, e2 = two_prod(s, b)
    return [p1, e1, p2, e2]


def component_z(fid: int, D: int, comps, c: int, x) -> np.ndarray:
    """z of component c for candidate x, each entry the correctly rounded
    value of R_b (s_b (x - o)[S_b]) + c_b over the given doubles."""
    comp = comps[c]
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    scale, offset = oracle.block_affine(fid, D, c)
    z = np.zeros(D)
    if not comp.rotated:
        parts = _y_parts(x, comp.o, scale[0])
        for j in range(D):
            z[j] = math.fsum([p[j] for p in parts] + [offset[0]])
        return z
    off = 0
    for b, (n, R) in enumerate(zip(comp.blocks, comp.R)):
        idx = comp.S[off:off + n]
        parts = _y_parts(x[idx], comp.o[idx], scale[b])
        terms = []
        for p in parts:
            P, E = two_prod(R, p[None, :])
            terms += [P, E]
        M = np.concatenate(terms, axis=1)
        for i in range(n):
            z[off + i] = math.fsum(M[i].tolist() + [offset[b]])
        off += n
    return z


def sq_distance(x, o) -> float:
    """||x - o||^2 correctly rounded."""
    a, b = two_sum(np.asarray(x, dtype=np.float64), -np.asarray(o, dtype=np.float64))
    p1, e1 = two_prod(a, a)
    p2, e2 = two_prod(2.0 * a, b)
    p3, e3 = two_prod(b, b)
    return math.fsum(np.concatenate([p1, e1, p2, e2, p3, e3]).tolist())


def evaluate(fid: int, D: int, comps, x) -> np.ndarray:
    """f (f_opt included) of each row of x from correctly rounded z (and d^2),
    assembled by the oracle."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, D)
    out = np.zeros(x.shape[0])
    for r in range(x.shape[0]):
        zs = [component_z(fid, D, comps, c, x[r]) for c in range(len(comps))]
        d2 = [sq_distance(x[r], comp.o) for comp in comps]
        out[r] = oracle.evaluate_from_z(fid, D, zs, d2)
    return out
