"""Pins for the oracle's instance generator (General Setup section).

Each check compares the oracle against something other than itself: numpy's
Philox4x64-10 bit generator, numpy's QR factorisation, or a closed form.
"""
import numpy as np
import pytest

M64 = (1 << 64) - 1


def numpy_philox_block(ctr, key):
    """philox4x64_10(ctr, key) from numpy's bit generator, which increments
    its counter before producing each 4-word block."""
    c = [int(v) for v in ctr]
    # numpy adds one (with carry) before generating: start one below.
    val = (c[0] | (c[1] << 64) | (c[2] << 128) | (c[3] << 192)) - 1
    val &= (1 << 256) - 1
    start = np.array([(val >> (64 * i)) & M64 for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=start)
    return bg.random_raw(4)


@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([M64, M64, M64, M64], [M64, M64]),
    ([1, 2, 3, 4], [5, 6]),
    ([0x243F6A8885A308D3, 0x13198A2E03707344, 0xA4093822299F31D0,
      0x082EFA98EC4E6C89], [0x452821E638D01377, 0xBE5466CF34E90C6C]),
    ([12345, 0 | (2 << 8), 29, 4], [2024, 0]),
])
def test_philox_matches_numpy(orc, ctr, key):
    got = orc.philox4x64_10(ctr, key)
    exp = numpy_philox_block(ctr, key)
    assert np.array_equal(got, exp)


def test_philox_known_answer_zero(orc):
    # published known-answer vector for philox4x64-10 with zero counter/key
    got = orc.philox4x64_10([0, 0, 0, 0], [0, 0])
    assert [int(v) for v in got] == [0x16554D9ECA36314C, 0xDB20FE9D672D0FDC,
                                     0xD7E772CEE186176B, 0x7E68B68AEC7BA23B]


def _word(seed, purpose, block, fid, comp, index):
    blk = numpy_philox_block([index // 4, purpose | (block << 8), fid, comp], [seed, 0])
    return int(blk[index % 4])


@pytest.mark.parametrize("fid,D,seed,comp", [(0, 10, 0, 0), (16, 37, 7, 0),
                                            (29, 12, 3, 1), (23, 20, 11, 0)])
def test_shift_and_permutation_from_numpy_words(orc, fid, D, seed, comp):
    """o_k = 140 u_k - 70 and the Fisher-Yates split, rebuilt from numpy's
    Philox words; bit-exact."""
    comps = orc.generate(fid, D, seed)
    c = comps[comp]
    u = np.array([(_word(seed, 0, 0, fid, comp, k) >> 11) * 2.0 ** -53 for k in range(D)])
    o = (140.0 * u) - 70.0
    assert np.array_equal(c.o, o)
    assert np.all(np.abs(c.o) <= 70.0)
    perm = list(range(D))
    for i in range(D - 1, 0, -1):
        w = _word(seed, 1, 0, fid, comp, i)
        j = (w * (i + 1)) >> 64
        perm[i], perm[j] = perm[j], perm[i]
    off = 0
    exp = []
    for n in c.blocks:
        exp += sorted(perm[off:off + n])
        off += n
    assert list(c.S) == exp


def test_third_composition_member_at_origin(orc):
    for fid in range(29, 37):
        comps = orc.generate(fid, 12, 5)
        assert np.all(comps[2].o == 0.0)
        assert not np.all(comps[0].o == 0.0)


def test_shift_is_uniform_in_box(orc):
    from scipy import stats
    o = orc.generate(0, 5000, 1)[0].o
    assert o.min() >= -70 and o.max() <= 70
    assert stats.kstest((o + 70) / 140, "uniform").pvalue > 1e-4


def _gaussians(seed, fid, comp, b, n):
    g = np.zeros(n * n)
    for t in range(n * n):
        w1 = _word(seed, 2, b, fid, comp, 2 * t)
        w2 = _word(seed, 2, b, fid, comp, 2 * t + 1)
        u1 = ((w1 >> 11) + 1) * 2.0 ** -53
        u2 = (w2 >> 11) * 2.0 ** -53
        g[t] = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return g.reshape(n, n)


@pytest.mark.parametrize("fid,D,seed", [(0, 30, 0), (8, 50, 3), (25, 40, 1)])
def test_gram_schmidt_equals_qr(orc, fid, D, seed):
    """Row-wise Gram-Schmidt of G equals Q^T of the QR factorisation of G^T
    with the signs fixed so that diag(R) > 0."""
    c = orc.generate(fid, D, seed)[0]
    for b, n in enumerate(c.blocks):
        if n == 0:
            continue
        G = _gaussians(seed, fid, 0, b, n)
        Q, Rq = np.linalg.qr(G.T)
        Q = Q * np.sign(np.diag(Rq))[None, :]
        assert np.abs(c.R[b] - Q.T).max() < 1e-12


def test_gaussian_entries_are_standard_normal():
    from scipy import stats
    g = _gaussians(9, 0, 0, 0, 40).reshape(-1)
    assert stats.kstest(g, "norm").pvalue > 1e-4


@pytest.mark.parametrize("fid,D", [(0, 10), (11, 100), (2, 1000), (27, 1000), (36, 64)])
def test_rotation_is_orthogonal(orc, fid, D):
    for c in orc.generate(fid, D, 0):
        assert sorted(c.S.tolist()) == list(range(D))
        for R in c.R:
            n = R.shape[0]
            if n:
                assert np.abs(R.T @ R - np.eye(n)).max() <= 1e-13
                assert np.abs(R @ R.T - np.eye(n)).max() <= 1e-13


def test_basic_block_sizes(orc):
    assert orc.layout(0, 10) == ([3, 3, 4], True)
    assert orc.layout(0, 1000) == ([333, 333, 334], True)
    assert orc.layout(0, 2) == ([0, 0, 2], True)
    assert orc.layout(10, 50) == ([50], False)
    assert orc.layout(15, 50) == ([50], False)


def _golden_hybrid_sizes():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "hybrid_sizes.txt")
    rows = []
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            f, d, sizes = line.split(None, 2)
            rows.append((int(f), int(d), [int(s) for s in sizes.split(",")]))
    return rows


@pytest.mark.parametrize("fid,D,sizes", _golden_hybrid_sizes())
def test_hybrid_block_sizes_golden(orc, fid, D, sizes):
    assert orc.layout(fid, D)[0] == sizes


def test_hybrid_block_sizes_nonnegative(orc):
    for fid in range(23, 29):
        for D in range(10, 2001):
            sizes, _ = orc.layout(fid, D)
            assert sum(sizes) == D and min(sizes) >= 0


def test_invalid_dimensions_rejected(orc):
    with pytest.raises(ValueError):
        orc.layout(0, 1)
    with pytest.raises(ValueError):
        orc.layout(23, 9)
    with pytest.raises(ValueError):
        orc.layout(35, 9)
    with pytest.raises(ValueError):
        orc.layout(37, 10)
