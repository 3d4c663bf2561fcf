"""Seeded synthetic candidate populations.

The paper times its functions on "uniform random" candidates in the search box
(Sec. 2, Speedup); the library's accuracy tests add a slice of candidates
around a known optimum.  This module only draws numbers: it holds none of the
benchmark's arithmetic, so it can feed both the GPU library and the oracle.
"""
from __future__ import annotations

import numpy as np

BOX = 100.0  # search domain [-100, 100]^D (General Setup, "Search Space")


def uniform(N: int, D: int, seed: int) -> np.ndarray:
    """N x D candidates uniform in the search box, FP64."""
    rng = np.random.default_rng([seed, 0x5EED, D, N])
    return rng.uniform(-BOX, BOX, size=(N, D))


def near(center: np.ndarray, N: int, sigma: float, seed: int) -> np.ndarray:
    """N candidates center + N(0, sigma^2) per coordinate, FP64."""
    center = np.asarray(center, dtype=np.float64).reshape(-1)
    rng = np.random.default_rng([seed, 0x0A7, center.size, N])
    return center[None, :] + sigma * rng.standard_normal((N, center.size))


def mixed(N: int, D: int, seed: int, center=None, frac_near: float = 0.1,
          sigma: float = 1e-3) -> np.ndarray:
    """Uniform candidates with the first ``frac_near`` of rows replaced by a
    Gaussian cloud of width ``sigma`` around ``center`` (when given)."""
    x = uniform(N, D, seed)
    if center is not None and frac_near > 0:
        m = int(round(frac_near * N))
        if m:
            x[:m] = near(center, m, sigma, seed + 1)
    return x


def ragged_instances(n_inst: int, seed: int, dims=(10, 30, 50, 100, 500, 1000),
                     nmin: int = 32, nmax: int = 8192, n_fid: int = 37):
    """(fid, D, N) triples for a mixed batch: fid uniform over the suite,
    D uniform over ``dims``, N log-uniform in [nmin, nmax]."""
    rng = np.random.default_rng([seed, 0xBA7C])
    fids = rng.integers(0, n_fid, size=n_inst)
    Ds = rng.choice(np.asarray(dims), size=n_inst)
    Ns = np.round(np.exp(rng.uniform(np.log(nmin), np.log(nmax), size=n_inst)))
    return [(int(f), int(d), int(n)) for f, d, n in zip(fids, Ds, Ns)]


def shuffled_mixture(N: int, D: int, seed: int, center, frac_near: float = 0.3,
                     sigma: float = 10.0) -> np.ndarray:
    """Training and screening pools of the learned pre-screen: ``frac_near``
    of the rows Gaussian around ``center`` (width ``sigma``), the rest uniform
    in the box, rows in random order."""
    x = mixed(N, D, seed, center, frac_near, sigma)
    rng = np.random.default_rng([seed, 0x5A1F, D, N])
    return x[rng.permutation(N)]
