"""2-D landscapes of the benchmark functions (the paper's App. A plots, as
data): f on a res x res grid over [lo, hi]^2 at D = 2, evaluated on the GPU
through curob_evaluate (FP64) or curob_evaluatef (FP32), written as CSV or as a
binary PGM image (log-scaled f - f_opt, 16-bit grey).  No graphics API: the
grid is one batched evaluation of res^2 candidates.

    python -m paper_1407_7737_gb300.landscape --fid 8 --res 512 --out weierstrass.pgm

Hybrid functions (IDs 23-28) and the compositions built from them (35, 36)
need D >= 10 and have no 2-D landscape.
"""
from __future__ import annotations

import argparse

import numpy as np

from . import binding as cu


def grid_points(res: int, lo: float = -100.0, hi: float = 100.0) -> np.ndarray:
    """The res^2 x 2 candidates of the grid, row-major: point (i, j) has
    x_1 = the j-th abscissa and x_2 = the i-th (i counts from lo upwards)."""
    t = np.linspace(lo, hi, res)
    X1, X2 = np.meshgrid(t, t)
    return np.stack([X1.ravel(), X2.ravel()], axis=1)


def landscape(fid: int, res: int = 256, lo: float = -100.0, hi: float = 100.0, seed: int = 0,
              fp32: bool = False) -> np.ndarray:
    """f_fid on the grid (res x res array, FOPT included) for the instance
    (D = 2, seed).  Initialises and disposes the library around the call."""
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("landscape needs a CUDA device")
    pts = grid_points(res, lo, hi)
    n = pts.shape[0]
    cu.curob_initialize(2, n, seed)
    try:
        dtype = torch.float32 if fp32 else torch.float64
        x = torch.from_numpy(pts).to(device="cuda", dtype=dtype).contiguous()
        out = cu.evaluate(fid, x)
        torch.cuda.synchronize()
        cu.curob_get_device_status(None)
        return out.double().cpu().numpy().reshape(res, res)
    finally:
        cu.curob_dispose()


def to_grey(f: np.ndarray, fopt: float = cu.FOPT) -> np.ndarray:
    """log10(1 + f - f_opt) scaled to 0..65535 (uint16); the minimum is black."""
    v = np.log10(1.0 + np.maximum(f - fopt, 0.0))
    span = float(v.max() - v.min())
    g = (v - v.min()) / span if span > 0 else np.zeros_like(v)
    return np.round(g * 65535.0).astype(np.uint16)


def write_pgm(path: str, f: np.ndarray) -> None:
    """Binary 16-bit PGM (P5, big-endian samples), top row = largest x_2."""
    g = to_grey(f)[::-1]
    h, w = g.shape
    with open(path, "wb") as fh:
        fh.write(f"P5\n{w} {h}\n65535\n".encode())
        fh.write(g.astype(">u2").tobytes())


def write_csv(path: str, f: np.ndarray, lo: float = -100.0, hi: float = 100.0) -> None:
    """One line per grid point: x_1, x_2, f."""
    res = f.shape[0]
    pts = grid_points(res, lo, hi)
    np.savetxt(path, np.column_stack([pts, f.ravel()]), delimiter=",", fmt="%.17g",
               header="x1,x2,f", comments="")


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--fid", type=int, required=True)
    ap.add_argument("--res", type=int, default=256)
    ap.add_argument("--lo", type=float, default=-100.0)
    ap.add_argument("--hi", type=float, default=100.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--fp32", action="store_true")
    ap.add_argument("--out", required=True, help="a .pgm or .csv path")
    a = ap.parse_args()
    f = landscape(a.fid, a.res, a.lo, a.hi, a.seed, a.fp32)
    if a.out.endswith(".csv"):
        write_csv(a.out, f, a.lo, a.hi)
    else:
        write_pgm(a.out, f)


if __name__ == "__main__":
    main()
