"""Helpers for the GPU tests: library (re)initialisation, loading the oracle's
instance into the library, and the tolerance rules.

Tolerances:
  FP64 path   |f_gpu - f_ref| <= 1e-12 |f_ref|  (same FP64 arithmetic; only the
              summation order and the rotation's accumulation differ)
  FP32 paths  |f_gpu - f_ref| <= max(1e-5 |f_ref|, 1e-6 f_scale), f_ref the
              oracle at the FP32-rounded x, f_scale = median |f - f_opt| over
              uniform candidates of the same instance.
"""
import numpy as np

FOPT = 100.0
_state = {"cfg": None}


def cu():
    from paper_1407_7737_gb300 import binding
    return binding


def ensure(D, max_conc, seed=0):
    """Initialise the library for (D, max_conc, seed) unless it already is."""
    b = cu()
    cfg = (D, max_conc, seed)
    if _state["cfg"] == cfg:
        return b
    if _state["cfg"] is not None:
        b.curob_dispose()
    _state["cfg"] = None
    b.curob_initialize(D, max_conc, seed)
    _state["cfg"] = cfg
    return b


def invalidate():
    """The instance was modified (oracle data loaded): re-init on next use."""
    if _state["cfg"] is not None:
        cu().curob_dispose()
    _state["cfg"] = None


def load_oracle_instance(orc, fid, D, seed):
    """Replace the library's components of fid with the oracle's own."""
    comps = orc.generate(fid, D, seed)
    for c, comp in enumerate(comps):
        cu().curob_set_component(fid, c, comp.o, comp.S, comp.R)
    return comps


def gpu_eval(fid, x_np, dtype):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to(device="cuda", dtype=dtype)
    out = cu().evaluate(fid, x)
    torch.cuda.synchronize()
    cu().curob_get_device_status(None)
    return out.cpu().numpy().astype(np.float64)


def rel_err(a, b):
    return np.abs(a - b) / np.abs(b)


def f_scale(orc, fid, D, seed, n=256):
    from paper_1407_7737_gb300 import inputs
    x = inputs.uniform(n, D, 9999)
    f = orc.evaluate(fid, D, seed, x, nthreads=8)
    return float(np.median(np.abs(f - FOPT)))


def fp32_ok(got, ref, fscale):
    tol = np.maximum(1e-5 * np.abs(ref), 1e-6 * fscale)
    return np.abs(got - ref) <= tol, tol


# Discontinuous kinds (Sec. 4.1 Step: floor(z + 1/2) jumps at half-integers;
# Sec. 4.9 Modified Schwefel: g1 jumps where mod(w, 500) wraps, |w| = 1000,
# 1500, ...).  Where such a variable sits within 1e-5 (|v| + 1) of a jump, an
# FP32 result on the other side is rounding deciding the branch, not an error
# of the path; those rows are excused (and counted).  Members holding them:
# fid -> [(component, block or None for all blocks, kind, scale)].
_DISC = {
    7: [(0, None, "step", 1.0)],
    15: [(0, None, "schwefel", 10.0)], 16: [(0, None, "schwefel", 10.0)],
    23: [(0, 0, "schwefel", 10.0)], 27: [(0, 3, "schwefel", 10.0)],
    28: [(0, 3, "schwefel", 10.0)],
    30: [(0, None, "schwefel", 10.0)], 31: [(0, None, "schwefel", 10.0)],
    32: [(0, None, "schwefel", 10.0)], 33: [(2, None, "schwefel", 10.0)],
    34: [(2, None, "schwefel", 10.0)], 35: [(0, 0, "schwefel", 10.0)],
    36: [(1, 3, "schwefel", 10.0), (2, 3, "schwefel", 10.0)],
}


def _component_z(c, x, scale):
    """Per-block z of one oracle component in FP64 (block order)."""
    y = np.asarray(x, dtype=np.float64) - c.o[None, :]
    if not c.rotated:
        return [scale * y]
    zs, off = [], 0
    for n, R in zip(c.blocks, c.R):
        zs.append((scale * y[:, c.S[off:off + n]]) @ R.T)
        off += n
    return zs


def near_discontinuity(orc, fid, D, seed, x):
    """Boolean per row: some Step or Modified Schwefel variable is within
    1e-5 (|v| + 1) of a jump of its function."""
    x = np.asarray(x, dtype=np.float64)
    flag = np.zeros(x.shape[0], dtype=bool)
    if fid not in _DISC:
        return flag
    comps = orc.generate(fid, D, seed)
    for comp, block, kind, scale in _DISC[fid]:
        zs = _component_z(comps[comp], x, scale)
        if block is not None:
            zs = [zs[block]]
        for z in zs:
            if kind == "step":
                v = z + 0.5
                dist = np.abs(v - np.round(v))
            else:
                w = np.abs(z + 420.9687462275036)
                m = np.mod(w, 500.0)
                dist = np.where(w >= 999.0, np.minimum(m, 500.0 - m), np.inf)
                v = w
            flag |= (dist <= 1e-5 * (np.abs(v) + 1.0)).any(axis=1)
    return flag


def fp32_check(orc, fid, D, seed, x32, got, rows=None):
    """(ok, worst ratio, excused count) of FP32 results against the oracle at
    the FP32-rounded inputs."""
    r = np.arange(x32.shape[0]) if rows is None else rows
    xr = np.asarray(x32[r], dtype=np.float64)
    ref = orc.evaluate(fid, D, seed, xr, nthreads=16)
    ok, tol = fp32_ok(got[r], ref, f_scale(orc, fid, D, seed))
    excused = 0
    if fid in _DISC and not ok.all():
        edge = near_discontinuity(orc, fid, D, seed, xr)
        excused = int((~ok & edge).sum())
        ok = ok | edge
    ratio = np.abs(got[r] - ref) / tol
    return bool(ok.all()), float(ratio[ok].max() if ok.any() else np.inf), excused, float(ratio.max())
