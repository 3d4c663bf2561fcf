"""Parity rules of the GPU checks (FP64 and FP32 tolerances, the discontinuity
excuse), stated once for the tests and the smoke check.

TEST INFRASTRUCTURE ONLY (tests and the smoke check import it; the product
path never does).

Tolerances:
  FP64 path   |f_gpu - f_ref| <= 1e-12 |f_ref|
  FP32 paths  |f_gpu - f_ref| <= max(1e-5 |f_ref|, 1e-6 f_scale), f_ref the
              oracle at the FP32-rounded x, f_scale = median |f - f_opt| over
              uniform candidates of the same instance.
Discontinuous kinds (Sec. 4.1 Step: floor(z + 1/2) jumps at half-integers;
Sec. 4.9 Modified Schwefel: g1 jumps where mod(w, 500) wraps, |w| = 1000,
1500, ...): where such a variable sits within 1e-5 (|v| + 1) of a jump, an
FP32 result on the other side is rounding deciding the branch, not an error
of the path; those rows are excused (and counted).
"""
from __future__ import annotations

import numpy as np

import oracle

FOPT = 100.0

# fid -> [(component, block or None for all blocks, kind, scale)] of the
# members holding a discontinuous kind
DISC = {
    7: [(0, None, "step", 1.0)],
    15: [(0, None, "schwefel", 10.0)], 16: [(0, None, "schwefel", 10.0)],
    23: [(0, 0, "schwefel", 10.0)], 27: [(0, 3, "schwefel", 10.0)],
    28: [(0, 3, "schwefel", 10.0)],
    30: [(0, None, "schwefel", 10.0)], 31: [(0, None, "schwefel", 10.0)],
    32: [(0, None, "schwefel", 10.0)], 33: [(2, None, "schwefel", 10.0)],
    34: [(2, None, "schwefel", 10.0)], 35: [(0, 0, "schwefel", 10.0)],
    36: [(1, 3, "schwefel", 10.0), (2, 3, "schwefel", 10.0)],
}


def f_scale(fid, D, seed, n=256):
    """Median |f - f_opt| over n uniform candidates of the instance."""
    from paper_1407_7737_gb300 import inputs
    x = inputs.uniform(n, D, 9999)
    f = oracle.evaluate(fid, D, seed, x, nthreads=8)
    return float(np.median(np.abs(f - FOPT)))


def fp32_ok(got, ref, fscale):
    tol = np.maximum(1e-5 * np.abs(ref), 1e-6 * fscale)
    return np.abs(got - ref) <= tol, tol


def component_z64(c, x, scale):
    """Per-block z of one oracle component in FP64 (block order)."""
    y = np.asarray(x, dtype=np.float64) - c.o[None, :]
    if not c.rotated:
        return [scale * y]
    zs, off = [], 0
    for n, R in zip(c.blocks, c.R):
        zs.append((scale * y[:, c.S[off:off + n]]) @ R.T)
        off += n
    return zs


def jump_distance(kind, z):
    """(distance of each z entry to the nearest jump of its kind, the value the
    relative margin is taken of)."""
    if kind == "step":
        v = z + 0.5
        return np.abs(v - np.round(v)), v
    w = np.abs(z + 420.9687462275036)
    m = np.mod(w, 500.0)
    return np.where(w >= 999.0, np.minimum(m, 500.0 - m), np.inf), w


def near_discontinuity(fid, D, seed, x, comps=None):
    """Boolean per row: some Step or Modified Schwefel variable is within
    1e-5 (|v| + 1) of a jump of its function."""
    x = np.asarray(x, dtype=np.float64)
    flag = np.zeros(x.shape[0], dtype=bool)
    if fid not in DISC:
        return flag
    comps = comps if comps is not None else oracle.generate(fid, D, seed)
    for comp, block, kind, scale in DISC[fid]:
        zs = component_z64(comps[comp], x, scale)
        if block is not None:
            zs = [zs[block]]
        for z in zs:
            dist, v = jump_distance(kind, z)
            flag |= (dist <= 1e-5 * (np.abs(v) + 1.0)).any(axis=1)
    return flag


def fp32_check(fid, D, seed, x32, got, rows=None, fscale=None, ref=None):
    """(ok, worst ratio among passing rows, excused count, worst raw ratio) of
    FP32 results against the oracle at the FP32-rounded inputs."""
    r = np.arange(x32.shape[0]) if rows is None else rows
    xr = np.asarray(x32[r], dtype=np.float64)
    if ref is None:
        ref = oracle.evaluate(fid, D, seed, xr, nthreads=16)
    fs = f_scale(fid, D, seed) if fscale is None else fscale
    ok, tol = fp32_ok(got[r], ref, fs)
    excused = 0
    if fid in DISC and not ok.all():
        edge = near_discontinuity(fid, D, seed, xr)
        excused = int((~ok & edge).sum())
        ok = ok | edge
    ratio = np.abs(got[r] - ref) / tol
    return bool(ok.all()), float(ratio[ok].max() if ok.any() else np.inf), excused, float(ratio.max())


def _mirror(kind, zj):
    """zj reflected across the nearest jump of its kind (same distance, other
    side)."""
    if kind == "step":
        v = zj + 0.5
        return 2.0 * np.round(v) - v - 0.5
    c = 420.9687462275036
    w = zj + c
    a = abs(w)
    jump = np.round(a / 500.0) * 500.0
    return np.copysign(2.0 * jump - a, w) - c


def explain_excused(fid, D, seed, x32, got, rows=None, fscale=None, max_vars=12):
    """For each row fp32_check excuses: the discontinuous variables within the
    excuse margin of a jump (nearest first, at most max_vars), the oracle's f
    at the FP32-rounded x (its FP64 z), and the smallest set of those
    variables which, reflected to the other side of their jumps, gives the GPU
    value within the FP32 tolerance (found from the single-variable changes,
    then confirmed by one evaluation with all of them reflected) -- i.e.
    whether the FP32 rounding of z crossing those jumps explains the value."""
    r = np.arange(x32.shape[0]) if rows is None else np.asarray(rows)
    xr = np.asarray(x32[r], dtype=np.float64)
    ref = oracle.evaluate(fid, D, seed, xr, nthreads=16)
    fs = f_scale(fid, D, seed) if fscale is None else fscale
    ok, tol = fp32_ok(got[r], ref, fs)
    if fid not in DISC or ok.all():
        return []
    edge = near_discontinuity(fid, D, seed, xr)
    comps = oracle.generate(fid, D, seed)
    out = []
    for i in np.nonzero(~ok & edge)[0]:
        x = xr[i]
        g = float(got[r[i]])
        zs = [oracle.component_z(fid, D, comps, c, x) for c in range(len(comps))]
        d2 = [float(np.sum((x - cc.o) ** 2)) for cc in comps]
        cand = []  # (relative distance, member, index, kind, distance)
        for comp, block, kind, scale in DISC[fid]:
            sizes = comps[comp].blocks
            lo = 0 if block is None else int(sum(sizes[:block]))
            hi = D if block is None else lo + int(sizes[block])
            dist, v = jump_distance(kind, zs[comp][lo:hi])
            rel = dist / (np.abs(v) + 1.0)
            for j in np.nonzero(rel <= 1e-5)[0]:
                cand.append((float(rel[j]), comp, lo + int(j), kind, float(dist[j])))
        cand.sort()
        cand = cand[:max_vars]

        def flipped(sel):
            zo = [z.copy() for z in zs]
            for (_, comp, j, kind, _) in sel:
                zo[comp][j] = _mirror(kind, zs[comp][j])
            return oracle.evaluate_from_z(fid, D, zo, d2)

        delta = np.array([flipped([c]) - ref[i] for c in cand])
        found = None
        if cand:
            n = len(cand)
            masks = (np.arange(1, 1 << n)[:, None] >> np.arange(n)[None, :]) & 1
            hit = np.nonzero(np.abs(ref[i] + masks @ delta - g) <= tol[i])[0]
            for m in hit[np.argsort(masks[hit].sum(axis=1), kind="stable")][:8]:  # smallest sets first
                sub = tuple(int(k) for k in np.nonzero(masks[m])[0])
                f_all = flipped([cand[k] for k in sub])
                if abs(f_all - g) <= tol[i]:
                    found = (sub, f_all)
                    break
        rec = {"row": int(r[i]), "gpu": g, "oracle": float(ref[i]), "tol": float(tol[i]),
               "ratio": float(abs(g - ref[i]) / tol[i]), "near_jump_variables": len(cand),
               "gpu_on_other_side": found is not None}
        if found:
            sub, f_all = found
            rec["oracle_other_side"] = f_all
            rec["crossed"] = [{"member": cand[s][1], "z_index": cand[s][2], "kind": cand[s][3],
                               "z": float(zs[cand[s][1]][cand[s][2]]),
                               "distance_to_jump": cand[s][4]} for s in sub]
        out.append(rec)
    return out
