"""Helpers for the GPU tests: library (re)initialisation, loading the oracle's
instance into the library, and the tolerance rules (stated once, in
oracle.parity: FP64 |df| <= 1e-12 |f|; FP32 |df| <= max(1e-5 |f|, 1e-6
f_scale) with the oracle at the FP32-rounded x and the discontinuity excuse).
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
    from oracle import parity
    return parity.f_scale(fid, D, seed, n)


def fp32_ok(got, ref, fscale):
    from oracle import parity
    return parity.fp32_ok(got, ref, fscale)


def near_discontinuity(orc, fid, D, seed, x):
    from oracle import parity
    return parity.near_discontinuity(fid, D, seed, x)


def fp32_check(orc, fid, D, seed, x32, got, rows=None):
    """(ok, worst ratio, excused count, worst raw ratio) of FP32 results
    against the oracle at the FP32-rounded inputs."""
    from oracle import parity
    return parity.fp32_check(fid, D, seed, x32, got, rows)
