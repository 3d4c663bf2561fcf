"""Helpers for the GPU tests: library (re)initialisation, loading the oracle's
instance into the library, and the tolerance rules.

Tolerances (derived in the design doc from the arithmetic):
  FP64 path   |f_gpu - f_ref| <= 1e-12 |f_ref|
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
