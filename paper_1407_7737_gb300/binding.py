"""ctypes binding of libcurob (include/curob.h).

Argument marshalling only: every function forwards to the C entry point of the
same name, and every step of the evaluation runs in the library's CUDA
kernels.  There is no fallback: if ``libcurob.so`` is missing or cannot be
loaded, the first call raises.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

STATUS = {
    0: "CUROB_OK", 1: "CUROB_ERR_NOT_INITIALIZED", 2: "CUROB_ERR_ALREADY_INITIALIZED",
    3: "CUROB_ERR_INVALID_FID", 4: "CUROB_ERR_INVALID_DIM", 5: "CUROB_ERR_CAPACITY",
    6: "CUROB_ERR_NULL_POINTER", 7: "CUROB_ERR_CUDA", 8: "CUROB_ERR_DEVICE_TIMEOUT",
    9: "CUROB_ERR_OUT_OF_MEMORY", 10: "CUROB_ERR_INVALID_ARGUMENT", 11: "CUROB_ERR_UNSUPPORTED",
}
CODES = {v: k for k, v in STATUS.items()}

PRECISION_AUTO, PRECISION_TF32X3, PRECISION_BF16X3, PRECISION_SIMT, PRECISION_EXACT = 0, 1, 2, 3, 4
PRECISION_MIXED = 5  # reported for compositions whose members take different precisions
PRECISION_FP16X3 = 6
PRECISION64_AUTO = 0
PRECISION64_SIMT = 1
PRECISION64_TENSOR = 2
NUM_FUNCTIONS = 37
FOPT = 100.0

# (name, restype, argtypes) of every exported entry point
_P = ctypes.c_void_p
_I = ctypes.c_int
_F = ctypes.c_float
_LL = ctypes.c_longlong
_SIGS = [
    ("curob_initialize", _I, [_I, _I, ctypes.c_uint64]),
    ("curob_dispose", _I, []),
    ("curob_evaluate", _I, [_I, _P, _I, _P, _P]),
    ("curob_evaluatef", _I, [_I, _P, _I, _P, _P]),
    ("curob_h_evaluate", _I, [_I, _P, _I, _P]),
    ("curob_h_evaluatef", _I, [_I, _P, _I, _P]),
    ("curob_set_precision", _I, [_I]),
    ("curob_set_small_batch", _I, [_I]),
    ("curob_query_small", _I, [_I, _I, _P]),
    ("curob_query_precision", _I, [_I, _P]),
    ("curob_query_component_precision", _I, [_I, _I, _P]),
    ("curob_query_launches", _I, [_I, _I, _P]),
    ("curob_set_precision64", _I, [_I]),
    ("curob_query_precision64", _I, [_I, _P]),
    ("curob_query_launches64", _I, [_I, _I, _P]),
    ("curob_get_device_status", _I, [_P]),
    ("curob_selftest_bounded_wait", _I, [_P]),
    ("curob_status_string", ctypes.c_char_p, [_I]),
    ("curob_get_config", _I, [_P, _P]),
    ("curob_num_components", _I, [_I, _P]),
    ("curob_component_layout", _I, [_I, _I, _P, _P, _P]),
    ("curob_component_kinds", _I, [_I, _I, _P, _P]),
    ("curob_get_component", _I, [_I, _I, _P, _P, _P]),
    ("curob_set_component", _I, [_I, _I, _P, _P, _P]),
    ("curob_get_optimum", _I, [_I, _P]),
    ("curob_batch_create", _I, [_P, _I, _P]),
    ("curob_batch_run", _I, [_P, _P]),
    ("curob_batch_run_separate", _I, [_P, _P]),
    ("curob_batch_run_auto", _I, [_P, _P]),
    ("curob_batch_plan", _I, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    ("curob_batch_schedule", _I, [_P, _P, _P, _P]),
    ("curob_batch_status", _I, [_P, _P]),
    ("curob_batch_destroy", _I, [_P]),
    ("curob_evaluatef_multi_noalloc", _I, [_P, _P, _P, _P, _I, _P]),
    ("curob_last_error", ctypes.c_char_p, []),
    ("curob_surrogate_create", _I, [_I, ctypes.c_uint64, _P]),
    ("curob_surrogate_destroy", _I, [_P]),
    ("curob_surrogate_set_hyper", _I, [_P, _F, _F, _F, _F, _F]),
    ("curob_surrogate_get_params", _I, [_P, _P]),
    ("curob_surrogate_set_params", _I, [_P, _P]),
    ("curob_surrogate_get_grads", _I, [_P, _P]),
    ("curob_surrogate_set_standardisation", _I, [_P, _F, _F]),
    ("curob_surrogate_get_standardisation", _I, [_P, _P, _P]),
    ("curob_surrogate_standardise", _I, [_P, _P, _LL, _F, _P]),
    ("curob_surrogate_step", _I, [_P, _P, _P, _I, _F, _F, _I, _P, _P]),
    ("curob_surrogate_fit", _I, [_P, _P, _P, _LL, _F, _I, _I, _F, ctypes.c_uint64, _P, _P]),
    ("curob_surrogate_predict", _I, [_P, _P, _LL, _P, _P]),
    ("curob_surrogate_device_status", _I, [_P, _P]),
    ("curob_select_smallest", _I, [_P, _LL, _I, _P, _P]),
    ("curob_gather_rows", _I, [_P, _I, _P, _I, _P, _P]),
    ("curob_surrogate_screen", _I, [_P, _I, _P, _LL, _I, _P, _P, _P, _P, _P]),
]
EXPORTS = [s[0] for s in _SIGS]


class CurobError(RuntimeError):
    def __init__(self, fn, code):
        self.code = code
        super().__init__(f"{fn}: {STATUS.get(code, code)}")


_lib = None


def library_path() -> str:
    return _build.SO


def load(build_if_missing: bool = True):
    """Load libcurob.so (building it if absent).  Raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.SO):
        if not build_if_missing:
            raise OSError(f"libcurob.so not built: {_build.SO}")
        _build.build()
    L = ctypes.CDLL(_build.SO)
    for name, res, args in _SIGS:
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _call(name, *args, check=True):
    rc = getattr(load(), name)(*args)
    if check and rc != 0:
        err = CurobError(name, rc)
        detail = load().curob_last_error()
        if rc == CODES["CUROB_ERR_CUDA"] and detail:
            err.args = (f"{err.args[0]} ({detail.decode(errors='replace')})",)
        raise err
    return rc


def _ptr(t):
    """Address of a tensor / numpy array / raw integer pointer (or None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    raise TypeError(f"cannot take the address of {type(t)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


# ----- thin wrappers, same names as the C ABI -------------------------------
def curob_initialize(D: int, max_concurrency: int, seed: int, check=True):
    return _call("curob_initialize", D, max_concurrency, seed, check=check)


def curob_dispose(check=True):
    return _call("curob_dispose", check=check)


def curob_evaluate(fid, x, N, out, stream=None, check=True):
    return _call("curob_evaluate", fid, _ptr(x), N, _ptr(out), _stream(stream), check=check)


def curob_evaluatef(fid, x, N, out, stream=None, check=True):
    return _call("curob_evaluatef", fid, _ptr(x), N, _ptr(out), _stream(stream), check=check)


def curob_h_evaluate(fid, x, N, out, check=True):
    return _call("curob_h_evaluate", fid, _ptr(x), N, _ptr(out), check=check)


def curob_h_evaluatef(fid, x, N, out, check=True):
    return _call("curob_h_evaluatef", fid, _ptr(x), N, _ptr(out), check=check)


def curob_set_precision(mode, check=True):
    return _call("curob_set_precision", mode, check=check)


def curob_set_small_batch(max_n, check=True):
    return _call("curob_set_small_batch", max_n, check=check)


def curob_query_small(fid, N):
    v = ctypes.c_int()
    _call("curob_query_small", fid, N, ctypes.addressof(v))
    return bool(v.value)


def curob_query_precision(fid):
    m = ctypes.c_int()
    _call("curob_query_precision", fid, ctypes.addressof(m))
    return m.value


def curob_query_component_precision(fid, comp):
    m = ctypes.c_int()
    _call("curob_query_component_precision", fid, comp, ctypes.addressof(m))
    return m.value


def curob_query_launches(fid, N):
    n = ctypes.c_int()
    _call("curob_query_launches", fid, N, ctypes.addressof(n))
    return n.value


def curob_set_precision64(mode, check=True):
    return _call("curob_set_precision64", mode, check=check)


def curob_query_precision64(fid):
    m = ctypes.c_int()
    _call("curob_query_precision64", fid, ctypes.addressof(m))
    return m.value


def curob_query_launches64(fid, N):
    n = ctypes.c_int()
    _call("curob_query_launches64", fid, N, ctypes.addressof(n))
    return n.value


def curob_selftest_bounded_wait(stream=None, check=False):
    """Returns the status code (CUROB_ERR_DEVICE_TIMEOUT when the wait ran out)."""
    return _call("curob_selftest_bounded_wait", _stream(stream), check=check)


def curob_get_device_status(stream=None, check=True):
    return _call("curob_get_device_status", _stream(stream), check=check)


def curob_status_string(code) -> str:
    return load().curob_status_string(code).decode()


def curob_get_config():
    D, M = ctypes.c_int(), ctypes.c_int()
    _call("curob_get_config", ctypes.addressof(D), ctypes.addressof(M))
    return D.value, M.value


def curob_num_components(fid):
    n = ctypes.c_int()
    _call("curob_num_components", fid, ctypes.addressof(n))
    return n.value


def curob_component_layout(fid, comp):
    nb, rot = ctypes.c_int(), ctypes.c_int()
    sizes = (ctypes.c_int * 5)()
    _call("curob_component_layout", fid, comp, ctypes.addressof(nb), ctypes.addressof(sizes),
          ctypes.addressof(rot))
    return [sizes[i] for i in range(nb.value)], bool(rot.value)


def curob_component_kinds(fid, comp):
    """Basic-function kind (Table 1 row 0..22) of each block of a component."""
    nb = ctypes.c_int()
    kinds = (ctypes.c_int * 5)()
    _call("curob_component_kinds", fid, comp, ctypes.addressof(nb), ctypes.addressof(kinds))
    return [kinds[i] for i in range(nb.value)]


def curob_get_component(fid, comp):
    """(o, S, [R_b ...]) of one component, as numpy arrays."""
    import numpy as np
    D, _ = curob_get_config()
    sizes, rot = curob_component_layout(fid, comp)
    o = np.zeros(D)
    S = np.zeros(D, dtype=np.int32)
    rs = sum(n * n for n in sizes) if rot else 0
    R = np.zeros(max(rs, 1))
    _call("curob_get_component", fid, comp, o.ctypes.data, S.ctypes.data,
          R.ctypes.data if rot else None)
    blocks, off = [], 0
    if rot:
        for n in sizes:
            blocks.append(R[off: off + n * n].reshape(n, n).copy())
            off += n * n
    return o, S, blocks


def curob_set_component(fid, comp, o, S, R_blocks, check=True):
    import numpy as np
    o = np.ascontiguousarray(o, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.int32)
    parts = [np.asarray(r, dtype=np.float64).reshape(-1) for r in R_blocks]
    R = np.ascontiguousarray(np.concatenate(parts)) if parts else None
    return _call("curob_set_component", fid, comp, o.ctypes.data, S.ctypes.data,
                 R.ctypes.data if R is not None else None, check=check)


def curob_get_optimum(fid):
    import numpy as np
    D, _ = curob_get_config()
    o = np.zeros(D)
    _call("curob_get_optimum", fid, o.ctypes.data)
    return o


# ----- ragged batches ---------------------------------------------------------
class BatchItem(ctypes.Structure):
    _fields_ = [("fid", ctypes.c_int), ("D", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("N", ctypes.c_int), ("x", ctypes.c_void_p), ("out", ctypes.c_void_p)]


def curob_batch_create(items):
    """items: sequence of (fid, D, seed, N, x, out) with x/out device tensors or
    pointers.  Returns the opaque batch handle."""
    arr = (BatchItem * len(items))()
    for i, (fid, D, seed, N, x, out) in enumerate(items):
        arr[i] = BatchItem(fid, D, seed, N, _ptr(x), _ptr(out))
    h = ctypes.c_void_p()
    _call("curob_batch_create", ctypes.addressof(arr), len(items), ctypes.addressof(h))
    return h.value


def curob_batch_run(batch, stream=None, check=True):
    return _call("curob_batch_run", batch, _stream(stream), check=check)


def curob_batch_run_separate(batch, stream=None, check=True):
    return _call("curob_batch_run_separate", batch, _stream(stream), check=check)


def curob_batch_run_auto(batch, stream=None, check=True):
    return _call("curob_batch_run_auto", batch, _stream(stream), check=check)


def curob_batch_plan(batch):
    """dict of the autotuner's choices per precision."""
    v = [ctypes.c_int() for _ in range(9)]
    _call("curob_batch_plan", batch, *[ctypes.addressof(a) for a in v])
    keys = ("items_exact", "items_tf32", "work_exact", "work_tf32", "grid_exact", "grid_tf32",
            "order_exact", "order_tf32", "concurrent")
    return {k: a.value for k, a in zip(keys, v)}


def curob_batch_schedule(batch):
    n, g, o = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _call("curob_batch_schedule", batch, ctypes.addressof(n), ctypes.addressof(g),
          ctypes.addressof(o))
    return n.value, g.value, o.value


def curob_batch_status(batch, stream=None, check=True):
    return _call("curob_batch_status", batch, _stream(stream), check=check)


def curob_batch_destroy(batch, check=True):
    return _call("curob_batch_destroy", batch, check=check)


def curob_evaluatef_multi_noalloc(fids, xs, Ns, outs, stream=None, check=True):
    """Several functions of the current instance in one launch that allocates
    no device memory; xs / outs are device tensors or pointers."""
    n = len(fids)
    f = (ctypes.c_int * n)(*fids)
    nn = (ctypes.c_int * n)(*Ns)
    xp = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    op = (ctypes.c_void_p * n)(*[_ptr(o) for o in outs])
    return _call("curob_evaluatef_multi_noalloc", ctypes.addressof(f), ctypes.addressof(xp),
                 ctypes.addressof(nn), ctypes.addressof(op), n, _stream(stream), check=check)


SURROGATE_INPUT = 100
SURROGATE_HIDDEN = 256
SURROGATE_PARAMS = 91905
# offsets of the flat parameter vector
SURROGATE_LAYOUT = {"W1": (0, (256, 100)), "b1": (25600, (256,)), "W2": (25856, (256, 256)),
                    "b2": (91392, (256,)), "w3": (91648, (256,)), "b3": (91904, ())}


def curob_last_error():
    """Text of the last CUDA failure recorded on this thread ('' if none)."""
    return load().curob_last_error().decode(errors="replace")


def curob_surrogate_create(max_batch, seed, check=True):
    """Returns the surrogate handle (an integer)."""
    h = ctypes.c_void_p()
    _call("curob_surrogate_create", max_batch, seed, ctypes.byref(h), check=check)
    return h.value


def curob_surrogate_destroy(s, check=True):
    return _call("curob_surrogate_destroy", s, check=check)


def curob_surrogate_set_hyper(s, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=1e-4,
                              check=True):
    return _call("curob_surrogate_set_hyper", s, lr, beta1, beta2, eps, weight_decay, check=check)


def curob_surrogate_get_params(s):
    import numpy as np
    out = np.empty(SURROGATE_PARAMS, dtype=np.float32)
    _call("curob_surrogate_get_params", s, out.ctypes.data)
    return out


def curob_surrogate_set_params(s, params, check=True):
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == SURROGATE_PARAMS
    return _call("curob_surrogate_set_params", s, p.ctypes.data, check=check)


def curob_surrogate_get_grads(s):
    import numpy as np
    out = np.empty(SURROGATE_PARAMS, dtype=np.float32)
    _call("curob_surrogate_get_grads", s, out.ctypes.data)
    return out


def surrogate_unflatten(v):
    """Flat parameter (or gradient) vector -> dict of arrays (W1, b1, ...)."""
    return {k: (v[o:o + int(__import__("numpy").prod(sh))].reshape(sh) if sh else float(v[o]))
            for k, (o, sh) in SURROGATE_LAYOUT.items()}


def curob_surrogate_set_standardisation(s, mu, sd, check=True):
    return _call("curob_surrogate_set_standardisation", s, mu, sd, check=check)


def curob_surrogate_get_standardisation(s):
    mu, sd = ctypes.c_float(), ctypes.c_float()
    _call("curob_surrogate_get_standardisation", s, ctypes.byref(mu), ctypes.byref(sd))
    return mu.value, sd.value


def curob_surrogate_standardise(s, f, n, f_opt=FOPT, stream=None, check=True):
    return _call("curob_surrogate_standardise", s, _ptr(f), n, f_opt, _stream(stream), check=check)


def curob_surrogate_step(s, x, f, B, f_opt=FOPT, lr=1e-3, update=1, loss_out=None, stream=None,
                         check=True):
    return _call("curob_surrogate_step", s, _ptr(x), _ptr(f), B, f_opt, lr, update,
                 _ptr(loss_out), _stream(stream), check=check)


def curob_surrogate_fit(s, x, f, n, f_opt=FOPT, epochs=4, batch=4096, lr_max=2e-3,
                        shuffle_seed=0, loss_hist=None, stream=None, check=True):
    return _call("curob_surrogate_fit", s, _ptr(x), _ptr(f), n, f_opt, epochs, batch, lr_max,
                 shuffle_seed, _ptr(loss_hist), _stream(stream), check=check)


def curob_surrogate_predict(s, x, N, out, stream=None, check=True):
    return _call("curob_surrogate_predict", s, _ptr(x), N, _ptr(out), _stream(stream), check=check)


def curob_surrogate_device_status(s, stream=None, check=True):
    return _call("curob_surrogate_device_status", s, _stream(stream), check=check)


def curob_select_smallest(v, N, k, idx, stream=None, check=True):
    return _call("curob_select_smallest", _ptr(v), N, k, _ptr(idx), _stream(stream), check=check)


def curob_gather_rows(x, D, idx, k, out, stream=None, check=True):
    return _call("curob_gather_rows", _ptr(x), D, _ptr(idx), k, _ptr(out), _stream(stream),
                 check=check)


def curob_surrogate_screen(s, fid, pool, N, k, pred, idx, x_sel, f_sel, stream=None, check=True):
    return _call("curob_surrogate_screen", s, fid, _ptr(pool), N, k, _ptr(pred), _ptr(idx),
                 _ptr(x_sel), _ptr(f_sel), _stream(stream), check=check)


# ----- tensor conveniences ---------------------------------------------------
def evaluate(fid, x, out=None, stream=None):
    """f(x) for a CUDA tensor x (N x D): FP64 -> curob_evaluate, FP32 ->
    curob_evaluatef.  Returns out (allocated if None)."""
    import torch
    if not (x.is_cuda and x.is_contiguous() and x.dim() == 2):
        raise ValueError("x must be a contiguous 2-D CUDA tensor")
    N = x.shape[0]
    if out is None:
        out = torch.empty(N, dtype=x.dtype, device=x.device)
    if stream is None:
        stream = torch.cuda.current_stream(x.device)
    if x.dtype == torch.float64:
        curob_evaluate(fid, x, N, out, stream)
    elif x.dtype == torch.float32:
        curob_evaluatef(fid, x, N, out, stream)
    else:
        raise TypeError("x must be float64 or float32")
    return out
