"""Plain FP64 CPU oracle for the cuROB benchmark functions.

TEST INFRASTRUCTURE ONLY.  This package is the independent reference that the
GPU library is checked against; only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA library: the C source here (``curob_oracle.c``) re-states every formula of
the paper on its own, and this module only compiles it and marshals arrays.

Parity unpinned: the readings of points the paper leaves silent or garbled
(listed in ``curob_oracle.c``) and the instance-generation choices are checked
for self-consistency only; every formula is pinned by the CPU tests.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "curob_oracle.c")
_HDR = os.path.join(_HERE, "curob_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

NUM_FUNCTIONS = 37
F_OPT = 100.0

# basic kinds, in the order of enum oracle_gkind
GKINDS = [
    "sphere", "ellipsoid", "elliptic", "discus", "cigar", "powers", "sharpv",
    "step", "weierstrass", "griewank", "rastrigin", "schafferf7", "egr",
    "rosenbrock", "schwefel", "katsuura", "lunacek", "ackley", "happycat",
    "hgbat", "schafferf6",
]
GK = {name: i for i, name in enumerate(GKINDS)}

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math"]
    if platform.machine() in ("x86_64", "AMD64"):
        cmd.append("-mfma")  # inline the hardware fma(); results are identical
    cmd += ["-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_philox4x64_10.argtypes = [u64p, u64p, u64p]
        L.oracle_philox4x64_10.restype = None
        L.oracle_G.argtypes = [ctypes.c_int, dp, ctypes.c_int]
        L.oracle_G.restype = ctypes.c_double
        L.oracle_num_components.argtypes = [ctypes.c_int]
        L.oracle_num_components.restype = ctypes.c_int
        L.oracle_component_layout.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ip, ip, ip]
        L.oracle_component_layout.restype = ctypes.c_int
        L.oracle_component_rsize.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.oracle_component_rsize.restype = ctypes.c_long
        L.oracle_generate_component.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                                ctypes.c_int, dp, ip, dp]
        L.oracle_generate_component.restype = ctypes.c_int
        L.oracle_evaluate_given.argtypes = [ctypes.c_int, ctypes.c_int, dp, ip, dp, dp,
                                            ctypes.c_long, dp, ctypes.c_int]
        L.oracle_evaluate_given.restype = ctypes.c_int
        L.oracle_evaluate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, dp,
                                      ctypes.c_long, dp, ctypes.c_int]
        L.oracle_evaluate.restype = ctypes.c_int
        L.oracle_component_z.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ip, dp,
                                         dp, ctypes.c_int, dp]
        L.oracle_component_z.restype = ctypes.c_int
        L.oracle_evaluate_from_z.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.oracle_evaluate_from_z.restype = ctypes.c_int
        L.oracle_compose.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.oracle_compose.restype = ctypes.c_int
        L.oracle_block_affine.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        L.oracle_block_affine.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def philox4x64_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib().oracle_philox4x64_10(c.ctypes.data_as(u64p), k.ctypes.data_as(u64p),
                               out.ctypes.data_as(u64p))
    return out


def G(kind, z) -> float:
    """Basic function value (no f_opt) on an already transformed vector z."""
    k = GK[kind] if isinstance(kind, str) else int(kind)
    zz = np.ascontiguousarray(z, dtype=np.float64).reshape(-1)
    return lib().oracle_G(k, _dp(zz), zz.size)


def num_components(fid: int) -> int:
    return lib().oracle_num_components(fid)


def layout(fid: int, D: int, comp: int = 0):
    """(block sizes, rotated) of one component; raises on invalid input."""
    nb = ctypes.c_int()
    rot = ctypes.c_int()
    sizes = np.zeros(5, dtype=np.int32)
    rc = lib().oracle_component_layout(fid, D, comp, ctypes.byref(nb), _ip(sizes),
                                       ctypes.byref(rot))
    if rc:
        raise ValueError(f"oracle_component_layout({fid},{D},{comp}) -> {rc}")
    return [int(s) for s in sizes[: nb.value]], bool(rot.value)


@dataclass
class Component:
    o: np.ndarray          # (D,) shift x^opt
    S: np.ndarray          # (D,) variable indices in block order
    blocks: list           # [(n_b,) ...] block sizes
    R: list                # [n_b x n_b arrays], empty if unrotated
    rotated: bool


def generate(fid: int, D: int, seed: int):
    """All components of the instance (fid, D, seed)."""
    comps = []
    for c in range(num_components(fid)):
        sizes, rot = layout(fid, D, c)
        rs = lib().oracle_component_rsize(fid, D, c)
        o = np.zeros(D)
        S = np.zeros(D, dtype=np.int32)
        R = np.zeros(max(rs, 1))
        rc = lib().oracle_generate_component(fid, D, seed, c, _dp(o), _ip(S), _dp(R))
        if rc:
            raise ValueError(f"oracle_generate_component -> {rc}")
        blocks = []
        off = 0
        if rot:
            for n in sizes:
                blocks.append(R[off: off + n * n].reshape(n, n).copy())
                off += n * n
        comps.append(Component(o=o, S=S, blocks=sizes, R=blocks, rotated=rot))
    return comps


def evaluate_given(fid: int, D: int, comps, x, nthreads: int = 1) -> np.ndarray:
    """f(x) for explicitly given instance data (list of Component)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, D)
    o = np.ascontiguousarray(np.stack([c.o for c in comps]), dtype=np.float64)
    S = np.ascontiguousarray(np.stack([c.S for c in comps]), dtype=np.int32)
    parts = [r.reshape(-1) for c in comps for r in c.R]
    R = np.ascontiguousarray(np.concatenate(parts) if parts else np.zeros(1))
    out = np.zeros(x.shape[0])
    rc = lib().oracle_evaluate_given(fid, D, _dp(o), _ip(S), _dp(R), _dp(x), x.shape[0],
                                     _dp(out), nthreads)
    if rc:
        raise ValueError(f"oracle_evaluate_given -> {rc}")
    return out


def evaluate(fid: int, D: int, seed: int, x, nthreads: int = 1) -> np.ndarray:
    """f(x) on the seeded instance, f_opt = 100 included."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, D)
    out = np.zeros(x.shape[0])
    rc = lib().oracle_evaluate(fid, D, seed, _dp(x), x.shape[0], _dp(out), nthreads)
    if rc:
        raise ValueError(f"oracle_evaluate({fid},{D}) -> {rc}")
    return out


def _packed_R(comp):
    parts = [r.reshape(-1) for r in comp.R]
    return np.ascontiguousarray(np.concatenate(parts) if parts else np.zeros(1))


def component_z(fid: int, D: int, comps, c: int, x, plain: bool = False) -> np.ndarray:
    """z of component c (block order) for one candidate x: one fma per term
    in index order (as the evaluation), or plain=True for rounded products
    added in index order."""
    comp = comps[c]
    xx = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    o = np.ascontiguousarray(comp.o, dtype=np.float64)
    S = np.ascontiguousarray(comp.S, dtype=np.int32)
    z = np.zeros(D)
    rc = lib().oracle_component_z(fid, D, c, _dp(o), _ip(S), _dp(_packed_R(comp)), _dp(xx),
                                  int(plain), _dp(z))
    if rc:
        raise ValueError(f"oracle_component_z -> {rc}")
    return z


def evaluate_from_z(fid: int, D: int, zs, d2=None) -> float:
    """f (f_opt included) from every component's z (list of D-vectors) and,
    for a composition, the squared distances d2[c] = ||x - o_c||^2."""
    z = np.ascontiguousarray(np.concatenate([np.asarray(v, dtype=np.float64) for v in zs]))
    dd = np.ascontiguousarray(np.zeros(max(len(zs), 1)) if d2 is None else d2, dtype=np.float64)
    out = np.zeros(1)
    rc = lib().oracle_evaluate_from_z(fid, D, _dp(z), _dp(dd), _dp(out))
    if rc:
        raise ValueError(f"oracle_evaluate_from_z -> {rc}")
    return float(out[0])


def compose(fid: int, D: int, G, d2) -> float:
    """A composition's f (f_opt included) from its members' values G_c and
    squared distances d2_c (Eq. composition, Eq. weight)."""
    g = np.ascontiguousarray(G, dtype=np.float64)
    dd = np.ascontiguousarray(d2, dtype=np.float64)
    out = np.zeros(1)
    rc = lib().oracle_compose(fid, D, _dp(g), _dp(dd), _dp(out))
    if rc:
        raise ValueError(f"oracle_compose -> {rc}")
    return float(out[0])


def block_affine(fid: int, D: int, comp: int = 0):
    """([s_b], [c_b]) of component comp's blocks: z_b = R_b (s_b y_b) + c_b."""
    sc = np.zeros(5)
    of = np.zeros(5)
    rc = lib().oracle_block_affine(fid, D, comp, _dp(sc), _dp(of))
    if rc:
        raise ValueError(f"oracle_block_affine -> {rc}")
    nb = len(layout(fid, D, comp)[0])
    return sc[:nb].tolist(), of[:nb].tolist()
