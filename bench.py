"""Throughput benchmark of libcurob: evaluations/s of the cuROB functions at
D = 1000, N = 16384 (FP32 candidates, the mixed-precision path), next to the
FP64 path and the FP64 CPU oracle.

One step evaluates, for every one of the 37 functions, its own batch of
N = 16384 candidates uniform in [-100, 100]^1000 (37 distinct FP32 batches,
2.4 GB resident in HBM, so consecutive launches do not find their input in
L2).  value = 37 * N * n_gpus / (step time), max over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank evaluates its own batches on its own GPU (weak
scaling, no collective on the data path).  --impl reference times the FP64
CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

D = 1000
N = 16384
NFUN = 37
SEED = 0
METRIC = "evals/s at D=1000,N=16384: TF32/bf16x3 vs FP64 (rel err<=1e-5); % roofline"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="curob", choices=["curob", "reference"])
    ap.add_argument("--precision", default="auto",
                    choices=["auto", "tf32x3", "bf16x3", "simt", "exact", "fp16x3"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the FP64 and forced-precision side measurements")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="skip the learned pre-screen side measurement")
    ap.add_argument("--surrogate-fids", default="all",
                    help="functions of the learned pre-screen measurement (all, or a,b,c)")
    ap.add_argument("--surrogate-n", type=int, default=1_000_000,
                    help="training samples and pool size of the pre-screen measurement")
    ap.add_argument("--streams", type=int, default=8,
                    help="streams the step's 37 independent calls are spread over (1: one stream)")
    ap.add_argument("--order", default="longest", choices=["longest", "fid"],
                    help="issue order of the step's calls over the streams: longest first (per-call "
                         "times measured during warm-up) or function ID")
    ap.add_argument("--paper-protocol", action="store_true",
                    help="the paper's small-batch timing (N = 50 per call, D in 10/32/64/96, FP32 and "
                         "FP64, against the oracle on one core): one JSON line, no benchmark line")
    ap.add_argument("--profile-fid", type=int, default=None,
                    help="profiling case: two launches of one function, no JSON")
    ap.add_argument("--profile-fp64", type=str, default=None,
                    help="profiling case of curob_evaluate (FP64 tensor-core path): two calls of "
                         "each listed function ('all' or comma-separated IDs), no JSON")
    return ap.parse_args()


# --------------------------------------------------------------------------
# distributed plumbing (barrier + max over ranks only)
# --------------------------------------------------------------------------
def dist_setup(args, backend=None):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend or ("nccl" if args.impl == "curob" else "gloo"))
        pg = dist
    return rank, world, local, pg


def weak_throughput(evals_per_rank, world, ms_step_max):
    """Whole-job evaluations/s: every rank evaluates its own batches (no
    exchange), the step time is the slowest rank's."""
    return evals_per_rank * world / (ms_step_max / 1e3)


def dist_max(pg, v, device):
    if pg is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg):
    if pg is not None:
        pg.barrier()


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi every 50 ms; each line is stamped on arrival and only the
    lines stamped between mark_start() and mark_end() (plus one interval)
    count, so the figures describe the timed region and not its set-up."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.first = threading.Event()
        self.t_start = self.t_end = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            self.first.wait(timeout=10.0)  # sampler running before the region opens
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))
            self.first.set()

    def mark_start(self):
        self.t_start = time.monotonic()

    def mark_end(self):
        self.t_end = time.monotonic()
        # one more sample after the region closes, so short regions get one
        time.sleep(1.5 * self.INTERVAL_MS / 1e3)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lo = self.t_start if self.t_start is not None else float("-inf")
        hi = (self.t_end + self.INTERVAL_MS / 1e3) if self.t_end is not None else float("inf")
        for t, ln in self.lines:
            if not lo <= t <= hi:
                continue
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "interval_ms": self.INTERVAL_MS}


# --------------------------------------------------------------------------
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# Algorithmic work per variable of each basic function on the FP32 path
# (Table 1 rows 0..22, the order curob_component_kinds reports): (SFU
# operations, FP32 ALU instructions, an FMA counting one), the minimum the
# formula needs; pair kinds count per pair.  Weierstrass: 21 cosines and a
# phase multiply and an FMA per term; Katsuura: 32 terms of (double, round,
# |.| FMA) and a power (lg2, ex2); Schaffer F7: two square roots, a power and
# a sine per pair; the others their transcendentals (one SFU operation each)
# and a few arithmetic instructions.
KIND_OPS = [
    (0, 1), (0, 2), (0, 2), (0, 1), (0, 1), (2, 4), (0, 1), (0, 3),   # sphere .. step
    (21, 42), (2, 4), (1, 3), (5, 8), (1, 8), (0, 5), (2, 4),          # weierstrass .. schwefel
    (2, 100), (1, 6), (1, 2), (0, 2), (0, 3), (3, 8),                  # katsuura .. schaffer F6
]
# partial sums a kind keeps (FP64 additions per 32 columns in the epilogue)
KIND_SUMS = [1, 1, 1, 2, 2, 1, 2, 1, 1, 2, 1, 1, 1, 1, 1, 2, 3, 2, 2, 3, 1]
SMS = 152
SFU_PER_CLK = 16     # SFU results per clock per SM
FP32_PER_CLK = 128   # FP32 lanes per clock per SM
FP64_NOMINAL = 1.25e12  # FP64 FLOP/s of the part (an FMA counting two)
TF32_OVER_BF16 = 1.1 / 2.25  # dense TF32 / BF16 tensor rate, nominal


def _profile_traffic():
    """DRAM bytes per call of the dominant group from the committed ncu
    summary, when it was taken of the kernel sources as they are now; else
    None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_per_call.txt")
    if not os.path.exists(path):
        return None, None
    h = hashlib.sha256()
    for f in ("curob_mma.cu", "curob_device.cuh", "curob_tc.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1407_7737_gb300", "csrc", f), "rb").read())
    want = h.hexdigest()[:16]
    sha, table = None, {}
    for ln in open(path):
        ln = ln.strip()
        if ln.startswith("kernel_sources_sha256_16:"):
            sha = ln.split(":", 1)[1].strip()
        elif ln.startswith("group ") and ":" in ln:
            k, v = ln[6:].split(":", 1)
            table[k.strip()] = float(v.split()[0])
    return (table if sha == want else None), want


def fp64_summary(cu, N, per_path):
    """curob_evaluate's two paths at the bench workload; the tensor-core
    path's executed BF16 products (28 per algorithmic multiply-add of the
    block rotations) over the whole call time, against the measured BF16
    peak."""
    pk, src = peaks()
    t_ms, s_ms = per_path["tensor"], per_path["simt"]
    prod = 0.0
    for f in range(len(t_ms)):
        for c in range(cu.curob_num_components(f)):
            sizes, rot = cu.curob_component_layout(f, c)
            if rot:
                prod += 28 * 2.0 * sum(n * n for n in sizes) * N
    achieved = prod / (sum(t_ms) / 1e3) / 1e12
    peak = pk.get("bf16_tflops")
    return {
        "path": "tensor (AUTO): seven BF16 digits per operand, 28 products, exact class sums, "
                "z rounded once; terms and sums in FP64",
        "tensor_evals_s": round(len(t_ms) * N / (sum(t_ms) / 1e3), 1),
        "simt_evals_s": round(len(s_ms) * N / (sum(s_ms) / 1e3), 1),
        "speedup_vs_simt": round(sum(s_ms) / sum(t_ms), 2),
        "per_function_ms_tensor": [round(v, 4) for v in t_ms],
        "per_function_ms_simt": [round(v, 4) for v in s_ms],
        "launches_per_call": [cu.curob_query_launches64(f, N) for f in range(len(t_ms))],
        "bf16_products_tflops_over_call_time": round(achieved, 1),
        "bf16_peak_tflops": peak,
        "frac_of_bf16_peak": round(achieved / peak, 4) if peak else None,
        "peak_source": src,
    }


def roofline(cu, pk, src, modes, launch_ms, launches, args):
    """Per-function binding roofline and the dominant group's tensor line.

    Per function, the time each unit would need at its peak for the work
    the function algorithmically requires: tensor (2 sum_b n_b^2 FLOP per
    candidate and rotated component, at the rate of algorithmic products the
    member's precision reaches), HBM (4 D + 4 bytes per candidate: x read
    once, f written), SFU and FP32 ALU (KIND_OPS per variable), FP64 (the
    partial sums per 32 columns, ||x - o||^2 of composition members per 16
    columns, the composition's weights); the binding bound is the largest,
    and frac_of_binding = bound / measured time.  The dominant group (the
    precision holding most of the step's time) is reported as a tensor line:
    achieved = its algorithmic FLOP / its CUDA-event time, peak = the rate its
    members' precisions reach."""
    bf16 = pk["bf16_tflops"]
    clk = pk.get("sm_max_mhz", 2070.0) * 1e6
    mode_peak = {1: bf16 * TF32_OVER_BF16 / 3.0, 2: bf16 / 3.0, 4: bf16 / 10.0, 6: bf16 / 3.0,
                 3: SMS * FP32_PER_CLK * 2 * clk / 1e12 / 6.0}
    sfu_rate = SMS * SFU_PER_CLK * clk
    alu_rate = SMS * FP32_PER_CLK * clk
    f64_rate = FP64_NOMINAL / 2.0
    hbm = pk["hbm_gbs"] * 1e9
    flops = np.zeros(NFUN)
    per_fn = []
    units = ("tensor", "hbm", "sfu", "alu", "fp64")
    t_bind = np.zeros(NFUN)
    t_tensor = np.zeros(NFUN)
    for f in range(NFUN):
        t = dict.fromkeys(units, 0.0)
        ncomp = cu.curob_num_components(f)
        sfu = alu = f64 = 0.0
        for c in range(ncomp):
            sizes, rot = cu.curob_component_layout(f, c)
            kinds = cu.curob_component_kinds(f, c)
            if rot:
                fl = 2.0 * sum(n * n for n in sizes) * N
                flops[f] += fl
                t["tensor"] += fl / (mode_peak[cu.curob_query_component_precision(f, c)] * 1e12)
            for n, k in zip(sizes if rot else [D], kinds):
                sfu += KIND_OPS[k][0] * n
                alu += KIND_OPS[k][1] * n
                f64 += KIND_SUMS[k] * n / 32.0
            if ncomp > 1:
                f64 += D / 16.0 + 20.0
        t["hbm"] = (4.0 * D + 4.0) * N / hbm
        t["sfu"] = sfu * N / sfu_rate
        t["alu"] = alu * N / alu_rate
        t["fp64"] = f64 * N / f64_rate
        b = max(units, key=lambda u: t[u])
        t_bind[f] = t[b]
        t_tensor[f] = t["tensor"]
        per_fn.append({"fid": f, "ms": round(float(launch_ms[f]), 4),
                       "bound_ms": {u: round(t[u] * 1e3, 4) for u in units},
                       "binding": b, "frac_of_binding": round(t[b] * 1e3 / float(launch_ms[f]), 4)})
    modes_a = np.array(modes)
    share = {m: launch_ms[modes_a == m].sum() for m in set(modes)}
    dom = max(share, key=share.get)
    sel = (modes_a == dom) & (flops > 0)
    achieved = flops[sel].sum() / (launch_ms[sel].sum() / 1e3) / 1e12
    peak = flops[sel].sum() / t_tensor[sel].sum() / 1e12
    names = {1: "mma_eval_kernel<TF32X3> (+ finish_kernel for heavy kinds)",
             2: "mma_eval_kernel<BF16X3> (+ finish_kernel for heavy kinds)",
             4: "mma_eval_kernel<EXACT> (+ finish_kernel for heavy kinds)",
             6: "mma_eval_kernel<FP16X3> (+ finish_kernel for heavy kinds)",
             3: "eval_simt_f32_kernel",
             5: "mma_eval_kernel<EXACT> + <TF32X3> + finish_kernel (mixed compositions)"}
    group = {1: "tf32x3", 2: "bf16x3", 4: "exact", 3: "simt", 5: "mixed", 6: "fp16x3"}[dom]
    table, sha = _profile_traffic()
    traffic = table.get(group) if (table and args.precision == "auto") else None
    roof = {"bound": "tensor" if dom != 3 else "alu", "kernel": names[dom],
            "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4),
            "traffic": traffic, "traffic_unit": "DRAM bytes per function call (ncu)",
            "traffic_kernel_sources_sha256_16": sha,
            "algorithmic_bytes_per_call": (4 * D + 4) * N,
            "peak_source": f"{src} bf16 burst; per algorithmic product: EXACT / 10 BF16 products, "
                           "FP16X3 / 3 FP16 products (FP16 and BF16 share the dense rate), "
                           "TF32X3 x 1.1/2.25 (TF32/BF16 dense, nominal) / 3 TF32 products",
            "share_of_step": round(share[dom] / launch_ms.sum(), 3),
            "launches_per_step": int(np.array(launches)[sel].sum()),
            "frac_of_binding": round(float(t_bind[sel].sum() / (launch_ms[sel].sum() / 1e3)), 4),
            "binding_units": {u: int(sum(1 for f in np.nonzero(sel)[0]
                                         if per_fn[f]["binding"] == u)) for u in units},
            "step_frac_of_binding": round(float(t_bind.sum() / (launch_ms.sum() / 1e3)), 4),
            "peaks": {"sfu_per_s": sfu_rate, "fp32_alu_per_s": alu_rate, "fp64_fma_per_s": f64_rate,
                      "hbm_bytes_per_s": hbm, "clock_hz": clk,
                      "source": "SFU 16 and FP32 128 per clock per SM x 152 SMs x the maximum SM "
                                "clock of MEASURED_PEAKS; FP64 1.25 TFLOP/s nominal; HBM measured"},
            "note": "achieved = algorithmic flops (2*sum n_b^2 per candidate and rotated "
                    "component) / CUDA-event time of those functions' calls"}
    return roof, per_fn


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                v = ln.split(":", 1)[1].strip()
                if v and not v.isdigit():
                    return v
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def run_curob(args):
    import torch
    from paper_1407_7737_gb300 import binding as cu
    from paper_1407_7737_gb300 import inputs

    rank, world, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cu.curob_initialize(D, N, SEED)
    mode = {"auto": 0, "tf32x3": 1, "bf16x3": 2, "simt": 3, "exact": 4, "fp16x3": 6}[args.precision]
    cu.curob_set_precision(mode)

    # 37 FP32 batches, resident in HBM before timing starts (one for a
    # profiling case)
    nb = NFUN if (args.profile_fid is None and args.profile_fp64 is None) else 1
    X = torch.empty((nb, N, D), dtype=torch.float32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(1234 + rank)
    X.uniform_(-100.0, 100.0, generator=g)
    OUT = torch.empty((nb, N), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    if args.profile_fid is not None:
        for _ in range(2):
            cu.curob_evaluatef(args.profile_fid, X[0], N, OUT[0], stream)
        torch.cuda.synchronize()
        cu.curob_get_device_status(stream)
        cu.curob_dispose()
        return
    if args.profile_fp64 is not None:
        fids = (list(range(NFUN)) if args.profile_fp64 == "all"
                else [int(v) for v in args.profile_fp64.split(",")])
        x64 = X[0].double()
        o64 = torch.empty(N, dtype=torch.float64, device=dev)
        for fid in fids:
            for _ in range(2):
                cu.curob_evaluate(fid, x64, N, o64, stream)
        torch.cuda.synchronize()
        cu.curob_get_device_status(stream)
        cu.curob_dispose()
        return

    def step(evs=None):
        for fid in range(NFUN):
            if evs is not None:
                evs[fid][0].record(stream)
            cu.curob_evaluatef(fid, X[fid], N, OUT[fid], stream)
            if evs is not None:
                evs[fid][1].record(stream)

    # The step's 37 calls are independent: spread round-robin over S
    # streams forked from and joined back into the timing stream, so that a
    # call's CTAs and the small finish blocks fill SMs another call leaves
    # idle (a 128-candidate tile per CTA occupies 128 of the 152 SMs at
    # N = 16384).
    S = max(1, args.streams)
    side = [torch.cuda.Stream(dev) for _ in range(S)] if S > 1 else []

    order = list(range(NFUN))  # issue order of the calls (longest first after warm-up)

    def step_streams():
        fork = torch.cuda.Event()
        fork.record(stream)
        for sd in side:
            sd.wait_event(fork)
        for k, fid in enumerate(order):
            cu.curob_evaluatef(fid, X[fid], N, OUT[fid], side[k % S])
        for sd in side:
            join = torch.cuda.Event()
            join.record(sd)
            stream.wait_event(join)

    timed_step = step_streams if S > 1 else step
    for _ in range(args.warmup):
        timed_step()
    torch.cuda.synchronize()
    cu.curob_get_device_status(stream)
    if S > 1 and args.order == "longest":
        # one warm-up step on one stream with every call timed; the timed
        # steps then issue the calls longest first, so that the short ones
        # fill the streams' tails (the work is the same 37 calls)
        wev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(NFUN)]
        step(wev)
        torch.cuda.synchronize()
        wt = [wev[f][0].elapsed_time(wev[f][1]) for f in range(NFUN)]
        order[:] = sorted(range(NFUN), key=lambda f: -wt[f])
        timed_step()
        torch.cuda.synchronize()

    barrier(pg)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        clk.mark_start()
        t0.record(stream)
        for s in range(args.steps):
            timed_step()
        t1.record(stream)
        torch.cuda.synchronize()
        clk.mark_end()
    barrier(pg)
    cu.curob_get_device_status(stream)
    ms_total = t0.elapsed_time(t1)
    ms_step = dist_max(pg, ms_total / args.steps, dev)
    value = weak_throughput(NFUN * N, world, ms_step)

    # the same steps on one stream, with every call timed by its own events
    # (per-function times and the roofline need calls that do not overlap)
    for _ in range(max(1, args.warmup // 2)):
        step()
    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(NFUN)] for _ in range(args.steps)]
    launch_ms = np.zeros(NFUN)
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for s in range(args.steps):
        step(evs[s])
    a1.record(stream)
    torch.cuda.synchronize()
    cu.curob_get_device_status(stream)
    ms_seq = a0.elapsed_time(a1) / args.steps
    for s in range(args.steps):
        for fid in range(NFUN):
            launch_ms[fid] += evs[s][fid][0].elapsed_time(evs[s][fid][1])
    launch_ms /= args.steps

    modes = [cu.curob_query_precision(f) for f in range(NFUN)]
    launches = [cu.curob_query_launches(f, N) for f in range(NFUN)]  # kernels per call

    def timed_pass(mode):
        """Step time (ms) of all 37 functions with the precision forced."""
        cu.curob_set_precision(mode)
        step()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize()
        cu.curob_set_precision(0)
        return a.elapsed_time(b)

    extra = {}
    fp64 = None
    if rank == 0 and not args.no_extra:
        # whether the forced precision meets the FP32 tolerance on every
        # function at this size (GPU parity tests): TF32X3 and BF16X3 do not
        # on the functions that magnify contraction error, which AUTO routes
        # to EXACT
        meets = {"tf32x3": False, "bf16x3": False, "fp16x3": False, "exact": True, "simt": True}
        forced = {}
        for name, m in (("tf32x3", 1), ("bf16x3", 2), ("fp16x3", 6), ("exact", 4), ("simt", 3)):
            forced[name] = {"evals_s": round(NFUN * N / (timed_pass(m) / 1e3), 1),
                            "meets_fp32_tolerance_on_all_functions": meets[name]}
        extra["forced_precision"] = forced
        # FP64 path (curob_evaluate) on the same workload, FP64 copies of the
        # batches: the tensor-core path (AUTO) and the FP64-pipe path
        x64 = torch.empty((N, D), dtype=torch.float64, device=dev)
        o64 = torch.empty(N, dtype=torch.float64, device=dev)
        per_path = {}
        for name, pm in (("tensor", 2), ("simt", 1)):
            cu.curob_set_precision64(pm)
            ms = []
            for fid in range(NFUN):
                x64.copy_(X[fid])
                cu.curob_evaluate(fid, x64, N, o64, stream)  # warm
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                cu.curob_evaluate(fid, x64, N, o64, stream)
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            per_path[name] = ms
        cu.curob_set_precision64(0)
        fp64 = NFUN * N / (sum(per_path["tensor"]) / 1e3)
        extra["fp64"] = fp64_summary(cu, N, per_path)

    ragged = None
    if rank == 0 and not args.no_extra:
        ragged = ragged_batch(cu, torch, dev, stream, reps=max(3, args.steps))

    pk, src = peaks()
    roof, per_fn = roofline(cu, pk, src, modes, launch_ms, launches, args)
    e2e = None
    if not args.no_e2e:
        # End to end through the boundary's host-pointer call (the paper's
        # h_func_evaluatef): every call copies its batch in from pinned host
        # memory, evaluates and copies the values back (the library overlaps
        # the copy of one chunk with the kernels of the others); one step is
        # the 37 calls.  Beside it, the device-pointer API with the copies
        # issued by the caller over the step's streams, so that copies overlap
        # other calls' kernels.
        hx = torch.empty((N, D), dtype=torch.float32, pin_memory=True)
        hx.uniform_(-100, 100)
        hout = torch.empty((NFUN, N), dtype=torch.float32, pin_memory=True)
        lanes = side if S > 1 else [stream]
        for fid in range(NFUN):
            cu.curob_h_evaluatef(fid, hx, N, hout[fid])
        reps = max(1, args.steps // 2)
        barrier(pg)
        tt = time.perf_counter()
        for _ in range(reps):
            for fid in range(NFUN):
                cu.curob_h_evaluatef(fid, hx, N, hout[fid])
        el_h = dist_max(pg, (time.perf_counter() - tt) / reps, dev)

        def e2e_step():
            for fid in range(NFUN):
                sd = lanes[fid % len(lanes)]
                with torch.cuda.stream(sd):
                    X[fid].copy_(hx, non_blocking=True)
                cu.curob_evaluatef(fid, X[fid], N, OUT[fid], sd)
                with torch.cuda.stream(sd):
                    hout[fid].copy_(OUT[fid], non_blocking=True)
            torch.cuda.synchronize()

        e2e_step()
        barrier(pg)
        tt = time.perf_counter()
        for _ in range(reps):
            e2e_step()
        el = dist_max(pg, (time.perf_counter() - tt) / reps, dev)
        e2e = {"value": round(NFUN * N * world / el_h, 1), "unit": "evals/s",
               "h2d_bytes_per_step": NFUN * N * D * 4, "d2h_bytes_per_step": NFUN * N * 4,
               "api": "curob_h_evaluatef (host buffers, pinned), 37 calls per step",
               "device_api_overlapped_evals_s": round(NFUN * N * world / el, 1),
               "device_api_overlapped": f"caller's copies + curob_evaluatef on {len(lanes)} "
                                        "stream(s), copies overlapping other calls' kernels"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(sample_n=8)

    surrogate = None
    if rank == 0 and not args.no_surrogate:
        cu.curob_dispose()
        surrogate = surrogate_bench(cu, torch, dev, stream, args)
        cu.curob_initialize(D, N, SEED)

    small = None
    if rank == 0 and not args.no_extra:
        cu.curob_dispose()
        small = small_batch_latency(cu, torch, stream)
        cu.curob_initialize(D, N, SEED)

    gpu_launches = int(sum(launches)) * args.steps
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 in/out; rotation on tensor cores as tf32x3 (3 TF32 products) or exact "
                     "(BF16 integer slices), per function and member (auto); FP64 sums",
            "data": "synthetic",
            "config": {"workload": f"37 functions x N={N} candidates U[-100,100]^{D}, FP32",
                       "D": D, "N": N, "functions": NFUN, "precision": args.precision,
                       "l2": "37 distinct input batches (2.4 GB) > L2 per step",
                       "streams": S,
                       "step": f"37 curob_evaluatef calls, round-robin over {S} stream(s) "
                               "forked from and joined into the timing stream"
                               + (", longest first" if S > 1 and args.order == "longest" else ""),
                       "parallelism": f"replicas x{world} (independent batches)"},
            "one_stream_ms_per_step": round(ms_seq, 4),
            "one_stream_evals_s": round(NFUN * N / (ms_seq / 1e3), 1),
            "fp64_evals_s": round(fp64, 1) if fp64 else None,
            **extra,
            "per_function_ms": [round(v, 4) for v in launch_ms.tolist()],
            "per_function_path": [{1: "tf32x3", 2: "bf16x3", 3: "simt", 4: "exact",
                                   5: "mixed", 6: "fp16x3"}[m] for m in modes],
            "per_function_launches": launches,
            "roofline": roof, "roofline_per_function": per_fn, "cpu_baseline": cpu, "e2e": e2e, "ragged_batch": ragged,
            "surrogate": surrogate, "small_batch": small,
            "clocks": clk.summary(), "gpu_launches": gpu_launches,
        }
        print(json.dumps(line))
    cu.curob_dispose()
    if pg is not None:
        pg.destroy_process_group()


def small_batch_latency(cu, torch, stream, runs=200, n=50):
    """The paper's timing setting (Sec. 2): N = 50 candidates per call, every
    function at D = 10, 32, 64, 96, FP32 (curob_evaluatef, AUTO) and FP64
    (curob_evaluate), each call repeated `runs` times back to back on one
    stream (CUDA events); mean microseconds per call over the functions."""
    from paper_1407_7737_gb300 import inputs
    per_d = {}
    for d in (10, 32, 64, 96):
        cu.curob_initialize(d, n, SEED)
        x64 = torch.from_numpy(inputs.uniform(n, d, 900 + d)).cuda()
        x32 = x64.float()
        o64 = torch.empty(n, dtype=torch.float64, device="cuda")
        o32 = torch.empty(n, dtype=torch.float32, device="cuda")
        t32, t64, nsmall = [], [], 0
        for fid in range(NFUN):
            try:
                cu.curob_query_precision(fid)
            except cu.CurobError:
                continue  # not defined at this D
            nsmall += int(cu.curob_query_small(fid, n))
            for call, xx, oo, acc in ((cu.curob_evaluatef, x32, o32, t32),
                                      (cu.curob_evaluate, x64, o64, t64)):
                for _ in range(5):
                    call(fid, xx, n, oo, stream)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(runs):
                    call(fid, xx, n, oo, stream)
                b.record(stream)
                torch.cuda.synchronize()
                acc.append(a.elapsed_time(b) * 1e3 / runs)
        cu.curob_get_device_status(stream)
        cu.curob_dispose()
        per_d[str(d)] = {"functions": len(t32), "small_kernel_functions": nsmall,
                         "f32_us_per_call_mean": round(float(np.mean(t32)), 2),
                         "f32_us_per_call_max": round(float(np.max(t32)), 2),
                         "f64_us_per_call_mean": round(float(np.mean(t64)), 2),
                         "f64_us_per_call_max": round(float(np.max(t64)), 2)}
    return {"N": n, "runs": runs, "per_D": per_d}


def _rank_corr(torch, a, b):
    """Spearman's rank correlation of two device vectors (ties broken by
    position; the values are continuous)."""
    def ranks(v):
        r = torch.empty_like(v, dtype=torch.float64)
        r[torch.argsort(v)] = torch.arange(v.numel(), device=v.device, dtype=torch.float64)
        return r - r.mean()
    ra, rb = ranks(a), ranks(b)
    return float((ra * rb).sum() / torch.sqrt((ra * ra).sum() * (rb * rb).sum()))


def _mixture(torch, dev, n, xopt, seed, frac_near=0.3, sigma=10.0):
    """n x 100 candidates: frac_near Gaussian around xopt (width sigma), the
    rest uniform in [-100, 100]^100, rows in random order."""
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    x = torch.empty((n, 100), dtype=torch.float32, device=dev).uniform_(-100.0, 100.0, generator=g)
    m = int(round(frac_near * n))
    x[:m] = xopt[None, :] + sigma * torch.randn((m, 100), device=dev, generator=g)
    return x[torch.randperm(n, device=dev, generator=g)].contiguous()


def surrogate_bench(cu, torch, dev, stream, args, D_s=100, epochs=4, batch=4096, frac=0.05):
    """Learned pre-screen at D = 100: for each function, an MLP 100-256-256-1
    trained on n exact evaluations (70 % uniform, 30 % around x_opt with
    sigma 10) screens a fresh pool of n candidates; the best 5 % by the
    surrogate are evaluated exactly.  Reports the training and screening
    throughput, Spearman's rho of prediction against exact value over the
    pool, the regret (best exact value kept minus best in the pool) next to
    the mean regret of a random 5 %, and the exact evaluations saved."""
    n = args.surrogate_n
    fids = list(range(NFUN)) if args.surrogate_fids == "all" else \
        [int(v) for v in args.surrogate_fids.split(",")]
    k = int(n * frac)
    cu.curob_initialize(D_s, n, SEED)
    s = cu.curob_surrogate_create(batch, 7)
    rows = []
    t_fit = t_screen = 0.0
    try:
        for fid in fids:
            xopt = torch.from_numpy(cu.curob_get_optimum(fid)).to(dev, torch.float32)
            x = _mixture(torch, dev, n, xopt, 1000 + fid)
            f = torch.empty(n, device=dev)
            cu.curob_evaluatef(fid, x, n, f, stream)
            init = cu.curob_surrogate_get_params(s) if not rows else init
            cu.curob_surrogate_set_params(s, init)
            steps = epochs * (n // batch)
            hist = torch.zeros(steps, device=dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            cu.curob_surrogate_fit(s, x, f, n, 100.0, epochs, batch, 2e-3, fid, hist, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            fit_ms = e0.elapsed_time(e1)
            del x, f
            pool = _mixture(torch, dev, n, xopt, 5000 + fid)
            pred = torch.empty(n, device=dev)
            idx = torch.empty(k, dtype=torch.int32, device=dev)
            xs = torch.empty((k, D_s), device=dev)
            fs = torch.empty(k, device=dev)
            cu.curob_surrogate_screen(s, fid, pool, n, k, pred, idx, xs, fs, stream)  # warm
            torch.cuda.synchronize()
            e0.record(stream)
            cu.curob_surrogate_screen(s, fid, pool, n, k, pred, idx, xs, fs, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            scr_ms = e0.elapsed_time(e1)
            cu.curob_surrogate_device_status(s, stream)
            fpool = torch.empty(n, device=dev)
            cu.curob_evaluatef(fid, pool, n, fpool, stream)
            torch.cuda.synchronize()
            best = float(fpool.min())
            reg = float(fs.min()) - best
            gr = torch.Generator(device=dev)
            gr.manual_seed(fid)
            reg_rand = float(np.mean([float(fpool[torch.randperm(n, device=dev, generator=gr)[:k]].min())
                                      - best for _ in range(10)]))
            h = hist.cpu().numpy()
            per = n // batch
            rows.append({"fid": fid, "rho": round(_rank_corr(torch, pred, fpool), 4),
                         "regret": reg, "random_regret": reg_rand,
                         "beats_random": reg < reg_rand,
                         "loss_first_epoch": round(float(h[:per].mean()), 4),
                         "loss_last_epoch": round(float(h[-per:].mean()), 4),
                         "fit_ms": round(fit_ms, 2), "screen_ms": round(scr_ms, 3)})
            t_fit += fit_ms
            t_screen += scr_ms
            del pool, pred, fpool
    finally:
        cu.curob_surrogate_destroy(s)
        cu.curob_dispose()
    rhos = [r["rho"] for r in rows]
    return {
        "D": D_s, "model": "MLP 100-256-256-1 GELU, BF16 operands, FP32 accumulation, AdamW",
        "train_samples": n, "pool": n, "screened_fraction": frac, "epochs": epochs, "batch": batch,
        "functions": len(rows),
        "train_samples_per_s": round(epochs * (n // batch) * batch * len(rows) / (t_fit / 1e3), 1),
        "screen_candidates_per_s": round(n * len(rows) / (t_screen / 1e3), 1),
        "exact_evals_saved": round(1.0 / frac, 2),
        "median_rho": float(np.median(rhos)) if rhos else None,
        "beats_random": int(sum(r["beats_random"] for r in rows)),
        "per_function": rows,
    }


def ragged_batch(cu, torch, dev, stream, reps=5, n_items=64, seed=2024):
    """64 items, fid uniform over the suite, D uniform over {10, 30, 50, 100,
    500, 1000}, N log-uniform in [32, 8192]: the persistent launches (one per
    precision) replayed from a CUDA graph, against every item as a
    curob_evaluatef call under AUTO and against one fused launch per item."""
    from paper_1407_7737_gb300 import inputs
    items = inputs.ragged_instances(n_items, seed)
    xs, outs, spec = [], [], []
    for i, (fid, D, N) in enumerate(items):
        x = torch.empty((N, D), dtype=torch.float32, device=dev).uniform_(-100.0, 100.0)
        o = torch.empty(N, dtype=torch.float32, device=dev)
        xs.append(x)
        outs.append(o)
        spec.append((fid, D, 1000 + D, N, x, o))
    b = cu.curob_batch_create(spec)
    evals = sum(N for (_, _, N) in items)
    try:
        cu.curob_batch_run(b, stream)  # autotune + capture
        cu.curob_batch_status(b, stream)

        def timed(fn):
            fn(b, stream)
            a = torch.cuda.Event(enable_timing=True)
            z = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            for _ in range(reps):
                fn(b, stream)
            z.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(z) / reps

        ms_p = timed(cu.curob_batch_run)
        ms_a = timed(cu.curob_batch_run_auto)
        ms_s = timed(cu.curob_batch_run_separate)
        cu.curob_batch_status(b, stream)
        nwork, grid, order = cu.curob_batch_schedule(b)
        plan = cu.curob_batch_plan(b)
    finally:
        cu.curob_batch_destroy(b)
    names = ["longest-first", "round-robin", "item-order"]
    return {"items": n_items, "evals_per_run": evals,
            "dims": sorted({D for (_, D, _) in items}),
            "persistent_graph_ms": round(ms_p, 4),
            "per_item_auto_calls_ms": round(ms_a, 4),
            "separate_fused_launches_ms": round(ms_s, 4),
            "persistent_evals_s": round(evals / (ms_p / 1e3), 1),
            "per_item_auto_evals_s": round(evals / (ms_a / 1e3), 1),
            "speedup_vs_per_item_auto": round(ms_a / ms_p, 3),
            "speedup_vs_separate_fused": round(ms_s / ms_p, 3),
            "schedule": {"work_items": nwork, "grid": grid, "order": names[order]},
            "autotuner": {"items_exact": plan["items_exact"], "items_tf32x3": plan["items_tf32"],
                          "work_exact": plan["work_exact"], "work_tf32x3": plan["work_tf32"],
                          "grid_exact": plan["grid_exact"], "grid_tf32x3": plan["grid_tf32"],
                          "order_exact": names[plan["order_exact"]],
                          "order_tf32x3": names[plan["order_tf32"]],
                          "launches": "side by side" if plan["concurrent"] else "in sequence"},
            "precision": "per item, AUTO's rule (TF32X3 or EXACT)"}


def cpu_baseline(sample_n=8, budget_s=25.0):
    """The FP64 oracle on the host's cores: every function on sample_n
    candidates of the D = 1000 workload (bounded to ~budget_s of CPU work),
    on all cores and on one core; instance setup excluded."""
    import oracle
    from paper_1407_7737_gb300 import inputs
    cores = os.cpu_count() or 1
    comps = {fid: oracle.generate(fid, D, SEED) for fid in range(NFUN)}  # setup, not timed
    x = inputs.uniform(max(sample_n, cores), D, 77)
    t = time.perf_counter()
    for fid in range(NFUN):
        oracle.evaluate_given(fid, D, comps[fid], x, nthreads=cores)
    ev = max(time.perf_counter() - t, 1e-9)
    x1 = x[:2]
    t = time.perf_counter()
    for fid in range(NFUN):
        oracle.evaluate_given(fid, D, comps[fid], x1, nthreads=1)
    ev1 = max(time.perf_counter() - t, 1e-9)
    return {"value": round(NFUN * x.shape[0] / ev, 2), "unit": "evals/s", "cores": cores,
            "kind": "oracle", "cpu_model": cpu_model(),
            "one_core_evals_s": round(NFUN * x1.shape[0] / ev1, 2),
            "sample": f"{x.shape[0]} candidates x 37 functions at D={D} on {cores} threads, "
                      f"{x1.shape[0]} x 37 on one thread (instance setup excluded)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1407_7737_gb300 import inputs
    cores = os.cpu_count() or 1
    n = max(cores, 16)
    x = inputs.uniform(n, D, 78)
    comps = {fid: oracle.generate(fid, D, SEED) for fid in range(NFUN)}
    def step():
        for fid in range(NFUN):
            oracle.evaluate_given(fid, D, comps[fid], x, nthreads=cores)
    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = (time.perf_counter() - t) / args.steps
    value = NFUN * n / el
    line = {"metric": METRIC, "value": round(value, 2), "unit": "evals/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": f"37 functions x N={N} candidates U[-100,100]^{D}, FP32",
                       "D": D, "N": N, "functions": NFUN,
                       "sample": f"{n} candidates per function per step"},
            "cpu_baseline": {"value": round(value, 2), "unit": "evals/s", "cores": cores,
                             "kind": "oracle", "cpu_model": cpu_model(),
                             "sample": f"{n} candidates x 37 functions at D={D} per step"},
            "e2e": {"value": round(value, 2), "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_paper_protocol(args, runs=1000, oracle_runs=3):
    """Sec. 1.4's timing: N = 50 candidates per call, every function at D =
    10, 32, 64, 96, FP32 (curob_evaluatef, AUTO) and FP64 (curob_evaluate),
    each call repeated `runs` times back to back on one stream (CUDA events),
    against the FP64 oracle on one host core (its instance setup excluded).
    Speedup per function = oracle time / GPU time per call; reported per D as
    the mean over the functions defined at that D."""
    import torch
    import oracle
    from paper_1407_7737_gb300 import binding as cu
    from paper_1407_7737_gb300 import inputs
    n = 50
    stream = torch.cuda.current_stream()
    per_d = {}
    for d in (10, 32, 64, 96):
        cu.curob_initialize(d, n, SEED)
        x64h = inputs.uniform(n, d, 900 + d)
        x64 = torch.from_numpy(x64h).cuda()
        x32 = x64.float()
        o64 = torch.empty(n, dtype=torch.float64, device="cuda")
        o32 = torch.empty(n, dtype=torch.float32, device="cuda")
        rows = []
        for fid in range(NFUN):
            try:
                cu.curob_query_precision(fid)
            except cu.CurobError:
                continue  # not defined at this D
            times = []
            for call, xx, oo in ((cu.curob_evaluatef, x32, o32), (cu.curob_evaluate, x64, o64)):
                for _ in range(5):
                    call(fid, xx, n, oo, stream)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(runs):
                    call(fid, xx, n, oo, stream)
                b.record(stream)
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b) * 1e3 / runs)  # us per call
            comps = oracle.generate(fid, d, SEED)
            oracle.evaluate_given(fid, d, comps, x64h, nthreads=1)
            t = time.perf_counter()
            for _ in range(oracle_runs):
                oracle.evaluate_given(fid, d, comps, x64h, nthreads=1)
            t_cpu = (time.perf_counter() - t) * 1e6 / oracle_runs
            rows.append((fid, times[0], times[1], t_cpu))
        cu.curob_get_device_status(stream)
        cu.curob_dispose()
        r = np.array([[f32, f64, cpu] for _, f32, f64, cpu in rows])
        per_d[str(d)] = {
            "functions": len(rows),
            "f32_us_per_call_mean": round(float(r[:, 0].mean()), 2),
            "f64_us_per_call_mean": round(float(r[:, 1].mean()), 2),
            "oracle_us_per_call_mean": round(float(r[:, 2].mean()), 1),
            "speedup_f32_mean": round(float((r[:, 2] / r[:, 0]).mean()), 1),
            "speedup_f64_mean": round(float((r[:, 2] / r[:, 1]).mean()), 1),
            "per_function": [{"fid": f, "f32_us": round(a, 2), "f64_us": round(b, 2),
                              "oracle_us": round(c, 1)} for f, a, b, c in rows]}
    print(json.dumps({"protocol": "paper small-batch timing (N = 50 per call)", "runs": runs,
                      "oracle": "FP64 oracle, 1 host core", "per_D": per_d}))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.paper_protocol:
        run_paper_protocol(a)
    else:
        run_curob(a)
