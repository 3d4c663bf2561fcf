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
                    choices=["auto", "tf32x3", "bf16x3", "simt", "exact"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the FP64 and forced-precision side measurements")
    ap.add_argument("--profile-fid", type=int, default=None,
                    help="profiling case: two launches of one function, no JSON")
    return ap.parse_args()


# --------------------------------------------------------------------------
# distributed plumbing (barrier + max over ranks only)
# --------------------------------------------------------------------------
def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "curob" else "gloo")
        pg = dist
    return rank, world, local, pg


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
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

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
        for ln in self.lines:
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
                "samples": len(sm)}


# --------------------------------------------------------------------------
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def algorithmic_flops(cu, fid):
    """2 * sum_b n_b^2 per candidate over every rotated block of fid (the
    contraction z_b = R_b y_b), the unit of the tensor roofline."""
    total = 0
    for c in range(cu.curob_num_components(fid)):
        sizes, rot = cu.curob_component_layout(fid, c)
        if rot:
            total += 2 * sum(n * n for n in sizes)
    return total


def run_curob(args):
    import torch
    from paper_1407_7737_gb300 import binding as cu
    from paper_1407_7737_gb300 import inputs

    rank, world, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cu.curob_initialize(D, N, SEED)
    mode = {"auto": 0, "tf32x3": 1, "bf16x3": 2, "simt": 3, "exact": 4}[args.precision]
    cu.curob_set_precision(mode)

    # 37 FP32 batches, resident in HBM before timing starts (one for a
    # profiling case)
    nb = NFUN if args.profile_fid is None else 1
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

    def step(evs=None):
        for fid in range(NFUN):
            if evs is not None:
                evs[fid][0].record(stream)
            cu.curob_evaluatef(fid, X[fid], N, OUT[fid], stream)
            if evs is not None:
                evs[fid][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    cu.curob_get_device_status(stream)

    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(NFUN)] for _ in range(args.steps)]
    launch_ms = np.zeros(NFUN)
    barrier(pg)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t0.record(stream)
        for s in range(args.steps):
            step(evs[s])
        t1.record(stream)
        torch.cuda.synchronize()
    barrier(pg)
    cu.curob_get_device_status(stream)
    ms_total = t0.elapsed_time(t1)
    for s in range(args.steps):
        for fid in range(NFUN):
            launch_ms[fid] += evs[s][fid][0].elapsed_time(evs[s][fid][1])
    launch_ms /= args.steps
    ms_step = dist_max(pg, ms_total / args.steps, dev)
    evals = NFUN * N * world
    value = evals / (ms_step / 1e3)

    modes = [cu.curob_query_precision(f) for f in range(NFUN)]

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
        for name, m in (("tf32x3", 1), ("bf16x3", 2), ("exact", 4), ("simt", 3)):
            extra[name + "_evals_s"] = round(NFUN * N / (timed_pass(m) / 1e3), 1)
        # FP64 path on the same workload (FP64 copy of the batches)
        x64 = torch.empty((N, D), dtype=torch.float64, device=dev)
        o64 = torch.empty(N, dtype=torch.float64, device=dev)
        fp64_ms = 0.0
        for fid in range(NFUN):
            x64.copy_(X[fid])
            cu.curob_evaluate(fid, x64, N, o64, stream)  # warm
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            cu.curob_evaluate(fid, x64, N, o64, stream)
            b.record(stream)
            torch.cuda.synchronize()
            fp64_ms += a.elapsed_time(b)
        fp64 = NFUN * N / (fp64_ms / 1e3)

    ragged = None
    if rank == 0 and not args.no_extra:
        ragged = ragged_batch(cu, torch, dev, stream, reps=max(3, args.steps))

    # roofline of the dominant kernel (the path holding most of the step)
    pk, src = peaks()
    flops = np.array([algorithmic_flops(cu, f) * N for f in range(NFUN)], dtype=np.float64)
    mma = np.array([m in (1, 2, 4) for m in modes])
    t_mma, t_simt = launch_ms[mma].sum(), launch_ms[~mma].sum()
    if t_mma >= t_simt:
        sel = mma & (flops > 0)
        achieved = flops[sel].sum() / (launch_ms[sel].sum() / 1e3) / 1e12
        peak = pk["bf16_tflops"] * (1.1 / 2.25)  # TF32 dense = bf16 x nominal ratio
        roof = {"bound": "tensor", "kernel": "mma_eval_kernel (tcgen05 TF32x3)",
                "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "peak_source": f"{src} bf16 x 1.1/2.25 (TF32/BF16 nominal ratio)",
                "share_of_step": round(t_mma / launch_ms.sum(), 3),
                "note": "algorithmic flops 2*sum(n_b^2) per candidate; three split products execute 3x"}
    else:
        sel = (~mma) & (flops > 0)
        achieved = flops[sel].sum() / (launch_ms[sel].sum() / 1e3) / 1e12
        peak = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 FMA lanes x 2 flop x max SM clock
        roof = {"bound": "alu", "kernel": "eval_simt_f32_kernel (compensated FP32)",
                "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                "share_of_step": round(t_simt / launch_ms.sum(), 3),
                "note": "algorithmic flops 2*sum(n_b^2) per candidate; the compensated dot product executes ~6x"}

    e2e = None
    if not args.no_e2e:
        hx = torch.empty((N, D), dtype=torch.float32, pin_memory=True)
        hx.uniform_(-100, 100)
        hout = torch.empty(N, dtype=torch.float32, pin_memory=True)
        for fid in range(NFUN):
            cu.curob_h_evaluatef(fid, hx, N, hout)
        barrier(pg)
        tt = time.perf_counter()
        for _ in range(max(1, args.steps // 2)):
            for fid in range(NFUN):
                cu.curob_h_evaluatef(fid, hx, N, hout)
        el = (time.perf_counter() - tt) / max(1, args.steps // 2)
        el = dist_max(pg, el, dev)
        e2e = {"value": round(NFUN * N * world / el, 1), "unit": "evals/s",
               "h2d_bytes_per_step": NFUN * N * D * 4, "d2h_bytes_per_step": NFUN * N * 4,
               "api": "curob_h_evaluatef (pinned host buffers)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(sample_n=8)

    gpu_launches = NFUN * args.steps
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (tf32x3/bf16x3 rotation, f64 shift)", "data": "synthetic",
            "config": {"workload": f"37 functions x N={N} candidates U[-100,100]^{D}, FP32",
                       "D": D, "N": N, "functions": NFUN, "precision": args.precision,
                       "l2": "37 distinct input batches (2.4 GB) > L2 per step",
                       "parallelism": f"replicas x{world} (independent batches)"},
            "fp64_evals_s": round(fp64, 1) if fp64 else None,
            **extra,
            "per_function_ms": [round(v, 4) for v in launch_ms.tolist()],
            "per_function_path": [{1: "tf32x3", 2: "bf16x3", 3: "simt", 4: "exact"}[m]
                                  for m in modes],
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "ragged_batch": ragged,
            "clocks": clk.summary(), "gpu_launches": gpu_launches,
        }
        print(json.dumps(line))
    cu.curob_dispose()
    if pg is not None:
        pg.destroy_process_group()


def ragged_batch(cu, torch, dev, stream, reps=5, n_items=64, seed=2024):
    """64 items, fid uniform over the suite, D uniform over {10, 30, 50, 100,
    500, 1000}, N log-uniform in [32, 8192]: one persistent launch replayed
    from a CUDA graph against one launch per item (same EXACT arithmetic)."""
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
        ms_s = timed(cu.curob_batch_run_separate)
        cu.curob_batch_status(b, stream)
        nwork, grid, order = cu.curob_batch_schedule(b)
    finally:
        cu.curob_batch_destroy(b)
    return {"items": n_items, "evals_per_run": evals,
            "dims": sorted({D for (_, D, _) in items}),
            "persistent_graph_ms": round(ms_p, 4), "separate_launches_ms": round(ms_s, 4),
            "persistent_evals_s": round(evals / (ms_p / 1e3), 1),
            "separate_evals_s": round(evals / (ms_s / 1e3), 1),
            "speedup": round(ms_s / ms_p, 3),
            "schedule": {"work_items": nwork, "grid": grid,
                         "order": ["longest-first", "round-robin", "item-order"][order]},
            "precision": "exact (all items)"}


def cpu_baseline(sample_n=8, budget_s=25.0):
    """The FP64 oracle on the machine's host cores: every function on sample_n
    candidates of the D = 1000 workload (bounded to ~budget_s of CPU work)."""
    import oracle
    from paper_1407_7737_gb300 import inputs
    cores = os.cpu_count() or 1
    x = inputs.uniform(max(sample_n, cores), D, 77)
    t = time.perf_counter()
    n_done = 0
    for fid in range(NFUN):
        oracle.evaluate(fid, D, SEED, x, nthreads=cores)  # includes instance setup
        n_done += x.shape[0]
    total = time.perf_counter() - t
    # setup (generation) is not evaluation: time it alone and subtract
    t = time.perf_counter()
    for fid in range(NFUN):
        oracle.generate(fid, D, SEED)
    gen = time.perf_counter() - t
    ev = max(total - gen, 1e-9)
    return {"value": round(n_done / ev, 2), "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": f"{x.shape[0]} candidates x 37 functions at D={D} (instance setup excluded)"}


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
                             "kind": "oracle",
                             "sample": f"{n} candidates x 37 functions at D={D} per step"},
            "e2e": {"value": round(value, 2), "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_curob(a)
