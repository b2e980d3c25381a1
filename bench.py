#!/usr/bin/env python
"""Benchmark: periodic Ewald-RPY Brownian-dynamics steps per second at
N = 8000 beads (400 chains x 20 beads, theta solution at c/c* = 4, excluded
volume off, overlap-corrected RPY, 16 Wiener vectors, N_Ch = 40).

One step = the whole hot path on one configuration: forces, dense D(R)
assembly (self + real-space images + reciprocal sum + M*), Lanczos bounds,
the first product D.[F, dW], the Chebyshev terms and the Euler update.

  python bench.py [--gpus N --steps K --warmup W] [--precision fp64|mixed_f16|mixed_bf16]
  python bench.py --impl reference ...     # the CPU oracle on the host cores

Prints one JSON line (rank 0).  N > 1 runs independent replicas, one per
rank (weak scaling; the path has no data-path exchange).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BD steps/sec at N=8000 (D build + Chebyshev), FP64 vs mixed; % of roofline"
WORKLOAD = ("theta solution N=8000 (400 chains x 20 beads), c/c*=4, EV off, overlap-corrected "
            "RPY, dense D 24000x24000, 16 Wiener vectors, N_Ch=40")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="both",
                    choices=["both", "fp64", "fp64_df", "mixed_f16", "mixed_bf16"],
                    help="both: FP64 (FP64 multiply-adds and double-float on the FP32 "
                         "pipe) and mixed (IEEE-half) on the same system; the headline "
                         "value is the mixed step, the FP64 steps are reported beside it")
    ap.add_argument("--nch", type=int, default=40)
    ap.add_argument("--m", type=int, default=16)
    ap.add_argument("--alpha-factor", default="auto",
                    help="alpha = f sqrt(pi)/L; 'auto' times bd_build_D for a few f first "
                         "(untimed) and keeps the fastest per precision")
    ap.add_argument("--lanczos", type=int, default=30)
    ap.add_argument("--bounds", default="lagged", choices=["lagged", "fresh"],
                    help="mixed plans: lagged = bounds from the previous step's Lanczos "
                         "carried in the products; fresh = --lanczos products per step")
    ap.add_argument("--shape", default="auto", choices=["auto", "1", "2", "3"],
                    help="launch shape of the mixed product: auto = autotuned on the first "
                         "warm-up step; 1/2 = stream-K with 1/2 CTAs per SM; 3 = symmetric "
                         "(upper triangle of D16).  Profiles fix it (a profiler distorts the "
                         "autotuner's timings)")
    ap.add_argument("--no-graph", action="store_true",
                    help="mixed plans: time direct bd_step calls only (default: the step "
                         "captured once with bd_step_capture and replayed with "
                         "bd_step_replay, the direct steps reported beside it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--workload", default="n8000",
                    choices=["n8000", "batch", "theta", "lma", "spectral", "lambda"],
                    help="batch: 64 replicas, N ~ U[200, 2000], mixed, one graph launch "
                         "per step (replica-steps/s); theta: the theta-solution statics "
                         "validation (N_b = 20 and 40, N_c = 20, a = 0.5, dt = 0.01, five "
                         "concentrations), reported against Eqs. (Re2), (Rg2); lma: dense D "
                         "(HMA) against matrix-free products (LMA) at N = 8000 and larger N")
    ap.add_argument("--replicas", type=int, default=64)
    ap.add_argument("--chains", type=int, default=400,
                    help="chains of 20 beads (400 = the N=8000 workload; smaller only for "
                         "profiler captures)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms, ws, device):
    """The slowest rank's time: every rank gets the max over ranks (one
    all-reduce; no collective on the data path)."""
    if ws <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(ws, steps, ms):
    """Whole-job throughput: every rank advances its own replica `steps`
    times in the (max-over-ranks) time ms."""
    return ws * steps / (ms * 1e-3)


def replica_chains(cfg, rank):
    """The rank's replica: the same system shape, its own seeded chains."""
    from paper_1203_6208_gb300 import inputs
    return inputs.make_chains(cfg, seed=cfg.seed + 17 * rank)


def system(alpha_factor, chains=400):
    from paper_1203_6208_gb300 import inputs
    cfg, extra = inputs.preset("c4", alpha_factor=alpha_factor, n_chains=chains)
    return cfg, cfg.params()


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample of the same workload)

def oracle_sample_step(p, R, m, nch, rows):
    """Oracle work of one step restricted to `rows` bead rows: those rows of
    D plus the N_Ch - 1 products restricted to them.  Returns seconds."""
    import numpy as np
    import oracle
    n3 = 3 * p["n"]
    X = np.random.default_rng(0).standard_normal((m, n3))
    Y = np.zeros((m, n3))
    t0 = time.perf_counter()
    Drows = oracle.build_D_rows(p, R, 0, rows)
    for _ in range(nch - 1):
        oracle.lib().oracle_apply_rows(n3, 0, 3 * rows, oracle._ptr(Drows), oracle._ptr(X), m,
                                       oracle._ptr(Y))
    return time.perf_counter() - t0


# Ewald splits the oracle is tried at (alpha = f sqrt(pi)/L)
ORACLE_ALPHAS = (0.75, 1.0, 1.25, 1.5)


def oracle_alpha(chains, R, rows=16):
    """The oracle's own best Ewald split: the factor f whose D rows the oracle
    (as it stands) builds fastest on this system; the products do not depend
    on alpha.  Both CPU figures of the benchmark use it."""
    import oracle
    best = None
    for f in ORACLE_ALPHAS:
        _, p = system(f, chains)
        t0 = time.perf_counter()
        oracle.build_D_rows(p, R, 0, rows)
        t = time.perf_counter() - t0
        if best is None or t < best[1]:
            best = (f, t)
    return best[0]


def cpu_baseline(chains, R, m, nch, target_s=12.0):
    import oracle
    f = oracle_alpha(chains, R)
    _, p = system(f, chains)
    n = p["n"]
    t_small = oracle_sample_step(p, R, m, nch, 32)
    rows = int(min(n, max(32, 32 * target_s / max(t_small, 1e-3))))
    t = oracle_sample_step(p, R, m, nch, rows)
    step_s = t * n / rows
    return {"value": 1.0 / step_s, "unit": "steps/s", "cores": oracle.num_threads(),
            "kind": "oracle", "alpha_factor": f,
            "sample": f"D rows and the {nch - 1} products for {rows} of {n} beads "
                      f"({t:.1f} s), scaled by N/rows to one step ({step_s:.1f} s); "
                      f"alpha = {f} sqrt(pi)/L, the oracle's fastest of {list(ORACLE_ALPHAS)}"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_1203_6208_gb300 import inputs
    import oracle
    oracle.build()
    cfg, _ = system(1.0, args.chains)
    R = inputs.make_chains(cfg)
    f = oracle_alpha(args.chains, R) if args.alpha_factor == "auto" else float(args.alpha_factor)
    cfg, p = system(f, args.chains)
    n = p["n"]
    rows = 64
    for _ in range(args.warmup):
        oracle_sample_step(p, R, args.m, args.nch, rows)
    ts = [oracle_sample_step(p, R, args.m, args.nch, rows) for _ in range(args.steps)]
    step_s = sum(ts) / len(ts) * n / rows
    v = 1.0 / step_s
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp64 oracle", "alpha_factor": f},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "alpha_factor": f,
                             "sample": f"each step: D rows + {args.nch - 1} products for {rows} "
                                       f"of {n} beads, scaled by N/rows; alpha = {f} sqrt(pi)/L, "
                                       f"the oracle's fastest of {list(ORACLE_ALPHAS)}"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.lines = []
        self.proc = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        if vis.strip().isdigit():
            cmd += ["-i", vis.strip()]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        first_idx = None
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            if first_idx is None:
                first_idx = f[0]
            if f[0] != first_idx:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def probe_fp64_peak(which=0):
    """FP64 DFMA (which=0) or FP32 FFMA (which=2) throughput of this GPU
    (probe kernel), flop/s."""
    import ctypes
    from paper_1203_6208_gb300 import build
    L = ctypes.CDLL(build.PROBE_LIB)
    L.bd_probe_peak.restype = ctypes.c_double
    L.bd_probe_peak.argtypes = [ctypes.c_int] * 4
    sms = 152
    best = 0.0
    for blocks_per_sm in (4, 8):
        best = max(best, L.bd_probe_peak(which, 4096, sms * blocks_per_sm, 256))
    return best


def kernel_source_hash(path, name):
    """sha256 (16 hex) of the code between the kernel's begin/end markers,
    comments and whitespace removed (a comment edit leaves the kernel, and
    its recorded traffic, as it was)."""
    txt = open(os.path.join(ROOT, path)).read()
    a = txt.index(f"// -- kernel begin: {name}")
    b = txt.index(f"// -- kernel end: {name}")
    code = re.sub(r"/\*.*?\*/", " ", txt[a:b], flags=re.S)
    code = re.sub(r"//[^\n]*", " ", code)
    return hashlib.sha256(" ".join(code.split()).encode()).hexdigest()[:16]


KERNELS = {"fp64": ("paper_1203_6208_gb300/csrc/dense_f64.cu", "k_gemm_f64"),
           "fp64_df": ("paper_1203_6208_gb300/csrc/dense_f64.cu", "k_gemm_df"),
           "mixed": ("paper_1203_6208_gb300/csrc/tc_gemm.cu", "k_tc_gemm"),
           "sym": ("paper_1203_6208_gb300/csrc/sym_gemm.cu", "k_sym_gemm")}


def traffic_per_launch(kind):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"traffic_{kind}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != kernel_source_hash(*KERNELS[kind]):
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


ALPHA_FACTORS = (1.0, 1.25, 1.5, 1.75, 2.0, 2.25, 2.5)


def pick_alpha(args, p, R, precision):
    if args.alpha_factor != "auto":
        return float(args.alpha_factor), None
    from paper_1203_6208_gb300 import tune
    best, times = tune.tune_alpha(p, R, precision, factors=ALPHA_FACTORS, reps=1)
    return best, {str(k): round(v, 3) for k, v in times.items()}


def spectrum_check(plan, D, st, is64):
    """Sec. IV's bound condition d_min <= lambda_min, d_max >= lambda_max on
    the D of the last timed step (exact extremes from an FP32 symmetric
    eigensolver on the device, upper triangle; for mixed plans also of the
    16-bit copy the Chebyshev products multiply by).  Untimed."""
    import torch
    out = {"d_min": st["d_min"], "d_max": st["d_max"],
           "eigensolver": "torch.linalg.eigvalsh (FP32, upper triangle) of the step's D"}
    for which in (("f32",) if is64 else ("f32", "f16")):
        try:
            w = torch.linalg.eigvalsh(plan.D_view(D, which).float(), UPLO="U")
        except RuntimeError as e:          # a missing dense eigensolver must not end the run
            out["error"] = str(e).splitlines()[0]
            return out
        lmin, lmax = float(w[0]), float(w[-1])
        del w
        torch.cuda.empty_cache()
        key = "" if which == "f32" else "_f16"
        out["lambda_min" + key] = lmin
        out["lambda_max" + key] = lmax
        out["d_min_over_lambda_min" + key] = st["d_min"] / lmin
        out["d_max_over_lambda_max" + key] = st["d_max"] / lmax
        out["brackets" + key] = bool(st["d_min"] <= lmin and lmax <= st["d_max"])
    return out


def mixed_error_vs_fp64(args, p, R0, shape_code):
    """Error of the benchmark's mixed step against the FP64 path on the same
    configuration: two lagged mixed steps with given Wiener increments (the
    second uses the first's Lanczos bounds, as in the timed loop), then the
    FP64 plan's D.F and Chebyshev dS for the positions, dW and bounds of that
    second step.  Max-norm relative errors."""
    import torch
    from paper_1203_6208_gb300 import binding as bnd, inputs
    n3, m, nch = 3 * p["n"], args.m, args.nch
    dW = torch.tensor(inputs.make_wiener(n3, m, p["dt"], 4343), device="cuda")
    plan = bnd.Plan(p, "mixed_f16", max_rhs=m, max_cheb=nch)
    if shape_code:
        plan.set_shape(shape_code)
    R = torch.tensor(R0, device="cuda")
    D = plan.alloc_D()
    stats = bnd.new_stats()
    DF = torch.empty(n3, dtype=torch.float64, device="cuda")
    dS = torch.empty(m, n3, dtype=torch.float64, device="cuda")
    kw = dict(m=m, n_cheb=nch, lanczos_iters=args.lanczos, bound_safety=0.05,
              dmin_fraction=0.5, bounds_mode=1, stats=stats)
    plan.step(R, D, dW, **kw)
    R1 = R.clone()
    plan.step(R, D, dW, DF=DF, dS=dS, **kw)
    torch.cuda.synchronize()
    st = bnd.read_stats(stats)
    plan.close()
    del D
    torch.cuda.empty_cache()
    ref = bnd.Plan(p, "fp64", max_rhs=m, max_cheb=nch)
    D64 = ref.alloc_D()
    ref.build_D(R1, D64)
    F = torch.empty(n3, dtype=torch.float64, device="cuda")
    ref.forces(R1, F)
    DF64 = torch.empty_like(F)
    ref.apply(D64, F, DF64)
    bounds = torch.tensor([st["d_min"], st["d_max"]], dtype=torch.float64, device="cuda")
    dS64 = torch.empty_like(dS)
    ref.chebyshev(D64, bounds, nch, dW, dS64)
    torch.cuda.synchronize()
    rel = lambda a, b: float((a - b).abs().max() / b.abs().max())
    out = {"DF": rel(DF, DF64), "dS": rel(dS, dS64), "norm": "max|mixed - FP64| / max|FP64|",
           "reference": "the FP64 GPU path (parity with the FP64 oracle at 1e-11) on the same "
                        "positions, dW and bounds", "bounds": [st["d_min"], st["d_max"]],
           "targets": {"DF": 1e-5, "dS": 1e-3}}
    ref.close()
    del D64
    torch.cuda.empty_cache()
    return out


def adaptive_figure(args, p, R0, shape_code, tol=1e-3, steps=3, precision="mixed_f16"):
    """Sec. IV's adaptive N_Ch on the benchmark's system: N_Ch starts at
    Eq. (nint) and grows until E_f < tol (fresh Lanczos + pair bounds, as the
    lagged recurrence needs a fixed N_Ch).  The adaptive series reads E_f back
    on the host per candidate, so the step time is host wall clock."""
    import torch
    from paper_1203_6208_gb300 import binding as bnd
    plan = bnd.Plan(p, precision, max_rhs=args.m, max_cheb=256)
    if shape_code:
        plan.set_shape(shape_code)
    R = torch.tensor(R0, device="cuda")
    D = plan.alloc_D()
    stats = bnd.new_stats()
    kw = dict(m=args.m, n_cheb=0, ef_tol=tol, lanczos_iters=args.lanczos, bound_safety=0.05,
              dmin_fraction=0.5, seed=99, bounds_mode=0, stats=stats)
    plan.step(R, D, None, step_index=0, **kw)
    torch.cuda.synchronize()
    rows = []
    t0 = time.perf_counter()
    for k in range(steps):
        plan.step(R, D, None, step_index=1 + k, **kw)
        torch.cuda.synchronize()
        st = bnd.read_stats(stats)
        rows.append({"n_cheb": st["n_cheb"], "ef_max": st["ef_max"], "status": st["status"]})
    ms = (time.perf_counter() - t0) / steps * 1e3
    plan.close()
    del D
    torch.cuda.empty_cache()
    return {"precision": precision, "ef_tol": tol, "ms_per_step": ms, "steps_per_s": 1e3 / ms,
            "steps": rows, "max_cheb": 256, "bounds": "fresh Lanczos (30 steps) + pair estimate",
            "note": "status 6 = BD_ERR_CHEB_NOCONV (max_cheb reached); E_f is recomputed "
                    "from the final dS (the moment estimate that stops the growth is "
                    "taken on the same products)"}


def measure(args, precision, p, R0, rank, ws):
    """Warm up, then time exactly args.steps bd_step calls on the device."""
    import torch
    from paper_1203_6208_gb300 import binding as bnd
    is64 = precision.startswith("fp64")
    plan = bnd.Plan(p, "fp64" if is64 else precision, max_rhs=args.m, max_cheb=max(args.nch, 2))
    if precision == "fp64_df":
        plan.set_shape(bnd.BD_SHAPE_F64_DOUBLE_FLOAT)
    R = torch.tensor(R0, device="cuda")
    D = plan.alloc_D()
    stats = bnd.new_stats()
    # mixed steps take their bounds from the previous step's Lanczos recurrence,
    # which rides as one extra column of the products (no extra pass over D)
    bounds_mode = 1 if (not is64 and args.bounds == "lagged") else 0
    kw = dict(m=args.m, n_cheb=args.nch, lanczos_iters=args.lanczos, bound_safety=0.05,
              dmin_fraction=0.5, seed=4242 + rank, stats=stats, bounds_mode=bounds_mode)
    shape = None
    for w in range(args.warmup):
        plan.step(R, D, None, step_index=w, **kw)
        if w == 0 and not is64:
            # launch shape of the tensor-core product, timed on this D (or fixed)
            if args.shape != "auto":
                plan.set_shape(int(args.shape))
                cps, pms = int(args.shape), float("nan")
            else:
                cps, pms = plan.autotune(D)
            shape = ({"kernel": "symmetric (upper triangle of D16)"}
                     if cps == bnd.BD_SHAPE_SYMMETRIC else
                     {"kernel": "stream-K (all of D16)", "ctas_per_sm": cps})
            shape["autotune_ms"] = None if args.shape != "auto" else round(pms, 4)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(args.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for row in evs:             # torch creates the CUDA event on its first record
        for ev in row:
            ev.record(stream)
    torch.cuda.synchronize()
    clocks = ClockSampler()
    clocks.start()
    time.sleep(0.4)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    l0 = bnd.kernel_launches()
    plan.product_timing(True)
    e0.record(stream)
    torch.cuda.nvtx.range_push("timed_direct_steps")
    for k in range(args.steps):
        plan.set_phase_events(evs[k])
        plan.step(R, D, None, step_index=args.warmup + k, **kw)
    torch.cuda.nvtx.range_pop()
    e1.record(stream)
    torch.cuda.synchronize()
    prod_ms, prod_n = plan.product_timing(False)
    launches = bnd.kernel_launches() - l0
    plan.set_phase_events(None)
    ms = e0.elapsed_time(e1)
    direct_ms = ms
    graph = not is64 and not args.no_graph
    if graph:
        # the same step recorded once as a CUDA graph (noise from the device
        # step counter) and replayed: no host launch gaps between its kernels
        kwg = {k: v for k, v in kw.items()}
        plan.set_step_counter(7_000_000)
        l1 = bnd.kernel_launches()
        plan.step_capture(R, D, flags=bnd.BD_STEP_DEVICE_COUNTER, **kwg)
        launches = (bnd.kernel_launches() - l1) * args.steps     # kernels of the replays
        for _ in range(3):
            plan.step_replay()
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        torch.cuda.nvtx.range_push("timed_steps")     # a profiler can select these launches
        for k in range(args.steps):
            plan.step_replay()
        torch.cuda.nvtx.range_pop()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ms, ws, "cuda")
    st = bnd.read_stats(stats)
    # the exact spectrum is checked on the benchmark's own system only (the
    # reduced sizes serve profiler captures)
    bounds_check = spectrum_check(plan, D, st, is64) if args.chains == 400 else None
    phases = {name: sum(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(args.steps))
              / args.steps for i, name in enumerate(bnd.PHASES)}

    # roofline of the dominant kernel: the Chebyshev product (N_Ch - 2 launches
    # per step), its average launch duration from events around each launch
    n3 = 3 * p["n"]
    cheb_launch_ms = prod_ms / max(prod_n, 1)
    peaks, peak_src = measured_peaks()
    if precision == "fp64":
        flops = 2.0 * n3 * n3 * args.m
        fp64_peak = probe_fp64_peak()
        achieved = flops / (cheb_launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "k_gemm_f64<16,cheb>", "achieved": achieved,
                "peak": fp64_peak / 1e12, "unit": "TFLOP/s", "frac": achieved * 1e12 / fp64_peak,
                "peak_source": "FP64 DFMA probe (probe/peaks.cu) on this GPU (measured)",
                "traffic": traffic_per_launch("fp64"),
                "algorithmic_per_launch": f"2*(3N)^2*m = {flops:.3e} flop",
                "launch_ms": cheb_launch_ms, "launches_timed": prod_n}
    elif precision == "fp64_df":
        # 12 FP32 lane instructions per multiply-add (exact hi x hi product,
        # two cross terms, two-sum into the pair); peak = FFMA lanes x clock
        ins = 12.0 * n3 * n3 * args.m
        lane_peak = probe_fp64_peak(2) / 2.0
        achieved = ins / (cheb_launch_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "k_gemm_df<16,cheb>", "achieved": achieved,
                "peak": lane_peak / 1e12, "unit": "T FP32 lane-instructions/s",
                "frac": achieved * 1e12 / lane_peak,
                "peak_source": "FP32 FFMA probe (probe/peaks.cu) on this GPU (measured), "
                               "one FFMA = one lane instruction",
                "traffic": traffic_per_launch("fp64_df"),
                "algorithmic_per_launch": f"12*(3N)^2*m = {ins:.3e} FP32 lane instructions "
                                          f"(2*(3N)^2*m = {2.0 * n3 * n3 * args.m:.3e} FP64-"
                                          f"equivalent flop, {2.0 * n3 * n3 * args.m / (cheb_launch_ms * 1e-3) / 1e12:.3f} TFLOP/s)",
                "launch_ms": cheb_launch_ms, "launches_timed": prod_n}
    else:
        lag = args.bounds == "lagged"
        cols = args.m + (1 if lag else 0)
        bn = 16 if cols <= 16 else 32
        sym = "ctas_per_sm" not in (shape or {"ctas_per_sm": 2})
        # the 16-bit operand in and out, V_{p-1}, V_{p-2}, dS read and V_p, dS
        # written (FP64), the Lanczos column's q_j, q_{j-1} read and w written
        vec = n3 * args.m * (2 + 2 + 8 * 5) + (n3 * (2 + 8 * 3) if lag else 0)
        if sym:
            # the tiles on and above the diagonal of the 16-bit D (diagonal
            # tiles whole): the unique half of a symmetric D
            t = -(-n3 // 128)
            tiles = t * (t + 1) // 2
            dbytes = min(tiles * 128 * 128, n3 * (n3 + 128) // 2) * 2.0
            kernel = f"k_sym_gemm<{bn}> + k_sym_reduce<{bn}> (upper triangle, Chebyshev epilogue)"
            what = "upper-triangle 16-bit D + vectors"
        else:
            cps = shape["ctas_per_sm"] if shape else 2
            st = (224 * 1024 if cps == 1 else 110 * 1024) // (128 * 64 * 2 + bn * 64 * 2)
            dbytes = n3 * n3 * 2.0
            kernel = f"k_tc_gemm<{bn},{st}> (stream-K, Chebyshev epilogue)"
            what = "16-bit D + vectors"
        bytes_ = dbytes + vec
        achieved = bytes_ / (cheb_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": kernel,
                "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "peak_source": f"hbm_gbs ({peak_src} copy bandwidth)",
                "traffic": traffic_per_launch("sym" if sym else "mixed"),
                "algorithmic_per_launch": f"{what} = {bytes_:.3e} B",
                "launch_ms": cheb_launch_ms, "launches_timed": prod_n}

    # end to end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        Rh = torch.tensor(R0, dtype=torch.float64).pin_memory()
        sh = torch.empty(bnd.STATS_BYTES, dtype=torch.uint8).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            R.copy_(Rh, non_blocking=True)
            if graph:
                plan.step_replay()
            else:
                plan.step(R, D, None, step_index=10_000 + k, **kw)
            Rh.copy_(R, non_blocking=True)
            sh.copy_(stats, non_blocking=True)
            stream.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        e2e = {"value": ws / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": 8 * n3,
               "d2h_bytes_per_step": 8 * n3 + bnd.STATS_BYTES,
               "note": "per step: positions H2D from pinned memory, the step (bd_step_replay "
                       "of the captured step on mixed plans, else bd_step), positions + stats "
                       "D2H, stream sync (wall clock)"}
    out = {"value": job_value(ws, args.steps, ms), "ms_per_step": ms / args.steps,
           "launch": "CUDA graph replay (bd_step_capture / bd_step_replay)" if graph
                     else "direct bd_step calls",
           "direct_ms_per_step": direct_ms / args.steps,
           "phases_ms": phases, "step_stats": st, "roofline": roof, "gpu_launches": launches,
           "clocks": clk, "e2e": e2e, "n_kvec_half": plan.info.n_kvec,
           "bounds_check": bounds_check,
           "d_gb": plan.info.d_bytes / 1e9, "product_shape": shape}
    del D
    plan.close()
    torch.cuda.empty_cache()
    return out


def dtype_of(precision):
    return {"fp64": "f64", "fp64_df": "f64 (double-float f32 products)", "mixed_f16": "f16+f32+f64",
            "mixed_bf16": "bf16+f32+f64"}[precision]


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(local)
    else:
        torch.cuda.set_device(0)
    from paper_1203_6208_gb300 import build, inputs
    build.build()
    precs = ["fp64", "fp64_df", "mixed_f16"] if args.precision == "both" else [args.precision]
    cfg, p1 = system(1.0, args.chains)
    R0 = replica_chains(cfg, rank)
    results, alphas = {}, {}
    for prec in precs:
        if prec == "fp64_df" and "fp64" in alphas:
            f, sweep = alphas["fp64"][0], "as fp64 (the same FP64 assembly)"
        else:
            Rt = torch.tensor(R0, device="cuda")
            f, sweep = pick_alpha(args, p1, Rt, "fp64" if prec == "fp64_df" else prec)
            del Rt
        _, p = system(f, args.chains)
        alphas[prec] = (f, sweep, p)
        results[prec] = measure(args, prec, p, R0, rank, ws)
    if rank != 0:
        return
    head = precs[-1]
    r = results[head]
    f, sweep, p = alphas[head]
    line = {"metric": METRIC, "value": r["value"], "unit": "steps/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_of(head), "data": "synthetic",
            "config": {"workload": WORKLOAD if args.chains == 400 else
                       f"reduced: {args.chains} chains x 20 beads (profiling only)",
                       "n_beads": p["n"], "box_L": p["L"], "precision": head,
                       "alpha": p["alpha"], "alpha_factor": f, "alpha_sweep_ms": sweep,
                       "r_c": p["rc"], "n2max": p["n2max"], "n_kvec_half": r["n_kvec_half"],
                       "m": args.m, "n_cheb": args.nch, "lanczos_iters": args.lanczos,
                       "bounds": args.bounds if not head.startswith("fp64") else "fresh",
                       "l2": "inputs larger than L2 (D alone is %.2f GB)" % r["d_gb"],
                       "parallelism": "replicas" if ws > 1 else "single",
                       "product_shape": r["product_shape"], "launch": r["launch"]},
            "direct_ms_per_step": r["direct_ms_per_step"],
            "phases_ms": r["phases_ms"], "step_stats": r["step_stats"],
            "bounds_check": r["bounds_check"], "roofline": r["roofline"],
            "gpu_launches": r["gpu_launches"], "clocks": r["clocks"], "e2e": r["e2e"]}
    for key in ("fp64", "fp64_df"):
        if key not in results or key == head:
            continue
        q = results[key]
        fq, sq, pq = alphas[key]
        line["fp64" if key == "fp64" else "fp64_double_float"] = {
            "value": q["value"], "unit": "steps/s", "ms_per_step": q["ms_per_step"],
            "products": "FP64 multiply-adds" if key == "fp64" else
                        "double-float on the FP32 pipe (launch shape 4)",
            "alpha_factor": fq, "alpha_sweep_ms": sq, "phases_ms": q["phases_ms"],
            "step_stats": q["step_stats"], "bounds_check": q["bounds_check"],
            "roofline": q["roofline"],
            "gpu_launches": q["gpu_launches"], "clocks": q["clocks"], "e2e": q["e2e"]}
    if "fp64" in results and head != "fp64":
        line["mixed_speedup_over_fp64"] = r["value"] / results["fp64"]["value"]
    if head.startswith("mixed") and args.chains == 400:
        sh = r["product_shape"] or {}
        code = 3 if "ctas_per_sm" not in sh else int(sh["ctas_per_sm"])
        line["error_vs_fp64"] = mixed_error_vs_fp64(args, p, R0, code)
        line["adaptive_nch"] = adaptive_figure(args, p, R0, code)
        if "fp64_df" in alphas:
            # the same series in FP64 (double-float products), where E_f can
            # reach the tolerance (the 16-bit D of the mixed products sets a
            # floor near 2e-3)
            line["adaptive_nch_fp64"] = adaptive_figure(args, alphas["fp64_df"][2], R0, 4,
                                                        steps=1, precision="fp64")
    if ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        line["cpu_baseline"] = cpu_baseline(args.chains, R0, args.m, args.nch)
    print(json.dumps(line), flush=True)


def run_batch(args):
    """Batched replicas: one bd_batch_step (a single CUDA-graph launch after the
    first two calls) advances every replica; value = replica steps per second."""
    import torch
    torch.cuda.set_device(0)
    import numpy as np
    from paper_1203_6208_gb300 import binding as bnd, build, inputs
    build.build()
    cfgs = inputs.batch_systems(count=args.replicas)
    # the Ewald split of every replica at 1.75 sqrt(pi)/L: the fastest batched
    # step of a sweep over 1.5 .. 2.5 (beyond 2.0 the reciprocal sum leaves
    # the tensor-core product)
    alpha_factor = 1.75
    plist = []
    for c in cfgs:
        c.alpha_factor = alpha_factor
        plist.append(c.params())
    m = 1
    nch = 30
    b = bnd.Batch(plist, "mixed_f16", max_rhs=m, max_cheb=nch)
    R = torch.tensor(np.concatenate([inputs.make_chains(c).reshape(-1) for c in cfgs]),
                     device="cuda")
    D = b.alloc_D()
    stats = torch.zeros(b.count * bnd.STATS_BYTES, dtype=torch.uint8, device="cuda")
    kw = dict(m=m, n_cheb=nch, lanczos_iters=30, seed=77, step_index=0, stats=stats,
              bounds_mode=1)
    for _ in range(max(args.warmup, 3)):
        b.step(R, D, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler()
    clocks.start()
    time.sleep(0.4)
    l0 = bnd.kernel_launches()
    e0.record()
    for _ in range(args.steps):
        b.step(R, D, **kw)
    e1.record()
    torch.cuda.synchronize()
    host_launches = bnd.kernel_launches() - l0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    st = [bnd.BdStepStats.from_buffer_copy(bytes(stats[i * bnd.STATS_BYTES:(i + 1) * bnd.STATS_BYTES]
                                                 .cpu().numpy().tobytes())) for i in range(b.count)]
    nbeads = sum(c.n for c in cfgs)
    # the batched Chebyshev loop alone: the same batch at N_Ch = nch and at
    # N_Ch = 8 (the smallest with the lagged Lanczos column), the difference
    # over the terms between (each term streams every replica's D16 once)
    def batch_ms(n_cheb, reps):
        bb = bnd.Batch(plist, "mixed_f16", max_rhs=m, max_cheb=nch)
        kk = dict(kw, n_cheb=n_cheb)
        for _ in range(3):
            bb.step(R, D, **kk)
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            bb.step(R, D, **kk)
        z.record()
        torch.cuda.synchronize()
        bb.close()
        return a.elapsed_time(z) / reps
    t_long, t_short = batch_ms(nch, args.steps), batch_ms(8, args.steps)
    term_ms = (t_long - t_short) / (nch - 8)
    d16 = sum(9.0 * c.n * c.n * 2.0 for c in cfgs)
    vec = sum(3.0 * c.n * (m * (8 * 5 + 4 * 2) + (8 * 5 + 4)) for c in cfgs)
    peaks, peak_src = measured_peaks()
    achieved = (d16 + vec) / (term_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": "k_rows_cheb (all replicas' Chebyshev terms, one launch)",
            "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"],
            "peak_source": f"hbm_gbs ({peak_src} copy bandwidth)", "traffic": None,
            "algorithmic_per_term": f"every replica's 16-bit D + vectors = {d16 + vec:.3e} B",
            "term_ms": term_ms,
            "how": f"(step at N_Ch = {nch} - step at N_Ch = 8) / {nch - 8} terms, graph replays"}
    line = {"metric": "batched replica steps/sec (64 replicas, N ~ U[200, 2000], mixed)",
            "value": b.count * args.steps / (ms * 1e-3), "unit": "replica-steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16+f32+f64", "data": "synthetic",
            "config": {"workload": "batch", "replicas": b.count, "beads_total": nbeads,
                       "n_range": [min(c.n for c in cfgs), max(c.n for c in cfgs)],
                       "m": m, "n_cheb": nch, "bounds": "lagged", "alpha_factor": alpha_factor,
                       "d_arena_gb": b.d_total / 1e9},
            "bead_steps_per_s": nbeads * args.steps / (ms * 1e-3),
            "graph_launches": host_launches,
            "accepted": sum(x.accepted for x in st), "max_ef": max(x.ef_max for x in st),
            "roofline": roof, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_theta(args):
    """Theta-solution statics: batched trajectories from the exact equilibrium;
    per N_b and c/c*, <R_e^2> / 3(N_b - 1) and <R_g^2> / ((N_b^2 - 1)/2N_b) with
    standard errors over independent replicas.  --steps is the trajectory
    length (default 5 is raised to 4000)."""
    import torch
    torch.cuda.set_device(0)
    import numpy as np
    from paper_1203_6208_gb300 import binding as bnd, build, inputs
    build.build()
    nsteps = args.steps if args.steps > 100 else 4000
    every = 20
    burn = nsteps // 5
    out = {}
    t_all = 0.0
    steps_all = 0
    for nb in (20, 40):
        cfgs = inputs.theta_systems(nb=nb, replicas=8)
        b = bnd.Batch([c.params() for c in cfgs], "mixed_f16", max_rhs=1, max_cheb=24)
        R = torch.tensor(np.concatenate([inputs.make_chains(c).reshape(-1) for c in cfgs]),
                         device="cuda")
        D = b.alloc_D()
        stats = torch.zeros(b.count * bnd.STATS_BYTES, dtype=torch.uint8, device="cuda")
        acc = torch.zeros(b.count, 2, dtype=torch.float64, device="cuda")
        ns = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(nsteps):
            b.step(R, D, m=1, n_cheb=24, seed=91 + nb, stats=stats, bounds_mode=1)
            if k >= burn and k % every == 0:
                rows = []
                for i, c in enumerate(cfgs):
                    r = R[b.r_off[i]:b.r_off[i] + b.n3[i]].view(c.n_chains, c.nb, 3)
                    re2 = ((r[:, -1] - r[:, 0]) ** 2).sum(-1).mean()
                    rg2 = ((r - r.mean(1, keepdim=True)) ** 2).sum(-1).mean()
                    rows.append(torch.stack([re2, rg2]))
                acc += torch.stack(rows)
                ns += 1
        torch.cuda.synchronize()
        t_all += time.perf_counter() - t0
        steps_all += nsteps * b.count
        per = (acc / ns).cpu().numpy()
        ref = np.array([3.0 * (nb - 1), (nb * nb - 1) / (2.0 * nb)])
        res = {}
        for ci, c in enumerate(inputs.THETA_CONCENTRATIONS):
            blk = per[8 * ci:8 * (ci + 1)] / ref
            res[str(c)] = {"Re2_ratio": float(blk[:, 0].mean()),
                           "Re2_se": float(blk[:, 0].std(ddof=1) / math.sqrt(len(blk))),
                           "Rg2_ratio": float(blk[:, 1].mean()),
                           "Rg2_se": float(blk[:, 1].std(ddof=1) / math.sqrt(len(blk)))}
        out[f"Nb={nb}"] = res
        b.close()
        del D
        torch.cuda.empty_cache()
    line = {"metric": "theta-solution statics: <R_e^2>/3(N_b-1), <R_g^2>/((N_b^2-1)/2N_b)",
            "value": steps_all / t_all, "unit": "replica-steps/s (wall clock, incl. sampling)",
            "n_gpus": 1, "steps": nsteps, "warmup": 0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16+f32+f64", "data": "synthetic",
            "config": {"workload": "theta", "n_chains": 20, "a": 0.5, "dt": 0.01,
                       "c_over_cstar": list(inputs.THETA_CONCENTRATIONS), "replicas_per_c": 8,
                       "n_cheb": 24, "bounds": "lagged", "burn_in_steps": burn,
                       "sample_every": every},
            "statics": out}
    print(json.dumps(line), flush=True)


def fft_size(k):
    """Smallest multiple of 8 >= k whose prime factors are 2, 3 and 5 (the
    mesh transforms take radix-2, 3, 4 and 5 passes)."""
    K = int(math.ceil(k / 8.0)) * 8
    while True:
        r = K
        for f in (2, 3, 5):
            while r % f == 0:
                r //= f
        if r == 1:
            return K
        K += 8


def spectral_params(cfg, r_c=6.0, order=8, mesh_per_L=2.5):
    """Spectral-path parameters for a system: r_c = 6 l_H (alpha = M/r_c), the
    k-sphere of the same accuracy target, order-8 B-splines on a mesh of
    2.5 L points per edge (rounded up by fft_size).  Measured on the N = 8000
    system against a converged mesh (order 10, 6 L points): the mesh error
    is 3.3e-7 in FP64 there, below the FP32 floor of the mixed product
    (1.0e-6, the same as with 3.5 L points)."""
    from paper_1203_6208_gb300 import inputs
    L = cfg.params()["L"]
    f = cfg.M / r_c * L / inputs.SQRT_PI
    q = replace_cfg(cfg, alpha_factor=f).params()
    kmax = math.sqrt(q["n2max"])
    K = max(mesh_per_L * L, 2 * math.ceil(kmax) + 2)
    q.update(pme_grid=fft_size(K), pme_order=order)
    return q


def replace_cfg(cfg, **kw):
    from dataclasses import replace
    return replace(cfg, **kw)


def run_lma(args):
    """Dense-D steps (HMA, D assembled once per step) against matrix-free
    steps (LMA, D(R) X recomputed in every product) and spectral matrix-free
    steps (real space over cell lists, reciprocal sum on a mesh) on the theta
    workload of the headline (c/c* = 4, 20-bead chains, m = 16, N_Ch = 40,
    mixed), at N = 8000 and larger N; dense runs only where D fits in device
    memory, the pair-sum LMA only up to N = 32 000 (53 s per step at N = 100 000),
    the spectral path up to N = 300 000."""
    import torch
    torch.cuda.set_device(0)
    from paper_1203_6208_gb300 import binding as bnd, build, inputs
    build.build()
    free, _ = torch.cuda.mem_get_info()
    res = {}
    for chains in (400, 1600, 5000, 15000):
        cfg, _ = inputs.preset("c4", alpha_factor=1.75, n_chains=chains)
        p = cfg.params()
        R0 = inputs.make_chains(cfg)
        row = {}
        for mode in ("dense", "matfree", "spectral"):
            q = spectral_params(cfg) if mode == "spectral" else p
            if mode == "matfree" and chains > 1600:
                row[mode] = {"skipped": "pair-sum LMA too slow at this N"}
                continue
            plan = bnd.Plan(q, "mixed_f16", max_rhs=args.m, max_cheb=args.nch)
            if mode == "dense" and plan.info.d_bytes > 0.8 * free:
                row[mode] = {"skipped": "D needs %.0f GB" % (plan.info.d_bytes / 1e9)}
                plan.close()
                continue
            D = plan.alloc_D() if mode == "dense" else None
            R = torch.tensor(R0.reshape(-1), device="cuda")
            flags = 0 if mode == "dense" else bnd.BD_STEP_MATRIX_FREE
            kw = dict(m=args.m, n_cheb=args.nch, bounds_mode=3, fixman_c=8.0, flags=flags,
                      seed=7)
            reps = 1 if (mode != "dense" and chains > 400) else 2
            plan.step(R, D, None, step_index=0, **kw)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for k in range(reps):
                plan.step(R, D, None, step_index=1 + k, **kw)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            row[mode] = {"ms_per_step": ms, "steps_per_s": 1e3 / ms, "timed_steps": reps}
            if mode == "spectral":
                row[mode].update(r_c=q["rc"], n2max=q["n2max"], mesh=q["pme_grid"],
                                 order=q["pme_order"])
            del D
            plan.close()
            torch.cuda.empty_cache()
        res[f"N={cfg.n}"] = row
        print(f"N={cfg.n}", json.dumps(row), file=sys.stderr, flush=True)
    head = res["N=8000"]
    line = {"metric": "steps/sec, dense D (HMA) vs matrix-free (LMA) vs spectral, mixed",
            "value": head["spectral"]["steps_per_s"], "unit": "steps/s (spectral, N=8000)",
            "n_gpus": 1, "steps": args.steps, "warmup": 1, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "lma", "m": args.m, "n_cheb": args.nch,
                       "bounds": "fixman semidilute (C = 8)", "alpha_factor": 1.75},
            "results": res}
    print(json.dumps(line), flush=True)


def run_spectral(args):
    """The spectral matrix-free product Y = D(R) X of m + 1 columns (drift and
    Wiener columns, as in a Chebyshev product), each call building the
    per-position tables too (cell list, neighbour table, mesh-tile bins) --
    the unit the spectral step repeats; c/c* = 4, 20-bead chains, mixed."""
    import torch
    torch.cuda.set_device(0)
    from paper_1203_6208_gb300 import binding as bnd, build, inputs
    build.build()
    cfg, _ = inputs.preset("c4", alpha_factor=1.75, n_chains=args.chains)
    q = spectral_params(cfg)
    m = args.m + 1
    plan = bnd.Plan(q, "mixed_f16", max_rhs=args.m, max_cheb=args.nch)
    R = torch.tensor(inputs.make_chains(cfg).reshape(-1), device="cuda")
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn(m, 3 * cfg.n, dtype=torch.float64, device="cuda", generator=g)
    Y = torch.empty_like(X)
    for _ in range(max(args.warmup, 3)):
        plan.apply_matfree(R, X, Y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        plan.apply_matfree(R, X, Y)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    line = {"metric": "spectral products/sec (tables included)", "value": 1e3 / ms,
            "unit": "products/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "spectral", "n_beads": cfg.n, "columns": m, "r_c": q["rc"],
                       "n2max": q["n2max"], "mesh": q["pme_grid"], "order": q["pme_order"],
                       "l2": "mesh larger than L2"}}
    plan.close()
    print(json.dumps(line), flush=True)


def run_lambda(args):
    """Sec. IV's eigenvalue study behind Eqs. (fmax) and (fmin): for N_b = 10
    chains at c/c* = 4.44 and a = 0.5, N_c = 10 .. 300 (three conformations
    each), Fixman's estimates lambda^F_max,min = U+-.D.U+- / 3N (Eq.
    lmax-lmin-dilute, from the library's own FP64 products) against the exact
    extreme eigenvalues of the FP64 D (a dense symmetric eigensolver, as the
    paper's GSL routine) and the library's Lanczos bounds (60 steps).  Reports
    lambda^exact_max / lambda^F_max beside 0.35 N^0.6, C = (lambda_max /
    lambda_min) / N^0.6, and the fitted log-log slopes over N."""
    import numpy as np
    import torch
    torch.cuda.set_device(0)
    from paper_1203_6208_gb300 import binding as bnd, build, inputs
    build.build()
    rows = []
    t0 = time.perf_counter()
    for nc in (10, 20, 40, 80, 160, 300):
        for k in range(3):
            cfg = inputs.SystemConfig(n_chains=nc, nb=10, c_over_cstar=4.44,
                                      hstar=0.5 / inputs.SQRT_PI, seed=5000 + 10 * nc + k)
            p = cfg.params()
            plan = bnd.Plan(p, "fp64", max_rhs=2, max_cheb=8)
            R = torch.tensor(inputs.make_chains(cfg).reshape(-1), device="cuda")
            D = plan.alloc_D()
            plan.build_D(R, D)
            n3 = 3 * cfg.n
            U = torch.ones(2, n3, dtype=torch.float64, device="cuda")
            U[1, 1::2] = -1.0
            Y = torch.empty_like(U)
            plan.apply(D, U, Y)
            lF_max = float((U[0] * Y[0]).sum()) / n3
            lF_min = float((U[1] * Y[1]).sum()) / n3
            ev = torch.linalg.eigvalsh(plan.D_view(D))
            lmin, lmax = float(ev[0]), float(ev[-1])
            bounds = torch.empty(2, dtype=torch.float64, device="cuda")
            plan.eig_bounds(D, 60, 0.0, 1.0, bounds)
            th = bounds.cpu().numpy()
            n06 = cfg.n ** 0.6
            rows.append({"N": cfg.n, "lambdaF_max": lF_max, "lambdaF_min": lF_min,
                         "lambda_max": lmax, "lambda_min": lmin,
                         "lanczos_max": float(th[1]), "lanczos_min": float(th[0]),
                         "ratio_max": lmax / lF_max, "eq_fmax": 0.35 * n06,
                         "C": lmax / lmin / n06})
            del D, ev
            plan.close()
            torch.cuda.empty_cache()
    Ns = np.array([r["N"] for r in rows], dtype=np.float64)
    slope = lambda key: float(np.polyfit(np.log(Ns), np.log([r[key] for r in rows]), 1)[0])
    fits = {"lambda_max": slope("lambda_max"), "lambda_min": slope("lambda_min"),
            "lambdaF_max": slope("lambdaF_max"), "ratio_max": slope("ratio_max"),
            "kappa": float(np.polyfit(np.log(Ns), np.log([r["lambda_max"] / r["lambda_min"]
                                                          for r in rows]), 1)[0])}
    line = {"metric": "eigenvalue study (Sec. IV, Eqs. fmax, fmin): fitted exponents over N",
            "value": fits["ratio_max"], "unit": "d log(lambda_max/lambda^F_max) / d log N",
            "n_gpus": 1, "higher_is_better": None, "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "wall_s": round(time.perf_counter() - t0, 1),
            "config": {"workload": "lambda", "nb": 10, "c_over_cstar": 4.44, "a": 0.5,
                       "n_chains": [10, 20, 40, 80, 160, 300], "conformations": 3},
            "fits": fits, "rows": rows}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "theta":
        run_theta(args)
    elif args.workload == "lma":
        run_lma(args)
    elif args.workload == "spectral":
        run_spectral(args)
    elif args.workload == "lambda":
        run_lambda(args)
    elif args.workload == "batch":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
