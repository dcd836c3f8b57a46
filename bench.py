#!/usr/bin/env python
"""Throughput of the odd-even Kalman smoother on GB300: smoothed steps per second.

One step of the benchmark is one pass of the whole path over one synthetic problem already
resident in HBM: whitening, the odd-even QR factorization (all levels), back substitution and
the odd-even SelInv covariances of every state, all through the C ABI (libks.so).

Default workload: k = 1,000,000 states, n = m = 6, F = 0.99 * random orthogonal, H = I,
G_i ~ N(0, 1/6), K_i, C_i = L L^T (L lower triangular, diagonal U[0.5, 1.5], off-diagonal std
0.1), FP64.  Its inputs (1.5 GB) are larger than L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  Under torchrun each rank smooths its own problem (seed = rank):
the method has no exchange step between independent problems, so N GPUs are N replicas.
``--impl reference`` times the CPU oracle on a bounded sample of the same workload instead.
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

METRIC = "smoothed steps/s (FP64 plain vs FP32+refine batched) on 1 GB300; % roofline; p99 ms"
UNIT = "steps/s"
# Nominal rates, quoted as context beside the measured ones (ks_measure_fma_rate).
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (recipe table)
FP32_NOMINAL_TFLOPS = 80.5   # 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz

_PEAKS = {}
_T0 = time.perf_counter()


def log(msg):
    """Progress of the run on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench +{time.perf_counter() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def measured_peaks(device=0):
    """FMA rates the device sustains, measured by the library (TFLOP/s): the denominators of
    the arithmetic-bound rooflines."""
    if not _PEAKS:
        from paper_2502_11686_gb300 import native
        _PEAKS["fp64"] = max(native.ks_measure_fma_rate(device, native.KS_FP64) for _ in range(2))
        _PEAKS["fp32"] = max(native.ks_measure_fma_rate(device, native.KS_FP32_REFINE)
                             for _ in range(2))
    return _PEAKS


def alu_roofline(kernel, flops, ms, fp64, device=0):
    """Roofline record of an arithmetic-bound phase: algorithmic flops / its GPU time against
    the measured FMA rate of its precision (nominal rate as context)."""
    pk = measured_peaks(device)
    achieved = flops / (ms / 1e3) / 1e12
    peak = pk["fp64"] if fp64 else pk["fp32"]
    nominal = FP64_NOMINAL_TFLOPS if fp64 else FP32_NOMINAL_TFLOPS
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": ("measured DFMA rate of this GPU (ks_measure_fma_rate)" if fp64 else
                            "measured FFMA rate of this GPU (ks_measure_fma_rate)"),
            "peak_nominal": nominal, "frac_of_nominal": achieved / nominal, "traffic": None}

WORKLOADS = {
    "long_k1e6_n6": dict(k=1_000_000, n=6, m=6, f_scale=0.99, sample_k=1_000_000,
                         ref_sample_k=100_000,
                         desc="k=1,000,000 states, n=m=6, F=0.99*orth, H=I, G~N(0,1/6), "
                              "K,C=LL^T per step; states + all covariances"),
    "cv_k1000_n4": dict(k=1000, n=4, m=2, cv=True, sample_k=1000, ref_sample_k=1000,
                        desc="k=1000, 2-D constant velocity n=4, m=2, G~N(0,1), K=0.01I, "
                             "C=0.25I; states + all covariances"),
    "dense_k1e5_n48": dict(k=100_000, n=48, m=48, f_scale=0.995, sample_k=1500, ref_sample_k=300,
                           desc="k=100,000 states, n=m=48, F=0.995*orth, H=I, G~N(0,1/48), "
                                "K,C=LL^T per step; states + all covariances"),
    "large_k1e4_n128": dict(k=10_000, n=128, m=128, f_scale=0.995, sample_k=200, ref_sample_k=60,
                            desc="k=10,000 states, n=m=128, F=0.995*orth, H=I, G~N(0,1/128), "
                                 "K,C=LL^T per step; states + all covariances"),
    "huge_k500_n500": dict(k=500, n=500, m=500, f_scale=0.995, sample_k=8, ref_sample_k=3,
                           desc="k=500 states, n=m=500 (the paper's large-n regime), "
                                "F=0.995*orth, H=I, G~N(0,1/500), K,C=LL^T per step; states + "
                                "all covariances"),
}


BATCH_WORKLOADS = {
    "batch_c4": dict(nprob=512, k_lo=100, k_hi=20000, ns=(4, 8, 16, 32),
                     desc="512 independent problems, k log-uniform [100, 20000], n in {4, 8, 16, "
                          "32}, m = n/2 or n, problem i from seed i; states + all covariances"),
}


def make_problem(wl, seed, k=None):
    from paper_2502_11686_gb300 import inputs
    k = k or wl["k"]
    if wl.get("cv"):
        return inputs.cv_problem(k=k, seed=seed)
    return inputs.random_problem(k, wl["n"], wl["m"], seed=seed, f_scale=wl["f_scale"])


def flops_per_step(n, m, precision):
    """Algorithmic flops per smoothed step of each phase, counted as the kernels perform them
    (an FMA is 2 flops; a divide or square root 1).  The Householder steps use the structured
    "triangle over full block" reflectors: a reflector touches one row of the triangle and the
    p rows of the full block."""
    def factor(p):      # QR of [T (n x n upper) ; M (p x n)]
        return 2 * p * n * (n - 1) + 3 * p * n + 4 * n
    def apply(p, cols):  # n reflectors applied to `cols` companion columns
        return cols * n * (4 * p + 2)
    tri = n * (n + 1) // 2
    whiten = (n ** 3 + m ** 3) / 3 + (2 * n + 1) * n * n + n * m * m + m * m \
        + factor(m) + apply(m, 1)
    level = 3 * factor(n) + apply(n, n + 1) + apply(n, 2 * n + 1) + apply(n, 1)
    backsub = 5 * n * n
    ri = 2 * sum(c - i for c in range(n) for i in range(c + 1)) + tri
    selinv = ri + 2 * 2 * n * tri + 2 * sum((j + 1) * (n - j) for j in range(n)) \
        + 2 * 2 * n * (2 * n * n + tri)
    refine = (20 * n * n + 4 * m * n + 2 * m * m + n) if precision == "fp32_refine" else 0
    return {"whiten": whiten, "level": level, "backsub": backsub, "selinv": selinv,
            "refine": refine}


def measured_traffic(phase, precision, n):
    """DRAM bytes per unit from a committed ncu capture, if the kernel source still matches."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except (OSError, ValueError):
        return None
    key = f"{phase} phase {precision} n={n}"
    r = rec.get(key)
    if not r:
        return None
    csrc = os.path.join(ROOT, "paper_2502_11686_gb300", "csrc")
    src = open(os.path.join(csrc, "ks_small.cuh"), "rb").read() + \
        open(os.path.join(csrc, "ks_small_n.cu"), "rb").read()
    if hashlib.sha256(src).hexdigest()[:16] != r["source_digest"]:
        return None
    return r


def bytes_per_step(n, m, precision):
    """Algorithmic HBM bytes per smoothed step of each phase (each array read or written once)."""
    t = 4 if precision == "fp32_refine" else 8
    rec = (3 * n * n + 2 * n) * t           # level-buffer record
    rrec = (3 * n * n + n) * t              # R-store record
    inputs = (3 * n * n + m * n + m * m + m) * 8
    return {"whiten": inputs + rec + (8 * (n * n + m * m) if t == 4 else 0),
            "level": 2 * rec + rrec,        # read the level (2 columns -> 1), write R row
            "backsub": rrec + 3 * n * 8,
            "selinv": rrec + 3 * n * n * 8 + 2 * n * n * t + n * n * 8,
            "refine": (inputs + 8 * (n * n + m * m) + 10 * n * 8) if t == 4 else 0}


class ClockSampler:
    """nvidia-smi samples of SM clock, power and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 9:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        pw = [float(r[3]) for r in self.rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


def oracle_rate(wl, budget_s=10.0):
    """Steps/s of the CPU oracle (1 host core) on a bounded sample of the workload."""
    import oracle
    p = make_problem(wl, seed=0, k=wl["sample_k"])
    oracle.smooth(p)  # load + warm
    steps, t0 = 0, time.perf_counter()
    while True:
        oracle.smooth(p, covariances=True)
        steps += p.k
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    sample = (f"{wl['sample_k']} states of the same recipe (n={wl['n']}, m={wl['m']}), states + "
              f"covariances, repeated for {el:.1f} s")
    return steps / el, sample


def reference_arm(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    p = make_problem(wl, seed=0, k=wl["ref_sample_k"])
    oracle.smooth(p)
    for _ in range(args.warmup):
        oracle.smooth(p, covariances=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.smooth(p, covariances=True)
    el = time.perf_counter() - t0
    value = p.k * args.steps / el
    sample = f"{p.k} states of the {args.workload} recipe per step, states + covariances"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {wl['desc']}", "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _oracle_batch_task(task):
    """Worker of the problem-parallel CPU baseline: one uneven-batch problem, drawn on the host
    from its seed, smoothed by the oracle (states + covariances); returns (states, seconds)."""
    seed, k_lo, k_hi, ns = task
    import oracle
    from paper_2502_11686_gb300 import inputs
    k, n, m = inputs.uneven_shape(seed, k_lo, k_hi, ns)
    p = inputs.random_problem(k, n, m, seed=seed, f_scale=0.99)
    t0 = time.perf_counter()
    oracle.smooth(p, covariances=True)
    return k, time.perf_counter() - t0


def oracle_pool():
    """Process pool for the problem-parallel oracle: spawn (never fork after CUDA is up), one
    worker per host core."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    return mp.get_context("spawn").Pool(cores), cores


def batch_cpu_baseline(wl, pool, cores, budget_s=12.0):
    """The oracle on all host cores, problem-parallel (problems are independent), over the
    first problems of the batch until about budget_s of wall time."""
    tasks = [(i, wl["k_lo"], wl["k_hi"], wl["ns"]) for i in range(wl["nprob"])]
    t0 = time.perf_counter()
    steps, busy, done = 0, 0.0, 0
    for k, sec in pool.imap_unordered(_oracle_batch_task, tasks):
        steps += k
        busy += sec
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    wall = time.perf_counter() - t0
    return {"value": steps / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} problems of the batch recipe (same seeds, drawn on the host), "
                      f"{steps} states + covariances, problem-parallel on {cores} host cores, "
                      f"{wall:.1f} s wall ({busy:.1f} core-seconds in the oracle)"}


def batch_record(args, nprob, precision, pool=None, cores=1, want_e2e=True, steps=None,
                 warmup=None):
    """The batched form (C4): every step is one ks_smooth_batch call over 512 resident problems
    (states + covariances).  Inputs are drawn on the device (ks_generate_steps, the batch recipe
    with the library's counter-based generator, problem i from seed i)."""
    import torch

    from paper_2502_11686_gb300 import inputs, native

    wl = dict(BATCH_WORKLOADS["batch_c4"], nprob=nprob)
    steps = steps or args.steps
    warmup = warmup or args.warmup
    dev = "cuda:0"
    shapes = [inputs.uneven_shape(i, wl["k_lo"], wl["k_hi"], wl["ns"]) for i in range(nprob)]
    total_k = sum(k for k, _, _ in shapes)
    stream = torch.cuda.Stream()
    prec = native.KS_FP64 if precision == "fp64" else native.KS_FP32_REFINE

    # The autotuner's choices (grid and level kernel family per group) go to a tune cache that
    # every ctx of this record shares, and into the record.
    import tempfile
    tune_dir = tempfile.mkdtemp(prefix="ks_tune_")
    tune_path = os.path.join(tune_dir, "tune.txt").encode()

    def make_ctx(profile):
        o = native.ks_default_options()
        o.precision = prec
        o.stream = stream.cuda_stream
        o.profile = 1 if profile else 0
        o.sync = 0
        o.tune_cache = tune_path
        return native.ks_create(o)

    log(f"batched record: drawing {nprob} problems ({total_k} states) on the device")
    gctx = make_ctx(False)
    batch = []
    in_bytes = 0
    with torch.cuda.stream(stream):
        for i, (k, n, m) in enumerate(shapes):
            T = lambda *sh: torch.empty(sh, dtype=torch.float64, device=dev)   # noqa: E731
            d = {"k": k, "n": n, "m": np.full(k, m, np.int32), "F": T(k - 1, n, n),
                 "H": T(k - 1, n, n), "c": None, "K": T(k - 1, n, n), "G": T(k, m, n),
                 "o": T(k, m), "C": T(k, m, m), "u_out": T(k, n), "cov_out": T(k, n, n)}
            native.ks_generate_steps(gctx, k, n, m, i, 0.99, d["F"], d["H"], d["K"], d["G"],
                                     d["C"], d["o"])
            in_bytes += sum(d[x].numel() * 8 for x in ("F", "H", "K", "G", "o", "C")) + k * 4
            batch.append(d)
    native.ks_sync(gctx)
    native.ks_destroy(gctx)
    log("batched record: warm-up (graph capture, grid tuning)")
    ctx = make_ctx(False)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            native.ks_smooth_batch(ctx, batch)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(steps):
                native.ks_smooth_batch(ctx, batch)
            ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    st, info = native.ks_sync(ctx)
    if st != native.KS_OK:
        raise native.KsError(st, native.ks_last_error(ctx), info)
    prof_graph = native.ks_profile_read(ctx)
    native.ks_destroy(ctx)
    value = total_k * steps / (ms / 1e3)

    log(f"batched record: {steps} timed passes, {ms / steps:.1f} ms each")
    # One profiled pass (launches issued one by one, each timed into its phase).
    pctx = make_ctx(True)
    with torch.cuda.stream(stream):
        native.ks_smooth_batch(pctx, batch)
        native.ks_profile_read(pctx, reset=True)
        native.ks_smooth_batch(pctx, batch)
    prof = native.ks_profile_read(pctx)
    native.ks_destroy(pctx)
    phase_ms = {k: v for k, v in prof["phase_ms"].items() if v > 0 and k != "copy"}

    # End to end: the same call with pinned host arrays (the H2D copy of every input and the D2H
    # copy of every state and covariance inside the timed region, every step).
    e2e = None
    if want_e2e:
        log("batched record: pinned host copies of the inputs for the end-to-end pass")
        hbatch = []
        for d in batch:
            h = dict(d)
            for x in ("F", "H", "K", "G", "o", "C", "u_out", "cov_out"):
                h[x] = torch.empty(d[x].shape, dtype=torch.float64).pin_memory()
                if x not in ("u_out", "cov_out"):
                    h[x].copy_(d[x])
            hbatch.append(h)
        ectx = make_ctx(False)
        native.ks_smooth_batch(ectx, hbatch)
        native.ks_sync(ectx)
        e_steps = max(1, min(steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            native.ks_smooth_batch(ectx, hbatch)
        native.ks_sync(ectx)
        torch.cuda.synchronize()
        e_s = time.perf_counter() - t0
        native.ks_destroy(ectx)
        out_bytes = sum(d["u_out"].numel() * 8 + d["cov_out"].numel() * 8 for d in batch)
        e2e = {"value": total_k * e_steps / e_s, "unit": UNIT, "h2d_bytes_per_step": int(in_bytes),
               "d2h_bytes_per_step": int(out_bytes), "steps": e_steps,
               "timing": "wall clock, device synchronized on both sides"}
        del hbatch
        log(f"batched record: end to end {e_s / e_steps * 1e3:.1f} ms per pass")

    flops = {ph: 0.0 for ph in ("whiten", "level", "backsub", "selinv", "refine")}
    for k, n, m in shapes:
        f = flops_per_step(n, m, precision)
        for ph in flops:
            flops[ph] += f[ph] * k
    top = max(flops, key=lambda ph: phase_ms.get(ph, 0.0))
    fp64_phase = precision == "fp64" or top in ("whiten", "refine")
    roof = alu_roofline(f"{top} phase (batched launches)", flops[top], phase_ms[top], fp64_phase)
    tuned = read_tuning(tune_path.decode())
    import shutil
    shutil.rmtree(tune_dir, ignore_errors=True)
    cpu = None
    if pool is not None:
        log(f"batched record: CPU baseline on {cores} host cores")
        cpu = batch_cpu_baseline(wl, pool, cores)
    return {
        "metric": "smoothed steps/s, batched", "value": value, "unit": UNIT,
        "ms_per_step": ms / steps, "steps": steps, "warmup": warmup,
        "dtype": "f64" if precision == "fp64" else "f32+f64",
        "config": {"workload": f"batch_c4: {wl['desc']}", "problems": nprob,
                   "total_states": total_k, "precision": precision,
                   "inputs": "drawn on the device per problem seed (ks_generate_steps)",
                   "l2": f"inputs ({in_bytes / 1e9:.1f} GB) larger than L2, no flush"},
        "roofline": roof, "phase_ms_per_step": phase_ms, "cpu_baseline": cpu, "e2e": e2e,
        "tuned": tuned,
        "gpu_launches": prof_graph["launches"] // max(1, steps + warmup) * steps,
        "clocks": clk.summary(),
    }


def read_tuning(path):
    """The batched autotuner's choices from its tune cache: per group signature (precision,
    state dimension, s = small-state path or g = block kernels, largest observation count), the
    level kernel family (0: the default kernel for that dimension -- register-column where one
    is compiled; 1: column owner) and the persistent grid in blocks per SM (cache value =
    family * 64 + blocks per SM)."""
    out = {}
    try:
        with open(path) as fh:
            for line in fh:
                sig, v = line.split()
                v = int(v)
                out[sig] = {"level_kernel_family": v // 64, "blocks_per_sm": v % 64}
    except OSError:
        pass
    return out


def batch_arm(args):
    pool, cores = oracle_pool() if not args.no_cpu_baseline else (None, 1)
    rec = batch_record(args, args.nprob or BATCH_WORKLOADS[args.workload]["nprob"],
                       args.precision, pool, cores, want_e2e=not args.no_e2e)
    if pool is not None:
        pool.terminate()
    line = dict(rec, metric=METRIC, n_gpus=1, higher_is_better=True, scaling="weak",
                vs_baseline=None, data="synthetic")
    line["config"]["parallelism"] = "replicas only (independent problems)"
    print(json.dumps(line), flush=True)
    return 0


WAIT_LIMIT_MS = 120000.0   # requests still running this long after the last arrival are reported, not awaited


def serve_record(args, rates, duration, ns, precision, max_queue, verbose=True):
    """The serving loop: Poisson arrivals of synthetic requests (inputs generated on the device at
    admission), k log-uniform in [1e2, 1e5], n uniform over the served state sizes, m = n; 10 %
    of the requests get a covariance follow-up on their kept factor.  Sweeps the offered rates
    upward (stopping at the first saturated one) and reports, per rate, the completed throughput
    and the p50 / p99 latency from submission to completion; the record's headline is the
    highest rate that did not saturate."""
    import torch

    from paper_2502_11686_gb300 import native

    torch.cuda.set_device(0)
    o = native.ks_default_options()
    o.precision = native.KS_FP64 if precision == "fp64" else native.KS_FP32_REFINE
    ctx = native.ks_create(o)
    results = []
    rng = np.random.default_rng(2024)
    seed = 0
    for rate in rates:
        srv = native.ks_server_create(ctx, keep_factors=True)
        lat, qms, cov_lat, done_steps = [], [], [], 0
        lock = threading.Lock()
        pending = []
        stop = threading.Event()

        stuck = []
        abort = threading.Event()

        def waiter():
            # Polls every outstanding request (never blocks on one): a completed request is
            # released at once, so its memory can admit the next one; a covariance follow-up is
            # submitted when its request completes and awaited the same way.  Waiting on the
            # requests one at a time could hold a finished request's memory while its
            # predecessor's follow-up waits for memory.
            nonlocal done_steps
            live = []   # [rid, k, follow, fid]
            while not abort.is_set() and (not stop.is_set() or pending or live):
                with lock:
                    while pending:
                        live.append(list(pending.pop(0)) + [None])
                still = []
                for it in live:
                    rid, k, follow, fid = it
                    if fid is None:
                        info = native.ks_server_wait(srv, rid, 0.0)
                        if not info["done"]:
                            still.append(it)
                            continue
                        with lock:
                            lat.append(info["latency_ms"])
                            qms.append(info["queue_ms"])
                            done_steps += k
                        if follow and info["status"] == native.KS_OK:
                            it[3] = native.ks_server_covariances(srv, rid)
                            still.append(it)
                            continue
                        native.ks_server_release(srv, rid)
                    else:
                        finfo = native.ks_server_wait(srv, fid, 0.0)
                        if not finfo["done"]:
                            still.append(it)
                            continue
                        with lock:
                            cov_lat.append(finfo["latency_ms"])
                        native.ks_server_release(srv, fid)
                        native.ks_server_release(srv, rid)
                live = still
                time.sleep(0.0005)
            if live:
                stuck.append(live[0][0])

        th = threading.Thread(target=waiter, daemon=True)
        th.start()
        t0 = time.perf_counter()
        t_next = t0
        submitted = 0
        saturated = False
        while True:
            now = time.perf_counter()
            if now - t0 >= duration or stuck:
                break
            if submitted % 8 == 0 and native.ks_server_stats(srv)["queued"] > max_queue:
                saturated = True   # offered load above capacity: stop before the backlog grows
                break
            if now < t_next:
                time.sleep(min(t_next - now, 0.001))
                continue
            k = int(round(np.exp(rng.uniform(np.log(1e2), np.log(1e5)))))
            n = int(rng.choice(ns))
            rid = native.ks_server_submit_synthetic(srv, k, n, n, seed, want_cov=False)
            seed += 1
            with lock:
                pending.append((rid, k, rng.uniform() < 0.1))
            submitted += 1
            t_next += rng.exponential(1.0 / rate)
        submit_window = time.perf_counter() - t0
        log(f"serve: {rate} req/s, {submitted} submitted in {submit_window:.1f} s; draining")
        stop.set()
        th.join(timeout=WAIT_LIMIT_MS / 1e3)
        if th.is_alive():
            abort.set()
            th.join()
        if stuck:
            # A request did not complete within the limit: report it and leave the server (and
            # its scheduler thread) alone rather than wait on it.
            log(f"serve: request {stuck[0]} not done {WAIT_LIMIT_MS / 1e3:.0f} s after the last arrival")
            return {"metric": "served smoothed steps/s; p50 / p99 latency", "value": None,
                    "unit": UNIT, "error": f"request {stuck[0]} not complete "
                                           f"{WAIT_LIMIT_MS / 1e3:.0f} s after the last arrival at "
                                           f"{rate} req/s", "rates": results}
        total = time.perf_counter() - t0
        stats = native.ks_server_stats(srv)
        native.ks_server_destroy(srv)
        lat_a = np.array(lat)
        # Every submitted request completes, so the served rate is window / (window + drain) of
        # the offered one: a drain longer than 30 % of the window means the loop fell behind.
        lagged = (total - submit_window) > 0.3 * submit_window
        results.append({
            "offered_req_per_s": rate, "saturated": saturated or lagged,
            "queue_overflow": saturated, "submitted": submitted,
            "completed": len(lat),
            "submit_window_s": submit_window, "drain_s": total - submit_window,
            "throughput_steps_per_s": done_steps / total,
            "throughput_req_per_s": len(lat) / total,
            "p50_ms": float(np.percentile(lat_a, 50)) if len(lat_a) else None,
            "p99_ms": float(np.percentile(lat_a, 99)) if len(lat_a) else None,
            "p50_queue_ms": float(np.percentile(qms, 50)) if qms else None,
            "cov_followups": len(cov_lat),
            "p99_cov_ms": float(np.percentile(cov_lat, 99)) if cov_lat else None,
            "ticks": stats["ticks"], "launches": stats["launches"],
            "shared_launches": stats["shared_launches"],
            "max_requests_per_launch": stats["max_requests_per_launch"]})
        if verbose:
            print(json.dumps({"serve_rate": results[-1]}), flush=True)
        if saturated or lagged:
            break
    native.ks_destroy(ctx)
    ok = [r for r in results if not r["saturated"]] or results
    best = max(ok, key=lambda r: r["offered_req_per_s"])
    return {"metric": "served smoothed steps/s; p50 / p99 latency", "value":
            best["throughput_steps_per_s"], "unit": UNIT,
            "dtype": "f64" if precision == "fp64" else "f32+f64",
            "data": "synthetic (generated on the device at admission)",
            "config": {"workload": "serve: Poisson arrivals, k log-uniform [1e2, 1e5], n in "
                                   f"{ns}, m = n, 10 % covariance follow-ups",
                       "precision": precision, "duration_s_per_rate": duration,
                       "offered_req_per_s": best["offered_req_per_s"]},
            "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"],
            "saturated_at_req_per_s": next((r["offered_req_per_s"] for r in results
                                            if r["saturated"]), None),
            "rates": results}


def serve_arm(args):
    rec = serve_record(args, [float(x) for x in args.rates.split(",")], args.duration,
                       [int(x) for x in args.serve_n.split(",")], args.precision, args.max_queue)
    line = dict(rec, metric=METRIC, n_gpus=1, steps=len(rec["rates"]), warmup=0,
                higher_is_better=True, scaling="weak", vs_baseline=None)
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="long_k1e6_n6",
                    choices=sorted(WORKLOADS) + sorted(BATCH_WORKLOADS) + ["serve"])
    ap.add_argument("--nprob", type=int, default=None, help="batched workloads: problem count")
    ap.add_argument("--rates", default="25,100,400,2000",
                    help="serve workload: offered request rates (req/s) to sweep, ascending; the "
                         "sweep stops at the first saturated rate")
    ap.add_argument("--duration", type=float, default=3.0,
                    help="serve workload: seconds of arrivals per rate (each rate then drains)")
    ap.add_argument("--serve-n", default="6,24,48,128", help="serve workload: state sizes")
    ap.add_argument("--max-queue", type=int, default=32,
                    help="serve workload: a rate whose admission queue exceeds this is saturated")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_refine"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--k", type=int, default=None,
                    help="override the number of states (smaller cases for profiling)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: leave out the batched and served records")
    ap.add_argument("--batch-steps", type=int, default=3,
                    help="default line: timed steps of the batched record")
    ap.add_argument("--serve-rates", default="2,5,10",
                    help="default line: offered rates (req/s) of the served record")
    ap.add_argument("--serve-duration", type=float, default=5.0,
                    help="default line: seconds of arrivals per rate of the served record")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "serve":
        if args.impl == "reference":
            return 0
        if args.precision == "fp64" and "--precision" not in sys.argv:
            args.precision = "fp32_refine"
        return serve_arm(args)
    if args.workload in BATCH_WORKLOADS:
        if args.impl == "reference":
            return 0
        return batch_arm(args)
    wl = dict(WORKLOADS[args.workload])
    if args.k:
        wl["k"] = args.k
        wl["sample_k"] = min(wl["sample_k"], args.k)
        wl["ref_sample_k"] = min(wl["ref_sample_k"], args.k)
        wl["desc"] = wl["desc"].replace(f"k={WORKLOADS[args.workload]['k']:,}", f"k={args.k:,}")
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args, wl)

    import torch
    import torch.distributed as dist

    from paper_2502_11686_gb300 import native, problem_arrays

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    extras = (world == 1 and not args.no_extras and args.workload == "long_k1e6_n6"
              and args.k is None)
    pool, cores = (None, 1)
    if extras and not args.no_cpu_baseline:
        pool, cores = oracle_pool()   # spawn: safe beside the CUDA context

    p = make_problem(wl, seed=rank)
    k, n = p.k, p.n
    m = int(p.m[0])
    arr = problem_arrays(p, f"cuda:{local}")
    stream = torch.cuda.Stream()
    opts = native.ks_default_options()
    opts.device = local
    opts.precision = native.KS_FP64 if args.precision == "fp64" else native.KS_FP32_REFINE
    opts.stream = stream.cuda_stream
    opts.sync = 0
    opts.profile = 1
    ctx = native.ks_create(opts)
    u = torch.empty((k, n), dtype=torch.float64, device=f"cuda:{local}")
    cov = torch.empty((k, n, n), dtype=torch.float64, device=f"cuda:{local}")
    h = None

    def step(a, uo, co):
        nonlocal h
        _, h, _ = native.ks_smooth(ctx, k, n, a["m"], a["F"], a["H"], a["c"], a["K"], a["G"],
                                   a["o"], a["C"], uo, keep=True, reuse=h)
        native.ks_covariances(ctx, h, co)

    log(f"{args.workload}: {args.warmup} warm-up passes")
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(arr, u, cov)
    st, info = native.ks_sync(ctx)
    if st != native.KS_OK:
        raise native.KsError(st, native.ks_last_error(ctx), info)
    native.ks_profile_read(ctx, reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(args.steps):
                step(arr, u, cov)
            ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    st, info = native.ks_sync(ctx)
    if st != native.KS_OK:
        raise native.KsError(st, native.ks_last_error(ctx), info)
    ms = ev0.elapsed_time(ev1)
    prof = native.ks_profile_read(ctx, reset=True)
    t = torch.tensor([ms], dtype=torch.float64, device=f"cuda:{local}")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * k * args.steps / (ms_max / 1e3)
    log(f"{args.workload}: {args.steps} timed passes, {ms_max / args.steps:.3f} ms each")

    # End to end through the same C ABI with pinned host buffers: every step copies its
    # inputs in and its states and covariances out inside the timed region.
    e2e = None
    if not args.no_e2e:
        harr = {nm: (torch.from_numpy(np.ascontiguousarray(getattr(p, nm))).pin_memory()
                     if getattr(p, nm) is not None and nm != "m" else getattr(p, nm))
                for nm in ("m", "F", "H", "c", "K", "G", "o", "C")}
        hu = torch.empty((k, n), dtype=torch.float64).pin_memory()
        hc = torch.empty((k, n, n), dtype=torch.float64).pin_memory()
        e_steps = max(3, min(args.steps, 10))
        with torch.cuda.stream(stream):
            step(harr, hu, hc)
            step(harr, hu, hc)
            native.ks_sync(ctx)
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(e_steps):
                step(harr, hu, hc)
            st, info = native.ks_sync(ctx)
            torch.cuda.synchronize()
            e_wall = time.perf_counter() - t0
        if st != native.KS_OK:
            raise native.KsError(st, native.ks_last_error(ctx), info)
        e_ms = torch.tensor([e_wall * 1e3], dtype=torch.float64, device=f"cuda:{local}")
        if world > 1:
            dist.all_reduce(e_ms, op=dist.ReduceOp.MAX)
        in_bytes = sum(int(v.numel() * v.element_size()) for nm, v in harr.items()
                       if v is not None and nm != "m") + int(p.m.nbytes)
        e2e = {"value": world * k * e_steps / (float(e_ms.item()) / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": in_bytes,
               "d2h_bytes_per_step": int(hu.numel() * 8 + hc.numel() * 8),
               "steps": e_steps, "timing": "wall clock, device synchronized on both sides; "
                                           "the input copy of a call overlaps the previous "
                                           "call's kernels"}
        native.ks_profile_read(ctx, reset=True)
        log(f"{args.workload}: end to end {e_wall * 1e3 / e_steps:.3f} ms per pass")

    if h is not None:
        native.ks_release(ctx, h)
    native.ks_destroy(ctx)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    fl = flops_per_step(n, m, args.precision)
    by = bytes_per_step(n, m, args.precision)
    phase_ms = {ph: v / args.steps for ph, v in prof["phase_ms"].items() if v > 0}
    top = max(("whiten", "level", "backsub", "selinv", "refine"), key=lambda ph: phase_ms.get(ph, 0))
    fp64_phase = args.precision == "fp64" or top in ("whiten", "refine")
    roof = alu_roofline(f"{top} phase", fl[top] * k, phase_ms[top], fp64_phase, local)
    roof.update({"flops_per_step": fl[top], "hbm_bytes_per_step": by[top],
                 "achieved_hbm_gbs": by[top] * k / (phase_ms[top] / 1e3) / 1e9})
    tr = measured_traffic(top, args.precision, n)
    if tr is not None and top == "level":
        launches = max(1, prof["phase_launches"]["level"] // args.steps)
        roof["traffic"] = tr["dram_bytes_per_tile"] * (k - 1) / launches
        roof["traffic_unit"] = "bytes per launch (average over the level launches of a pass)"
        roof["traffic_source"] = tr["capture"]
        roof["algorithmic_bytes_per_launch"] = by[top] * k / launches
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        log(f"{args.workload}: CPU baseline (oracle, 1 host core)")
        rate, sample = oracle_rate(wl)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm_peak = peaks.get("hbm_gbs")
    except (OSError, ValueError):
        hbm_peak = 6800.0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {wl['desc']}", "k": k, "n": n, "m": m,
                   "precision": args.precision,
                   "l2": f"inputs ({p.input_bytes() / 1e9:.2f} GB) larger than L2 (129 MB), no flush",
                   "parallelism": "replicas only (one independent problem per GPU)"},
        "roofline": roof,
        "hbm_frac_of_measured": roof["achieved_hbm_gbs"] / hbm_peak if hbm_peak else None,
        "phase_ms_per_step": phase_ms,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": prof["launches"],
        "clocks": clk.summary(),
    }
    if extras:
        line["fp32_refine_batched"] = batch_record(args, BATCH_WORKLOADS["batch_c4"]["nprob"],
                                                   "fp32_refine", pool, cores,
                                                   steps=args.batch_steps, warmup=3)
        log("served record")
        line["serve"] = serve_record(args, [float(x) for x in args.serve_rates.split(",")],
                                     args.serve_duration, [6, 24, 48, 128], "fp32_refine",
                                     args.max_queue, verbose=False)
    if pool is not None:
        pool.terminate()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
