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
FP64_PEAK_TFLOPS = 1.25      # nominal GB300 FP64 rate (no measured FP64 peak is provided)
FP32_PEAK_TFLOPS = 80.5      # 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz

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


def batch_arm(args):
    """The batched form: every step is one ks_smooth_batch call over resident inputs."""
    import torch

    import oracle
    from paper_2502_11686_gb300 import inputs, native, problem_arrays

    wl = BATCH_WORKLOADS[args.workload]
    nprob = args.nprob or wl["nprob"]
    torch.cuda.set_device(0)
    probs = inputs.uneven_batch(nprob, 0, wl["k_lo"], wl["k_hi"], wl["ns"])
    total_k = sum(p.k for p in probs)
    batch = []
    for p in probs:
        arr = problem_arrays(p, "cuda:0")
        d = dict(arr, k=p.k, n=p.n, m=np.ascontiguousarray(p.m, dtype=np.int32),
                 u_out=torch.empty((p.k, p.n), dtype=torch.float64, device="cuda:0"),
                 cov_out=torch.empty((p.k, p.n, p.n), dtype=torch.float64, device="cuda:0"))
        batch.append(d)
    stream = torch.cuda.Stream()
    prec = native.KS_FP64 if args.precision == "fp64" else native.KS_FP32_REFINE

    def make_ctx(profile):
        o = native.ks_default_options()
        o.precision = prec
        o.stream = stream.cuda_stream
        o.profile = 1 if profile else 0
        return native.ks_create(o)

    ctx = make_ctx(False)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            native.ks_smooth_batch(ctx, batch)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for _ in range(args.steps):
                native.ks_smooth_batch(ctx, batch)
            ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    prof_graph = native.ks_profile_read(ctx)
    native.ks_destroy(ctx)
    value = total_k * args.steps / (ms / 1e3)

    # One profiled pass (launches issued one by one, each timed into its phase).
    pctx = make_ctx(True)
    with torch.cuda.stream(stream):
        native.ks_smooth_batch(pctx, batch)
        native.ks_profile_read(pctx, reset=True)
        native.ks_smooth_batch(pctx, batch)
    prof = native.ks_profile_read(pctx)
    native.ks_destroy(pctx)
    phase_ms = {k: v for k, v in prof["phase_ms"].items() if v > 0 and k != "copy"}

    # The same problems one at a time in FP64 (ks_smooth + ks_covariances per problem).
    o = native.ks_default_options()
    o.stream = stream.cuda_stream
    o.sync = 0
    c64 = native.ks_create(o)
    def per_problem():
        for b in batch:
            _, h, _ = native.ks_smooth(c64, b["k"], b["n"], b["m"], b["F"], b["H"], b["c"], b["K"],
                                       b["G"], b["o"], b["C"], b["u_out"], keep=True)
            native.ks_covariances(c64, h, b["cov_out"])
            native.ks_release(c64, h)
    with torch.cuda.stream(stream):
        per_problem()
        torch.cuda.synchronize()
        ev0.record(stream)
        per_problem()
        ev1.record(stream)
    torch.cuda.synchronize()
    per_problem_fp64 = total_k / (ev0.elapsed_time(ev1) / 1e3)
    native.ks_destroy(c64)

    # Roofline of the dominant phase: algorithmic flops summed over the problems.
    flops = {ph: 0.0 for ph in ("whiten", "level", "backsub", "selinv", "refine")}
    for p in probs:
        f = flops_per_step(p.n, int(p.m[0]), args.precision)
        for ph in flops:
            flops[ph] += f[ph] * p.k
    top = max(flops, key=lambda ph: phase_ms.get(ph, 0.0))
    achieved = flops[top] / (phase_ms[top] / 1e3) / 1e12
    fp64_phase = args.precision == "fp64" or top in ("whiten", "refine")
    peak = FP64_PEAK_TFLOPS if fp64_phase else FP32_PEAK_TFLOPS
    roof = {"bound": "alu", "kernel": f"{top} phase (batched launches)", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": ("nominal FP64 rate of the GB300 (1.25 TFLOP/s)" if fp64_phase else
                            "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"),
            "traffic": None}
    cpu = None
    if not args.no_cpu_baseline:
        t0, steps, i = time.perf_counter(), 0, 0
        while time.perf_counter() - t0 < 10.0:
            p = probs[i % len(probs)]
            oracle.smooth(p)
            steps += p.k
            i += 1
        el = time.perf_counter() - t0
        cpu = {"value": steps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"the first {i} problems of the batch, one after another, states + "
                         f"covariances, {el:.1f} s"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {wl['desc']}", "problems": nprob,
                   "total_states": total_k, "precision": args.precision,
                   "l2": "inputs larger than L2, no flush",
                   "parallelism": "replicas only (independent problems)"},
        "per_problem_fp64_steps_per_s": per_problem_fp64,
        "roofline": roof, "phase_ms_per_step": phase_ms, "cpu_baseline": cpu, "e2e": None,
        "gpu_launches": prof_graph["launches"] // max(1, args.steps + args.warmup) * args.steps,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def serve_arm(args):
    """The serving loop: Poisson arrivals of synthetic requests (inputs generated on the device at
    admission), k log-uniform in [1e2, 1e5], n uniform over the served state sizes, m = n; 10 %
    of the requests get a covariance follow-up on their kept factor.  Reports per offered rate the
    completed throughput and the p50 / p99 latency from submission to completion."""
    import torch

    from paper_2502_11686_gb300 import native

    torch.cuda.set_device(0)
    o = native.ks_default_options()
    o.precision = native.KS_FP64 if args.precision == "fp64" else native.KS_FP32_REFINE
    ctx = native.ks_create(o)
    ns = [int(x) for x in args.serve_n.split(",")]
    rates = [float(x) for x in args.rates.split(",")]
    results = []
    rng = np.random.default_rng(2024)
    seed = 0
    for rate in rates:
        srv = native.ks_server_create(ctx, keep_factors=True)
        lat, qms, cov_lat, done_steps = [], [], [], 0
        lock = threading.Lock()
        pending = []
        stop = threading.Event()

        def waiter():
            nonlocal done_steps
            while not stop.is_set() or pending:
                with lock:
                    item = pending.pop(0) if pending else None
                if item is None:
                    time.sleep(0.0005)
                    continue
                rid, k, follow = item
                info = native.ks_server_wait(srv, rid)
                with lock:
                    lat.append(info["latency_ms"])
                    qms.append(info["queue_ms"])
                    done_steps += k
                if follow:
                    fid = native.ks_server_covariances(srv, rid)
                    finfo = native.ks_server_wait(srv, fid)
                    with lock:
                        cov_lat.append(finfo["latency_ms"])
                    native.ks_server_release(srv, fid)
                native.ks_server_release(srv, rid)

        th = threading.Thread(target=waiter, daemon=True)
        th.start()
        t0 = time.perf_counter()
        t_next = t0
        submitted = 0
        saturated = False
        while True:
            now = time.perf_counter()
            if now - t0 >= args.duration:
                break
            if submitted % 8 == 0 and native.ks_server_stats(srv)["queued"] > args.max_queue:
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
        stop.set()
        th.join()
        total = time.perf_counter() - t0
        stats = native.ks_server_stats(srv)
        native.ks_server_destroy(srv)
        lat_a = np.array(lat)
        results.append({
            "offered_req_per_s": rate, "saturated": saturated, "submitted": submitted,
            "completed": len(lat),
            "submit_window_s": submit_window, "drain_s": total - submit_window,
            "throughput_steps_per_s": done_steps / total,
            "throughput_req_per_s": len(lat) / total,
            "p50_ms": float(np.percentile(lat_a, 50)) if len(lat_a) else None,
            "p99_ms": float(np.percentile(lat_a, 99)) if len(lat_a) else None,
            "p50_queue_ms": float(np.percentile(qms, 50)) if qms else None,
            "cov_followups": len(cov_lat),
            "p99_cov_ms": float(np.percentile(cov_lat, 99)) if cov_lat else None,
            "ticks": stats["ticks"], "launches": stats["launches"]})
        print(json.dumps({"serve_rate": results[-1]}), flush=True)
        if saturated:
            break
    native.ks_destroy(ctx)
    best = max(results, key=lambda r: r["throughput_steps_per_s"])
    line = {"metric": METRIC, "value": best["throughput_steps_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": len(rates), "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic (generated on the device at admission)",
            "config": {"workload": "serve: Poisson arrivals, k log-uniform [1e2, 1e5], n in "
                                   f"{ns}, m = n, 10 % covariance follow-ups",
                       "precision": args.precision, "duration_s_per_rate": args.duration},
            "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"], "rates": results}
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
            native.ks_sync(ctx)
            barrier()
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(e_steps):
                step(harr, hu, hc)
            ev1.record(stream)
        torch.cuda.synchronize()
        st, info = native.ks_sync(ctx)
        if st != native.KS_OK:
            raise native.KsError(st, native.ks_last_error(ctx), info)
        e_ms = torch.tensor([ev0.elapsed_time(ev1)], dtype=torch.float64, device=f"cuda:{local}")
        if world > 1:
            dist.all_reduce(e_ms, op=dist.ReduceOp.MAX)
        in_bytes = sum(int(v.numel() * v.element_size()) for nm, v in harr.items()
                       if v is not None and nm != "m") + int(p.m.nbytes)
        e2e = {"value": world * k * e_steps / (float(e_ms.item()) / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": in_bytes,
               "d2h_bytes_per_step": int(hu.numel() * 8 + hc.numel() * 8),
               "steps": e_steps}
        native.ks_profile_read(ctx, reset=True)

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
    peak = FP64_PEAK_TFLOPS if args.precision == "fp64" else FP32_PEAK_TFLOPS
    achieved = fl[top] * k / (phase_ms[top] / 1e3) / 1e12
    roof = {"bound": "alu", "kernel": f"{top} phase", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": ("nominal FP64 rate of the GB300 (1.25 TFLOP/s), no measured FP64 peak"
                            if args.precision == "fp64" else
                            "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"),
            "flops_per_step": fl[top], "hbm_bytes_per_step": by[top],
            "achieved_hbm_gbs": by[top] * k / (phase_ms[top] / 1e3) / 1e9,
            "traffic": None}
    tr = measured_traffic(top, args.precision, n)
    if tr is not None and top == "level":
        launches = max(1, prof["phase_launches"]["level"] // args.steps)
        roof["traffic"] = tr["dram_bytes_per_tile"] * (k - 1) / launches
        roof["traffic_unit"] = "bytes per launch (average over the level launches of a pass)"
        roof["traffic_source"] = tr["capture"]
        roof["algorithmic_bytes_per_launch"] = by[top] * k / launches
    cpu = None
    if not args.no_cpu_baseline and world == 1:
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
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
