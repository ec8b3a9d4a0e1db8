#!/usr/bin/env python3
"""Benchmark of the Sketched Leverage Score Ordering hot path on one GB300 (or N replicas).

One step = slso_leverage (sketch -> FP64 QR -> certified R^-1 or SVD -> M -> scores) followed by
slso_order (radix argsort into the "dec" order) over the whole matrix, X already resident in HBM.
Workload: X 1,000,000 x 1024 float32 (rank-200 signal + noise at SNR 10, Student-t(3) row
scaling), CountSketch s = 16384, JL width k = 128.  X (4.1 GB) is larger than L2, so no flush is
needed between steps.

Printed: one JSON line (rank 0).  `value` is scored rows/s of the float32 path over all ranks;
the bfloat16 path, the end-to-end host-buffer call, per-stage times, the roofline of the dominant
kernel, clocks, precision against the FP64 oracle and the oracle's own CPU throughput ride along.

--impl reference times the FP64 CPU oracle instead (the only reference this method has), on a
bounded sample of the same workload per step, scaled to rows/s.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "scored rows/s (BF16 vs FP32, ≤2% median rel err) + roofline %; p99 job latency"
WORKLOAD = dict(n=1_000_000, d=1024, s=16384, k=128, kind="countsketch", xseed=1003, seed_S=2003, seed_Pi=3003)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070 / 1e3  # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz = 1.26
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070 / 1e3
# float-float multiply-add (TwoProd by FMA, TwoSum and the renormalisation): about 12 float32
# instructions, so the float32 pipe's issue rate bounds float-float work at this many TFLOP/s
FF_PEAK_TFLOPS = 152 * 128 * 2.070 / 12 * 2 / 1e3
# bfloat16 digit products of the exact Gram split: 8 digits a column, the 36 pairs (p, q) with
# p + q <= 7 (a symmetric pair counted once per product)
GRAM_DIGIT_PRODUCTS = 36
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of each stage's kernel on the
# 1,000,000 x 1024 workload (s = 16384, k = 128), from one ncu capture of its current source; None
# whenever the kernel changed since, until it is captured again.
# scores: captured on 131072 rows (X read once), scaled by 10^6 / 131072 rows; syrk (gram_tc_kernel)
# and chol (chol_ff_kernel): the sketch and the solve do not depend on n (s = 16384, d = 1024 in both).
TRAFFIC_BYTES = {"scores": 4_153_843_750, "sketch": None, "syrk": 272_007_936, "chol": 6_848_000}
CORRECT_FRAC = 0.015  # rescore the top 1.5% rows in float32 (1% target plus margin)
OSNAP_NNZ = 4  # nonzeros per column of the OSNAP sketch
STREAM_BLOCK = 262144  # rows per block of the out-of-core entry point


def stage_rooflines(per, n, d, s, k, peaks, peak_src):
    """Roofline of each timed stage's dominant kernel on the n x d float32 step (k = JL width):
    algorithmic bytes or flops per call over the stage's CUDA-event time."""
    out = {}
    full = (n, d, s, k) == (WORKLOAD["n"], WORKLOAD["d"], WORKLOAD["s"], WORKLOAD["k"])
    tr = (lambda nm: TRAFFIC_BYTES.get(nm)) if full else (lambda nm: None)
    hbm = peaks["hbm_gbs"]
    if "scores" in per:  # X read once, l written; Y = X M never leaves the SM
        b = n * d * 4.0 + n * 4.0
        a = b / (per["scores"] / 1e3) / 1e9
        out["scores"] = {"kernel": "score_tm_kernel (X M on tcgen05: tf32 products from X's raw tile, bf16 pieces in TMEM; row norms)", "bound": "hbm",
                         "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm, "traffic": tr("scores"),
                         "algorithmic": b, "peak_source": peak_src, "ms": per["scores"]}
    if "sketch" in per:  # X read once, SX (float64) written once
        b = n * d * 4.0 + s * d * 8.0
        a = b / (per["sketch"] / 1e3) / 1e9
        out["sketch"] = {"kernel": "cs_gather_kernel (CountSketch bucket sums + FP8 column maxima)", "bound": "hbm",
                         "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm, "traffic": tr("sketch"),
                         "algorithmic": b, "peak_source": peak_src, "ms": per["sketch"]}
    if "syrk" in per:  # 36 bf16 digit SYRKs over the lower triangle, 2 flops a multiply-add
        f = GRAM_DIGIT_PRODUCTS * float(s) * d * (d + 1)
        a = f / (per["syrk"] / 1e3) / 1e12
        pk = peaks["bf16_tflops_sustained"]
        out["syrk"] = {"kernel": "gram_tc_kernel (exact G = SX^T SX from bfloat16 digits on tcgen05)",
                       "bound": "tensor", "achieved": a, "peak": pk, "unit": "TFLOP/s", "frac": a / pk,
                       "traffic": tr("syrk"), "algorithmic": f, "peak_source": peak_src + " (bf16 sustained)",
                       "ms": per["syrk"]}
    if "chol" in per:  # Cholesky d^3/3 + triangular inverse d^3/3 + M and probes d^2 (k + 4), float-float
        f = 2.0 * d ** 3 / 3.0 + d * d * (k + 4.0)
        a = f / (per["chol"] / 1e3) / 1e12
        out["chol"] = {"kernel": "chol_ff_kernel (float-float Cholesky, R^-1, M in one cooperative launch)",
                       "bound": "alu", "achieved": a, "peak": FF_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "frac": a / FF_PEAK_TFLOPS, "traffic": tr("chol"), "algorithmic": f,
                       "peak_source": "derived: 152 SM x 128 FP32 lanes x 2.07 GHz / 12 instructions per "
                                      "float-float multiply-add x 2 flops", "ms": per["chol"]}
    if "qr" in per and per["qr"] > 0.01:
        f = 2.0 * s * d * d - 2.0 * d ** 3 / 3.0
        a = f / (per["qr"] / 1e3) / 1e12
        out["qr"] = {"kernel": "qr_kernel (FP64 Householder, cooperative)", "bound": "alu", "achieved": a,
                     "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": a / FP64_PEAK_TFLOPS, "traffic": None,
                     "algorithmic": f, "peak_source": "derived: 152 SM x 2 FP64 FMA/clk x 2.07 GHz",
                     "ms": per["qr"]}
    if "order" in per:  # scores read, 64-bit order written, one 32-bit key pass per radix digit pass
        b = n * 4.0 + n * 8.0
        a = b / (per["order"] / 1e3) / 1e9
        out["order"] = {"kernel": "radix order (key/index passes)", "bound": "hbm", "achieved": a, "peak": hbm,
                        "unit": "GB/s", "frac": a / hbm, "traffic": None, "algorithmic": b,
                        "peak_source": peak_src, "ms": per["order"]}
    return out


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def _config(n, d, s, k, kind):
    return {
        "workload": f"snr_student_t {n}x{d} float32 (rank-200 + SNR 10 noise, t(3) rows), "
                    f"{kind} s={s}, JL k={k}; leverage + dec order",
        "n": n, "d": d, "s": s, "k": k, "sketch": kind,
        "l2": "inputs larger than L2 (X is 4.1 GB > 129 MB); no flush",
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle timing
def oracle_job(Xn, kind, s, k, seed_S, seed_Pi):
    """One whole sketched-score job of the FP64 oracle (Oracle B, the same S and Pi as the GPU), timed:
    sketch, R by LAPACK's QR, SVD of R, M, all row scores, then the "dec" order.  Returns
    (scores, oracle_rank, seconds for the scores, seconds for the order)."""
    from oracle import slso_oracle as O

    t0 = time.perf_counter()
    SX = O.sketch(Xn, kind, s, seed_S)
    sv = O.sketched_svd(SX, qr="lapack")
    M = O.m_matrix(sv["sigma"], sv["V"], sv["U_R"], sv["rank"], O.jl_matrix(Xn.shape[1], k, seed_Pi) if k else None)
    want = O.row_scores(Xn, M)
    t1 = time.perf_counter()
    O.order_dec(want)
    t2 = time.perf_counter()
    return want, sv["rank"], t1 - t0, t2 - t1


def oracle_exact_seconds(Xn):
    """Oracle A (exact scores, the hat-matrix diagonal from R of X by blocked QR and its SVD) on all rows of Xn."""
    import numpy as np

    from oracle import slso_oracle as O

    t0 = time.perf_counter()
    O.exact_leverage_rows(Xn, np.arange(Xn.shape[0]))
    return time.perf_counter() - t0


ONE_THREAD_CODE = r"""
import os, sys, json, time
for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
    os.environ[v] = "1"
sys.path.insert(0, sys.argv[1])
import numpy as np
import bench
from paper_1812_07903_gb300 import inputs
a = json.loads(sys.argv[2])
X = inputs.snr_student_t(a["n"], a["d"], seed=a["xseed"], device="cpu").numpy()
_, _, t_sc, t_od = bench.oracle_job(X, a["kind"], a["s"], a["k"], a["seed_S"], a["seed_Pi"])
print(json.dumps({"seconds": t_sc + t_od}))
"""


def oracle_one_thread(n, d, s, k, kind, seed_S, seed_Pi, xseed):
    """The same whole job on n rows with the BLAS limited to one thread (a child process, so that the
    thread limits are set before numpy loads its BLAS)."""
    import subprocess

    args = json.dumps({"n": n, "d": d, "s": s, "k": k, "kind": kind, "seed_S": seed_S, "seed_Pi": seed_Pi,
                       "xseed": xseed})
    r = subprocess.run([sys.executable, "-c", ONE_THREAD_CODE, ROOT, args], capture_output=True, text=True,
                       timeout=900)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])["seconds"]


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


REF_ROWS = 65536  # the reference arm's bounded sample: a whole job on the first rows of the workload


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    W = WORKLOAD
    n, d, s, k = W["n"], W["d"], W["s"], W["k"]
    from paper_1812_07903_gb300 import inputs

    Xn = inputs.snr_student_t(REF_ROWS, d, seed=W["xseed"], device="cpu").numpy()
    secs = []
    for it in range(args.warmup + args.steps):
        _, _, t_sc, t_od = oracle_job(Xn, W["kind"], s, k, W["seed_S"], W["seed_Pi"])
        if it >= args.warmup:
            secs.append(t_sc + t_od)
    t = statistics.median(secs)
    v = REF_ROWS / t
    sample = (f"whole sketched-score job (sketch, LAPACK QR, SVD of R, M, scores, dec order) on {REF_ROWS} rows "
              f"of the {n}-row workload, measured per step; the s x d factor does not shrink with the sample")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "rows/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(n, d, s, k, W["kind"]),
        "cpu_baseline": {"value": v, "unit": "rows/s", "cores": host_cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- serving
def serving_bench(api, inputs, torch, n_jobs, slots=4, load=0.7, seed=4004):
    """Poisson trace of mixed leverage jobs through slso_server at `load` x one-at-a-time capacity.

    Jobs: n = round(2^U[12,20]), d from {64,128,256,300,784}, 8-cluster Gaussian-mixture rows,
    sketch kind 1/3 each, k = 64.  Capacity is calibrated by running the first 16 jobs one at a time
    through the direct entry points; arrivals are then Poisson at `load` x that rate.
    """
    import numpy as np

    jobs = inputs.serving_jobs(n_jobs=n_jobs, seed=seed, rate_per_s=1.0)
    # every job's rows are a window of a per-width pool of mixture rows (seeded offset), so that the
    # trace fits the device whatever its length
    pools = {}
    gen = np.random.default_rng(seed + 1)
    pool_rows = 2 << 20
    for jb in jobs:
        if jb["d"] not in pools:
            pools[jb["d"]] = inputs.gaussian_mixture(pool_rows, jb["d"], seed=20000 + jb["d"], device="cuda")
        off = int(gen.integers(0, pool_rows - jb["n"] + 1))
        jb["X"] = pools[jb["d"]][off: off + jb["n"]]
    torch.cuda.synchronize()
    calib = jobs[: min(16, n_jobs)]
    for jb in calib[:2]:  # warm-up
        api.leverage(jb["X"], jb["kind"], jb["s"], jb["k"], jb["seed"], jb["seed"] + 1, want_info=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for jb in calib:
        sc, _ = api.leverage(jb["X"], jb["kind"], jb["s"], jb["k"], jb["seed"], jb["seed"] + 1, want_info=False)
        api.order(sc)
        torch.cuda.synchronize()
    service_s = (time.perf_counter() - t0) / len(calib)
    rate = load / service_s
    gaps = [jobs[0]["arrival_s"]] + [b["arrival_s"] - a["arrival_s"] for a, b in zip(jobs, jobs[1:])]
    srv = api.Server(slots=slots, mem_budget_bytes=24 << 30)
    tickets = []
    start = time.perf_counter()
    t_arr = 0.0
    for jb, g in zip(jobs, gaps):
        t_arr += g / rate  # inter-arrival gaps of the unit-rate trace, rescaled
        delay = start + t_arr - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.submit_leverage(jb["X"], jb["kind"], jb["s"], jb["k"], jb["seed"], jb["seed"] + 1))
    lat, bad = [], 0
    for t in tickets:
        st, info, times, _ = srv.poll(t, timeout_ms=600000)
        bad += st != 0
        lat.append(times[2])
    makespan = time.perf_counter() - start
    counters = srv.counters()
    srv.close()
    # each job's own service time, run alone through the direct entry points: the slowdown
    # (latency in the trace / time alone) separates queueing from the spread of job sizes
    alone = []
    for jb in jobs:
        t1 = time.perf_counter()
        sc, _ = api.leverage(jb["X"], jb["kind"], jb["s"], jb["k"], jb["seed"], jb["seed"] + 1, want_info=False)
        api.order(sc)
        torch.cuda.synchronize()
        alone.append((time.perf_counter() - t1) * 1e3)
    slow = sorted(l_ / a for l_, a in zip(lat, alone))
    lat.sort()
    pct = lambda q: lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]  # noqa: E731
    rows = sum(jb["n"] for jb in jobs)
    return {
        "workload": f"{n_jobs} jobs, Poisson arrivals at {load} x calibrated capacity, n=2^U[12,20], "
                    "d in {64,128,256,300,784}, rows a seeded window of a per-d pool of 8-cluster mixture rows, "
                    "CountSketch/SRHT/Gaussian 1/3 each, k=64",
        "slots": slots, "jobs": n_jobs, "failed": bad, "calibrated_service_ms": service_s * 1e3,
        "arrival_rate_per_s": rate, "p50_ms": pct(0.50), "p99_ms": pct(0.99), "max_ms": lat[-1],
        "slowdown": {"p50": slow[len(slow) // 2], "p99": slow[min(len(slow) - 1, int(math.ceil(0.99 * len(slow))) - 1)],
                     "max": slow[-1], "alone_p50_ms": sorted(alone)[len(alone) // 2],
                     "alone_p99_ms": sorted(alone)[min(len(alone) - 1, int(math.ceil(0.99 * len(alone))) - 1)]},
        "makespan_s": makespan, "jobs_per_s": n_jobs / makespan, "rows_per_s": rows / makespan,
        "graphs": {k: counters[k] for k in ("graphs_new", "graphs_updated", "direct")},
        "grouped": {k: counters[k] for k in ("group_launches", "grouped_jobs")},
        "repeated_shape": repeated_shape_latency(api, inputs, torch),
    }


def repeated_shape_latency(api, inputs, torch, n=65536, d=256, jobs=24):
    """Latency of back-to-back jobs of one shape through a 1-slot server: the first runs direct,
    the second is captured into a CUDA graph, the rest replay it (arguments updated in place)."""
    X = [inputs.gaussian_mixture(n, d, seed=500 + i, device="cuda") for i in range(4)]
    srv = api.Server(slots=1, mem_budget_bytes=4 << 30)
    lat = []
    for i in range(jobs):
        t = srv.submit_leverage(X[i % 4], "countsketch", 4096, 64, 9, 10)
        st, info, times, _ = srv.poll(t, timeout_ms=600000)
        lat.append(times[2])
    c = srv.counters()
    srv.close()
    direct = []  # the same jobs through the direct entry points, one at a time
    for i in range(jobs):
        t0 = time.perf_counter()
        sc, _ = api.leverage(X[i % 4], "countsketch", 4096, 64, 9, 10, want_info=False)
        api.order(sc)
        torch.cuda.synchronize()
        direct.append((time.perf_counter() - t0) * 1e3)
    rest = sorted(lat[2:])
    direct = sorted(direct[2:])
    return {"workload": f"{jobs} sequential jobs, n={n}, d={d}, CountSketch s=4096, k=64, 1 slot",
            "first_ms": lat[0], "captured_ms": lat[1], "replay_p50_ms": rest[len(rest) // 2],
            "direct_call_p50_ms": direct[len(direct) // 2],
            "graphs": {k: c[k] for k in ("graphs_new", "graphs_updated", "direct")}}


# ----------------------------------------------------------------------------- large workload
LARGE = dict(n=4_000_000, d=3072, s=6144, k=256, kind="gaussian", xseed=1005, seed_S=2005, seed_Pi=3005)


def large_bench(args):
    """4M x 3072 bfloat16 rows (1% from a rank-16 subspace x 20), Gaussian sketch s = 6144 on tensor
    cores, k = 256, scores in float32 / bfloat16 / FP8; one JSON line with stage times and the
    sketch's tensor throughput."""
    import torch

    from paper_1812_07903_gb300 import api, inputs

    L = dict(LARGE)
    n = args.n if args.n != WORKLOAD["n"] else L["n"]
    d, s, k = L["d"], L["s"], L["k"]
    torch.cuda.set_device(0)
    X, _ = inputs.outlier_subspace(n, d, seed=L["xseed"], device="cuda", dtype=torch.bfloat16)
    h = api.Handle(0)
    scores = torch.empty(n, dtype=torch.float32, device="cuda")
    order = torch.empty(n, dtype=torch.int64, device="cuda")
    peaks, peak_src = _peaks()
    out = {"config": {"workload": f"outlier_subspace {n}x{d} bfloat16 (1% rank-16 rows x 20), gaussian s={s} "
                                  f"(tensor cores), JL k={k}; leverage + dec order", "n": n, "d": d, "s": s, "k": k,
                      "sketch": "gaussian", "l2": "X larger than L2; no flush"},
           "metric": "scored rows/s", "unit": "rows/s", "steps": args.steps, "warmup": args.warmup}
    ref = None  # the float32-accurate scores: the precision ladder's reference at this size
    top = max(1, n // 100)
    for compute, corr in (("f32", 0.0), ("bf16", 0.0), ("bf16", CORRECT_FRAC), ("fp8", 0.0), ("fp8", CORRECT_FRAC)):
        def step():
            api.leverage(X, "gaussian", s, k, L["seed_S"], L["seed_Pi"], compute=compute, out=scores,
                         want_info=False, handle=h, correct_frac=corr)
            api.order(scores, out=order, handle=h)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        api.profile(True, handle=h)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            step()
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        stages, launches = api.profile_read(handle=h)
        api.profile(False, handle=h)
        per = {nm: v_ / args.steps for nm, (v_, c) in stages.items() if c}
        tf = 2.0 * s * n * d / (per["sketch"] / 1e3) / 1e12
        line = {"value": n / (ms / 1e3), "ms_per_step": ms, "gpu_launches": int(launches),
                "stages_ms_per_step": {nm: round(v_, 3) for nm, v_ in per.items()},
                "sketch_tensor_tflops": tf,
                "sketch_frac_of_bf16_peak": tf / peaks["bf16_tflops_sustained"],
                "peak": {"bf16_tflops_sustained": peaks["bf16_tflops_sustained"], "source": peak_src}}
        if ref is None:
            ref = scores.double().clone()
            ref_top = set(torch.topk(ref, top).indices.cpu().tolist())
        else:
            rel = ((scores.double() - ref).abs() / ref.abs().clamp_min(1e-300))
            got_top = set(torch.topk(scores.double(), top).indices.cpu().tolist())
            line["vs_float32_path"] = {"median_rel_err": float(rel.median()), "max_rel_err": float(rel.max()),
                                       "top1pct_overlap": len(ref_top & got_top) / top}
        out[compute + ("_corrected" if corr else "")] = line
    print(json.dumps(out))


SHAPES = {
    # the paper's SST sentence matrix (56 steps x 300-d word vectors) and CMU-MOSI early-fusion
    # matrix (325 features per step, d = 9750 as printed); synthetic rows of those layouts
    "text": dict(n=131072, d=16800, s=32768, k=128, gen="text_sequences", xseed=1006, seed_S=2006, seed_Pi=3006,
                 desc="text_sequences 131072x16800 float32 (SST-shaped: 56 steps x 300-d word vectors, Zipf "
                      "words, left zero padding)"),
    "multimodal": dict(n=131072, d=9750, s=16384, k=128, gen="multimodal_sequences", xseed=1007, seed_S=2007,
                       seed_Pi=3007, desc="multimodal_sequences 131072x9750 float32 (CMU-MOSI-shaped: 325 "
                                          "early-fused features per step, d = 9750)"),
}


def shape_bench(args, name):
    """The paper's text- and multimodal-shaped feature matrices: CountSketch leverage + dec order in
    float32 and bfloat16; one JSON line with stage times and the Gram product's tensor rate."""
    import torch

    from paper_1812_07903_gb300 import api, inputs

    W = SHAPES[name]
    n = args.n if args.n != WORKLOAD["n"] else W["n"]
    d, s, k = W["d"], W["s"], W["k"]
    torch.cuda.set_device(0)
    X = getattr(inputs, W["gen"])(n, seed=W["xseed"], device="cuda")
    h = api.Handle(0)
    scores = torch.empty(n, dtype=torch.float32, device="cuda")
    order = torch.empty(n, dtype=torch.int64, device="cuda")
    peaks, peak_src = _peaks()
    out = {"config": {"workload": W["desc"] + f", countsketch s={s}, JL k={k}; leverage + dec order", "n": n, "d": d,
                      "s": s, "k": k, "sketch": "countsketch", "l2": "X larger than L2; no flush"},
           "metric": "scored rows/s", "unit": "rows/s", "steps": args.steps, "warmup": args.warmup}
    for compute in ("f32", "bf16"):
        def step(info=False):
            r = api.leverage(X, "countsketch", s, k, W["seed_S"], W["seed_Pi"], compute=compute, out=scores,
                             want_info=info, handle=h)
            api.order(scores, out=order, handle=h)
            return r
        _, info = step(True)
        for _ in range(max(0, args.warmup - 1)):
            step()
        torch.cuda.synchronize()
        api.profile(True, handle=h)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            step()
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        stages, launches = api.profile_read(handle=h)
        api.profile(False, handle=h)
        per = {nm: v_ / args.steps for nm, (v_, c) in stages.items() if c}
        # the Gram product: 36 digit products over the 128 x 64 tiles of the lower triangle
        nbi, nbj = -(-d // 128), -(-d // 64)
        tiles = sum(min(2 * i + 2, nbj) for i in range(nbi))
        digit_flops = 36.0 * tiles * 128 * 64 * 2.0 * s
        syrk_ms = per.get("syrk", float("nan"))
        out[compute] = {"value": n / (ms / 1e3), "ms_per_step": ms, "gpu_launches": int(launches),
                        "stages_ms_per_step": {nm: round(v_, 3) for nm, v_ in per.items()},
                        "gram_route": info["gram_route"], "gram_resid": info["gram_resid"], "rank": info["rank"],
                        "gram_digit_tflops": digit_flops / (syrk_ms / 1e3) / 1e12,
                        "gram_frac_of_bf16_peak": digit_flops / (syrk_ms / 1e3) / 1e12 / peaks["bf16_tflops"],
                        "peak": {"bf16_tflops": peaks["bf16_tflops"], "source": peak_src}}
    print(json.dumps(out))


IMAGE = dict(n=60000, d=784, k=64, xseed=1002, seed_S=2002, seed_Pi=3002,
             kinds=(("srht", 2048), ("countsketch", 8192)))


def image_bench(args):
    """The MNIST-shaped image matrix (60000 x 784, 68 zero columns, rank 716): the SRHT (s = 2048,
    padded to 65536 rows) and CountSketch (s = 8192) sketches alone and the whole leverage + dec
    order in float32; one JSON line with the sketch's achieved HBM rate."""
    import torch

    from paper_1812_07903_gb300 import api, inputs

    W = IMAGE
    n, d, k = W["n"], W["d"], W["k"]
    torch.cuda.set_device(0)
    X, _ = inputs.image_like(n, d, seed=W["xseed"], device="cuda")
    h = api.Handle(0)
    scores = torch.empty(n, dtype=torch.float32, device="cuda")
    order = torch.empty(n, dtype=torch.int64, device="cuda")
    peaks, peak_src = _peaks()
    out = {"config": {"workload": f"image_like {n}x{d} float32 (MNIST-shaped: uint8/255 pixels, rank-50 "
                                  "structure + noise, 68 zero columns); leverage + dec order, JL k=64",
                      "n": n, "d": d, "k": k, "l2": "X (188 MB) larger than L2; no flush"},
           "metric": "scored rows/s", "unit": "rows/s", "steps": args.steps, "warmup": args.warmup}

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        api.profile(True, handle=h)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.steps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        stages, launches = api.profile_read(handle=h)
        api.profile(False, handle=h)
        return e0.elapsed_time(e1) / args.steps, stages, launches

    for kind, s in W["kinds"]:
        ms_sk, _, l_sk = timed(lambda: api.sketch(X, kind, s, W["seed_S"], handle=h))
        _, info = api.leverage(X, kind, s, k, W["seed_S"], W["seed_Pi"], compute="f32", out=scores, handle=h)

        def step():
            api.leverage(X, kind, s, k, W["seed_S"], W["seed_Pi"], compute="f32", out=scores, want_info=False,
                         handle=h)
            api.order(scores, out=order, handle=h)
        ms, stages, launches = timed(step)
        xbytes = n * d * 4.0
        out[kind] = {"s": s, "sketch_ms": ms_sk, "sketch_launches_per_call": l_sk / args.steps,
                     "sketch_x_read_gbs": xbytes / (ms_sk / 1e3) / 1e9,
                     "sketch_frac_of_hbm": xbytes / (ms_sk / 1e3) / 1e9 / peaks["hbm_gbs"],
                     "value": n / (ms / 1e3), "ms_per_step": ms, "gpu_launches": int(launches),
                     "stages_ms_per_step": {nm: round(v_ / args.steps, 4) for nm, (v_, c) in stages.items() if c},
                     "rank": info["rank"], "svd_route": info["svd_route"], "gram_route": info["gram_route"]}
    out["peak"] = {"hbm_gbs": peaks["hbm_gbs"], "source": peak_src}
    print(json.dumps(out))


# ----------------------------------------------------------------------------- GPU arm
def max_over_ranks(ms, world, device):
    """The slowest rank's time: every rank of an N-rank run gets the same value (weak scaling times
    the whole job by its slowest replica)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rows_per_s(n_per_rank, world, ms):
    """Whole-job throughput: every rank scores its own n rows per step, the step takes ms."""
    return world * n_per_rank / (ms / 1e3)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=WORKLOAD["n"])
    ap.add_argument("--no-precision", action="store_true", help="skip the FP64 oracle comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--serving-jobs", type=int, default=512, help="jobs in the serving trace (0 skips it)")
    ap.add_argument("--config", default="benchmark", choices=["benchmark", "large", "text", "multimodal", "image"],
                    help="large: the 4M x 3072 bfloat16 Gaussian-sketch workload; text / multimodal: the SST- and "
                         "CMU-MOSI-shaped matrices (each its own JSON line)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "large":
        return large_bench(args)
    if args.config in SHAPES:
        return shape_bench(args, args.config)
    if args.config == "image":
        return image_bench(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1812_07903_gb300 import api, inputs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    W = dict(WORKLOAD)
    n, d, s, k, kind = args.n, W["d"], W["s"], W["k"], W["kind"]
    X = inputs.snr_student_t(n, d, seed=W["xseed"] + rank, device="cuda")
    h = api.Handle(local)
    scores = torch.empty(n, dtype=torch.float32, device="cuda")
    scores_bf = torch.empty(n, dtype=torch.float32, device="cuda")
    order = torch.empty(n, dtype=torch.int64, device="cuda")

    def step(compute, out, correct=0.0):
        api.leverage(X, kind, s, k, W["seed_S"], W["seed_Pi"], compute=compute, correct_frac=correct, out=out,
                     want_info=False, handle=h)
        api.order(out, out=order, handle=h)

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(compute, out, steps, clocks=False, correct=0.0):
        for _ in range(args.warmup):
            step(compute, out, correct)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if clocks else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        api.profile(True, handle=h)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            step(compute, out, correct)
        e1.record(st)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        stages, launches = api.profile_read(handle=h)
        api.profile(False, handle=h)
        clk = sampler.stop() if sampler else None
        return max_over_ranks(ms, world, "cuda"), stages, launches, clk

    ms32, stages32, launches32, clk = timed("f32", scores, args.steps, clocks=True)
    ms16, stages16, _, _ = timed("bf16", scores_bf, args.steps)
    scores_bc = torch.empty(n, dtype=torch.float32, device="cuda")
    msbc, stagesbc, _, _ = timed("bf16", scores_bc, args.steps, correct=CORRECT_FRAC)
    scores_f8 = torch.empty(n, dtype=torch.float32, device="cuda")
    ms8, stages8, _, _ = timed("fp8", scores_f8, args.steps)
    scores_f8c = torch.empty(n, dtype=torch.float32, device="cuda")
    ms8c, stages8c, _, _ = timed("fp8", scores_f8c, args.steps, correct=CORRECT_FRAC)
    _, info = api.leverage(X, kind, s, k, W["seed_S"], W["seed_Pi"], compute="f32", out=scores, handle=h)

    value = job_rows_per_s(n, world, ms32)
    value16 = job_rows_per_s(n, world, ms16)
    peaks, peak_src = _peaks()

    # ---- roofline of every stage's kernel, and the dominant one
    per = {name: ms_ / args.steps for name, (ms_, c) in stages32.items() if c}
    roofs = stage_rooflines(per, n, d, s, k, peaks, peak_src)
    dom = max(roofs, key=lambda nm: roofs[nm]["ms"])
    roof = dict(roofs[dom])

    line = {
        "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": _config(n, d, s, k, kind),
        "roofline": roof, "stage_rooflines": roofs, "gpu_launches": int(launches32),
        "stages_ms_per_step": {nm: round(v_ / args.steps, 4) for nm, (v_, c) in stages32.items() if c},
        "bf16": {"value": value16, "unit": "rows/s", "ms_per_step": ms16,
                 "stages_ms_per_step": {nm: round(v_ / args.steps, 4) for nm, (v_, c) in stages16.items() if c}},
        "bf16_corrected": {"value": job_rows_per_s(n, world, msbc), "unit": "rows/s", "ms_per_step": msbc,
                           "correct_frac": CORRECT_FRAC,
                           "stages_ms_per_step": {nm: round(v_ / args.steps, 4) for nm, (v_, c) in stagesbc.items() if c}},
        "fp8": {"value": job_rows_per_s(n, world, ms8), "unit": "rows/s", "ms_per_step": ms8,
                "stages_ms_per_step": {nm: round(v_ / args.steps, 4) for nm, (v_, c) in stages8.items() if c}},
        "fp8_corrected": {"value": job_rows_per_s(n, world, ms8c), "unit": "rows/s", "ms_per_step": ms8c,
                          "correct_frac": CORRECT_FRAC,
                          "stages_ms_per_step": {nm: round(v_ / args.steps, 4) for nm, (v_, c) in stages8c.items() if c}},
        "solve": "G = SX^T SX exactly split into bfloat16 digits on the tensor cores; float-float Cholesky, "
                 "R^-1 and M = R^-1 Pi in one cooperative kernel; kept by a 4-probe orthogonality check "
                 "(else fp64 Householder QR)",
        "rank_info": {"rank": info["rank"], "svd_route": info["svd_route"], "score_sum": info["score_sum"],
                      "gram_route": info["gram_route"], "gram_resid": info["gram_resid"]},
        "clocks": clk,
        "hbm_floor_ms": (2 * n * d * 4 + n * 12) / (peaks["hbm_gbs"] * 1e6),
    }
    line["hbm_roofline_frac_whole_step"] = line["hbm_floor_ms"] / ms32

    # ---- approximate left singular vectors (Algorithm 2 step 3) on the same matrix
    if rank == 0:
        U = torch.empty(n, d, dtype=torch.float32, device="cuda")
        api.approx_u(X, kind, s, W["seed_S"], out=U, handle=h)
        torch.cuda.synchronize()
        api.profile(True, handle=h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(2):
            api.approx_u(X, kind, s, W["seed_S"], out=U, handle=h)
        e1.record()
        torch.cuda.synchronize()
        st_u, _ = api.profile_read(handle=h)
        api.profile(False, handle=h)
        ms_u = e0.elapsed_time(e1) / 2
        line["approx_u"] = {"value": n / (ms_u / 1e3), "unit": "rows/s", "ms_per_call": ms_u,
                            "output": f"U {n}x{d} float32 ({n * d * 4 / 1e9:.1f} GB)",
                            "stages_ms_per_call": {nm: round(v_ / 2, 3) for nm, (v_, c) in st_u.items() if c}}
        del U

    # ---- OSNAP sketch (4 nonzeros per column of S) in place of CountSketch, same step
    if rank == 0:
        scores_os = torch.empty(n, dtype=torch.float32, device="cuda")

        def osnap_step():
            api.leverage(X, "osnap", s, k, W["seed_S"], W["seed_Pi"], compute="f32", out=scores_os, want_info=False,
                         handle=h, nnz=OSNAP_NNZ)
            api.order(scores_os, out=order, handle=h)
        for _ in range(args.warmup):
            osnap_step()
        torch.cuda.synchronize()
        api.profile(True, handle=h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            osnap_step()
        e1.record()
        torch.cuda.synchronize()
        st_o, _ = api.profile_read(handle=h)
        api.profile(False, handle=h)
        ms_o = e0.elapsed_time(e1) / args.steps
        line["osnap"] = {"value": n / (ms_o / 1e3), "unit": "rows/s", "ms_per_step": ms_o, "nnz": OSNAP_NNZ,
                         "stages_ms_per_step": {nm: round(v_ / args.steps, 4) for nm, (v_, c) in st_o.items() if c}}
        del scores_os

    # ---- end to end through the host-buffer entry points
    if not args.no_e2e:
        Xh = X.cpu().pin_memory()
        ke = max(3, args.steps)
        sc_h = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(2)]
        od_h = [torch.empty(n, dtype=torch.int64).pin_memory() for _ in range(2)]
        st = torch.cuda.current_stream()

        def e2e_timed(fn):
            fn()  # warm-up
            barrier()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            return max_over_ranks(e0.elapsed_time(e1) / ke, world, "cuda")

        def single_calls():
            for i in range(ke):
                api.rank_rows_host(Xh, kind, s, k, W["seed_S"], W["seed_Pi"], compute="f32", scores_out=sc_h[i & 1],
                                   order_out=od_h[i & 1], handle=h)

        def batch_call():
            api.rank_rows_host_batch([Xh] * ke, kind, s, k, W["seed_S"], W["seed_Pi"], compute="f32",
                                     scores_out=[sc_h[i & 1] for i in range(ke)],
                                     order_out=[od_h[i & 1] for i in range(ke)], handle=h)

        def streamed_calls():
            for i in range(ke):
                api.rank_rows_streamed(Xh, kind, s, k, W["seed_S"], W["seed_Pi"], compute="f32",
                                       block_rows=STREAM_BLOCK, scores_out=sc_h[i & 1], order_out=od_h[i & 1],
                                       handle=h)

        ms_single = e2e_timed(single_calls)
        ms_e = e2e_timed(batch_call)
        ms_stream = e2e_timed(streamed_calls)
        nblk = -(-n // STREAM_BLOCK)
        reloads = max(0, nblk - 2)  # the second pass finds the last two blocks still on the device
        line["out_of_core"] = {
            "value": job_rows_per_s(n, world, ms_stream), "unit": "rows/s", "ms_per_step": ms_stream,
            "api": "slso_rank_rows_streamed: X stays in pinned host memory and is streamed through the device "
                   "twice in blocks (sketch pass, then score pass); device memory independent of n x d",
            "block_rows": STREAM_BLOCK, "blocks": nblk,
            "h2d_bytes_per_step": (n + reloads * STREAM_BLOCK) * d * 4,
            "d2h_bytes_per_step": n * (4 + 8)}
        line["e2e"] = {"value": job_rows_per_s(n, world, ms_e), "unit": "rows/s", "ms_per_step": ms_e,
                       "h2d_bytes_per_step": n * d * 4, "d2h_bytes_per_step": n * (4 + 8),
                       "api": f"slso_rank_rows_host_batch over {ke} host matrices (pinned): each step copies its X "
                              "in and its scores + order out; copies overlap the neighbouring steps' compute",
                       "single_call_ms_per_step": ms_single,
                       "single_call_value": job_rows_per_s(n, world, ms_single)}
        del Xh

    # ---- precision against the FP64 oracle, and the oracle's own measured throughput (rank 0, N = 1)
    if rank == 0 and world == 1 and not args.no_precision:
        from oracle import slso_oracle as O

        Xn = X.cpu().numpy()
        want, orank, t_or, t_od = oracle_job(Xn, kind, s, k, W["seed_S"], W["seed_Pi"])
        stats = {}
        for name, got in (("f32", scores), ("bf16", scores_bf), ("bf16_corrected", scores_bc), ("fp8", scores_f8),
                          ("fp8_corrected", scores_f8c)):
            g = got.cpu().numpy().astype(np.float64)
            pos = want > 0
            rel = np.abs(g[pos] - want[pos]) / want[pos]
            top = max(1, math.ceil(0.01 * n))
            og = set(O.order_dec(g)[:top].tolist())
            ow = set(O.order_dec(want)[:top].tolist())
            stats[name] = {"median_rel_err": float(np.median(rel)), "max_rel_err": float(np.max(rel)),
                           "top1pct_overlap": len(og & ow) / top,
                           "zero_rows": int(np.sum(~pos)), "zero_rows_nonzero_gpu": int(np.sum(g[~pos] != 0))}
        line["precision_vs_fp64_oracle"] = stats
        line["precision_vs_fp64_oracle"]["oracle_rank"] = orank
        if not args.no_cpu_baseline:
            cores = host_cores()
            rows_a = 131072
            t_a = oracle_exact_seconds(Xn[:rows_a])
            t_1 = oracle_one_thread(REF_ROWS, d, s, k, kind, W["seed_S"], W["seed_Pi"], W["xseed"])
            line["cpu_baseline"] = {
                "value": n / (t_or + t_od), "unit": "rows/s", "cores": cores, "kind": "oracle",
                "sample": f"whole job, all {n} rows, measured: sketch + LAPACK QR + SVD of R + M + scores (Oracle B, "
                          "same S and Pi) then the dec order",
                "seconds": t_or + t_od, "scores_seconds": t_or, "order_seconds": t_od,
                "exact_scores": {"kind": "oracle A (exact, blocked QR of X + SVD)", "rows": rows_a,
                                 "seconds": t_a, "rows_per_s": rows_a / t_a, "cores": cores},
                "one_thread": ({"rows": REF_ROWS, "seconds": t_1, "rows_per_s": REF_ROWS / t_1, "cores": 1,
                                "sample": f"whole job on the first {REF_ROWS} rows, BLAS on one thread"}
                               if t_1 else None),
            }
    if rank == 0 and world == 1 and args.serving_jobs > 0:
        del X
        torch.cuda.empty_cache()
        line["serving"] = serving_bench(api, inputs, torch, args.serving_jobs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
