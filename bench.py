"""Benchmark: BinSketch hot path on one GB300 (or N, one process per GPU).

One step = sketch a CSR batch of n binary vectors (Definition "BinSketch") and
run the all-pairs top-k ranking by estimated Jaccard (Alg. 1-3, Experiment 2
as top-k), i.e. every row of the hot path.  The workload is the text-BoW
configuration: n = 100,000 vectors over d = 1,000,000, nnz per row log-normal
(median 200, sigma 1) clipped to [1, 5000], Zipf(1.0) columns, N = 4096,
top-50 by Jaccard.  Inputs are synthetic and seeded (per rank: seed = rank).

Prints one JSON line (rank 0).  ``value`` is pair estimates per second
(ordered pairs q != j, each scored and filtered into the fused top-k), summed
over ranks; ``e2e`` is the same through the C ABI with the CSR copied in from
pinned host memory and the top-k copied back inside the timed region.
``--impl reference`` times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
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

METRIC = ("CSR→sketch GB/s; sketch-pair estimates/s (top-k fused); "
          "query p99 at fixed MSE")
WORKLOAD = dict(workload="text-BoW all-pairs top-k", n=100_000, d=1_000_000, N=4096, k=50,
                by="js", nnz="lognormal(median 200, sigma 1) clip [1,5000]", columns="Zipf(1.0)")


def sketch_bytes(n, nnz, N):
    """Algorithmic HBM bytes of one sketch launch: indices + offsets in, sketches + counts out."""
    return 4 * nnz + 8 * (n + 1) + n * N // 8 + 4 * n


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # the sampler is running (first line printed) before the timed region starts
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.005)
            self.lines.clear()
        except OSError:
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
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def profile_traffic(files, name):
    """dram bytes per call recorded under profiles/ for the current sources (the
    kernel, and the host file that schedules its launches), else None."""
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1910_04658_gb300", "csrc", f), "rb").read())
    sha = h.hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", f"{name}.txt")
    try:
        rec = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
        if rec.get("source_sha256_16") == sha:
            return float(rec["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        pass
    return None


# ----------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on a bounded sample of the same workload
# ----------------------------------------------------------------------------

def oracle_sample(csr, N, k, budget_s):
    """Time the oracle: full sketch, then top-k for as many query rows as fit
    in budget_s; returns (pair estimates/s, sketch GB/s, rows, seconds, threads)."""
    import oracle
    t0 = time.perf_counter()
    sk, pc = oracle.sketch(csr.row_ptr, csr.col, csr.d, N, 0)
    t_sketch = time.perf_counter() - t0
    rows, t_topk, batch = 0, 0.0, min(16, csr.n)
    rng = np.random.default_rng(1)
    while t_topk < budget_s:
        q = rng.choice(csr.n, batch, replace=False)
        t0 = time.perf_counter()
        oracle.topk(sk[q], sk, N, oracle.JS, k, exclude_self=False)
        t_topk += time.perf_counter() - t0
        rows += batch
        batch = min(batch * 2, 1024, csr.n)
    pairs_per_s = rows * (csr.n - 1) / t_topk
    n = csr.n
    step_s = t_sketch + n * (t_topk / rows)
    total_pairs = n * (n - 1)
    gbs = sketch_bytes(n, csr.nnz, N) / t_sketch / 1e9
    return total_pairs / step_s, pairs_per_s, gbs, rows, t_topk + t_sketch, oracle.num_threads()


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_1910_04658_gb300 import inputs
    csr = inputs.bow_corpus(0, n=args.n)    # the corpus our arm's rank 0 sketches
    N, k = WORKLOAD["N"], WORKLOAD["k"]
    vals = []
    info = None
    timed_s = 0.0   # CPU seconds the timed steps actually ran (sketch + sampled rows)
    for step in range(args.warmup + args.steps):
        budget = 2.0 if step < args.warmup else 8.0
        res = oracle_sample(csr, N, k, budget)
        if step >= args.warmup:
            vals.append(res[0])
            info = res
            timed_s += res[4]
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pair-estimates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": (csr.n * (csr.n - 1)) / value * 1e3,
        "ms_per_step_is": "extrapolated from the sampled rows to the full step",
        "timed_s": timed_s,
        "timed_ms_per_step": timed_s / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(WORKLOAD, n=csr.n, step="oracle: full sketch + sampled top-k rows"),
        "cpu_baseline": {"kind": "oracle", "value": value, "unit": "pair-estimates/s",
                         "cores": info[5],
                         "sample": f"full sketch of {csr.n:,} rows + top-{k} of {info[3]} sampled "
                                   f"query rows per step, extrapolated to all rows"},
        "e2e": {"value": value, "unit": "pair-estimates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def run_ours(args, rank, world, dist):
    import torch

    from paper_1910_04658_gb300 import binding as B, build, inputs, sharded

    build.build()
    B.lib()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    N, k = WORKLOAD["N"], WORKLOAD["k"]
    csr = inputs.bow_corpus(seed=rank, n=args.n)
    n, nnz = csr.n, csr.nnz
    rp = torch.from_numpy(csr.row_ptr.view(np.int64)).to(dev)
    col = torch.from_numpy(csr.col.view(np.int32)).to(dev)
    sk = torch.empty((n, N // 32), dtype=torch.int32, device=dev)
    pc = torch.empty((n,), dtype=torch.int32, device=dev)
    score = torch.empty((n, k), dtype=torch.float32, device=dev)
    idx = torch.empty((n, k), dtype=torch.int32, device=dev)
    wsb = B.bs_topk_workspace_bytes(n, n, N, k)
    ws = torch.empty((max(wsb, 16),), dtype=torch.uint8, device=dev)
    use_tc, splits, topk_launches = B.bs_topk_plan(n, n, N, k, B.BS_VARIANT_AUTO, True)
    launches_per_step = 1 + topk_launches       # sketch + (re-layout, count+top-k, merge)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty((256 << 20,), dtype=torch.uint8, device=dev)   # > 129 MB L2

    def step(ev=None):
        if ev: ev[0].record(stream)
        B.bs_sketch(rp, col, n, nnz, csr.d, N, 0, sk, pc, stream)
        if ev: ev[1].record(stream)
        B.bs_topk(sk, pc, n, sk, pc, n, N, B.BS_JS, k, 1, score, idx, ws if wsb else None, wsb,
                  stream)
        if ev: ev[2].record(stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    assert B.bs_get_async_error(stream) == 0

    def barrier():
        if dist is not None:
            dist.barrier()

    # device-timed region: inputs resident; L2 flushed before every step (outside the events)
    t_sk, t_tk = [], []
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        wall0 = time.perf_counter()
        for s in range(args.steps):
            flush.zero_()
            step(evs[s])
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    barrier()
    for e in evs:
        t_sk.append(e[0].elapsed_time(e[1]) / 1e3)
        t_tk.append(e[1].elapsed_time(e[2]) / 1e3)
    step_s = [a + b for a, b in zip(t_sk, t_tk)]
    total_s = sum(step_s)
    pairs = n * (n - 1)

    # end to end through the C ABI: pinned host CSR in, top-k out, every step
    h_rp = torch.from_numpy(csr.row_ptr.view(np.int64)).pin_memory()
    h_col = torch.from_numpy(csr.col.view(np.int32)).pin_memory()
    h_score = torch.empty((n, k), dtype=torch.float32).pin_memory()
    h_idx = torch.empty((n, k), dtype=torch.int32).pin_memory()
    e2e_s = []
    for s in range(args.warmup + args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rp.copy_(h_rp, non_blocking=True)
        col.copy_(h_col, non_blocking=True)
        step()
        h_score.copy_(score, non_blocking=True)
        h_idx.copy_(idx, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if s >= args.warmup:
            e2e_s.append(e0.elapsed_time(e1) / 1e3)
    h2d = csr.row_ptr.nbytes + csr.col.nbytes
    d2h = n * k * 8

    # max over ranks, sums of units
    t_max, e2e_max = sharded.max_over_ranks([total_s, sum(e2e_s)], device=dev)
    value = world * pairs * args.steps / t_max
    e2e_value = world * pairs * args.steps / e2e_max

    # the CUDA-core (POPC) variant on the same workload, once, for comparison
    t_popc = None
    if not args.no_popc_compare:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        B.bs_topk_ex(sk, pc, n, sk, pc, n, N, B.BS_JS, k, 1, score, idx, ws if wsb else None, wsb,
                     B.BS_VARIANT_POPC, stream)
        e1.record(stream)
        e1.synchronize()
        t_popc = e0.elapsed_time(e1) / 1e3

    # roofline of the dominant kernel (the fused count + top-k launch)
    W = N // 32
    t_tk_sorted = sorted(t_tk)
    tk_mean = sum(t_tk) / len(t_tk)
    pk = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max_mhz = pk.get("sm_max_mhz", 2070.0)
    if use_tc:
        # dense 0/1 contraction on the block-scaled FP4 tensor pipe: 2 flops
        # per (pair, bit); the FP4 peak is the measured bf16 peak times the
        # nominal dense fp4/bf16 ratio 13.5 / 2.25 = 6
        flops = 2.0 * pairs * N
        bf16 = pk.get("bf16_tflops")
        peak = (bf16 if bf16 else 1900.0) * (13.5 / 2.25)
        roof = {"bound": "tensor", "kernel": "pair_tc_kernel<TOPK,JS> (tcgen05.mma kind::mxf4)",
                "achieved": flops / tk_mean / 1e12, "peak": peak, "unit": "TFLOP/s",
                "frac": flops / tk_mean / 1e12 / peak,
                "traffic": profile_traffic(("bs_tc_kernel.cuh", "bs_pairs_tc.cu"), "pair_tc_topk_traffic"),
                "peak_source": ("measured cuBLAS bf16 burst x 6 (nominal dense fp4/bf16 ratio 13.5/2.25), of measured"
                                if bf16 else "fallback 1.9 PF bf16 x 6, of fallback")}
    else:
        popc_peak = 16 * sm_count * sm_max_mhz * 1e6 / 1e12   # 16 POPC/clk/SM
        achieved = pairs * W / tk_mean / 1e12
        roof = {"bound": "alu", "kernel": "pair_kernel<TOPK,JS> (AND+POPC)",
                "achieved": achieved, "peak": popc_peak, "unit": "Tword-popc/s",
                "frac": achieved / popc_peak,
                "traffic": profile_traffic(("bs_pairs.cu",), "pair_topk_traffic"),
                "peak_source": "16 POPC/clk/SM x SMs x max SM clock (recipe units/clocks)"}
    sk_med = sorted(t_sk)[len(t_sk) // 2]
    sk_gbs = sketch_bytes(n, nnz, N) / sk_med / 1e9
    hbm_peak = pk.get("hbm_gbs", 6800.0)

    line = {
        "metric": METRIC, "value": value, "unit": "pair-estimates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32+f32",
        "data": "synthetic",
        "config": dict(WORKLOAD, n=n, l2="flushed (256 MB write) before every timed step",
                       parallelism=f"independent corpus per rank x{world}"),
        "roofline": roof,
        "components": {
            "sketch_ms_median": sk_med * 1e3, "sketch_GBps": sk_gbs,
            "sketch_frac_of_measured_hbm": sk_gbs / hbm_peak,
            "topk_ms": tk_mean * 1e3, "topk_ms_min": t_tk_sorted[0] * 1e3,
            "topk_pair_estimates_per_s": pairs / tk_mean,
            "topk_variant": "tensor cores (tcgen05)" if use_tc else "CUDA cores (POPC)",
            "topk_db_splits": splits,
            "popc_variant_topk_ms": t_popc * 1e3 if t_popc else None,
            "wall_s_timed_region": wall,
            "e2e_ms_steps": [round(x * 1e3, 3) for x in e2e_s]},
        "e2e": {"value": e2e_value, "unit": "pair-estimates/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_serving and n == WORKLOAD["n"]:
        # third leg of the metric: query p50 / p99 at fixed MSE (N = 4096, closed
        # form) against a resident 1,000,000-sketch database, Poisson arrivals at
        # 0.8 x a saturation measured on the same request mix (outside the timed region)
        del ws, flush
        torch.cuda.empty_cache()
        sat, mean_q, lat = serving_run(SERVING["db_rows"], args.serving_leg_requests, [0.8],
                                       args.slots, args.max_batch)
        st = lat[0.8]
        line["components"].update({
            "serving_p50_ms": st["p50_ms"], "serving_p99_ms": st["p99_ms"],
            "serving_qps": st["queries_per_s"], "serving_saturation_qps": sat,
            "serving_load": 0.8, "serving_requests": st["requests"],
            "serving_mean_request_queries": mean_q, "serving_db_rows": SERVING["db_rows"],
            "serving_N": SERVING["N"], "serving_k": SERVING["k"],
            "serving_fixed_mse": "N = 4096 bits, closed-form JS estimator"})
    if rank == 0 and world == 1 and not args.no_cpu_baseline and n == WORKLOAD["n"]:
        v, pps, gbs, rows, secs, thr = oracle_sample(csr, N, k, args.cpu_budget)
        line["cpu_baseline"] = {
            "value": v, "unit": "pair-estimates/s", "cores": thr, "kind": "oracle",
            "sample": f"oracle: full sketch ({gbs:.3f} GB/s) + top-{k} of {rows} sampled query "
                      f"rows vs all 100,000, extrapolated to the full step ({secs:.1f} s of CPU work)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# serving workload: a resident 1,000,000-sketch database, Poisson query stream
# ----------------------------------------------------------------------------

SERVING = dict(workload="serving: top-k against a resident sketch database", db_rows=1_000_000,
               d=1_000_000, N=4096, k=100, by="js", request_queries="log-uniform [1, 4096]",
               arrivals="Poisson")


def serving_run(db_rows, n_requests, loads, slots, max_q, seed=7):
    """Build the resident database of db_rows sketches, measure saturation
    (every request queued at t = 0), then serve a Poisson stream at each load
    (fraction of saturation).  Returns (saturation q/s, mean request size,
    {load: latency stats})."""
    import torch

    from paper_1910_04658_gb300 import binding as B, build, inputs
    from paper_1910_04658_gb300.serving import (GpuExecutor, Scheduler, SketchDB,
                                                latency_stats, poisson_requests)

    build.build()
    B.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    N, k = SERVING["N"], SERVING["k"]
    rp, col = inputs.bow_corpus_device(0, db_rows, SERVING["d"])
    db = SketchDB(rp, col, SERVING["d"], N, seed=0)
    del rp, col
    torch.cuda.synchronize()
    assert B.bs_get_async_error() == 0
    rng = np.random.default_rng(seed)
    zc = inputs.ZipfColumns(np.random.default_rng(seed + 1), SERVING["d"])
    make = lambda r, q: inputs.query_batch(r, q, zc)
    arena = 6 << 30

    def serve(reqs):
        ex = GpuExecutor(db, k=k, by="js", slots=slots, arena_bytes=arena, max_queries=max_q)
        sch = Scheduler(ex, arena_bytes=arena, slots=slots, max_batch_queries=max_q)
        t0 = time.perf_counter()
        res = sch.run(reqs)
        torch.cuda.synchronize()
        return res, time.perf_counter() - t0, sch

    # warm-up, then saturation: every request queued at t = 0
    serve(poisson_requests(rng, 12, 1e9, make))
    sat_reqs = poisson_requests(rng, n_requests, 1e9, make)
    for r in sat_reqs:
        r.arrival = 0.0
    res, wall, _ = serve(sat_reqs)
    sat_qps = sum(r.n_queries for r in sat_reqs) / wall
    mean_q = float(np.mean([r.n_queries for r in sat_reqs]))
    lines = {}
    for load in loads:
        reqs = poisson_requests(rng, n_requests, load * sat_qps / mean_q, make)
        res, wall, sch = serve(reqs)
        st = latency_stats(res, wall)
        st["batches"] = sch.batches_launched
        st["max_inflight"] = sch.max_inflight
        lines[load] = st
    assert B.bs_get_async_error() == 0
    del db
    torch.cuda.empty_cache()
    return sat_qps, mean_q, lines


def run_serving(args):
    from paper_1910_04658_gb300 import binding as B

    slots, max_q = args.slots, args.max_batch
    sat_qps, mean_q, lines = serving_run(args.db_rows, args.serving_requests, args.loads, slots, max_q)
    head = lines[0.8] if 0.8 in lines else lines[args.loads[-1]]
    line = {
        "metric": METRIC, "value": head["p99_ms"], "unit": "ms (query p99 at 0.8 x saturation)",
        "n_gpus": 1, "steps": args.serving_requests, "warmup": 12,
        "ms_per_step": head["mean_ms"], "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32+f32", "data": "synthetic",
        "config": dict(SERVING, db_rows=args.db_rows, slots=slots, max_batch_queries=max_q,
                       fixed_mse="N = 4096, closed-form estimator"),
        "components": {"saturation_queries_per_s": sat_qps, "mean_request_queries": mean_q,
                       "loads": {str(kk): v for kk, v in lines.items()}},
        "e2e": {"value": head["p99_ms"], "unit": "ms", "h2d_bytes_per_step": None,
                "d2h_bytes_per_step": None,
                "note": "latency is end to end: pinned-host CSR in, top-k back on the host"},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# batched workload: 64 independent datasets, autotuned, one graph launch
# ----------------------------------------------------------------------------

BATCHED = dict(workload="batched: 64 datasets, sketch + within-dataset top-20 cosine",
               datasets=64, n="uniform [2000, 50000]", d="log-uniform [1e4, 1e7]",
               N="{256,...,8192}", nnz="lognormal(median U[50,500], sigma 1) clip [1,5000]",
               k=20, by="cos")


def run_batched(args):
    import tempfile

    import torch

    from paper_1910_04658_gb300 import binding as B, build
    from paper_1910_04658_gb300.batched import Autotuner, BatchedJob, make_datasets

    build.build()
    B.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ds = make_datasets(0, n_datasets=args.datasets)
    pairs = sum(d.n * (d.n - 1) for d in ds)
    flops = sum(2.0 * d.n * (d.n - 1) * d.N for d in ds)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return ts

    # reference form: one bs_topk_ex per dataset (default kernel choice), eager
    per = BatchedJob(ds, k=20, by="cos", mode="per_dataset")
    timed(per.run_eager, args.warmup)
    t_per = timed(per.run_eager, args.steps)
    # plain persistent form: one ranking launch for all datasets, default configuration
    plain = BatchedJob(ds, k=20, by="cos")
    timed(plain.run_eager, args.warmup)
    t_plain = timed(plain.run_eager, args.steps)
    # autotuned + graph
    cache = os.path.join(tempfile.mkdtemp(), "autotune.json")
    tuner = Autotuner(cache_path=cache)
    job = BatchedJob(ds, k=20, by="cos", autotuner=tuner)
    t0 = time.perf_counter()
    job.tune()
    tune_s = time.perf_counter() - t0
    job.capture()
    timed(job.replay, args.warmup)
    t_eager_tuned = timed(job.run_eager, args.steps)
    with ClockSampler(0) as clk:
        t_graph = timed(job.replay, args.steps)
    assert B.bs_get_async_error() == 0
    same = all(torch.equal(job.idx[j], per.idx[j]) and torch.equal(job.score[j], per.score[j]) and
               torch.equal(plain.idx[j], per.idx[j]) and torch.equal(plain.score[j], per.score[j])
               for j in range(len(ds)))
    tg = sum(t_graph) / len(t_graph)

    def name(v):
        return "popc" if (v & 15) == B.BS_VARIANT_POPC else (
            f"tc{((v >> 4) & 15) - 1}" if (v >> 4) else ("tc" if (v & 15) == B.BS_VARIANT_TC else "auto"))
    choice = {"batched_launch": name(job.bvariant)}
    for j in job.side:
        choice[name(job.variants[j])] = choice.get(name(job.variants[j]), 0) + 1
    pk = measured_peaks()
    bf16 = pk.get("bf16_tflops")
    peak = (bf16 if bf16 else 1900.0) * (13.5 / 2.25)
    line = {
        "metric": METRIC, "value": pairs / tg, "unit": "pair-estimates/s (whole batched job)",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tg * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32+f32",
        "data": "synthetic",
        "config": dict(BATCHED, datasets=len(ds), rows=sum(d.n for d in ds),
                       nnz=int(sum(d.col.numel() for d in ds)), launches_per_job=job.launches(),
                       l2="inputs (>3 GB of indices) larger than L2"),
        "roofline": {"bound": "tensor", "kernel": "whole job (mixed N), graph replay",
                     "achieved": flops / tg / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "frac": flops / tg / 1e12 / peak, "traffic": None,
                     "peak_source": "measured cuBLAS bf16 burst x 6 (nominal dense fp4/bf16 ratio), of measured"},
        "components": {"graph_replay_ms": tg * 1e3,
                       "eager_tuned_ms": sum(t_eager_tuned) / len(t_eager_tuned) * 1e3,
                       "eager_persistent_default_ms": sum(t_plain) / len(t_plain) * 1e3,
                       "eager_per_dataset_ms": sum(t_per) / len(t_per) * 1e3,
                       "launches_persistent": job.launches(), "launches_per_dataset": per.launches(),
                       "autotune_s": tune_s, "kernel_choices": choice,
                       "autotune_timings_ms": {k: v for t in tuner.timings.values() for k, v in t.items()}
                       if len(tuner.timings) == 1 else None,
                       "results_identical_to_per_dataset": same},
        "gpu_launches": job.launches() * args.steps,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# learned estimator in the dense regime
# ----------------------------------------------------------------------------

LEARNED = dict(workload="learned estimator, dense regime", d=100_000, Ns=[256, 1024],
               sizes="uniform [N/4, 4N]", train_pairs=10_000_000, heldout_pairs=1_000_000,
               mlp="4-64-64-4 GELU (tanh form), BF16 weights/activations, FP32 accumulation")


def run_learned(args):
    import torch

    from paper_1910_04658_gb300 import binding as B, build
    from paper_1910_04658_gb300 import learned as L

    build.build()
    B.lib()
    torch.cuda.set_device(0)
    per_n_train = args.train_pairs // 2
    per_n_test = args.heldout_pairs // 2
    t0 = time.perf_counter()
    train = [L.dense_pairs(per_n_train, N, pair_seed=1 + i) for i, N in enumerate(LEARNED["Ns"])]
    test = [L.dense_pairs(per_n_test, N, pair_seed=101 + i) for i, N in enumerate(LEARNED["Ns"])]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    mlp = L.MLPEstimator(seed=0)
    t0 = time.perf_counter()
    hist = mlp.train(train, epochs=args.epochs, batch=8192, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    table = {}
    rates = {"closed_form": [], "mlp": [], "mlp_cuda_cores": []}
    flush = torch.empty((256 << 20,), dtype=torch.uint8, device="cuda")   # > 129 MB L2
    for s in test:
        exact = L.exact_similarities(s.sizes.cpu().numpy().view(np.uint32))
        def mlp_cuda_cores(ps):
            out = torch.empty((ps.n, 4), dtype=torch.float32, device="cuda")
            B.bs_mlp_estimate_ex(mlp.params, ps.counts, ps.n, ps.N, out, B.BS_VARIANT_POPC)
            return out
        for name, fn in (("closed_form", L.closed_form), ("mlp", mlp.estimate),
                         ("mlp_cuda_cores", mlp_cuda_cores)):
            for _ in range(max(args.warmup, 3)):
                fn(s)
            ms = []
            for _ in range(max(args.steps, 1)):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                est = fn(s)
                e1.record()
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            rates[name].append(s.n / (float(np.mean(ms)) / 1e3))
            if name != "mlp_cuda_cores":
                table[f"N={s.N} {name}"] = L.mse_table(est.cpu().numpy(), exact)
    infer_rates = rates["mlp"]
    assert B.bs_get_async_error() == 0
    better = {m: all(table[f"N={s.N} mlp"][m] <= table[f"N={s.N} closed_form"][m] for s in test)
              for m in L.MEASURES}
    # MLP inference: the 64 x 64 hidden layer (2 x 64 x 64 flops per pair) on
    # the tensor cores, the 4 -> 64 and 64 -> 4 layers and both GELUs on the
    # FP32 CUDA cores; reported against the FP32 FMA peak (152 SMs x 128
    # lanes x 2 flops x 2.07 GHz), which the CUDA-core layers are bound by
    flops_pair = 2 * (4 * 64 + 64 * 64 + 64 * 4)
    alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    achieved = float(np.mean(infer_rates)) * flops_pair / 1e12
    line = {
        "metric": METRIC, "value": float(np.mean(infer_rates)),
        "unit": "pair-estimates/s (MLP inference from counts)", "n_gpus": 1,
        "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": float(np.mean([per_n_test / r for r in infer_rates])) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32",
        "data": "synthetic",
        "config": dict(LEARNED, train_pairs=args.train_pairs, heldout_pairs=args.heldout_pairs,
                       epochs=args.epochs, l2="flushed (256 MB write) before each timed launch"),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved / alu_peak, "traffic": None,
                     "kernel": "infer_tc_kernel (hidden layer on tcgen05 kind::f16)",
                     "peak_source": "FP32 FMA lanes x 2.07 GHz (all 9216 flops/pair counted)"},
        "components": {"mse_heldout": table, "mlp_mse_at_or_below_closed_form": better,
                       "closed_form_estimates_per_s": float(np.mean(rates["closed_form"])),
                       "mlp_cuda_cores_only_estimates_per_s": float(np.mean(rates["mlp_cuda_cores"])),
                       "train_loss_per_epoch": hist, "epochs": args.epochs,
                       "train_pairs_per_s": args.train_pairs * args.epochs / train_s,
                       "generate_s": gen_s, "train_s": train_s},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# ranking-quality evaluation (Experiment 2): thresholded retrieval vs exact
# ----------------------------------------------------------------------------

RANKING = dict(workload="ranking quality (Experiment 2): 90/10 split of the text-BoW corpus",
               n=100_000, d=1_000_000, query_frac=0.1, Ns=[512, 1024, 2048, 4096],
               measures=["js", "cos", "ip"])


def run_ranking(args):
    import torch

    from paper_1910_04658_gb300 import binding as B, build, inputs, ranking

    build.build()
    B.lib()
    torch.cuda.set_device(0)
    csr = inputs.bow_corpus(seed=0, n=args.n)
    ev_t0 = torch.cuda.Event(enable_timing=True)
    ev_t1 = torch.cuda.Event(enable_timing=True)
    ev_t0.record()
    ev = ranking.Evaluation(csr, seed=0, query_frac=RANKING["query_frac"])
    ev_t1.record()
    ev_t1.synchronize()
    exact_ms = ev_t0.elapsed_time(ev_t1)
    pairs = ev.nq * ev.ndb
    table, times = {}, {}
    for N in RANKING["Ns"]:
        ev.evaluate(N, RANKING["measures"])           # warm-up (kernel attributes, allocations)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = ev.evaluate(N, RANKING["measures"])
        e1.record()
        e1.synchronize()
        times[N] = e0.elapsed_time(e1)
        for m in RANKING["measures"]:
            table[f"N={N} {m}"] = [
                {"threshold": round(th, 4), "f1": r["f1"], "precision": r["precision"], "recall": r["recall"],
                 "accuracy": r["accuracy"], "pooled_f1": r["pooled_f1"], "truth_pairs": r["truth_pairs"],
                 "queries_with_truth": r["queries_with_truth"]}
                for th, r in zip(res[m]["thresholds"], res[m]["metrics"])]
    assert B.bs_get_async_error() == 0
    N0 = RANKING["Ns"][-1]
    value = pairs / (times[N0] / 1e3)
    line = {
        "metric": METRIC, "value": value,
        "unit": "query x training pairs evaluated per second (sketch + 3 estimates + threshold sets)",
        "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": times[N0], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32+f32 (exact side f64)", "data": "synthetic",
        "config": dict(RANKING, n=csr.n, queries=ev.nq, training=ev.ndb, pairs=pairs),
        "components": {"exact_counts_ms": exact_ms, "evaluate_ms_per_N": times,
                       "max_inner_product": ev.max_inner_product(), "by_N_and_measure": table},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-popc-compare", action="store_true",
                    help="skip the one-off CUDA-core variant launch reported for comparison")
    ap.add_argument("--n", type=int, default=WORKLOAD["n"],
                    help="rows of the corpus (smaller only for profiling captures)")
    ap.add_argument("--workload", choices=["bow", "serving", "batched", "learned", "ranking"],
                    default="bow")
    ap.add_argument("--train-pairs", type=int, default=10_000_000)
    ap.add_argument("--heldout-pairs", type=int, default=1_000_000)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--datasets", type=int, default=64)
    ap.add_argument("--db-rows", type=int, default=SERVING["db_rows"])
    ap.add_argument("--serving-requests", type=int, default=300)
    ap.add_argument("--loads", type=float, nargs="+", default=[0.5, 0.8, 0.95])
    ap.add_argument("--slots", type=int, default=3, help="serving: concurrent micro-batches")
    ap.add_argument("--no-serving", action="store_true",
                    help="default workload: skip the serving leg (p50/p99 on the 1M-sketch database)")
    ap.add_argument("--serving-leg-requests", type=int, default=100)
    ap.add_argument("--max-batch", type=int, default=4096, help="serving: queries per micro-batch")
    args = ap.parse_args()
    if args.workload == "serving":
        run_serving(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "learned":
        run_learned(args)
        return
    if args.workload == "ranking":
        run_ranking(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist_mod
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    try:
        run_ours(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
