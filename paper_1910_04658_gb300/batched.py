"""Many independent BinSketch datasets as one batched, autotuned, graph-captured job.

Each dataset (its own d, N and seed) is sketched (Definition "BinSketch") and
ranked within itself by an estimated similarity (Alg. 1-4, Experiment 2 as a
top-k).  The job runs as:

* one persistent launch that sketches every dataset (`bs_sketch_batched`,
  driven by a device job table);
* one top-k call per dataset, each with the kernel and block configuration an
  autotuner picked for its shape, spread over several streams;

and the whole sequence is captured once into a CUDA graph, so one graph
launch replays the job.  The autotuner times the candidate kernels
(CUDA-core POPC, tensor-core configurations 0-9) on the dataset itself and
caches the winner per (GPU, N, log2 n, k, measure) in a JSON file.  The
candidates compute identical estimates, so tuning changes speed, never
results.
"""
from __future__ import annotations

import json
import math
import os
import threading
from dataclasses import dataclass
from typing import Dict, List, Optional

import numpy as np

from . import binding as B

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "binsketch", "autotune.json")


@dataclass
class Dataset:
    row_ptr: "object"     # device int64 [n + 1] (uint64 offsets)
    col: "object"         # device int32 [nnz] (uint32 ids)
    d: int
    N: int
    seed: int = 0

    @property
    def n(self) -> int:
        return int(self.row_ptr.numel() - 1)


class Autotuner:
    """Picks the fastest top-k kernel per shape class and remembers it."""

    def __init__(self, cache_path: Optional[str] = None, reps: int = 2):
        self.path = cache_path or os.environ.get("BS_AUTOTUNE_CACHE", DEFAULT_CACHE)
        self.reps = reps
        self.lock = threading.Lock()
        self.table: Dict[str, int] = {}
        self.timings: Dict[str, Dict[str, float]] = {}
        try:
            with open(self.path) as f:
                self.table = {k: int(v) for k, v in json.load(f).items()}
        except (OSError, ValueError):
            self.table = {}

    @staticmethod
    def candidates():
        return [("popc", B.BS_VARIANT_POPC)] + [
            (f"tc{c}", B.BS_VARIANT_TC | B.BS_VARIANT_TC_CFG(c)) for c in range(B.BS_TC_CONFIGS)]

    @staticmethod
    def key(gpu: str, N: int, n: int, k: int, by: str) -> str:
        return f"{gpu}|N={N}|log2n={round(math.log2(max(n, 1)))}|k={k}|by={by}"

    def choose(self, gpu, sk, pc, n, N, k, by, score, idx, ws, wsb, stream) -> int:
        import torch
        key = self.key(gpu, N, n, k, by)
        with self.lock:
            if key in self.table:
                return self.table[key]
        best, best_t, times = None, float("inf"), {}
        for name, code in self.candidates():
            try:
                for _ in range(1 + self.reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    B.bs_topk_ex(sk, pc, n, sk, pc, n, N, B.MEASURE_BITS[by], k, 1, score, idx,
                                 ws, wsb, code, stream)
                    e1.record(stream)
                e1.synchronize()
                t = e0.elapsed_time(e1)
            except B.BinSketchError:
                continue            # configuration does not fit this shape
            times[name] = t
            if t < best_t:
                best, best_t = code, t
        if best is None:
            best = B.BS_VARIANT_AUTO
        with self.lock:
            self.table[key] = best
            self.timings[key] = times
        return best

    def save(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        tmp = self.path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.table, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


class BatchedJob:
    """Sketch + within-dataset top-k for a list of datasets."""

    def __init__(self, datasets: List[Dataset], k: int = 20, by: str = "cos",
                 autotuner: Optional[Autotuner] = None, n_streams: int = 4):
        import torch
        self.torch = torch
        self.ds = datasets
        self.k, self.by = k, by
        self.dev = datasets[0].row_ptr.device
        self.tuner = autotuner
        self.sk, self.pc, self.score, self.idx, self.ws, self.wsb = [], [], [], [], [], []
        for d in datasets:
            n = d.n
            self.sk.append(torch.empty((n, d.N // 32), dtype=torch.int32, device=self.dev))
            self.pc.append(torch.empty((n,), dtype=torch.int32, device=self.dev))
            self.score.append(torch.empty((n, k), dtype=torch.float32, device=self.dev))
            self.idx.append(torch.empty((n, k), dtype=torch.int32, device=self.dev))
            wsb = B.bs_topk_workspace_bytes(n, n, d.N, k)
            self.wsb.append(wsb)
            self.ws.append(torch.empty((max(wsb, 256),), dtype=torch.uint8, device=self.dev))
        # device job table for the batched sketch
        jobs = (B.bs_sketch_job * len(datasets))()
        for j, d in enumerate(datasets):
            jobs[j] = B.bs_sketch_job(d.row_ptr.data_ptr(), d.col.data_ptr(), d.col.numel(), d.seed,
                                      d.n, d.d, d.N, 0, self.sk[j].data_ptr(), self.pc[j].data_ptr())
        raw = np.frombuffer(bytes(jobs), dtype=np.uint8)
        self.jobs = torch.from_numpy(raw.copy()).to(self.dev)
        self.max_N = max(d.N for d in datasets)
        self.variants = [B.BS_VARIANT_AUTO] * len(datasets)
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(n_streams)]
        self.graph = None
        self.gpu = torch.cuda.get_device_name(self.dev)

    def launches(self) -> int:
        n = 1
        for d, v in zip(self.ds, self.variants):
            n += B.bs_topk_plan(d.n, d.n, d.N, self.k, v, True)[2]
        return n

    def sketch_all(self, stream):
        B.bs_sketch_batched(self.jobs, len(self.ds), self.max_N, stream)

    def tune(self):
        """Sketch once, then let the autotuner choose each dataset's kernel."""
        if self.tuner is None:
            return
        s = self.torch.cuda.current_stream(self.dev)
        self.sketch_all(s)
        for j, d in enumerate(self.ds):
            self.variants[j] = self.tuner.choose(self.gpu, self.sk[j], self.pc[j], d.n, d.N, self.k,
                                                 self.by, self.score[j], self.idx[j], self.ws[j],
                                                 self.wsb[j], s)
        s.synchronize()

    def _enqueue(self, main):
        self.sketch_all(main)
        order = sorted(range(len(self.ds)), key=lambda j: -self.ds[j].n * self.ds[j].n * self.ds[j].N)
        for t, j in enumerate(order):
            s = self.streams[t % len(self.streams)]
            s.wait_stream(main)
            d = self.ds[j]
            B.bs_topk_ex(self.sk[j], self.pc[j], d.n, self.sk[j], self.pc[j], d.n, d.N,
                         B.MEASURE_BITS[self.by], self.k, 1, self.score[j], self.idx[j],
                         self.ws[j], self.wsb[j], self.variants[j], s)
        for s in self.streams:
            main.wait_stream(s)

    def run_eager(self):
        main = self.torch.cuda.current_stream(self.dev)
        self._enqueue(main)

    def capture(self):
        """Record the whole job (one batched sketch + every top-k) as a CUDA graph."""
        torch = self.torch
        self.run_eager()                       # warm-up: kernel attributes are set outside capture
        torch.cuda.synchronize(self.dev)
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(device=self.dev)
        cap.wait_stream(torch.cuda.current_stream(self.dev))
        with torch.cuda.graph(g, stream=cap):
            self._enqueue(cap)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def results(self, j: int):
        return self.score[j], self.idx[j]


def make_datasets(seed: int, n_datasets: int = 64, n_lo: int = 2000, n_hi: int = 50000,
                  d_lo: float = 1e4, d_hi: float = 1e7, Ns=(256, 512, 1024, 2048, 4096, 8192),
                  med_lo: float = 50, med_hi: float = 500, device="cuda") -> List[Dataset]:
    """The batched workload: n uniform in [n_lo, n_hi], d log-uniform in
    [d_lo, d_hi], N from Ns, log-normal nnz with a per-dataset median in
    [med_lo, med_hi] (sigma 1, clipped to [1, 5000]), Zipf(1.0) columns."""
    from . import inputs
    rng = np.random.default_rng(seed)
    out = []
    for j in range(n_datasets):
        n = int(rng.integers(n_lo, n_hi + 1))
        d = int(round(math.exp(rng.uniform(math.log(d_lo), math.log(d_hi)))))
        N = int(rng.choice(Ns))
        med = float(rng.uniform(med_lo, med_hi))
        rp, col = inputs.bow_corpus_device(seed * 1000 + j, n, d, median=med, device=device)
        out.append(Dataset(rp, col, d, N, seed=j))
    return out
