"""Many independent BinSketch datasets as one batched, autotuned, graph-captured job.

Each dataset (its own d, N and seed) is sketched (Definition "BinSketch") and
ranked within itself by an estimated similarity (Alg. 1-4, Experiment 2 as a
top-k).  The job runs as:

* one persistent launch that sketches every dataset (`bs_sketch_batched`,
  driven by a device job table);
* one persistent tensor-core launch that ranks every dataset
  (`bs_topk_batched`): the (dataset, query block, database tile) work units
  of all datasets form one queue cut into equal-cost ranges per SM, so small
  datasets fill the gaps of large ones -- plus one re-layout launch before it
  and one merge launch after it when a query block is split between SMs;
* datasets outside the tensor-core shape (N not a multiple of 128, N < 256
  or N > 8192) ranked one `bs_topk_ex` call each on side streams;

and the whole sequence is captured once into a CUDA graph, so one graph
launch replays the job.  The autotuner times the tensor-core block
configurations on the batched launch itself and caches the winner per
(GPU, job table signature, k, measure) in a JSON file.  The candidates compute
identical estimates, so tuning changes speed, never results.  mode =
"per_dataset" keeps the earlier form -- one autotuned `bs_topk_ex` per
dataset on several streams -- as the reference the persistent form is
checked and timed against.
"""
from __future__ import annotations

import hashlib
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

    @staticmethod
    def batch_key(gpu: str, shapes, k: int, by: str) -> str:
        """Key of a batched launch: the GPU, the sorted (n, N) of its datasets, k, measure."""
        sig = hashlib.sha1(repr(sorted(shapes)).encode()).hexdigest()[:12]
        return f"{gpu}|batched|jobs={len(shapes)}|sig={sig}|k={k}|by={by}"

    def choose_batched(self, key: str, run, stream) -> int:
        """Time run(variant) for each tensor-core configuration; keep the fastest."""
        import torch
        with self.lock:
            if key in self.table:
                return self.table[key]
        best, best_t, times = None, float("inf"), {}
        for name, code in self.candidates()[1:]:
            try:
                for _ in range(1 + self.reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    run(code)
                    e1.record(stream)
                e1.synchronize()
                t = e0.elapsed_time(e1)
            except B.BinSketchError:
                continue            # configuration does not fit k
            times[name] = t
            if t < best_t:
                best, best_t = code, t
        if best is None:
            best = B.BS_VARIANT_TC
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


def tc_shape(N: int) -> bool:
    """Whether the tensor-core kernels take sketches of N bits."""
    return N % 128 == 0 and 256 <= N <= 8192


class BatchedJob:
    """Sketch + within-dataset top-k for a list of datasets."""

    def __init__(self, datasets: List[Dataset], k: int = 20, by: str = "cos",
                 autotuner: Optional[Autotuner] = None, n_streams: int = 4,
                 mode: str = "persistent"):
        import torch
        if mode not in ("persistent", "per_dataset"):
            raise ValueError(f"mode: {mode}")
        self.torch = torch
        self.ds = datasets
        self.k, self.by = k, by
        self.mode = mode
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
        # the batched ranking: tensor-core datasets in one host job table, the rest one call each
        self.in_batch = [j for j, d in enumerate(datasets) if mode == "persistent" and tc_shape(d.N)]
        self.side = [j for j in range(len(datasets)) if j not in set(self.in_batch)]
        self.tjobs = None
        self.bws, self.bwsb, self.bvariant = None, 0, B.BS_VARIANT_TC
        if self.in_batch:
            if len(self.in_batch) > B.BS_TOPK_BATCH_MAX:
                raise ValueError(f"at most {B.BS_TOPK_BATCH_MAX} tensor-core datasets per batched launch")
            self.tjobs = B._job_table([dict(Q=self.sk[j], pcQ=self.pc[j], DB=self.sk[j], pcDB=self.pc[j],
                                            score=self.score[j], idx=self.idx[j], nQ=datasets[j].n,
                                            nDB=datasets[j].n, N=datasets[j].N, exclude_self=True, k=k)
                                       for j in self.in_batch])
            self.bwsb = B.bs_topk_batched_workspace_bytes(self.tjobs, k)
            self.bws = torch.empty((max(self.bwsb, 256),), dtype=torch.uint8, device=self.dev)
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(n_streams)]
        self.graph = None
        self.gpu = torch.cuda.get_device_name(self.dev)

    def launches(self) -> int:
        """Kernels one replay of the job launches."""
        n = 1
        if self.tjobs is not None:
            n += B.bs_topk_batched_plan(self.tjobs, self.k)[1]
        for j in self.side:
            d = self.ds[j]
            n += B.bs_topk_plan(d.n, d.n, d.N, self.k, self.variants[j], True)[2]
        return n

    def sketch_all(self, stream):
        B.bs_sketch_batched(self.jobs, len(self.ds), self.max_N, stream)

    def _rank_batch(self, variant, stream):
        B.bs_topk_batched(self.tjobs, B.MEASURE_BITS[self.by], self.k, self.bws, self.bwsb, variant, stream)

    def tune(self):
        """Sketch once, then let the autotuner choose the batched launch's block
        configuration (and each side dataset's kernel)."""
        if self.tuner is None:
            return
        s = self.torch.cuda.current_stream(self.dev)
        self.sketch_all(s)
        if self.tjobs is not None:
            shapes = [(self.ds[j].n, self.ds[j].N) for j in self.in_batch]
            key = Autotuner.batch_key(self.gpu, shapes, self.k, self.by)
            self.bvariant = self.tuner.choose_batched(key, lambda v: self._rank_batch(v, s), s)
        for j in self.side:
            d = self.ds[j]
            self.variants[j] = self.tuner.choose(self.gpu, self.sk[j], self.pc[j], d.n, d.N, self.k,
                                                 self.by, self.score[j], self.idx[j], self.ws[j],
                                                 self.wsb[j], s)
        s.synchronize()

    def _enqueue(self, main):
        self.sketch_all(main)
        order = sorted(self.side, key=lambda j: -self.ds[j].n * self.ds[j].n * self.ds[j].N)
        for t, j in enumerate(order):
            s = self.streams[t % len(self.streams)]
            s.wait_stream(main)
            d = self.ds[j]
            B.bs_topk_ex(self.sk[j], self.pc[j], d.n, self.sk[j], self.pc[j], d.n, d.N,
                         B.MEASURE_BITS[self.by], self.k, 1, self.score[j], self.idx[j],
                         self.ws[j], self.wsb[j], self.variants[j], s)
        if self.tjobs is not None:
            self._rank_batch(self.bvariant, main)
        for s in self.streams[:len(order)]:
            main.wait_stream(s)

    def run_eager(self):
        main = self.torch.cuda.current_stream(self.dev)
        self._enqueue(main)

    def capture(self):
        """Record the whole job (one batched sketch + the ranking) as a CUDA graph."""
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
