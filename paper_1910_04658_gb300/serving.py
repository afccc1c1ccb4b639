"""Top-k query serving against a device-resident sketch database.

Requests (a CSR batch of query vectors each) arrive over time.  The server
keeps the database sketched and tiled in HBM, and continuously batches the
requests: whenever a launch slot (a CUDA stream) is free, the queued requests
that fit into the free part of a device memory arena are packed into one
micro-batch, which is sketched on arrival (Definition "BinSketch") and ranked
against the whole database by estimated similarity (Experiment 2 as a top-k,
Alg. 1-4) with one tensor-core top-k launch.  Requests that arrive while
others run are admitted as slots and memory free up, and the batches of
different slots overlap on the device.  Every query row is ranked
independently, so a request's result does not depend on what it was batched
with.

The scheduler (`Scheduler`) is pure host logic over an `Executor` interface;
`GpuExecutor` runs batches through the C ABI.  All device memory comes from
torch; the kernels are the library's.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass
from typing import Dict, List, Optional

import numpy as np


# ----------------------------------------------------------------------------
# requests and results
# ----------------------------------------------------------------------------

@dataclass
class Request:
    rid: int
    arrival: float            # seconds from the start of the run
    row_ptr: np.ndarray       # uint64 [q + 1]
    col: np.ndarray           # uint32 [nnz]

    @property
    def n_queries(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


@dataclass
class Result:
    rid: int
    score: np.ndarray         # float32 [q][k]
    idx: np.ndarray           # uint32 [q][k]
    arrival: float
    launched: float
    done: float
    batch: int                # id of the micro-batch that carried it

    @property
    def latency(self) -> float:
        return self.done - self.arrival


# ----------------------------------------------------------------------------
# device memory arena: admission by free HBM
# ----------------------------------------------------------------------------

class Arena:
    """First-fit allocator of byte ranges in one fixed region (256-byte aligned)."""

    ALIGN = 256

    def __init__(self, size: int):
        self.size = int(size)
        self.free = [(0, self.size)]          # sorted (offset, length)

    def _round(self, n):
        return (int(n) + self.ALIGN - 1) // self.ALIGN * self.ALIGN

    def alloc(self, n: int) -> Optional[int]:
        n = self._round(max(n, 1))
        for i, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, ln - n)
                return off
        return None

    def release(self, off: int, n: int):
        n = self._round(max(n, 1))
        self.free.append((off, n))
        self.free.sort()
        merged = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged

    @property
    def free_bytes(self) -> int:
        return sum(ln for _, ln in self.free)


# ----------------------------------------------------------------------------
# scheduler
# ----------------------------------------------------------------------------

@dataclass
class Batch:
    bid: int
    requests: List[Request]
    slot: int
    offset: int = 0
    nbytes: int = 0
    launched: float = 0.0
    handle: object = None

    @property
    def n_queries(self):
        return sum(r.n_queries for r in self.requests)

    @property
    def nnz(self):
        return sum(r.nnz for r in self.requests)


class Executor:
    """What the scheduler needs from a device."""

    def footprint(self, n_queries: int, nnz: int) -> int:
        raise NotImplementedError

    def launch(self, batch: Batch):           # asynchronous
        raise NotImplementedError

    def done(self, batch: Batch) -> bool:
        raise NotImplementedError

    def results(self, batch: Batch) -> Dict[int, tuple]:   # rid -> (score, idx)
        raise NotImplementedError


class Scheduler:
    """Continuous batching with admission by slots and arena memory.

    max_batch_queries bounds the queries of one micro-batch; a request larger
    than that runs alone.  Requests are served in arrival order (a request
    that does not fit in memory holds the queue, so none is starved)."""

    def __init__(self, executor: Executor, arena_bytes: int, slots: int = 3,
                 max_batch_queries: int = 4096, clock=time.perf_counter, poll_s: float = 2e-5):
        self.ex = executor
        self.arena = Arena(arena_bytes)
        self.slots = slots
        self.max_batch_queries = max_batch_queries
        self.clock = clock
        self.poll_s = poll_s
        self.batches_launched = 0
        self.max_inflight = 0
        self.peak_arena_bytes = 0

    def _form_batch(self, pending: deque, slot: int) -> Optional[Batch]:
        take: List[Request] = []
        nq = nnz = 0
        while pending:
            r = pending[0]
            if take and nq + r.n_queries > self.max_batch_queries:
                break
            need = self.ex.footprint(nq + r.n_queries, nnz + r.nnz)
            if need > self.arena.size and not take:
                raise MemoryError(f"request {r.rid} needs {need} bytes, arena holds {self.arena.size}")
            if take and need > self.arena.free_bytes:
                break
            take.append(pending.popleft())
            nq += r.n_queries
            nnz += r.nnz
        if not take:
            return None
        nbytes = self.ex.footprint(nq, nnz)
        off = self.arena.alloc(nbytes)
        if off is None:                     # not enough free HBM yet: wait
            for r in reversed(take):
                pending.appendleft(r)
            return None
        b = Batch(self.batches_launched, take, slot, off, nbytes)
        self.batches_launched += 1
        used = self.arena.size - self.arena.free_bytes
        self.peak_arena_bytes = max(self.peak_arena_bytes, used)
        return b

    def run(self, requests: List[Request]) -> List[Result]:
        reqs = sorted(requests, key=lambda r: r.arrival)
        pending: deque = deque()
        inflight: List[Batch] = []
        free_slots = list(range(self.slots))
        out: List[Result] = []
        t0 = self.clock()
        i = 0
        while i < len(reqs) or pending or inflight:
            now = self.clock() - t0
            while i < len(reqs) and reqs[i].arrival <= now:
                pending.append(reqs[i])
                i += 1
            progressed = False
            for b in list(inflight):
                if self.ex.done(b):
                    t = self.clock() - t0
                    res = self.ex.results(b)
                    for r in b.requests:
                        s, ix = res[r.rid]
                        out.append(Result(r.rid, s, ix, r.arrival, b.launched, t, b.bid))
                    self.arena.release(b.offset, b.nbytes)
                    inflight.remove(b)
                    free_slots.append(b.slot)
                    progressed = True
            while free_slots and pending:
                b = self._form_batch(pending, free_slots[0])
                if b is None:
                    break
                free_slots.pop(0)
                b.launched = self.clock() - t0
                self.ex.launch(b)
                inflight.append(b)
                self.max_inflight = max(self.max_inflight, len(inflight))
                progressed = True
            if not progressed:
                if not inflight and not pending and i < len(reqs):
                    wait = reqs[i].arrival - (self.clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                else:
                    time.sleep(self.poll_s)
        return sorted(out, key=lambda r: r.rid)


def latency_stats(results: List[Result], wall_s: Optional[float] = None) -> dict:
    lat = np.array([r.latency for r in results], np.float64)
    nq = sum(r.score.shape[0] for r in results)
    span = wall_s if wall_s is not None else (max(r.done for r in results) -
                                             min(r.arrival for r in results))
    return {"requests": len(results), "queries": int(nq),
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
            "mean_ms": float(lat.mean() * 1e3) if lat.size else None,
            "queries_per_s": nq / span if span > 0 else None}


def poisson_requests(rng: np.random.Generator, n_requests: int, rate_per_s: float, make_csr,
                     q_lo: int = 1, q_hi: int = 4096) -> List[Request]:
    """Poisson arrivals; request sizes log-uniform in [q_lo, q_hi];
    make_csr(rng, q) -> (row_ptr, col)."""
    t = 0.0
    out = []
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        q = int(round(math.exp(rng.uniform(math.log(q_lo), math.log(q_hi)))))
        q = min(max(q, q_lo), q_hi)
        rp, col = make_csr(rng, q)
        out.append(Request(rid, t, rp, col))
    return out


# ----------------------------------------------------------------------------
# GPU executor
# ----------------------------------------------------------------------------

class SketchDB:
    """Sketches of a corpus kept in HBM with the two copies the tensor-core
    search reads: tiled (bs_topk_pretiled) and FP4 (bs_topk_prewidened, the
    one the executor uses: both operands by TMA, 4x the packed size)."""

    def __init__(self, row_ptr, col, d: int, N: int, seed: int = 0, stream=None):
        import torch
        from . import binding as B
        n = row_ptr.numel() - 1
        dev = row_ptr.device
        self.n, self.d, self.N, self.seed = n, d, N, seed
        self.sketch = torch.empty((n, N // 32), dtype=torch.int32, device=dev)
        self.pc = torch.empty((n,), dtype=torch.int32, device=dev)
        B.bs_sketch(row_ptr, col, n, col.numel(), d, N, seed, self.sketch, self.pc, stream)
        self._copies(stream)

    def _copies(self, stream=None):
        import torch
        from . import binding as B
        dev = self.sketch.device
        self.tiled = torch.empty((B.bs_tiled_bytes(self.n, self.N),), dtype=torch.uint8, device=dev)
        B.bs_tile_sketches(self.sketch, self.n, self.N, self.tiled, stream)
        self.fp4 = torch.empty((B.bs_fp4_bytes(self.n, self.N),), dtype=torch.uint8, device=dev)
        B.bs_fp4_sketches(self.sketch, self.n, self.N, self.fp4, stream)

    def save(self, path: str) -> None:
        """Write the sketches with their (N, seed) (checkpoint.py format)."""
        from . import checkpoint
        checkpoint.save_sketches(path, self.sketch, self.pc, self.N, self.seed, self.d)

    @classmethod
    def load(cls, path: str, device: str = "cuda", expect_N: int = None, expect_seed: int = None,
             stream=None) -> "SketchDB":
        """A database from a checkpoint, its tensor-core copies rebuilt;
        refuses one sketched with another (N, seed) than expected."""
        from . import checkpoint
        sk, pc, meta = checkpoint.load_sketches(path, device, expect_N, expect_seed)
        db = cls.__new__(cls)
        db.n, db.d, db.N, db.seed = meta.n, meta.d, meta.N, meta.seed
        db.sketch, db.pc = sk, pc
        db._copies(stream)
        return db


class GpuExecutor(Executor):
    """Runs a micro-batch on its slot's stream: pinned-host CSR in, sketch,
    tensor-core top-k against the database, top-k back to pinned host."""

    def __init__(self, db: SketchDB, k: int = 100, by: str = "js", slots: int = 3,
                 arena_bytes: int = 1 << 30, max_queries: int = 4096, max_nnz: int = 4096 * 1500):
        import torch
        from . import binding as B
        self.B, self.torch = B, torch
        self.db, self.k, self.by = db, k, B.MEASURE_BITS[by]
        dev = db.sketch.device
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(slots)]
        self.arena = torch.empty((arena_bytes,), dtype=torch.uint8, device=dev)
        self.base = self.arena.data_ptr()
        # pinned staging per slot, reused once the slot's batch has completed
        self.stage = [self._pinned(max_queries, max_nnz) for _ in range(slots)]
        self.events = {}
        self.host = {}

    def _pinned(self, nq, nnz):
        t = self.torch
        return {"rp": t.empty((nq + 1,), dtype=t.int64).pin_memory(),
                "col": t.empty((max(nnz, 1),), dtype=t.int32).pin_memory(),
                "score": t.empty((nq, self.k), dtype=t.float32).pin_memory(),
                "idx": t.empty((nq, self.k), dtype=t.int32).pin_memory(), "nq": nq, "nnz": nnz}

    def footprint(self, n_queries, nnz):
        return sum(v for _, v in self._parts(n_queries, nnz))

    def _parts(self, nq, nnz):
        N, k = self.db.N, self.k
        ws = self.B.bs_topk_prewidened_workspace_bytes(nq, self.db.n, N, k)
        a = lambda x: (int(x) + 255) // 256 * 256
        return [("rp", a(8 * (nq + 1))), ("col", a(4 * max(nnz, 1))), ("sk", a(nq * N // 8)),
                ("pc", a(4 * nq)), ("score", a(4 * nq * k)), ("idx", a(4 * nq * k)), ("ws", a(ws))]

    def launch(self, b: Batch):
        torch, B = self.torch, self.B
        nq, nnz = b.n_queries, b.nnz
        st = self.stage[b.slot]
        if nq > st["nq"] or nnz > st["nnz"]:
            st = self.stage[b.slot] = self._pinned(max(nq, st["nq"]), max(nnz, st["nnz"]))
        rp = st["rp"].numpy()[:nq + 1].view(np.uint64)
        col = st["col"].numpy()[:max(nnz, 1)].view(np.uint32)
        rp[0] = 0
        pos, base = 0, 0
        for r in b.requests:
            q, z = r.n_queries, r.nnz
            rp[pos + 1:pos + q + 1] = r.row_ptr[1:] + np.uint64(base)
            col[base:base + z] = r.col
            pos += q
            base += z
        ptr = {}
        off = b.offset
        for name, ln in self._parts(nq, nnz):
            ptr[name] = off
            off += ln
        A = self.arena
        s = self.streams[b.slot]
        with torch.cuda.stream(s):
            A[ptr["rp"]:ptr["rp"] + 8 * (nq + 1)].copy_(st["rp"][:nq + 1].view(torch.uint8),
                                                          non_blocking=True)
            if nnz:
                A[ptr["col"]:ptr["col"] + 4 * nnz].copy_(st["col"][:nnz].view(torch.uint8),
                                                           non_blocking=True)
            g = {name: self.base + o for name, o in ptr.items()}
            B.bs_sketch(g["rp"], g["col"], nq, nnz, self.db.d, self.db.N, self.db.seed,
                        g["sk"], g["pc"], s)
            ws_bytes = B.bs_topk_prewidened_workspace_bytes(nq, self.db.n, self.db.N, self.k)
            B.bs_topk_prewidened(g["sk"], g["pc"], nq, self.db.fp4, self.db.pc, self.db.n,
                                 self.db.N, self.by, self.k, g["score"], g["idx"], g["ws"],
                                 ws_bytes, s)
            kk = self.k
            st["score"][:nq].view(torch.uint8).view(-1).copy_(
                A[ptr["score"]:ptr["score"] + 4 * nq * kk], non_blocking=True)
            st["idx"][:nq].view(torch.uint8).view(-1).copy_(
                A[ptr["idx"]:ptr["idx"] + 4 * nq * kk], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        self.events[b.bid] = ev
        self.host[b.bid] = (st, nq)

    def done(self, b: Batch) -> bool:
        return self.events[b.bid].query()

    def results(self, b: Batch):
        st, nq = self.host.pop(b.bid)
        self.events.pop(b.bid)
        sc = st["score"].numpy()[:nq]
        ix = st["idx"].numpy()[:nq].view(np.uint32)
        out, pos = {}, 0
        for r in b.requests:
            q = r.n_queries
            out[r.rid] = (sc[pos:pos + q].copy(), ix[pos:pos + q].copy())
            pos += q
        return out
