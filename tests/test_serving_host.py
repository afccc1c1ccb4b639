"""Host logic of the serving loop (no GPU): the arena allocator and the
continuous-batching scheduler, driven by a fake executor."""
import numpy as np
import pytest

from paper_1910_04658_gb300.serving import Arena, Executor, Request, Scheduler, latency_stats


def test_arena_first_fit_and_coalescing():
    a = Arena(10_000)
    o1 = a.alloc(1000)
    o2 = a.alloc(3000)
    o3 = a.alloc(500)
    assert (o1, o2, o3) == (0, 1024, 4096)
    assert a.alloc(10_000) is None
    a.release(o2, 3000)
    assert a.alloc(2000) == 1024                  # first fit reuses the hole
    a.release(o1, 1000)
    a.release(1024, 2000)
    a.release(o3, 500)
    assert a.free == [(0, 10_000)]                # everything coalesced again


class FakeExecutor(Executor):
    """Completes a batch after `latency` polls; results encode request and row."""

    def __init__(self, latency=3):
        self.latency = latency
        self.polls = {}
        self.launched = []

    def footprint(self, nq, nnz):
        return 256 * nq + 4 * nnz + 1024

    def launch(self, b):
        self.polls[b.bid] = 0
        self.launched.append(b)

    def done(self, b):
        self.polls[b.bid] += 1
        return self.polls[b.bid] >= self.latency

    def results(self, b):
        out = {}
        for r in b.requests:
            q = r.n_queries
            out[r.rid] = (np.full((q, 2), r.rid, np.float32), np.arange(q * 2, dtype=np.uint32).reshape(q, 2))
        return out


def _reqs(sizes, arrivals=None):
    out = []
    for i, q in enumerate(sizes):
        rp = np.arange(q + 1, dtype=np.uint64) * 3
        out.append(Request(i, 0.0 if arrivals is None else arrivals[i], rp,
                           np.zeros(3 * q, np.uint32)))
    return out


def test_scheduler_batches_respect_limits_and_serve_everyone():
    ex = FakeExecutor()
    sizes = [1, 5, 300, 2, 900, 40, 1000, 7, 64, 3]
    sch = Scheduler(ex, arena_bytes=600_000, slots=2, max_batch_queries=1024, poll_s=0)
    res = sch.run(_reqs(sizes))
    assert [r.rid for r in res] == list(range(len(sizes)))
    for r, q in zip(res, sizes):
        assert r.score.shape == (q, 2) and np.all(r.score == r.rid)
    for b in ex.launched:
        assert b.n_queries <= 1024 or len(b.requests) == 1
        assert ex.footprint(b.n_queries, b.nnz) <= 600_000
    # arrival order is kept across batches
    order = [r.rid for b in ex.launched for r in b.requests]
    assert order == sorted(order)
    assert sch.max_inflight <= 2
    assert sch.peak_arena_bytes <= 600_000
    assert len(ex.launched) < len(sizes)          # requests were batched together


def test_memory_bound_requests_wait_for_free_hbm():
    ex = FakeExecutor(latency=2)
    # each 1000-query request needs ~262 KB; the arena holds one at a time
    sch = Scheduler(ex, arena_bytes=300_000, slots=3, max_batch_queries=4096, poll_s=0)
    res = sch.run(_reqs([1000, 1000, 1000]))
    assert len(res) == 3
    assert sch.max_inflight == 1                  # admission by memory, not by slots
    with pytest.raises(MemoryError):
        Scheduler(FakeExecutor(), arena_bytes=10_000, slots=1).run(_reqs([1000]))


def test_latency_stats():
    ex = FakeExecutor()
    res = Scheduler(ex, arena_bytes=1 << 20, slots=2, poll_s=0).run(_reqs([3, 4, 5], [0.0, 0.001, 0.002]))
    st = latency_stats(res)
    assert st["requests"] == 3 and st["queries"] == 12
    assert st["p50_ms"] >= 0 and st["p99_ms"] >= st["p50_ms"]


def test_arena_random_alloc_release_keeps_its_invariants():
    # live ranges never overlap and stay aligned, free + live = size, and
    # releasing everything leaves one free range covering the arena
    rng = np.random.default_rng(7)
    size = 1 << 20
    for _ in range(20):
        a = Arena(size)
        live = {}
        for step in range(400):
            if live and (rng.random() < 0.45 or len(live) > 60):
                off = list(live)[int(rng.integers(len(live)))]
                a.release(off, live.pop(off))
            else:
                n = int(rng.integers(1, 60_000))
                off = a.alloc(n)
                if off is None:
                    assert all(ln < a._round(n) for _, ln in a.free)   # first fit found no hole
                    continue
                assert off % Arena.ALIGN == 0 and off + a._round(n) <= size
                live[off] = n
            spans = sorted((o, o + a._round(n)) for o, n in live.items())
            assert all(e <= s for (_, e), (s, _) in zip(spans, spans[1:]))
            assert a.free_bytes + sum(a._round(n) for n in live.values()) == size
            assert all(o1 + l1 < o2 for (o1, l1), (o2, _) in zip(a.free, a.free[1:]))   # coalesced
        for off, n in list(live.items()):
            a.release(off, n)
        assert a.free == [(0, size)]
