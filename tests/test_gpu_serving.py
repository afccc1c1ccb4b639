"""Serving on the GPU: continuous batching gives every request exactly the
result it gets alone, and those results match the oracle."""
import numpy as np
import pytest

import oracle
from paper_1910_04658_gb300 import inputs
from tests.helpers import check_topk_row, to_dev, u32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1910_04658_gb300 import binding as B  # noqa: E402
from paper_1910_04658_gb300.serving import (GpuExecutor, Request, Scheduler, SketchDB,  # noqa: E402
                                            latency_stats)

N, K = 4096, 100


@pytest.fixture(scope="module")
def served():
    db_csr = inputs.random_csr(31, 20_000, 1_000_000, 1, 400)
    rp, col = to_dev(db_csr)
    db = SketchDB(rp, col, db_csr.d, N, seed=5)
    torch.cuda.synchronize()
    assert B.bs_get_async_error() == 0
    rng = np.random.default_rng(3)
    reqs = []
    t = 0.0
    for rid, q in enumerate([1, 7, 300, 2, 64, 128, 33, 500, 5, 90, 256, 11]):
        c = inputs.random_csr(100 + rid, q, 1_000_000, 1, 400)
        t += rng.exponential(0.0005)
        reqs.append(Request(rid, t, c.row_ptr, c.col))
    return db_csr, db, reqs


def _serve(db, reqs, slots, max_q):
    ex = GpuExecutor(db, k=K, by="js", slots=slots, arena_bytes=256 << 20, max_queries=max_q)
    sch = Scheduler(ex, arena_bytes=256 << 20, slots=slots, max_batch_queries=max_q)
    res = sch.run(reqs)
    torch.cuda.synchronize()
    assert B.bs_get_async_error() == 0
    return res, sch


def test_mixed_equals_alone(served):
    _, db, reqs = served
    mixed, sch = _serve(db, reqs, slots=3, max_q=512)
    assert sch.batches_launched < len(reqs)            # requests really were batched
    assert len({r.batch for r in mixed}) == sch.batches_launched
    for r in reqs:
        alone, _ = _serve(db, [Request(r.rid, 0.0, r.row_ptr, r.col)], slots=1, max_q=4096)
        m = mixed[r.rid]
        assert np.array_equal(alone[0].idx, m.idx)
        assert np.array_equal(alone[0].score, m.score)
    st = latency_stats(mixed)
    assert st["queries"] == sum(r.n_queries for r in reqs)


def test_served_results_match_oracle(served):
    db_csr, db, reqs = served
    res, _ = _serve(db, reqs, slots=2, max_q=256)
    dsk, _ = oracle.sketch(db_csr.row_ptr, db_csr.col, db_csr.d, N, seed=5)
    assert np.array_equal(u32(db.sketch), dsk)
    for r in [reqs[1], reqs[4], reqs[9]]:
        qsk, _ = oracle.sketch(r.row_ptr, r.col, db_csr.d, N, seed=5)
        oest, _ = oracle.estimate_pairs(qsk, dsk, N)
        got = res[r.rid]
        for i in range(r.n_queries):
            check_topk_row(got.score[i], got.idx[i], oest[2, i], K, 2)


def test_pretiled_matches_topk(served):
    db_csr, db, reqs = served
    r = reqs[7]
    rp = torch.from_numpy(r.row_ptr.view(np.int64)).cuda()
    col = torch.from_numpy(r.col.view(np.int32)).cuda()
    q = r.n_queries
    sk = torch.empty((q, N // 32), dtype=torch.int32, device="cuda")
    pc = torch.empty((q,), dtype=torch.int32, device="cuda")
    B.bs_sketch(rp, col, q, r.nnz, db.d, N, 5, sk, pc)
    s1 = torch.empty((q, K), dtype=torch.float32, device="cuda")
    i1 = torch.empty((q, K), dtype=torch.int32, device="cuda")
    wsb = B.bs_topk_pretiled_workspace_bytes(q, db.n, N, K)
    ws = torch.empty((wsb,), dtype=torch.uint8, device="cuda")
    B.bs_topk_pretiled(sk, pc, q, db.tiled, db.pc, db.n, N, B.BS_JS, K, s1, i1, ws, wsb)
    s2 = torch.empty_like(s1)
    i2 = torch.empty_like(i1)
    wsb2 = B.bs_topk_workspace_bytes(q, db.n, N, K)
    ws2 = torch.empty((wsb2,), dtype=torch.uint8, device="cuda")
    B.bs_topk_ex(sk, pc, q, db.sketch, db.pc, db.n, N, B.BS_JS, K, 0, s2, i2, ws2, wsb2,
                 B.BS_VARIANT_TC)
    assert np.array_equal(u32(i1), u32(i2)) and np.array_equal(s1.cpu().numpy(), s2.cpu().numpy())


def test_prewidened_matches_pretiled_and_fp4_layout(served):
    # the FP4 copy is the documented widening of every word, and the search
    # against it returns, bit for bit, the lists of the tiled database
    db_csr, db, reqs = served
    w = u32(db.sketch[:64])
    M = np.uint32(0x22222222)
    want = np.stack([(w << np.uint32(1)) & M, w & M, (w >> np.uint32(1)) & M, (w >> np.uint32(2)) & M],
                    axis=-1).reshape(64, -1)
    got = db.fp4[:64 * (N // 2)].cpu().numpy().view(np.uint32).reshape(64, -1)
    assert np.array_equal(got, want)
    r = reqs[3]
    rp = torch.from_numpy(r.row_ptr.view(np.int64)).cuda()
    col = torch.from_numpy(r.col.view(np.int32)).cuda()
    q = r.n_queries
    sk = torch.empty((q, N // 32), dtype=torch.int32, device="cuda")
    pc = torch.empty((q,), dtype=torch.int32, device="cuda")
    B.bs_sketch(rp, col, q, r.nnz, db.d, N, 5, sk, pc)
    out = []
    for fn, wsfn, base in ((B.bs_topk_pretiled, B.bs_topk_pretiled_workspace_bytes, db.tiled),
                           (B.bs_topk_prewidened, B.bs_topk_prewidened_workspace_bytes, db.fp4)):
        s = torch.empty((q, K), dtype=torch.float32, device="cuda")
        i = torch.empty((q, K), dtype=torch.int32, device="cuda")
        wsb = wsfn(q, db.n, N, K)
        ws = torch.empty((wsb,), dtype=torch.uint8, device="cuda")
        fn(sk, pc, q, base, db.pc, db.n, N, B.BS_JS, K, s, i, ws, wsb)
        assert B.bs_get_async_error() == 0
        out.append((s, i))
    assert torch.equal(out[0][1], out[1][1]) and torch.equal(out[0][0], out[1][0])


def test_device_corpus_generator_shape():
    rp, col = inputs.bow_corpus_device(0, 5000, 100_000)
    lens = (rp[1:] - rp[:-1]).cpu().numpy()
    assert lens.min() >= 1 and lens.max() <= 5000 and 100 < np.median(lens) < 400
    c = col.cpu().numpy().view(np.uint32)
    assert c.max() < 100_000
