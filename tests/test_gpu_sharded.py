"""Database-sharded ranking on one GPU: P in-process shards (bs_topk_shard)
merged by bs_topk_merge must equal the unsharded bs_topk exactly -- the same
indices and bit-identical scores -- for both pair-counting kernels, in
all-pairs mode (self pair excluded through the shard offset) and in
query-vs-database mode, with ragged shards and a shard smaller than k.  The
merged lists are also checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1910_04658_gb300 import inputs, sharded
from tests.helpers import check_topk_row, to_dev, u32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1910_04658_gb300 import api, binding as B  # noqa: E402


def _sketch(seed, n, N):
    c = inputs.random_csr(seed, n, 50_000, 1, 400)
    rp, col = to_dev(c)
    sk, pc = api.sketch(rp, col, c.d, N, 7)
    return sk, pc


def _oracle_sketch(seed, n, N):
    """The oracle's own sketches of the batch _sketch(seed, n, N) sketches."""
    c = inputs.random_csr(seed, n, 50_000, 1, 400)
    return oracle.sketch(c.row_ptr, c.col, c.d, N, 7)[0]


def _unsharded(Q, pcQ, DB, pcDB, N, by, k, excl, variant):
    nQ, nDB = pcQ.numel(), pcDB.numel()
    s = torch.empty((nQ, k), dtype=torch.float32, device="cuda")
    i = torch.empty((nQ, k), dtype=torch.int32, device="cuda")
    wsb = B.bs_topk_workspace_bytes(nQ, nDB, N, k)
    ws = torch.empty((max(wsb, 256),), dtype=torch.uint8, device="cuda")
    B.bs_topk_ex(Q, pcQ, nQ, DB, pcDB, nDB, N, by, k, excl, s, i, ws, wsb, variant)
    return s, i


def _sharded(Q, pcQ, DB, pcDB, N, by, k, excl, variant, bounds):
    nQ = pcQ.numel()
    parts_s, parts_i = [], []
    for lo, hi in zip(bounds, bounds[1:]):
        s = torch.empty((nQ, k), dtype=torch.float32, device="cuda")
        i = torch.empty((nQ, k), dtype=torch.int32, device="cuda")
        wsb = B.bs_topk_workspace_bytes(nQ, hi - lo, N, k)
        ws = torch.empty((max(wsb, 256),), dtype=torch.uint8, device="cuda")
        B.bs_topk_shard(Q, pcQ, nQ, DB[lo:hi], pcDB[lo:hi], hi - lo, lo, N, by, k, excl, s, i,
                        ws, wsb, variant)
        parts_s.append(s)
        parts_i.append(i)
    sp, ip = torch.stack(parts_s), torch.stack(parts_i)
    out_s = torch.empty((nQ, k), dtype=torch.float32, device="cuda")
    out_i = torch.empty((nQ, k), dtype=torch.int32, device="cuda")
    B.bs_topk_merge(sp, ip, len(parts_s), nQ, k, bounds[:-1], by, out_s, out_i)
    assert B.bs_get_async_error() == 0
    return out_s, out_i


@pytest.mark.parametrize("variant", ["popc", "tc"])
@pytest.mark.parametrize("by", ["js", "ham", "cos", "ip"])
def test_all_pairs_sharded_equals_unsharded(variant, by):
    N, k = 1024, 20
    sk, pc = _sketch(11, 2500, N)
    bounds = [0, 700, 1717, 1730, 2500]          # ragged; one shard smaller than k
    v, m = B.VARIANTS[variant], B.MEASURE_BITS[by]
    ref_s, ref_i = _unsharded(sk, pc, sk, pc, N, m, k, True, v)
    got_s, got_i = _sharded(sk, pc, sk, pc, N, m, k, True, v, bounds)
    assert torch.equal(got_i, ref_i)
    assert torch.equal(got_s, ref_s)


@pytest.mark.parametrize("variant", ["popc", "tc"])
def test_query_vs_sharded_db_matches_oracle(variant):
    N, k = 2048, 50
    db, pdb = _sketch(21, 3000, N)
    q, pq = _sketch(22, 333, N)
    bounds = sharded.shard_offsets(3000, 3) + [3000]
    v = B.VARIANTS[variant]
    ref_s, ref_i = _unsharded(q, pq, db, pdb, N, B.BS_JS, k, False, v)
    got_s, got_i = _sharded(q, pq, db, pdb, N, B.BS_JS, k, False, v, bounds)
    assert torch.equal(got_i, ref_i) and torch.equal(got_s, ref_s)
    oq, odb = _oracle_sketch(22, 333, N), _oracle_sketch(21, 3000, N)
    assert np.array_equal(u32(q), oq) and np.array_equal(u32(db), odb)
    est, _ = oracle.estimate_pairs(oq, odb, N)
    gs, gi = got_s.cpu().numpy(), u32(got_i)
    for r in range(0, 333, 7):
        check_topk_row(gs[r], gi[r], est[oracle.JS][r], k, oracle.JS)


def test_sharded_topk_class_single_process():
    N, k = 1024, 10
    sk, pc = _sketch(31, 900, N)
    lo, hi = 300, 900
    st = sharded.ShardedTopK(sk[lo:hi], pc[lo:hi], lo, N, k, by="cos")
    s, i = st.search(sk, pc, exclude_self=True)
    # one process holds one shard: the result is that shard's top-k, global indices
    ref_s, ref_i = _unsharded(sk, pc, sk[lo:hi], pc[lo:hi], N, B.BS_COS, k, False, 0)
    ref_i = torch.where(ref_i >= 0, ref_i + lo, ref_i)
    rows = torch.arange(lo, hi, device="cuda")
    keep = torch.ones(900, dtype=torch.bool, device="cuda")
    keep[rows] = False               # rows inside the shard had their self pair dropped
    assert torch.equal(i[keep], ref_i[keep]) and torch.equal(s[keep], ref_s[keep])
    assert not (i[lo:hi] == rows[:, None]).any()


def test_merge_argument_errors():
    s = torch.zeros((1, 4, 5), device="cuda")
    i = torch.zeros((1, 4, 5), dtype=torch.int32, device="cuda")
    o_s = torch.empty((4, 5), device="cuda")
    o_i = torch.empty((4, 5), dtype=torch.int32, device="cuda")
    with pytest.raises(B.BinSketchError):
        B.bs_topk_merge(s, i, 0, 4, 5, None, B.BS_JS, o_s, o_i)
    with pytest.raises(B.BinSketchError):
        B.bs_topk_merge(s, i, B.BS_TOPK_MERGE_PARTS_MAX + 1, 4, 5, None, B.BS_JS, o_s, o_i)
    with pytest.raises(B.BinSketchError):
        B.bs_topk_merge(s, i, 1, 4, 0, None, B.BS_JS, o_s, o_i)
