"""CUDA path vs the FP64 oracle, through the C ABI.

Sketches, popcounts and common-bit counts must match bit for bit; estimates
within the tolerance of tests/helpers.py; top-k lists by the tolerance-band
rule.  Sizes span several tiles with ragged tails; the full text-BoW workload
(100,000 x 1,000,000, N = 4096, top-50 by Jaccard) runs in the launch
configuration the benchmark uses and is checked on sampled query rows.
"""
import numpy as np
import pytest

import oracle
from paper_1910_04658_gb300 import inputs
from tests.helpers import assert_close, check_topk_row, to_dev, u32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1910_04658_gb300 import api, binding as B  # noqa: E402


@pytest.fixture(scope="module")
def tiny():
    return inputs.tiny_corpus(0)


def _gpu_sketch(c, N, seed, parity=False):
    rp, col = to_dev(c)
    sk, pc = api.sketch(rp, col, c.d, N, seed, parity=parity)
    assert B.bs_get_async_error() == 0
    return sk, pc


def _sketch_both(c, N, seed):
    """The GPU's sketches of a CSR batch (device) and the oracle's own
    sketches of the same batch (host), checked equal bit for bit.  The
    oracle's estimates are computed from the oracle's copy: no oracle input
    comes from the GPU."""
    sk, pc = _gpu_sketch(c, N, seed)
    osk, opc = oracle.sketch(c.row_ptr, c.col, c.d, N, seed)
    assert np.array_equal(u32(sk), osk) and np.array_equal(u32(pc), opc)
    return sk, pc, osk


# ------------------------------------------------------------------ sketching

def test_sketch_tiny_corpus_bit_exact(tiny):
    N = 1024
    sk, pc = _gpu_sketch(tiny, N, 0)
    osk, opc = oracle.sketch(tiny.row_ptr, tiny.col, tiny.d, N, 0)
    assert np.array_equal(u32(sk), osk)
    assert np.array_equal(u32(pc), opc)


@pytest.mark.parametrize("N", [32, 96, 256, 1024, 4096, 8192, 65536])
def test_sketch_sizes_bit_exact(N):
    c = inputs.random_csr(N % 977, 333, 200_000, 0, 700)
    sk, pc = _gpu_sketch(c, N, 12345)
    osk, opc = oracle.sketch(c.row_ptr, c.col, c.d, N, 12345)
    assert np.array_equal(u32(sk), osk) and np.array_equal(u32(pc), opc)


def test_sketch_unaligned_column_pointer_and_empty_rows():
    c = inputs.random_csr(5, 257, 50_000, 0, 90)
    N = 512
    osk, opc = oracle.sketch(c.row_ptr, c.col, c.d, N, 3)
    for shift in (1, 2, 3, 4, 5):
        # the same rows stored `shift` words into the column buffer: every
        # offset of the first 16-byte boundary the kernel peels up to
        col = torch.zeros(c.col.size + 8, dtype=torch.int32, device="cuda")
        col[shift:shift + c.col.size] = torch.from_numpy(c.col.view(np.int32)).cuda()
        rp = torch.from_numpy(c.row_ptr.view(np.int64)).cuda()
        sk = torch.empty((c.n, N // 32), dtype=torch.int32, device="cuda")
        pc = torch.empty((c.n,), dtype=torch.int32, device="cuda")
        B.bs_sketch(rp, col.data_ptr() + 4 * shift, c.n, c.nnz, c.d, N, 3, sk, pc)
        assert B.bs_get_async_error() == 0
        assert np.array_equal(u32(sk), osk) and np.array_equal(u32(pc), opc)


def test_sketch_long_rows_and_duplicates():
    rng = np.random.default_rng(2)
    sizes = [0, 1, 5000, 12000, 33, 4096, 4088, 4089, 4085, 3, 0, 4087, 2, 4088]
    rows = [rng.integers(0, 1000, int(m)).astype(np.uint32) for m in sizes]
    rp = np.zeros(len(rows) + 1, np.uint64)
    rp[1:] = np.cumsum([r.size for r in rows])
    c = inputs.CSR(rp, np.concatenate(rows).astype(np.uint32), 1000)
    for N in (64, 2048):
        sk, pc = _gpu_sketch(c, N, 77)
        osk, opc = oracle.sketch(c.row_ptr, c.col, c.d, N, 77)
        assert np.array_equal(u32(sk), osk) and np.array_equal(u32(pc), opc)


@pytest.mark.parametrize("N", [64, 4096])
def test_sketch_many_short_rows(N):
    # 40,000 rows of 0-3 indices: most of a row's lanes idle, empty rows,
    # several rows per warp (the grid strides over them)
    rng = np.random.default_rng(N)
    n = 40_000
    nnz = rng.integers(0, 4, n)
    rp = np.zeros(n + 1, np.uint64)
    rp[1:] = np.cumsum(nnz)
    col = rng.integers(0, 70_000, int(rp[-1])).astype(np.uint32)
    c = inputs.CSR(rp, col, 70_000)
    for parity in (False, True):
        sk, pc = _gpu_sketch(c, N, 5, parity=parity)
        osk, opc = oracle.sketch(c.row_ptr, c.col, c.d, N, 5, parity=parity)
        assert np.array_equal(u32(sk), osk) and np.array_equal(u32(pc), opc)


def test_bcs_parity_sketch_bit_exact(tiny):
    sk, pc = _gpu_sketch(tiny, 1024, 4, parity=True)
    osk, opc = oracle.sketch(tiny.row_ptr, tiny.col, tiny.d, 1024, 4, parity=True)
    assert np.array_equal(u32(sk), osk) and np.array_equal(u32(pc), opc)


def test_sketch_data_errors_are_reported_not_faulted():
    c = inputs.random_csr(9, 40, 1000, 1, 30)
    bad = c.col.copy()
    r = 7
    bad[int(c.row_ptr[r])] = 1000          # == d: out of range
    c2 = inputs.CSR(c.row_ptr, bad, c.d)
    rp, col = to_dev(c2)
    sk, pc = api.sketch(rp, col, c.d, 256, 1)
    assert B.bs_get_async_error() == 2      # BS_ERR_INDEX_RANGE
    assert B.bs_get_async_error() == 0      # cleared
    osk, opc = oracle.sketch(c.row_ptr, c.col, c.d, 256, 1)
    got, gpc = u32(sk), u32(pc)
    assert not got[r].any() and gpc[r] == 0
    keep = np.arange(c.n) != r
    assert np.array_equal(got[keep], osk[keep])
    # decreasing row offsets and an offset past nnz
    rp_bad = c.row_ptr.copy()
    rp_bad[3], rp_bad[4] = rp_bad[4], rp_bad[3]
    rp_t = torch.from_numpy(rp_bad.view(np.int64)).cuda()
    sk2 = torch.empty((c.n, 8), dtype=torch.int32, device="cuda")
    B.bs_sketch(rp_t, col, c.n, c.nnz, c.d, 256, 1, sk2, None)
    assert B.bs_get_async_error() == 3      # BS_ERR_ROWPTR
    with pytest.raises(B.BinSketchError):
        B.bs_sketch(rp_t, col, c.n, c.nnz, c.d, 100, 1, sk2, None)   # N not a multiple of 32


def test_popcount_rows(tiny):
    sk, pc = _gpu_sketch(tiny, 1024, 0)
    pc2 = torch.empty_like(pc)
    B.bs_popcount_rows(sk, tiny.n, 1024, pc2)
    assert np.array_equal(u32(pc2), u32(pc))


# --------------------------------------------------------- counts + estimates

def _check_pairs(Ask, Apc, oA, Bsk, Bpc, oB, N):
    out, cnt = api.estimate_pairs(Ask, Apc, Bsk, Bpc, N)
    oest, ocnt = oracle.estimate_pairs(oA, oB, N)
    assert np.array_equal(u32(cnt), ocnt)
    for m in range(4):
        assert_close(out[m].cpu().numpy(), oest[m], m)


def test_estimates_tiny_corpus_all_pairs(tiny):
    N = 1024
    sk, pc, osk = _sketch_both(tiny, N, 0)
    _check_pairs(sk, pc, osk, sk, pc, osk, N)


@pytest.mark.parametrize("N", [96, 256, 1024, 4096, 8192])
def test_estimates_ragged_tiles(N):
    a = inputs.random_csr(1, 77, 300_000, 1, 900)
    b = inputs.random_csr(2, 301, 300_000, 1, 900)
    ask, apc, oa = _sketch_both(a, N, 5)
    bsk, bpc, ob = _sketch_both(b, N, 5)
    _check_pairs(ask, apc, oa, bsk, bpc, ob, N)


@pytest.mark.parametrize("N", [256, 1024])
def test_estimates_saturated_regime(N):
    # nnz uniform in [N/4, 4N]: sketches near saturation (clamp reading)
    # plus a few rows of 20N columns, whose sketches fill up (|a_s| = N)
    c = inputs.uniform_csr(3, 90, 100_000, N // 4, 4 * N)
    f = inputs.uniform_csr(4, 6, 100_000, 20 * N, 20 * N)
    rp = np.concatenate([c.row_ptr, f.row_ptr[1:] + c.row_ptr[-1]]).astype(np.uint64)
    c = inputs.CSR(rp, np.concatenate([c.col, f.col]), c.d)
    sk, pc, osk = _sketch_both(c, N, 8)
    assert (u32(pc) == N).any()
    _check_pairs(sk, pc, osk, sk, pc, osk, N)


def test_estimates_measure_subsets_and_counts_only(tiny):
    N = 1024
    sk, pc, osk = _sketch_both(tiny, N, 0)
    oest, ocnt = oracle.estimate_pairs(osk[:50], osk[:70], N)
    out, cnt = api.estimate_pairs(sk[:50], pc[:50], sk[:70], pc[:70], N, measures=("js", "cos"))
    assert_close(out[0].cpu().numpy(), oest[2], 2)
    assert_close(out[1].cpu().numpy(), oest[3], 3)
    out2, cnt2 = api.estimate_pairs(sk[:50], pc[:50], sk[:70], pc[:70], N, measures=())
    assert out2 is None and np.array_equal(u32(cnt2), ocnt)


# ------------------------------------------------------------------------ top-k

@pytest.mark.parametrize("variant", ["popc", "tc"])
@pytest.mark.parametrize("by,m", [("js", 2), ("cos", 3), ("ip", 0), ("ham", 1)])
@pytest.mark.parametrize("k", [1, 20, 50, 100, 128])
def test_topk_all_pairs_tiny(tiny, by, m, k, variant):
    N = 1024
    sk, pc, osk = _sketch_both(tiny, N, 0)
    score, idx = api.topk(sk, pc, sk, pc, N, k, by=by, exclude_self=True, variant=variant)
    oest, _ = oracle.estimate_pairs(osk, osk, N)
    s, ix = score.cpu().numpy(), u32(idx)
    for q in range(tiny.n):
        check_topk_row(s[q], ix[q], oest[m, q], k, m, exclude_q=q)


@pytest.mark.parametrize("variant", ["popc", "tc"])
def test_topk_fewer_db_rows_than_k(tiny, variant):
    N = 1024
    sk, pc, osk = _sketch_both(tiny, N, 0)
    score, idx = api.topk(sk[:40], pc[:40], sk[:30], pc[:30], N, 50, by="js", variant=variant)
    oest, _ = oracle.estimate_pairs(osk[:40], osk[:30], N)
    for q in range(40):
        check_topk_row(score[q].cpu().numpy(), u32(idx[q]), oest[2, q], 50, 2)


@pytest.mark.parametrize("variant", ["popc", "tc"])
@pytest.mark.parametrize("N,by,m", [(4096, "js", 2), (1024, "cos", 3), (256, "ham", 1),
                                    (8192, "ip", 0)])
def test_topk_split_database_merge(N, by, m, variant):
    # few queries against a large database: the database is split across
    # blocks and the per-split lists are merged by a second kernel
    db = inputs.random_csr(11, 20_000, 1_000_000, 1, 400)
    q = inputs.random_csr(12, 37, 1_000_000, 1, 400)
    dsk, dpc, odb = _sketch_both(db, N, 2)
    qsk, qpc, oq = _sketch_both(q, N, 2)
    assert B.bs_topk_workspace_bytes(37, 20_000, N, 100) > 0
    score, idx = api.topk(qsk, qpc, dsk, dpc, N, 100, by=by, variant=variant)
    oest, _ = oracle.estimate_pairs(oq, odb, N)
    s, ix = score.cpu().numpy(), u32(idx)
    for r in range(37):
        check_topk_row(s[r], ix[r], oest[m, r], 100, m)


@pytest.mark.parametrize("same", [False, True])
def test_topk_aligned_parts_after_rounds(same):
    # a database whose FP4 copy (N / 2 bytes a row, 82 MB here) is too large to
    # stay in L2: the query rows left after the rounds of whole row blocks run
    # with every row block cut into the same aligned parts of the database
    # (rows ending inside a 240-row tile, a ragged last query block), merged
    # by the call -- bit for bit the CUDA-core kernel's lists
    N, k = 4096, 50
    dc = inputs.random_csr(42, 40_001, 1_000_000, 1, 400)
    ds, dp = _gpu_sketch(dc, N, 6)
    if same:
        qs, qp, nq = ds, dp, dc.n
    else:
        qc = inputs.random_csr(41, 20_000, 1_000_000, 1, 400)
        qs, qp = _gpu_sketch(qc, N, 6)
        nq = qc.n
    uses_tc, splits, launches = B.bs_topk_plan(nq, dc.n, N, k, B.BS_VARIANT_TC, int(same))
    assert uses_tc and splits > 1
    ref_s, ref_i = api.topk(qs, qp, ds, dp, N, k, by="js", exclude_self=same, variant="popc")
    s, i = api.topk(qs, qp, ds, dp, N, k, by="js", exclude_self=same, variant="tc")
    assert B.bs_get_async_error() == 0
    assert torch.equal(i, ref_i) and torch.equal(s, ref_s)


@pytest.mark.parametrize("N,by,m", [(256, "ip", 0), (1024, "js", 2), (8192, "cos", 3)])
def test_topk_tc_dense_and_saturated(N, by, m):
    # counts up to N: the FP4 products must still sum exactly in FP32
    c = inputs.uniform_csr(3, 300, 100_000, N // 4, 4 * N)
    f = inputs.uniform_csr(4, 6, 100_000, 20 * N, 20 * N)
    rp = np.concatenate([c.row_ptr, f.row_ptr[1:] + c.row_ptr[-1]]).astype(np.uint64)
    c = inputs.CSR(rp, np.concatenate([c.col, f.col]), c.d)
    sk, pc, osk = _sketch_both(c, N, 8)
    oest, _ = oracle.estimate_pairs(osk, osk, N)
    for variant in ("tc", "popc"):
        score, idx = api.topk(sk, pc, sk, pc, N, 30, by=by, exclude_self=True, variant=variant)
        s, ix = score.cpu().numpy(), u32(idx)
        for q in range(c.n):
            check_topk_row(s[q], ix[q], oest[m, q], 30, m, exclude_q=q)


@pytest.mark.parametrize("cfg", range(B.BS_TC_CONFIGS))
@pytest.mark.parametrize("N,by,k", [(1024, "js", 50), (4096, "ham", 20), (256, "cos", 100), (2048, "ip", 1)])
def test_topk_tc_block_configurations_agree(cfg, N, by, k):
    # every operand-slot width / ring depth / epilogue split gives the same
    # lists as the CUDA-core kernel, bit for bit
    c = inputs.random_csr(21, 1500, 300_000, 1, 500)
    sk, pc = _gpu_sketch(c, N, 9)
    n = c.n
    ref_s, ref_i = api.topk(sk, pc, sk, pc, N, k, by=by, exclude_self=True, variant="popc")
    s = torch.empty((n, k), dtype=torch.float32, device="cuda")
    i = torch.empty((n, k), dtype=torch.int32, device="cuda")
    wsb = B.bs_topk_workspace_bytes(n, n, N, k)
    ws = torch.empty((wsb,), dtype=torch.uint8, device="cuda")
    try:
        B.bs_topk_ex(sk, pc, n, sk, pc, n, N, B.MEASURE_BITS[by], k, 1, s, i, ws, wsb,
                     B.BS_VARIANT_TC | B.BS_VARIANT_TC_CFG(cfg))
    except B.BinSketchError as e:
        assert e.code == 7     # this configuration's heaps do not fit k
        return
    assert B.bs_get_async_error() == 0
    assert torch.equal(i, ref_i) and torch.equal(s, ref_s)


@pytest.mark.parametrize("cfg", range(B.BS_TC_FIRST_TMA, B.BS_TC_CONFIGS))
@pytest.mark.parametrize("N,by", [(384, "js"), (640, "ip"), (8192, "cos")])
def test_topk_tma_database_operand_ragged(cfg, N, by):
    # the configurations that read the FP4 database copy by TMA: a database
    # whose rows end inside a 208-row tile (rows past the end arrive as zeros)
    # and N with an odd number of 128-bit chunks (the last 256-bit slot is
    # half outside the row); queries against another matrix, no self pair --
    # bit for bit the CUDA-core kernel's lists
    k = 20
    qc = inputs.random_csr(31, 300, 300_000, 1, 400)
    dc = inputs.random_csr(32, 1000, 300_000, 1, 400)
    qs, qp = _gpu_sketch(qc, N, 4)
    ds, dp = _gpu_sketch(dc, N, 4)
    ref_s, ref_i = api.topk(qs, qp, ds, dp, N, k, by=by, variant="popc")
    s = torch.empty((qc.n, k), dtype=torch.float32, device="cuda")
    i = torch.empty((qc.n, k), dtype=torch.int32, device="cuda")
    wsb = B.bs_topk_workspace_bytes(qc.n, dc.n, N, k)
    ws = torch.empty((wsb,), dtype=torch.uint8, device="cuda")
    B.bs_topk_ex(qs, qp, qc.n, ds, dp, dc.n, N, B.MEASURE_BITS[by], k, 0, s, i, ws, wsb,
                 B.BS_VARIANT_TC | B.BS_VARIANT_TC_CFG(cfg))
    assert B.bs_get_async_error() == 0
    assert torch.equal(i, ref_i) and torch.equal(s, ref_s)


def test_topk_tc_rejects_unsupported_shapes(tiny):
    sk, pc, osk = _sketch_both(tiny, 96, 0)
    score = torch.empty((10, 5), dtype=torch.float32, device="cuda")
    idx = torch.empty((10, 5), dtype=torch.int32, device="cuda")
    with pytest.raises(B.BinSketchError) as e:     # N = 96: not a multiple of 128
        B.bs_topk_ex(sk, pc, 10, sk, pc, 100, 96, B.BS_JS, 5, 0, score, idx, None, 0, B.BS_VARIANT_TC)
    assert e.value.code == 7
    # the automatic choice falls back to the CUDA-core kernel and still works
    s2, i2 = api.topk(sk[:10], pc[:10], sk[:100], pc[:100], 96, 5, by="js")
    oest, _ = oracle.estimate_pairs(osk[:10], osk[:100], 96)
    for q in range(10):
        check_topk_row(s2[q].cpu().numpy(), u32(i2[q]), oest[2, q], 5, 2)


def test_topk_rejects_small_workspace():
    N = 1024
    db = inputs.random_csr(1, 5000, 100_000, 1, 100)
    dsk, dpc = _gpu_sketch(db, N, 0)
    need = B.bs_topk_workspace_bytes(3, 5000, N, 10)
    assert need > 16
    score = torch.empty((3, 10), dtype=torch.float32, device="cuda")
    idx = torch.empty((3, 10), dtype=torch.int32, device="cuda")
    ws = torch.empty((16,), dtype=torch.uint8, device="cuda")
    for variant in (B.BS_VARIANT_AUTO, B.BS_VARIANT_POPC, B.BS_VARIANT_TC):
        with pytest.raises(B.BinSketchError) as e:
            B.bs_topk_ex(dsk, dpc, 3, dsk, dpc, 5000, N, B.BS_JS, 10, 0, score, idx, ws, 16, variant)
        assert e.value.code == 5


# --------------------------------------------- full text-BoW workload (sampled)

@pytest.fixture(scope="module")
def bow():
    return inputs.bow_corpus(0)


def test_bow_scale_sketch_and_topk50_sampled(bow):
    N, k = 4096, 50
    # all 100,000 sketches and counts bit exact against the oracle's own
    sk, pc, osk = _sketch_both(bow, N, 0)
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(bow.n, 64, replace=False))
    # all-pairs top-50 by Jaccard, the benchmark's launch, checked on sampled queries
    score, idx = api.topk(sk, pc, sk, pc, N, k, by="js", exclude_self=True)
    assert B.bs_get_async_error() == 0
    s, ix = score.cpu().numpy(), u32(idx)
    # both counting kernels feed identical integer counts to identical FP32
    # arithmetic, so the two variants must agree exactly
    s_p, i_p = api.topk(sk, pc, sk, pc, N, k, by="js", exclude_self=True, variant="popc")
    assert np.array_equal(u32(i_p), ix)
    assert np.array_equal(s_p.cpu().numpy(), s)
    q = rows[:24]
    oest, _ = oracle.estimate_pairs(osk[q], osk, N)
    for t, r in enumerate(q):
        check_topk_row(s[r], ix[r], oest[2, t], k, 2, exclude_q=int(r))
