"""Ranking-quality evaluation (Experiment 2, Sec. 4) on the GPU vs the oracle:
exact common counts bit for bit, retrieval-set counts exactly (both sides
threshold the oracle's estimates, rounded to FP32 as the GPU path holds them,
in FP64), and the end-to-end evaluation."""
import numpy as np
import pytest

import oracle
from paper_1910_04658_gb300 import inputs, ranking
from tests.helpers import to_dev, u32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1910_04658_gb300 import api, binding as B  # noqa: E402


def _counts(q, t, d):
    q_rp, q_col = to_dev(q)
    t_rp, t_col = to_dev(t)
    cnt = torch.empty((q.n, t.n), dtype=torch.int32, device="cuda")
    qs = torch.empty((q.n,), dtype=torch.int32, device="cuda")
    ts = torch.empty((t.n,), dtype=torch.int32, device="cuda")
    B.bs_exact_counts(q_rp, q_col, q.n, q.nnz, t_rp, t_col, t.n, t.nnz, d, cnt, qs, ts)
    assert B.bs_get_async_error() == 0
    return cnt, qs, ts


def _oracle_exact(q, t):
    both = inputs.CSR(np.concatenate([q.row_ptr, q.row_ptr[-1] + t.row_ptr[1:]]).astype(np.uint64),
                      np.concatenate([q.col, t.col]).astype(np.uint32), q.d)
    pa, pb = np.meshgrid(np.arange(q.n), q.n + np.arange(t.n), indexing="ij")
    return oracle.exact_pairs(both.row_ptr, both.col, pa.ravel(), pb.ravel()).reshape(q.n, t.n, 4)


@pytest.mark.parametrize("d", [1000, 100_000, 1_572_864])
def test_exact_counts_bit_exact(d):
    c = inputs.random_csr(d % 97, 700, d, 0, 300)
    qr, tr = ranking.split(c.n, seed=1)
    q, t = ranking.take_rows(c, qr), ranking.take_rows(c, tr)
    cnt, qs, ts = _counts(q, t, d)
    ex = _oracle_exact(q, t)
    assert np.array_equal(u32(cnt).astype(np.float64), ex[:, :, 0])
    assert np.array_equal(u32(qs), np.diff(q.row_ptr).astype(np.uint32))
    assert np.array_equal(u32(ts), np.diff(t.row_ptr).astype(np.uint32))


def test_exact_counts_query_duplicates_and_bad_index():
    d = 5000
    q = inputs.CSR(np.array([0, 5, 5], np.uint64), np.array([3, 3, 9, 4999, 9], np.uint32), d)
    t = inputs.CSR(np.array([0, 3, 4], np.uint64), np.array([3, 9, 17, 4999], np.uint32), d)
    cnt, qs, _ = _counts(q, t, d)
    assert u32(cnt).tolist() == [[2, 1], [0, 0]] and u32(qs).tolist() == [3, 0]
    bad = inputs.CSR(t.row_ptr, np.array([3, 9, 5000, 1], np.uint32), d)
    q_rp, q_col = to_dev(q)
    b_rp, b_col = to_dev(bad)
    out = torch.empty((2, 2), dtype=torch.int32, device="cuda")
    B.bs_exact_counts(q_rp, q_col, 2, q.nnz, b_rp, b_col, 2, bad.nnz, d, out)
    assert B.bs_get_async_error() == 2      # BS_ERR_INDEX_RANGE
    with pytest.raises(B.BinSketchError):
        B.bs_exact_counts(q_rp, q_col, 2, q.nnz, b_rp, b_col, 2, bad.nnz, B.BS_EXACT_D_MAX + 1, out)


@pytest.mark.parametrize("N", [256, 2048])
def test_threshold_eval_matches_oracle(N):
    c = inputs.random_csr(17, 1200, 50_000, 1, 250)
    qr, tr = ranking.split(c.n, seed=3)
    q, t = ranking.take_rows(c, qr), ranking.take_rows(c, tr)
    cnt, qs, ts = _counts(q, t, c.d)
    ex = _oracle_exact(q, t)
    assert np.array_equal(u32(cnt).astype(np.float64), ex[:, :, 0])
    # the estimates both sides threshold: the oracle's, from its own sketches,
    # rounded to the FP32 the GPU path keeps them in
    oqs, _ = oracle.sketch(q.row_ptr, q.col, c.d, N, 4)
    ots, _ = oracle.sketch(t.row_ptr, t.col, c.d, N, 4)
    e32 = oracle.estimate_pairs(oqs, ots, N)[0].astype(np.float32)
    est = torch.from_numpy(e32).cuda()
    e = e32.astype(np.float64)
    max_ip = float(ex[:, :, 0].max())
    cases = [("js", 2, ranking.THRESHOLDS), ("cos", 3, ranking.THRESHOLDS),
             ("ip", 0, tuple(f * max_ip for f in ranking.THRESHOLDS)), ("ham", 1, (5.0, 40.0, 200.0, 400.0))]
    for by, m, th in cases:
        out = torch.empty((q.n, len(th), 3), dtype=torch.int32, device="cuda")
        B.bs_threshold_eval(est[m], cnt, qs, ts, q.n, t.n, B.MEASURE_BITS[by], th, out)
        ref = oracle.threshold_sets(e[m], ex[:, :, m], th, distance=(by == "ham"))
        assert np.array_equal(u32(out).astype(np.int64), ref), by


def test_evaluation_end_to_end():
    c = inputs.random_csr(23, 3000, 200_000, 5, 300)
    ev = ranking.Evaluation(c, seed=0)
    assert ev.nq == 300 and ev.ndb == 2700
    lo, hi = ev.evaluate(256, ("js", "cos", "ip")), ev.evaluate(4096, ("js", "cos", "ip"))
    assert B.bs_get_async_error() == 0
    for res in (lo, hi):
        for by in ("js", "cos", "ip"):
            cnt = res[by]["counts"]
            assert (cnt[:, :, 2] <= np.minimum(cnt[:, :, 0], cnt[:, :, 1])).all()
            # thresholds fall: the ground-truth sets only grow
            assert (np.diff(cnt[:, :, 0].astype(np.int64), axis=1) >= 0).all()
    # the near-duplicate rows give ground truth at the high thresholds, and a
    # 16x longer sketch retrieves it at least as well (pooled F1 at JS >= 0.5)
    t = ranking.THRESHOLDS.index(0.5)
    assert hi["js"]["metrics"][t]["truth_pairs"] > 0
    assert hi["js"]["metrics"][t]["pooled_f1"] >= lo["js"]["metrics"][t]["pooled_f1"] - 0.02
