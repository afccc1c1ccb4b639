"""Ranking-quality evaluation of Experiment 2 (Sec. 4): the oracle's
retrieval sets and the host-side split, gather and metric arithmetic,
pinned on hand-worked examples (no GPU)."""
import math

import numpy as np

import oracle
from paper_1910_04658_gb300 import inputs, ranking


def test_threshold_sets_hand_example():
    # one query, five training points; exact JS and estimates
    exact = np.array([[0.95, 0.90, 0.50, 0.10, 0.0]])
    est = np.array([[0.97, 0.85, 0.55, 0.12, 0.3]])
    cnt = oracle.threshold_sets(est, exact, [0.9, 0.5, 0.1])
    # thr 0.9: O = {0, 1}, O' = {0}          -> (2, 1, 1)
    # thr 0.5: O = {0, 1, 2}, O' = {0, 1, 2} -> (3, 3, 3)
    # thr 0.1: O = {0, 1, 2, 3}, O' = all 5  -> (4, 5, 4)
    assert cnt.tolist() == [[[2, 1, 1], [3, 3, 3], [4, 5, 4]]]
    # a distance (Hamming): retrieved when at most the threshold
    cnt = oracle.threshold_sets(np.array([[3.0, 7.0]]), np.array([[2.0, 9.0]]), [5.0], distance=True)
    assert cnt.tolist() == [[[1, 1, 1]]]


def test_metrics_hand_example():
    # |O| = 4, |O'| = 5, |O n O'| = 3: acc 3/6, P 3/5, R 3/4, F1 2PR/(P+R) = 2/3
    m = ranking.metrics(np.array([[[4, 5, 3]]]))[0]
    assert math.isclose(m["accuracy"], 0.5) and math.isclose(m["precision"], 0.6)
    assert math.isclose(m["recall"], 0.75) and math.isclose(m["f1"], 2 * 0.6 * 0.75 / 1.35)
    # undefined parts are left out of the means; pooled counts add up
    m = ranking.metrics(np.array([[[4, 5, 3]], [[0, 2, 0]], [[0, 0, 0]]]))[0]
    assert math.isclose(m["precision"], (0.6 + 0.0) / 2)
    assert math.isclose(m["recall"], 0.75) and m["queries_with_truth"] == 1
    assert math.isclose(m["accuracy"], (0.5 + 0.0) / 2)
    assert math.isclose(m["pooled_precision"], 3 / 7) and math.isclose(m["pooled_recall"], 3 / 4)
    assert m["truth_pairs"] == 4 and m["retrieved_pairs"] == 7


def test_split_and_take_rows():
    c = inputs.random_csr(3, 501, 10_000, 0, 40)
    q, t = ranking.split(c.n, seed=7)
    assert q.size == 50 and t.size == 451
    assert np.array_equal(np.sort(np.concatenate([q, t])), np.arange(c.n))
    sub = ranking.take_rows(c, q)
    for k, r in enumerate(q):
        a = c.col[c.row_ptr[r]:c.row_ptr[r + 1]]
        b = sub.col[sub.row_ptr[k]:sub.row_ptr[k + 1]]
        assert np.array_equal(a, b)
    assert ranking.split(c.n, seed=7)[0].tolist() == q.tolist()     # seeded


def test_oracle_ground_truth_matches_dense_vectors():
    # exact similarities from sorted-list intersection vs dense 0/1 vectors,
    # then the retrieval sets from them
    c = inputs.random_csr(5, 40, 300, 1, 60)
    dense = np.zeros((c.n, c.d), np.int64)
    for r in range(c.n):
        dense[r, c.col[c.row_ptr[r]:c.row_ptr[r + 1]]] = 1
    pa, pb = np.meshgrid(np.arange(5), np.arange(5, 40), indexing="ij")
    ex = oracle.exact_pairs(c.row_ptr, c.col, pa.ravel(), pb.ravel())[:, 2].reshape(5, 35)
    I = dense[:5] @ dense[5:].T
    U = dense[:5].sum(1)[:, None] + dense[5:].sum(1)[None, :] - I
    js = np.where(U > 0, I / np.maximum(U, 1), 0.0)
    assert np.array_equal(ex, js)
    cnt = oracle.threshold_sets(js, ex, ranking.THRESHOLDS)
    assert (cnt[:, :, 0] == cnt[:, :, 1]).all() and (cnt[:, :, 0] == cnt[:, :, 2]).all()
