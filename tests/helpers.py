"""Shared helpers of the parity tests: device transfer and the comparison rules.

Tolerances (estimates are FP32 on the GPU, FP64 in the oracle):
    |gpu - oracle| <= 1e-5 * max(|oracle|, floor)
with floor 0.1 set elements for IP and Ham (estimates at or near 0 occur when
a*b = N*c; 0.1 is far below the estimator's own spread, Lemma 4) and 1e-7 for
JS and Cos.  Counts and sketches are compared bit for bit.
"""
import numpy as np

REL = 1e-5
FLOORS = {0: 0.1, 1: 0.1, 2: 1e-7, 3: 1e-7}   # IP, Ham, JS, Cos


def to_dev(csr, device="cuda"):
    import torch
    rp = torch.from_numpy(np.ascontiguousarray(csr.row_ptr).view(np.int64)).to(device)
    col = torch.from_numpy(np.ascontiguousarray(csr.col).view(np.int32)).to(device)
    return rp, col


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def dev_u32(a, device="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).to(device)


def assert_close(gpu, ref, measure):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    tol = REL * np.maximum(np.abs(ref), FLOORS[measure])
    bad = np.abs(gpu - ref) > tol
    if bad.any():
        i = np.flatnonzero(bad.ravel())[:5]
        raise AssertionError(f"measure {measure}: {bad.sum()} of {bad.size} outside tolerance; "
                             f"gpu={gpu.ravel()[i]} oracle={ref.ravel()[i]}")


def check_topk_row(g_score, g_idx, o_row_scores, k, measure, exclude_q=None):
    """Tolerance-band parity of one query row's top-k.

    o_row_scores: oracle estimates of this query against every DB row.
    (i) every returned index carries the oracle's score within tolerance;
    (ii) every DB row whose oracle score beats the oracle's k-th best by more
         than the tolerance is returned;
    (iii) the returned scores are ordered best first, indices are distinct;
    (iv) unused slots are (-inf | +inf for Ham, 0xFFFFFFFF)."""
    sign = -1.0 if measure == 1 else 1.0
    cand = np.arange(o_row_scores.size)
    if exclude_q is not None:
        cand = cand[cand != exclude_q]
    n_valid = min(k, cand.size)
    g_idx = np.asarray(g_idx, np.uint32)
    g_score = np.asarray(g_score, np.float64)
    used = g_idx[:n_valid].astype(np.int64)
    assert np.all(g_idx[n_valid:] == 0xFFFFFFFF)
    if n_valid < k:
        assert np.all(g_score[n_valid:] == (np.inf if measure == 1 else -np.inf))
    assert np.all(used < o_row_scores.size)
    assert len(set(used.tolist())) == n_valid
    if exclude_q is not None:
        assert exclude_q not in set(used.tolist())
    assert_close(g_score[:n_valid], o_row_scores[used], measure)
    key = sign * g_score[:n_valid]
    assert np.all(np.diff(key) <= 1e-12)
    if n_valid:
        okey = np.sort(sign * o_row_scores[cand])[::-1]
        kth = okey[n_valid - 1]
        tol = REL * max(abs(kth), FLOORS[measure])
        must = cand[sign * o_row_scores[cand] > kth + 2 * tol]
        missing = set(must.tolist()) - set(used.tolist())
        assert not missing, f"missing {sorted(missing)[:5]}"
