"""Ranking-quality evaluation of Experiment 2 (Sec. 4, "Ranking") on the GPU.

The corpus is split at random into a training partition (90%) and a query
partition (10%).  For every query row and similarity threshold, the ground
truth O is the set of training rows whose exact similarity (from the
uncompressed vectors) reaches the threshold, and O' the set whose estimate
from the sketches (Alg. 1-4) does.  Per query: accuracy = |O n O'| / |O u O'|,
precision = |O n O'| / |O'|, recall = |O n O'| / |O|, F1 = 2PR / (P + R).

Thresholds: for Jaccard and cosine the paper's list {0.95, 0.9, 0.85, 0.8,
0.6, 0.5, 0.2, 0.1}; for inner product the same fractions of the largest
exact inner product between a query and a training row.  Each metric is the
mean over the queries for which it is defined (accuracy: O u O' not empty;
precision: O' not empty; recall: O not empty; F1: both), and the pooled
counts are reported beside it.

Device work runs in the library's kernels: the sketches (bs_sketch), the
estimates (bs_estimate_pairs), the exact common counts (bs_exact_counts) and
the retrieval-set counts (bs_threshold_eval).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import binding as B
from .inputs import CSR

THRESHOLDS = (0.95, 0.9, 0.85, 0.8, 0.6, 0.5, 0.2, 0.1)
MEASURE_INDEX = {"ip": 0, "ham": 1, "js": 2, "cos": 3}


def split(n: int, seed: int, query_frac: float = 0.1) -> Tuple[np.ndarray, np.ndarray]:
    """Random partition of rows 0..n-1: (query rows, training rows), each sorted."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    nq = max(1, int(round(n * query_frac))) if n > 1 else 0
    return np.sort(perm[:nq]), np.sort(perm[nq:])


def take_rows(c: CSR, rows: np.ndarray) -> CSR:
    """The CSR batch of the given rows, in that order."""
    rows = np.asarray(rows, np.int64)
    lens = (c.row_ptr[rows + 1] - c.row_ptr[rows]).astype(np.int64)
    rp = np.zeros(rows.size + 1, np.uint64)
    rp[1:] = np.cumsum(lens)
    starts = c.row_ptr[rows].astype(np.int64)
    idx = np.repeat(starts - rp[:-1].astype(np.int64), lens) + np.arange(int(rp[-1]), dtype=np.int64)
    return CSR(rp, c.col[idx].astype(np.uint32), c.d)


def metrics(cnt: np.ndarray) -> List[Dict[str, float]]:
    """cnt[q][t] = (|O|, |O'|, |O n O'|) -> per threshold the mean accuracy,
    precision, recall and F1 over the queries where each is defined, and the
    pooled (summed-count) values."""
    cnt = np.asarray(cnt, np.float64)
    out = []
    for t in range(cnt.shape[1]):
        o, r, i = cnt[:, t, 0], cnt[:, t, 1], cnt[:, t, 2]
        u = o + r - i
        with np.errstate(divide="ignore", invalid="ignore"):
            acc = np.where(u > 0, i / u, np.nan)
            prec = np.where(r > 0, i / r, np.nan)
            rec = np.where(o > 0, i / o, np.nan)
            both = (r > 0) & (o > 0)
            f1 = np.where(both & (prec + rec > 0), 2 * prec * rec / (prec + rec), np.where(both, 0.0, np.nan))

        def mean(x):
            x = x[~np.isnan(x)]
            return float(x.mean()) if x.size else float("nan")

        O, R, I = o.sum(), r.sum(), i.sum()
        pp = I / R if R else float("nan")
        pr = I / O if O else float("nan")
        out.append({"accuracy": mean(acc), "precision": mean(prec), "recall": mean(rec), "f1": mean(f1),
                    "queries_with_truth": int((o > 0).sum()), "pooled_precision": pp, "pooled_recall": pr,
                    "pooled_f1": (2 * pp * pr / (pp + pr)) if (O and R and pp + pr > 0) else float("nan"),
                    "truth_pairs": int(O), "retrieved_pairs": int(R)})
    return out


@dataclass
class Split:
    query: CSR
    train: CSR
    query_rows: np.ndarray
    train_rows: np.ndarray


class Evaluation:
    """Exact counts of one corpus split, kept on the device, and the
    per-threshold retrieval quality of BinSketch estimates at any N."""

    def __init__(self, c: CSR, seed: int = 0, query_frac: float = 0.1, device: str = "cuda"):
        import torch
        self.torch = torch
        qr, tr = split(c.n, seed, query_frac)
        self.split = Split(take_rows(c, qr), take_rows(c, tr), qr, tr)
        self.d = c.d
        self.device = device
        q, t = self.split.query, self.split.train
        self.nq, self.ndb = q.n, t.n
        dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a).view(dt)).to(device)
        self.q_rp, self.q_col = dev(q.row_ptr, np.int64), dev(q.col, np.int32)
        self.t_rp, self.t_col = dev(t.row_ptr, np.int64), dev(t.col, np.int32)
        self.counts = torch.empty((self.nq, self.ndb), dtype=torch.int32, device=device)
        self.q_sizes = torch.empty((self.nq,), dtype=torch.int32, device=device)
        self.t_sizes = torch.empty((self.ndb,), dtype=torch.int32, device=device)
        B.bs_exact_counts(self.q_rp, self.q_col, self.nq, q.nnz, self.t_rp, self.t_col, self.ndb, t.nnz,
                          self.d, self.counts, self.q_sizes, self.t_sizes)

    def max_inner_product(self) -> int:
        return int(self.torch.amax(self.counts).item())

    def thresholds(self, by: str) -> Tuple[float, ...]:
        if by in ("js", "cos"):
            return THRESHOLDS
        if by == "ip":
            m = self.max_inner_product()
            return tuple(f * m for f in THRESHOLDS)
        raise ValueError("ranking thresholds are defined for ip, js and cos")

    def sketches(self, N: int, hash_seed: int = 0):
        torch = self.torch
        out = []
        for rp, col, n, nnz in ((self.q_rp, self.q_col, self.nq, self.split.query.nnz),
                                (self.t_rp, self.t_col, self.ndb, self.split.train.nnz)):
            sk = torch.empty((n, N // 32), dtype=torch.int32, device=self.device)
            pc = torch.empty((n,), dtype=torch.int32, device=self.device)
            B.bs_sketch(rp, col, n, nnz, self.d, N, hash_seed, sk, pc)
            out.append((sk, pc))
        return out

    def evaluate(self, N: int, measures: Sequence[str] = ("js", "cos", "ip"), hash_seed: int = 0):
        """{measure: {"thresholds": [...], "metrics": [per-threshold dict], "counts": array}}"""
        torch = self.torch
        (qs, qp), (ts, tp) = self.sketches(N, hash_seed)
        bits = 0
        for m in measures:
            bits |= B.MEASURE_BITS[m]
        order = [m for m in ("ip", "ham", "js", "cos") if B.MEASURE_BITS[m] & bits]
        est = torch.empty((len(order), self.nq, self.ndb), dtype=torch.float32, device=self.device)
        B.bs_estimate_pairs(qs, qp, self.nq, ts, tp, self.ndb, N, bits, est, None)
        res = {}
        for m in measures:
            th = self.thresholds(m)
            out = torch.empty((self.nq, len(th), 3), dtype=torch.int32, device=self.device)
            B.bs_threshold_eval(est[order.index(m)], self.counts, self.q_sizes, self.t_sizes, self.nq,
                                self.ndb, B.MEASURE_BITS[m], th, out)
            cnt = out.cpu().numpy().view(np.uint32)
            res[m] = {"thresholds": list(th), "metrics": metrics(cnt), "counts": cnt}
        return res
