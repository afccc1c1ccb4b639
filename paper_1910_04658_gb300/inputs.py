"""Seeded synthetic inputs shaped like bag-of-words corpora.

This module only draws random data; it holds none of BinSketch's arithmetic and
serves the CUDA path and the CPU oracle alike.  The paper's corpora (NYTimes,
Enron, KOS, BBC; Sec. 4 "Datasets") are sparse binary bag-of-words matrices
with power-law feature frequencies; they are not available here, so these
generators stand in for them:

* per-row nnz: Zipf(1.1) clipped to [5, 200], log-normal (median m, sigma)
  clipped to [lo, hi], or uniform;
* columns: Zipf(s = 1.0) over feature ranks 1..d (inverse CDF over the
  harmonic weights), mapped to column ids through a seeded permutation so hot
  features are not index-adjacent; no repeats within a row; rows are stored
  as uint32 CSR with uint64 row offsets and increasing columns;
* near-duplicates: a fraction of rows (default 20%) are children of another
  row -- each parent column is kept with probability p ~ U[0.5, 1] and the row
  is topped up with fresh Zipf draws -- because the paper's experiments look
  at pairs above a similarity threshold (Sec. 4, Experiments 1-2), which
  independent power-law rows would almost never produce.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    row_ptr: np.ndarray  # uint64 [n + 1]
    col: np.ndarray      # uint32 [nnz]
    d: int

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def row(self, r: int) -> np.ndarray:
        return self.col[int(self.row_ptr[r]):int(self.row_ptr[r + 1])]

    def slice(self, r0: int, r1: int) -> "CSR":
        b, e = int(self.row_ptr[r0]), int(self.row_ptr[r1])
        return CSR((self.row_ptr[r0:r1 + 1] - np.uint64(b)).astype(np.uint64),
                   self.col[b:e].copy(), self.d)


class ZipfColumns:
    """Column ids drawn from Zipf(s) over ranks, through a rank->id permutation."""

    def __init__(self, rng: np.random.Generator, d: int, s: float = 1.0, permute: bool = True):
        w = 1.0 / np.power(np.arange(1, d + 1, dtype=np.float64), s)
        cdf = np.cumsum(w)
        cdf /= cdf[-1]
        self.cdf = cdf
        self.perm = (rng.permutation(d).astype(np.uint32) if permute
                     else np.arange(d, dtype=np.uint32))
        self.d = d

    def draw(self, rng: np.random.Generator, m: int) -> np.ndarray:
        r = np.searchsorted(self.cdf, rng.random(m), side="right")
        np.minimum(r, self.d - 1, out=r)
        return self.perm[r]


def nnz_zipf_clipped(rng, n, a=1.1, lo=5, hi=200):
    return np.clip(rng.zipf(a, n), lo, hi).astype(np.int64)


def nnz_lognormal(rng, n, median, sigma=1.0, lo=1, hi=5000):
    x = rng.lognormal(np.log(median), sigma, n)
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


def _sorted_unique(x: np.ndarray) -> np.ndarray:
    x = np.sort(x)
    if x.size:
        keep = np.empty(x.size, bool)
        keep[0] = True
        np.not_equal(x[1:], x[:-1], out=keep[1:])
        x = x[keep]
    return x


def _fill_unique(rng, target, rows0, cols0, draw, d):
    """Complete every row r to exactly target[r] distinct columns.

    (rows0, cols0) are initial entries (may repeat); fresh columns come from
    draw(m).  Returns sorted unique keys row * d + col."""
    n = target.shape[0]
    done = []
    key = _sorted_unique(rows0.astype(np.int64) * d + cols0.astype(np.int64))
    active = np.arange(n, dtype=np.int64)
    tgt = target.copy()
    while True:
        rws = key // d
        have = np.bincount(rws, minlength=n)
        full = have[active] >= tgt[active]
        if full.any():
            fin = np.zeros(n, bool)
            fin[active[full]] = True
            sel = fin[rws]
            done.append(key[sel])
            key = key[~sel]
            active = active[~full]
        if active.size == 0:
            break
        need = (tgt[active] - have[active])
        m = int(need.sum())
        r_new = np.repeat(active, need)
        c_new = draw(m).astype(np.int64)
        key = _sorted_unique(np.concatenate([key, r_new * d + c_new]))
    out = np.concatenate(done) if done else np.zeros(0, np.int64)
    out.sort()
    return out


def powerlaw_csr(rng: np.random.Generator, n: int, d: int, nnz: np.ndarray,
                 s: float = 1.0, child_frac: float = 0.2, permute: bool = True) -> CSR:
    """n rows over d columns with the given per-row nnz (see module doc)."""
    nnz = np.minimum(np.asarray(nnz, np.int64), d)
    zc = ZipfColumns(rng, d, s, permute)
    n_child = int(round(child_frac * n)) if n > 1 else 0
    is_child = np.zeros(n, bool)
    if n_child:
        is_child[rng.choice(n, n_child, replace=False)] = True
    parents = np.flatnonzero(~is_child)
    # independent rows first
    tgt = np.where(is_child, 0, nnz)
    draw = lambda m: zc.draw(rng, m)
    key = _fill_unique(rng, tgt, np.zeros(0, np.int64), np.zeros(0, np.int64), draw, d)
    rows0 = np.zeros(0, np.int64)
    cols0 = np.zeros(0, np.int64)
    if n_child:
        children = np.flatnonzero(is_child)
        par = parents[rng.integers(0, parents.size, children.size)]
        rws, cls = key // d, key % d
        start = np.searchsorted(rws, np.arange(n + 1))
        plen = start[par + 1] - start[par]
        c_rep = np.repeat(children, plen)
        p_idx = np.concatenate([np.arange(start[p], start[p + 1]) for p in par]) \
            if par.size else np.zeros(0, np.int64)
        keep_p = np.repeat(rng.uniform(0.5, 1.0, children.size), plen)
        keep = rng.random(c_rep.size) < keep_p
        c_rep, p_idx = c_rep[keep], p_idx[keep]
        # cap each child at its own nnz: keep a random subset of the kept parent columns
        order = np.lexsort((rng.random(c_rep.size), c_rep))
        c_rep, p_idx = c_rep[order], p_idx[order]
        first = np.searchsorted(c_rep, c_rep, side="left")
        rank = np.arange(c_rep.size) - first
        ok = rank < nnz[c_rep]
        rows0, cols0 = c_rep[ok], cls[p_idx[ok]]
        tgt_c = np.where(is_child, nnz, 0)
        key_c = _fill_unique(rng, tgt_c, rows0, cols0, draw, d)
        key = np.concatenate([key, key_c])
        key.sort()
    rws = key // d
    counts = np.bincount(rws, minlength=n)
    row_ptr = np.zeros(n + 1, np.uint64)
    row_ptr[1:] = np.cumsum(counts).astype(np.uint64)
    return CSR(row_ptr, (key % d).astype(np.uint32), d)


# ----------------------------------------------------------------------------
# Workloads (sizes of the benchmark configurations)
# ----------------------------------------------------------------------------

def tiny_corpus(seed: int = 0, n: int = 1000, d: int = 10_000) -> CSR:
    """n=1000 rows over d=10,000; nnz ~ Zipf(1.1) clipped to [5, 200]."""
    rng = np.random.default_rng(seed)
    return powerlaw_csr(rng, n, d, nnz_zipf_clipped(rng, n))


def bow_corpus(seed: int = 0, n: int = 100_000, d: int = 1_000_000, median: float = 200.0,
               sigma: float = 1.0, lo: int = 1, hi: int = 5000) -> CSR:
    """Text-BoW scale: nnz log-normal (median 200, sigma 1) clipped to [1, 5000]."""
    rng = np.random.default_rng(seed)
    return powerlaw_csr(rng, n, d, nnz_lognormal(rng, n, median, sigma, lo, hi))


def random_csr(seed: int, n: int, d: int, nnz_lo: int, nnz_hi: int, child_frac=0.2,
               permute=True, s=1.0) -> CSR:
    """Small corpora for tests: nnz uniform in [nnz_lo, nnz_hi]."""
    rng = np.random.default_rng(seed)
    nnz = rng.integers(nnz_lo, nnz_hi + 1, n)
    return powerlaw_csr(rng, n, d, nnz, s=s, child_frac=child_frac, permute=permute)


def uniform_csr(seed: int, n: int, d: int, nnz_lo: int, nnz_hi: int) -> CSR:
    """Rows of uniformly random distinct columns (dense / saturated regime)."""
    rng = np.random.default_rng(seed)
    nnz = rng.integers(nnz_lo, nnz_hi + 1, n)
    nnz = np.minimum(nnz, d)
    cols = [np.sort(rng.choice(d, int(k), replace=False)).astype(np.uint32) for k in nnz]
    row_ptr = np.zeros(n + 1, np.uint64)
    row_ptr[1:] = np.cumsum(nnz).astype(np.uint64)
    col = np.concatenate(cols) if cols else np.zeros(0, np.uint32)
    return CSR(row_ptr, col.astype(np.uint32), d)


def random_sketches(seed: int, n: int, N: int, density: float = 0.5) -> np.ndarray:
    """Packed random bit rows [n][N/32] (for count-only tests)."""
    rng = np.random.default_rng(seed)
    bits = rng.random((n, N)) < density
    return np.packbits(bits, axis=1, bitorder="little").view(np.uint32).reshape(n, N // 32)


def bow_corpus_device(seed: int, n: int, d: int, median: float = 200.0, sigma: float = 1.0,
                      lo: int = 1, hi: int = 5000, device="cuda", s: float = 1.0):
    """A large text-BoW-shaped corpus drawn directly on the GPU (torch RNG).

    Same shape as bow_corpus -- log-normal nnz per row clipped to [lo, hi],
    Zipf(s) columns through a seeded rank -> id permutation -- but columns are
    drawn with replacement (a repeated column is harmless: OR is idempotent)
    and no near-duplicate children are planted.  Returns device tensors
    (row_ptr int64 [n + 1], col int32 [nnz]) holding uint64 offsets and
    uint32 ids."""
    import torch
    g = torch.Generator().manual_seed(seed)
    ln = torch.randn(n, generator=g, dtype=torch.float64) * sigma + math.log(median)
    nnz = torch.clamp(torch.round(torch.exp(ln)), lo, hi).to(torch.int64)
    row_ptr = torch.zeros(n + 1, dtype=torch.int64)
    row_ptr[1:] = torch.cumsum(nnz, 0)
    total = int(row_ptr[-1])
    perm = torch.randperm(d, generator=g).to(torch.int32).to(device)
    w = 1.0 / torch.arange(1, d + 1, dtype=torch.float64, device=device) ** s
    cdf = torch.cumsum(w, 0)
    cdf /= cdf[-1].clone()
    gd = torch.Generator(device=device).manual_seed(seed + 1)
    col = torch.empty(total, dtype=torch.int32, device=device)
    step = 1 << 26
    for a in range(0, total, step):
        b = min(total, a + step)
        u = torch.rand(b - a, generator=gd, dtype=torch.float64, device=device)
        r = torch.searchsorted(cdf, u, right=True).clamp_(max=d - 1)
        col[a:b] = perm[r]
    return row_ptr.to(device), col


def query_batch(rng: np.random.Generator, q: int, zipf: "ZipfColumns", median: float = 200.0,
                sigma: float = 1.0, lo: int = 1, hi: int = 5000):
    """q query vectors shaped like bow_corpus rows (log-normal nnz, Zipf
    columns, drawn with replacement).  Returns (row_ptr uint64, col uint32)."""
    nnz = nnz_lognormal(rng, q, median, sigma, lo, hi)
    row_ptr = np.zeros(q + 1, np.uint64)
    row_ptr[1:] = np.cumsum(nnz).astype(np.uint64)
    col = zipf.draw(rng, int(row_ptr[-1])).astype(np.uint32)
    return row_ptr, col
