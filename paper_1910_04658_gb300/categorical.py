"""Categorical data front end (Sec. 1, "Extension for categorical data
compression").

A categorical row has F features; the distance between two rows is the number
of features on which they differ.  Label encoding maps the m distinct values
of a feature to 0 .. m-1 (in sorted order of the values, as scikit-learn's
LabelEncoder does); one-hot encoding then turns feature f into m_f binary
columns with one set bit.  Two encoded rows differ in exactly two bits per
differing feature, so the categorical distance is half the Hamming distance
of the binary rows, and BinSketch's Hamming estimate (Alg. 2) divided by two
estimates it.

Label encoding runs on the host (it sees arbitrary values); the one-hot
encoding (bs_onehot_csr), the sketches and the estimates run in the
library's kernels.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

from . import binding as B


def label_encode(columns: Sequence[Sequence]) -> Tuple[np.ndarray, List[np.ndarray]]:
    """columns[f] = the n values of feature f (any sortable values).  Returns
    labels uint32[n][F] and, per feature, its sorted distinct values (label v
    stands for classes[f][v])."""
    labels, classes = [], []
    for values in columns:
        cls, inv = np.unique(np.asarray(values), return_inverse=True)
        labels.append(inv.astype(np.uint32))
        classes.append(cls)
    return np.stack(labels, 1) if labels else np.zeros((0, 0), np.uint32), classes


def feature_offsets(cardinalities: Sequence[int]) -> np.ndarray:
    """uint32[F + 1]: first binary column of each feature, then d."""
    off = np.zeros(len(cardinalities) + 1, np.uint64)
    off[1:] = np.cumsum(np.asarray(cardinalities, np.uint64))
    if off[-1] >= 2 ** 32:
        raise ValueError("binary dimension exceeds 2^32")
    return off.astype(np.uint32)


def onehot(labels, offsets):
    """Device one-hot CSR of device labels int32/uint32 [n][F] and offsets
    [F + 1]: (row_ptr int64 [n + 1], col int32 [n * F], d)."""
    import torch
    n, F = int(labels.shape[0]), int(labels.shape[1])
    dev = labels.device
    rp = torch.empty((n + 1,), dtype=torch.int64, device=dev)
    col = torch.empty((max(n * F, 1),), dtype=torch.int32, device=dev)
    B.bs_onehot_csr(labels, n, F, offsets, rp, col)
    d = int(offsets[-1].item())
    return rp, col, d


def distance_estimates(ham_estimates):
    """Categorical distance estimate = Hamming estimate / 2."""
    return ham_estimates * 0.5


def synthetic(seed: int, n: int, cardinalities: Sequence[int], dup_frac: float = 0.2,
              change_frac: float = 0.2) -> np.ndarray:
    """Labels uint32[n][F]: each feature Zipf(1.0)-distributed over its
    values; a fraction of the rows copy an earlier row and redraw about
    change_frac of its features (so close pairs exist)."""
    rng = np.random.default_rng(seed)
    F = len(cardinalities)
    out = np.empty((n, F), np.uint32)
    for f, m in enumerate(cardinalities):
        p = 1.0 / np.arange(1, m + 1)
        out[:, f] = rng.choice(m, size=n, p=p / p.sum())
    kids = np.flatnonzero(rng.random(n) < dup_frac)
    kids = kids[kids > 0]
    for i in kids:
        j = rng.integers(0, i)
        row = out[j].copy()
        redraw = rng.random(F) < change_frac
        for f in np.flatnonzero(redraw):
            row[f] = rng.integers(0, cardinalities[f])
        out[i] = row
    return out
