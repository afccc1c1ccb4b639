"""Learned estimator for saturated sketches: data, training, evaluation.

BinSketch's closed-form estimators (Alg. 1-4) invert the expected occupancy
N (1 - (1 - 1/N)^|a|); when sketches fill up (|a| comparable to N or larger)
the inversion becomes ill-conditioned.  This module trains the library's
4 -> 64 -> 64 -> 4 BF16 MLP to correct the closed form in that regime (its
inputs are the closed-form set sizes and inner product, its outputs are added
to the closed-form estimates), on pairs that the
library's own generator sketches (`bs_dense_pairs`: exact sizes are known by
construction), and compares its mean squared error with the closed form on
held-out pairs.  All arithmetic runs in the library's kernels; torch only
holds the buffers.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List

import numpy as np

from . import binding as B

MEASURES = ["ip", "ham", "js", "cos"]


@dataclass
class PairSet:
    N: int
    counts: "object"    # device int32 [n][3]
    sizes: "object"     # device int32 [n][3]

    @property
    def n(self):
        return int(self.counts.shape[0])


def dense_pairs(n: int, N: int, d: int = 100_000, pair_seed: int = 1, hash_seed: int = 0,
                lo_frac: float = 0.25, hi_frac: float = 4.0, device="cuda") -> PairSet:
    """n pairs with |a|, |b| uniform in [N/4, 4N] over d columns (the dense regime)."""
    import torch
    counts = torch.empty((n, 3), dtype=torch.int32, device=device)
    sizes = torch.empty((n, 3), dtype=torch.int32, device=device)
    B.bs_dense_pairs(n, N, d, int(lo_frac * N), int(hi_frac * N), pair_seed, hash_seed, counts, sizes)
    return PairSet(N, counts, sizes)


def exact_similarities(sizes: np.ndarray) -> np.ndarray:
    """IP, Ham, JS, Cos [n][4] (float64) from exact (|a|, |b|, |a AND b|)."""
    A, Bs, I = (sizes[:, i].astype(np.float64) for i in range(3))
    U = A + Bs - I
    js = np.divide(I, U, out=np.zeros_like(I), where=U > 0)
    den = np.sqrt(A * Bs)
    cs = np.divide(I, den, out=np.zeros_like(I), where=den > 0)
    return np.stack([I, A + Bs - 2 * I, js, cs], 1)


class MLPEstimator:
    def __init__(self, device="cuda", seed: int = 0):
        import torch
        self.torch = torch
        g = torch.Generator().manual_seed(seed)
        p = torch.zeros(B.BS_MLP_PARAMS, dtype=torch.float32)
        # W1[64][4], b1[64], W2[64][64], b2[64], W3[4][64], b3[4]; He initialisation
        p[0:256] = torch.randn(256, generator=g) * (2.0 / 4) ** 0.5
        p[320:4416] = torch.randn(4096, generator=g) * (2.0 / 64) ** 0.5
        # W3, b3 start at zero: the untrained MLP is exactly the closed form
        self.params = p.to(device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.step = 0
        self.device = device

    def train(self, sets: List[PairSet], epochs: int = 3, batch: int = 8192, lr: float = 2e-3,
              seed: int = 0) -> List[float]:
        """Adam on the mean squared error of the scaled targets; returns the
        mean batch loss of each epoch."""
        torch = self.torch
        xs, ts = [], []
        for s in sets:
            x = torch.empty((s.n, 4), dtype=torch.float32, device=self.device)
            t = torch.empty((s.n, 4), dtype=torch.float32, device=self.device)
            B.bs_mlp_prepare(s.counts, s.sizes, s.n, s.N, x, t)
            xs.append(x)
            ts.append(t)
        X, T = torch.cat(xs), torch.cat(ts)
        n = X.shape[0]
        g = torch.Generator(device=self.device).manual_seed(seed)
        steps_per_epoch = (n + batch - 1) // batch
        total = epochs * steps_per_epoch
        hist = []
        done = 0   # steps of this call (the Adam step count self.step runs on across calls)
        for ep in range(epochs):
            perm = torch.randperm(n, generator=g, device=self.device)
            Xp, Tp = X[perm].contiguous(), T[perm].contiguous()
            self.loss.zero_()
            for i in range(steps_per_epoch):
                a = i * batch
                b = min(n, a + batch)
                self.step += 1
                # cosine decay of the step size over this call's steps
                frac = done / max(1, total)
                done += 1
                rate = lr * 0.5 * (1 + np.cos(np.pi * min(frac, 1.0)))
                B.bs_mlp_train_step(self.params, self.m, self.v, self.grad, self.step, float(rate),
                                    Xp[a:b], Tp[a:b], b - a, self.loss)
            hist.append(float(self.loss.item()) / steps_per_epoch)
        return hist

    def estimate(self, s: PairSet):
        out = self.torch.empty((s.n, 4), dtype=self.torch.float32, device=self.device)
        B.bs_mlp_estimate(self.params, s.counts, s.n, s.N, out)
        return out


def closed_form(s: PairSet):
    import torch
    out = torch.empty((s.n, 4), dtype=torch.float32, device=s.counts.device)
    B.bs_estimate_counts(s.counts, s.n, s.N, out)
    return out


def mse_table(est: np.ndarray, exact: np.ndarray) -> Dict[str, float]:
    err = (est.astype(np.float64) - exact) ** 2
    return {m: float(err[:, i].mean()) for i, m in enumerate(MEASURES)}
