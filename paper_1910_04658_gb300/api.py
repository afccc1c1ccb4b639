"""Torch-facing helpers over the C ABI: allocate outputs, call the binding.

These only allocate device memory with torch and forward to ``binding``; all
arithmetic runs in libbinsketch's kernels.
"""
from __future__ import annotations

import torch

from . import binding as B


def sketch(row_ptr: torch.Tensor, col: torch.Tensor, d: int, N: int, seed: int = 0,
           parity: bool = False, stream=None):
    """CSR on the GPU -> (sketch [n][N/32], |a_s| [n]).

    row_ptr holds uint64 offsets and col uint32 indices (any 8- or 4-byte
    integer tensor dtype: only the bits matter).  Outputs are int32 tensors
    carrying the uint32 words and counts."""
    n = row_ptr.numel() - 1
    dev = row_ptr.device
    sk = torch.empty((n, N // 32), dtype=torch.int32, device=dev)
    pc = torch.empty((n,), dtype=torch.int32, device=dev)
    fn = B.bs_sketch_parity if parity else B.bs_sketch
    fn(row_ptr, col, n, col.numel(), d, N, seed, sk, pc, stream)
    return sk, pc


def estimate_pairs(A, pcA, Bm, pcB, N: int, measures=("ip", "ham", "js", "cos"), counts=True,
                   stream=None, variant: str = "auto"):
    """Counts and estimates of every (A row, B row) pair (bs_estimate_pairs_ex);
    variant: "auto", "popc" or "tc"."""
    mask = 0
    for m in measures:
        mask |= B.MEASURE_BITS[m]
    nA, nB = A.shape[0], Bm.shape[0]
    nm = bin(mask).count("1")
    out = torch.empty((nm, nA, nB), dtype=torch.float32, device=A.device) if nm else None
    cnt = torch.empty((nA, nB), dtype=torch.int32, device=A.device) if counts else None
    B.bs_estimate_pairs_ex(A, pcA, nA, Bm, pcB, nB, N, mask, out, cnt, B.VARIANTS[variant], stream)
    return out, cnt


def topk(Q, pcQ, DB, pcDB, N: int, k: int, by: str = "js", exclude_self: bool = False,
         stream=None, workspace=None, variant: str = "auto"):
    """Top-k of every query row by `by` (bs_topk_ex); variant: "auto",
    "popc", "tc" or "tc0" .. "tc14" (a tensor-core block configuration)."""
    nQ, nDB = Q.shape[0], DB.shape[0]
    score = torch.empty((nQ, k), dtype=torch.float32, device=Q.device)
    idx = torch.empty((nQ, k), dtype=torch.int32, device=Q.device)
    wsb = B.bs_topk_workspace_bytes(nQ, nDB, N, k)
    if wsb and (workspace is None or workspace.numel() * workspace.element_size() < wsb):
        workspace = torch.empty((wsb,), dtype=torch.uint8, device=Q.device)
    B.bs_topk_ex(Q, pcQ, nQ, DB, pcDB, nDB, N, B.MEASURE_BITS[by], k, exclude_self, score, idx,
                 workspace if wsb else None, wsb, B.VARIANTS[variant], stream)
    return score, idx
