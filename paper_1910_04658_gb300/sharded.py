"""Ranking over a database sharded across ranks (one GPU per rank).

The ranking of Experiment 2 (Sec. 4), as a top-k, splits over database rows
with one exchange step: every rank ranks the queries against its own
contiguous shard (``bs_topk_shard``), the ranks all-gather their nQ x k
lists (8 bytes per entry), and every rank merges them (``bs_topk_merge``).
Each shard's list holds that shard's k best, so the merged list is the
unsharded top-k exactly, index for index and bit for bit.  Sketching needs no
exchange at all: every rank sketches its own rows with the shared (seed, N).

The collectives go through ``torch.distributed`` (NCCL between GPUs; the
host-side helpers also run on gloo with CPU tensors).
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

from . import binding as B


def shard_range(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Rows [lo, hi) of shard `rank` when n rows are split into `world`
    contiguous shards whose sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard request")
    return n * rank // world, n * (rank + 1) // world


def shard_offsets(n: int, world: int) -> List[int]:
    return [shard_range(n, r, world)[0] for r in range(world)]


def _world(group=None) -> Tuple[int, int]:
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def max_over_ranks(values: Sequence[float], group=None, device=None) -> List[float]:
    """Element-wise maximum of `values` over the ranks of `group` (the
    benchmark's per-rank times); the identity without a process group."""
    import torch
    import torch.distributed as dist
    _, world = _world(group)
    if world == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return [float(v) for v in t.tolist()]


def gather_lists(score, idx, group=None):
    """All-gather every rank's [nQ, k] top-k lists into [world, nQ, k]
    tensors on every rank (same device as the inputs)."""
    import torch
    import torch.distributed as dist
    _, world = _world(group)
    if world == 1:
        return score.unsqueeze(0), idx.unsqueeze(0)
    s_parts = torch.empty((world,) + tuple(score.shape), dtype=score.dtype, device=score.device)
    i_parts = torch.empty((world,) + tuple(idx.shape), dtype=idx.dtype, device=idx.device)
    dist.all_gather(list(s_parts.unbind(0)), score.contiguous(), group=group)
    dist.all_gather(list(i_parts.unbind(0)), idx.contiguous(), group=group)
    return s_parts, i_parts


class ShardedTopK:
    """This rank's shard of a sketch database and the cross-rank top-k.

    sk, pc: the shard's rows (device int32 [n_shard, N/32] and [n_shard]),
    which are rows db_offset .. db_offset + n_shard - 1 of the whole database.
    """

    def __init__(self, sk, pc, db_offset: int, N: int, k: int, by: str = "js", group=None,
                 variant: int = B.BS_VARIANT_AUTO):
        self.sk, self.pc = sk, pc
        self.n = int(pc.numel())
        self.off = int(db_offset)
        self.N, self.k, self.by = N, k, by
        self.group = group
        self.variant = variant
        self.rank, self.world = _world(group)
        self._ws = None

    def _workspace(self, nQ):
        import torch
        need = B.bs_topk_workspace_bytes(nQ, self.n, self.N, self.k)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty((max(need, 256),), dtype=torch.uint8, device=self.pc.device)
        return self._ws, need

    def offsets(self) -> List[int]:
        """Every rank's db_offset (an all-gather of one integer)."""
        import torch
        import torch.distributed as dist
        if self.world == 1:
            return [self.off]
        t = torch.tensor([self.off], dtype=torch.int64, device=self.pc.device)
        out = torch.empty((self.world, 1), dtype=torch.int64, device=self.pc.device)
        dist.all_gather(list(out.unbind(0)), t, group=self.group)
        return [int(v) for v in out.flatten().tolist()]

    def search(self, Q, pcQ, exclude_self: bool = False, offsets: Optional[List[int]] = None):
        """Top-k of every query row over the whole (all ranks') database, on
        the current CUDA stream (where the collectives also order).
        exclude_self: query row q is database row q (all-pairs mode)."""
        import torch
        nQ = int(pcQ.numel())
        dev = self.pc.device
        score = torch.empty((nQ, self.k), dtype=torch.float32, device=dev)
        idx = torch.empty((nQ, self.k), dtype=torch.int32, device=dev)
        ws, wsb = self._workspace(nQ)
        by = B.MEASURE_BITS[self.by]
        B.bs_topk_shard(Q, pcQ, nQ, self.sk, self.pc, self.n, self.off, self.N, by, self.k,
                        exclude_self, score, idx, ws, wsb, self.variant)
        offs = offsets if offsets is not None else self.offsets()
        s_parts, i_parts = gather_lists(score, idx, self.group)
        out_s = torch.empty_like(score)
        out_i = torch.empty_like(idx)
        B.bs_topk_merge(s_parts, i_parts, len(offs), nQ, self.k, offs, by, out_s, out_i)
        return out_s, out_i
