"""Host side of the database-sharded ranking (no GPU): shard ranges, the
max-over-ranks reduction the benchmark uses, and the all-gather of per-shard
top-k lists, run as two gloo ranks on CPU.  The decomposition itself (merged
per-shard lists == the unsharded top-k) is checked on oracle lists."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_1910_04658_gb300 import inputs, sharded


def test_shard_range_partitions():
    for n in (0, 1, 7, 128, 1000, 100_003):
        for world in (1, 2, 3, 8):
            ranges = [sharded.shard_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (lo, hi), (lo2, _) in zip(ranges, ranges[1:]):
                assert hi == lo2
            sizes = [hi - lo for lo, hi in ranges]
            assert max(sizes) - min(sizes) <= 1
            assert sharded.shard_offsets(n, world) == [lo for lo, _ in ranges]
    with pytest.raises(ValueError):
        sharded.shard_range(10, 2, 2)


def test_single_process_helpers_are_identity():
    assert sharded.max_over_ranks([1.5, 2.0]) == [1.5, 2.0]
    s = torch.zeros((3, 4))
    i = torch.zeros((3, 4), dtype=torch.int32)
    sp, ip = sharded.gather_lists(s, i)
    assert sp.shape == (1, 3, 4) and ip.shape == (1, 3, 4)


N, K, SEED = 256, 12, 5


def _corpus():
    csr = inputs.random_csr(seed=SEED, n=301, d=5000, nnz_lo=1, nnz_hi=120)
    sk, pc = oracle.sketch(csr.row_ptr, csr.col, csr.d, N, seed=3)
    return sk, pc


def _shard_topk(sk, lo, hi, measure, exclude_self):
    """The k best rows of sk[lo:hi] for every row of sk, local indices,
    ranked like the library (score desc / Ham asc, then index asc)."""
    est, _ = oracle.estimate_pairs(sk, sk[lo:hi], N)
    e = est[measure]
    key = -e if measure == oracle.HAM else e
    n = sk.shape[0]
    score = np.zeros((n, K))
    idx = np.zeros((n, K), np.int64)
    for q in range(n):
        order = sorted((j for j in range(hi - lo) if not (exclude_self and lo + j == q)),
                       key=lambda j: (-key[q, j], j))[:K]
        score[q] = e[q, order]
        idx[q] = order
    return score, idx


def _merge(score_parts, idx_parts, offsets, measure):
    n = score_parts.shape[1]
    out_s = np.zeros((n, K))
    out_i = np.zeros((n, K), np.int64)
    for q in range(n):
        items = []
        for p, off in enumerate(offsets):
            for t in range(K):
                v = score_parts[p, q, t]
                items.append((v if measure == oracle.HAM else -v, int(idx_parts[p, q, t]) + off))
        items.sort()
        out_s[q] = [(v if measure == oracle.HAM else -v) for v, _ in items[:K]]
        out_i[q] = [g for _, g in items[:K]]
    return out_s, out_i


def _rank_main(rank, world, port, errfile):
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
        # max over ranks (the benchmark's timing reduction)
        got = sharded.max_over_ranks([1.0 + rank, 10.0 - rank])
        assert got == [float(world), 10.0], got
        sk, _ = _corpus()
        n = sk.shape[0]
        lo, hi = sharded.shard_range(n, rank, world)
        # every rank learns every shard's offset (host metadata only)
        meta = sharded.ShardedTopK(None, torch.zeros(hi - lo, dtype=torch.int32), lo, N, K)
        assert meta.world == world and meta.rank == rank
        assert meta.offsets() == sharded.shard_offsets(n, world)
        for measure in (oracle.JS, oracle.HAM):
            s, i = _shard_topk(sk, lo, hi, measure, exclude_self=True)
            sp, ip = sharded.gather_lists(torch.from_numpy(s), torch.from_numpy(i))
            assert sp.shape == (world, n, K)
            # every rank received every rank's lists, in rank order
            s_own, i_own = sp[rank].numpy(), ip[rank].numpy()
            assert np.array_equal(s_own, s) and np.array_equal(i_own, i)
            ms, mi = _merge(sp.numpy(), ip.numpy(), sharded.shard_offsets(n, world), measure)
            ref_s, ref_i, _ = oracle.topk(sk, sk, N, measure, K, exclude_self=True)
            assert np.array_equal(mi, ref_i.astype(np.int64)), measure
            assert np.array_equal(ms, ref_s), measure
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    except BaseException as e:  # reported to the parent through the file
        with open(errfile, "a") as f:
            f.write(f"rank {rank}: {type(e).__name__}: {e}\n")
        raise


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2])
def test_gloo_ranks_gather_and_merge(tmp_path, world):
    oracle.build()
    errfile = str(tmp_path / "err.txt")
    mp.start_processes(_rank_main, args=(world, _free_port(), errfile), nprocs=world,
                       start_method="spawn", join=True)
    assert not os.path.exists(errfile) or open(errfile).read() == ""
