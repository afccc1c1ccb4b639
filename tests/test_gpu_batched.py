"""Batched datasets: the persistent batched sketch equals per-dataset sketches;
the autotuned, graph-captured top-k equals the plain per-dataset calls."""
import numpy as np
import pytest

import oracle
from tests.helpers import check_topk_row, dev_u32, u32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1910_04658_gb300 import api, binding as B  # noqa: E402
from paper_1910_04658_gb300.batched import Autotuner, BatchedJob, make_datasets  # noqa: E402


@pytest.fixture(scope="module")
def datasets():
    ds = make_datasets(3, n_datasets=7, n_lo=300, n_hi=3000, d_lo=1e3, d_hi=1e6,
                       Ns=(96, 256, 1024, 4096, 8192), med_lo=20, med_hi=300)
    return ds


def test_batched_sketch_equals_single(datasets):
    job = BatchedJob(datasets, k=20, by="cos")
    job.sketch_all(torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert B.bs_get_async_error() == 0
    for j, d in enumerate(datasets):
        sk, pc = api.sketch(d.row_ptr, d.col, d.d, d.N, d.seed)
        assert torch.equal(sk, job.sk[j]) and torch.equal(pc, job.pc[j])


def test_tuned_graph_equals_plain_topk(datasets, tmp_path):
    tuner = Autotuner(cache_path=str(tmp_path / "tune.json"))
    job = BatchedJob(datasets, k=20, by="cos", autotuner=tuner)
    job.tune()
    tuner.save()
    assert len(Autotuner(cache_path=str(tmp_path / "tune.json")).table) >= 1
    job.capture()
    for _ in range(2):
        job.replay()
        torch.cuda.synchronize()
        assert B.bs_get_async_error() == 0
        for j, d in enumerate(datasets):
            s_ref, i_ref = api.topk(job.sk[j], job.pc[j], job.sk[j], job.pc[j], d.N, 20, by="cos",
                                    exclude_self=True)
            s, i = job.results(j)
            assert torch.equal(i, i_ref) and torch.equal(s, s_ref)


def test_batched_results_match_oracle(datasets):
    job = BatchedJob(datasets, k=20, by="cos")
    job.run_eager()
    torch.cuda.synchronize()
    for j in (0, 3):
        d = datasets[j]
        # the oracle sketches the dataset's input CSR itself
        osk, _ = oracle.sketch(d.row_ptr.cpu().numpy().view(np.uint64), d.col.cpu().numpy().view(np.uint32),
                               d.d, d.N, d.seed)
        assert np.array_equal(u32(job.sk[j]), osk)
        rows = np.arange(0, d.n, max(1, d.n // 12))
        oest, _ = oracle.estimate_pairs(osk[rows], osk, d.N)
        s, i = job.results(j)
        s, i = s.cpu().numpy(), u32(i)
        for t, r in enumerate(rows):
            check_topk_row(s[r], i[r], oest[3, t], 20, 3, exclude_q=int(r))


def test_persistent_batch_equals_per_dataset_calls(datasets):
    # one persistent ranking launch over every tensor-core dataset (the N = 96
    # dataset goes through its own CUDA-core call) gives, list for list and
    # bit for bit, what one bs_topk_ex per dataset gives
    per = BatchedJob(datasets, k=20, by="cos", mode="per_dataset")
    per.run_eager()
    job = BatchedJob(datasets, k=20, by="cos")
    job.run_eager()
    torch.cuda.synchronize()
    assert B.bs_get_async_error() == 0
    assert job.side == [j for j, d in enumerate(datasets) if d.N == 96]
    for j in range(len(datasets)):
        s0, i0 = per.results(j)
        s1, i1 = job.results(j)
        assert torch.equal(i0, i1) and torch.equal(s0, s1), j
    # launches: the batched sketch, the re-layout, the ranking, and the side
    # dataset's own calls -- far fewer than one top-k per dataset
    assert job.launches() < per.launches()
    assert B.bs_topk_batched_plan(job.tjobs, 20) == (1, 2)


def test_batched_topk_rejects_bad_tables(datasets):
    job = BatchedJob(datasets, k=20, by="cos")
    ws = torch.empty((job.bwsb,), dtype=torch.uint8, device="cuda")
    with pytest.raises(B.BinSketchError) as e:     # workspace too small
        B.bs_topk_batched(job.tjobs, B.BS_COS, 20, ws[:64], 64, 0)
    assert e.value.code == 5
    d = datasets[job.side[0]]
    j96 = job.side[0]
    bad = B._job_table([dict(Q=job.sk[j96], pcQ=job.pc[j96], DB=job.sk[j96], pcDB=job.pc[j96],
                             score=job.score[j96], idx=job.idx[j96], nQ=d.n, nDB=d.n, N=d.N,
                             exclude_self=True, k=20)])
    with pytest.raises(B.BinSketchError) as e:     # N = 96: not a tensor-core shape
        B.bs_topk_batched(bad, B.BS_COS, 20, ws, job.bwsb, 0)
    assert e.value.code == 7


def test_dynamic_schedule_many_small_jobs_repeatable():
    # 64 problems (the table maximum) of mixed shapes, self-joins and
    # query-vs-database pairs, many more row blocks than resident blocks:
    # whichever block claims a row block, each list equals the single-problem
    # tensor-core call's, and a second call on the same workspace (its claim
    # counter reset by the re-layout launch) gives the same lists again
    from paper_1910_04658_gb300.inputs import random_sketches

    rng = np.random.default_rng(21)
    k, dev = 16, torch.device("cuda", 0)
    jobs, refs = [], []
    for j in range(B.BS_TOPK_BATCH_MAX):
        N = int(rng.choice([256, 512, 1024, 4096]))
        nq = int(rng.integers(1, 700))
        self_join = j % 3 == 0
        ndb = nq if self_join else int(rng.integers(1, 2500))
        dens = float(rng.uniform(0.02, 0.4))
        q = dev_u32(random_sketches(1000 + j, nq, N, dens))
        db = q if self_join else dev_u32(random_sketches(5000 + j, ndb, N, dens))
        pcq = torch.empty((nq,), dtype=torch.int32, device=dev)
        pcdb = pcq if self_join else torch.empty((ndb,), dtype=torch.int32, device=dev)
        B.bs_popcount_rows(q, nq, N, pcq)
        if not self_join:
            B.bs_popcount_rows(db, ndb, N, pcdb)
        score = torch.empty((nq, k), dtype=torch.float32, device=dev)
        idx = torch.empty((nq, k), dtype=torch.int32, device=dev)
        jobs.append(dict(Q=q, pcQ=pcq, DB=db, pcDB=pcdb, score=score, idx=idx, nQ=nq, nDB=ndb, N=N,
                         exclude_self=self_join, k=k))
        s_ref = torch.empty_like(score)
        i_ref = torch.empty_like(idx)
        wsb = B.bs_topk_workspace_bytes(nq, ndb, N, k)
        ws = torch.empty((max(wsb, 1),), dtype=torch.uint8, device=dev)
        B.bs_topk_ex(q, pcq, nq, db, pcdb, ndb, N, B.BS_JS, k, self_join, s_ref, i_ref, ws, wsb, B.BS_VARIANT_TC)
        refs.append((s_ref, i_ref))
    tab = B._job_table(jobs)
    wsb = B.bs_topk_batched_workspace_bytes(tab, k)
    ws = torch.empty((wsb,), dtype=torch.uint8, device=dev)
    for _ in range(2):
        for jb in jobs:
            jb["score"].fill_(7.0)
            jb["idx"].fill_(-7)
        B.bs_topk_batched(tab, B.BS_JS, k, ws, wsb, 0)
        torch.cuda.synchronize()
        assert B.bs_get_async_error() == 0
        for j, (jb, (s_ref, i_ref)) in enumerate(zip(jobs, refs)):
            assert torch.equal(jb["idx"], i_ref) and torch.equal(jb["score"], s_ref), j
