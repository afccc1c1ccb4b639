"""Tensor-core counting (block-scaled FP4 MMA) against the oracle, through the C ABI.

The common-bit counts n_{a_s,b_s} of Alg. 1 step 2 come out of the tensor
cores as FP32 accumulators; they must equal the oracle's integer counts bit
for bit, including dense and saturated sketches (counts up to N) and sketch
lengths whose 128-bit k-chunk count is odd (the kernel pads those to whole
256-bit operand slots).  Estimates stay within the tolerance of
tests/helpers.py.  A fault-injected call must end in BS_ERR_TIMEOUT without
faulting, and the next call on the stream must be correct.
"""
import numpy as np
import pytest

import oracle
from paper_1910_04658_gb300 import inputs
from tests.helpers import assert_close, check_topk_row, to_dev, u32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1910_04658_gb300 import api, binding as B  # noqa: E402


def _sketch_both(c, N, seed):
    rp, col = to_dev(c)
    sk, pc = api.sketch(rp, col, c.d, N, seed)
    assert B.bs_get_async_error() == 0
    osk, opc = oracle.sketch(c.row_ptr, c.col, c.d, N, seed)
    assert np.array_equal(u32(sk), osk) and np.array_equal(u32(pc), opc)
    return sk, pc, osk


def _dense(N, n=300, seed=3):
    # nnz uniform in [N/4, 4N] plus a few rows of 20N columns (|a_s| = N)
    c = inputs.uniform_csr(seed, n, 100_000, N // 4, 4 * N)
    f = inputs.uniform_csr(seed + 1, 6, 100_000, 20 * N, 20 * N)
    rp = np.concatenate([c.row_ptr, f.row_ptr[1:] + c.row_ptr[-1]]).astype(np.uint64)
    return inputs.CSR(rp, np.concatenate([c.col, f.col]), c.d)


@pytest.mark.parametrize("N", [256, 384, 1024, 4096, 8192])
def test_tc_counts_bit_exact_dense_and_saturated(N):
    c = _dense(N)
    sk, pc, osk = _sketch_both(c, N, 8)
    assert (u32(pc) == N).any()
    out, cnt = api.estimate_pairs(sk, pc, sk, pc, N, variant="tc")
    assert B.bs_get_async_error() == 0
    oest, ocnt = oracle.estimate_pairs(osk, osk, N)
    assert np.array_equal(u32(cnt), ocnt)
    assert ocnt.max() == N            # some pair reaches the full sketch length
    for m in range(4):
        assert_close(out[m].cpu().numpy(), oest[m], m)


@pytest.mark.parametrize("N", [256, 640, 4096])
@pytest.mark.parametrize("nA,nB", [(1, 1), (77, 301), (129, 481), (300, 239)])
def test_tc_counts_ragged_shapes(N, nA, nB):
    # query blocks of 128 and database tiles of 240 rows with ragged tails
    a = inputs.random_csr(1, nA, 300_000, 1, 900)
    b = inputs.random_csr(2, nB, 300_000, 1, 900)
    ask, apc, oa = _sketch_both(a, N, 5)
    bsk, bpc, ob = _sketch_both(b, N, 5)
    out, cnt = api.estimate_pairs(ask, apc, bsk, bpc, N, variant="tc")
    oest, ocnt = oracle.estimate_pairs(oa, ob, N)
    assert np.array_equal(u32(cnt), ocnt)
    for m in range(4):
        assert_close(out[m].cpu().numpy(), oest[m], m)


def test_tc_and_popc_counts_identical_and_subsets():
    N = 2048
    c = inputs.random_csr(7, 700, 500_000, 1, 3000)
    sk, pc, osk = _sketch_both(c, N, 1)
    o_tc, c_tc = api.estimate_pairs(sk, pc, sk[:333], pc[:333], N, measures=("js", "cos"), variant="tc")
    o_pp, c_pp = api.estimate_pairs(sk, pc, sk[:333], pc[:333], N, measures=("js", "cos"), variant="popc")
    assert torch.equal(c_tc, c_pp)
    assert torch.equal(o_tc, o_pp)        # same integers, same FP32 arithmetic
    _, c_only = api.estimate_pairs(sk, pc, sk[:333], pc[:333], N, measures=(), variant="tc")
    assert torch.equal(c_only, c_tc)


def test_tc_estimate_rejects_unsupported_shape():
    N = 96
    c = inputs.random_csr(7, 20, 50_000, 1, 30)
    sk, pc, _ = _sketch_both(c, N, 1)
    with pytest.raises(B.BinSketchError) as e:
        api.estimate_pairs(sk, pc, sk, pc, N, variant="tc")
    assert e.value.code == 7


@pytest.mark.parametrize("N,by,m", [(384, "js", 2), (640, "cos", 3), (1152, "ham", 1)])
def test_tc_topk_odd_kchunk_counts(N, by, m):
    c = inputs.random_csr(13, 900, 300_000, 1, 600)
    sk, pc, osk = _sketch_both(c, N, 4)
    score, idx = api.topk(sk, pc, sk, pc, N, 25, by=by, exclude_self=True, variant="tc")
    oest, _ = oracle.estimate_pairs(osk, osk, N)
    s, ix = score.cpu().numpy(), u32(idx)
    for q in range(c.n):
        check_topk_row(s[q], ix[q], oest[m, q], 25, m, exclude_q=q)


def test_tc_topk_largest_k():
    # k = BS_TOPK_K_MAX: only the single-operand-slot configuration fits its heaps
    N, k = 1024, B.BS_TOPK_K_MAX
    assert B.bs_topk_plan(500, 500, N, k, B.BS_VARIANT_TC)[0]
    c = inputs.random_csr(15, 500, 200_000, 1, 400)
    sk, pc, osk = _sketch_both(c, N, 2)
    score, idx = api.topk(sk, pc, sk, pc, N, k, by="js", exclude_self=True, variant="tc")
    oest, _ = oracle.estimate_pairs(osk, osk, N)
    s, ix = score.cpu().numpy(), u32(idx)
    for q in range(0, c.n, 7):
        check_topk_row(s[q], ix[q], oest[2, q], k, 2, exclude_q=q)


def test_injected_stall_times_out_and_the_next_call_is_correct():
    # the fault is made on purpose inside the kernel's own protocol: its MMA
    # thread never announces the first accumulator, every wait of that launch
    # is bounded at ~2e6 cycles, so the waiting warps give up, raise
    # BS_ERR_TIMEOUT and the block drains and exits -- no trap, no fault
    N, k = 1024, 10
    c = inputs.random_csr(9, 2000, 200_000, 1, 300)
    sk, pc, osk = _sketch_both(c, N, 3)
    n = c.n
    score = torch.empty((n, k), dtype=torch.float32, device="cuda")
    idx = torch.empty((n, k), dtype=torch.int32, device="cuda")
    wsb = B.bs_topk_workspace_bytes(n, n, N, k)
    ws = torch.empty((wsb,), dtype=torch.uint8, device="cuda")
    B.bs_topk_ex(sk, pc, n, sk, pc, n, N, B.BS_JS, k, 1, score, idx, ws, wsb,
                 B.BS_VARIANT_TC | B.BS_VARIANT_INJECT_STALL)
    assert B.bs_get_async_error() == 6          # BS_ERR_TIMEOUT, read and cleared
    assert B.bs_get_async_error() == 0
    # the injector exists only in the tensor-core kernel
    with pytest.raises(B.BinSketchError) as e:
        B.bs_topk_ex(sk, pc, n, sk, pc, n, N, B.BS_JS, k, 1, score, idx, ws, wsb,
                     B.BS_VARIANT_POPC | B.BS_VARIANT_INJECT_STALL)
    assert e.value.code == 7
    # the same stream, the next normal call: correct against the oracle
    B.bs_topk_ex(sk, pc, n, sk, pc, n, N, B.BS_JS, k, 1, score, idx, ws, wsb, B.BS_VARIANT_TC)
    assert B.bs_get_async_error() == 0
    oest, _ = oracle.estimate_pairs(osk[:200], osk, N)
    s, ix = score.cpu().numpy(), u32(idx)
    for q in range(200):
        check_topk_row(s[q], ix[q], oest[2, q], k, 2, exclude_q=q)
