"""bs_topk_noalloc: the top-k for callers that may not allocate GPU memory.

Some callers cannot hand the library a freshly allocated workspace -- for
instance a serving process whose memory arena owns the whole device, or a
plugin running inside another framework's allocator.  bs_topk_noalloc keeps
the scratch that bs_topk would need in a fixed array inside the library.  This
file checks it through the C ABI against bs_topk (which gets a torch-allocated
workspace) on two calls in a row, and that shapes needing more scratch than
the array holds are refused.  It is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1910_04658_gb300 import inputs
from tests.helpers import assert_close, to_dev, u32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1910_04658_gb300 import api, binding as B  # noqa: E402


def _sketch(c, N):
    rp, col = to_dev(c)
    sk, pc = api.sketch(rp, col, c.d, N, 1)
    assert B.bs_get_async_error() == 0
    return sk, pc


def test_noalloc_topk_matches_topk_twice_in_a_row():
    N, k = 1024, 40
    db = inputs.random_csr(21, 12_000, 500_000, 1, 300)
    dsk, dpc = _sketch(db, N)
    queries = [inputs.random_csr(22, 50, 500_000, 1, 300), inputs.random_csr(23, 19, 500_000, 5, 200)]
    for qc, by, m in zip(queries, ("js", "cos"), (2, 3)):
        qsk, qpc = _sketch(qc, N)
        nQ, nDB = qc.n, db.n
        need = B.bs_topk_workspace_bytes(nQ, nDB, N, k)
        assert 0 < need <= B.BS_TOPK_NOALLOC_SCRATCH_BYTES   # the scratch is really used
        ref_s, ref_i = api.topk(qsk, qpc, dsk, dpc, N, k, by=by)
        s = torch.full((nQ, k), float("nan"), dtype=torch.float32, device="cuda")
        i = torch.zeros((nQ, k), dtype=torch.int32, device="cuda")
        B.bs_topk_noalloc(qsk, qpc, nQ, dsk, dpc, nDB, N, B.MEASURE_BITS[by], k, 0, s, i)
        torch.cuda.synchronize()
        assert B.bs_get_async_error() == 0
        assert np.array_equal(u32(i), u32(ref_i))
        assert_close(s.cpu().numpy(), ref_s.cpu().numpy(), m)


def test_noalloc_topk_refuses_shapes_beyond_its_scratch():
    N, k, nDB = 1024, 128, 300_000
    # a query count whose split top-k needs more scratch than the fixed array
    nQ = next(n for n in (9500, 6000, 4700, 3100, 12000, 2400)
              if B.bs_topk_workspace_bytes(n, nDB, N, k) > B.BS_TOPK_NOALLOC_SCRATCH_BYTES)
    q = torch.zeros((nQ, N // 32), dtype=torch.int32, device="cuda")
    qpc = torch.zeros((nQ,), dtype=torch.int32, device="cuda")
    db = torch.zeros((nDB, N // 32), dtype=torch.int32, device="cuda")
    dpc = torch.zeros((nDB,), dtype=torch.int32, device="cuda")
    s = torch.empty((nQ, k), dtype=torch.float32, device="cuda")
    i = torch.empty((nQ, k), dtype=torch.int32, device="cuda")
    with pytest.raises(B.BinSketchError) as e:
        B.bs_topk_noalloc(q, qpc, nQ, db, dpc, nDB, N, B.BS_JS, k, 0, s, i)
    assert e.value.code == 5   # BS_ERR_NO_MEMORY
    # a refusal leaves nothing behind: the next call on the stream succeeds
    s2 = torch.empty((3, 5), dtype=torch.float32, device="cuda")
    i2 = torch.empty((3, 5), dtype=torch.int32, device="cuda")
    B.bs_topk_noalloc(q[:3], qpc[:3], 3, db[:1000], dpc[:1000], 1000, N, B.BS_JS, 5, 0, s2, i2)
    torch.cuda.synchronize()
    assert B.bs_get_async_error() == 0
