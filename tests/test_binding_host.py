"""The Python binding refuses, before any kernel launch, tensors the C entry
points cannot take: host tensors, strided views and tensors smaller than the
call's sizes imply (runs without a GPU)."""
import pytest

torch = pytest.importorskip("torch")

from paper_1910_04658_gb300 import binding as B  # noqa: E402


class FakeCuda:
    """Stands in for a CUDA tensor of `nbytes` bytes (no device needed)."""

    def __init__(self, nbytes, contiguous=True):
        self.nbytes_, self.contiguous = nbytes, contiguous
        self.is_cuda = True
        self.device = "cuda:0"

    def is_contiguous(self):
        return self.contiguous

    def numel(self):
        return self.nbytes_

    def element_size(self):
        return 1

    def data_ptr(self):
        return 1 << 40


def test_host_tensor_is_refused():
    with pytest.raises(ValueError, match="CUDA tensor"):
        B._p(torch.zeros(4, dtype=torch.int32))


def test_strided_view_is_refused():
    with pytest.raises(ValueError, match="contiguous"):
        B._p(FakeCuda(64, contiguous=False))


def test_size_is_checked_against_the_call():
    assert B._p(FakeCuda(64), 64) == 1 << 40
    with pytest.raises(ValueError, match="needs 65"):
        B._p(FakeCuda(64), 65, "sketch")
    assert B._p(None, 100) is None and B._p(12345, 100) == 12345   # raw addresses pass as is


def test_entry_points_check_their_tensors():
    n, N, nnz = 10, 256, 40
    rp, col = FakeCuda(8 * (n + 1)), FakeCuda(4 * nnz)
    # one sketch row short
    with pytest.raises(ValueError, match="sketch"):
        B.bs_sketch(rp, col, n, nnz, 1000, N, 0, FakeCuda((n - 1) * N // 8), FakeCuda(4 * n))
    with pytest.raises(ValueError, match="col"):
        B.bs_sketch_parity(rp, FakeCuda(4 * nnz - 4), n, nnz, 1000, N, 0, FakeCuda(n * N // 8), None)
    sk, pc = FakeCuda(n * N // 8), FakeCuda(4 * n)
    # three measures need 3 * nA * nB floats
    with pytest.raises(ValueError, match="out"):
        B.bs_estimate_pairs(sk, pc, n, sk, pc, n, N, B.BS_IP | B.BS_JS | B.BS_COS, FakeCuda(4 * 2 * n * n))
    with pytest.raises(ValueError, match="idx"):
        B.bs_topk(sk, pc, n, sk, pc, n, N, B.BS_JS, 5, 1, FakeCuda(4 * n * 5), FakeCuda(4 * n * 4))
    with pytest.raises(ValueError, match="workspace"):
        B.bs_topk_ex(sk, pc, n, sk, pc, n, N, B.BS_JS, 5, 1, FakeCuda(4 * n * 5), FakeCuda(4 * n * 5),
                     FakeCuda(100), 200)
    with pytest.raises(ValueError, match="DB"):
        B.bs_topk_noalloc(sk, pc, n, FakeCuda(N // 8), pc, n, N, B.BS_JS, 5, 1, FakeCuda(4 * n * 5),
                          FakeCuda(4 * n * 5))
