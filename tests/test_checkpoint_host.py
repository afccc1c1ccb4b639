"""Checkpoint format (no GPU): round trips of the learned estimator's state
and of sketch databases, and rejection of damaged or mismatched files."""
import numpy as np
import pytest
import torch

from paper_1910_04658_gb300 import checkpoint
from paper_1910_04658_gb300.learned import MLPEstimator


def test_mlp_roundtrip(tmp_path):
    m = MLPEstimator(device="cpu", seed=3)
    m.params += torch.linspace(-1, 1, m.params.numel())
    m.m.fill_(0.25)
    m.v.copy_(torch.arange(m.v.numel(), dtype=torch.float32))
    m.step = 1234
    p = str(tmp_path / "mlp.bsck")
    checkpoint.save_mlp(p, m)
    r = checkpoint.load_mlp(p, device="cpu")
    assert r.step == 1234
    for a, b in ((m.params, r.params), (m.m, r.m), (m.v, r.v)):
        assert torch.equal(a, b)


def test_sketch_roundtrip_and_hash_check(tmp_path):
    rng = np.random.default_rng(0)
    sk = torch.from_numpy(rng.integers(0, 2**32, (37, 8), dtype=np.uint64).astype(np.uint32).view(np.int32))
    pc = torch.from_numpy(np.array([bin(int(x)).count("1") for x in range(37)], np.int32))
    p = str(tmp_path / "db.bsck")
    checkpoint.save_sketches(p, sk, pc, N=256, seed=99, d=5000)
    s2, p2, meta = checkpoint.load_sketches(p, device="cpu", expect_N=256, expect_seed=99)
    assert torch.equal(s2, sk) and torch.equal(p2, pc)
    assert (meta.N, meta.seed, meta.n, meta.d) == (256, 99, 37, 5000)
    with pytest.raises(checkpoint.CheckpointError, match="seed"):
        checkpoint.load_sketches(p, device="cpu", expect_seed=98)
    with pytest.raises(checkpoint.CheckpointError, match="N ="):
        checkpoint.load_sketches(p, device="cpu", expect_N=512)
    with pytest.raises(checkpoint.CheckpointError):
        checkpoint.save_sketches(p, sk, pc, N=512, seed=1, d=1)     # shape does not match N


def test_damaged_files_are_rejected(tmp_path):
    m = MLPEstimator(device="cpu")
    p = str(tmp_path / "mlp.bsck")
    checkpoint.save_mlp(p, m)
    raw = bytearray(open(p, "rb").read())
    bad = bytearray(raw)
    bad[-5] ^= 0x40
    open(p, "wb").write(bad)
    with pytest.raises(checkpoint.CheckpointError, match="checksum"):
        checkpoint.load_mlp(p, device="cpu")
    open(p, "wb").write(raw[:-12])
    with pytest.raises(checkpoint.CheckpointError, match="size"):
        checkpoint.load_mlp(p, device="cpu")
    open(p, "wb").write(b"XXXX" + raw[4:])
    with pytest.raises(checkpoint.CheckpointError, match="not a BinSketch"):
        checkpoint.load_mlp(p, device="cpu")
    open(p, "wb").write(raw)
    with pytest.raises(checkpoint.CheckpointError, match="kind"):
        checkpoint.load_sketches(p, device="cpu")
