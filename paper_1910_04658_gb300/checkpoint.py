"""Checkpoints: the learned estimator's training state and sketch databases.

One binary format for both: a 32-byte header

    magic  b"BSCK"   (4 bytes)
    version          uint32 (1)
    kind             uint32 (1: MLP state, 2: sketch database)
    payload bytes    uint64
    payload crc32    uint32
    reserved         uint32 (0)
    meta bytes       uint32

then `meta bytes` of little-endian uint64 fields, then the payload.

* MLP state (kind 1): meta (step, n_params); payload = FP32 master weights,
  Adam first and second moments (n_params each).  The weights are kept in
  FP32 and rounded to BF16 by the kernels on use, so a resumed run continues
  from exactly the saved state.
* Sketch database (kind 2): meta (N, seed, n, words = N/32, d); payload =
  sketches uint32[n][words] then popcounts uint32[n].  A sketch means
  something only under its (seed, N), so both travel with it and a loader can
  refuse a database made with another hash.

Files are written to a temporary name and renamed, so a crash never leaves a
half-written checkpoint under the final name.
"""
from __future__ import annotations

import os
import struct
import zlib
from dataclasses import dataclass

import numpy as np

MAGIC = b"BSCK"
VERSION = 1
KIND_MLP, KIND_SKETCHES = 1, 2
_HDR = struct.Struct("<4sIIQIII")   # magic, version, kind, payload bytes, crc, reserved, meta bytes


class CheckpointError(ValueError):
    pass


def _write(path: str, kind: int, meta, payload: bytes):
    mb = struct.pack(f"<{len(meta)}Q", *[int(v) for v in meta])
    hdr = _HDR.pack(MAGIC, VERSION, kind, len(payload), zlib.crc32(payload) & 0xFFFFFFFF, 0, len(mb))
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "wb") as f:
        f.write(hdr)
        f.write(mb)
        f.write(payload)
    os.replace(tmp, path)


def _read(path: str, kind: int):
    with open(path, "rb") as f:
        raw = f.read()
    if len(raw) < _HDR.size:
        raise CheckpointError("truncated header")
    magic, ver, k, plen, crc, _, mlen = _HDR.unpack_from(raw, 0)
    if magic != MAGIC:
        raise CheckpointError("not a BinSketch checkpoint")
    if ver != VERSION:
        raise CheckpointError(f"unsupported version {ver}")
    if k != kind:
        raise CheckpointError(f"checkpoint kind {k}, expected {kind}")
    if mlen % 8 or len(raw) != _HDR.size + mlen + plen:
        raise CheckpointError("size mismatch (truncated or extended file)")
    meta = struct.unpack_from(f"<{mlen // 8}Q", raw, _HDR.size)
    payload = raw[_HDR.size + mlen:]
    if zlib.crc32(payload) & 0xFFFFFFFF != crc:
        raise CheckpointError("payload checksum mismatch")
    return meta, payload


def _host_f32(t) -> np.ndarray:
    return t.detach().to("cpu").contiguous().numpy().astype(np.float32, copy=False)


# ---------------------------------------------------------------------- MLP

def save_mlp(path: str, mlp) -> None:
    """Weights and Adam state of a learned.MLPEstimator."""
    p, m, v = _host_f32(mlp.params), _host_f32(mlp.m), _host_f32(mlp.v)
    _write(path, KIND_MLP, (mlp.step, p.size), p.tobytes() + m.tobytes() + v.tobytes())


def load_mlp(path: str, device: str = "cuda"):
    """A learned.MLPEstimator on `device` with the saved weights, moments and step."""
    import torch

    from . import binding as B
    from .learned import MLPEstimator
    (step, n), payload = _read(path, KIND_MLP)
    if n != B.BS_MLP_PARAMS or len(payload) != 3 * 4 * n:
        raise CheckpointError(f"{n} parameters, expected {B.BS_MLP_PARAMS}")
    arr = np.frombuffer(payload, np.float32).reshape(3, n)
    mlp = MLPEstimator(device=device)
    for dst, src in zip((mlp.params, mlp.m, mlp.v), arr):
        dst.copy_(torch.from_numpy(src.copy()))
    mlp.step = int(step)
    return mlp


# ------------------------------------------------------------- sketch database

@dataclass
class SketchMeta:
    N: int
    seed: int
    n: int
    d: int


def save_sketches(path: str, sketch, popcnt, N: int, seed: int, d: int) -> None:
    """sketch int32/uint32 [n][N/32], popcnt [n] (any device)."""
    sk = sketch.detach().to("cpu").contiguous().numpy().view(np.uint32)
    pc = popcnt.detach().to("cpu").contiguous().numpy().view(np.uint32)
    n = sk.shape[0]
    if sk.shape != (n, N // 32) or pc.shape != (n,):
        raise CheckpointError("sketch / popcount shapes do not match N")
    _write(path, KIND_SKETCHES, (N, seed, n, N // 32, d), sk.tobytes() + pc.tobytes())


def load_sketches(path: str, device: str = "cuda", expect_N: int = None, expect_seed: int = None):
    """(sketch int32 [n][N/32], popcnt int32 [n], SketchMeta) on `device`;
    refuses a database made with another (N, seed) than the one expected."""
    import torch
    (N, seed, n, words, d), payload = _read(path, KIND_SKETCHES)
    if words * 32 != N or len(payload) != 4 * n * (words + 1):
        raise CheckpointError("inconsistent sketch database header")
    if expect_N is not None and N != expect_N:
        raise CheckpointError(f"database sketched with N = {N}, expected {expect_N}")
    if expect_seed is not None and seed != expect_seed:
        raise CheckpointError(f"database sketched with seed {seed}, expected {expect_seed}")
    arr = np.frombuffer(payload, np.uint32)
    sk = torch.from_numpy(arr[: n * words].reshape(n, words).view(np.int32).copy()).to(device)
    pc = torch.from_numpy(arr[n * words:].view(np.int32).copy()).to(device)
    return sk, pc, SketchMeta(int(N), int(seed), int(n), int(d))
