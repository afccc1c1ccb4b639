"""Thin ctypes binding of libbinsketch.so (the C ABI in include/binsketch.h).

Each function has the name of the C entry point it calls and only marshals
arguments: tensors become device pointers, ``stream=None`` becomes the current
torch stream.  A tensor argument must be a contiguous CUDA tensor; for the
sketch, estimate and top-k entry points it must also hold at least the bytes
the call's sizes imply.  Anything else raises ValueError before a kernel sees
the address (an int is taken as a device address as is).  All work runs in
the library's CUDA kernels; if the library is missing, ``lib()`` raises --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "libbinsketch.so")

BS_IP, BS_HAM, BS_JS, BS_COS = 1, 2, 4, 8
BS_VARIANT_AUTO, BS_VARIANT_POPC, BS_VARIANT_TC = 0, 1, 2
VARIANTS = {"auto": 0, "popc": 1, "tc": 2}   # plus "tc0" .. "tc14" below


BS_TC_CONFIGS = 15
BS_TC_FIRST_TMA = 10   # configurations from here on read an FP4 copy of the database by TMA


def BS_VARIANT_TC_CFG(c: int) -> int:
    """Bits selecting tensor-core block configuration c (0..14) in bs_topk_ex's variant."""
    return (c + 1) << 4


VARIANTS.update({f"tc{c}": BS_VARIANT_TC | BS_VARIANT_TC_CFG(c) for c in range(BS_TC_CONFIGS)})


class bs_sketch_job(ctypes.Structure):
    """Mirror of the C struct bs_sketch_job (include/binsketch.h)."""
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("nnz", ctypes.c_uint64),
                ("seed", ctypes.c_uint64), ("n_rows", ctypes.c_uint32), ("d", ctypes.c_uint32),
                ("N", ctypes.c_uint32), ("pad_", ctypes.c_uint32), ("sketch", ctypes.c_void_p),
                ("popcnt", ctypes.c_void_p)]


class bs_topk_job(ctypes.Structure):
    """Mirror of the C struct bs_topk_job (include/binsketch.h)."""
    _fields_ = [("Q", ctypes.c_void_p), ("pcQ", ctypes.c_void_p), ("DB", ctypes.c_void_p),
                ("pcDB", ctypes.c_void_p), ("score", ctypes.c_void_p), ("idx", ctypes.c_void_p),
                ("nQ", ctypes.c_uint32), ("nDB", ctypes.c_uint32), ("N", ctypes.c_uint32),
                ("exclude_self", ctypes.c_int)]


BS_VARIANT_INJECT_STALL = 0x100
BS_TOPK_BATCH_MAX = 64
MEASURE_BITS = {"ip": BS_IP, "ham": BS_HAM, "js": BS_JS, "cos": BS_COS}
BS_TOPK_K_MAX = 128
BS_TOPK_MERGE_PARTS_MAX = 256
BS_EXACT_D_MAX = 1572864
BS_EVAL_THRESHOLDS_MAX = 16
BS_TOPK_NOALLOC_SCRATCH_BYTES = 16 << 20
BS_N_MAX = 65536
STATUS = {0: "BS_OK", 1: "BS_ERR_INVALID_ARG", 2: "BS_ERR_INDEX_RANGE", 3: "BS_ERR_ROWPTR",
          4: "BS_ERR_CUDA", 5: "BS_ERR_NO_MEMORY", 6: "BS_ERR_TIMEOUT", 7: "BS_ERR_UNSUPPORTED"}

_lock = threading.Lock()
_lib = None

# (name, restype, argtypes) of every exported entry point
_u32, _u64, _i32, _sz, _vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p
SIGNATURES = [
    ("bs_sketch", _i32, [_vp, _vp, _u32, _u64, _u32, _u32, _u64, _vp, _vp, _vp]),
    ("bs_sketch_parity", _i32, [_vp, _vp, _u32, _u64, _u32, _u32, _u64, _vp, _vp, _vp]),
    ("bs_sketch_batched", _i32, [_vp, _u32, _u32, _vp]),
    ("bs_popcount_rows", _i32, [_vp, _u32, _u32, _vp, _vp]),
    ("bs_estimate_pairs", _i32, [_vp, _vp, _u32, _vp, _vp, _u32, _u32, _u32, _vp, _vp, _vp]),
    ("bs_estimate_pairs_ex", _i32, [_vp, _vp, _u32, _vp, _vp, _u32, _u32, _u32, _vp, _vp, _u32, _vp]),
    ("bs_topk_workspace_bytes", _sz, [_u32, _u32, _u32, _u32]),
    ("bs_topk_batched_workspace_bytes", _sz, [_vp, _u32, _u32]),
    ("bs_topk_batched", _i32, [_vp, _u32, _u32, _u32, _vp, _sz, _u32, _vp]),
    ("bs_topk_batched_plan", _i32, [_vp, _u32, _u32, ctypes.POINTER(_u32), ctypes.POINTER(_u32)]),
    ("bs_topk", _i32, [_vp, _vp, _u32, _vp, _vp, _u32, _u32, _u32, _u32, _i32, _vp, _vp, _vp,
                       _sz, _vp]),
    ("bs_topk_ex", _i32, [_vp, _vp, _u32, _vp, _vp, _u32, _u32, _u32, _u32, _i32, _vp, _vp, _vp,
                          _sz, _u32, _vp]),
    ("bs_topk_shard", _i32, [_vp, _vp, _u32, _vp, _vp, _u32, _u32, _u32, _u32, _u32, _i32, _vp,
                             _vp, _vp, _sz, _u32, _vp]),
    ("bs_topk_merge", _i32, [_vp, _vp, _u32, _u32, _u32, ctypes.POINTER(_u32), _u32, _vp, _vp,
                             _vp]),
    ("bs_topk_plan", _i32, [_u32, _u32, _u32, _u32, _u32, _i32, ctypes.POINTER(_u32),
                            ctypes.POINTER(_u32), ctypes.POINTER(_u32)]),
    ("bs_tiled_bytes", _sz, [_u32, _u32]),
    ("bs_tile_sketches", _i32, [_vp, _u32, _u32, _vp, _vp]),
    ("bs_topk_pretiled_workspace_bytes", _sz, [_u32, _u32, _u32, _u32]),
    ("bs_topk_pretiled", _i32, [_vp, _vp, _u32, _vp, _vp, _u32, _u32, _u32, _u32, _vp, _vp, _vp,
                                _sz, _vp]),
    ("bs_fp4_bytes", _sz, [_u32, _u32]),
    ("bs_fp4_sketches", _i32, [_vp, _u32, _u32, _vp, _vp]),
    ("bs_topk_prewidened_workspace_bytes", _sz, [_u32, _u32, _u32, _u32]),
    ("bs_topk_prewidened", _i32, [_vp, _vp, _u32, _vp, _vp, _u32, _u32, _u32, _u32, _vp, _vp, _vp,
                                  _sz, _vp]),
    ("bs_topk_noalloc", _i32, [_vp, _vp, _u32, _vp, _vp, _u32, _u32, _u32, _u32, _i32, _vp, _vp,
                               _vp]),
    ("bs_onehot_csr", _i32, [_vp, _u32, _u32, _vp, _vp, _vp, _vp]),
    ("bs_exact_counts", _i32, [_vp, _vp, _u32, _u64, _vp, _vp, _u32, _u64, _u32, _vp, _vp, _vp, _vp]),
    ("bs_threshold_eval", _i32, [_vp, _vp, _vp, _vp, _u32, _u32, _u32, ctypes.POINTER(ctypes.c_double),
                                 _u32, _vp, _vp]),
    ("bs_dense_pairs", _i32, [_u32, _u32, _u32, _u32, _u32, _u64, _u64, _vp, _vp, _vp, _u32, _vp]),
    ("bs_estimate_counts", _i32, [_vp, _u32, _u32, _vp, _vp]),
    ("bs_mlp_prepare", _i32, [_vp, _vp, _u32, _u32, _vp, _vp, _vp]),
    ("bs_mlp_train_step", _i32, [_vp, _vp, _vp, _vp, _u32, ctypes.c_float, _vp, _vp, _u32, _vp, _vp]),
    ("bs_mlp_estimate", _i32, [_vp, _vp, _u32, _u32, _vp, _vp]),
    ("bs_mlp_estimate_ex", _i32, [_vp, _vp, _u32, _u32, _vp, _u32, _vp]),
    ("bs_get_async_error", _i32, [_vp]),
    ("bs_hash_params", None, [_u64, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    ("bs_status_string", ctypes.c_char_p, [_i32]),
    ("bs_version", _i32, []),
]


class BinSketchError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is not built; run paper_1910_04658_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(x, nbytes: int = 0, name: str = "argument"):
    """Device address of `x`: None, an int (taken as a device address as is),
    or a contiguous CUDA tensor of at least `nbytes` bytes.  A host tensor, a
    strided view or a tensor too small for the call raises ValueError here
    instead of reaching a kernel."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise ValueError(f"{name}: a CUDA tensor is required, got one on {x.device}")
    if not x.is_contiguous():
        raise ValueError(f"{name}: the tensor must be contiguous")
    have = x.numel() * x.element_size()
    if have < nbytes:
        raise ValueError(f"{name}: {have} bytes, the call needs {nbytes}")
    return x.data_ptr()


def _nmeasures(measures: int) -> int:
    return bin(int(measures) & 15).count("1")


def _s(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(rc, where):
    if rc != 0:
        raise BinSketchError(rc, where)


def _sketch_args(row_ptr, col, n_rows, nnz, N, sketch, popcnt):
    return (_p(row_ptr, 8 * (n_rows + 1) if n_rows else 0, "row_ptr"), _p(col, 4 * nnz, "col"), n_rows,
            nnz), (_p(sketch, n_rows * (N // 8), "sketch"), _p(popcnt, 4 * n_rows, "popcnt"))


def bs_sketch(row_ptr, col, n_rows, nnz, d, N, seed, sketch, popcnt=None, stream=None):
    (rp, c, n, z), (sk, pc) = _sketch_args(row_ptr, col, n_rows, nnz, N, sketch, popcnt)
    _check(lib().bs_sketch(rp, c, n, z, d, N, seed, sk, pc, _s(stream)), "bs_sketch")


def bs_sketch_batched(jobs_dev, n_jobs, max_N, stream=None):
    """jobs_dev: device pointer (or tensor) to n_jobs packed bs_sketch_job structs."""
    _check(lib().bs_sketch_batched(_p(jobs_dev), n_jobs, max_N, _s(stream)), "bs_sketch_batched")


def bs_sketch_parity(row_ptr, col, n_rows, nnz, d, N, seed, sketch, popcnt=None, stream=None):
    (rp, c, n, z), (sk, pc) = _sketch_args(row_ptr, col, n_rows, nnz, N, sketch, popcnt)
    _check(lib().bs_sketch_parity(rp, c, n, z, d, N, seed, sk, pc, _s(stream)), "bs_sketch_parity")


def bs_popcount_rows(sketch, n_rows, N, popcnt, stream=None):
    sk, pc = _p(sketch, n_rows * (N // 8), "sketch"), _p(popcnt, 4 * n_rows, "popcnt")
    _check(lib().bs_popcount_rows(sk, n_rows, N, pc, _s(stream)), "bs_popcount_rows")


def bs_estimate_pairs(A, pcA, nA, B, pcB, nB, N, measures, out=None, counts=None, stream=None):
    pairs = nA * nB
    a, pa = _p(A, nA * (N // 8), "A"), _p(pcA, 4 * nA, "pcA")
    b, pb = _p(B, nB * (N // 8), "B"), _p(pcB, 4 * nB, "pcB")
    o, c = _p(out, 4 * _nmeasures(measures) * pairs, "out"), _p(counts, 4 * pairs, "counts")
    _check(lib().bs_estimate_pairs(a, pa, nA, b, pb, nB, N, measures, o, c, _s(stream)),
           "bs_estimate_pairs")


def bs_estimate_pairs_ex(A, pcA, nA, B, pcB, nB, N, measures, out=None, counts=None, variant=0,
                         stream=None):
    pairs = nA * nB
    a, pa = _p(A, nA * (N // 8), "A"), _p(pcA, 4 * nA, "pcA")
    b, pb = _p(B, nB * (N // 8), "B"), _p(pcB, 4 * nB, "pcB")
    o, c = _p(out, 4 * _nmeasures(measures) * pairs, "out"), _p(counts, 4 * pairs, "counts")
    _check(lib().bs_estimate_pairs_ex(a, pa, nA, b, pb, nB, N, measures, o, c, variant, _s(stream)),
           "bs_estimate_pairs_ex")


def _job_table(jobs):
    """jobs: sequence of dicts with Q, pcQ, DB, pcDB, score, idx, nQ, nDB, N, exclude_self
    (tensors or device addresses) -> a HOST ctypes array of bs_topk_job."""
    arr = (bs_topk_job * len(jobs))()
    for i, j in enumerate(jobs):
        nQ, nDB, N = int(j["nQ"]), int(j["nDB"]), int(j["N"])
        k = int(j.get("k", 0))
        arr[i].Q = _p(j["Q"], nQ * (N // 8), "Q")
        arr[i].pcQ = _p(j["pcQ"], 4 * nQ, "pcQ")
        arr[i].DB = _p(j["DB"], nDB * (N // 8), "DB")
        arr[i].pcDB = _p(j["pcDB"], 4 * nDB, "pcDB")
        arr[i].score = _p(j["score"], 4 * nQ * k, "score")
        arr[i].idx = _p(j["idx"], 4 * nQ * k, "idx")
        arr[i].nQ, arr[i].nDB, arr[i].N = nQ, nDB, N
        arr[i].exclude_self = int(bool(j.get("exclude_self", False)))
    return arr


def bs_topk_batched_workspace_bytes(jobs, k) -> int:
    """jobs: a ctypes array from _job_table, or a sequence of job dicts."""
    arr = jobs if isinstance(jobs, ctypes.Array) else _job_table(jobs)
    return int(lib().bs_topk_batched_workspace_bytes(arr, len(arr), k))


def bs_topk_batched(jobs, by, k, workspace=None, workspace_bytes=0, variant=0, stream=None):
    """jobs: a sequence of job dicts (see _job_table; each with its k for the size checks)
    or a prepared ctypes array of bs_topk_job."""
    arr = jobs if isinstance(jobs, ctypes.Array) else _job_table([dict(j, k=k) for j in jobs])
    _check(lib().bs_topk_batched(arr, len(arr), by, k, _p(workspace, workspace_bytes, "workspace"),
                                 workspace_bytes, variant, _s(stream)), "bs_topk_batched")


def bs_topk_batched_plan(jobs, k):
    """(splits, launches) of a bs_topk_batched call on this job table."""
    arr = jobs if isinstance(jobs, ctypes.Array) else _job_table(jobs)
    s, l = _u32(), _u32()
    _check(lib().bs_topk_batched_plan(arr, len(arr), k, ctypes.byref(s), ctypes.byref(l)),
           "bs_topk_batched_plan")
    return int(s.value), int(l.value)


def bs_topk_workspace_bytes(nQ, nDB, N, k) -> int:
    return int(lib().bs_topk_workspace_bytes(nQ, nDB, N, k))


def _topk_args(Q, pcQ, nQ, DB, pcDB, nDB, N, k, score, idx, workspace, workspace_bytes):
    return (_p(Q, nQ * (N // 8), "Q"), _p(pcQ, 4 * nQ, "pcQ"), _p(DB, nDB * (N // 8), "DB"),
            _p(pcDB, 4 * nDB, "pcDB"), _p(score, 4 * nQ * k, "score"), _p(idx, 4 * nQ * k, "idx"),
            _p(workspace, workspace_bytes, "workspace"))


def bs_topk(Q, pcQ, nQ, DB, pcDB, nDB, N, by, k, exclude_self, score, idx, workspace=None,
            workspace_bytes=0, stream=None):
    q, pq, db, pdb, sc, ix, ws = _topk_args(Q, pcQ, nQ, DB, pcDB, nDB, N, k, score, idx, workspace,
                                            workspace_bytes)
    _check(lib().bs_topk(q, pq, nQ, db, pdb, nDB, N, by, k, int(exclude_self), sc, ix, ws,
                         workspace_bytes, _s(stream)), "bs_topk")


def bs_topk_ex(Q, pcQ, nQ, DB, pcDB, nDB, N, by, k, exclude_self, score, idx, workspace=None,
               workspace_bytes=0, variant=0, stream=None):
    q, pq, db, pdb, sc, ix, ws = _topk_args(Q, pcQ, nQ, DB, pcDB, nDB, N, k, score, idx, workspace,
                                            workspace_bytes)
    _check(lib().bs_topk_ex(q, pq, nQ, db, pdb, nDB, N, by, k, int(exclude_self), sc, ix, ws,
                            workspace_bytes, variant, _s(stream)), "bs_topk_ex")


def bs_topk_shard(Q, pcQ, nQ, DB, pcDB, nDB, db_offset, N, by, k, exclude_self, score, idx,
                  workspace=None, workspace_bytes=0, variant=0, stream=None):
    q, pq, db, pdb, sc, ix, ws = _topk_args(Q, pcQ, nQ, DB, pcDB, nDB, N, k, score, idx, workspace,
                                            workspace_bytes)
    _check(lib().bs_topk_shard(q, pq, nQ, db, pdb, nDB, db_offset, N, by, k, int(exclude_self), sc,
                               ix, ws, workspace_bytes, variant, _s(stream)), "bs_topk_shard")


def bs_topk_merge(score_parts, idx_parts, parts, nQ, k, part_offset, by, score, idx, stream=None):
    """part_offset: a sequence of `parts` ints (host), or None."""
    offs = None if part_offset is None else (_u32 * parts)(*[int(o) for o in part_offset])
    _check(lib().bs_topk_merge(_p(score_parts), _p(idx_parts), parts, nQ, k, offs, by, _p(score),
                               _p(idx), _s(stream)), "bs_topk_merge")


def bs_onehot_csr(labels, n, F, offsets, row_ptr, col, stream=None):
    _check(lib().bs_onehot_csr(_p(labels), n, F, _p(offsets), _p(row_ptr), _p(col), _s(stream)),
           "bs_onehot_csr")


def bs_exact_counts(q_row_ptr, q_col, nq, q_nnz, db_row_ptr, db_col, ndb, db_nnz, d, counts,
                    q_sizes=None, db_sizes=None, stream=None):
    _check(lib().bs_exact_counts(_p(q_row_ptr), _p(q_col), nq, q_nnz, _p(db_row_ptr), _p(db_col), ndb,
                                 db_nnz, d, _p(counts), _p(q_sizes), _p(db_sizes), _s(stream)),
           "bs_exact_counts")


def bs_threshold_eval(est, counts, q_sizes, db_sizes, nq, ndb, by, thresholds, out, stream=None):
    """thresholds: a sequence of floats (host)."""
    th = (ctypes.c_double * len(thresholds))(*[float(t) for t in thresholds])
    _check(lib().bs_threshold_eval(_p(est), _p(counts), _p(q_sizes), _p(db_sizes), nq, ndb, by, th,
                                   len(thresholds), _p(out), _s(stream)), "bs_threshold_eval")


def bs_topk_plan(nQ, nDB, N, k, variant=0, same_matrix=False):
    """(uses_tc, splits, launches) of a bs_topk_ex call of this shape."""
    u, s, l = _u32(), _u32(), _u32()
    _check(lib().bs_topk_plan(nQ, nDB, N, k, variant, int(same_matrix), ctypes.byref(u),
                              ctypes.byref(s), ctypes.byref(l)), "bs_topk_plan")
    return bool(u.value), int(s.value), int(l.value)


def bs_tiled_bytes(n_rows, N) -> int:
    return int(lib().bs_tiled_bytes(n_rows, N))


def bs_tile_sketches(sketch, n_rows, N, tiled, stream=None):
    _check(lib().bs_tile_sketches(_p(sketch), n_rows, N, _p(tiled), _s(stream)), "bs_tile_sketches")


def bs_topk_pretiled_workspace_bytes(nQ, nDB, N, k) -> int:
    return int(lib().bs_topk_pretiled_workspace_bytes(nQ, nDB, N, k))


def bs_topk_pretiled(Q, pcQ, nQ, DB_tiled, pcDB, nDB, N, by, k, score, idx, workspace=None,
                     workspace_bytes=0, stream=None):
    _check(lib().bs_topk_pretiled(_p(Q), _p(pcQ), nQ, _p(DB_tiled), _p(pcDB), nDB, N, by, k,
                                  _p(score), _p(idx), _p(workspace), workspace_bytes, _s(stream)),
           "bs_topk_pretiled")


def bs_fp4_bytes(n_rows, N) -> int:
    return int(lib().bs_fp4_bytes(n_rows, N))


def bs_fp4_sketches(sketch, n_rows, N, fp4, stream=None):
    _check(lib().bs_fp4_sketches(_p(sketch, n_rows * (N // 8), "sketch"), n_rows, N,
                                 _p(fp4, n_rows * (N // 2), "fp4"), _s(stream)), "bs_fp4_sketches")


def bs_topk_prewidened_workspace_bytes(nQ, nDB, N, k) -> int:
    return int(lib().bs_topk_prewidened_workspace_bytes(nQ, nDB, N, k))


def bs_topk_prewidened(Q, pcQ, nQ, DB_fp4, pcDB, nDB, N, by, k, score, idx, workspace=None,
                       workspace_bytes=0, stream=None):
    _check(lib().bs_topk_prewidened(_p(Q, nQ * (N // 8), "Q"), _p(pcQ, 4 * nQ, "pcQ"), nQ,
                                    _p(DB_fp4, nDB * (N // 2), "DB_fp4"), _p(pcDB, 4 * nDB, "pcDB"),
                                    nDB, N, by, k, _p(score, 4 * nQ * k, "score"), _p(idx, 4 * nQ * k, "idx"),
                                    _p(workspace), workspace_bytes, _s(stream)), "bs_topk_prewidened")


def bs_topk_noalloc(Q, pcQ, nQ, DB, pcDB, nDB, N, by, k, exclude_self, score, idx, stream=None):
    q, pq, db, pdb, sc, ix, _ = _topk_args(Q, pcQ, nQ, DB, pcDB, nDB, N, k, score, idx, None, 0)
    _check(lib().bs_topk_noalloc(q, pq, nQ, db, pdb, nDB, N, by, k, int(exclude_self), sc, ix,
                                 _s(stream)), "bs_topk_noalloc")


BS_MLP_PARAMS = 4740


def bs_dense_pairs(n_pairs, N, d, size_lo, size_hi, pair_seed, hash_seed, counts, sizes=None,
                   cols=None, max_cols=0, stream=None):
    _check(lib().bs_dense_pairs(n_pairs, N, d, size_lo, size_hi, pair_seed, hash_seed, _p(counts),
                                _p(sizes), _p(cols), max_cols, _s(stream)), "bs_dense_pairs")


def bs_estimate_counts(counts, n, N, out, stream=None):
    _check(lib().bs_estimate_counts(_p(counts), n, N, _p(out), _s(stream)), "bs_estimate_counts")


def bs_mlp_prepare(counts, sizes, n, N, x, t=None, stream=None):
    _check(lib().bs_mlp_prepare(_p(counts), _p(sizes), n, N, _p(x), _p(t), _s(stream)),
           "bs_mlp_prepare")


def bs_mlp_train_step(params, adam_m, adam_v, grad, step, lr, x, t, n, loss=None, stream=None):
    _check(lib().bs_mlp_train_step(_p(params), _p(adam_m), _p(adam_v), _p(grad), step, lr, _p(x),
                                   _p(t), n, _p(loss), _s(stream)), "bs_mlp_train_step")


def bs_mlp_estimate(params, counts, n, N, out, stream=None):
    _check(lib().bs_mlp_estimate(_p(params), _p(counts), n, N, _p(out), _s(stream)),
           "bs_mlp_estimate")


def bs_mlp_estimate_ex(params, counts, n, N, out, variant=0, stream=None):
    _check(lib().bs_mlp_estimate_ex(_p(params), _p(counts), n, N, _p(out), variant, _s(stream)),
           "bs_mlp_estimate_ex")


def bs_get_async_error(stream=None) -> int:
    return int(lib().bs_get_async_error(_s(stream)))


def bs_hash_params(seed: int):
    m, a = _u64(), _u64()
    lib().bs_hash_params(seed, ctypes.byref(m), ctypes.byref(a))
    return m.value, a.value


def bs_status_string(code: int) -> str:
    return lib().bs_status_string(code).decode()


def bs_version() -> int:
    return int(lib().bs_version())
