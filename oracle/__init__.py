"""BinSketch CPU oracle (FP64) -- test infrastructure only.

A plain restatement of BinSketch (arXiv 1910.04658) used to check the CUDA
library: sketching (Definition "BinSketch", Sec. 3), the sketch counts and the
estimators of Alg. 1-4 (Sec. 3.1-3.4), the ranking of Experiment 2 (Sec. 4) as
a top-k and as thresholded retrieval sets, the categorical front end, and
exact similarities as ground truth.  Only ``tests/``, the smoke
check and the CPU-baseline leg of the benchmark may import this package; the
product path never does.  It shares no code with the CUDA library.

The arithmetic lives in ``bs_oracle.c`` (plain C, FP64, OpenMP over rows) and is
compiled with gcc on first use; this module only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libbs_oracle.so")
_lock = threading.Lock()
_lib = None

IP, HAM, JS, COS = 0, 1, 2, 3
MEASURES = {"ip": IP, "ham": HAM, "js": JS, "cos": COS}


def compile_library(src: str, out: str) -> str:
    """gcc with the oracle's flags (portable, no FMA contraction): src -> out."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC",
           "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile bs_oracle.c into _build/ unless the library is up to date."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_library(_SRC, _LIB_PATH)


def _library_path() -> str:
    # BS_ORACLE_LIB names another build of bs_oracle.c to load instead; the
    # mutation tests use it to run the pins against copies with a planted
    # mistake and check that a pin fails.
    alt = os.environ.get("BS_ORACLE_LIB")
    return alt if alt else build()


def _P(t):
    return ctypes.POINTER(t)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(_library_path())
            u32, u64, i32, f64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
            L.bso_hash_params.argtypes = [u64, _P(u64), _P(u64)]
            L.bso_bucket.argtypes = [u64, u64, u32, u32]
            L.bso_bucket.restype = u32
            L.bso_mapping_table.argtypes = [u64, u32, u32, _P(u32)]
            L.bso_sketch_map.argtypes = [_P(u64), _P(u32), u32, u32, u32, _P(u32), _P(u32), _P(u32)]
            L.bso_sketch_map.restype = i32
            L.bso_sketch.argtypes = [_P(u64), _P(u32), u32, u32, u32, u64, _P(u32), _P(u32)]
            L.bso_sketch.restype = i32
            L.bso_sketch_parity.argtypes = [_P(u64), _P(u32), u32, u32, u32, u64, _P(u32), _P(u32)]
            L.bso_sketch_parity.restype = i32
            L.bso_popcount_row.argtypes = [_P(u32), u32]
            L.bso_popcount_row.restype = u32
            L.bso_counts.argtypes = [_P(u32), u32, _P(u32), u32, u32, _P(u32)]
            L.bso_estimate.argtypes = [f64, f64, f64, u32, i32, _P(f64), _P(f64), _P(f64)]
            L.bso_estimate_pairs.argtypes = [_P(u32), u32, _P(u32), u32, u32, _P(f64), _P(u32)]
            L.bso_topk.argtypes = [_P(u32), u32, _P(u32), u32, u32, i32, u32, i32,
                                   _P(f64), _P(u32), _P(u32)]
            L.bso_exact_pairs.argtypes = [_P(u64), _P(u32), _P(u32), _P(u32), u64, _P(f64)]
            L.bso_num_threads.restype = i32
            _lib = L
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(_P(t))


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(lib().bso_num_threads())


def hash_params(seed: int):
    m, a = ctypes.c_uint64(), ctypes.c_uint64()
    lib().bso_hash_params(ctypes.c_uint64(seed), ctypes.byref(m), ctypes.byref(a))
    return m.value, a.value


def bucket(seed: int, N: int, i: int) -> int:
    m, a = hash_params(seed)
    return int(lib().bso_bucket(m, a, N, i))


def mapping_table(seed: int, N: int, d: int) -> np.ndarray:
    pi = np.empty(d, np.uint32)
    lib().bso_mapping_table(seed, N, d, _ptr(pi, ctypes.c_uint32))
    return pi


def sketch(row_ptr, col, d: int, N: int, seed: int = 0, pi=None, parity: bool = False):
    """Packed sketches [n][ceil(N/32)] uint32 and |a_s| [n] uint32.

    ``pi`` (optional, uint32[d]) replaces the seeded hash by an explicit random
    mapping.  ``parity`` gives the BCS sketch (Definition "BCS", Sec. 2)."""
    row_ptr = _c(row_ptr, np.uint64)
    col = _c(col, np.uint32)
    n = row_ptr.shape[0] - 1
    sk = np.zeros((n, (N + 31) // 32), np.uint32)
    pc = np.zeros(n, np.uint32)
    L = lib()
    if pi is not None:
        pi = _c(pi, np.uint32)
        assert pi.shape[0] >= d
        rc = L.bso_sketch_map(_ptr(row_ptr, ctypes.c_uint64), _ptr(col, ctypes.c_uint32), n, d, N,
                              _ptr(pi, ctypes.c_uint32), _ptr(sk, ctypes.c_uint32),
                              _ptr(pc, ctypes.c_uint32))
    elif parity:
        rc = L.bso_sketch_parity(_ptr(row_ptr, ctypes.c_uint64), _ptr(col, ctypes.c_uint32), n, d,
                                 N, seed, _ptr(sk, ctypes.c_uint32), _ptr(pc, ctypes.c_uint32))
    else:
        rc = L.bso_sketch(_ptr(row_ptr, ctypes.c_uint64), _ptr(col, ctypes.c_uint32), n, d, N,
                          seed, _ptr(sk, ctypes.c_uint32), _ptr(pc, ctypes.c_uint32))
    if rc == -1:
        raise ValueError("column index >= d")
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return sk, pc


def counts(A, B) -> np.ndarray:
    A = _c(A, np.uint32)
    B = _c(B, np.uint32)
    assert A.shape[1] == B.shape[1]
    c = np.zeros((A.shape[0], B.shape[0]), np.uint32)
    lib().bso_counts(_ptr(A, ctypes.c_uint32), A.shape[0], _ptr(B, ctypes.c_uint32), B.shape[0],
                     A.shape[1], _ptr(c, ctypes.c_uint32))
    return c


def estimate(nas: float, nbs: float, nasbs: float, N: int, paper_literal_ham: bool = False):
    """(IP, Ham, JS, Cos, n_a, n_b) for one pair of counts (Alg. 1-4)."""
    out = (ctypes.c_double * 4)()
    na, nb = ctypes.c_double(), ctypes.c_double()
    lib().bso_estimate(float(nas), float(nbs), float(nasbs), N, int(paper_literal_ham), out,
                       ctypes.byref(na), ctypes.byref(nb))
    return out[0], out[1], out[2], out[3], na.value, nb.value


def estimate_pairs(A, B, N: int):
    """All estimates [4][nA][nB] (IP, Ham, JS, Cos) and counts [nA][nB]."""
    A = _c(A, np.uint32)
    B = _c(B, np.uint32)
    nA, nB = A.shape[0], B.shape[0]
    out = np.zeros((4, nA, nB), np.float64)
    c = np.zeros((nA, nB), np.uint32)
    lib().bso_estimate_pairs(_ptr(A, ctypes.c_uint32), nA, _ptr(B, ctypes.c_uint32), nB, N,
                             _ptr(out, ctypes.c_double), _ptr(c, ctypes.c_uint32))
    return out, c


def topk(Q, DB, N: int, measure: int, k: int, exclude_self: bool = False):
    """Per query row the k best DB rows: (score[nQ][k], idx[nQ][k], count[nQ][k])."""
    Q = _c(Q, np.uint32)
    DB = _c(DB, np.uint32)
    nQ, nDB = Q.shape[0], DB.shape[0]
    score = np.zeros((nQ, k), np.float64)
    idx = np.zeros((nQ, k), np.uint32)
    cnt = np.zeros((nQ, k), np.uint32)
    lib().bso_topk(_ptr(Q, ctypes.c_uint32), nQ, _ptr(DB, ctypes.c_uint32), nDB, N, int(measure),
                   k, int(exclude_self), _ptr(score, ctypes.c_double), _ptr(idx, ctypes.c_uint32),
                   _ptr(cnt, ctypes.c_uint32))
    return score, idx, cnt


def exact_pairs(row_ptr, col, pa, pb) -> np.ndarray:
    """Exact (IP, Ham, JS, Cos) [n_pairs][4] of CSR rows pa[t], pb[t]."""
    row_ptr = _c(row_ptr, np.uint64)
    col = _c(col, np.uint32)
    pa = _c(pa, np.uint32)
    pb = _c(pb, np.uint32)
    out = np.zeros((pa.shape[0], 4), np.float64)
    lib().bso_exact_pairs(_ptr(row_ptr, ctypes.c_uint64), _ptr(col, ctypes.c_uint32),
                          _ptr(pa, ctypes.c_uint32), _ptr(pb, ctypes.c_uint32), pa.shape[0],
                          _ptr(out, ctypes.c_double))
    return out


def threshold_sets(est, exact, thresholds, distance: bool = False) -> np.ndarray:
    """Experiment 2 (Sec. 4, "Ranking"): for each query row q and threshold
    thr, the ground-truth set O = {j : exact[q, j] >= thr} (a distance: <=),
    the retrieved set O' = {j : est[q, j] >= thr} (<=), and their overlap.
    Returns counts [nq][T][3] = (|O|, |O'|, |O n O'|); both sides are compared
    with thr in FP64."""
    est = np.asarray(est, np.float64)
    exact = np.asarray(exact, np.float64)
    out = np.zeros((est.shape[0], len(thresholds), 3), np.int64)
    for t, thr in enumerate(thresholds):
        thr = float(thr)
        O = exact <= thr if distance else exact >= thr
        R = est <= thr if distance else est >= thr
        out[:, t, 0] = O.sum(1)
        out[:, t, 1] = R.sum(1)
        out[:, t, 2] = (O & R).sum(1)
    return out


def categorical_distance(u, v) -> int:
    """Sec. 1, categorical extension: the number of features on which the
    categorical rows u and v differ (the sum over features of 1[u_i != v_i])."""
    return sum(1 for a, b in zip(u, v) if a != b)


def onehot(labels, cardinalities):
    """One-hot encoding of label-encoded rows (Sec. 1, categorical extension):
    feature f, label l -> binary column (m_0 + ... + m_{f-1}) + l.  Returns
    (row_ptr, col, d) as a CSR batch."""
    labels = np.asarray(labels)
    n, F = labels.shape
    starts = [0]
    for m in cardinalities:
        starts.append(starts[-1] + int(m))
    row_ptr = np.zeros(n + 1, np.uint64)
    cols = []
    for i in range(n):
        for f in range(F):
            cols.append(starts[f] + int(labels[i, f]))
        row_ptr[i + 1] = len(cols)
    return row_ptr, np.array(cols, np.uint32), starts[-1]

