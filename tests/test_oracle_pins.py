"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each compares the oracle with an
independent route -- brute force from a definition, exact enumeration of the
expectation lemma (Sec. 3.1), high-precision algebra, published generator
values, limits and invariants.
"""
import itertools
import math
import os
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1910_04658_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _csr(rows, d):
    row_ptr = np.zeros(len(rows) + 1, np.uint64)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([c for r in rows for c in r], np.uint32)
    return row_ptr, col


def _unpack(sk, N):
    bits = np.unpackbits(sk.view(np.uint8), axis=1, bitorder="little")
    return bits[:, :N]


# --------------------------------------------------------------------------
# the random mapping (hash) -- build reading R1
# --------------------------------------------------------------------------

def test_splitmix64_published_values():
    vals = {}
    for line in open(os.path.join(GOLDEN, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = int(v, 0)
    mult, add = oracle.hash_params(vals["seed"])
    assert mult == vals["out1"] | 1
    assert add == vals["out2"]


@pytest.mark.parametrize("seed", [0, 1, 12345, 2**63 + 7])
@pytest.mark.parametrize("logN", [5, 10, 12, 13, 16])
def test_hash_is_top_bits_multiply_shift_for_power_of_two_N(seed, logN):
    # classic multiply-shift: the top log2(N) bits of (a*i + b) mod 2^64
    N = 1 << logN
    mult, add = oracle.hash_params(seed)
    pi = oracle.mapping_table(seed, N, 5000)
    rng = np.random.default_rng(seed % 2**32)
    idx = np.concatenate([np.arange(5000), rng.integers(0, 5000, 64)])
    for i in idx[:300].tolist() + idx[-64:].tolist():
        top = ((mult * i + add) % 2**64) >> (64 - logN)
        assert pi[i] == top


def test_hash_bucket_is_floor_of_scaled_fraction_for_any_N():
    # for any N the bucket is floor(N * h32 / 2^32), i.e. in [0, N)
    mult, add = oracle.hash_params(7)
    for N in [3, 100, 1000, 4097, 65535]:
        pi = oracle.mapping_table(7, N, 2000)
        for i in range(0, 2000, 37):
            h32 = ((mult * i + add) % 2**64) >> 32
            assert pi[i] == (h32 * N) // 2**32 < N


@pytest.mark.parametrize("consecutive", [True, False])
def test_hash_uniformity_chi_square(consecutive):
    N, m = 1024, 1_000_000
    if consecutive:
        keys = np.arange(m, dtype=np.uint32)
        pi = oracle.mapping_table(3, N, m)[keys]
    else:
        d = 50_000_000
        keys = np.random.default_rng(1).integers(0, d, m).astype(np.uint32)
        mult, add = oracle.hash_params(3)
        pi = np.array([oracle.lib().bso_bucket(mult, add, N, int(k)) for k in keys[:200_000]])
        m = pi.size
    hist = np.bincount(pi, minlength=N)
    e = m / N
    chi2 = float(((hist - e) ** 2 / e).sum())
    dof = N - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)


# --------------------------------------------------------------------------
# sketching (Definition "BinSketch", Sec. 3)
# --------------------------------------------------------------------------

def test_sketch_equals_definition_brute_force():
    rng = np.random.default_rng(0)
    for trial in range(40):
        d = int(rng.integers(1, 65))
        N = int(rng.integers(1, 70))
        pi = rng.integers(0, N, d).astype(np.uint32)
        dense = rng.random((5, d)) < rng.random()
        rows = [np.flatnonzero(v).tolist() for v in dense]
        rp, col = _csr(rows, d)
        sk, pc = oracle.sketch(rp, col, d, N, pi=pi)
        got = _unpack(sk, N)
        for r in range(5):
            # a_s[j] = OR over i with pi(i) = j of a[i]
            want = [int(any(dense[r, i] for i in range(d) if pi[i] == j)) for j in range(N)]
            assert got[r].tolist() == want
            assert pc[r] == sum(want)
        # padding bits above N stay zero
        allbits = np.unpackbits(sk.view(np.uint8), axis=1, bitorder="little")
        assert not allbits[:, N:].any()


def test_hash_sketch_equals_table_sketch():
    c = inputs.random_csr(2, 50, 3000, 1, 300)
    for N in [64, 1024, 4096]:
        a, pa = oracle.sketch(c.row_ptr, c.col, c.d, N, seed=9)
        b, pb = oracle.sketch(c.row_ptr, c.col, c.d, N, pi=oracle.mapping_table(9, N, c.d))
        assert np.array_equal(a, b) and np.array_equal(pa, pb)


def test_sketch_invariants():
    c = inputs.random_csr(3, 200, 20000, 1, 600)
    N = 512
    sk, pc = oracle.sketch(c.row_ptr, c.col, c.d, N, seed=5)
    lens = np.diff(c.row_ptr.astype(np.int64))
    assert np.all(pc <= np.minimum(lens, N))                  # |a_s| <= min(|a|, N)
    assert np.all(pc[lens == 1] == 1)                          # |a| = 1 -> |a_s| = 1
    assert np.array_equal(pc, np.unpackbits(sk.view(np.uint8), axis=1).sum(1))
    cnt = oracle.counts(sk, sk)
    bits = _unpack(sk, N).astype(np.int64)
    for i in range(0, 200, 17):
        for j in range(0, 200, 13):
            a, b, cc = int(pc[i]), int(pc[j]), int(cnt[i, j])
            assert cc <= min(a, b)
            assert a + b - cc == int((bits[i] | bits[j]).sum())   # union count
            # sketch(a OR b) = sketch(a) OR sketch(b)
            u = np.union1d(c.row(i), c.row(j)).astype(np.uint32)
            rp, col = _csr([u.tolist()], c.d)
            su, _ = oracle.sketch(rp, col, c.d, N, seed=5)
            assert np.array_equal(su[0], sk[i] | sk[j])


def test_bcs_parity_sketch_is_linear():
    # Definition "BCS" (Sec. 2): parity of the bits in each bucket, so the
    # sketch of the symmetric difference is the XOR of the sketches
    c = inputs.random_csr(4, 60, 5000, 1, 200)
    N = 256
    sk, _ = oracle.sketch(c.row_ptr, c.col, c.d, N, seed=1, parity=True)
    for i, j in [(0, 1), (5, 9), (10, 40)]:
        x = np.setxor1d(c.row(i), c.row(j)).astype(np.uint32)
        rp, col = _csr([x.tolist()], c.d)
        sx, _ = oracle.sketch(rp, col, c.d, N, seed=1, parity=True)
        assert np.array_equal(sx[0], sk[i] ^ sk[j])


def test_out_of_range_column_is_rejected():
    # columns are 0 .. d-1: d itself is the first index out of range
    for bad in (50, 99):
        rp, col = _csr([[1, 2], [3, bad]], 50)
        for parity in (False, True):
            with pytest.raises(ValueError):
                oracle.sketch(rp, col, 50, 64, seed=0, parity=parity)
    rp, col = _csr([[1, 2], [3, 49]], 50)
    sk, pc = oracle.sketch(rp, col, 50, 64, seed=0)
    assert pc[1] >= 1


def test_counts_brute_force():
    A = inputs.random_sketches(1, 37, 320, 0.3)
    B = inputs.random_sketches(2, 29, 320, 0.6)
    c = oracle.counts(A, B)
    a = _unpack(A, 320).astype(np.int64)
    b = _unpack(B, 320).astype(np.int64)
    assert np.array_equal(c, a @ b.T)


# --------------------------------------------------------------------------
# the expectation lemma (Sec. 3.1), exactly, by enumerating every mapping
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N,d,a_set,b_set", [
    (2, 6, [0, 1, 2], [2, 3]),
    (3, 6, [0, 1, 2, 3], [1, 2, 4, 5]),
    (4, 5, [0, 1], [0, 1]),
    (4, 6, [0, 2, 4], [1, 3, 5]),
    (3, 5, [0, 1, 2, 3, 4], [4]),
    (4, 6, [], [1, 2]),
])
def test_expectation_lemma_exact_enumeration(N, d, a_set, b_set):
    rp, col = _csr([a_set, b_set], d)
    tot_a = tot_b = tot_c = 0
    count = 0
    for pi in itertools.product(range(N), repeat=d):
        sk, pc = oracle.sketch(rp, col, d, N, pi=np.array(pi, np.uint32))
        c = oracle.counts(sk[:1], sk[1:])[0, 0]
        tot_a += int(pc[0])
        tot_b += int(pc[1])
        tot_c += int(c)
        count += 1
    n = 1 - Fraction(1, N)
    A, B = len(a_set), len(b_set)
    ip = len(set(a_set) & set(b_set))
    assert Fraction(tot_a, count) == N * (1 - n ** A)
    assert Fraction(tot_b, count) == N * (1 - n ** B)
    # E<a_s,b_s>/N = 1 - n^|a| - n^|b| + n^(|a|+|b|-<a,b>)  (the lemma's proof)
    assert Fraction(tot_c, count) == N * (1 - n ** A - n ** B + n ** (A + B - ip))


def test_expectation_monte_carlo_realistic_sizes():
    rng = np.random.default_rng(11)
    d, N, T = 20000, 256, 1500
    common = rng.choice(d, 70, replace=False)
    rest = np.setdiff1d(np.arange(d), common)
    extra = rng.choice(rest, 30 + 50, replace=False)
    a_set = np.sort(np.concatenate([common, extra[:30]]))
    b_set = np.sort(np.concatenate([common, extra[30:]]))
    rp, col = _csr([a_set.tolist(), b_set.tolist()], d)
    sa, sc = [], []
    for _ in range(T):
        pi = rng.integers(0, N, d).astype(np.uint32)
        sk, pc = oracle.sketch(rp, col, d, N, pi=pi)
        sa.append(int(pc[0]))
        sc.append(int(oracle.counts(sk[:1], sk[1:])[0, 0]))
    n = 1 - 1 / N
    A, B, ip = 100, 120, 70
    ea = N * (1 - n ** A)
    ec = N * (1 - n ** A - n ** B + n ** (A + B - ip))
    sa, sc = np.array(sa, float), np.array(sc, float)
    assert abs(sa.mean() - ea) < 5 * sa.std() / math.sqrt(T)
    assert abs(sc.mean() - ec) < 5 * sc.std() / math.sqrt(T)


# --------------------------------------------------------------------------
# the estimators (Alg. 1-4)
# --------------------------------------------------------------------------

def _expected_counts(A, B, ip, N):
    n = 1 - 1 / N
    return N * (1 - n ** A), N * (1 - n ** B), N * (1 - n ** A - n ** B + n ** (A + B - ip))


@pytest.mark.parametrize("A,B,ip,N", [
    (100, 80, 40, 1024), (200, 200, 200, 4096), (5, 3, 0, 64), (300, 50, 49, 8192),
    (1000, 900, 850, 4096), (20, 20, 1, 256), (2000, 1500, 700, 2048), (1, 1, 1, 32),
])
def test_estimators_invert_the_expectation_lemma(A, B, ip, N):
    # feeding the expected counts back must return the exact set sizes and
    # similarities: IP (Alg. 1), Ham = |a|+|b|-2IP, JS = IP/|a u b|, Cos
    nas, nbs, nasbs = _expected_counts(A, B, ip, N)
    IP, Ham, JS, Cos, na, nb = oracle.estimate(nas, nbs, nasbs, N)
    assert na == pytest.approx(A, rel=1e-9, abs=1e-9)
    assert nb == pytest.approx(B, rel=1e-9, abs=1e-9)
    assert IP == pytest.approx(ip, rel=1e-8, abs=1e-7)
    assert Ham == pytest.approx(A + B - 2 * ip, rel=1e-8, abs=1e-7)
    assert JS == pytest.approx(ip / (A + B - ip), rel=1e-8, abs=1e-9)
    assert Cos == pytest.approx(ip / math.sqrt(A * B), rel=1e-8, abs=1e-9)


def _rearranged_decimal(a, b, c, N):
    """Alg. 1-4 through the exact rearrangement n^{n_a} = (N-a)/N, evaluated in
    50-digit decimal: IP = ln(A*B/(N*U))/ln n with A = N-a, B = N-b,
    U = N-(a+b-c), n_a = ln(A/N)/ln n, n_u = ln(U/N)/ln n.  Counts are clamped
    so that A, B, U >= 1 (saturation reading)."""
    getcontext().prec = 50
    A = max(N - a, 1)
    B = max(N - b, 1)
    U = max(N - (a + b - c), 1)
    D = Decimal
    L = (D(N - 1) / D(N)).ln()
    na = (D(A) / D(N)).ln() / L
    nb = (D(B) / D(N)).ln() / L
    ip = (D(A) * D(B) / (D(N) * D(U))).ln() / L
    nu = (D(U) / D(N)).ln() / L
    ham = na + nb - 2 * ip
    js = ip / nu if nu != 0 else D(0)
    cs = ip / (na * nb).sqrt() if na * nb > 0 else D(0)
    return [float(ip), float(ham), float(js), float(cs)]


def test_estimators_match_high_precision_rearrangement():
    rng = np.random.default_rng(5)
    cases = []
    for N in [32, 256, 1024, 4096, 8192]:
        for _ in range(60):
            a = int(rng.integers(0, N + 1))
            b = int(rng.integers(0, N + 1))
            lo = max(0, a + b - N)
            c = int(rng.integers(lo, min(a, b) + 1))
            cases.append((a, b, c, N))
        cases += [(N, N, N, N), (N - 1, N - 1, N - 2, N), (0, 0, 0, N), (0, 5, 0, N),
                  (N, 3, 3, N), (1, 1, 0, N), (7, 7, 7, N)]
    for a, b, c, N in cases:
        got = oracle.estimate(a, b, c, N)[:4]
        want = _rearranged_decimal(a, b, c, N)
        for g, w, floor in zip(got, want, [1e-3, 1e-3, 1e-9, 1e-9]):
            assert abs(g - w) <= 1e-9 * max(abs(w), floor), (a, b, c, N, got, want)


def test_estimator_special_cases():
    N = 1024
    for a in [1, 17, 300, 1000]:
        IP, Ham, JS, Cos, na, nb = oracle.estimate(a, a, a, N)   # identical sketches
        assert IP == pytest.approx(na, rel=1e-12)
        assert abs(Ham) < 1e-9 and JS == pytest.approx(1.0, abs=1e-12)
        assert Cos == pytest.approx(1.0, abs=1e-12)
    assert oracle.estimate(1, 1, 1, N)[4] == pytest.approx(1.0, abs=1e-13)  # one bit -> |a| = 1
    assert oracle.estimate(50, 60, 0, N)[0] < 0                             # no overlap -> IP < 0
    IP, Ham, JS, Cos, na, nb = oracle.estimate(0, 40, 0, N)                 # empty row
    assert IP == 0.0 and Cos == 0.0 and JS == 0.0 and na == 0.0
    assert Ham == pytest.approx(nb, rel=1e-12)
    assert oracle.estimate(0, 0, 0, N)[2] == 0.0                            # JS(empty, empty) = 0
    for a, b, c in [(N, N, N), (N, 10, 10), (N - 1, N - 1, N - 1)]:         # saturation stays finite
        assert all(math.isfinite(v) for v in oracle.estimate(a, b, c, N))


def test_paper_literal_hamming_is_the_union():
    # Alg. 2 as printed returns n_a + n_b - n_{a,b}: the union size, not the
    # Hamming distance; Alg. 3 built on it is not Jaccard (reading R2)
    A, B, ip, N = 100, 80, 40, 1 << 20
    nas, nbs, nasbs = _expected_counts(A, B, ip, N)
    lit = oracle.estimate(nas, nbs, nasbs, N, paper_literal_ham=True)
    assert lit[1] == pytest.approx(A + B - ip, rel=1e-6)
    assert lit[2] == pytest.approx(ip / (A + B), rel=1e-6)
    assert abs(lit[2] - ip / (A + B - ip)) > 0.05


def test_estimate_converges_as_N_grows():
    # collisions vanish as N grows, so the IP estimate tends to the exact IP
    rng = np.random.default_rng(8)
    d = 1_000_000
    common = rng.choice(d, 60, replace=False)
    rest = rng.choice(np.setdiff1d(np.arange(200000), common), 230, replace=False)
    a_set = np.sort(np.concatenate([common, rest[:140]]))
    b_set = np.sort(np.concatenate([common, rest[140:]]))
    rp, col = _csr([a_set.tolist(), b_set.tolist()], d)
    errs = []
    for logN in [8, 10, 12, 14, 16, 18, 20]:
        N = 1 << logN
        e = []
        for seed in range(12):
            sk, pc = oracle.sketch(rp, col, d, N, seed=seed)
            c = oracle.counts(sk[:1], sk[1:])[0, 0]
            e.append(abs(oracle.estimate(pc[0], pc[1], c, N)[0] - 60))
        errs.append(float(np.mean(e)))
    assert errs[-1] < 0.5
    assert errs[-1] < errs[0] / 5
    assert all(errs[i + 2] <= errs[i] + 0.5 for i in range(len(errs) - 2))


def test_lemma_concentration_bounds():
    # Lemma 1 (|n_{a_s} - E|a_s|| < sqrt(psi/2 ln 2/delta)) w.p. >= 1-delta;
    # Lemma 3 likewise for n_{a_s,b_s}; Lemma 4 for IP w.p. >= 1-3 delta, with
    # N chosen by Theorem 1
    rng = np.random.default_rng(21)
    psi, delta, d = 60, 0.1, 50000
    # Theorem 1's sketch length N = psi sqrt((psi / 2) ln(2 / delta)), worked by
    # hand for psi = 60, delta = 0.1: 60 sqrt(30 ln 20) = 60 sqrt(89.87197) =
    # 60 x 9.480083 = 568.805, so N = 569
    N = math.ceil(psi * math.sqrt(psi / 2 * math.log(2 / delta)))
    assert N == 569
    common = rng.choice(d, 30, replace=False)
    rest = np.setdiff1d(np.arange(d), common)
    ex = rng.choice(rest, 60, replace=False)
    a_set = np.sort(np.concatenate([common, ex[:30]]))
    b_set = np.sort(np.concatenate([common, ex[30:]]))
    rp, col = _csr([a_set.tolist(), b_set.tolist()], d)
    ea, eb, ec = _expected_counts(60, 60, 30, N)
    bound = math.sqrt(psi / 2 * math.log(2 / delta))
    T, ok1, ok3, ok4 = 400, 0, 0, 0
    for _ in range(T):
        pi = rng.integers(0, N, d).astype(np.uint32)
        sk, pc = oracle.sketch(rp, col, d, N, pi=pi)
        c = int(oracle.counts(sk[:1], sk[1:])[0, 0])
        ok1 += abs(pc[0] - ea) < bound
        ok3 += abs(c - ec) < bound
        ok4 += abs(oracle.estimate(pc[0], pc[1], c, N)[0] - 30) < 14 * bound
    assert ok1 / T >= 1 - delta and ok3 / T >= 1 - delta and ok4 / T >= 1 - 3 * delta


# --------------------------------------------------------------------------
# ranking (Experiment 2 as a top-k) and exact similarities
# --------------------------------------------------------------------------

@pytest.mark.parametrize("measure", [0, 1, 2, 3])
@pytest.mark.parametrize("k,exclude", [(5, True), (40, False), (70, True)])
def test_topk_matches_full_sort(measure, k, exclude):
    c = inputs.random_csr(6, 64, 4000, 3, 120)
    N = 256
    sk, _ = oracle.sketch(c.row_ptr, c.col, c.d, N, seed=2)
    Q, DB = sk[:20], sk
    est, cnt = oracle.estimate_pairs(Q, DB, N)
    score, idx, cc = oracle.topk(Q, DB, N, measure, k, exclude)
    for q in range(20):
        items = [(est[measure, q, j], j) for j in range(DB.shape[0]) if not (exclude and j == q)]
        sign = 1 if measure == 1 else -1
        items.sort(key=lambda t: (sign * t[0], t[1]))
        for t in range(k):
            if t < len(items):
                assert idx[q, t] == items[t][1] and score[q, t] == items[t][0]
                assert cc[q, t] == cnt[q, items[t][1]]
            else:
                assert idx[q, t] == 0xFFFFFFFF
                assert score[q, t] == (math.inf if measure == 1 else -math.inf)


def test_estimate_pairs_agree_with_single_pair_estimates():
    A = inputs.random_sketches(3, 9, 512, 0.2)
    B = inputs.random_sketches(4, 7, 512, 0.7)
    est, cnt = oracle.estimate_pairs(A, B, 512)
    pa = oracle.counts(A, A).diagonal()
    pb = oracle.counts(B, B).diagonal()
    for i in range(9):
        for j in range(7):
            e = oracle.estimate(pa[i], pb[j], cnt[i, j], 512)
            assert list(est[:, i, j]) == list(e[:4])


def test_exact_similarities_dense():
    c = inputs.random_csr(7, 40, 3000, 0, 150)
    dense = np.zeros((c.n, c.d), np.int64)
    for r in range(c.n):
        dense[r, c.row(r)] = 1
    pa = np.repeat(np.arange(c.n), c.n).astype(np.uint32)
    pb = np.tile(np.arange(c.n), c.n).astype(np.uint32)
    ex = oracle.exact_pairs(c.row_ptr, c.col, pa, pb)
    ip = dense @ dense.T
    sz = dense.sum(1)
    for t in range(0, pa.size, 7):
        i, j = pa[t], pb[t]
        assert ex[t, 0] == ip[i, j]
        assert ex[t, 1] == int(np.sum(dense[i] != dense[j]))
        uni = int(np.sum(dense[i] | dense[j]))
        assert ex[t, 2] == (ip[i, j] / uni if uni else 0.0)
        assert ex[t, 3] == pytest.approx(ip[i, j] / math.sqrt(sz[i] * sz[j]) if sz[i] * sz[j] else 0.0)
