/*
 * BinSketch CPU oracle -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * Plain, slow, obviously-correct FP64 restatement of BinSketch
 * (Pratap, Bera, Revanuru, "Efficient Sketching Algorithm for Sparse Binary
 * Data", arXiv 1910.04658).  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Every function cites the passage of the paper it follows.  Where the paper
 * is silent or misprinted the reading taken is stated at the function:
 *   R1  the random mapping pi is realised by a seeded multiply-shift hash
 *       (Definition "BinSketch", Sec. 3 only asks for a random mapping);
 *   R2  Alg. 2 prints ham = n_a + n_b - n_{a,b}; that is the union size.  The
 *       Hamming identity Ham = |a| + |b| - 2 IP is used instead (Sec. 3.2);
 *       the printed form is kept behind a flag for documentation only;
 *   R3  saturation: the inversion ln(1 - n_{a_s}/N) needs n_{a_s} < N and the
 *       log argument of Alg. 1 needs the union count < N.  Counts are clamped
 *       so that N - n_{a_s}, N - n_{b_s} and N - union are all >= 1;
 *   R4  zero denominators: Cos = 0 when n_a * n_b = 0, JS = 0 when the
 *       estimated union is 0;
 *   R5  estimates are returned raw (never clamped to [0,1] or [0, min]);
 *   R6  0-based column indices, LSB-first packing of sketch bit j into
 *       word j >> 5, bit j & 31; a row holds ceil(N/32) words, the bits at
 *       and above N stay 0 (the oracle accepts any N >= 1 so that tiny N can
 *       be enumerated).
 *
 * Parity of the hash (R1) is pinned only by its own properties (top-bits
 * equality for power-of-two N, uniformity); everything else is pinned against
 * the expectation lemma (exact enumeration), the inversion identity and brute
 * force in the test-suite.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Random mapping pi : [d] -> [N]  (Definition "BinSketch", Sec. 3; R1)       */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): a Weyl sequence with step
 * 0x9E3779B97F4A7C15 followed by the "variant 13" 64-bit finaliser. */
static uint64_t splitmix64_next(uint64_t *state)
{
    uint64_t z;
    *state = *state + 0x9E3779B97F4A7C15ULL;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* The multiplier (forced odd) and the increment of the multiply-add-shift
 * hash are the first two SplitMix64 outputs for the given seed. */
void bso_hash_params(uint64_t seed, uint64_t *mult, uint64_t *add)
{
    uint64_t s = seed;
    *mult = splitmix64_next(&s) | 1ULL;
    *add = splitmix64_next(&s);
}

/* Dietzfelbinger multiply-add-shift to a 32-bit value, then the range [0, N)
 * by the high half of a 32x32-bit product: bucket = floor(h32 * N / 2^32). */
uint32_t bso_bucket(uint64_t mult, uint64_t add, uint32_t N, uint32_t i)
{
    uint64_t h = mult * (uint64_t)i + add; /* arithmetic mod 2^64 */
    uint32_t h32 = (uint32_t)(h >> 32);
    return (uint32_t)(((uint64_t)h32 * (uint64_t)N) >> 32);
}

/* pi as an explicit table, pi[i] for i in [0, d). */
void bso_mapping_table(uint64_t seed, uint32_t N, uint32_t d, uint32_t *pi)
{
    uint64_t mult, add;
    uint32_t i;
    bso_hash_params(seed, &mult, &add);
    for (i = 0; i < d; i++)
        pi[i] = bso_bucket(mult, add, N, i);
}

/* ------------------------------------------------------------------------ */
/* Sketching (Definition "BinSketch", Sec. 3):                               */
/*   a_s[j] = OR over i with pi(i) = j of a[i]                               */
/* A CSR row lists the i with a[i] = 1; only those can set a bit, so the OR  */
/* is "set bit pi(i) for every listed i" (the O(psi) cost noted in Sec. 3).  */
/* ------------------------------------------------------------------------ */

/* One row into an unpacked 0/1 byte vector a_s[0..N). */
static void sketch_row_bits(const uint32_t *idx, uint64_t len, const uint32_t *pi,
                            uint32_t N, unsigned char *a_s)
{
    uint64_t k;
    memset(a_s, 0, N);
    for (k = 0; k < len; k++)
        a_s[pi[idx[k]]] = 1; /* a_s[pi(i)] = a_s[pi(i)] OR 1 */
}

/* Pack the 0/1 vector LSB-first (R6) and count |a_s| (Alg. 1 step 1). */
static void pack_row(const unsigned char *a_s, uint32_t N, uint32_t *words, uint32_t *pc)
{
    uint32_t j, cnt = 0;
    memset(words, 0, (size_t)((N + 31) / 32) * sizeof(uint32_t));
    for (j = 0; j < N; j++) {
        if (a_s[j]) {
            words[j >> 5] |= 1u << (j & 31);
            cnt++;
        }
    }
    if (pc) *pc = cnt;
}

/* Sketch n CSR rows with an explicit mapping pi[0..d).  Returns -1 when a
 * column index is >= d (nothing written for that row), else 0. */
int bso_sketch_map(const uint64_t *row_ptr, const uint32_t *col, uint32_t n_rows,
                   uint32_t d, uint32_t N, const uint32_t *pi,
                   uint32_t *sketch, uint32_t *popcnt)
{
    uint32_t r;
    int bad = 0;
    unsigned char *a_s = (unsigned char *)malloc(N ? N : 1);
    if (!a_s) return -2;
    for (r = 0; r < n_rows; r++) {
        uint64_t k, b = row_ptr[r], e = row_ptr[r + 1];
        int row_ok = 1;
        for (k = b; k < e; k++)
            if (col[k] >= d) row_ok = 0;
        if (!row_ok) { bad = 1; continue; }
        sketch_row_bits(col + b, e - b, pi, N, a_s);
        pack_row(a_s, N, sketch + (size_t)r * ((N + 31) / 32), popcnt ? popcnt + r : NULL);
    }
    free(a_s);
    return bad ? -1 : 0;
}

/* Sketch with the seeded hash mapping (R1). */
int bso_sketch(const uint64_t *row_ptr, const uint32_t *col, uint32_t n_rows,
               uint32_t d, uint32_t N, uint64_t seed, uint32_t *sketch, uint32_t *popcnt)
{
    int rc;
    uint32_t *pi = (uint32_t *)malloc((size_t)(d ? d : 1) * sizeof(uint32_t));
    if (!pi) return -2;
    bso_mapping_table(seed, N, d, pi);
    rc = bso_sketch_map(row_ptr, col, n_rows, d, N, pi, sketch, popcnt);
    free(pi);
    return rc;
}

/* BCS (Definition "BCS", Sec. 2): u_s[j] = sum over i with pi(i)=j of u[i]
 * mod 2.  Same mapping, parity instead of OR. */
int bso_sketch_parity(const uint64_t *row_ptr, const uint32_t *col, uint32_t n_rows,
                      uint32_t d, uint32_t N, uint64_t seed, uint32_t *sketch,
                      uint32_t *popcnt)
{
    uint32_t r;
    int bad = 0;
    uint32_t *pi = (uint32_t *)malloc((size_t)(d ? d : 1) * sizeof(uint32_t));
    unsigned char *u_s = (unsigned char *)malloc(N ? N : 1);
    if (!pi || !u_s) { free(pi); free(u_s); return -2; }
    bso_mapping_table(seed, N, d, pi);
    for (r = 0; r < n_rows; r++) {
        uint64_t k, b = row_ptr[r], e = row_ptr[r + 1];
        int row_ok = 1;
        for (k = b; k < e; k++)
            if (col[k] >= d) row_ok = 0;
        if (!row_ok) { bad = 1; continue; }
        memset(u_s, 0, N);
        for (k = b; k < e; k++)
            u_s[pi[col[k]]] = (unsigned char)((u_s[pi[col[k]]] + 1) % 2);
        pack_row(u_s, N, sketch + (size_t)r * ((N + 31) / 32), popcnt ? popcnt + r : NULL);
    }
    free(pi);
    free(u_s);
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Sketch counts (Alg. 1 steps 1-2): n_{a_s} = |a_s|, n_{a_s,b_s} = <a_s,b_s> */
/* ------------------------------------------------------------------------ */

static uint32_t popcount32(uint32_t x)
{
    return (uint32_t)__builtin_popcount(x);
}

uint32_t bso_popcount_row(const uint32_t *w, uint32_t n_words)
{
    uint32_t k, s = 0;
    for (k = 0; k < n_words; k++) s += popcount32(w[k]);
    return s;
}

/* Number of common 1-bits of every (A row i, B row j): c[i*nB + j]. */
void bso_counts(const uint32_t *A, uint32_t nA, const uint32_t *B, uint32_t nB,
                uint32_t n_words, uint32_t *c)
{
    int64_t i;
#pragma omp parallel for schedule(dynamic, 4)
    for (i = 0; i < (int64_t)nA; i++) {
        uint32_t j, k;
        const uint32_t *a = A + (size_t)i * n_words;
        for (j = 0; j < nB; j++) {
            const uint32_t *b = B + (size_t)j * n_words;
            uint32_t s = 0;
            for (k = 0; k < n_words; k++) s += popcount32(a[k] & b[k]);
            c[(size_t)i * nB + j] = s;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Estimation (Alg. 1-4, Sec. 3.1-3.4) in FP64.                               */
/* ------------------------------------------------------------------------ */

enum { BSO_IP = 0, BSO_HAM = 1, BSO_JS = 2, BSO_COS = 3 };

/* Saturation clamp (R3) in the paper's notation: n_{a_s}, n_{b_s} and the
 * union n_{a_s}+n_{b_s}-n_{a_s,b_s} are capped at N-1; the common count is
 * then re-derived from the capped union so that the Alg. 1 log argument
 * n^{n_a} + n^{n_b} + n_{a_s,b_s}/N - 1 equals (N - union)/N >= 1/N. */
static void clamp_counts(double N, double *nas, double *nbs, double *nasbs)
{
    double uni = *nas + *nbs - *nasbs;
    if (*nas > N - 1) *nas = N - 1;
    if (*nbs > N - 1) *nbs = N - 1;
    if (uni > N - 1) uni = N - 1;
    *nasbs = *nas + *nbs - uni;
}

/* Alg. 1 (IP), Alg. 2 (Ham, read as R2), Alg. 3 (JS), Alg. 4 (Cos) for one
 * pair, from the counts n_{a_s}, n_{b_s}, n_{a_s,b_s} (taken as reals so that
 * expectations can be fed in as well).  out[0..3] = IP, Ham, JS, Cos.
 * out_na/out_nb (may be NULL) receive the set-size estimates n_a, n_b.
 * paper_literal_ham != 0 returns Alg. 2 exactly as printed (union size) and
 * JS accordingly -- documentation only, never a parity target. */
void bso_estimate(double nas, double nbs, double nasbs, uint32_t N_,
                  int paper_literal_ham, double *out, double *out_na, double *out_nb)
{
    const double N = (double)N_;
    const double n = 1.0 - 1.0 / N;   /* n = 1 - 1/N   (Sec. 3.1) */
    const double ln_n = log(n);
    double n_a, n_b, n_ab, ham, js, cs, arg;

    clamp_counts(N, &nas, &nbs, &nasbs);

    /* Alg. 1 step 3: n_a = ln(1 - n_{a_s}/N) / ln n, likewise n_b. */
    n_a = log(1.0 - nas / N) / ln_n;
    n_b = log(1.0 - nbs / N) / ln_n;

    /* Alg. 1 step 4: n_{a,b} = n_a + n_b - (1/ln n) ln(n^{n_a} + n^{n_b} + n_{a_s,b_s}/N - 1). */
    arg = pow(n, n_a) + pow(n, n_b) + nasbs / N - 1.0;
    n_ab = n_a + n_b - log(arg) / ln_n;

    /* Alg. 2: Hamming distance. */
    if (paper_literal_ham)
        ham = n_a + n_b - n_ab;          /* as printed: this is the union */
    else
        ham = n_a + n_b - 2.0 * n_ab;    /* Ham = |a| + |b| - 2 IP (R2) */

    /* Alg. 3: JS = n_{a,b} / (n_{a,b} + ham_{a,b}); 0 for an empty union (R4). */
    js = (n_ab + ham != 0.0) ? n_ab / (n_ab + ham) : 0.0;

    /* Alg. 4: Cos = n_{a,b} / sqrt(n_a n_b); 0 when n_a n_b = 0 (R4). */
    cs = (n_a * n_b > 0.0) ? n_ab / sqrt(n_a * n_b) : 0.0;

    out[BSO_IP] = n_ab;
    out[BSO_HAM] = ham;
    out[BSO_JS] = js;
    out[BSO_COS] = cs;
    if (out_na) *out_na = n_a;
    if (out_nb) *out_nb = n_b;
}

/* All four estimates for every (A row, B row) pair from packed sketches.
 * out is [4][nA][nB]; counts (may be NULL) receives n_{a_s,b_s}. */
void bso_estimate_pairs(const uint32_t *A, uint32_t nA, const uint32_t *B, uint32_t nB,
                        uint32_t N, double *out, uint32_t *counts)
{
    const uint32_t W = (N + 31) / 32;
    const size_t plane = (size_t)nA * nB;
    int64_t i;
#pragma omp parallel for schedule(dynamic, 4)
    for (i = 0; i < (int64_t)nA; i++) {
        uint32_t j, k;
        const uint32_t *a = A + (size_t)i * W;
        uint32_t na = bso_popcount_row(a, W);
        for (j = 0; j < nB; j++) {
            const uint32_t *b = B + (size_t)j * W;
            uint32_t nb = bso_popcount_row(b, W), c = 0;
            double e[4];
            size_t o = (size_t)i * nB + j;
            for (k = 0; k < W; k++) c += popcount32(a[k] & b[k]);
            bso_estimate((double)na, (double)nb, (double)c, N, 0, e, NULL, NULL);
            out[0 * plane + o] = e[0];
            out[1 * plane + o] = e[1];
            out[2 * plane + o] = e[2];
            out[3 * plane + o] = e[3];
            if (counts) counts[o] = c;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Ranking (Experiment 2, Sec. 4): the most similar DB rows of each query.    */
/* The paper thresholds; a top-k by (score desc, index asc) is used here,     */
/* Hamming ranked by ascending distance.  Self pairs are skipped on request.  */
/* ------------------------------------------------------------------------ */

typedef struct { double key; double val; uint32_t idx; } bso_item;

static int cmp_item(const void *x, const void *y)
{
    const bso_item *p = (const bso_item *)x, *q = (const bso_item *)y;
    if (p->key > q->key) return -1;
    if (p->key < q->key) return 1;
    if (p->idx < q->idx) return -1;
    if (p->idx > q->idx) return 1;
    return 0;
}

/* measure: 0 IP, 1 Ham, 2 JS, 3 Cos.  score/idx are [nQ][k]; missing
 * entries are (-inf, 0xFFFFFFFF) for IP/JS/Cos and (+inf, 0xFFFFFFFF) for
 * Ham.  cnt (may be NULL) gets n_{a_s,b_s} of each returned pair. */
void bso_topk(const uint32_t *Q, uint32_t nQ, const uint32_t *DB, uint32_t nDB,
              uint32_t N, int measure, uint32_t k, int exclude_self,
              double *score, uint32_t *idx, uint32_t *cnt)
{
    const uint32_t W = (N + 31) / 32;
    int64_t q;
#pragma omp parallel for schedule(dynamic, 1)
    for (q = 0; q < (int64_t)nQ; q++) {
        bso_item *items = (bso_item *)malloc((size_t)(nDB ? nDB : 1) * sizeof(bso_item));
        uint32_t *cc = (uint32_t *)malloc((size_t)(nDB ? nDB : 1) * sizeof(uint32_t));
        const uint32_t *a = Q + (size_t)q * W;
        uint32_t na = bso_popcount_row(a, W), j, m = 0, t;
        for (j = 0; j < nDB; j++) {
            const uint32_t *b = DB + (size_t)j * W;
            uint32_t nb = bso_popcount_row(b, W), c = 0, k2;
            double e[4];
            if (exclude_self && j == (uint32_t)q) continue;
            for (k2 = 0; k2 < W; k2++) c += popcount32(a[k2] & b[k2]);
            bso_estimate((double)na, (double)nb, (double)c, N, 0, e, NULL, NULL);
            items[m].val = e[measure];
            items[m].key = (measure == BSO_HAM) ? -e[measure] : e[measure];
            items[m].idx = j;
            cc[j] = c;
            m++;
        }
        qsort(items, m, sizeof(bso_item), cmp_item);
        for (t = 0; t < k; t++) {
            size_t o = (size_t)q * k + t;
            if (t < m) {
                score[o] = items[t].val;
                idx[o] = items[t].idx;
                if (cnt) cnt[o] = cc[items[t].idx];
            } else {
                score[o] = (measure == BSO_HAM) ? INFINITY : -INFINITY;
                idx[o] = 0xFFFFFFFFu;
                if (cnt) cnt[o] = 0;
            }
        }
        free(items);
        free(cc);
    }
}

/* ------------------------------------------------------------------------ */
/* Exact similarities from sorted index lists (Sec. 1, the exact baseline;    */
/* definitions in Sec. 2 and 3.2-3.4).  Used only as MSE ground truth.        */
/* ------------------------------------------------------------------------ */

/* |a cap b| of two strictly increasing index lists by a merge walk. */
static uint64_t intersect_sorted(const uint32_t *x, uint64_t nx, const uint32_t *y, uint64_t ny)
{
    uint64_t i = 0, j = 0, s = 0;
    while (i < nx && j < ny) {
        if (x[i] == y[j]) { s++; i++; j++; }
        else if (x[i] < y[j]) i++;
        else j++;
    }
    return s;
}

/* For each listed pair (pa[t], pb[t]) of CSR rows (columns sorted, unique):
 * out[t*4 + 0..3] = IP, Ham, JS, Cos exactly.  JS(empty, empty) = 0 and
 * Cos = 0 for an empty row (R4). */
void bso_exact_pairs(const uint64_t *row_ptr, const uint32_t *col,
                     const uint32_t *pa, const uint32_t *pb, uint64_t n_pairs, double *out)
{
    int64_t t;
#pragma omp parallel for schedule(static)
    for (t = 0; t < (int64_t)n_pairs; t++) {
        uint64_t a0 = row_ptr[pa[t]], a1 = row_ptr[pa[t] + 1];
        uint64_t b0 = row_ptr[pb[t]], b1 = row_ptr[pb[t] + 1];
        double sa = (double)(a1 - a0), sb = (double)(b1 - b0);
        double ip = (double)intersect_sorted(col + a0, a1 - a0, col + b0, b1 - b0);
        double uni = sa + sb - ip;
        out[t * 4 + 0] = ip;
        out[t * 4 + 1] = sa + sb - 2.0 * ip;
        out[t * 4 + 2] = uni > 0 ? ip / uni : 0.0;
        out[t * 4 + 3] = (sa * sb > 0) ? ip / sqrt(sa * sb) : 0.0;
    }
}

int bso_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
