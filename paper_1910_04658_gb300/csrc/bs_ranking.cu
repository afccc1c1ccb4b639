// Ranking-quality evaluation of Experiment 2 (Sec. 4, "Ranking"): ground
// truth from the uncompressed vectors, and the retrieval sets at a list of
// similarity thresholds.
//
//  * bs_exact_counts: exact |a AND b| for every (query row, database row)
//    pair.  One block per query row: the row becomes a bitmap of d bits in
//    shared memory, then the block's warps stream the database rows (warp per
//    row, 16-byte loads) and count the indices whose bit is set.
//  * bs_threshold_eval: for every query row and threshold, |O| (exact
//    similarity at or beyond the threshold), |O'| (estimate at or beyond it)
//    and |O n O'|, from the exact counts, the set sizes and the estimates.
#include <math.h>

#include "bs_internal.cuh"

namespace bs {
namespace rank {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxT = BS_EVAL_THRESHOLDS_MAX;   // thresholds per call

__global__ void __launch_bounds__(kThreads)
    exact_counts_kernel(const uint64_t *__restrict__ q_rp, const uint32_t *__restrict__ q_col, uint32_t nq,
                        uint64_t q_nnz, const uint64_t *__restrict__ db_rp,
                        const uint32_t *__restrict__ db_col, uint32_t ndb, uint64_t db_nnz, uint32_t d,
                        uint32_t *__restrict__ counts, uint32_t *__restrict__ q_sizes,
                        uint32_t *__restrict__ db_sizes, unsigned int *err) {
    extern __shared__ __align__(16) uint32_t bitmap[];
    __shared__ uint32_t s_size;
    const uint32_t words = (d + 31) >> 5;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t q = blockIdx.x; q < nq; q += gridDim.x) {
        for (uint32_t w = tid; w < words; w += kThreads) bitmap[w] = 0u;
        if (tid == 0) s_size = 0u;
        __syncthreads();
        const uint64_t qb = q_rp[q], qe = q_rp[q + 1];
        const bool qok = qb <= qe && qe <= q_nnz;
        bool bad = false;
        if (qok) {
            for (uint64_t k = qb + tid; k < qe; k += kThreads) {
                const uint32_t i = __ldg(q_col + k);
                if (i < d) {
                    const uint32_t m = 1u << (i & 31);
                    const uint32_t old = atomicOr(&bitmap[i >> 5], m);
                    if (!(old & m)) atomicAdd(&s_size, 1u);   // distinct indices only
                } else {
                    bad = true;
                }
            }
        }
        if (__syncthreads_or(bad) && tid == 0) raise_error(err, BS_ERR_INDEX_RANGE);
        if (!qok && tid == 0) raise_error(err, BS_ERR_ROWPTR);
        if (q_sizes && tid == 0) q_sizes[q] = s_size;
        // database rows, one warp each
        for (uint32_t j = warp; j < ndb; j += kWarps) {
            const uint64_t b = db_rp[j], e = db_rp[j + 1];
            const bool ok = b <= e && e <= db_nnz;
            uint32_t c = 0;
            bool rbad = false;
            if (ok) {
                const uint32_t *p = db_col + b;
                const uint64_t len64 = e - b;
                const uint32_t len = len64 > 0x7FFFFFFFull ? 0x7FFFFFFFu : (uint32_t)len64;
                const uint32_t mis = (uint32_t)((reinterpret_cast<uintptr_t>(p) >> 2) & 3u);
                uint32_t peel = (4u - mis) & 3u;
                peel = peel < len ? peel : len;
                auto test = [&](uint32_t i) {
                    if (i < d) c += (bitmap[i >> 5] >> (i & 31)) & 1u;
                    else rbad = true;
                };
                if ((uint32_t)lane < peel) test(__ldg(p + lane));
                const uint4 *v = reinterpret_cast<const uint4 *>(p + peel);
                const uint32_t nvec = (len - peel) >> 2;
                for (uint32_t t = lane; t < nvec; t += 32) {
                    const uint4 x = __ldg(v + t);
                    test(x.x);
                    test(x.y);
                    test(x.z);
                    test(x.w);
                }
                const uint32_t k = peel + (nvec << 2) + lane;
                if (k < len) test(__ldg(p + k));
                if (len64 > 0x7FFFFFFFull) rbad = true;
            }
            c = __reduce_add_sync(0xffffffffu, c);
            rbad = __any_sync(0xffffffffu, rbad);
            if (lane == 0) {
                if (!ok) raise_error(err, BS_ERR_ROWPTR);
                else if (rbad) raise_error(err, BS_ERR_INDEX_RANGE);
                counts[(size_t)q * ndb + j] = c;
                if (db_sizes && q == 0) db_sizes[j] = ok ? (uint32_t)(e - b) : 0u;
            }
        }
        __syncthreads();
    }
}

struct Thresholds {
    double v[kMaxT];
};

// exact similarity of measure m from the common count and the two set sizes
__device__ __forceinline__ double exact_sim(int m, double c, double a, double b) {
    if (m == M_IP) return c;
    if (m == M_HAM) return a + b - 2.0 * c;
    if (m == M_JS) {
        const double u = a + b - c;
        return u > 0.0 ? c / u : 0.0;
    }
    return (a * b > 0.0) ? c / sqrt(a * b) : 0.0;
}

__global__ void __launch_bounds__(256)
    threshold_eval_kernel(const float *__restrict__ est, const uint32_t *__restrict__ counts,
                          const uint32_t *__restrict__ q_sizes, const uint32_t *__restrict__ db_sizes,
                          uint32_t nq, uint32_t ndb, int m, const Thresholds thr, uint32_t T,
                          uint32_t *__restrict__ out) {
    __shared__ uint32_t acc[kMaxT * 3];
    for (uint32_t q = blockIdx.x; q < nq; q += gridDim.x) {
        for (uint32_t i = threadIdx.x; i < T * 3; i += blockDim.x) acc[i] = 0u;
        __syncthreads();
        uint32_t loc[kMaxT * 3];
#pragma unroll
        for (int i = 0; i < kMaxT * 3; ++i) loc[i] = 0u;
        const double a = (double)q_sizes[q];
        for (uint32_t j = threadIdx.x; j < ndb; j += blockDim.x) {
            const size_t o = (size_t)q * ndb + j;
            const double ex = exact_sim(m, (double)counts[o], a, (double)db_sizes[j]);
            const double es = (double)est[o];
#pragma unroll
            for (int t = 0; t < kMaxT; ++t) {
                if ((uint32_t)t < T) {
                    // Ham: a pair is retrieved when the distance is at most
                    // the threshold; the other measures: at least
                    const bool in_o = m == M_HAM ? ex <= thr.v[t] : ex >= thr.v[t];
                    const bool in_r = m == M_HAM ? es <= thr.v[t] : es >= thr.v[t];
                    loc[3 * t] += in_o;
                    loc[3 * t + 1] += in_r;
                    loc[3 * t + 2] += in_o && in_r;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kMaxT * 3; ++i) {
            if ((uint32_t)i < T * 3) {
                const uint32_t v = __reduce_add_sync(0xffffffffu, loc[i]);
                if ((threadIdx.x & 31) == 0 && v) atomicAdd(&acc[i], v);
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < T * 3; i += blockDim.x) out[(size_t)q * T * 3 + i] = acc[i];
        __syncthreads();
    }
}

}  // namespace rank
}  // namespace bs

using namespace bs;

extern "C" {

bs_status bs_exact_counts(const uint64_t *q_row_ptr, const uint32_t *q_col, uint32_t nq, uint64_t q_nnz,
                          const uint64_t *db_row_ptr, const uint32_t *db_col, uint32_t ndb,
                          uint64_t db_nnz, uint32_t d, uint32_t *counts, uint32_t *q_sizes,
                          uint32_t *db_sizes, bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (d == 0 || d > BS_EXACT_D_MAX) return BS_ERR_INVALID_ARG;
    if (nq == 0 || ndb == 0) return BS_OK;
    if (!q_row_ptr || !db_row_ptr || !counts || (q_nnz > 0 && !q_col) || (db_nnz > 0 && !db_col))
        return BS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(q_col) & 3u) || (reinterpret_cast<uintptr_t>(db_col) & 3u))
        return BS_ERR_INVALID_ARG;
    unsigned int *err = error_word();
    if (!err) return BS_ERR_CUDA;
    const size_t smem = (size_t)((d + 31) / 32) * 4;
    if (ensure_smem((const void *)rank::exact_counts_kernel, smem) != cudaSuccess) return BS_ERR_CUDA;
    const uint32_t cap = (uint32_t)sm_count() * 4u;
    const uint32_t grid = nq < cap ? nq : cap;
    rank::exact_counts_kernel<<<grid, rank::kThreads, smem, (cudaStream_t)stream>>>(
        q_row_ptr, q_col, nq, q_nnz, db_row_ptr, db_col, ndb, db_nnz, d, counts, q_sizes, db_sizes, err);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

bs_status bs_threshold_eval(const float *est, const uint32_t *counts, const uint32_t *q_sizes,
                            const uint32_t *db_sizes, uint32_t nq, uint32_t ndb, uint32_t by,
                            const double *thresholds, uint32_t n_thresholds, uint32_t *out,
                            bs_stream_t stream) {
    BS_NVTX_RANGE();
    int m = -1;
    switch (by) {
        case BS_IP: m = M_IP; break;
        case BS_HAM: m = M_HAM; break;
        case BS_JS: m = M_JS; break;
        case BS_COS: m = M_COS; break;
        default: return BS_ERR_INVALID_ARG;
    }
    if (n_thresholds == 0 || n_thresholds > rank::kMaxT || !thresholds) return BS_ERR_INVALID_ARG;
    if (nq == 0) return BS_OK;
    if (!est || !counts || !q_sizes || !db_sizes || !out) return BS_ERR_INVALID_ARG;
    rank::Thresholds thr = {};
    for (uint32_t t = 0; t < n_thresholds; ++t) thr.v[t] = thresholds[t];
    const uint32_t cap = (uint32_t)sm_count() * 8u;
    const uint32_t grid = nq < cap ? nq : cap;
    rank::threshold_eval_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(est, counts, q_sizes, db_sizes, nq,
                                                                        ndb, m, thr, n_thresholds, out);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

}  // extern "C"
