// Batched sketching: many independent CSR datasets (each with its own d, N
// and seed) sketched by one persistent launch (Definition "BinSketch",
// Sec. 3, applied per dataset).  The job table lives in device memory; every
// block walks the global list of (job, row) warp tasks with a grid stride, so
// heterogeneous datasets share one grid and no per-dataset launch is needed.
#include "bs_internal.cuh"

namespace bs {

constexpr int kBatchWarps = 8;

// SplitMix64 (Steele, Lea, Flood 2014), device side, for per-job parameters.
__device__ __forceinline__ uint64_t splitmix64_dev(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void __launch_bounds__(kBatchWarps * 32)
    sketch_batched_kernel(const bs_sketch_job *__restrict__ jobs, uint32_t n_jobs, uint32_t max_N,
                          unsigned int *err) {
    extern __shared__ __align__(16) uint32_t smem_words[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint32_t *s = smem_words + (size_t)warp * (max_N >> 5);
    // total warp tasks = total rows (one warp per row)
    uint64_t total = 0;
    for (uint32_t j = 0; j < n_jobs; ++j) total += jobs[j].n_rows;
    const uint64_t nwarps = (uint64_t)gridDim.x * kBatchWarps;
    uint32_t job = 0;
    uint64_t job_base = 0;   // first global task of `job`
    for (uint64_t g = (uint64_t)blockIdx.x * kBatchWarps + warp; g < total; g += nwarps) {
        while (job < n_jobs && g >= job_base + jobs[job].n_rows) {   // tasks only move forward
            job_base += jobs[job].n_rows;
            ++job;
        }
        if (job >= n_jobs) break;
        const bs_sketch_job J = jobs[job];
        const uint32_t r = (uint32_t)(g - job_base);
        const uint32_t N = J.N;
        const bool job_ok = N >= 32 && N <= max_N && (N & 31u) == 0 && J.row_ptr && J.sketch &&
                            (J.nnz == 0 || J.col);
        if (!job_ok) {
            if (lane == 0) raise_error(err, BS_ERR_INVALID_ARG);
            continue;
        }
        const uint32_t W = N >> 5;
        uint64_t st = J.seed;
        const uint64_t mult = splitmix64_dev(st) | 1ull;
        const uint64_t add = splitmix64_dev(st);
        const HashParts h = {(uint32_t)mult, (uint32_t)(mult >> 32), (uint32_t)add,
                             (uint32_t)(add >> 32)};
        for (uint32_t w = lane; w < W; w += 32) s[w] = 0u;
        __syncwarp();
        const uint64_t b = J.row_ptr[r], e = J.row_ptr[r + 1];
        const bool ok = (b <= e) && (e <= J.nnz);
        bool bad = false;
        if (ok) {
            // pieces of at most 2^30 indices (one piece in practice)
            for (uint64_t q = b; q < e; q += (1ull << 30)) {
                const uint64_t rest = e - q;
                const uint32_t len = rest > (1ull << 30) ? (1u << 30) : (uint32_t)rest;
                scatter_row<false>(s, J.col + q, len, J.d, h, N, lane, bad);
            }
        }
        bad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
            if (!ok) raise_error(err, BS_ERR_ROWPTR);
            else if (bad) raise_error(err, BS_ERR_INDEX_RANGE);
        }
        const bool zero = !ok || bad;
        __syncwarp();
        uint32_t cnt = 0;
        uint32_t *out = J.sketch + (size_t)r * W;
        for (uint32_t t = lane; t < W; t += 32) {
            const uint32_t x = zero ? 0u : s[t];
            cnt += __popc(x);
            out[t] = x;
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (J.popcnt && lane == 0) J.popcnt[r] = cnt;
        __syncwarp();
    }
}

}  // namespace bs

using namespace bs;

extern "C" bs_status bs_sketch_batched(const bs_sketch_job *jobs, uint32_t n_jobs, uint32_t max_N,
                                       bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (n_jobs == 0) return BS_OK;
    if (!jobs || max_N < 32 || max_N > BS_N_MAX || (max_N % 32) != 0) return BS_ERR_INVALID_ARG;
    unsigned int *err = error_word();
    if (!err) return BS_ERR_CUDA;
    const size_t smem = (size_t)kBatchWarps * (max_N / 32) * sizeof(uint32_t);
    if (ensure_smem((const void *)sketch_batched_kernel, smem) != cudaSuccess) return BS_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sketch_batched_kernel,
                                                      kBatchWarps * 32, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const unsigned grid = (unsigned)(sm_count() * per_sm);
    sketch_batched_kernel<<<grid, kBatchWarps * 32, smem, (cudaStream_t)stream>>>(jobs, n_jobs, max_N,
                                                                                 err);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}
