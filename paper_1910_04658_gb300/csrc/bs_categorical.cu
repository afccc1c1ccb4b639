// Categorical data front end (Sec. 1, "Extension for categorical data
// compression"): label-encoded categorical rows become binary rows by one-hot
// encoding, so BinSketch (Definition "BinSketch") and the Hamming estimator
// (Alg. 2) apply.  Feature f with m_f values occupies columns
// offsets[f] .. offsets[f] + m_f - 1 of the binary row; a row of F features
// has exactly F set bits, at offsets[f] + label[f].  The CSR offsets are
// therefore row * F and the column indices of a row increase.
#include "bs_internal.cuh"

namespace bs {

__global__ void __launch_bounds__(256)
    onehot_kernel(const uint32_t *__restrict__ labels, uint32_t n, uint32_t F,
                  const uint32_t *__restrict__ offsets, uint64_t *__restrict__ row_ptr,
                  uint32_t *__restrict__ col, unsigned int *err) {
    const uint64_t total = (uint64_t)n * F;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const uint32_t f = (uint32_t)(t % F);
        const uint32_t lo = __ldg(offsets + f), hi = __ldg(offsets + f + 1);
        const uint32_t v = __ldg(labels + t);
        // an out-of-range label keeps the row well formed (first column of
        // its feature) and is reported
        const bool ok = v < hi - lo;
        bad |= !ok;
        col[t] = lo + (ok ? v : 0u);
    }
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= n; r += stride)
        row_ptr[r] = r * F;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_error(err, BS_ERR_INDEX_RANGE);
}

}  // namespace bs

using namespace bs;

extern "C" bs_status bs_onehot_csr(const uint32_t *labels, uint32_t n, uint32_t F, const uint32_t *offsets,
                                   uint64_t *row_ptr, uint32_t *col, bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (F == 0) return BS_ERR_INVALID_ARG;
    if (!row_ptr || !offsets) return BS_ERR_INVALID_ARG;
    if (n > 0 && (!labels || !col)) return BS_ERR_INVALID_ARG;
    unsigned int *err = error_word();
    if (!err) return BS_ERR_CUDA;
    const uint64_t total = (uint64_t)n * F + n + 1;
    const uint64_t want = (total + 255) / 256;
    const uint64_t cap = (uint64_t)sm_count() * 16u;
    const uint32_t grid = (uint32_t)(want < cap ? want : cap);
    onehot_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(labels, n, F, offsets, row_ptr, col, err);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}
