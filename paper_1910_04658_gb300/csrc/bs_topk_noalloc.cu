// bs_topk_noalloc: the top-k ranking for callers that may not allocate GPU
// memory.
//
// Some callers cannot call cudaMalloc or hand the library a freshly allocated
// buffer: a serving process whose memory arena owns the whole device and
// forbids allocations outside it, a plugin that runs inside another
// framework's allocator, or a request path that must never pay for an
// allocation (which can synchronise the device).  bs_topk needs scratch
// memory when it splits the database across blocks; this entry point keeps
// that scratch in a fixed array in the library's own device memory instead.
//
// The array is BS_TOPK_NOALLOC_SCRATCH_BYTES large.  CUDA loads a library's
// device code lazily, one module per translation unit, so the array is
// reserved on a device when this file's module is first loaded there -- at
// the first bs_topk_noalloc call made while that device is current, which
// also looks up the array's address.  Make that first call before the
// caller's own arena takes the whole device and before any stream capture;
// it may synchronise.  The reservation then lasts until the process exits.
// All calls
// share the one array: two calls whose kernels overlap on the GPU (for
// example on two streams) race on it and must be serialised by the caller.
// Nothing in it needs to start at zero: every slot a call reads was written
// earlier by the same call.
#include <mutex>

#include "bs_internal.cuh"

namespace bs {

static __device__ __align__(256) unsigned char g_topk_scratch[BS_TOPK_NOALLOC_SCRATCH_BYTES];

// Device address of g_topk_scratch on the current device (nullptr on failure).
static void *topk_scratch_address() {
    static std::mutex mu;
    static void *addr[256] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return nullptr;
    std::lock_guard<std::mutex> g(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_topk_scratch) != cudaSuccess) {
            cudaGetLastError();   // leave no error behind for the next call's launch check
            return nullptr;
        }
        addr[dev] = p;
    }
    return addr[dev];
}

}  // namespace bs

extern "C" bs_status bs_topk_noalloc(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ,
                                     const uint32_t *DB, const uint32_t *pcDB, uint32_t nDB,
                                     uint32_t N, uint32_t by, uint32_t k, int exclude_self,
                                     float *score, uint32_t *idx, bs_stream_t stream) {
    BS_NVTX_RANGE();
    const size_t need = bs_topk_workspace_bytes(nQ, nDB, N, k);
    if (need > (size_t)BS_TOPK_NOALLOC_SCRATCH_BYTES) return BS_ERR_NO_MEMORY;
    void *scratch = nullptr;
    if (need > 0) {
        scratch = bs::topk_scratch_address();
        if (!scratch) return BS_ERR_CUDA;
    }
    return bs_topk(Q, pcQ, nQ, DB, pcDB, nDB, N, by, k, exclude_self, score, idx, scratch,
                   need > 0 ? (size_t)BS_TOPK_NOALLOC_SCRATCH_BYTES : 0, stream);
}
