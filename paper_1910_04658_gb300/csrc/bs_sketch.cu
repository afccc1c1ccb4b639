// Sketching: Definition "BinSketch" (Sec. 3) and BCS (Definition "BCS", Sec. 2).
//
// One warp per CSR row.  The row's N/32-word sketch lives in shared memory,
// the warp streams the row's column indices with coalesced 16-byte loads
// (after peeling to 16-byte alignment, two loads per lane in flight), hashes
// each index to its bucket and sets the bucket bit with a shared-memory
// atomicOr (atomicXor for BCS).  The finished row is written to HBM with
// 16-byte stores, the shared sketch is cleared on the way, and the popcount
// |a_s| is reduced across the warp.  The next row's offsets are loaded before
// the current row is scattered.  HBM traffic per row is the algorithmic
// minimum: the row's indices and offsets in, N/8 + 4 bytes out.
#include <map>
#include <mutex>
#include <utility>

#include "bs_internal.cuh"

namespace bs {

// Sticky first data error per device; read and cleared by bs_get_async_error.
__device__ unsigned int g_async_error;

unsigned int *error_word() {
    static std::mutex mu;
    static unsigned int *ptr[256] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return nullptr;
    std::lock_guard<std::mutex> g(mu);
    if (!ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_async_error) != cudaSuccess) return nullptr;
        ptr[dev] = (unsigned int *)p;
    }
    return ptr[dev];
}

int sm_count() {
    static std::mutex mu;
    static int cnt[256] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return 148;
    std::lock_guard<std::mutex> g(mu);
    if (!cnt[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cnt[dev] = v > 0 ? v : 148;
    }
    return cnt[dev];
}

cudaError_t ensure_smem(const void *func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> done;
    if (bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_pair(dev, func);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done[key] = bytes;
    return e;
}

EncodeTiledFn encode_tiled() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// SplitMix64 (Steele, Lea, Flood 2014).
static uint64_t splitmix64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void hash_params(uint64_t seed, uint64_t *mult, uint64_t *add) {
    uint64_t s = seed;
    *mult = splitmix64(&s) | 1ull;
    *add = splitmix64(&s);
}

// ---------------------------------------------------------------------------
// K1: sketch kernel
// ---------------------------------------------------------------------------

constexpr int kSketchWarps = 8;

// One warp per row, rows strided over the grid.  The row's N/32-word sketch
// lives in shared memory (kept zero between rows: the write-out clears it);
// the next row's offsets are loaded before the current row is scattered.
// Off: the type the offsets are held in -- 32 bits when nnz < 2^32 (fewer
// registers: the kernel runs at 32 a thread), else 64 bits.
template <bool PARITY, typename Off>
__global__ void __launch_bounds__(kSketchWarps * 32, 8)
    sketch_kernel(const uint64_t *__restrict__ row_ptr, const uint32_t *__restrict__ col,
                  uint32_t n_rows, Off nnz, uint32_t d, uint32_t N, uint64_t mult,
                  uint64_t add, uint32_t *__restrict__ sketch, uint32_t *__restrict__ popcnt,
                  unsigned int *err) {
    extern __shared__ __align__(16) uint32_t smem_words[];
    const uint32_t W = N >> 5;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint32_t *s = smem_words + (size_t)warp * W;
    const uint32_t nwarps = gridDim.x * kSketchWarps;
    const bool vec_out = (W & 3u) == 0 && ((reinterpret_cast<uintptr_t>(sketch) & 15u) == 0);
    const HashParts h = {(uint32_t)mult, (uint32_t)(mult >> 32), (uint32_t)add, (uint32_t)(add >> 32)};
    for (uint32_t w = lane; w < W; w += 32) s[w] = 0u;
    __syncwarp();

    uint32_t r = blockIdx.x * kSketchWarps + warp;
    // offsets past the index array (or not representable in Off) fail the check below
    auto off = [nnz](uint64_t x) -> Off { return x > (uint64_t)nnz ? nnz + 1 : (Off)x; };
    Off b = 0, e = 0;
    if (r < n_rows) {
        b = off(__ldg(row_ptr + r));
        e = off(__ldg(row_ptr + r + 1));
    }
    for (; r < n_rows; r += nwarps) {
        const uint32_t rn = r + nwarps;
        Off nb = 0, ne = 0;
        if (rn < n_rows) {   // next row's offsets, in flight while this row is done
            nb = off(__ldg(row_ptr + rn));
            ne = off(__ldg(row_ptr + rn + 1));
        }
        const bool ok = (b <= e) && (e <= nnz);
        bool bad = false;
        if (ok) {
            if (sizeof(Off) == 4) {
                scatter_row<PARITY>(s, col + b, (uint32_t)(e - b), d, h, N, lane, bad);
            } else {
                // rows are done in pieces of at most 2^30 indices (one piece in practice)
                for (uint64_t q = b; q < e; q += (1ull << 30)) {
                    const uint64_t rest = e - q;
                    const uint32_t len = rest > (1ull << 30) ? (1u << 30) : (uint32_t)rest;
                    scatter_row<PARITY>(s, col + q, len, d, h, N, lane, bad);
                }
            }
        }
        bad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
            if (!ok) raise_error(err, BS_ERR_ROWPTR);
            else if (bad) raise_error(err, BS_ERR_INDEX_RANGE);
        }
        const bool zero = !ok || bad;
        __syncwarp();

        // write out (zeros for a bad row), clear the shared sketch, count bits
        uint32_t cnt = 0;
        uint32_t *out = sketch + (size_t)r * W;
        if (vec_out) {
            uint4 *sv = reinterpret_cast<uint4 *>(s);
            uint4 *ov = reinterpret_cast<uint4 *>(out);
            for (uint32_t t = lane; t < (W >> 2); t += 32) {
                uint4 x = sv[t];
                sv[t] = make_uint4(0, 0, 0, 0);
                if (zero) x = make_uint4(0, 0, 0, 0);
                cnt += __popc(x.x) + __popc(x.y) + __popc(x.z) + __popc(x.w);
                ov[t] = x;
            }
        } else {
            for (uint32_t t = lane; t < W; t += 32) {
                uint32_t x = s[t];
                s[t] = 0u;
                if (zero) x = 0u;
                cnt += __popc(x);
                out[t] = x;
            }
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (popcnt && lane == 0) popcnt[r] = cnt;
        __syncwarp();
        b = nb;
        e = ne;
    }
}

__global__ void popcount_rows_kernel(const uint32_t *__restrict__ sk, uint32_t n_rows, uint32_t W,
                                     uint32_t *__restrict__ pc) {
    const int lane = threadIdx.x & 31;
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n_rows; r += nwarps) {
        uint32_t cnt = 0;
        const uint32_t *row = sk + (size_t)r * W;
        for (uint32_t t = lane; t < W; t += 32) cnt += __popc(row[t]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) pc[r] = cnt;
    }
}

static bool valid_N(uint32_t N) { return N >= 32 && N <= BS_N_MAX && (N % 32) == 0; }

template <bool PARITY>
static bs_status launch_sketch(const uint64_t *row_ptr, const uint32_t *col, uint32_t n_rows,
                               uint64_t nnz, uint32_t d, uint32_t N, uint64_t seed,
                               uint32_t *sketch, uint32_t *popcnt, bs_stream_t stream) {
    if (!valid_N(N)) return BS_ERR_INVALID_ARG;
    if (n_rows == 0) return BS_OK;
    if (!row_ptr || !sketch || (nnz > 0 && !col)) return BS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(col) & 3u) != 0) return BS_ERR_INVALID_ARG;
    unsigned int *err = error_word();
    if (!err) return BS_ERR_CUDA;
    uint64_t mult, add;
    hash_params(seed, &mult, &add);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t smem = (size_t)kSketchWarps * (N / 32) * sizeof(uint32_t);
    const uint32_t want = (n_rows + kSketchWarps - 1) / kSketchWarps;
    const uint32_t cap = (uint32_t)sm_count() * 32u;
    const uint32_t grid = want < cap ? want : cap;
    if (nnz < 0xFFFFFFFFull) {
        auto kern = sketch_kernel<PARITY, uint32_t>;
        if (ensure_smem((const void *)kern, smem) != cudaSuccess) return BS_ERR_CUDA;
        kern<<<grid, kSketchWarps * 32, smem, st>>>(row_ptr, col, n_rows, (uint32_t)nnz, d, N, mult, add,
                                                    sketch, popcnt, err);
    } else {
        auto kern = sketch_kernel<PARITY, uint64_t>;
        if (ensure_smem((const void *)kern, smem) != cudaSuccess) return BS_ERR_CUDA;
        kern<<<grid, kSketchWarps * 32, smem, st>>>(row_ptr, col, n_rows, nnz, d, N, mult, add, sketch,
                                                    popcnt, err);
    }
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

}  // namespace bs

using namespace bs;

extern "C" {

bs_status bs_sketch(const uint64_t *row_ptr, const uint32_t *col, uint32_t n_rows, uint64_t nnz,
                    uint32_t d, uint32_t N, uint64_t seed, uint32_t *sketch, uint32_t *popcnt,
                    bs_stream_t stream) {
    BS_NVTX_RANGE();
    return launch_sketch<false>(row_ptr, col, n_rows, nnz, d, N, seed, sketch, popcnt, stream);
}

bs_status bs_sketch_parity(const uint64_t *row_ptr, const uint32_t *col, uint32_t n_rows,
                           uint64_t nnz, uint32_t d, uint32_t N, uint64_t seed, uint32_t *sketch,
                           uint32_t *popcnt, bs_stream_t stream) {
    BS_NVTX_RANGE();
    return launch_sketch<true>(row_ptr, col, n_rows, nnz, d, N, seed, sketch, popcnt, stream);
}

bs_status bs_popcount_rows(const uint32_t *sketch, uint32_t n_rows, uint32_t N, uint32_t *popcnt,
                           bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (!valid_N(N)) return BS_ERR_INVALID_ARG;
    if (n_rows == 0) return BS_OK;
    if (!sketch || !popcnt) return BS_ERR_INVALID_ARG;
    const uint32_t want = (n_rows + 7) / 8;
    const uint32_t cap = (uint32_t)sm_count() * 32u;
    popcount_rows_kernel<<<want < cap ? want : cap, 256, 0, (cudaStream_t)stream>>>(
        sketch, n_rows, N / 32, popcnt);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

bs_status bs_get_async_error(bs_stream_t stream) {
    unsigned int *err = error_word();
    if (!err) return BS_ERR_CUDA;
    unsigned int host = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BS_ERR_CUDA;
    if (cudaMemcpyAsync(&host, err, sizeof(host), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return BS_ERR_CUDA;
    if (cudaMemsetAsync(err, 0, sizeof(unsigned int), s) != cudaSuccess) return BS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BS_ERR_CUDA;
    return (bs_status)host;
}

void bs_hash_params(uint64_t seed, uint64_t *mult, uint64_t *add) {
    uint64_t m, a;
    hash_params(seed, &m, &a);
    if (mult) *mult = m;
    if (add) *add = a;
}

const char *bs_status_string(bs_status s) {
    switch (s) {
        case BS_OK: return "ok";
        case BS_ERR_INVALID_ARG: return "invalid argument";
        case BS_ERR_INDEX_RANGE: return "column index out of range";
        case BS_ERR_ROWPTR: return "malformed row offsets";
        case BS_ERR_CUDA: return "CUDA error";
        case BS_ERR_NO_MEMORY: return "workspace too small";
        case BS_ERR_TIMEOUT: return "device wait timed out";
        case BS_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

int bs_version(void) { return 100; }

}  // extern "C"
