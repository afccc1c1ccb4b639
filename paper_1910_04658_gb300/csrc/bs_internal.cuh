// Internal helpers shared by the CUDA translation units of libbinsketch.
// Nothing here is part of the C ABI (see include/binsketch.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "binsketch.h"

namespace bs {

// NVTX range around one C-ABI call, named after the call, so profiler
// timelines attribute each kernel to the entry point that launched it (a
// no-op unless a profiling tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define BS_NVTX_RANGE() ::bs::NvtxRange bs_nvtx_range_(__func__)

// ---------------------------------------------------------------------------
// Host-side shared state
// ---------------------------------------------------------------------------

// Device address of the sticky data-error word of the current device
// (defined in bs_sketch.cu); nullptr if it could not be resolved.
unsigned int *error_word();

// Number of SMs of the current device (cached).
int sm_count();

// cuTensorMapEncodeTiled resolved through the runtime (no -lcuda needed).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled();

// SplitMix64-derived hash parameters (host).
void hash_params(uint64_t seed, uint64_t *mult, uint64_t *add);

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device; the attribute is set once per (device, kernel, size), so
// launches made later -- including inside a CUDA-graph capture -- do no
// device-attribute calls.
cudaError_t ensure_smem(const void *func, size_t bytes);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// pi(i) = floor(N * hi32(mult * i + add mod 2^64) / 2^32)
__device__ __forceinline__ uint32_t bucket_of(uint32_t i, uint64_t mult, uint64_t add, uint32_t N) {
    const uint64_t h = mult * (uint64_t)i + add;
    return __umulhi((uint32_t)(h >> 32), N);
}

// Hash parameters split into 32-bit halves: hi32(mult * i + add mod 2^64)
// = mh * i + ah + hi32(ml * i + al) (mod 2^32) -- one wide multiply-add and
// one multiply-add per index.
struct HashParts {
    uint32_t ml, mh, al, ah;
};

// Set (OR; XOR for BCS) the bucket bit of index i in the shared sketch s.
// Branch-free: an index >= d only marks the row bad (the row is written as
// zeros), its bucket is still in [0, N) so the shared access stays in bounds.
template <bool PARITY>
__device__ __forceinline__ void set_bucket(uint32_t *s, uint32_t i, uint32_t d, const HashParts &h,
                                           uint32_t N, bool &bad) {
    bad |= (i >= d);
    const uint64_t t = (uint64_t)h.ml * i + h.al;
    const uint32_t x = h.mh * i + h.ah + (uint32_t)(t >> 32);
    const uint32_t j = __umulhi(x, N);
    if (PARITY)
        atomicXor(&s[j >> 5], 1u << (j & 31));
    else
        atomicOr(&s[j >> 5], 1u << (j & 31));
}

// Scatter `len` indices starting at p (any 4-byte alignment): peel to a
// 16-byte boundary, then two 16-byte loads per lane in flight (with 32
// registers a thread, 64 warps stay resident per SM).
template <bool PARITY>
__device__ __forceinline__ void scatter_row(uint32_t *s, const uint32_t *__restrict__ p, uint32_t len,
                                            uint32_t d, const HashParts &h, uint32_t N, int lane,
                                            bool &bad) {
    const uint32_t mis = (uint32_t)((reinterpret_cast<uintptr_t>(p) >> 2) & 3u);
    uint32_t peel = (4u - mis) & 3u;
    peel = peel < len ? peel : len;
    if ((uint32_t)lane < peel) set_bucket<PARITY>(s, __ldg(p + lane), d, h, N, bad);
    const uint4 *v = reinterpret_cast<const uint4 *>(p + peel);
    const uint32_t nvec = (len - peel) >> 2;
    for (uint32_t t = lane; t < nvec; t += 64) {
        uint4 x[2];
#pragma unroll
        for (int u = 0; u < 2; ++u)
            if (t + 32 * u < nvec) x[u] = __ldg(v + t + 32 * u);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (t + 32 * u < nvec) {
                set_bucket<PARITY>(s, x[u].x, d, h, N, bad);
                set_bucket<PARITY>(s, x[u].y, d, h, N, bad);
                set_bucket<PARITY>(s, x[u].z, d, h, N, bad);
                set_bucket<PARITY>(s, x[u].w, d, h, N, bad);
            }
        }
    }
    const uint32_t k = peel + (nvec << 2) + lane;
    if (k < len) set_bucket<PARITY>(s, __ldg(p + k), d, h, N, bad);
}

__device__ __forceinline__ void raise_error(unsigned int *err, unsigned int code) {
    if (err) atomicCAS(err, 0u, code);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- mbarrier ---------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: returns false after `limit` SM cycles (default ~4e9, about
// 2 s at full clock; longer at lower clocks) without the phase completing.
// The cycle counter is read only after a burst of polls, so the common short
// wait costs nothing beyond the polls themselves.
constexpr long long kWaitLimitCycles = 4000000000ll;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          long long limit = kWaitLimitCycles) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
#pragma unroll 1
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > limit) return false;
    }
}

// ---- TMA --------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// contiguous global -> shared copy of `bytes` (a multiple of 16; both
// addresses 16-byte aligned), completion counted on the mbarrier
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// consumer-warps-only named barrier
__device__ __forceinline__ void named_sync(uint32_t id, uint32_t nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ---------------------------------------------------------------------------
// Estimation (Alg. 1-4) from integer counts, FP32.
//
// With n = 1 - 1/N, L = ln n, A = N - a, B = N - b and U = N - (a + b - c)
// (a = |a_s|, b = |b_s|, c = <a_s, b_s>), Alg. 1 gives n^{n_a} = A/N, so its
// log argument n^{n_a} + n^{n_b} + c/N - 1 equals U/N and
//    IP * L = ln(A B / (N U)),  n_a * L = ln(A / N),  n_u * L = ln(U / N)
//   Ham * L = ln(U^2 / (A B))            (Ham = n_a + n_b - 2 IP)
//        JS = ln(A B / (N U)) / ln(U / N) (IP / (IP + Ham) = IP / n_u)
//       Cos = -ln(A B / (N U)) / sqrt(ln(A/N) ln(B/N))
// Every logarithm is of a ratio p/q of exact positive integers, taken as
// +log1p((p - q)/q) for p >= q and -log1p((q - p)/p) for p < q: the argument
// of log1p is never negative, so its condition number stays below 1 and the
// FP32 result keeps ~1e-7 relative accuracy even where the estimate itself is
// close to 0 -- with one log1p and no branch.  The quotients use the fast
// division (__fdividef, within 2 ulp; both operands are far from its
// 2^126 limit), which keeps the error at a few 1e-7.
// Saturation: a, b and the union a + b - c are capped at N - 1, so A, B, U >= 1.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float ln_ratio(long long p, long long q) {
    const long long diff = p - q;
    const long long ad = diff < 0 ? -diff : diff;
    const long long den = diff < 0 ? p : q;
    const float r = log1pf(__fdividef((float)ad, (float)den));   // <= 2 ulp, den >= 1
    return diff < 0 ? -r : r;
}

struct Clamped {
    long long A, B, U;
};

__device__ __forceinline__ Clamped clamp_counts(uint32_t a, uint32_t b, uint32_t c, uint32_t N) {
    const uint32_t cap = N - 1;
    uint32_t u = a + b - c;
    a = a < cap ? a : cap;
    b = b < cap ? b : cap;
    u = u < cap ? u : cap;
    Clamped r;
    r.A = (long long)(N - a);
    r.B = (long long)(N - b);
    r.U = (long long)(N - u);
    return r;
}

// ln(A/N) for a row count a (per row, reused across pairs).
__device__ __forceinline__ float row_log(uint32_t a, uint32_t N) {
    const uint32_t cap = N - 1;
    a = a < cap ? a : cap;
    return ln_ratio((long long)(N - a), (long long)N);
}

// measure codes used inside the kernels
enum { M_IP = 0, M_HAM = 1, M_JS = 2, M_COS = 3 };

// One estimate; lnA = row_log(a), lnB = row_log(b); invL = 1/ln(1 - 1/N).
template <int M>
__device__ __forceinline__ float estimate_one(uint32_t a, uint32_t b, uint32_t c, uint32_t N,
                                              float lnA, float lnB, float invL) {
    const Clamped k = clamp_counts(a, b, c, N);
    if (M == M_IP) {
        return ln_ratio(k.A * k.B, (long long)N * k.U) * invL;
    } else if (M == M_HAM) {
        return ln_ratio(k.U * k.U, k.A * k.B) * invL;
    } else if (M == M_JS) {
        const float lu = ln_ratio(k.U, (long long)N);
        if (lu == 0.0f) return 0.0f;
        return __fdividef(ln_ratio(k.A * k.B, (long long)N * k.U), lu);
    } else {
        const float p = lnA * lnB;
        if (!(p > 0.0f)) return 0.0f;
        return -ln_ratio(k.A * k.B, (long long)N * k.U) * rsqrtf(p);
    }
}

// better(a, b): (key a, index a) ranks strictly before (key b, index b) --
// larger key first, then smaller index
__device__ __forceinline__ bool better(float ka, uint32_t ia, float kb, uint32_t ib) {
    return ka > kb || (ka == kb && ia < ib);
}

// ranking key of a measure: the estimate, negated for Ham (smaller is better)
template <int M>
__device__ __forceinline__ float rank_key(uint32_t a, uint32_t b, uint32_t c, uint32_t N, float lnA,
                                          float lnB, float invL) {
    const float v = estimate_one<M>(a, b, c, N, lnA, lnB, invL);
    return M == M_HAM ? -v : v;
}

// ---- host: top-k variants (bs_pairs.cu, bs_pairs_tc.cu) ----------------------
enum { VARIANT_AUTO = 0, VARIANT_POPC = 1, VARIANT_TC = 2 };

// POPC variant (bs_pairs.cu)
uint32_t popc_splits(uint32_t nQ, uint32_t nDB);
// exclude_self drops the pairs with query index q == self_off + database index
bs_status topk_popc(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ, const uint32_t *DB,
                    const uint32_t *pcDB, uint32_t nDB, uint32_t N, int measure, uint32_t k,
                    int exclude_self, uint32_t self_off, float *score, uint32_t *idx, float *ws_key,
                    uint32_t *ws_idx, uint32_t splits, unsigned int *err, cudaStream_t stream);
// merge per-split lists ws_key/ws_idx [splits][nQ][k] into score/idx
bs_status launch_merge(int measure, const float *ws_key, const uint32_t *ws_idx, uint32_t nQ,
                       uint32_t k, uint32_t splits, float *score, uint32_t *idx, cudaStream_t stream);

// tensor-core variant (bs_pairs_tc.cu): query blocks of 128 rows (the MMA's
// M, one TMEM lane per row), database tiles of 208 rows (the MMA's N)
constexpr uint32_t kTcQueryRows = 128, kTcTileRows = 208;
bool tc_supported(const uint32_t *Q, const uint32_t *DB, uint32_t N, uint32_t k);
// partial lists per row of the balanced schedule with tb-row database tiles,
// or (aligned) of the equal parts the rows after a call's rounds are cut into
uint32_t tc_splits(uint32_t nQ, uint32_t nDB, uint32_t tb = 208, bool aligned = false);
// database rows per tile (the MMA's N) of a block configuration
uint32_t tc_cfg_tile_rows(int cfg);
// bytes of a k-chunk-tiled copy of an n-row sketch matrix in R-row blocks
// (R = 128 for queries, 208 for a database)
size_t tc_tiled_bytes(uint32_t n, uint32_t N, uint32_t R);
// bytes of the FP4 copy of an n-row database (N / 2 bytes a row) that the
// TMA configurations read
size_t tc_fp4_bytes(uint32_t n, uint32_t N);
// tensor-core block configurations: BS_VARIANT_TC_CFG(c), 0 <= c < kTcConfigCount;
// c >= kTcFirstTmaCfg read the database operand from the FP4 copy by TMA
// (those with no widening warps the query operand too, from an FP4 copy of Q)
constexpr int kTcConfigCount = 15, kTcFirstTmaCfg = 10;
// wait budget of the tensor-core kernel's bounded waits (cycles), and the
// shortened budget of a fault-injected call
constexpr long long kTcWaitLimit = kWaitLimitCycles;
constexpr long long kTcInjectWaitLimit = 2000000ll;
// The launches of one tensor-core top-k call (host only): the block
// configuration, which operands go through FP4 copies, the first launch's
// rounds of whole row blocks (rows [0, q_split)), the partial lists per row of
// the launch over the remaining rows, the kernels launched and the partial-
// list bytes the call needs.
// an FP4 database copy up to this size stays in L2 (129 MB) while a launch
// sweeps it, whatever order the blocks read it in
constexpr size_t kTcL2Resident = (size_t)64 << 20;
struct TcCallPlan {
    int cfg = -1;
    bool fp4_q = false, fp4_db = false;
    bool aligned = false;   // the rows after the rounds run in aligned equal parts
    uint32_t rounds = 0, q_split = 0, splits = 1, launches = 0, tile_rows = 208;
    size_t lists_bytes = 0;
};
// kept: how the caller keeps the database -- not at all (the call makes the
// operand copy it needs), tiled (bs_tile_sketches) or as the FP4 copy
// (bs_fp4_sketches)
enum { KEPT_NONE = 0, KEPT_TILED = 1, KEPT_FP4 = 2 };
bs_status tc_call_plan(uint32_t nQ, uint32_t nDB, uint32_t N, uint32_t k, int cfg, bool same, int kept,
                       TcCallPlan &pl);
// partial-list bytes that cover the plan of every configuration
size_t tc_lists_bytes(uint32_t nQ, uint32_t nDB, uint32_t k);
// lists: lists_bytes of scratch for the partial lists (tc_lists_bytes covers
// every configuration); tiled: scratch for the operand copies, the larger of
// tc_tiled_bytes(nQ, N, 128) and tc_fp4_bytes(nQ, N) rounded up to 256 bytes,
// then the larger of tc_tiled_bytes(nDB, N, 208) and tc_fp4_bytes(nDB, N)
// (the second part unused when the caller keeps the database: db_kept, tiled
// by bs_tile_sketches or the FP4 copy of bs_fp4_sketches as `kept` says);
// the call merges its partial lists itself.
// inject: test-only fault injection (0 = none, 1 = the MMA issuer never
// announces its first accumulator; waits give up after kTcInjectWaitLimit)
bs_status topk_tc(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ, const uint32_t *DB,
                  const uint32_t *pcDB, uint32_t nDB, uint32_t N, int measure, uint32_t k,
                  int exclude_self, uint32_t self_off, float *score, uint32_t *idx, void *lists,
                  size_t lists_bytes, void *tiled, const void *db_kept, int kept, int cfg, uint32_t inject,
                  unsigned int *err, cudaStream_t stream);
// row-major sketches [n][N/32] -> the FP4 copy [n][N/2 bytes] (N % 128 == 0)
bs_status fp4_sketches(const uint32_t *sk, uint32_t n, uint32_t N, void *fp4, cudaStream_t stream);
// full count / estimate matrices on the tensor cores (N % 128 == 0, 256 <= N
// <= 8192, 16-byte aligned A and B), reading the row-major sketches directly
bool tc_store_supported(const uint32_t *A, const uint32_t *B, uint32_t N);
bs_status estimate_tc(const uint32_t *A, const uint32_t *pcA, uint32_t nA, const uint32_t *B,
                      const uint32_t *pcB, uint32_t nB, uint32_t N, uint32_t measures, float *out,
                      uint32_t *counts, unsigned int *err, cudaStream_t stream);
// batched tensor-core top-k: workspace bytes (0 when some job is not
// supported) and the call
size_t tc_batched_workspace(const bs_topk_job *jobs, uint32_t n, uint32_t k);
// partial lists per row and non-empty jobs of a batch (host only)
bs_status tc_batched_plan(const bs_topk_job *jobs, uint32_t n, uint32_t k, uint32_t *splits,
                          uint32_t *jobs_run);
bs_status topk_tc_batched(const bs_topk_job *jobs, uint32_t n, int measure, uint32_t k, void *workspace,
                          size_t workspace_bytes, int cfg, unsigned int *err, cudaStream_t stream);
// tensor-core block configuration chosen for k when none is requested
// (allow_tma: the call may build the FP4 database copy); -1 if none fits
int tc_default_cfg(uint32_t k, bool allow_tma);
bool tc_cfg_tma(int cfg);
bool tc_cfg_fits(int cfg, uint32_t k);
bool tc_shape_ok(uint32_t N, uint32_t k);
// row-major sketches [n][N/32] -> k-chunk tiles of R-row blocks (N % 128 == 0)
bs_status tile_sketches(const uint32_t *sk, uint32_t n, uint32_t N, uint32_t R, void *tiled,
                        cudaStream_t stream);

}  // namespace bs
