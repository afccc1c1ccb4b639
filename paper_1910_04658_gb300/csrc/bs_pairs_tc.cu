// Pair counting on the 5th-generation tensor cores, fused with the estimates
// and the per-query top-k (Alg. 1 step 2, Alg. 1-4, Experiment 2 as top-k).
//
// The common-bit count <a_s, b_s> is a dot product of two 0/1 vectors, i.e.
// one entry of the product Q * DB^T of the 0/1 sketch matrices.  Packed bits
// cannot feed tcgen05.mma directly (kind::i8 is not available on sm_103a), so
// every bit is widened to one FP8 (E4M3) element in shared memory: a set bit
// becomes 0x08 = 2^-6 (a single set bit, so 4 elements cost two integer
// instructions), a clear bit 0.  Each product is 2^-12 and every partial sum is
// a multiple of 2^-12 not above N * 2^-12 <= 2, which FP32 holds exactly, so
// the TMEM accumulator times 4096 is the exact integer count.  The widening
// permutes the order of the K elements (word j of the output holds bits
// j, j+8, j+16, j+24), identically for both operands, which a dot product
// does not see.
//
// Block (288 or 416 threads, one per SM, persistent): the (128-row query
// block, 256-row database tile) pairs are numbered row block by row block and
// every block takes an equal contiguous range of them, so the work is even
// across SMs whatever the shape; a row block cut between two blocks yields two
// partial lists, merged by merge_topk_kernel.
//   warp 0     TMEM owner (512 columns) and single-thread MMA issuer:
//              4 x tcgen05.mma.kind::f8f6f4 (M=128, N=256, K=32) per 128-bit
//              k-chunk, into one of two TMEM accumulators
//   warps 1-4  fetch the packed bits of three rows each and widen them into
//              the 128-byte-swizzled K-major FP8 layout the MMA descriptors
//              point at (a 3-deep operand ring when the heap leaves room, else
//              2).  The fetches read a k-chunk-tiled copy of the sketches
//              (128 rows x 16 bytes contiguous per k-chunk, made by
//              tile_kchunks_kernel), so a warp's load is 512 contiguous bytes;
//              four k-chunks are in flight per thread.
//   warps 5+   epilogue, one or two groups of 4 warps: one query row per
//              thread, 32 TMEM columns per tcgen05.ld; a closed-form bound on
//              the union count admits only pairs that can beat the row's
//              current k-th best, whose exact FP32 estimate then enters a
//              per-row heap in shared memory.  With two groups each takes
//              half of every tile's columns into its own heap; the groups
//              publish their k-th best to each other (a pair below either is
//              out of the final list) and merge the two heaps at the end.
// All waits are bounded (mbarrier try_wait with a wall-clock budget); a
// timeout raises BS_ERR_TIMEOUT and the block drains instead of hanging.
#include <math.h>
#include <stdlib.h>

#include <type_traits>

#include "bs_internal.cuh"

namespace bs {
namespace tc {

constexpr int BM = 128;                    // query rows per block (UMMA M, TMEM lanes)
constexpr int BN = 256;                    // database rows per tile (UMMA N)
constexpr int KCW = 4;                     // packed words per k-chunk (128 bits)
// threads per block with NG epilogue groups
__host__ __device__ constexpr int threads_for(int NG) { return 32 * (5 + 4 * NG); }
// Operand slot geometry for SK bytes of K per row (SK = 128: one whole
// 128-bit k-chunk per slot, 128-byte swizzle; SK = 64 / 32: half / quarter
// k-chunks with the 64- / 32-byte swizzle, so the same shared memory holds 2x
// / 4x as many slots and a refill has more queued MMA work to hide behind).
template <int SK>
struct Geo {
    static_assert(SK == 128 || SK == 64 || SK == 32, "slot width");
    static constexpr int A = BM * SK;                       // query operand bytes
    static constexpr int B = BN * SK;                       // database operand bytes
    static constexpr int BYTES = A + B;                     // per slot
    static constexpr int MMAS = SK / 32;                    // K = 32 MMAs per slot
    static constexpr int SPK = 128 / SK;                    // slots per k-chunk
    static constexpr int SHIFT = SK == 128 ? 0 : (SK == 64 ? 1 : 2);
    static constexpr uint64_t LAYOUT = SK == 128 ? 2 : (SK == 64 ? 4 : 6);   // descriptor swizzle code
    static_assert(BYTES % (8 * SK) == 0 && A % (8 * SK) == 0, "swizzle atom alignment");
};
constexpr uint32_t TMEM_COLS = 512;
constexpr int CB = 8;                      // admitted pairs a row buffers within a tile
constexpr uint32_t NO_IDX = 0xFFFFFFFFu;
// Admit when U' >= bound * (1 - 2^-13).  U' is an exact integer and the bound
// carries ~1e-6 relative FP32 error (ex2.approx, the row constants, the key it
// was derived from), so 1.2e-4 keeps every pair whose FP32 key beats the
// threshold (checked against emulated FP32 keys one ulp above it) while
// letting through almost none that fall a full count short.
constexpr float FILTER_SLACK = 0.99987793f;

// Shared-memory layout for NOP operand slots and NG epilogue groups (offsets
// from the 1024-aligned base); the NG heaps of k entries per row follow.
template <int NOP, int NG, int SK>
struct Smem {
    static constexpr int op = 0;
    static constexpr int col = op + NOP * Geo<SK>::BYTES;       // 2 x 2 x 256 floats
    static constexpr int bars = col + 2 * 2 * BN * 4;
    static constexpr int thr = bars + 256;                      // [NG][BM] key, idx, size
    static constexpr int lock = thr + NG * BM * 12;             // [BM] shared-heap row locks
    static constexpr int cbuf = lock + BM * 4;                  // [NG][CB][BM] admitted pairs
    static constexpr int heap = cbuf + NG * CB * BM * 4;
    static_assert((2 * NOP + 4) * 8 + 8 <= 256, "barrier area");
};

struct Args {
    const uint4 *Q, *DB;        // k-chunk-tiled sketches [ceil(n/128)][nKc][128] x 16 bytes
    const uint32_t *pcQ, *pcDB;
    uint32_t nQ, nDB, N, W, nKc, nSl;
    uint32_t k, splits;   // splits: parts of a row's list (merged after)
    uint64_t units;    // row blocks x database tiles; block c covers [c U / G, (c + 1) U / G)
    int exclude_self;  // drop the pair q == self_off + j
    uint32_t self_off;
    float invL;        // 1 / ln(1 - 1/N)
    float log2N, lnN;
    float *score;      // splits == 1
    uint32_t *idx;
    float *ws_key;     // splits > 1: [splits][nQ][k]
    uint32_t *ws_idx;
    unsigned int *err;
};

// ---- tcgen05 wrappers -------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive TMEM columns of this thread's lane; completes at tmem_wait()
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, SK-byte swizzle, 8-row groups
// 8 * SK bytes apart (SBO), leading offset unused for this layout (1).
template <int SK>
__device__ __forceinline__ uint64_t sw_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                     // LBO (ignored for swizzled K-major)
    d |= (uint64_t)((8 * SK) >> 4) << 32;       // SBO
    d |= (uint64_t)1 << 46;                     // descriptor version for tcgen05
    d |= Geo<SK>::LAYOUT << 61;                 // swizzle mode
    return d;
}

// Instruction descriptor: D = F32, A = B = E4M3, both K-major, N = 256, M = 128.
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

// Widen slot h of one row's 128-bit k-chunk (words h * SK/32 ..) into SK
// FP8 bytes and store them into the SK-byte-swizzled K-major tile: row r at
// (r / 8) * 8 SK + (r % 8) * SK, 16-byte chunk c at position
// c ^ ((r % 8) >> SHIFT).  Word p of the slot becomes chunks 2p (bits
// {8b + j}, j = 0..3, as byte b of output word j) and 2p + 1 (j = 4..7).
template <int SK>
__device__ __forceinline__ void widen_store(uint8_t *op_tile, int r, const uint4 &w, int h) {
    const uint32_t x[4] = {w.x, w.y, w.z, w.w};
    constexpr int NW = SK / 32;
    uint8_t *row = op_tile + (r >> 3) * (8 * SK) + (r & 7) * SK;
    const int sw = (r & 7) >> Geo<SK>::SHIFT;
#pragma unroll
    for (int p = 0; p < NW; ++p) {
        const uint32_t v = x[h * NW + p];
        uint4 lo, hi;
        lo.x = (v << 3) & 0x08080808u;
        lo.y = (v << 2) & 0x08080808u;
        lo.z = (v << 1) & 0x08080808u;
        lo.w = v & 0x08080808u;
        hi.x = (v >> 1) & 0x08080808u;
        hi.y = (v >> 2) & 0x08080808u;
        hi.z = (v >> 3) & 0x08080808u;
        hi.w = (v >> 4) & 0x08080808u;
        *reinterpret_cast<uint4 *>(row + (((2 * p) ^ sw) << 4)) = lo;
        *reinterpret_cast<uint4 *>(row + (((2 * p + 1) ^ sw) << 4)) = hi;
    }
}

// Re-layout of a packed sketch matrix [n][W] (W = 4 nKc words) into
// k-chunk tiles: 16-byte chunk kc of row r goes to
// dst[((r / 128) * nKc + kc) * 128 + r % 128]; rows past n are zero.  One
// block moves 128 rows x 8 chunks through shared memory so that both the
// reads (128-byte row pieces) and the writes (2 KB runs) are coalesced.
__global__ void __launch_bounds__(256)
    tile_kchunks_kernel(const uint4 *__restrict__ src, uint32_t n, uint32_t nKc,
                        uint4 *__restrict__ dst) {
    __shared__ uint4 buf[8][129];
    const uint32_t blk = blockIdx.x;
    const uint32_t kc0 = blockIdx.y * 8;
    const int t = threadIdx.x;
    // read: 8 consecutive threads take 8 consecutive chunks of one row
    for (int i = t; i < 128 * 8; i += 256) {
        const uint32_t r = i >> 3, c = i & 7;
        const uint32_t row = blk * 128 + r, kc = kc0 + c;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (row < n && kc < nKc) v = src[(size_t)row * nKc + kc];
        buf[c][r] = v;
    }
    __syncthreads();
    // write: 128 consecutive threads cover one 2 KB run
    for (int i = t; i < 128 * 8; i += 256) {
        const uint32_t c = i >> 7, r = i & 127;
        const uint32_t kc = kc0 + c;
        if (kc < nKc) dst[((size_t)blk * nKc + kc) * 128 + r] = buf[c][r];
    }
}

// ---- per-row heap of the k best (root = worst), interleaved across rows ------
struct Heap {
    float *key;      // key[i * BM + t]
    uint32_t *ix;
    int t, size, cap, levels;
    __device__ float k_at(int i) const { return key[i * BM + t]; }
    __device__ uint32_t i_at(int i) const { return ix[i * BM + t]; }
    __device__ void put(int i, float kk, uint32_t ii) { key[i * BM + t] = kk; ix[i * BM + t] = ii; }
    // append and sift up: parents that rank below the new entry move down
    __device__ void push(float kk, uint32_t ii) {
        int i = size++;
        while (i > 0) {
            const int p = (i - 1) >> 1;
            const float pk = k_at(p);
            const uint32_t pi = i_at(p);
            if (!better(pk, pi, kk, ii)) break;
            put(i, pk, pi);
            i = p;
        }
        put(i, kk, ii);
    }
    // sift (kk, ii) down from slot i over the first n slots: the worse child
    // moves up while the new entry ranks above it
    __device__ void sift_down(int i, float kk, uint32_t ii, int n) {
        for (;;) {
            const int l = 2 * i + 1;
            if (l >= n) break;
            int m = l;
            float mk = k_at(l);
            uint32_t mi = i_at(l);
            if (l + 1 < n) {
                const float rk = k_at(l + 1);
                const uint32_t ri = i_at(l + 1);
                if (better(mk, mi, rk, ri)) { m = l + 1; mk = rk; mi = ri; }
            }
            if (!better(kk, ii, mk, mi)) break;
            put(i, mk, mi);
            i = m;
        }
        put(i, kk, ii);
    }
    __device__ void replace_root(float kk, uint32_t ii) { sift_down(0, kk, ii, size); }
    // in-place heapsort: best first in slots [0, size)
    __device__ void sort_best_first() {
        for (int end = size - 1; end > 0; --end) {
            const float rk = k_at(0);
            const uint32_t ri = i_at(0);
            const float ek = k_at(end);
            const uint32_t ei = i_at(end);
            put(end, rk, ri);
            sift_down(0, ek, ei, end);
        }
    }
};

__host__ __device__ constexpr int heap_levels(int cap) {
    int lv = 0;
    while ((1 << lv) <= cap) ++lv;   // a heap of cap entries has lv levels
    return lv;
}

// Per-row constants of the admission bound (see filter_bound).
struct RowFilter {
    float c0, c1;
    bool all;       // heap not full (or bound not applicable): admit everything
};

// Bound on U' = N - min(a+b-c, N-1) that a pair must reach to beat key theta:
//   JS : log2 U' >= (log2 A' + log2 B' + (theta-1) log2 N) / (1 + theta)   (theta > -1/2)
//   COS: log2 U' >= (theta s_a s_b - s_a^2 - s_b^2) / ln 2 + log2 N,  s = sqrt(-ln(X'/N))
//   IP : U' >= A' B' exp(-theta L) / N
//   HAM: U' >= sqrt(A' B') exp(-theta L / 2)            (theta = -Ham)
// Column values: JS f0 = log2 B'; COS f0 = s_b; IP f0 = B'; HAM f0 = sqrt(B').
// Row value (row_const): JS log2 A'; COS s_a; IP A'/N; HAM sqrt(A').
template <int M>
__device__ __forceinline__ float row_const(float A, uint32_t N) {
    if (M == M_JS) return log2f(A);
    if (M == M_COS) return sqrtf(fmaxf(-logf(A / (float)N), 0.0f));
    if (M == M_IP) return A / (float)N;
    return sqrtf(A);
}

template <int M>
__device__ __forceinline__ RowFilter make_filter(float theta, float rc, float invL, float log2N) {
    RowFilter f;
    f.all = false;
    const float ln2 = 0.69314718056f;
    if (M == M_JS) {
        if (!(theta > -0.5f)) { f.all = true; f.c0 = f.c1 = 0.f; return f; }
        const float e = 1.0f / (1.0f + theta);
        f.c0 = e;
        f.c1 = (rc + (theta - 1.0f) * log2N) * e;
    } else if (M == M_COS) {
        f.c0 = theta * rc / ln2;
        f.c1 = log2N - rc * rc / ln2;
    } else if (M == M_IP) {
        // L < 0, invL = 1/L
        f.c0 = rc * expf(-theta / invL);
        f.c1 = 0.f;
    } else {
        f.c0 = rc * expf(-0.5f * theta / invL);
        f.c1 = 0.f;
    }
    if (!isfinite(f.c0) || !isfinite(f.c1)) f.all = true;
    return f;
}

// 2^x on the special-function unit (relative error ~2^-22, far inside the
// 2^-8 slack of the bound)
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int M>
__device__ __forceinline__ bool admit(const RowFilter &f, float U, float f0) {
    if (f.all) return true;
    float bound;
    if (M == M_JS) bound = ex2_approx(fmaf(f.c0, f0, f.c1));
    else if (M == M_COS) bound = ex2_approx(fmaf(f0, f.c0 - f0 * 1.44269504089f, f.c1));
    else bound = f.c0 * f0;
    return U >= bound * FILTER_SLACK;
}

// Running state of one query row in the epilogue.
struct RowState {
    float thr_k;       // key and index of the heap root once the heap is full,
    uint32_t thr_i;    // else (-inf, none)
    int size;          // entries in the heap
};

// A pair that passed the bound: exact FP32 key, then the heap.  Kept out of
// line -- it runs for a small fraction of the pairs.
// (eff_k, eff_i) is the better of this heap's root (when full) and the other
// group's; a pair not ranking above it cannot reach the final list.
template <int M>
__device__ __forceinline__ RowState consider(RowState st, float *hkey, uint32_t *hix, int t, uint32_t col,
                                          uint32_t c, uint32_t b, uint32_t a, float lnA,
                                          float eff_k, uint32_t eff_i, uint32_t N, float invL,
                                          int cap) {
    const float lnB = M == M_COS ? row_log(b, N) : 0.0f;
    const float key = rank_key<M>(a, b, c, N, lnA, lnB, invL);
    if (!better(key, col, eff_k, eff_i)) return st;
    Heap h;
    h.key = hkey; h.ix = hix; h.t = t; h.size = st.size; h.cap = cap;
    if (h.size < h.cap) {
        h.push(key, col);
        st.size = h.size;
        if (h.size == h.cap) { st.thr_k = h.k_at(0); st.thr_i = h.i_at(0); }
    } else {
        h.replace_root(key, col);
        st.thr_k = h.k_at(0); st.thr_i = h.i_at(0);
    }
    return st;
}

// Shared-heap variant: both epilogue groups insert into one heap per row,
// serialised by a per-row lock (the two threads of a row sit in different
// warps; within a warp every lane has its own row).  The root key is
// published for the filters outside the lock: it only ever improves, so a
// stale value admits more pairs, never fewer, and the exact test against the
// root is repeated under the lock.  Returns the root key once the heap is
// full, else -inf.
template <int M>
__device__ __noinline__ float consider_shared(float *hkey, uint32_t *hix, float *root_key, int *hsize,
                                              unsigned int *lock, int t, uint32_t col, uint32_t c,
                                              uint32_t b, uint32_t a, float lnA, float eff_k,
                                              uint32_t N, float invL, int cap, unsigned int *err) {
    const float lnB = M == M_COS ? row_log(b, N) : 0.0f;
    const float key = rank_key<M>(a, b, c, N, lnA, lnB, invL);
    if (!(key >= eff_k)) return eff_k;            // below the row's known root: cannot enter
    uint32_t spins = 0;
    while (atomicCAS(&lock[t], 0u, 1u) != 0u) {
        if (++spins > (1u << 22)) {               // never expected: report, drop the pair
            raise_error(err, BS_ERR_TIMEOUT);
            return eff_k;
        }
    }
    __threadfence_block();
    Heap h;
    h.key = hkey; h.ix = hix; h.t = t; h.size = hsize[t]; h.cap = cap;
    float root = -INFINITY;
    if (h.size < cap) {
        h.push(key, col);
        hsize[t] = h.size;
        if (h.size == cap) root = h.k_at(0);
    } else {
        if (better(key, col, h.k_at(0), h.i_at(0))) h.replace_root(key, col);
        root = h.k_at(0);
    }
    if (root != -INFINITY) *reinterpret_cast<volatile float *>(&root_key[t]) = root;
    __threadfence_block();
    atomicExch(&lock[t], 0u);
    return root;
}

// v[j] for a per-lane index j, by a select tree over registers (no local memory)
__device__ __forceinline__ uint32_t select32(const uint32_t (&v)[32], uint32_t j) {
    uint32_t t16[16], t8[8], t4[4], t2[2];
#pragma unroll
    for (int i = 0; i < 16; ++i) t16[i] = (j & 16) ? v[i + 16] : v[i];
#pragma unroll
    for (int i = 0; i < 8; ++i) t8[i] = (j & 8) ? t16[i + 8] : t16[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) t4[i] = (j & 4) ? t8[i + 4] : t8[i];
#pragma unroll
    for (int i = 0; i < 2; ++i) t2[i] = (j & 2) ? t4[i + 2] : t4[i];
    return (j & 1) ? t2[1] : t2[0];
}

template <int M, int NOP, int NG, int SK, bool SHARED>
__global__ void __launch_bounds__(threads_for(NG), 1)
    pair_tc_kernel(const Args p) {
    using Smem = tc::Smem<NOP, NG, SK>;
    using G = Geo<SK>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *op = base + Smem::op;
    float *colv = reinterpret_cast<float *>(base + Smem::col);      // [2][2][BN]
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + Smem::bars);
    uint64_t *op_full = bars, *op_empty = bars + NOP;
    uint64_t *acc_full = bars + 2 * NOP, *acc_empty = acc_full + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    float *thr_key = reinterpret_cast<float *>(base + Smem::thr);     // [NG][BM]
    uint32_t *thr_idx = reinterpret_cast<uint32_t *>(thr_key + NG * BM);
    int *heap_size = reinterpret_cast<int *>(thr_idx + NG * BM);
    unsigned int *row_lock = reinterpret_cast<unsigned int *>(base + Smem::lock);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // Persistent schedule: the (row block, database tile) pairs are numbered
    // u = row_block * n_tiles + tile, and block c takes the contiguous range
    // [c U / G, (c + 1) U / G).  A row block split between blocks yields one
    // partial list per block ("part"), merged afterwards.
    const uint32_t n_tiles = (p.nDB + BN - 1) / BN;
    const uint64_t u_lo = p.units * blockIdx.x / gridDim.x;
    const uint64_t u_hi = p.units * (blockIdx.x + 1) / gridDim.x;
    const uint32_t n_my_tiles = (uint32_t)(u_hi - u_lo);

    if (tid == 0) {
        for (int i = 0; i < NOP; ++i) {
            mbar_init(&op_full[i], 4);
            mbar_init(&op_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], 4 * NG);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, TMEM_COLS);
        tmem_relinquish();
    }
    for (int i = tid; i < NG * BM; i += blockDim.x) {   // published thresholds start empty
        thr_key[i] = -INFINITY;
        thr_idx[i] = NO_IDX;
        heap_size[i] = 0;
    }
    for (int i = tid; i < BM; i += blockDim.x) row_lock[i] = 0u;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (*abort_flag) return;
        if (!mbar_wait(bar, parity)) {
            raise_error(p.err, BS_ERR_TIMEOUT);
            *abort_flag = 1;
        }
    };

    if (warp == 0) {
        // ----------------------------- MMA issuer -----------------------------
        if (lane == 0) {
            uint32_t sl = 0;   // operand slots consumed
            const uint32_t nsl = p.nKc * G::SPK;
            for (uint32_t t = 0; t < n_my_tiles; ++t) {
                const uint32_t ab = t & 1;
                if (t >= 2) wait(&acc_empty[ab], ((t >> 1) - 1) & 1);
                tc_fence_after();
                const uint32_t d_tmem = tmem + ab * BN;
                for (uint32_t c = 0; c < nsl; ++c, ++sl) {
                    const uint32_t o = sl % NOP;
                    wait(&op_full[o], (sl / NOP) & 1);
                    tc_fence_after();
                    if (!*abort_flag) {
                        const uint32_t a_addr = smem_u32(op + o * G::BYTES);
                        const uint32_t b_addr = a_addr + G::A;
#pragma unroll
                        for (int kk = 0; kk < G::MMAS; ++kk)
                            mma_f8(d_tmem, sw_desc<SK>(a_addr + kk * 32), sw_desc<SK>(b_addr + kk * 32),
                                   IDESC, (c | (uint32_t)kk) != 0);
                    }
                    mma_commit(&op_empty[o]);
                }
                mma_commit(&acc_full[ab]);
            }
        }
    } else if (warp < 5) {
        // ------------------------------ widening ------------------------------
        // thread e owns query row e and database rows e and e + 128 of a tile
        const int e = tid - 32;   // 0..127
        const uint32_t nblk_db = (p.nDB + 127) / 128;
        const uint4 z = make_uint4(0, 0, 0, 0);
        const uint32_t total = n_my_tiles * p.nKc;
        // k-chunk g of this block's sweep: three 16-byte pieces
        // fetch cursor (row block, tile, k-chunk) of the next k-chunk; fetch()
        // is called for g = 0, 1, 2, ... in order, so it only ever steps
        uint32_t f_rb = (uint32_t)(u_lo / n_tiles), f_tile = (uint32_t)(u_lo % n_tiles), f_kc = 0;
        auto fetch = [&](uint32_t g, uint4 &a_, uint4 &b0_, uint4 &b1_) {
            if (g < total) {
                const uint32_t rb = f_rb, kc = f_kc;
                const uint32_t bb = 2 * f_tile;
                if (++f_kc == p.nKc) {
                    f_kc = 0;
                    if (++f_tile == n_tiles) { f_tile = 0; ++f_rb; }
                }
                a_ = __ldg(p.Q + ((size_t)rb * p.nKc + kc) * 128 + e);
                b0_ = bb < nblk_db ? __ldg(p.DB + ((size_t)bb * p.nKc + kc) * 128 + e) : z;
                b1_ = bb + 1 < nblk_db ? __ldg(p.DB + ((size_t)(bb + 1) * p.nKc + kc) * 128 + e) : z;
            }
        };
        // four k-chunks in flight; a fixed rotation keeps them in registers
        uint4 ra[4], rb0[4], rb1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) fetch(u, ra[u], rb0[u], rb1[u]);
        for (uint32_t g0 = 0; g0 < total; g0 += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t kc = g0 + u;
                if (kc >= total) break;
#pragma unroll
                for (int h = 0; h < G::SPK; ++h) {
                    const uint32_t sl = kc * G::SPK + h;   // operand slot sequence number
                    const uint32_t o = sl % NOP;
                    if (sl >= NOP) wait(&op_empty[o], ((sl / NOP) - 1) & 1);
                    uint8_t *oA = op + o * G::BYTES;
                    uint8_t *oB = oA + G::A;
                    widen_store<SK>(oA, e, ra[u], h);
                    widen_store<SK>(oB, e, rb0[u], h);
                    widen_store<SK>(oB, e + 128, rb1[u], h);
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&op_full[o]);
                }
                fetch(kc + 4, ra[u], rb0[u], rb1[u]);
            }
        }
    } else {
        // ------------------------------ epilogue ------------------------------
        const int grp = (warp - 5) >> 2;           // epilogue group
        const int e = tid - 160 - 128 * grp;       // 0..127 within the group
        const int quarter = warp & 3;              // TMEM lanes this warp may access
        const int r = quarter * 32 + lane;         // row within the block
        // row constants of the current row block (set at each segment start)
        uint32_t q = 0, a = 0, rb = 0;
        bool row_ok = false;
        float rc = 0.0f, lnA = 0.0f, Na = 0.0f;
        float *hkey = reinterpret_cast<float *>(base + Smem::heap) + (size_t)(SHARED ? 0 : grp) * p.k * BM * 2;
        uint32_t *hix = reinterpret_cast<uint32_t *>(hkey + (size_t)p.k * BM);
        constexpr int COLS = BN / NG;              // tile columns of this group
        RowState st;
        st.thr_k = -INFINITY; st.thr_i = NO_IDX; st.size = 0;
        // this row's buffer of admitted pairs, (count << 8) | column in tile
        uint32_t *cb = reinterpret_cast<uint32_t *>(base + Smem::cbuf) + (size_t)grp * CB * BM;
        int nbuf = 0;
        uint32_t d_col0 = 0;          // first column of the tile the buffer belongs to
        const float *d_cv = colv;     // that tile's column values
        float eff_k = -INFINITY;                   // threshold the filter was built from
        uint32_t eff_i = NO_IDX;
        RowFilter filt;
        filt.all = true; filt.c0 = filt.c1 = 0.f;
        // insert every buffered pair of this row into its heap (warp-wide loop)
        auto drain = [&]() {
            while (__any_sync(0xffffffffu, nbuf > 0)) {
                if (nbuf > 0) {
                    --nbuf;
                    const uint32_t ent = cb[nbuf * BM + r];
                    const uint32_t j = ent & 255u;
                    st = consider<M>(st, hkey, hix, r, d_col0 + j, ent >> 8, (uint32_t)d_cv[j], a, lnA,
                                     eff_k, eff_i, p.N, p.invL, (int)p.k);
                    if (st.thr_i != NO_IDX && better(st.thr_k, st.thr_i, eff_k, eff_i)) {
                        eff_k = st.thr_k; eff_i = st.thr_i;
                    }
                }
            }
        };

        uint32_t tile = (uint32_t)(u_lo % n_tiles);   // tile of unit u_lo + t
        rb = (uint32_t)(u_lo / n_tiles);
        for (uint32_t t = 0; t < n_my_tiles; ++t) {
            const uint64_t u = u_lo + t;
            if (t > 0 && ++tile == n_tiles) { tile = 0; ++rb; }
            if (t == 0 || tile == 0) {
                // a new row block: its row constants, empty heaps, empty
                // published thresholds (the other group reads them after the
                // barrier below)
                q = rb * BM + r;
                row_ok = q < p.nQ;
                a = row_ok ? __ldg(p.pcQ + q) : 0u;
                const uint32_t a_cl = a < p.N - 1 ? a : p.N - 1;
                rc = row_const<M>((float)(p.N - a_cl), p.N);   // from A' >= 1
                lnA = row_log(a, p.N);
                Na = (float)(p.N - a);                         // N - a (raw)
                st.thr_k = -INFINITY; st.thr_i = NO_IDX; st.size = 0;
                eff_k = -INFINITY; eff_i = NO_IDX;
                filt.all = true; filt.c0 = filt.c1 = 0.f;
                if (!SHARED || grp == 0) {
                    thr_key[(SHARED ? 0 : grp) * BM + r] = -INFINITY;
                    thr_idx[(SHARED ? 0 : grp) * BM + r] = NO_IDX;
                    heap_size[(SHARED ? 0 : grp) * BM + r] = 0;
                }
                if (NG == 2) named_sync(5, 128 * NG);
            }
            float *cv = colv + (t & 1) * 2 * BN;
            // per-column values of this group's columns (one per thread)
            for (int j = grp * COLS + e; j < (grp + 1) * COLS; j += 128) {
                const uint32_t col = tile * BN + j;
                const uint32_t b = col < p.nDB ? __ldg(p.pcDB + col) : 0u;
                const uint32_t b_cl = b < p.N - 1 ? b : p.N - 1;
                const float Bf = (float)(p.N - b_cl);
                float f0;
                if (M == M_JS) f0 = log2f(Bf);
                else if (M == M_COS) f0 = sqrtf(fmaxf(-logf(Bf / (float)p.N), 0.0f));
                else if (M == M_IP) f0 = Bf;
                else f0 = sqrtf(Bf);
                cv[j] = (float)b;         // raw count: U' is formed from the raw a, b, c
                cv[BN + j] = f0;
            }
            named_sync(2 + grp, 128);
            const uint32_t ab = t & 1;
            wait(&acc_full[ab], (t >> 1) & 1);
            tc_fence_after();
            const uint32_t col0 = tile * BN;
            d_col0 = col0;
            d_cv = cv;
            // every lane stays in the loops below (they vote); dead rows admit nothing
            const bool live = row_ok && !*abort_flag;
            const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + ab * BN;
#pragma unroll 1
            for (int ch = grp * (COLS / 32); ch < (grp + 1) * (COLS / 32); ++ch) {
                uint32_t v[32];
                tmem_ld32_async(trow + ch * 32, v);
                // the threshold to beat: this heap's root or the other group's
                // (shared heap: the published root key, ties admitted)
                float tk = st.thr_k;
                uint32_t ti = st.thr_i;
                if (SHARED) {
                    tk = *reinterpret_cast<volatile float *>(&thr_key[r]);
                    ti = tk == -INFINITY ? NO_IDX : 0xFFFFFFFEu;
                } else if (NG == 2) {
                    const float ok = thr_key[(1 - grp) * BM + r];
                    const uint32_t oi = thr_idx[(1 - grp) * BM + r];
                    if (better(ok, oi, tk, ti)) { tk = ok; ti = oi; }
                }
                if (tk != eff_k || ti != eff_i) {
                    eff_k = tk; eff_i = ti;
                    if (ti == NO_IDX) { filt.all = true; }
                    else filt = make_filter<M>(tk, rc, p.invL, p.log2N);
                }
                tmem_wait();
                // pass 1: which of these 32 pairs can beat the threshold
                uint32_t mask = 0;
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    const int j = ch * 32 + jj;
                    const float cf = __uint_as_float(v[jj]) * 4096.0f;   // exact count
                    // U' = N - min(a + b - c, N - 1) = max(N - a - b + c, 1), exact in FP32
                    const float U = fmaxf(Na - cv[j] + cf, 1.0f);
                    if (admit<M>(filt, U, cv[BN + j])) mask |= 1u << jj;
                }
                // columns past the database end and the self pair never rank
                const uint32_t col_c = col0 + ch * 32;
                if (col_c + 32 > p.nDB)
                    mask &= col_c >= p.nDB ? 0u : (0xFFFFFFFFu >> (32 - (p.nDB - col_c)));
                if (p.exclude_self) {
                    const long long qs = (long long)q - (long long)p.self_off - (long long)col_c;
                    if (qs >= 0 && qs < 32) mask &= ~(1u << (uint32_t)qs);
                }
                if (!live) mask = 0;
                // pass 2: exact keys for the admitted pairs.  Per-group heaps: the
                // pairs are buffered per row and inserted once per tile (the
                // warp loops as often as its busiest row needs); a chunk that
                // does not fit some row's buffer empties the buffers and is
                // inserted directly.
                const int size_before = st.size;
                const uint32_t root_before = st.thr_i;
                const float rootk_before = st.thr_k;
                auto insert_direct = [&](uint32_t m) {
                    while (__any_sync(0xffffffffu, m != 0)) {
                        if (m) {
                            const uint32_t jj = __ffs(m) - 1;
                            m &= m - 1;
                            const uint32_t c = (uint32_t)(__uint_as_float(select32(v, jj)) * 4096.0f);
                            const int j = ch * 32 + (int)jj;
                            if (SHARED) {
                                const float root = consider_shared<M>(hkey, hix, thr_key, heap_size, row_lock,
                                                                      r, col_c + jj, c, (uint32_t)cv[j], a, lnA,
                                                                      eff_k, p.N, p.invL, (int)p.k, p.err);
                                if (root > eff_k) { eff_k = root; eff_i = 0xFFFFFFFEu; }
                            } else {
                                st = consider<M>(st, hkey, hix, r, col_c + jj, c, (uint32_t)cv[j], a, lnA,
                                                 eff_k, eff_i, p.N, p.invL, (int)p.k);
                                if (st.thr_i != NO_IDX && better(st.thr_k, st.thr_i, eff_k, eff_i)) {
                                    eff_k = st.thr_k; eff_i = st.thr_i;
                                }
                            }
                        }
                    }
                };
                if (SHARED) {
                    insert_direct(mask);
                } else if (__any_sync(0xffffffffu, __popc(mask) > CB - nbuf)) {
                    drain();
                    insert_direct(mask);
                } else {
                    while (__any_sync(0xffffffffu, mask != 0)) {
                        if (mask) {
                            const uint32_t jj = __ffs(mask) - 1;
                            mask &= mask - 1;
                            const uint32_t c = (uint32_t)(__uint_as_float(select32(v, jj)) * 4096.0f);
                            cb[nbuf * BM + r] = (c << 8) | (uint32_t)(ch * 32 + (int)jj);
                            ++nbuf;
                        }
                    }
                }
                // publish a changed root to the other group
                if (!SHARED && NG == 2 && (st.size != size_before || st.thr_i != root_before ||
                                           st.thr_k != rootk_before)) {
                    thr_key[grp * BM + r] = st.thr_k;
                    thr_idx[grp * BM + r] = st.thr_i;
                }
                if (eff_i != NO_IDX) filt = make_filter<M>(eff_k, rc, p.invL, p.log2N);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[ab]);
            if (!SHARED) {   // this tile's buffered pairs (TMEM no longer needed)
                const int sz0 = st.size;
                const uint32_t ri0 = st.thr_i;
                const float rk0 = st.thr_k;
                drain();
                if (NG == 2 && (st.size != sz0 || st.thr_i != ri0 || st.thr_k != rk0)) {
                    thr_key[grp * BM + r] = st.thr_k;
                    thr_idx[grp * BM + r] = st.thr_i;
                }
                if (eff_i != NO_IDX) filt = make_filter<M>(eff_k, rc, p.invL, p.log2N);
            }
            if (t + 1 < n_my_tiles && tile + 1 < n_tiles) continue;
            // ---- end of this row block's segment: its list for part `part`
            const uint64_t x0 = u - tile;   // first unit of this row block
            const uint32_t part = blockIdx.x - (uint32_t)(((x0 + 1) * gridDim.x - 1) / p.units);
            // sort each heap best first; with two groups the first merges both lists
            // (shared heap: one list, sorted by the first group once both are done)
            if (SHARED && NG == 2) named_sync(4, 128 * NG);
            if (SHARED) st.size = heap_size[r];
            Heap h;
            h.key = hkey; h.ix = hix; h.t = r; h.size = st.size; h.cap = (int)p.k;
            if (row_ok && (!SHARED || grp == 0)) h.sort_best_first();
            if (!SHARED && NG == 2) {
                heap_size[grp * BM + r] = st.size;
                named_sync(4, 128 * NG);
            }
            if (grp == 0 && row_ok) {
                const float *k1 = reinterpret_cast<float *>(base + Smem::heap) + (size_t)p.k * BM * 2;
                const uint32_t *i1 = reinterpret_cast<const uint32_t *>(k1 + (size_t)p.k * BM);
                const int n0 = st.size, n1 = (!SHARED && NG == 2) ? heap_size[BM + r] : 0;
                int x = 0, y = 0;
                for (int s = 0; s < (int)p.k; ++s) {
                    float kk = -INFINITY;
                    uint32_t ii = NO_IDX;
                    const bool hx = x < n0, hy = y < n1;
                    if (hx || hy) {
                        const float xk = hx ? h.k_at(x) : -INFINITY;
                        const uint32_t xi = hx ? h.i_at(x) : NO_IDX;
                        const float yk = hy ? k1[y * BM + r] : -INFINITY;
                        const uint32_t yi = hy ? i1[y * BM + r] : NO_IDX;
                        if (hx && (!hy || better(xk, xi, yk, yi))) { kk = xk; ii = xi; ++x; }
                        else { kk = yk; ii = yi; ++y; }
                    }
                    if (p.splits == 1) {
                        const size_t o = (size_t)q * p.k + s;
                        p.score[o] = M == M_HAM ? -kk : kk;
                        p.idx[o] = ii;
                    } else {
                        const size_t o = ((size_t)part * p.nQ + q) * p.k + s;
                        p.ws_key[o] = kk;
                        p.ws_idx[o] = ii;
                    }
                }
                // the block holding a row block's last tile also writes empty
                // lists for the part slots this row block does not use
                if (p.splits > 1 && tile + 1 == n_tiles) {
                    for (uint32_t pp = part + 1; pp < p.splits; ++pp)
                        for (int s = 0; s < (int)p.k; ++s) {
                            const size_t o = ((size_t)pp * p.nQ + q) * p.k + s;
                            p.ws_key[o] = -INFINITY;
                            p.ws_idx[o] = NO_IDX;
                        }
                }
            }
            // every heap read of this segment is done before the next one resets them
            if (NG == 2) named_sync(6, 128 * NG);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

}  // namespace tc

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <int NOP, int NG, int SK, bool SH>
static size_t tc_smem_bytes(uint32_t k) {
    return 1024 + tc::Smem<NOP, NG, SK>::heap + (size_t)(SH ? 1 : NG) * k * tc::BM * 8;
}
constexpr size_t kSmemLimit = 232448;   // 227 KB per block

// Block configurations (operand slots, epilogue groups, slot K bytes, one
// heap per row shared by the groups); the index is the c of
// BS_VARIANT_TC_CFG(c).
#define BS_TC_CONFIGS(X)         \
    X(0, 3, 2, 128, false)       \
    X(1, 2, 2, 128, false)       \
    X(2, 3, 1, 128, false)       \
    X(3, 2, 1, 128, false)       \
    X(4, 4, 2, 64, false)        \
    X(5, 8, 2, 32, false)        \
    X(6, 6, 1, 64, false)        \
    X(7, 4, 1, 64, false)        \
    X(8, 3, 2, 128, true)        \
    X(9, 2, 2, 128, true)
constexpr int kTcConfigs = 10;

static size_t tc_cfg_smem(int cfg, uint32_t k) {
    switch (cfg) {
#define X(c, nop, ng, sk, sh) \
    case c: return tc_smem_bytes<nop, ng, sk, sh>(k);
        BS_TC_CONFIGS(X)
#undef X
    }
    return ~size_t(0);
}

bool tc_cfg_fits(int cfg, uint32_t k) { return tc_cfg_smem(cfg, k) <= kSmemLimit; }

// default: the first configuration in this order that fits -- two epilogue
// groups before one, whole-k-chunk slots (measured fastest on the text-BoW
// workload: each slot hand-off has a fixed cost) before finer ones
int tc_default_cfg(uint32_t k) {
    static const int order[kTcConfigs] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9};
    for (int c : order)
        if (tc_cfg_fits(c, k)) return c;
    return -1;
}

bool tc_shape_ok(uint32_t N, uint32_t k) {
    return (N % 128) == 0 && N >= 256 && N <= 8192 && k >= 1 && tc_cfg_fits(3, k);
}

bool tc_supported(const uint32_t *Q, const uint32_t *DB, uint32_t N, uint32_t k) {
    return tc_shape_ok(N, k) && (reinterpret_cast<uintptr_t>(Q) & 15u) == 0 &&
           (reinterpret_cast<uintptr_t>(DB) & 15u) == 0;
}

// Persistent schedule of the tensor-core top-k: one block per SM (at most one
// per unit), block c taking units [c U / G, (c + 1) U / G) of the U = row
// blocks x database tiles.  Returns the most blocks any row block is spread
// over: the number of partial lists per row to merge (1: none).
static uint32_t tc_blocks(uint64_t units) {
    const uint64_t sms = (uint64_t)sm_count();
    return (uint32_t)(units < sms ? units : sms);
}

uint32_t tc_splits(uint32_t nQ, uint32_t nDB) {
    const uint64_t rbs = (nQ + tc::BM - 1) / tc::BM;
    const uint64_t T = (nDB + tc::BN - 1) / tc::BN;
    const uint64_t U = rbs * T;
    if (U == 0) return 1;
    const uint64_t G = tc_blocks(U);
    auto first = [&](uint64_t x) { return ((x + 1) * G - 1) / U; };   // block holding unit x
    uint64_t parts = 1;
    for (uint64_t rb = 0; rb < rbs; ++rb) {
        const uint64_t n = first(rb * T + T - 1) - first(rb * T) + 1;
        if (n > parts) parts = n;
    }
    return (uint32_t)parts;
}

size_t tc_tiled_bytes(uint32_t n, uint32_t N) {
    return (size_t)((n + 127) / 128) * 128 * (N / 8);
}

bs_status tile_sketches(const uint32_t *sk, uint32_t n, uint32_t N, void *tiled, cudaStream_t stream) {
    const uint32_t nKc = N / 128;
    dim3 g((n + 127) / 128, (nKc + 7) / 8);
    tc::tile_kchunks_kernel<<<g, 256, 0, stream>>>(reinterpret_cast<const uint4 *>(sk), n, nKc,
                                                   reinterpret_cast<uint4 *>(tiled));
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

bs_status topk_tc(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ, const uint32_t *DB,
                  const uint32_t *pcDB, uint32_t nDB, uint32_t N, int measure, uint32_t k,
                  int exclude_self, uint32_t self_off, float *score, uint32_t *idx, float *ws_key,
                  uint32_t *ws_idx, uint32_t splits, void *tiled, const void *db_tiled, int cfg_req,
                  unsigned int *err, cudaStream_t stream) {
    const uint32_t W = N / 32;
    const uint32_t nKc = W / tc::KCW;
    // k-chunk-tiled copies of the operands (one copy when Q and DB coincide;
    // none for DB when the caller keeps it tiled)
    uint4 *tQ = reinterpret_cast<uint4 *>(tiled);
    uint4 *tDB = tQ;
    const bool same = (Q == DB && nQ == nDB && !db_tiled);
    {
        dim3 g((nQ + 127) / 128, (nKc + 7) / 8);
        tc::tile_kchunks_kernel<<<g, 256, 0, stream>>>(reinterpret_cast<const uint4 *>(Q), nQ, nKc, tQ);
    }
    if (db_tiled) {
        tDB = const_cast<uint4 *>(reinterpret_cast<const uint4 *>(db_tiled));
    } else if (!same) {
        tDB = reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(tiled) + tc_tiled_bytes(nQ, N));
        dim3 g((nDB + 127) / 128, (nKc + 7) / 8);
        tc::tile_kchunks_kernel<<<g, 256, 0, stream>>>(reinterpret_cast<const uint4 *>(DB), nDB, nKc, tDB);
    }
    if (cudaGetLastError() != cudaSuccess) return BS_ERR_CUDA;
    tc::Args p = {};
    p.Q = tQ; p.DB = tDB;
    p.pcQ = pcQ; p.pcDB = pcDB; p.nQ = nQ; p.nDB = nDB; p.N = N; p.W = W;
    p.nKc = nKc;
    p.nSl = (nKc + 1) / 2;
    p.k = k; p.exclude_self = exclude_self; p.self_off = self_off; p.splits = splits;
    const uint32_t tiles = (nDB + tc::BN - 1) / tc::BN;
    p.units = (uint64_t)((nQ + tc::BM - 1) / tc::BM) * tiles;
    p.invL = (float)(1.0 / log1p(-1.0 / (double)N));
    p.log2N = (float)log2((double)N);
    p.lnN = (float)log((double)N);
    p.score = score; p.idx = idx; p.ws_key = ws_key; p.ws_idx = ws_idx; p.err = err;
    if (p.units == 0) return BS_OK;
    dim3 grid(tc_blocks(p.units));
    // two epilogue groups when two heaps per row fit, three operand slots
    // when there is room left (configuration order: most parallel first)
    const int cfg = cfg_req >= 0 ? cfg_req : tc_default_cfg(k);
    if (cfg < 0 || !tc_cfg_fits(cfg, k)) return BS_ERR_UNSUPPORTED;
    cudaError_t ce = cudaSuccess;
    auto go = [&](auto kern, size_t smem, int threads) {
        if (smem > kSmemLimit) { ce = cudaErrorInvalidConfiguration; return; }
        ce = ensure_smem((const void *)kern, smem);
        if (ce == cudaSuccess) kern<<<grid, threads, smem, stream>>>(p);
    };
    auto launch = [&](auto mtag) {
        constexpr int MM = decltype(mtag)::value;
        switch (cfg) {
#define X(c, nop, ng, sk, sh)                                                                      \
    case c:                                                                                        \
        go(tc::pair_tc_kernel<MM, nop, ng, sk, sh>, tc_smem_bytes<nop, ng, sk, sh>(k), tc::threads_for(ng)); \
        break;
            BS_TC_CONFIGS(X)
#undef X
        }
    };
    switch (measure) {
        case M_IP: launch(std::integral_constant<int, M_IP>()); break;
        case M_HAM: launch(std::integral_constant<int, M_HAM>()); break;
        case M_JS: launch(std::integral_constant<int, M_JS>()); break;
        default: launch(std::integral_constant<int, M_COS>()); break;
    }
    if (ce != cudaSuccess) return BS_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

}  // namespace bs
