// Host side of the tensor-core pair kernels (bs_tc_kernel.cuh): the persistent
// schedule, the operand re-layout, the launches of the top-k (one problem or
// a batch of problems) and of the full-matrix store.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "bs_tc_kernel.cuh"

namespace bs {
namespace tc {

// Re-layout of one block of a packed sketch matrix [n][W] (W = 4 nKc words)
// into k-chunk tiles of R-row blocks (R = 128 for queries, 208 for a
// database): 16-byte chunk kc of row r goes to dst[((r / R) * nKc + kc) * R +
// r % R]; rows past n are zero.  One block moves R rows x 8 chunks through
// shared memory so that both the reads (128-byte row pieces) and the writes
// (R x 16-byte runs) are coalesced.
__device__ __forceinline__ void tile_block(const uint4 *__restrict__ src, uint32_t n, uint32_t nKc,
                                           uint4 *__restrict__ dst, uint32_t R, uint32_t blk, uint32_t kc0,
                                           uint4 (&buf)[8][BN + 1]) {
    const int t = threadIdx.x;
    // read: 8 consecutive threads take 8 consecutive chunks of one row
    for (uint32_t i = t; i < R * 8; i += 256) {
        const uint32_t r = i >> 3, c = i & 7;
        const uint32_t row = blk * R + r, kc = kc0 + c;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (row < n && kc < nKc) v = src[(size_t)row * nKc + kc];
        buf[c][r] = v;
    }
    __syncthreads();
    // write: R consecutive threads cover one run
    for (uint32_t i = t; i < R * 8; i += 256) {
        const uint32_t c = i / R, r = i % R;
        const uint32_t kc = kc0 + c;
        if (kc < nKc) dst[((size_t)blk * nKc + kc) * R + r] = buf[c][r];
    }
}

__global__ void __launch_bounds__(256)
    tile_kchunks_kernel(const uint4 *__restrict__ src, uint32_t n, uint32_t nKc, uint32_t R,
                        uint4 *__restrict__ dst) {
    __shared__ uint4 buf[8][BN + 1];
    tile_block(src, n, nKc, dst, R, blockIdx.x, blockIdx.y * 8, buf);
}

// The re-layout of many matrices in one launch: matrix m owns the grid blocks
// [blk_base[m], blk_base[m+1]), ceil(n/R) row blocks x ceil(nKc/8) chunk groups.
struct TileJobs {
    const uint4 *src[2 * MAXJ];
    uint4 *dst[2 * MAXJ];
    uint32_t n[2 * MAXJ], nKc[2 * MAXJ], R[2 * MAXJ];
    uint32_t blk_base[2 * MAXJ + 1];
    uint32_t count;
    unsigned int *counter;   // when set: zeroed by block 0
};

__global__ void __launch_bounds__(256) tile_batched_kernel(const __grid_constant__ TileJobs tj) {
    __shared__ uint4 buf[8][BN + 1];
    const uint32_t b = blockIdx.x;
    if (tj.counter && b == 0 && threadIdx.x == 0) *tj.counter = 0u;
    uint32_t lo = 0, hi = tj.count - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (tj.blk_base[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const uint32_t local = b - tj.blk_base[lo];
    const uint32_t nkg = (tj.nKc[lo] + 7) / 8;
    tile_block(tj.src[lo], tj.n[lo], tj.nKc[lo], tj.dst[lo], tj.R[lo], local / nkg, (local % nkg) * 8, buf);
}

// 2-D tensor map over a row-major sketch matrix [rows][N/32] of uint32 words:
// boxes of box_words words (one operand slot: 4 or 8) x box_rows rows, no
// swizzle, out-of-range rows and words read as zero.  The row stride N/8
// bytes is a multiple of 16 for N % 128 == 0, and every box starts at a word
// index that is a multiple of box_words, i.e. on a 16-byte boundary.
static bool make_map(CUtensorMap *m, const uint32_t *ptr, uint32_t rows, uint32_t N, uint32_t box_words,
                     uint32_t box_rows) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc || rows == 0) return false;
    cuuint64_t dims[2] = {N / 32, rows};
    cuuint64_t strides[1] = {(cuuint64_t)(N / 8)};
    cuuint32_t box[2] = {box_words, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, (void *)ptr, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---- persistent schedule ------------------------------------------------------
// Cost of one work unit in k-chunks.  The MMA / widening sweep over nKc
// k-chunks and the epilogue of the previous tile run at the same time, so a
// tile costs the larger of the two plus a fixed part; the epilogue of a
// 128 x 208 tile was measured at about EPI_KC k-chunks of sweep (a tile of
// N = 256..1024 bits costs the same), the fixed part at FIX_KC.  Only the
// batched form mixes costs; a single problem's units all cost the same.
constexpr uint64_t EPI_KC = 24, FIX_KC = 8;
static uint64_t unit_cost(uint32_t nKc) { return (nKc > EPI_KC ? nKc : EPI_KC) + FIX_KC; }

struct Schedule {
    uint32_t grid = 0, splits = 1;
    uint64_t units = 0;
    uint64_t block_start[MAXG + 1];
};

static uint32_t max_blocks() {
    const int s = sm_count();
    return (uint32_t)(s < 1 ? 1 : (s > MAXG ? MAXG : s));
}

// block holding unit x: the last block whose range starts at or before x
static uint32_t host_block_of(const Schedule &s, uint64_t x) {
    const uint64_t *b = s.block_start;
    return (uint32_t)(std::upper_bound(b, b + s.grid, x) - b) - 1;
}

// Jobs j = 0..nj-1 with rbs[j] row blocks of tiles[j] tiles and unit cost
// cost[j] (all rbs, tiles >= 1).  unit_base[j] receives each job's first unit.
// Block c takes the units whose starting cost s satisfies
// c C <= s G < (c + 1) C, C the total cost, G the grid.
static void make_schedule(uint32_t nj, const uint32_t *rbs, const uint32_t *tiles, const uint64_t *cost,
                          uint64_t *unit_base, Schedule &s) {
    std::vector<uint64_t> cbase(nj + 1);
    uint64_t U = 0, C = 0;
    for (uint32_t j = 0; j < nj; ++j) {
        unit_base[j] = U;
        cbase[j] = C;
        const uint64_t u = (uint64_t)rbs[j] * tiles[j];
        U += u;
        C += u * cost[j];
    }
    cbase[nj] = C;
    s.units = U;
    s.grid = (uint32_t)std::min<uint64_t>(max_blocks(), U);
    if (U == 0) { s.grid = 0; s.splits = 1; return; }
    const uint64_t G = s.grid;
    uint32_t j = 0;
    for (uint64_t c = 0; c < G; ++c) {
        // first unit u with start_cost(u) * G >= c * C
        const unsigned __int128 target = (unsigned __int128)c * C;
        while (j < nj) {
            const uint64_t u_j = (uint64_t)rbs[j] * tiles[j];
            const uint64_t last_start = cbase[j] + (u_j - 1) * cost[j];
            if ((unsigned __int128)last_start * G >= target) break;
            ++j;
        }
        if (j == nj) { s.block_start[c] = U; continue; }
        uint64_t l = 0;
        const unsigned __int128 have = (unsigned __int128)cbase[j] * G;
        if (target > have) {
            const unsigned __int128 den = (unsigned __int128)cost[j] * G;
            l = (uint64_t)((target - have + den - 1) / den);
        }
        s.block_start[c] = unit_base[j] + l;
    }
    s.block_start[G] = U;
    // partial lists per row: the most blocks one row block is spread over
    uint32_t parts = 1;
    for (uint32_t jj = 0; jj < nj; ++jj)
        for (uint32_t rb = 0; rb < rbs[jj]; ++rb) {
            const uint64_t x0 = unit_base[jj] + (uint64_t)rb * tiles[jj];
            const uint32_t n = host_block_of(s, x0 + tiles[jj] - 1) - host_block_of(s, x0) + 1;
            parts = std::max(parts, n);
        }
    s.splits = parts;
}

static void single_schedule(uint32_t nQ, uint32_t nDB, Schedule &s, uint64_t *unit_base, uint32_t tb = BN) {
    const uint32_t rbs = (nQ + BM - 1) / BM, tiles = (nDB + tb - 1) / tb;
    const uint64_t cost = 1;
    make_schedule(1, &rbs, &tiles, &cost, unit_base, s);
}

// The rows left after the rounds of a call that reads the FP4 database copy
// (T < G row blocks): every row block is cut into the same P = min(G / T,
// tiles) parts of its tile sequence, one block per part (block c: row block
// c / P, part c % P), so the T blocks holding part p of the T row blocks
// start at the same tile and sweep the copy together, reading each tile from
// L2 while it is hot.  Balanced ranges over all G blocks would start nearly
// every block at a different tile of a copy larger than L2 and fetch most
// tiles from DRAM; the idle G - T P blocks cost less than that.
static void aligned_schedule(uint32_t nQ, uint32_t nDB, Schedule &s, uint64_t *unit_base, uint32_t tb) {
    const uint32_t rbs = (nQ + BM - 1) / BM, tiles = (nDB + tb - 1) / tb;
    const uint32_t G = max_blocks();
    if (rbs == 0 || tiles == 0 || rbs > G) {
        single_schedule(nQ, nDB, s, unit_base, tb);
        return;
    }
    const uint32_t P = std::max<uint32_t>(1, std::min(G / rbs, tiles));
    s.grid = rbs * P;
    s.units = (uint64_t)rbs * tiles;
    s.splits = P;
    for (uint32_t c = 0; c < s.grid; ++c)
        s.block_start[c] = (uint64_t)(c / P) * tiles + (uint64_t)(c % P) * tiles / P;
    s.block_start[s.grid] = s.units;
    *unit_base = 0;
}

static void fill_job(Job &J, const uint32_t *pcQ, const uint32_t *pcDB, uint32_t nQ, uint32_t nDB,
                     uint32_t N, uint32_t tb = BN) {
    J.pcQ = pcQ; J.pcDB = pcDB;
    J.nQ = nQ; J.nDB = nDB; J.N = N; J.nKc = N / 128;
    J.rbs = (nQ + BM - 1) / BM;
    J.tiles = (nDB + tb - 1) / tb;
    J.invL = (float)(1.0 / log1p(-1.0 / (double)N));
    J.log2N = (float)log2((double)N);
}

// The FP4 copy of a packed sketch matrix that the TMA configurations read as
// their database operand: 32-bit word w becomes the 16 bytes ((w << 1) & M,
// w & M, (w >> 1) & M, (w >> 2) & M), M = 0x22222222 (the widening the
// kernel applies to the query operand), rows stay contiguous (N / 2 bytes).
// One 16-byte input chunk per thread, 64 bytes out.
__global__ void __launch_bounds__(256) widen_fp4_kernel(const uint4 *__restrict__ src, size_t n_chunks,
                                                         uint4 *__restrict__ dst) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_chunks; i += stride) {
        const uint4 v = src[i];
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t)
            dst[4 * i + t] = make_uint4((w[t] << 1) & 0x22222222u, w[t] & 0x22222222u, (w[t] >> 1) & 0x22222222u,
                                        (w[t] >> 2) & 0x22222222u);
    }
}

// The FP4 copies of many matrices in one launch: matrix m's 16-byte input
// chunks are [chunk_base[m], chunk_base[m+1]) of the grid-stride range; block
// 0 also zeroes the batch's claim counter (when given).
struct WidenJobs {
    const uint4 *src[2 * MAXJ];   // a job adds DB, and Q unless Q is DB
    uint4 *dst[2 * MAXJ];
    uint64_t chunk_base[2 * MAXJ + 1];
    uint32_t count;
    unsigned int *counter;
};

__global__ void __launch_bounds__(256) widen_fp4_batched_kernel(const __grid_constant__ WidenJobs wj) {
    if (wj.counter && blockIdx.x == 0 && threadIdx.x == 0) *wj.counter = 0u;
    const uint64_t total = wj.chunk_base[wj.count];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        uint32_t lo = 0, hi = wj.count - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (wj.chunk_base[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const uint64_t x = i - wj.chunk_base[lo];
        const uint4 v = wj.src[lo][x];
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t)
            wj.dst[lo][4 * x + t] = make_uint4((w[t] << 1) & 0x22222222u, w[t] & 0x22222222u,
                                               (w[t] >> 1) & 0x22222222u, (w[t] >> 2) & 0x22222222u);
    }
}

// 2-D tensor map over the FP4 copy [rows][N / 2 bytes]: boxes of one 256-bit
// operand slot (128 bytes) x box_rows rows (BN for a database tile, BM for a
// query block) with the 128-byte swizzle, so a box lands
// in the layout the MMA's database descriptors read; rows past the end and
// the second half of a last 128-bit slot arrive as zeros.  N % 128 == 0 makes
// the row pitch a multiple of 64 bytes.
static bool make_map_fp4(CUtensorMap *m, const void *ptr, uint32_t rows, uint32_t N, uint32_t box_rows) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc || rows == 0) return false;
    cuuint64_t dims[2] = {N / 2, rows};
    cuuint64_t strides[1] = {(cuuint64_t)(N / 2)};
    cuuint32_t box[2] = {128, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tc

// ---------------------------------------------------------------------------
// configuration table
// ---------------------------------------------------------------------------

static size_t tc_cfg_smem(int cfg, uint32_t k) {
    switch (cfg) {
#define X(c, nop, ng, sk, rd, sh, nb, tb) \
    case c: return tc::smem_bytes<nop, ng, sk, rd, sh, nb, tb>(k);
        BS_TC_CONFIGS(X)
#undef X
    }
    return ~size_t(0);
}

bool tc_cfg_fits(int cfg, uint32_t k) { return tc_cfg_smem(cfg, k) <= tc::kSmemLimit; }

static_assert(tc::kTcConfigs == kTcConfigCount && tc::kTcFirstTma == kTcFirstTmaCfg, "configuration table");
bool tc_cfg_tma(int cfg) { return cfg >= tc::kTcFirstTma; }

// configurations with no widening warps: the query operand by TMA as well
// database rows per tile (the MMA's N) of a configuration
uint32_t tc_cfg_tile_rows(int cfg) {
    switch (cfg) {
#define X(c, nop, ng, sk, rd, sh, nb, tb) \
    case c: return tb;
        BS_TC_CONFIGS(X)
#undef X
    }
    return tc::BN;
}

static bool tc_cfg_query_tma(int cfg) {
    switch (cfg) {
#define X(c, nop, ng, sk, rd, sh, nb, tb) \
    case c: return nop == 0;
        BS_TC_CONFIGS(X)
#undef X
    }
    return false;
}

// default: where the call may build the FP4 database copy (one problem, the
// database not kept tiled by the caller), the first TMA configuration that
// fits; otherwise the first configuration in table order that fits -- deeper
// operand rings and two epilogue groups first
int tc_default_cfg(uint32_t k, bool allow_tma) {
    // measured order on the 100,000-row all-pairs top-50: both operands by
    // TMA with three epilogue groups first
    static const int tma_order[] = {12, 13, 14, 10, 11};
    static_assert(sizeof(tma_order) / sizeof(tma_order[0]) == tc::kTcConfigs - tc::kTcFirstTma, "TMA order");
    if (allow_tma)
        for (int c : tma_order)
            if (tc_cfg_fits(c, k)) return c;
    for (int c = 0; c < tc::kTcFirstTma; ++c)
        if (tc_cfg_fits(c, k)) return c;
    return -1;
}

// the batched form: the configurations with both operands by TMA (12, 13, 14)
// first, then the widening ones (the database-only TMA ones need one problem)
static int tc_default_cfg_batched(uint32_t k) {
    for (int c : {12, 13, 14})
        if (tc_cfg_fits(c, k)) return c;
    for (int c = 0; c < tc::kTcFirstTma; ++c)
        if (tc_cfg_fits(c, k)) return c;
    return -1;
}

bool tc_shape_ok(uint32_t N, uint32_t k) {
    return (N % 128) == 0 && N >= 256 && N <= 8192 && k >= 1 && tc_cfg_fits(tc::kTcFirstTma - 1, k);
}

bool tc_supported(const uint32_t *Q, const uint32_t *DB, uint32_t N, uint32_t k) {
    return tc_shape_ok(N, k) && (reinterpret_cast<uintptr_t>(Q) & 15u) == 0 &&
           (reinterpret_cast<uintptr_t>(DB) & 15u) == 0;
}

bool tc_store_supported(const uint32_t *A, const uint32_t *B, uint32_t N) {
    return (N % 128) == 0 && N >= 256 && N <= 8192 && (reinterpret_cast<uintptr_t>(A) & 15u) == 0 &&
           (reinterpret_cast<uintptr_t>(B) & 15u) == 0;
}

uint32_t tc_splits(uint32_t nQ, uint32_t nDB, uint32_t tb, bool aligned) {
    if (nQ == 0 || nDB == 0) return 1;
    tc::Schedule s;
    uint64_t ub;
    if (aligned) tc::aligned_schedule(nQ, nDB, s, &ub, tb);
    else tc::single_schedule(nQ, nDB, s, &ub, tb);
    return s.splits;
}

// Bytes of a k-chunk-tiled copy of n rows in R-row blocks (R = tc::BM for
// queries, tc::BN for a database).
size_t tc_tiled_bytes(uint32_t n, uint32_t N, uint32_t R) { return (size_t)((n + R - 1) / R) * R * (N / 8); }

// Bytes of the FP4 copy of n rows (the TMA configurations' database operand).
size_t tc_fp4_bytes(uint32_t n, uint32_t N) { return (size_t)n * (N / 2); }

bs_status fp4_sketches(const uint32_t *sk, uint32_t n, uint32_t N, void *fp4, cudaStream_t stream) {
    const size_t chunks = (size_t)n * (N / 128);
    if (chunks == 0) return BS_OK;
    const uint32_t blocks = (uint32_t)std::min<size_t>((chunks + 255) / 256, (size_t)sm_count() * 16);
    tc::widen_fp4_kernel<<<blocks, 256, 0, stream>>>(reinterpret_cast<const uint4 *>(sk), chunks,
                                                     reinterpret_cast<uint4 *>(fp4));
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

bs_status tile_sketches(const uint32_t *sk, uint32_t n, uint32_t N, uint32_t R, void *tiled, cudaStream_t stream) {
    if (n == 0) return BS_OK;
    const uint32_t nKc = N / 128;
    dim3 g((n + R - 1) / R, (nKc + 7) / 8);
    tc::tile_kchunks_kernel<<<g, 256, 0, stream>>>(reinterpret_cast<const uint4 *>(sk), n, nKc, R,
                                                   reinterpret_cast<uint4 *>(tiled));
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

template <int NJ>
static cudaError_t launch_measure(int measure, int cfg, const tc::Args<NJ> &p, uint32_t grid,
                                  cudaStream_t stream) {
    switch (measure) {
        case M_IP: return tc::launch_topk<M_IP, NJ>(cfg, p, grid, stream);
        case M_HAM: return tc::launch_topk<M_HAM, NJ>(cfg, p, grid, stream);
        case M_JS: return tc::launch_topk<M_JS, NJ>(cfg, p, grid, stream);
        default: return tc::launch_topk<M_COS, NJ>(cfg, p, grid, stream);
    }
}

// The launches of one tensor-core top-k call.  With the FP4 database copy
// (configurations 10..14) every query block streams the whole copy, which is
// larger than L2, so the first launch deals whole row blocks out in rounds --
// block c takes row blocks [c R, (c + 1) R) -- and all blocks sweep the
// database tiles in the same order at the same time, reading each tile from
// L2 while it is hot; the rows left over (fewer than one per block) run as a
// second launch whose row blocks are cut into equal, aligned parts (partial
// lists, merged by the call) when the copy is too large to stay in L2.
// Otherwise one launch with the balanced ranges.
bs_status tc_call_plan(uint32_t nQ, uint32_t nDB, uint32_t N, uint32_t k, int cfg_req, bool same,
                       int kept, TcCallPlan &pl) {
    pl = TcCallPlan();
    pl.cfg = cfg_req >= 0 ? cfg_req : tc_default_cfg(k, kept != KEPT_TILED);
    if (pl.cfg < 0 || !tc_cfg_fits(pl.cfg, k)) return BS_ERR_UNSUPPORTED;
    pl.fp4_db = tc_cfg_tma(pl.cfg);
    pl.fp4_q = tc_cfg_query_tma(pl.cfg);
    if (pl.fp4_db && kept == KEPT_TILED) return BS_ERR_UNSUPPORTED;   // a kept tiled database has no FP4 copy
    if (!pl.fp4_db && kept == KEPT_FP4) return BS_ERR_UNSUPPORTED;    // and a kept FP4 copy no tiles
    if (nQ == 0 || nDB == 0) return BS_OK;
    const uint32_t rbs = (nQ + tc::BM - 1) / tc::BM;
    const uint32_t G = tc::max_blocks();
    pl.rounds = pl.fp4_db ? rbs / G : 0;
    pl.q_split = (uint32_t)std::min<uint64_t>(nQ, (uint64_t)pl.rounds * G * tc::BM);
    const uint32_t nQ2 = nQ - pl.q_split;
    pl.tile_rows = tc_cfg_tile_rows(pl.cfg);
    pl.aligned = pl.fp4_db && tc_fp4_bytes(nDB, N) > kTcL2Resident;
    pl.splits = nQ2 > 0 ? tc_splits(nQ2, nDB, pl.tile_rows, pl.aligned) : 1;
    pl.lists_bytes = pl.splits > 1 ? (size_t)pl.splits * nQ2 * k * 8 : 0;
    pl.launches = (kept != KEPT_NONE ? 0 : 1) + (pl.fp4_q ? (same ? 0 : 1) : 1) +
                  (pl.rounds > 0 ? 1 : 0) + (nQ2 > 0 ? 1 : 0) + (pl.splits > 1 ? 1 : 0);
    return BS_OK;
}

// partial-list bytes that cover the call plan of every configuration
size_t tc_lists_bytes(uint32_t nQ, uint32_t nDB, uint32_t k) {
    if (nQ == 0 || nDB == 0) return 0;
    const uint32_t s = tc_splits(nQ, nDB);
    size_t b = s > 1 ? (size_t)s * nQ * k * 8 : 0;
    TcCallPlan pl;
    for (int c = tc::kTcFirstTma; c < tc::kTcConfigs; ++c)
        if (tc_cfg_fits(c, k) && tc_call_plan(nQ, nDB, 256, k, c, false, KEPT_NONE, pl) == BS_OK) {
            b = std::max(b, pl.lists_bytes);
            // the aligned parts a larger N's copy would take instead
            const uint32_t nQ2 = nQ - pl.q_split;
            const uint32_t sa = nQ2 > 0 ? tc_splits(nQ2, nDB, pl.tile_rows, true) : 1;
            if (sa > 1) b = std::max(b, (size_t)sa * nQ2 * k * 8);
        }
    return b;
}

bs_status topk_tc(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ, const uint32_t *DB,
                  const uint32_t *pcDB, uint32_t nDB, uint32_t N, int measure, uint32_t k,
                  int exclude_self, uint32_t self_off, float *score, uint32_t *idx, void *lists,
                  size_t lists_bytes, void *tiled, const void *db_kept, int kept, int cfg_req,
                  uint32_t inject, unsigned int *err, cudaStream_t stream) {
    const bool same = kept == KEPT_NONE && Q == DB && nQ == nDB;
    const void *db_tiled = kept == KEPT_TILED ? db_kept : nullptr;
    TcCallPlan pl;
    const bs_status ps = tc_call_plan(nQ, nDB, N, k, cfg_req, same, kept, pl);
    if (ps != BS_OK) return ps;
    if (nQ == 0 || nDB == 0) return BS_OK;
    if (pl.lists_bytes > lists_bytes || (pl.lists_bytes > 0 && !lists)) return BS_ERR_NO_MEMORY;
    const int cfg = pl.cfg;
    static thread_local tc::Args<1> p;   // ~2 KB of launch arguments, rebuilt per launch
    // operand copies: the FP4 copies for the TMA configurations (all-pairs: the
    // database's copy serves as the query operand too), else k-chunk tiles --
    // Q in 128-row, DB in 208-row blocks (none for DB when the caller keeps it tiled)
    auto widen = [&](const uint32_t *src, uint32_t rows, uint4 *dst) {
        const size_t chunks = (size_t)rows * (N / 128);
        const uint32_t blocks = (uint32_t)std::min<size_t>((chunks + 255) / 256, (size_t)sm_count() * 16);
        if (chunks == 0) return true;
        tc::widen_fp4_kernel<<<blocks, 256, 0, stream>>>(reinterpret_cast<const uint4 *>(src), chunks, dst);
        return cudaGetLastError() == cudaSuccess;
    };
    uint4 *tQ = reinterpret_cast<uint4 *>(tiled);
    const size_t q_bytes = std::max(tc_tiled_bytes(nQ, N, tc::BM), tc_fp4_bytes(nQ, N));
    uint4 *db_area = reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(tiled) + ((q_bytes + 255) & ~(size_t)255));
    if (pl.fp4_q) {
        if (!same && !widen(Q, nQ, tQ)) return BS_ERR_CUDA;
    } else if (tile_sketches(Q, nQ, N, tc::BM, tQ, stream) != BS_OK) {
        return BS_ERR_CUDA;
    }
    const uint4 *tDB = reinterpret_cast<const uint4 *>(db_tiled);
    if (kept == KEPT_FP4) {
        db_area = const_cast<uint4 *>(reinterpret_cast<const uint4 *>(db_kept));
    } else if (pl.fp4_db) {
        if (!widen(DB, nDB, db_area)) return BS_ERR_CUDA;
    } else if (!db_tiled) {
        if (tile_sketches(DB, nDB, N, tc::BN, db_area, stream) != BS_OK) return BS_ERR_CUDA;
        tDB = db_area;
    }
    const uint8_t *q_fp4 = same ? reinterpret_cast<const uint8_t *>(db_area) : reinterpret_cast<const uint8_t *>(tQ);
    // one launch over query rows [q_lo, q_lo + rows): in rounds of whole row
    // blocks, or with the balanced ranges (and partial lists when splits > 1)
    auto run = [&](uint32_t q_lo, uint32_t rows, bool rounds) -> bs_status {
        memset(&p, 0, sizeof(p));
        if (pl.fp4_db && !tc::make_map_fp4(&p.maps[1], db_area, nDB, N, pl.tile_rows)) return BS_ERR_CUDA;
        if (pl.fp4_q && !tc::make_map_fp4(&p.maps[0], q_fp4 + (size_t)q_lo * (N / 2), rows, N, tc::BM))
            return BS_ERR_CUDA;
        tc::Job &J = p.job[0];
        tc::fill_job(J, pcQ + q_lo, pcDB, rows, nDB, N, pl.tile_rows);
        J.tQ = tQ + (size_t)(q_lo / tc::BM) * (N / 128) * tc::BM;   // q_lo is a multiple of 128
        J.tDB = tDB;
        J.exclude_self = exclude_self;
        J.self_off = self_off;
        J.q_base = q_lo;
        J.score = score + (size_t)q_lo * k;
        J.idx = idx + (size_t)q_lo * k;
        tc::Schedule s;
        if (rounds) {
            s.grid = tc::max_blocks();
            s.splits = 1;
            const uint64_t per = (uint64_t)pl.rounds * J.tiles;
            for (uint32_t c = 0; c <= s.grid; ++c) s.block_start[c] = (uint64_t)c * per;
            J.unit_base = 0;
        } else if (pl.aligned) {
            tc::aligned_schedule(rows, nDB, s, &J.unit_base, pl.tile_rows);
        } else {
            tc::single_schedule(rows, nDB, s, &J.unit_base, pl.tile_rows);
        }
        if (s.splits > 1) {
            J.ws_key = reinterpret_cast<float *>(lists);
            J.ws_idx = reinterpret_cast<uint32_t *>(J.ws_key + (size_t)s.splits * rows * k);
        }
        memcpy(p.block_start, s.block_start, sizeof(uint64_t) * (s.grid + 1));
        p.njobs = 1;
        p.k = k; p.splits = s.splits;
        p.inject = inject ? tc::INJECT_STALL : tc::INJECT_NONE;
        p.wait_limit = inject ? kTcInjectWaitLimit : kTcWaitLimit;
        p.err = err;
        const cudaError_t ce = launch_measure(measure, cfg, p, s.grid, stream);
        if (ce == cudaErrorInvalidConfiguration) return BS_ERR_UNSUPPORTED;
        if (ce != cudaSuccess) return BS_ERR_CUDA;
        if (s.splits <= 1) return BS_OK;
        return launch_merge(measure, J.ws_key, J.ws_idx, rows, k, s.splits, J.score, J.idx, stream);
    };
    if (pl.q_split > 0) {
        const bs_status s1 = run(0, pl.q_split, true);
        if (s1 != BS_OK) return s1;
    }
    if (pl.q_split < nQ) return run(pl.q_split, nQ - pl.q_split, false);
    return BS_OK;
}

bs_status estimate_tc(const uint32_t *A, const uint32_t *pcA, uint32_t nA, const uint32_t *B,
                      const uint32_t *pcB, uint32_t nB, uint32_t N, uint32_t measures, float *out,
                      uint32_t *counts, unsigned int *err, cudaStream_t stream) {
    static thread_local tc::Args<1> p;
    memset(&p, 0, sizeof(p));
    tc::Job &J = p.job[0];
    tc::fill_job(J, pcA, pcB, nA, nB, N);
    J.out = out;
    J.counts = counts;
    tc::Schedule s;
    tc::single_schedule(nA, nB, s, &J.unit_base);
    if (s.units == 0) return BS_OK;
    // the store kernel runs 256-bit operand slots (8-word boxes)
    if (!tc::make_map(&p.maps[0], A, nA, N, 8, tc::BM) || !tc::make_map(&p.maps[1], B, nB, N, 8, tc::BN))
        return BS_ERR_CUDA;
    memcpy(p.block_start, s.block_start, sizeof(uint64_t) * (s.grid + 1));
    p.njobs = 1;
    p.splits = 1;
    p.measures = measures;
    p.wait_limit = kTcWaitLimit;
    p.err = err;
    return tc::launch_store(p, s.grid, stream) == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

// ---- batched form -------------------------------------------------------------

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

namespace {
// The non-empty jobs of a batch and their dynamic schedule.  The work items
// are the row blocks of all jobs (a row block: 128 queries against the whole
// database of its job, never split, so every list is written once and needs
// no merge).  Jobs run in decreasing cost of one row block (tiles x
// unit_cost) and the blocks of the grid claim items in that order from a
// device counter: the largest items go first and the smallest fill the tail.
struct BatchPlan {
    uint32_t nj = 0;
    uint32_t src[BS_TOPK_BATCH_MAX];        // index in the caller's table, in run order
    uint64_t item_base[BS_TOPK_BATCH_MAX];  // first item of each job
    uint64_t items = 0;
    uint32_t grid = 0;
};

bs_status plan_batch(const bs_topk_job *jobs, uint32_t n, uint32_t k, BatchPlan &bp) {
    bp.nj = 0;
    bp.items = 0;
    bp.grid = 0;
    uint64_t rb_cost[BS_TOPK_BATCH_MAX];
    for (uint32_t i = 0; i < n; ++i) {
        const bs_topk_job &jb = jobs[i];
        if (jb.nQ == 0) continue;
        if (jb.nDB == 0) return BS_ERR_UNSUPPORTED;
        if (!tc_shape_ok(jb.N, k)) return BS_ERR_UNSUPPORTED;
        if (jb.exclude_self && !(jb.Q == jb.DB && jb.nQ == jb.nDB)) return BS_ERR_INVALID_ARG;
        bp.src[bp.nj] = i;
        rb_cost[i] = (uint64_t)((jb.nDB + tc::BN - 1) / tc::BN) * tc::unit_cost(jb.N / 128);
        ++bp.nj;
    }
    std::stable_sort(bp.src, bp.src + bp.nj, [&](uint32_t x, uint32_t y) { return rb_cost[x] > rb_cost[y]; });
    for (uint32_t j = 0; j < bp.nj; ++j) {
        bp.item_base[j] = bp.items;
        bp.items += (jobs[bp.src[j]].nQ + tc::BM - 1) / tc::BM;
    }
    bp.grid = (uint32_t)std::min<uint64_t>(tc::max_blocks(), bp.items);
    return BS_OK;
}

// workspace: [claim counter, 256 bytes] then per job its operand copies --
// Q tiled in 128-row blocks and DB in 208-row blocks, or (configurations with
// both operands by TMA) the FP4 copies of DB and, unless Q is DB, of Q; each
// job's region holds either
constexpr size_t COUNTER_BYTES = 256;
size_t job_ws(const bs_topk_job &jb) {
    const bool same = jb.Q == jb.DB && jb.nQ == jb.nDB;
    const size_t tiled = align256(tc_tiled_bytes(jb.nQ, jb.N, tc::BM)) + align256(tc_tiled_bytes(jb.nDB, jb.N, tc::BN));
    const size_t fp4 = align256(tc_fp4_bytes(jb.nDB, jb.N)) + (same ? 0 : align256(tc_fp4_bytes(jb.nQ, jb.N)));
    return std::max(tiled, fp4);
}
}  // namespace

bs_status tc_batched_plan(const bs_topk_job *jobs, uint32_t n, uint32_t k, uint32_t *splits,
                          uint32_t *jobs_run) {
    static thread_local BatchPlan bp;
    const bs_status st = plan_batch(jobs, n, k, bp);
    if (st != BS_OK) return st;
    if (splits) *splits = 1;
    if (jobs_run) *jobs_run = bp.nj;
    return BS_OK;
}

size_t tc_batched_workspace(const bs_topk_job *jobs, uint32_t n, uint32_t k) {
    static thread_local BatchPlan bp;
    if (plan_batch(jobs, n, k, bp) != BS_OK || bp.nj == 0) return 0;
    size_t b = COUNTER_BYTES;
    for (uint32_t j = 0; j < bp.nj; ++j) b += job_ws(jobs[bp.src[j]]);
    return b;
}

bs_status topk_tc_batched(const bs_topk_job *jobs, uint32_t n, int measure, uint32_t k, void *workspace,
                          size_t workspace_bytes, int cfg_req, unsigned int *err, cudaStream_t stream) {
    for (uint32_t i = 0; i < n; ++i) {
        const bs_topk_job &jb = jobs[i];
        if (jb.nQ == 0) continue;
        if (!jb.Q || !jb.pcQ || !jb.DB || !jb.pcDB || !jb.score || !jb.idx) return BS_ERR_INVALID_ARG;
        if ((reinterpret_cast<uintptr_t>(jb.Q) & 15u) || (reinterpret_cast<uintptr_t>(jb.DB) & 15u))
            return BS_ERR_UNSUPPORTED;
    }
    const int cfg = cfg_req >= 0 ? cfg_req : tc_default_cfg_batched(k);
    if (cfg < 0 || !tc_cfg_fits(cfg, k)) return BS_ERR_UNSUPPORTED;
    const bool fp4 = tc_cfg_query_tma(cfg);   // both operands by TMA from FP4 copies
    if (tc_cfg_tma(cfg) && !fp4) return BS_ERR_UNSUPPORTED;   // database-only TMA: one problem
    static thread_local BatchPlan bp;
    const bs_status ps = plan_batch(jobs, n, k, bp);
    if (ps != BS_OK) return ps;
    if (bp.nj == 0) return BS_OK;
    size_t need = COUNTER_BYTES;
    for (uint32_t j = 0; j < bp.nj; ++j) need += job_ws(jobs[bp.src[j]]);
    if (!workspace || workspace_bytes < need) return BS_ERR_NO_MEMORY;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return BS_ERR_INVALID_ARG;

    static thread_local tc::Args<tc::MAXJ> p;
    static thread_local tc::TileJobs tj;
    static thread_local tc::WidenJobs wj;
    memset(&p, 0, sizeof(p));
    memset(&tj, 0, sizeof(tj));
    memset(&wj, 0, sizeof(wj));
    uint8_t *w = reinterpret_cast<uint8_t *>(workspace);
    unsigned int *counter = reinterpret_cast<unsigned int *>(w);
    w += COUNTER_BYTES;
    if (fp4) {   // the FP4 copies of every job (one launch, which also zeroes the counter) and their maps
        for (uint32_t j = 0; j < bp.nj; ++j) {
            const bs_topk_job &jb = jobs[bp.src[j]];
            uint8_t *region = w;
            w += job_ws(jb);
            const bool same = jb.Q == jb.DB && jb.nQ == jb.nDB;
            uint8_t *db4 = region;
            uint8_t *q4 = same ? db4 : region + align256(tc_fp4_bytes(jb.nDB, jb.N));
            auto add = [&](const uint32_t *src, uint32_t rows, uint8_t *dst) {
                const uint32_t m = wj.count++;
                wj.src[m] = reinterpret_cast<const uint4 *>(src);
                wj.dst[m] = reinterpret_cast<uint4 *>(dst);
                wj.chunk_base[m + 1] = wj.chunk_base[m] + (uint64_t)rows * (jb.N / 128);
            };
            add(jb.DB, jb.nDB, db4);
            if (!same) add(jb.Q, jb.nQ, q4);
            tc::Job &J = p.job[j];
            tc::fill_job(J, jb.pcQ, jb.pcDB, jb.nQ, jb.nDB, jb.N, tc_cfg_tile_rows(cfg));
            J.exclude_self = jb.exclude_self;
            J.self_off = 0;
            J.score = jb.score; J.idx = jb.idx; J.ws_key = nullptr; J.ws_idx = nullptr;
            J.unit_base = bp.item_base[j];
            if (!tc::make_map_fp4(&p.jmap[j][0], q4, jb.nQ, jb.N, tc::BM) ||
                !tc::make_map_fp4(&p.jmap[j][1], db4, jb.nDB, jb.N, tc_cfg_tile_rows(cfg)))
                return BS_ERR_CUDA;
        }
        wj.counter = counter;   // zeroed here, ahead of the pair kernel on this stream
        const uint64_t total = wj.chunk_base[wj.count];
        const uint32_t blocks = (uint32_t)std::min<uint64_t>((total + 255) / 256, (uint64_t)sm_count() * 16);
        tc::widen_fp4_batched_kernel<<<blocks > 0 ? blocks : 1, 256, 0, stream>>>(wj);
        if (cudaGetLastError() != cudaSuccess) return BS_ERR_CUDA;
        p.njobs = bp.nj;
        p.k = k;
        p.splits = 1;
        p.counter = counter;
        p.items = (uint32_t)bp.items;
        p.wait_limit = kTcWaitLimit;
        p.err = err;
        const cudaError_t ce = launch_measure(measure, cfg, p, bp.grid, stream);
        if (ce == cudaErrorInvalidConfiguration) return BS_ERR_UNSUPPORTED;
        return ce == cudaSuccess ? BS_OK : BS_ERR_CUDA;
    }
    uint32_t blk = 0;
    auto add_tile = [&](const uint32_t *src, uint32_t rows, uint32_t N, uint32_t R, uint8_t *&at) {
        uint4 *dst = reinterpret_cast<uint4 *>(at);
        at += align256(tc_tiled_bytes(rows, N, R));
        const uint32_t m = tj.count++;
        tj.src[m] = reinterpret_cast<const uint4 *>(src);
        tj.dst[m] = dst;
        tj.n[m] = rows;
        tj.nKc[m] = N / 128;
        tj.R[m] = R;
        tj.blk_base[m] = blk;
        blk += ((rows + R - 1) / R) * ((N / 128 + 7) / 8);
        return dst;
    };
    for (uint32_t j = 0; j < bp.nj; ++j) {
        const bs_topk_job &jb = jobs[bp.src[j]];
        tc::Job &J = p.job[j];
        tc::fill_job(J, jb.pcQ, jb.pcDB, jb.nQ, jb.nDB, jb.N);
        uint8_t *at = w;
        w += job_ws(jb);
        J.tQ = add_tile(jb.Q, jb.nQ, jb.N, tc::BM, at);
        J.tDB = add_tile(jb.DB, jb.nDB, jb.N, tc::BN, at);
        J.exclude_self = jb.exclude_self;
        J.self_off = 0;
        J.score = jb.score; J.idx = jb.idx; J.ws_key = nullptr; J.ws_idx = nullptr;
        J.unit_base = bp.item_base[j];
    }
    tj.blk_base[tj.count] = blk;
    tj.counter = counter;   // zeroed by the re-layout launch, ahead of the pair kernel on this stream
    tc::tile_batched_kernel<<<blk, 256, 0, stream>>>(tj);
    if (cudaGetLastError() != cudaSuccess) return BS_ERR_CUDA;
    p.njobs = bp.nj;
    p.k = k;
    p.splits = 1;
    p.counter = counter;
    p.items = (uint32_t)bp.items;
    p.wait_limit = kTcWaitLimit;
    p.err = err;
    const cudaError_t ce = launch_measure(measure, cfg, p, bp.grid, stream);
    if (ce == cudaErrorInvalidConfiguration) return BS_ERR_UNSUPPORTED;
    return ce == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

}  // namespace bs
