// Pair counting on the 5th-generation tensor cores, fused with the estimates
// and either the per-query top-k (Experiment 2 as top-k) or a store of the
// full count / estimate matrices (Alg. 1 step 2, Alg. 1-4).
//
// The common-bit count <a_s, b_s> is a dot product of two 0/1 vectors, i.e.
// one entry of the product Q * DB^T of the 0/1 sketch matrices.  Packed bits
// cannot feed tcgen05.mma directly (there is no 1-bit kind, and kind::i8 is
// not available on sm_103a), so every bit is widened to one 4-bit E2M1
// element of a block-scaled FP4 MMA (kind::mxf4): a set bit becomes 0x2 =
// 1.0, a clear bit 0, and every 32-element block carries the unit scale
// UE8M0 127 = 2^0, held once in TMEM.  Products are 0 or 1 and every partial
// sum is an integer <= N <= 8192 < 2^24, so the FP32 accumulator IS the exact
// count.  A 32-bit word w of a row becomes the 16 bytes
// ((w << 1) & M, w & M, (w >> 1) & M, (w >> 2) & M) with M = 0x22222222 --
// bit 4i + t of w lands in nibble i of output word t -- which permutes the K
// order identically for both operands; a dot product does not see it.
//
// Block (one per SM, persistent): a job table (one job for a single call,
// up to BS_TOPK_BATCH_MAX for the batched form) is cut into work units
// (job, 128-row query block, TB-row database tile).  One problem: block c
// takes the contiguous unit range [block_start[c], block_start[c+1]) (a row
// block cut between blocks yields one partial list per block, a "part",
// merged afterwards); a batch: blocks claim whole row blocks from a device
// counter at run time.  An operand slot covers SK * 2 sketch bits (128 or
// 256) of a tile.  Three ways to feed the operands:
//  - both by TMA (NOP = 0, the default): the host writes FP4 copies of Q and
//    DB once per call; per slot one stage holds the query block's and the
//    database tile's slices (128-byte swizzle, straight from the copies), the
//    MMA reads both from shared memory.  TB = 240 (TMEM: two 240-column
//    accumulators and the scale factors).  Warps: 0 MMA, 1 TMA, 2+ epilogue.
//  - database by TMA, query widened (NB > 0, NOP > 0): the database tile
//    from its FP4 copy, the query's packed bits through a raw ring and
//    widened into TMEM by warps 2-5 (tcgen05.st; A fed from TMEM).
//  - both widened (NB = 0): the packed bits of both (bulk copies of k-chunk
//    tiles, or 2-D tensor maps over row-major sketches for the full-matrix
//    store) through a raw ring; warps 2-5 widen the query row into TMEM and
//    database rows into swizzled shared memory (+ fence.proxy.async).
//    TB = 208: TMEM holds two 208-column accumulators, the query slots and
//    the scale factors.
//   warp 0     TMEM owner (all 512 columns) and single-thread MMA issuer:
//              tcgen05.mma.kind::mxf4.block_scale (M=128, N=TB, K=64), 2 or
//              4 per slot, completion by tcgen05.commit to mbarriers
//   warp 1     producer (one thread): TMA / bulk copies into the stage or
//              raw rings, completion on mbarriers
//   epilogue   one to three groups of 4 warps, one query row per thread, 32
//              or 16 TMEM columns per tcgen05.ld.  Top-k: a closed-form bound
//              on the union count admits only pairs that can beat the row's
//              current k-th best, whose exact FP32 estimate then enters a
//              per-row heap in shared memory (one per group, or one shared by
//              the groups under a per-row lock).  Store: the count and the
//              requested estimates of every pair are written out.
// All waits are bounded (mbarrier try_wait against a cycle budget carried in
// the arguments); a timeout raises BS_ERR_TIMEOUT, the block drains its
// outstanding MMAs (again bounded), frees its TMEM and exits instead of
// hanging.
#pragma once

#include <math.h>

#include "bs_internal.cuh"

namespace bs {
namespace tc {

constexpr int BM = kTcQueryRows;           // query rows per block (UMMA M, TMEM lanes)
constexpr int BN = kTcTileRows;            // database rows per tile (UMMA N)
constexpr int KCW = 4;                     // packed words per k-chunk (128 bits)
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t SF_COL = 480;           // unit scale factors (A at +0, B at +16)
constexpr int MAXG = 192;                  // most persistent blocks per launch
constexpr int MAXJ = BS_TOPK_BATCH_MAX;    // most jobs per batched launch
constexpr int MODE_TOPK = 0, MODE_STORE = 1;
constexpr int IR = 8;                      // dynamic schedule: row blocks published ahead
constexpr uint32_t ITEM_END = 0xFFFFFFFFu; // no row block left
enum { INJECT_NONE = 0, INJECT_STALL = 1 };

// threads per block with NG epilogue groups: MMA warp, producer warp, 4
// widening warps (none when both operands arrive by TMA), the epilogue groups
__host__ __device__ constexpr int epi_warp0(bool widen) { return widen ? 6 : 2; }
__host__ __device__ constexpr int threads_for(int NG, bool widen = true) { return 32 * (epi_warp0(widen) + 4 * NG); }

// Operand slot geometry for SK bytes of K per row: one FP4 byte holds two
// sketch bits, so a slot covers 2 SK bits -- SK = 128: 256 bits (two 128-bit
// k-chunks, 128-byte swizzle, 4 MMAs), SK = 64: 128 bits (64-byte swizzle, 2
// MMAs).  Shared memory holds the database operand (B); the query operand (A)
// sits in TMEM, SK / 4 columns per slot.  A raw slot holds the same bits
// packed as they arrive: tiled, [k-chunk][rows] x 16 bytes; through the tensor
// maps, [rows][SK / 4 bytes].
template <int SK, int TB = BN>
struct Geo {
    static_assert(SK == 128 || SK == 64, "slot width");
    static constexpr int BYTES = TB * SK;                   // database operand bytes per slot
    static constexpr int TCOLS = SK / 4;                    // TMEM columns of a query operand slot
    static constexpr int MMAS = SK / 32;                    // K = 64 (32 bytes) per MMA
    static constexpr int WPS = SK / 16;                     // packed words per slot and row
    static constexpr int KPS = WPS / KCW;                   // 128-bit k-chunks per slot (1, 2)
    static constexpr int SHIFT = SK == 128 ? 0 : 1;         // swizzle: chunk ^ ((row % 8) >> SHIFT)
    static constexpr uint64_t LAYOUT = SK == 128 ? 2 : 4;   // descriptor swizzle code
    static constexpr int RAW_ROW = WPS * 4;                 // packed bytes per row
    static constexpr int RAW_A = BM * RAW_ROW;
    static constexpr int RAW_B = TB * RAW_ROW;
    static constexpr int RAW_SLOT = (RAW_A + RAW_B + 1023) / 1024 * 1024;
    static_assert(BYTES % (8 * SK) == 0, "swizzle atom alignment");
    static_assert(RAW_A % 1024 == 0, "raw slot alignment");
};

// operand slots per tile (SK = 128 pairs the k-chunks; an odd count pads with zeros)
template <int SK>
__host__ __device__ __forceinline__ uint32_t slots_per_tile(uint32_t nKc) {
    return SK == 128 ? (nKc + 1) / 2 : nKc;
}

constexpr int GSPLIT = 96;                 // first column of the second epilogue group
static_assert(GSPLIT % 32 == 0 && GSPLIT <= 256 && BN - GSPLIT <= 256, "two columns a thread per group");
constexpr int CB = 8;                      // admitted pairs a row buffers within a tile
constexpr uint32_t NO_IDX = 0xFFFFFFFFu;
// Admit when U' >= bound * (1 - 2^-13).  U' is an exact integer and the bound
// carries ~1e-6 relative FP32 error (ex2.approx, the row constants, the key it
// was derived from), so 1.2e-4 keeps every pair whose FP32 key beats the
// threshold (checked against emulated FP32 keys one ulp above it) while
// letting through almost none that fall a full count short.
constexpr float FILTER_SLACK = 0.99987793f;
constexpr float LOG2_FILTER_SLACK = -1.76126e-4f;   // log2(FILTER_SLACK), folded into the bounds

// Shared-memory layout for NOP operand slots and RD raw slots of SK bytes
// per row and NG epilogue groups (offsets from the 1024-aligned base); the
// heaps follow.
template <int NOP, int NG, int SK, int RD, int NB = 0, bool SH = false, int TB = BN>
struct Smem {
    using G = Geo<SK, TB>;
    static_assert(NOP * G::TCOLS <= (int)SF_COL - 2 * TB, "query operand slots exceed their TMEM columns");
    static_assert(2 * TB <= (int)SF_COL, "two accumulators and the scale factors exceed TMEM");
    // NOP = 0: NB stages of both operands, filled by TMA from the FP4 copies
    // (query block BM x SK bytes, then database tile BN x SK bytes);
    // NB > 0: NB database slots filled by TMA from the FP4 copy, raw slots hold
    // the query operand only; NB = 0: NOP database slots the widening warps fill
    static constexpr int ABYTES = BM * SK;
    static constexpr int STAGE = ABYTES + G::BYTES;
    static_assert(ABYTES % 1024 == 0 && STAGE % 1024 == 0, "stage alignment");
    static constexpr int op = 0;
    static constexpr int raw = op + (NOP == 0 ? NB * STAGE : (NB > 0 ? NB : NOP) * G::BYTES);
    // per-column (b, f0) of a tile, one copy per epilogue warp for its
    // group's columns: 4 x TB float2
    static constexpr int col = raw + RD * (NB > 0 ? G::RAW_A : G::RAW_SLOT);
    static constexpr int bars = col + 4 * TB * 8;
    static constexpr int thr = bars + 512;                      // [NG][BM] key, idx, size
    static constexpr int lock = thr + NG * BM * 12;             // [BM] shared-heap row locks
    static constexpr int cbuf = lock + BM * 4;                  // [NG][CB][BM] admitted pairs
    static constexpr int heap = cbuf + NG * CB * BM * 4;
    static_assert((2 * NOP + 2 * RD + 2 * NB + 5 + 2 * IR) * 8 + 8 + 4 * IR <= 512, "barrier area");
};

// One problem of the job table: nQ query rows against nDB database rows.
// Top-k reads k-chunk-tiled copies of the sketches -- Q in 128-row blocks,
// DB in 208-row blocks, [block][k-chunk][rows of the block] x 16 bytes -- so
// a slot's bits of a query block or a database tile are one contiguous run;
// the store reads the row-major sketches through the tensor maps of Args.
struct Job {
    const uint4 *tQ, *tDB;      // top-k: tiled copies
    const uint32_t *pcQ, *pcDB;
    float *score;               // top-k, splits == 1: [nQ][k]
    uint32_t *idx;
    float *ws_key;              // top-k, splits > 1: [splits][nQ][k]
    uint32_t *ws_idx;
    float *out;                 // store: [planes][nQ][nDB]
    uint32_t *counts;           // store: [nQ][nDB] or NULL
    uint64_t unit_base;         // first work unit of this job
    uint32_t nQ, nDB, N, nKc;
    uint32_t rbs, tiles;        // row blocks, database tiles
    uint32_t self_off;          // exclude_self drops the pair q_base + q == self_off + j
    uint32_t q_base;            // global index of the job's first query row
    int exclude_self;
    float invL;                 // 1 / ln(1 - 1/N)
    float log2N;
};

template <int NJ>
struct Args {
    CUtensorMap maps[2];              // store: A (box SK/16 words x 128 rows), B (x 208 rows);
                                      // one TMA top-k problem: the FP4 copies of Q and DB
    CUtensorMap jmap[NJ > 1 ? NJ : 1][2];   // a batch's TMA configurations: each job's FP4 maps
    Job job[NJ];
    uint64_t block_start[MAXG + 1];   // block c: units [block_start[c], block_start[c+1])
    uint32_t njobs;
    uint32_t k, splits;               // top-k: list length, parts per row list
    uint32_t measures;                // store: BS_IP | BS_HAM | BS_JS | BS_COS
    uint32_t inject;                  // INJECT_STALL: test-only fault injection
    long long wait_limit;             // cycles a wait may take before it gives up
    unsigned int *err;
    unsigned int *counter;            // dynamic schedule: next row block to claim (zero at launch)
    uint32_t items;                   // dynamic schedule: row blocks of all jobs
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
// D (+)= A * B, A in TMEM at a_tmem, B in shared memory, with per-32-element
// block scales read from TMEM
__device__ __forceinline__ void mma_fp4(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                        uint32_t sfa, uint32_t sfb, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], [%1], %2, %3, [%5], [%6], p;\n\t}\n" ::"r"(
            d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate), "r"(sfa), "r"(sfb)
        : "memory");
}
// the same with the query operand in shared memory too (descriptor adesc)
__device__ __forceinline__ void mma_fp4_ss(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t sfa, uint32_t sfb, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%5], [%6], p;\n\t}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate), "r"(sfa), "r"(sfb)
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

// 32 (or 16) consecutive TMEM columns of this thread's lane; completes at tmem_wait()
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
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 16; i < 32; ++i) r[i] = 0u;
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 32 columns of this warp's 32 lanes set to one value
__device__ __forceinline__ void tmem_fill32(uint32_t taddr, uint32_t v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
        "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(v)
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

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

// Instruction descriptor of the block-scaled MMA: A = B = E2M1 (code 1 of the
// mxf4 kind), both K-major, scale factors UE8M0 (bit 23), N = 208, M = 128,
// scale-factor selectors 0, dense K = 64.
__host__ __device__ constexpr uint32_t idesc_for(int tb) {
    return (1u << 7) | (1u << 10) | ((uint32_t)(tb >> 3) << 17) | (1u << 23) | ((uint32_t)(BM >> 4) << 24);
}
constexpr uint32_t UNIT_SCALES = 0x7F7F7F7Fu;   // four UE8M0 2^0

// Widen the WPS packed words x[] of one row into FP4 and store them into the
// SK-byte-swizzled K-major tile: row r at (r / 8) * 8 SK + (r % 8) * SK, the
// 16-byte chunk of word c at position c ^ ((r % 8) >> SHIFT).
template <int SK>
__device__ __forceinline__ void widen_store(uint8_t *op_tile, int r, const uint32_t (&x)[Geo<SK>::WPS]) {
    uint8_t *row = op_tile + (r >> 3) * (8 * SK) + (r & 7) * SK;
    const int sw = (r & 7) >> Geo<SK>::SHIFT;
#pragma unroll
    for (int c = 0; c < Geo<SK>::WPS; ++c) {
        const uint32_t v = x[c];
        uint4 o;
        o.x = (v << 1) & 0x22222222u;
        o.y = v & 0x22222222u;
        o.z = (v >> 1) & 0x22222222u;
        o.w = (v >> 2) & 0x22222222u;
        *reinterpret_cast<uint4 *>(row + ((c ^ sw) << 4)) = o;
    }
}

// Widen the WPS packed words x[] of this thread's query row into FP4 and
// write them to the row's TMEM lane: widened word 4c + t (t = 0..3 as in
// widen_store) at column taddr + 4c + t, the order the shared-memory operand
// has once unswizzled, so both operands see the same K permutation.
template <int SK>
__device__ __forceinline__ void widen_tmem(uint32_t taddr, const uint32_t (&x)[Geo<SK>::WPS]) {
    uint32_t w[4 * Geo<SK>::WPS];
#pragma unroll
    for (int c = 0; c < Geo<SK>::WPS; ++c) {
        const uint32_t v = x[c];
        w[4 * c] = (v << 1) & 0x22222222u;
        w[4 * c + 1] = v & 0x22222222u;
        w[4 * c + 2] = (v >> 1) & 0x22222222u;
        w[4 * c + 3] = (v >> 2) & 0x22222222u;
    }
    if constexpr (SK == 128) {
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
            "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
            "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]), "r"(w[8]),
            "r"(w[9]), "r"(w[10]), "r"(w[11]), "r"(w[12]), "r"(w[13]), "r"(w[14]), "r"(w[15]), "r"(w[16]),
            "r"(w[17]), "r"(w[18]), "r"(w[19]), "r"(w[20]), "r"(w[21]), "r"(w[22]), "r"(w[23]), "r"(w[24]),
            "r"(w[25]), "r"(w[26]), "r"(w[27]), "r"(w[28]), "r"(w[29]), "r"(w[30]), "r"(w[31])
            : "memory");
    } else {
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
                taddr),
            "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]), "r"(w[8]),
            "r"(w[9]), "r"(w[10]), "r"(w[11]), "r"(w[12]), "r"(w[13]), "r"(w[14]), "r"(w[15])
            : "memory");
    }
}

// The WPS packed words of raw row r: k-chunk h of the row at raw + h * plane
// + r * stride (tiled raw slots: plane = rows x 16, stride 16; row-major raw
// slots: plane 16, stride RAW_ROW); k-chunks from `valid` on read as zero
// (the padding of an odd k-chunk count).
template <int SK>
__device__ __forceinline__ void raw_row(const uint8_t *raw, int plane, int stride, int r, int valid,
                                        uint32_t (&x)[Geo<SK>::WPS]) {
#pragma unroll
    for (int h = 0; h < Geo<SK>::KPS; ++h) {
        uint4 a = make_uint4(0, 0, 0, 0);
        if (h < valid) a = *reinterpret_cast<const uint4 *>(raw + h * plane + r * stride);
        x[4 * h] = a.x; x[4 * h + 1] = a.y; x[4 * h + 2] = a.z; x[4 * h + 3] = a.w;
    }
}

// ---- per-row heap of the k best (root = worst), interleaved across rows ------
// Entry i of row t is the 8-byte (key bits, index) at ent[i * BM + t]: one
// shared-memory load per child while sifting, consecutive rows in
// consecutive entries.
struct Heap {
    uint2 *ent;
    int t, size, cap;
    __device__ void get(int i, float &k, uint32_t &ix) const {
        const uint2 v = ent[i * BM + t];
        k = __uint_as_float(v.x);
        ix = v.y;
    }
    __device__ float k_at(int i) const { return __uint_as_float(ent[i * BM + t].x); }
    __device__ uint32_t i_at(int i) const { return ent[i * BM + t].y; }
    __device__ void put(int i, float kk, uint32_t ii) { ent[i * BM + t] = make_uint2(__float_as_uint(kk), ii); }
    // append and sift up: parents that rank below the new entry move down
    __device__ void push(float kk, uint32_t ii) {
        int i = size++;
        while (i > 0) {
            const int p = (i - 1) >> 1;
            float pk;
            uint32_t pi;
            get(p, pk, pi);
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
            float mk;
            uint32_t mi;
            get(l, mk, mi);
            if (l + 1 < n) {
                float rk;
                uint32_t ri;
                get(l + 1, rk, ri);
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
            float rk, ek;
            uint32_t ri, ei;
            get(0, rk, ri);
            get(end, ek, ei);
            put(end, rk, ri);
            sift_down(0, ek, ei, end);
        }
    }
};

// Per-row constants of the admission bound (see make_filter).
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
    // the slack rides in the constants: 2^(x + log2 s) = s 2^x, (s c0) f0 = s (c0 f0)
    if (M == M_JS || M == M_COS) f.c1 += LOG2_FILTER_SLACK;
    else f.c0 *= FILTER_SLACK;
    if (!isfinite(f.c0) || !isfinite(f.c1)) f.all = true;
    return f;
}

// 2^x on the special-function unit (relative error ~2^-22, far inside the
// 2^-13 slack of the bound)
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int M>
__device__ __forceinline__ bool admit(const RowFilter &f, float U, float f0) {
    if (f.all) return true;
    float bound;   // already lowered by the slack (make_filter)
    if (M == M_JS) bound = ex2_approx(fmaf(f.c0, f0, f.c1));
    else if (M == M_COS) bound = ex2_approx(fmaf(f0, f.c0 - f0 * 1.44269504089f, f.c1));
    else bound = f.c0 * f0;
    return U >= bound;
}

// Running state of one query row in the epilogue.
struct RowState {
    float thr_k;       // key and index of the heap root once the heap is full,
    uint32_t thr_i;    // else (-inf, none)
    int size;          // entries in the heap
};

// A pair that passed the bound: exact FP32 key, then the heap.
// (eff_k, eff_i) is the better of this heap's root (when full) and the other
// group's; a pair not ranking above it cannot reach the final list.
template <int M>
__device__ __forceinline__ RowState consider(RowState st, uint2 *hent, int t, uint32_t col,
                                             uint32_t c, uint32_t b, uint32_t a, float lnA, float eff_k,
                                             uint32_t eff_i, uint32_t N, float invL, int cap) {
    const float lnB = M == M_COS ? row_log(b, N) : 0.0f;
    const float key = rank_key<M>(a, b, c, N, lnA, lnB, invL);
    if (!better(key, col, eff_k, eff_i)) return st;
    Heap h;
    h.ent = hent; h.t = t; h.size = st.size; h.cap = cap;
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
__device__ __forceinline__ float consider_shared(uint2 *hent, float *root_key, int *hsize,
                                              unsigned int *lock, int t, uint32_t col, uint32_t c,
                                              uint32_t b, uint32_t a, float lnA, float eff_k,
                                              uint32_t N, float invL, int cap, unsigned int *err) {
    const float lnB = M == M_COS ? row_log(b, N) : 0.0f;
    const float key = rank_key<M>(a, b, c, N, lnA, lnB, invL);
    if (!(key >= eff_k)) return eff_k;            // below the row's known root: cannot enter
    uint32_t spins = 0;
    // test and test-and-set: a waiter polls with plain reads and sleeps
    // between them, leaving the sub-partition's issue slots and the
    // shared-memory atomics to the thread that holds the lock
    while (atomicCAS(&lock[t], 0u, 1u) != 0u) {
        do {
            if (++spins > (1u << 22)) {           // never expected: report, drop the pair
                raise_error(err, BS_ERR_TIMEOUT);
                return eff_k;
            }
            __nanosleep(32);
        } while (*reinterpret_cast<volatile unsigned int *>(&lock[t]) != 0u);
    }
    __threadfence_block();
    Heap h;
    h.ent = hent; h.t = t; h.size = hsize[t]; h.cap = cap;
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

// Position in the job table: job j, row block rb, database tile `tile`.
struct Cursor {
    uint32_t j, rb, tile;
    __device__ void start(const Job *jobs, uint32_t njobs, uint64_t u) {
        j = 0;
        while (j + 1 < njobs && jobs[j + 1].unit_base <= u) ++j;
        const uint64_t l = u - jobs[j].unit_base;
        rb = (uint32_t)(l / jobs[j].tiles);
        tile = (uint32_t)(l % jobs[j].tiles);
    }
    __device__ void step(const Job *jobs) {
        if (++tile == jobs[j].tiles) {
            tile = 0;
            if (++rb == jobs[j].rbs) { rb = 0; ++j; }
        }
    }
};

// The sequence of tiles one role of a block works through.  Static schedule:
// the contiguous unit range [u_lo, u_lo + count) of the block.  Dynamic
// schedule (DYN): whole row blocks ("items", numbered job by job from each
// job's unit_base), claimed one at a time from a device counter by the TMA
// producer and published in order through a ring of IR shared-memory slots;
// every other role reads the same sequence from the ring.  A row block is
// then never split between blocks.
template <bool DYN>
struct TileSeq {
    const Job *jobs;
    uint32_t njobs;
    Cursor cur;                    // static
    uint32_t left;
    bool started;
    uint64_t *item_full;           // dynamic
    const volatile uint32_t *ring;
    uint32_t it;                   // items read (including the end marker)
    uint32_t j, rb, tile;          // the current tile
    bool in_item;
    __device__ void init_static(const Job *jb, uint32_t nj, uint64_t u_lo, uint32_t count) {
        jobs = jb; njobs = nj; left = count; started = false; in_item = false; it = 0;
        cur.start(jb, nj, u_lo);
    }
    __device__ void init_dynamic(const Job *jb, uint32_t nj, uint64_t *full, const volatile uint32_t *rg) {
        jobs = jb; njobs = nj; item_full = full; ring = rg; it = 0; in_item = false; left = 0; started = false;
    }
    __device__ void set_item(uint32_t item) {
        j = 0;
        while (j + 1 < njobs && jobs[j + 1].unit_base <= item) ++j;
        rb = item - (uint32_t)jobs[j].unit_base;
        tile = 0;
        in_item = true;
    }
    // the next tile; false at the end of the sequence (or once the block aborted)
    template <class W>
    __device__ bool next(W &wait, volatile int *abort_flag) {
        if (!DYN) {
            if (left == 0) return false;
            if (started) cur.step(jobs);
            started = true;
            --left;
            j = cur.j; rb = cur.rb; tile = cur.tile;
            return true;
        }
        if (in_item && tile + 1 < jobs[j].tiles) { ++tile; return true; }
        in_item = false;
        if (*abort_flag) return false;
        const uint32_t slot = it % IR;
        wait(&item_full[slot], (it / IR) & 1);
        if (*abort_flag) return false;
        const uint32_t item = ring[slot];
        ++it;
        if (item == ITEM_END) return false;
        set_item(item);
        return true;
    }
    // this tile ends its row block's work in this block (its list is due)
    __device__ bool segment_end() const { return tile + 1 == jobs[j].tiles || (!DYN && left == 0); }
    // the ring slot of the current item (dynamic)
    __device__ uint32_t slot() const { return (it - 1) % IR; }
};

// The block holding unit x: the last block whose range starts at or before x.
template <int NJ>
__device__ __forceinline__ uint32_t block_of(const Args<NJ> &p, uint64_t x, uint32_t nblocks) {
    uint32_t lo = 0, hi = nblocks - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (p.block_start[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int MODE, int M, int NOP, int NG, int SK, int RD, bool SHARED, int NJ, int NB = 0, int TB = BN>
__global__ void __launch_bounds__(threads_for(NG, NOP > 0), 1)
    pair_tc_kernel(const __grid_constant__ Args<NJ> p) {
    // TB: database rows per tile (the MMA's N)
    using Smem = tc::Smem<NOP, NG, SK, RD, NB, SHARED, TB>;
    using G = Geo<SK, TB>;
    constexpr uint32_t IDESC_T = idesc_for(TB);
    constexpr uint32_t A_COL_T = 2 * TB;   // query operand slots in TMEM (when widened)
    static_assert(TB == BN || NOP == 0, "other tile heights: both operands by TMA");
    static_assert(TB % 16 == 0 && TB <= 256, "MMA N");
    // BT: the database operand arrives already widened, by TMA from an FP4
    // copy in global memory (tensor map p.maps[1], 128-byte swizzle), into NB
    // shared-memory slots; the widening warps write only the query operand.
    // AT (NOP = 0): the query operand too (tensor map p.maps[0], 128-row
    // boxes): NB stages of both operands, no widening warps, the MMA reads
    // both from shared memory
    constexpr bool BT = NB > 0;
    constexpr bool AT = NOP == 0;
    constexpr int EPI0 = epi_warp0(!AT);   // first epilogue warp
    static_assert(!BT || (MODE == MODE_TOPK && SK == 128 && (NJ == 1 || NOP == 0)),
                  "TMA database operand: one top-k problem, or a batch with both operands by TMA");
    static_assert(!AT || (BT && RD == 0), "TMA query operand: stages of both operands");
    static_assert(NG <= 2 || SHARED, "three epilogue groups share one heap per row");
    constexpr uint32_t NOPS = NOP > 0 ? NOP : 1, RDS = RD > 0 ? RD : 1, NBS = NB > 0 ? NB : 1;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *op = base + Smem::op;
    uint8_t *raw = base + Smem::raw;
    float2 *colv = reinterpret_cast<float2 *>(base + Smem::col);    // [4][TB] per-warp column values
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + Smem::bars);
    uint64_t *op_full = bars, *op_empty = bars + NOP;
    uint64_t *raw_full = bars + 2 * NOP, *raw_empty = raw_full + RD;
    uint64_t *acc_full = raw_empty + RD, *acc_empty = acc_full + 2;
    uint64_t *drain_bar = acc_empty + 2;
    uint64_t *item_full = drain_bar + 1, *item_empty = item_full + IR;   // dynamic schedule
    uint64_t *b_full = item_empty + IR, *b_empty = b_full + NB;           // TMA database slots
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(b_empty + NB);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile uint32_t *item_ring = reinterpret_cast<volatile uint32_t *>(tmem_slot + 2);   // [IR]
    // a batch of top-k problems claims whole row blocks at run time; one
    // problem (and the store) deals fixed unit ranges out to the blocks
    constexpr bool DYN = NJ > 1 && MODE == MODE_TOPK;
    float *thr_key = reinterpret_cast<float *>(base + Smem::thr);     // [NG][BM]
    uint32_t *thr_idx = reinterpret_cast<uint32_t *>(thr_key + NG * BM);
    int *heap_size = reinterpret_cast<int *>(thr_idx + NG * BM);
    unsigned int *row_lock = reinterpret_cast<unsigned int *>(base + Smem::lock);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // The job table: one job is read from parameter memory at constant
    // offsets; a batch's table is copied to shared memory once (reads of
    // parameter memory at a run-time index are slow).
    const Job *jobs = p.job;
    if (NJ > 1) {
        Job *sj = reinterpret_cast<Job *>(base + Smem::heap + (size_t)(SHARED ? 1 : NG) * p.k * BM * 8);
        const uint32_t *src = reinterpret_cast<const uint32_t *>(p.job);
        uint32_t *dst = reinterpret_cast<uint32_t *>(sj);
        for (uint32_t i = tid; i < p.njobs * (uint32_t)(sizeof(Job) / 4); i += blockDim.x) dst[i] = src[i];
        jobs = sj;
    }
    const uint32_t njobs = NJ > 1 ? p.njobs : 1u;
    const uint64_t u_lo = p.block_start[blockIdx.x];
    const uint32_t n_my_tiles = (uint32_t)(p.block_start[blockIdx.x + 1] - u_lo);

    if (tid == 0) {
        for (int i = 0; i < NOP; ++i) {
            mbar_init(&op_full[i], 4);
            mbar_init(&op_empty[i], 1);
        }
        for (int i = 0; i < RD; ++i) {
            mbar_init(&raw_full[i], 1);
            mbar_init(&raw_empty[i], 4);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], 4 * NG);
        }
        mbar_init(drain_bar, 1);
        for (int i = 0; i < IR; ++i) {
            mbar_init(&item_full[i], 1);
            mbar_init(&item_empty[i], 4 * NG);
        }
        for (int i = 0; i < NB; ++i) {
            mbar_init(&b_full[i], 1);
            mbar_init(&b_empty[i], 1);
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
    // unit block scales (all 128 lanes of columns SF_COL ..) before any MMA
    if (warp >= EPI0 && warp < EPI0 + 4) tmem_fill32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + SF_COL, UNIT_SCALES);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (*abort_flag) return;
        if (!mbar_wait(bar, parity, p.wait_limit)) {
            raise_error(p.err, BS_ERR_TIMEOUT);
            *abort_flag = 1;
        }
    };

    if (warp == 0) {
        // ----------------------------- MMA issuer -----------------------------
        if (lane == 0) {
            uint32_t sl = 0;   // operand slots consumed
            TileSeq<DYN> seq;
            if (DYN) seq.init_dynamic(jobs, njobs, item_full, item_ring);
            else seq.init_static(jobs, njobs, u_lo, n_my_tiles);
            const uint32_t sfa = tmem + SF_COL, sfb = tmem + SF_COL + 16;
            for (uint32_t t = 0; seq.next(wait, abort_flag); ++t) {
                const uint32_t nsl = slots_per_tile<SK>(jobs[seq.j].nKc);
                const uint32_t ab = t & 1;
                if (t >= 2) wait(&acc_empty[ab], ((t >> 1) - 1) & 1);
                tc_fence_after();
                const uint32_t d_tmem = tmem + ab * TB;
                for (uint32_t c = 0; c < nsl; ++c, ++sl) {
                    const uint32_t o = sl % NOPS;
                    const uint32_t ob = BT ? sl % NBS : o;   // database slot (AT: stage)
                    if (!AT) wait(&op_full[o], (sl / NOPS) & 1);
                    if (BT) wait(&b_full[ob], (sl / NBS) & 1);
                    tc_fence_after();
                    if (!*abort_flag) {
                        if (AT) {
                            const uint32_t a_addr = smem_u32(op + ob * Smem::STAGE);
                            const uint32_t b_addr = a_addr + Smem::ABYTES;
#pragma unroll
                            for (int kk = 0; kk < G::MMAS; ++kk)
                                mma_fp4_ss(d_tmem, sw_desc<SK>(a_addr + kk * 32), sw_desc<SK>(b_addr + kk * 32),
                                           IDESC_T, sfa, sfb, (c | (uint32_t)kk) != 0);
                        } else {
                            const uint32_t a_tmem = tmem + A_COL_T + o * G::TCOLS;
                            const uint32_t b_addr = smem_u32(op + ob * G::BYTES);
#pragma unroll
                            for (int kk = 0; kk < G::MMAS; ++kk)
                                mma_fp4(d_tmem, a_tmem + 8 * kk, sw_desc<SK>(b_addr + kk * 32), IDESC_T, sfa, sfb,
                                        (c | (uint32_t)kk) != 0);
                        }
                    }
                    if (!AT) mma_commit(&op_empty[o]);
                    if (BT) mma_commit(&b_empty[ob]);
                }
                // fault injection (tests only): the first accumulator is never
                // announced, as if this role had died
                if (!(p.inject == INJECT_STALL && t == 0)) mma_commit(&acc_full[ab]);
            }
            // every MMA issued here completes before the TMEM is freed
            mma_commit(drain_bar);
            if (!mbar_wait(drain_bar, 0, p.wait_limit)) raise_error(p.err, BS_ERR_TIMEOUT);
        }
    } else if (warp == 1) {
        // ----------------------------- TMA producer -----------------------------
        if (lane == 0) {
            uint32_t rs = 0;   // raw slots issued
            uint32_t bs = 0;   // TMA database slots (AT: stages) issued
            // the raw slots of one tile
            auto issue_tile = [&](uint32_t jx, uint32_t rb, uint32_t tile) {
                const Job &J = jobs[jx];
                const CUtensorMap *mapA = NJ > 1 ? &p.jmap[NJ > 1 ? jx : 0][0] : &p.maps[0];
                const CUtensorMap *mapB = NJ > 1 ? &p.jmap[NJ > 1 ? jx : 0][1] : &p.maps[1];
                const uint32_t nKc = J.nKc;
                const uint32_t nsl = slots_per_tile<SK>(nKc);
                for (uint32_t c = 0; c < nsl; ++c) {
                    if (AT) {   // one stage: the query block's and the database tile's slot, both by TMA
                        const uint32_t ob = bs % NBS;
                        if (bs >= (uint32_t)NBS) wait(&b_empty[ob], ((bs / NBS) - 1) & 1);
                        if (*abort_flag) return;
                        uint8_t *dst = op + ob * Smem::STAGE;
                        mbar_arrive_expect_tx(&b_full[ob], Smem::STAGE);
                        tma_load_2d(dst, mapA, &b_full[ob], (int)(c * SK), (int)(rb * BM));
                        tma_load_2d(dst + Smem::ABYTES, mapB, &b_full[ob], (int)(c * SK), (int)(tile * TB));
                        ++bs;
                        continue;
                    }
                    const uint32_t o = rs % RDS;
                    if (rs >= RDS) wait(&raw_empty[o], ((rs / RDS) - 1) & 1);
                    if (*abort_flag) return;
                    uint8_t *dst = raw + o * (BT ? G::RAW_A : G::RAW_SLOT);
                    if (BT) {   // the query operand's packed bits; the widened database tile by TMA
                        const uint32_t kc0 = c * G::KPS;
                        const uint32_t np = nKc - kc0 < (uint32_t)G::KPS ? nKc - kc0 : (uint32_t)G::KPS;
                        mbar_arrive_expect_tx(&raw_full[o], np * BM * 16);
                        bulk_load(dst, J.tQ + ((size_t)rb * nKc + kc0) * BM, np * BM * 16, &raw_full[o]);
                        ++rs;
                        const uint32_t ob = bs % NBS;
                        if (bs >= (uint32_t)NBS) wait(&b_empty[ob], ((bs / NBS) - 1) & 1);
                        if (*abort_flag) return;
                        mbar_arrive_expect_tx(&b_full[ob], G::BYTES);
                        tma_load_2d(op + ob * G::BYTES, &p.maps[1], &b_full[ob], (int)(c * SK), (int)(tile * TB));
                        ++bs;
                        continue;
                    }
                    if (MODE == MODE_STORE) {   // strided rows through the tensor maps
                        mbar_arrive_expect_tx(&raw_full[o], G::RAW_A + G::RAW_B);
                        tma_load_2d(dst, &p.maps[0], &raw_full[o], (int)(G::WPS * c), (int)(rb * BM));
                        tma_load_2d(dst + G::RAW_A, &p.maps[1], &raw_full[o], (int)(G::WPS * c), (int)(tile * TB));
                    } else {                    // one contiguous run per operand
                        const uint32_t kc0 = c * G::KPS;
                        const uint32_t np = nKc - kc0 < (uint32_t)G::KPS ? nKc - kc0 : (uint32_t)G::KPS;
                        mbar_arrive_expect_tx(&raw_full[o], np * (BM + TB) * 16);
                        bulk_load(dst, J.tQ + ((size_t)rb * nKc + kc0) * BM, np * BM * 16, &raw_full[o]);
                        bulk_load(dst + G::RAW_A, J.tDB + ((size_t)tile * nKc + kc0) * TB, np * TB * 16,
                                  &raw_full[o]);
                    }
                    ++rs;
                }
            };
            if (DYN) {
                // claim row blocks one at a time and publish each to the other
                // roles; the end marker once none is left (or on abort)
                TileSeq<true> cur;
                cur.init_dynamic(jobs, njobs, item_full, item_ring);
                for (uint32_t it = 0;; ++it) {
                    const uint32_t slot = it % IR;
                    if (it >= (uint32_t)IR) wait(&item_empty[slot], ((it / IR) - 1) & 1);
                    uint32_t item = ITEM_END;
                    if (!*abort_flag) {
                        item = atomicAdd(p.counter, 1u);
                        if (item >= p.items) item = ITEM_END;
                    }
                    item_ring[slot] = item;
                    mbar_arrive(&item_full[slot]);   // release: the entry is visible to the waiters
                    if (item == ITEM_END) break;
                    cur.set_item(item);
                    const Job &J = jobs[cur.j];
                    for (uint32_t tile = 0; tile < J.tiles && !*abort_flag; ++tile) issue_tile(cur.j, cur.rb, tile);
                }
            } else {
                TileSeq<false> seq;
                seq.init_static(jobs, njobs, u_lo, n_my_tiles);
                while (seq.next(wait, abort_flag) && !*abort_flag) issue_tile(seq.j, seq.rb, seq.tile);
            }
            // every copy issued here has landed before the block may exit
            for (uint32_t i = rs > RDS ? rs - RDS : 0; i < rs; ++i)
                if (!mbar_wait(&raw_full[i % RDS], (i / RDS) & 1, p.wait_limit)) raise_error(p.err, BS_ERR_TIMEOUT);
            for (uint32_t i = bs > (uint32_t)NBS ? bs - NBS : 0; i < bs; ++i)
                if (!mbar_wait(&b_full[i % NBS], (i / NBS) & 1, p.wait_limit)) raise_error(p.err, BS_ERR_TIMEOUT);
        }
    } else if (!AT && warp < 6) {
        // ------------------------------ widening ------------------------------
        // thread e owns query row e -- the row of its warp's TMEM lane quarter --
        // and database rows e and e + 128 of a slot
        const int e = (warp & 3) * 32 + lane;   // 0..127
        const bool two_b = e + 128 < TB;
        const uint32_t a_lane = tmem + ((uint32_t)((warp & 3) * 32) << 16) + A_COL_T;
        uint32_t sl = 0;
        TileSeq<DYN> seq;
        if (DYN) seq.init_dynamic(jobs, njobs, item_full, item_ring);
        else seq.init_static(jobs, njobs, u_lo, n_my_tiles);
        while (seq.next(wait, abort_flag)) {
            const uint32_t nKc = jobs[seq.j].nKc;
            const uint32_t nsl = slots_per_tile<SK>(nKc);
            for (uint32_t c = 0; c < nsl; ++c, ++sl) {
                const uint32_t ro = sl % RDS, o = sl % NOPS;
                wait(&raw_full[ro], (sl / RDS) & 1);
                const uint8_t *src = raw + ro * (BT ? G::RAW_A : G::RAW_SLOT);
                uint32_t xa[G::WPS], xb0[G::WPS], xb1[G::WPS];
                if (MODE == MODE_STORE) {
                    raw_row<SK>(src, 16, G::RAW_ROW, e, G::KPS, xa);
                    raw_row<SK>(src + G::RAW_A, 16, G::RAW_ROW, e, G::KPS, xb0);
                    if (two_b) raw_row<SK>(src + G::RAW_A, 16, G::RAW_ROW, e + 128, G::KPS, xb1);
                } else {
                    const int valid = (int)(nKc - c * G::KPS);
                    raw_row<SK>(src, BM * 16, 16, e, valid, xa);
                    if (!BT) raw_row<SK>(src + G::RAW_A, TB * 16, 16, e, valid, xb0);
                    if (!BT && two_b) raw_row<SK>(src + G::RAW_A, TB * 16, 16, e + 128, valid, xb1);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&raw_empty[ro]);   // the raw slot may be refilled
                if (sl >= NOPS) wait(&op_empty[o], ((sl / NOPS) - 1) & 1);
                uint8_t *oB = op + o * G::BYTES;
                widen_tmem<SK>(a_lane + o * G::TCOLS, xa);
                if (!BT) widen_store<SK>(oB, e, xb0);
                if (!BT && two_b) widen_store<SK>(oB, e + 128, xb1);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                if (!BT) fence_async_smem();   // the generic-proxy stores, before the MMA reads them
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&op_full[o]);
            }
        }
    } else {
        // ------------------------------ epilogue ------------------------------
        const int grp = (warp - EPI0) >> 2;        // epilogue group
        const int quarter = warp & 3;              // TMEM lanes this warp may access
        const int r = quarter * 32 + lane;         // row within the block
        // tile columns of this group
        // (two groups: 96 and 112 of 208 columns; three: 64, 64 and 80 of 208,
        // 80 each of 240 -- even splits whose TMEM loads of 32 or 16 columns
        // all start at a multiple of their width)
        constexpr int G3 = TB == 240 ? 80 : 64;
        const int c_lo = NG == 1 ? 0 : (NG == 2 ? grp * GSPLIT : grp * G3);
        const int c_hi = NG == 1 ? TB : (NG == 2 ? (grp == 1 ? TB : GSPLIT) : (grp == NG - 1 ? TB : (grp + 1) * G3));
        // the widest group's columns, and the columns each lane prepares
        constexpr int GW = NG == 1 ? TB
                         : (NG == 2 ? (TB - GSPLIT > GSPLIT ? TB - GSPLIT : GSPLIT)
                                    : (TB - 2 * G3 > G3 ? TB - 2 * G3 : G3));
        constexpr int CPL = (GW + 31) / 32;
        // this warp's own copy of its group's per-column values (raw b, bound
        // term f0), indexed by column - c_lo: every read of them (bound test,
        // buffered and direct insertions) stays within the warp, so the
        // group's warps need no barrier between tiles
        float2 *cv = colv + 4 * c_lo + ((warp - EPI0) & 3) * (c_hi - c_lo);
        // row constants of the current row block (set at each segment start)
        uint32_t q = 0, a = 0;
        bool row_ok = false;
        float rc = 0.0f, lnA = 0.0f, Na = 0.0f;
        uint2 *hent = reinterpret_cast<uint2 *>(base + Smem::heap) + (size_t)(SHARED ? 0 : grp) * p.k * BM;
        RowState st;
        st.thr_k = -INFINITY; st.thr_i = NO_IDX; st.size = 0;
        // this row's buffer of admitted pairs, (count << 8) | column in tile
        uint32_t *cb = reinterpret_cast<uint32_t *>(base + Smem::cbuf) + (size_t)grp * CB * BM;
        int nbuf = 0;
        uint32_t d_col0 = 0;          // first column of the tile the buffer belongs to
        const float2 *d_cv = cv;      // that tile's (b, f0) per column (column - c_lo)
        float eff_k = -INFINITY;                   // threshold the filter was built from
        uint32_t eff_i = NO_IDX;
        RowFilter filt;
        filt.all = true; filt.c0 = filt.c1 = 0.f;
        TileSeq<DYN> seq;
        if (DYN) seq.init_dynamic(jobs, njobs, item_full, item_ring);
        else seq.init_static(jobs, njobs, u_lo, n_my_tiles);
        uint32_t b_pre[CPL];            // counts of this lane's columns of the next tile
        bool b_pre_ok = false;          // b_pre holds them
        uint32_t N = jobs[0].N;
        float invL = jobs[0].invL;
        // insert every buffered pair of this row into its heap (warp-wide loop)
        auto drain = [&]() {
            while (__any_sync(0xffffffffu, nbuf > 0)) {
                if (nbuf > 0) {
                    --nbuf;
                    const uint32_t ent = cb[nbuf * BM + r];
                    const uint32_t j = ent & 255u;
                    if (SHARED) {
                        const float root = consider_shared<M>(hent, thr_key, heap_size, row_lock, r, d_col0 + j,
                                                              ent >> 8, (uint32_t)d_cv[j - c_lo].x, a, lnA, eff_k, N,
                                                              invL, (int)p.k, p.err);
                        if (root > eff_k) { eff_k = root; eff_i = 0xFFFFFFFEu; }
                    } else {
                        st = consider<M>(st, hent, r, d_col0 + j, ent >> 8, (uint32_t)d_cv[j - c_lo].x, a, lnA,
                                         eff_k, eff_i, N, invL, (int)p.k);
                        if (st.thr_i != NO_IDX && better(st.thr_k, st.thr_i, eff_k, eff_i)) {
                            eff_k = st.thr_k; eff_i = st.thr_i;
                        }
                    }
                }
            }
        };

        for (uint32_t t = 0; seq.next(wait, abort_flag); ++t) {
            const Job &J = jobs[seq.j];
            const uint32_t tile = seq.tile;
            if (t == 0 || tile == 0) {
                // a new row block: its row constants, empty heaps, empty
                // published thresholds (the other group reads them after the
                // barrier below)
                N = J.N;
                invL = J.invL;
                q = seq.rb * BM + r;
                row_ok = q < J.nQ;
                a = row_ok ? __ldg(J.pcQ + q) : 0u;
                const uint32_t a_cl = a < N - 1 ? a : N - 1;
                if (MODE == MODE_TOPK) rc = row_const<M>((float)(N - a_cl), N);   // from A' >= 1
                lnA = row_log(a, N);
                Na = (float)(N - a);                         // N - a (raw)
                st.thr_k = -INFINITY; st.thr_i = NO_IDX; st.size = 0;
                eff_k = -INFINITY; eff_i = NO_IDX;
                filt.all = true; filt.c0 = filt.c1 = 0.f;
                if (MODE == MODE_TOPK && (!SHARED || grp == 0)) {
                    thr_key[(SHARED ? 0 : grp) * BM + r] = -INFINITY;
                    thr_idx[(SHARED ? 0 : grp) * BM + r] = NO_IDX;
                    heap_size[(SHARED ? 0 : grp) * BM + r] = 0;
                }
                if (MODE == MODE_TOPK && NG >= 2) named_sync(9, 128 * NG);
            }
            // per-column values (raw b, bound term f0) of this group's columns,
            // CPL per lane, into the warp's own copy (its previous tile's
            // insertions are done); their counts were fetched during the
            // previous tile (the first tile fetches its own)
            __syncwarp();
            if (!b_pre_ok) {
#pragma unroll
                for (int i = 0; i < CPL; ++i) {
                    const uint32_t j = (uint32_t)(c_lo + lane + 32 * i);
                    const uint32_t col = tile * TB + j;
                    b_pre[i] = (j < (uint32_t)c_hi && col < J.nDB) ? __ldg(J.pcDB + col) : 0u;
                }
            }
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const int j = c_lo + lane + 32 * i;
                if (j >= c_hi) continue;
                const uint32_t b = b_pre[i];
                const uint32_t b_cl = b < N - 1 ? b : N - 1;
                const float Bf = (float)(N - b_cl);
                float f0;
                if (MODE == MODE_STORE) f0 = row_log(b, N);
                else if (M == M_JS) f0 = log2f(Bf);
                else if (M == M_COS) f0 = sqrtf(fmaxf(-logf(Bf / (float)N), 0.0f));
                else if (M == M_IP) f0 = Bf;
                else f0 = sqrtf(Bf);
                cv[j - c_lo] = make_float2((float)b, f0);   // raw count: U' is formed from the raw a, b, c
            }
            // the next tile's counts, in flight during this one (when the next
            // tile is known: the rest of a static range, or of the same row block)
            b_pre_ok = false;
            {
                uint32_t nj = 0, ntile = 0;
                if (!DYN && seq.left > 0) {
                    Cursor nx = seq.cur;
                    nx.step(jobs);
                    nj = nx.j; ntile = nx.tile; b_pre_ok = true;
                } else if (DYN && tile + 1 < J.tiles) {
                    nj = seq.j; ntile = tile + 1; b_pre_ok = true;
                }
                if (b_pre_ok) {
                    const Job &J2 = jobs[nj];
#pragma unroll
                    for (int i = 0; i < CPL; ++i) {
                        const uint32_t j = (uint32_t)(c_lo + lane + 32 * i);
                        const uint32_t col = ntile * TB + j;
                        b_pre[i] = (j < (uint32_t)c_hi && col < J2.nDB) ? __ldg(J2.pcDB + col) : 0u;
                    }
                }
            }
            __syncwarp();   // the warp's column values are written
            const uint32_t ab = t & 1;
            wait(&acc_full[ab], (t >> 1) & 1);
            tc_fence_after();
            const uint32_t col0 = tile * TB;
            d_col0 = col0;
            // every lane stays in the loops below (they vote); dead rows admit nothing
            const bool live = row_ok && !*abort_flag;
            const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + ab * TB;
#pragma unroll 1
            for (int c0 = c_lo, width = 0; c0 < c_hi; c0 += width) {
                // 32 columns where aligned and in range, else 16
                width = ((c0 & 31) == 0 && c0 + 32 <= c_hi) ? 32 : 16;
                uint32_t v[32];
                if (width == 32) tmem_ld32_async(trow + c0, v);
                else tmem_ld16_async(trow + c0, v);
                const uint32_t col_c = col0 + c0;
                if (MODE == MODE_STORE) {
                    tmem_wait();
                    if (live) {
                        const size_t plane = (size_t)J.nQ * J.nDB;
                        const size_t o0 = (size_t)q * J.nDB + col_c;
#pragma unroll 4
                        for (int jj = 0; jj < 32; ++jj) {
                            if (jj >= width || col_c + jj >= J.nDB) break;
                            const int j = c0 + jj;
                            const uint32_t c = (uint32_t)__uint_as_float(v[jj]);
                            const uint32_t b = (uint32_t)cv[j - c_lo].x;
                            const float lnB = cv[j - c_lo].y;
                            const size_t o = o0 + jj;
                            if (J.counts) J.counts[o] = c;
                            float *out = J.out + o;
                            if (p.measures & BS_IP) { *out = estimate_one<M_IP>(a, b, c, N, lnA, lnB, invL); out += plane; }
                            if (p.measures & BS_HAM) { *out = estimate_one<M_HAM>(a, b, c, N, lnA, lnB, invL); out += plane; }
                            if (p.measures & BS_JS) { *out = estimate_one<M_JS>(a, b, c, N, lnA, lnB, invL); out += plane; }
                            if (p.measures & BS_COS) *out = estimate_one<M_COS>(a, b, c, N, lnA, lnB, invL);
                        }
                    }
                    continue;
                }
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
                    else filt = make_filter<M>(tk, rc, invL, J.log2N);
                }
                tmem_wait();
                // pass 1: which of these 32 pairs can beat the threshold
                uint32_t mask = 0;
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    const int j = c0 + jj;
                    const float cf = __uint_as_float(v[jj]);   // exact count
                    // U' = N - min(a + b - c, N - 1) = max(N - a - b + c, 1), exact in FP32
                    const float2 bf = cv[j - c_lo];
                    const float U = fmaxf(Na - bf.x + cf, 1.0f);
                    if (admit<M>(filt, U, bf.y)) mask |= 1u << jj;
                }
                if (width < 32) mask &= 0xFFFFu;
                // columns past the database end and the self pair never rank
                if (col_c + 32 > J.nDB)
                    mask &= col_c >= J.nDB ? 0u : (0xFFFFFFFFu >> (32 - (J.nDB - col_c)));
                if (J.exclude_self) {
                    const long long qs = (long long)q + (long long)J.q_base - (long long)J.self_off - (long long)col_c;
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
                const float effk_before = eff_k;
                const uint32_t effi_before = eff_i;
                auto insert_direct = [&](uint32_t m) {
                    while (__any_sync(0xffffffffu, m != 0)) {
                        if (m) {
                            const uint32_t jj = __ffs(m) - 1;
                            m &= m - 1;
                            const uint32_t c = (uint32_t)__uint_as_float(select32(v, jj));
                            const int j = c0 + (int)jj;
                            if (SHARED) {
                                const float root = consider_shared<M>(hent, thr_key, heap_size, row_lock,
                                                                      r, col_c + jj, c, (uint32_t)cv[j - c_lo].x, a, lnA,
                                                                      eff_k, N, invL, (int)p.k, p.err);
                                if (root > eff_k) { eff_k = root; eff_i = 0xFFFFFFFEu; }
                            } else {
                                st = consider<M>(st, hent, r, col_c + jj, c, (uint32_t)cv[j - c_lo].x, a, lnA,
                                                 eff_k, eff_i, N, invL, (int)p.k);
                                if (st.thr_i != NO_IDX && better(st.thr_k, st.thr_i, eff_k, eff_i)) {
                                    eff_k = st.thr_k; eff_i = st.thr_i;
                                }
                            }
                        }
                    }
                };
                if (__any_sync(0xffffffffu, __popc(mask) > CB - nbuf)) {
                    drain();
                    insert_direct(mask);
                } else {
                    while (__any_sync(0xffffffffu, mask != 0)) {
                        if (mask) {
                            const uint32_t jj = __ffs(mask) - 1;
                            mask &= mask - 1;
                            const uint32_t c = (uint32_t)__uint_as_float(select32(v, jj));
                            cb[nbuf * BM + r] = (c << 8) | (uint32_t)(c0 + (int)jj);
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
                // the bound again only if this chunk's insertions raised the threshold
                if (eff_i != NO_IDX && (eff_k != effk_before || eff_i != effi_before))
                    filt = make_filter<M>(eff_k, rc, invL, J.log2N);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[ab]);
            if (MODE == MODE_STORE) continue;
            if (SHARED) {    // this tile's buffered pairs (TMEM no longer needed)
                drain();
                if (eff_i != NO_IDX) filt = make_filter<M>(eff_k, rc, invL, J.log2N);
            } else {
                const int sz0 = st.size;
                const uint32_t ri0 = st.thr_i;
                const float rk0 = st.thr_k;
                drain();
                if (NG == 2 && (st.size != sz0 || st.thr_i != ri0 || st.thr_k != rk0)) {
                    thr_key[grp * BM + r] = st.thr_k;
                    thr_idx[grp * BM + r] = st.thr_i;
                }
                if (eff_i != NO_IDX) filt = make_filter<M>(eff_k, rc, invL, J.log2N);
            }
            if (!seq.segment_end()) continue;
            // ---- end of this row block's segment: its list for part `part`
            // (a dynamically scheduled row block is whole: part 0 of 1)
            uint32_t part = 0;
            if (!DYN) {
                const uint64_t x0 = J.unit_base + (uint64_t)seq.rb * J.tiles;   // first unit of this row block
                part = blockIdx.x - block_of(p, x0, gridDim.x);
            }
            // sort each heap best first; with two groups the first merges both lists
            // (shared heap: one list, sorted by the first group once both are done)
            if (SHARED && NG >= 2) named_sync(8, 128 * NG);
            if (SHARED) st.size = heap_size[r];
            Heap h;
            h.ent = hent; h.t = r; h.size = st.size; h.cap = (int)p.k;
            if (row_ok && (!SHARED || grp == 0)) h.sort_best_first();
            if (!SHARED && NG == 2) {
                heap_size[grp * BM + r] = st.size;
                named_sync(8, 128 * NG);
            }
            if (grp == 0 && row_ok) {
                const uint2 *e1 = reinterpret_cast<const uint2 *>(base + Smem::heap) + (size_t)p.k * BM;
                const int n0 = st.size, n1 = (!SHARED && NG == 2) ? heap_size[BM + r] : 0;
                int x = 0, y = 0;
                for (int s = 0; s < (int)p.k; ++s) {
                    float kk = -INFINITY;
                    uint32_t ii = NO_IDX;
                    const bool hx = x < n0, hy = y < n1;
                    if (hx || hy) {
                        const float xk = hx ? h.k_at(x) : -INFINITY;
                        const uint32_t xi = hx ? h.i_at(x) : NO_IDX;
                        const uint2 yv = hy ? e1[y * BM + r] : make_uint2(__float_as_uint(-INFINITY), NO_IDX);
                        const float yk = __uint_as_float(yv.x);
                        const uint32_t yi = yv.y;
                        if (hx && (!hy || better(xk, xi, yk, yi))) { kk = xk; ii = xi; ++x; }
                        else { kk = yk; ii = yi; ++y; }
                    }
                    if (p.splits == 1) {
                        const size_t o = (size_t)q * p.k + s;
                        J.score[o] = M == M_HAM ? -kk : kk;
                        J.idx[o] = ii;
                    } else {
                        const size_t o = ((size_t)part * J.nQ + q) * p.k + s;
                        J.ws_key[o] = kk;
                        J.ws_idx[o] = ii;
                    }
                }
                // the block holding a row block's last tile also writes empty
                // lists for the part slots this row block does not use
                if (p.splits > 1 && tile + 1 == J.tiles) {
                    for (uint32_t pp = part + 1; pp < p.splits; ++pp)
                        for (int s = 0; s < (int)p.k; ++s) {
                            const size_t o = ((size_t)pp * J.nQ + q) * p.k + s;
                            J.ws_key[o] = -INFINITY;
                            J.ws_idx[o] = NO_IDX;
                        }
                }
            }
            // every heap read of this segment is done before the next one resets them
            if (NG >= 2) named_sync(10, 128 * NG);
            if (DYN) {   // this row block is done: its ring entry may be reused
                __syncwarp();
                if (lane == 0) mbar_arrive(&item_empty[seq.slot()]);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// Block configurations (operand slots, epilogue groups, slot K bytes SK,
// raw-slot ring depth, one heap per row shared by the groups); the index is
// the c of BS_VARIANT_TC_CFG(c).  The default is the first that fits k in this order.
// The last, a single operand slot, keeps k up to BS_TOPK_K_MAX on the tensor
// cores at the cost of overlap between widening and MMA.
// ---------------------------------------------------------------------------
#define BS_TC_CONFIGS(X)             \
    X(0, 2, 2, 128, 4, false, 0, 208)     \
    X(1, 2, 2, 128, 4, true, 0, 208)      \
    X(2, 4, 2, 64, 8, false, 0, 208)      \
    X(3, 4, 2, 64, 8, true, 0, 208)       \
    X(4, 2, 1, 128, 4, false, 0, 208)     \
    X(5, 2, 2, 128, 6, false, 0, 208)     \
    X(6, 2, 2, 128, 2, false, 0, 208)     \
    X(7, 2, 2, 128, 6, true, 0, 208)      \
    X(8, 2, 1, 128, 2, false, 0, 208)     \
    X(9, 1, 1, 128, 2, false, 0, 208)     \
    X(10, 2, 2, 128, 4, false, 3, 208)    \
    X(11, 2, 2, 128, 4, true, 4, 208)     \
    X(12, 0, 3, 128, 0, true, 3, 240)     \
    X(13, 0, 3, 128, 0, true, 2, 240)     \
    X(14, 0, 2, 128, 0, true, 3, 208)
constexpr int kTcConfigs = 15;
constexpr int kTcFirstTma = 10;         // configurations from here on read the FP4 database copy
constexpr size_t kSmemLimit = 232448;   // 227 KB per block

template <int NOP, int NG, int SK, int RD, bool SH, int NB = 0, int TB = BN>
__host__ __device__ constexpr size_t smem_bytes(uint32_t k) {
    return 1024 + Smem<NOP, NG, SK, RD, NB, SH, TB>::heap + (size_t)(SH ? 1 : NG) * k * BM * 8;
}

// Launch of one configuration for one measure (defined in the per-measure
// translation units); cudaErrorInvalidConfiguration when it does not fit k.
template <int M, int NJ>
cudaError_t launch_topk(int cfg, const Args<NJ> &p, uint32_t grid, cudaStream_t stream);
// Store of the full count / estimate matrices (bs_tc_store.cu).
cudaError_t launch_store(const Args<1> &p, uint32_t grid, cudaStream_t stream);

}  // namespace tc
}  // namespace bs
