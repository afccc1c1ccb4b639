// Pair counting and estimation: Alg. 1 step 2 (n_{a_s,b_s} = <a_s, b_s>),
// the estimators of Alg. 1-4, and the ranking of Experiment 2 (Sec. 4) as a
// fused per-query top-k.  Variant "LOP3+POPC": the common-bit count of two
// packed rows is the sum over words of popc(a_w & b_w).
//
// Block layout: one producer warp streams 128-byte-wide k-chunks of a BM-row
// query tile and a BN-row database tile into a STAGES-deep shared-memory ring
// with TMA (cp.async.bulk.tensor, 128-byte swizzle, mbarrier completion); 8
// consumer warps (16x16 threads, each owning 2 query rows x 8 database rows)
// read 16-byte swizzled words, AND them and accumulate popcounts in
// registers.  Either the estimates are written out (bs_estimate_pairs) or
// each pair's score is filtered against the running k-th best of its query
// row and kept in a per-row candidate buffer that is bitonic-sorted and cut
// back to k whenever it could overflow (bs_topk); the count matrix never
// reaches HBM.  When few query tiles exist the database is split across
// blocks and a second kernel merges the per-split top-k lists.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "bs_internal.cuh"

namespace bs {

constexpr int KC = 32;            // words per k-chunk (128 bytes of a row)
constexpr int BM = 32;            // query rows per block
constexpr int BN = 128;           // database rows per tile
constexpr int STAGES = 4;
constexpr int CONSUMERS = 256;    // 8 warps
constexpr int THREADS = CONSUMERS + 32;
constexpr int CAP = 256;          // candidate slots per query row
constexpr int A_TILE_BYTES = BM * KC * 4;
constexpr int B_TILE_BYTES = BN * KC * 4;
constexpr int STAGE_BYTES = A_TILE_BYTES + B_TILE_BYTES;
constexpr uint32_t NO_IDX = 0xFFFFFFFFu;

static_assert(STAGE_BYTES % 1024 == 0, "stages must keep 1024-byte alignment for the swizzle");
static_assert(BN <= CAP - BS_TOPK_K_MAX, "a full tile of candidates must fit after a merge");

enum { MODE_ESTIMATE = 0, MODE_TOPK = 1 };

struct PairArgs {
    const uint32_t *Q;      // [nQ][W]   (LDG producer path)
    const uint32_t *DB;     // [nDB][W]
    const uint32_t *pcQ;
    const uint32_t *pcDB;
    uint32_t nQ, nDB, N, W, nK;
    float invL;             // 1 / ln(1 - 1/N)
    // estimate mode
    uint32_t measures;      // bit mask
    float *out;
    uint32_t *counts;
    // top-k mode
    uint32_t k;
    int exclude_self;       // drop the pair q == self_off + c
    uint32_t self_off;
    uint32_t splits;        // database splits (grid.y)
    uint32_t tiles_per_split;
    float *score;           // final output (splits == 1)
    uint32_t *idx;
    float *ws_key;          // [splits][nQ][k] (splits > 1)
    uint32_t *ws_idx;
    unsigned int *err;
};

struct __align__(8) PairSmemHdr {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    int abort_flag;
};

// Bitonic sort (best first) of n = power of two entries by one warp.
__device__ void warp_sort_best_first(float *key, uint32_t *ix, int n, int lane) {
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < (n >> 1); t += 32) {
                const int i = 2 * t - (t & (stride - 1));
                const int j = i + stride;
                const bool up = (i & size) == 0;
                const float ki = key[i], kj = key[j];
                const uint32_t ii = ix[i], ij = ix[j];
                if (better(kj, ij, ki, ii) == up) {
                    key[i] = kj; key[j] = ki;
                    ix[i] = ij; ix[j] = ii;
                }
            }
            __syncwarp();
        }
    }
}

// Sort a candidate row and keep its best min(cnt, k); returns the new count.
__device__ int shrink_row(float *key, uint32_t *ix, int cnt, int k, int lane) {
    int n = 32;
    while (n < cnt) n <<= 1;
    for (int t = cnt + lane; t < n; t += 32) {
        key[t] = -INFINITY;
        ix[t] = NO_IDX;
    }
    __syncwarp();
    warp_sort_best_first(key, ix, n, lane);
    return cnt < k ? cnt : k;
}

// word (4-word group q of row r) inside a 128-byte-swizzled tile of 32-word rows
__device__ __forceinline__ const uint4 *swz(const uint32_t *tile, int r, int q) {
    return reinterpret_cast<const uint4 *>(tile + r * KC + (((q ^ (r & 7)) << 2)));
}

// Producer (LDG path, any N multiple of 32): one warp copies a tile with plain
// loads into the same swizzled layout TMA would produce.
__device__ __forceinline__ void ldg_fill(uint32_t *tile, const uint32_t *src, uint32_t n_src,
                                         int row0, int rows, int kc, uint32_t W, int lane) {
    const uint32_t w = (uint32_t)kc * KC + lane;
    for (int r0 = 0; r0 < rows; r0 += 8) {
        uint32_t v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int r = r0 + u;
            const uint32_t gr = (uint32_t)(row0 + r);
            v[u] = (r < rows && gr < n_src && w < W) ? __ldg(src + (size_t)gr * W + w) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int r = r0 + u;
            if (r < rows) tile[r * KC + ((((lane >> 2) ^ (r & 7)) << 2) | (lane & 3))] = v[u];
        }
    }
}

template <int MODE, int M, bool TMA>
__global__ void __launch_bounds__(THREADS, 1)
    pair_kernel(const __grid_constant__ CUtensorMap mapQ, const __grid_constant__ CUtensorMap mapDB,
                const PairArgs p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte aligned base for the swizzled tiles
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint32_t *tiles = reinterpret_cast<uint32_t *>(base);
    PairSmemHdr *hdr = reinterpret_cast<PairSmemHdr *>(base + STAGES * STAGE_BYTES);
    uint8_t *after_hdr = base + STAGES * STAGE_BYTES + sizeof(PairSmemHdr);
    // per-row data
    float *row_ln = reinterpret_cast<float *>(after_hdr);            // [BM]
    uint32_t *row_pc = reinterpret_cast<uint32_t *>(row_ln + BM);    // [BM]
    int *cand_cnt = reinterpret_cast<int *>(row_pc + BM);            // [BM]
    float *thr_key = reinterpret_cast<float *>(cand_cnt + BM);       // [BM]
    uint32_t *thr_idx = reinterpret_cast<uint32_t *>(thr_key + BM);  // [BM]
    float *cand_key = reinterpret_cast<float *>(thr_idx + BM);       // [BM][CAP]
    uint32_t *cand_idx = reinterpret_cast<uint32_t *>(cand_key + BM * CAP);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;

    const uint32_t row0 = blockIdx.x * BM;
    uint32_t tile_begin, tile_end;
    const uint32_t n_tiles_total = (p.nDB + BN - 1) / BN;
    if (MODE == MODE_TOPK) {
        tile_begin = blockIdx.y * p.tiles_per_split;
        tile_end = min(n_tiles_total, tile_begin + p.tiles_per_split);
        if (tile_begin > tile_end) tile_begin = tile_end;
    } else {
        tile_begin = blockIdx.y;
        tile_end = blockIdx.y + 1;
    }

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&hdr->full[s], TMA ? 1u : 32u);
            mbar_init(&hdr->empty[s], CONSUMERS / 32);
        }
        hdr->abort_flag = 0;
        fence_mbar_init();
    }
    if (tid < BM) {
        const uint32_t q = row0 + tid;
        const uint32_t a = q < p.nQ ? p.pcQ[q] : 0u;
        row_pc[tid] = a;
        row_ln[tid] = row_log(a, p.N);
        cand_cnt[tid] = 0;
        thr_key[tid] = -INFINITY;
        thr_idx[tid] = NO_IDX;
    }
    __syncthreads();

    volatile int *abort_flag = &hdr->abort_flag;

    if (warp == CONSUMERS / 32) {
        // ------------------------------ producer ------------------------------
        uint32_t it = 0;
        for (uint32_t t = tile_begin; t < tile_end; ++t) {
            for (uint32_t kc = 0; kc < p.nK; ++kc, ++it) {
                const uint32_t s = it % STAGES;
                const uint32_t use = it / STAGES;
                if (use > 0 && !*abort_flag) {
                    bool ok = true;
                    if (lane == 0) ok = mbar_wait(&hdr->empty[s], (use - 1) & 1u);
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) {
                        if (lane == 0) {
                            raise_error(p.err, BS_ERR_TIMEOUT);
                            *abort_flag = 1;
                        }
                    }
                }
                __syncwarp();
                if (*abort_flag) continue;
                uint32_t *tA = tiles + (size_t)s * (STAGE_BYTES / 4);
                uint32_t *tB = tA + A_TILE_BYTES / 4;
                if (TMA) {
                    if (lane == 0) {
                        mbar_arrive_expect_tx(&hdr->full[s], STAGE_BYTES);
                        tma_load_2d(tA, &mapQ, &hdr->full[s], (int)(kc * KC), (int)row0);
                        tma_load_2d(tB, &mapDB, &hdr->full[s], (int)(kc * KC), (int)(t * BN));
                    }
                } else {
                    ldg_fill(tA, p.Q, p.nQ, (int)row0, BM, (int)kc, p.W, lane);
                    ldg_fill(tB, p.DB, p.nDB, (int)(t * BN), BN, (int)kc, p.W, lane);
                    mbar_arrive(&hdr->full[s]);
                }
            }
        }
        // drain: make sure no copy into this block's shared memory is still in flight
        if (TMA && lane == 0 && it > 0) {
            const uint32_t first = it > (uint32_t)STAGES ? it - STAGES : 0u;
            for (uint32_t j = first; j < it; ++j) mbar_wait(&hdr->full[j % STAGES], (j / STAGES) & 1u);
        }
        return;
    }

    // ------------------------------- consumers --------------------------------
    const int ty = tid >> 4;   // 0..15
    const int tx = tid & 15;   // 0..15
    uint32_t it = 0;
    for (uint32_t t = tile_begin; t < tile_end; ++t) {
        uint32_t acc[2][8];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0u;

        for (uint32_t kc = 0; kc < p.nK; ++kc, ++it) {
            const uint32_t s = it % STAGES;
            if (!*abort_flag && !mbar_wait(&hdr->full[s], (it / STAGES) & 1u)) {
                raise_error(p.err, BS_ERR_TIMEOUT);
                *abort_flag = 1;
            }
            const uint32_t *tA = tiles + (size_t)s * (STAGE_BYTES / 4);
            const uint32_t *tB = tA + A_TILE_BYTES / 4;
#pragma unroll 2
            for (int q = 0; q < KC / 4; ++q) {
                uint4 a[2], b[8];
#pragma unroll
                for (int i = 0; i < 2; ++i) a[i] = *swz(tA, ty + 16 * i, q);
#pragma unroll
                for (int j = 0; j < 8; ++j) b[j] = *swz(tB, tx + 16 * j, q);
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        acc[i][j] += __popc(a[i].x & b[j].x) + __popc(a[i].y & b[j].y) +
                                     __popc(a[i].z & b[j].z) + __popc(a[i].w & b[j].w);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&hdr->empty[s]);
        }

        // ------------------------------ epilogue ------------------------------
        const uint32_t col0 = t * BN;
        if (MODE == MODE_ESTIMATE) {
            const size_t plane = (size_t)p.nQ * p.nDB;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = ty + 16 * i;
                const uint32_t q = row0 + r;
                if (q >= p.nQ) continue;
                const uint32_t a = row_pc[r];
                const float lnA = row_ln[r];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t c = col0 + tx + 16 * j;
                    if (c >= p.nDB) continue;
                    const size_t o = (size_t)q * p.nDB + c;
                    const uint32_t cnt = acc[i][j];
                    if (p.counts) p.counts[o] = cnt;
                    if (p.measures) {
                        const uint32_t b = __ldg(p.pcDB + c);
                        const float lnB = row_log(b, p.N);
                        float *dst = p.out + o;
                        if (p.measures & BS_IP) { *dst = estimate_one<M_IP>(a, b, cnt, p.N, lnA, lnB, p.invL); dst += plane; }
                        if (p.measures & BS_HAM) { *dst = estimate_one<M_HAM>(a, b, cnt, p.N, lnA, lnB, p.invL); dst += plane; }
                        if (p.measures & BS_JS) { *dst = estimate_one<M_JS>(a, b, cnt, p.N, lnA, lnB, p.invL); dst += plane; }
                        if (p.measures & BS_COS) { *dst = estimate_one<M_COS>(a, b, cnt, p.N, lnA, lnB, p.invL); }
                    }
                }
            }
        } else {
            uint32_t bcnt[8];
            float lnB[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t c = col0 + tx + 16 * j;
                bcnt[j] = c < p.nDB ? __ldg(p.pcDB + c) : 0u;
                lnB[j] = M == M_COS ? row_log(bcnt[j], p.N) : 0.0f;
            }
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = ty + 16 * i;
                const uint32_t q = row0 + r;
                if (q >= p.nQ) continue;
                const float tk = thr_key[r];
                const uint32_t ti = thr_idx[r];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint32_t c = col0 + tx + 16 * j;
                    if (c >= p.nDB || (p.exclude_self && (uint64_t)c + p.self_off == q)) continue;
                    const float key = rank_key<M>(row_pc[r], bcnt[j], acc[i][j], p.N, row_ln[r],
                                                  lnB[j], p.invL);
                    if (better(key, c, tk, ti)) {
                        const int slot = atomicAdd(&cand_cnt[r], 1);
                        if (slot < CAP) {   // always true: a shrink leaves room for a tile
                            cand_key[r * CAP + slot] = key;
                            cand_idx[r * CAP + slot] = c;
                        }
                    }
                }
            }
            named_sync(1, CONSUMERS);
            // shrink rows that could not take another full tile
            for (int r = warp; r < BM; r += CONSUMERS / 32) {
                const int cnt = cand_cnt[r];
                if (cnt > CAP - BN) {
                    const int kept = shrink_row(cand_key + r * CAP, cand_idx + r * CAP, cnt,
                                                (int)p.k, lane);
                    if (lane == 0) {
                        cand_cnt[r] = kept;
                        if (kept == (int)p.k) {
                            thr_key[r] = cand_key[r * CAP + kept - 1];
                            thr_idx[r] = cand_idx[r * CAP + kept - 1];
                        }
                    }
                }
                __syncwarp();
            }
            named_sync(1, CONSUMERS);
        }
    }

    if (MODE == MODE_TOPK) {
        for (int r = warp; r < BM; r += CONSUMERS / 32) {
            const uint32_t q = row0 + r;
            if (q >= p.nQ) continue;
            const int kept = shrink_row(cand_key + r * CAP, cand_idx + r * CAP, cand_cnt[r],
                                        (int)p.k, lane);
            for (int s = lane; s < (int)p.k; s += 32) {
                float kk = s < kept ? cand_key[r * CAP + s] : -INFINITY;
                uint32_t ii = s < kept ? cand_idx[r * CAP + s] : NO_IDX;
                if (p.splits == 1) {
                    const size_t o = (size_t)q * p.k + s;
                    p.score[o] = (M == M_HAM) ? -kk : kk;
                    p.idx[o] = ii;
                } else {
                    const size_t o = ((size_t)blockIdx.y * p.nQ + q) * p.k + s;
                    p.ws_key[o] = kk;
                    p.ws_idx[o] = ii;
                }
            }
            __syncwarp();
        }
    }
}

// Index offsets of the parts of a cross-shard merge (bs_topk_merge).
struct PartOffsets {
    uint32_t v[BS_TOPK_MERGE_PARTS_MAX];
};

// Merge the per-split top-k lists of each query row (one warp per row).
// Lists hold ranking keys (SCORES = false: split lists of one call) or output
// scores (SCORES = true: the final lists of database shards, whose indices
// are shifted by their shard's offset).
template <int M, bool SCORES>
__global__ void __launch_bounds__(256)
    merge_topk_kernel(const float *__restrict__ ws_key, const uint32_t *__restrict__ ws_idx,
                      uint32_t nQ, uint32_t k, uint32_t splits, float *__restrict__ score,
                      uint32_t *__restrict__ idx, const __grid_constant__ PartOffsets offs) {
    __shared__ float skey[8][CAP];
    __shared__ uint32_t sidx[8][CAP];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *key = skey[warp];
    uint32_t *ix = sidx[warp];
    for (uint32_t q = blockIdx.x * 8 + warp; q < nQ; q += gridDim.x * 8) {
        int cnt = 0;
        float tk = -INFINITY;
        uint32_t ti = NO_IDX;
        for (uint32_t s = 0; s < splits; ++s) {
            const size_t o = ((size_t)s * nQ + q) * k;
            for (uint32_t t0 = 0; t0 < k; t0 += 32) {
                const uint32_t t = t0 + lane;
                float kk = -INFINITY;
                uint32_t ii = NO_IDX;
                if (t < k) {
                    kk = ws_key[o + t];
                    ii = ws_idx[o + t];
                    if (SCORES) {
                        if (M == M_HAM) kk = -kk;
                        if (ii != NO_IDX) ii += offs.v[s];
                    }
                }
                const bool take = t < k && ii != NO_IDX && better(kk, ii, tk, ti);
                const uint32_t m = __ballot_sync(0xffffffffu, take);
                const int slot = cnt + __popc(m & ((1u << lane) - 1u));
                if (take && slot < CAP) {
                    key[slot] = kk;
                    ix[slot] = ii;
                }
                cnt += __popc(m);
            }
            __syncwarp();
            if (cnt > CAP - (int)k) {
                cnt = shrink_row(key, ix, cnt, (int)k, lane);
                if (cnt == (int)k) {
                    tk = key[k - 1];
                    ti = ix[k - 1];
                }
            }
        }
        const int kept = shrink_row(key, ix, cnt, (int)k, lane);
        for (uint32_t t = lane; t < k; t += 32) {
            const float kk = (int)t < kept ? key[t] : -INFINITY;
            score[(size_t)q * k + t] = (M == M_HAM) ? -kk : kk;
            idx[(size_t)q * k + t] = (int)t < kept ? ix[t] : NO_IDX;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static size_t pair_smem_bytes(int mode) {
    size_t b = 1024 /* alignment slack */ + (size_t)STAGES * STAGE_BYTES + sizeof(PairSmemHdr) +
               5 * BM * 4;
    if (mode == MODE_TOPK) b += (size_t)BM * CAP * 8;
    return b;
}

static bool make_map(CUtensorMap *m, const uint32_t *ptr, uint32_t rows, uint32_t W, int box_rows) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    cuuint64_t dims[2] = {W, rows};
    cuuint64_t strides[1] = {(cuuint64_t)W * 4};
    cuuint32_t box[2] = {KC, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, (void *)ptr, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool tma_ok(const uint32_t *A, const uint32_t *B, uint32_t N) {
    return (N % 128) == 0 && N >= 1024 && (reinterpret_cast<uintptr_t>(A) & 15u) == 0 &&
           (reinterpret_cast<uintptr_t>(B) & 15u) == 0;
}

template <int MODE, int M>
static bs_status launch_pairs(const PairArgs &p, dim3 grid, cudaStream_t stream) {
    CUtensorMap mq, md;
    memset(&mq, 0, sizeof(mq));
    memset(&md, 0, sizeof(md));
    bool use_tma = tma_ok(p.Q, p.DB, p.N);
    if (use_tma) {
        use_tma = make_map(&mq, p.Q, p.nQ, p.W, BM) && make_map(&md, p.DB, p.nDB, p.W, BN);
    }
    const size_t smem = pair_smem_bytes(MODE);
    if (use_tma) {
        auto kern = pair_kernel<MODE, M, true>;
        if (ensure_smem((const void *)kern, smem) != cudaSuccess) return BS_ERR_CUDA;
        kern<<<grid, THREADS, smem, stream>>>(mq, md, p);
    } else {
        auto kern = pair_kernel<MODE, M, false>;
        if (ensure_smem((const void *)kern, smem) != cudaSuccess) return BS_ERR_CUDA;
        kern<<<grid, THREADS, smem, stream>>>(mq, md, p);
    }
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

static bool valid_N(uint32_t N) { return N >= 32 && N <= BS_N_MAX && (N % 32) == 0; }

static float inv_ln_n(uint32_t N) { return (float)(1.0 / log1p(-1.0 / (double)N)); }

// database splits of the POPC top-k on this device
uint32_t popc_splits(uint32_t nQ, uint32_t nDB) {
    const uint32_t row_blocks = (nQ + BM - 1) / BM;
    const uint32_t tiles = (nDB + BN - 1) / BN;
    if (row_blocks == 0 || tiles == 0) return 1;
    const uint32_t target = 2u * (uint32_t)sm_count();
    uint32_t s = (target + row_blocks - 1) / row_blocks;
    // keep at least 4 tiles per split
    const uint32_t max_s = (tiles + 3) / 4;
    if (s > max_s) s = max_s;
    if (s < 1) s = 1;
    // make the split count match the per-split tile count exactly
    const uint32_t per = (tiles + s - 1) / s;
    return (tiles + per - 1) / per;
}

template <bool SCORES>
static bs_status merge_lists(int measure, const float *key, const uint32_t *ix, uint32_t nQ,
                             uint32_t k, uint32_t parts, float *score, uint32_t *idx,
                             const PartOffsets &offs, cudaStream_t st) {
    const uint32_t blocks = (nQ + 7) / 8;
    switch (measure) {
        case M_IP: merge_topk_kernel<M_IP, SCORES><<<blocks, 256, 0, st>>>(key, ix, nQ, k, parts, score, idx, offs); break;
        case M_HAM: merge_topk_kernel<M_HAM, SCORES><<<blocks, 256, 0, st>>>(key, ix, nQ, k, parts, score, idx, offs); break;
        case M_JS: merge_topk_kernel<M_JS, SCORES><<<blocks, 256, 0, st>>>(key, ix, nQ, k, parts, score, idx, offs); break;
        default: merge_topk_kernel<M_COS, SCORES><<<blocks, 256, 0, st>>>(key, ix, nQ, k, parts, score, idx, offs); break;
    }
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

bs_status launch_merge(int measure, const float *ws_key, const uint32_t *ws_idx, uint32_t nQ,
                       uint32_t k, uint32_t splits, float *score, uint32_t *idx, cudaStream_t st) {
    static const PartOffsets zero = {};
    return merge_lists<false>(measure, ws_key, ws_idx, nQ, k, splits, score, idx, zero, st);
}

bs_status topk_popc(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ, const uint32_t *DB,
                    const uint32_t *pcDB, uint32_t nDB, uint32_t N, int measure, uint32_t k,
                    int exclude_self, uint32_t self_off, float *score, uint32_t *idx, float *ws_key,
                    uint32_t *ws_idx, uint32_t splits, unsigned int *err, cudaStream_t st) {
    PairArgs p = {};
    p.Q = Q; p.DB = DB; p.pcQ = pcQ; p.pcDB = pcDB;
    p.nQ = nQ; p.nDB = nDB; p.N = N; p.W = N / 32; p.nK = (p.W + KC - 1) / KC;
    p.invL = inv_ln_n(N);
    p.k = k; p.exclude_self = exclude_self; p.self_off = self_off; p.err = err;
    p.score = score; p.idx = idx;
    const uint32_t tiles = (nDB + BN - 1) / BN;
    p.splits = splits;
    p.tiles_per_split = splits ? (tiles + splits - 1) / splits : 0;
    p.ws_key = ws_key;
    p.ws_idx = ws_idx;
    dim3 grid((nQ + BM - 1) / BM, splits);
    if (grid.y > 65535) return BS_ERR_UNSUPPORTED;
    switch (measure) {
        case M_IP: return launch_pairs<MODE_TOPK, M_IP>(p, grid, st);
        case M_HAM: return launch_pairs<MODE_TOPK, M_HAM>(p, grid, st);
        case M_JS: return launch_pairs<MODE_TOPK, M_JS>(p, grid, st);
        default: return launch_pairs<MODE_TOPK, M_COS>(p, grid, st);
    }
}

static int measure_code(uint32_t by) {
    switch (by) {
        case BS_IP: return M_IP;
        case BS_HAM: return M_HAM;
        case BS_JS: return M_JS;
        case BS_COS: return M_COS;
    }
    return -1;
}

static size_t ws_bytes(uint32_t splits, uint32_t nQ, uint32_t k) {
    return splits <= 1 ? 0 : (size_t)splits * nQ * k * (sizeof(float) + sizeof(uint32_t));
}

}  // namespace bs

using namespace bs;

// Kernel choice forced by the environment for calls that leave it to the
// library (BS_VARIANT_AUTO): BS_VARIANT=popc forces the CUDA-core kernel,
// BS_VARIANT=tc<c> (c = 0..9) picks tensor-core configuration c where the
// tensor-core kernel applies.  Read once.  Returns -2: not set, -1: POPC,
// c >= 0: configuration c.
static int env_variant() {
    static std::once_flag once;
    static int v = -2;
    std::call_once(once, [] {
        const char *e = getenv("BS_VARIANT");
        if (!e) return;
        if (!strcmp(e, "popc")) v = -1;
        else if (e[0] == 't' && e[1] == 'c' && e[2] >= '0' && e[2] <= '9') {
            int c = e[2] - '0';
            if (e[3] >= '0' && e[3] <= '9' && e[4] == 0) c = 10 * c + (e[3] - '0');
            else if (e[3] != 0) return;
            if (c < kTcConfigCount) v = c;
        }
    });
    return v;
}

extern "C" {

bs_status bs_estimate_pairs_ex(const uint32_t *A, const uint32_t *pcA, uint32_t nA, const uint32_t *B,
                               const uint32_t *pcB, uint32_t nB, uint32_t N, uint32_t measures,
                               float *out, uint32_t *counts, uint32_t variant, bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (!valid_N(N) || (measures & ~15u) || variant > BS_VARIANT_TC) return BS_ERR_INVALID_ARG;
    if (nA == 0 || nB == 0) return BS_OK;
    if (!A || !B || !pcA || !pcB) return BS_ERR_INVALID_ARG;
    if (measures && !out) return BS_ERR_INVALID_ARG;
    if (!measures && !counts) return BS_OK;
    unsigned int *err = error_word();
    if (!err) return BS_ERR_CUDA;
    if (variant == BS_VARIANT_AUTO && env_variant() == -1) variant = BS_VARIANT_POPC;
    const bool tc_ok = tc_store_supported(A, B, N);
    if (variant == BS_VARIANT_TC && !tc_ok) return BS_ERR_UNSUPPORTED;
    if (variant != BS_VARIANT_POPC && tc_ok)
        return estimate_tc(A, pcA, nA, B, pcB, nB, N, measures, out, counts, err, (cudaStream_t)stream);
    PairArgs p = {};
    p.Q = A; p.DB = B; p.pcQ = pcA; p.pcDB = pcB;
    p.nQ = nA; p.nDB = nB; p.N = N; p.W = N / 32; p.nK = (p.W + KC - 1) / KC;
    p.invL = inv_ln_n(N);
    p.measures = measures; p.out = out; p.counts = counts;
    p.splits = 1; p.err = err;
    dim3 grid((nA + BM - 1) / BM, (nB + BN - 1) / BN);
    if (grid.y > 65535) return BS_ERR_UNSUPPORTED;
    return launch_pairs<MODE_ESTIMATE, 0>(p, grid, (cudaStream_t)stream);
}

bs_status bs_estimate_pairs(const uint32_t *A, const uint32_t *pcA, uint32_t nA, const uint32_t *B,
                            const uint32_t *pcB, uint32_t nB, uint32_t N, uint32_t measures,
                            float *out, uint32_t *counts, bs_stream_t stream) {
    return bs_estimate_pairs_ex(A, pcA, nA, B, pcB, nB, N, measures, out, counts, BS_VARIANT_AUTO, stream);
}

// Workspace of one top-k call: the per-split lists (when the database is split
// across blocks) and, for the tensor-core kernel, the k-chunk-tiled copies of
// both operands; each part starts on a 256-byte boundary.
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// tensor-core call: [partial lists, every configuration's plan][Q copy][DB copy]
static size_t tc_workspace(uint32_t nQ, uint32_t nDB, uint32_t N, uint32_t k) {
    const size_t q = std::max(tc_tiled_bytes(nQ, N, kTcQueryRows), tc_fp4_bytes(nQ, N));
    const size_t db = std::max(tc_tiled_bytes(nDB, N, kTcTileRows), tc_fp4_bytes(nDB, N));
    return align256(tc_lists_bytes(nQ, nDB, k)) + align256(q) + align256(db);
}

size_t bs_topk_workspace_bytes(uint32_t nQ, uint32_t nDB, uint32_t N, uint32_t k) {
    if (nQ == 0 || nDB == 0 || k == 0) return 0;
    size_t need = ws_bytes(popc_splits(nQ, nDB), nQ, k);
    if (valid_N(N) && tc_shape_ok(N, k)) {
        const size_t t = tc_workspace(nQ, nDB, N, k);
        if (t > need) need = t;
    }
    return need;
}

static bs_status topk_impl(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ, const uint32_t *DB,
                           const uint32_t *pcDB, uint32_t nDB, uint32_t N, uint32_t by, uint32_t k,
                           int exclude_self, uint32_t self_off, float *score, uint32_t *idx,
                           void *workspace, size_t workspace_bytes, uint32_t variant,
                           cudaStream_t st) {
    if (!valid_N(N)) return BS_ERR_INVALID_ARG;
    if (k == 0 || k > BS_TOPK_K_MAX) return BS_ERR_INVALID_ARG;
    const int m = measure_code(by);
    const uint32_t inject = (variant & BS_VARIANT_INJECT_STALL) ? 1u : 0u;
    variant &= ~BS_VARIANT_INJECT_STALL;
    int tc_cfg = (int)((variant >> 4) & 15u) - 1;   // -1: default configuration
    if (variant >> 8) return BS_ERR_INVALID_ARG;
    variant &= 15u;
    if (m < 0 || variant > BS_VARIANT_TC || tc_cfg >= kTcConfigCount) return BS_ERR_INVALID_ARG;
    if (variant == BS_VARIANT_AUTO && tc_cfg < 0) {
        const int ev = env_variant();
        if (ev == -1) variant = BS_VARIANT_POPC;
        else if (ev >= 0 && tc_cfg_fits(ev, k)) tc_cfg = ev;
    }
    if (nQ == 0) return BS_OK;
    if (!Q || !pcQ || !score || !idx) return BS_ERR_INVALID_ARG;
    if (nDB > 0 && (!DB || !pcDB)) return BS_ERR_INVALID_ARG;
    unsigned int *err = error_word();
    if (!err) return BS_ERR_CUDA;

    bool use_tc = false;
    if (variant == BS_VARIANT_TC) {
        if (nDB == 0 || !tc_supported(Q, DB, N, k)) return BS_ERR_UNSUPPORTED;
        use_tc = true;
    } else if (variant == BS_VARIANT_AUTO) {
        use_tc = nDB > 0 && tc_supported(Q, DB, N, k);
    }
    if (inject && !use_tc) return BS_ERR_UNSUPPORTED;   // the injector lives in the tensor-core kernel
    if (use_tc) {   // the tensor-core call plans, launches and merges by itself
        const size_t lists = tc_lists_bytes(nQ, nDB, k);
        const size_t need = tc_workspace(nQ, nDB, N, k);
        if (!workspace || workspace_bytes < need) return BS_ERR_NO_MEMORY;
        if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return BS_ERR_INVALID_ARG;
        uint8_t *w = reinterpret_cast<uint8_t *>(workspace);
        return topk_tc(Q, pcQ, nQ, DB, pcDB, nDB, N, m, k, exclude_self, self_off, score, idx, w, lists,
                       w + align256(lists), nullptr, KEPT_NONE, tc_cfg, inject, err, st);
    }
    const uint32_t splits = popc_splits(nQ, nDB);
    const size_t need = ws_bytes(splits, nQ, k);
    float *ws_key = nullptr;
    uint32_t *ws_idx = nullptr;
    if (need > 0) {
        if (!workspace || workspace_bytes < need) return BS_ERR_NO_MEMORY;
        if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return BS_ERR_INVALID_ARG;
        ws_key = reinterpret_cast<float *>(workspace);
        ws_idx = reinterpret_cast<uint32_t *>(ws_key + (size_t)splits * nQ * k);
    }
    bs_status s1 = topk_popc(Q, pcQ, nQ, DB, pcDB, nDB, N, m, k, exclude_self, self_off, score, idx,
                             ws_key, ws_idx, splits, err, st);
    if (s1 != BS_OK || splits <= 1) return s1;
    return launch_merge(m, ws_key, ws_idx, nQ, k, splits, score, idx, st);
}

bs_status bs_topk_ex(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ, const uint32_t *DB,
                     const uint32_t *pcDB, uint32_t nDB, uint32_t N, uint32_t by, uint32_t k,
                     int exclude_self, float *score, uint32_t *idx, void *workspace,
                     size_t workspace_bytes, uint32_t variant, bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (exclude_self && nQ > nDB) return BS_ERR_INVALID_ARG;
    return topk_impl(Q, pcQ, nQ, DB, pcDB, nDB, N, by, k, exclude_self, 0, score, idx, workspace,
                     workspace_bytes, variant, (cudaStream_t)stream);
}

bs_status bs_topk_shard(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ, const uint32_t *DB,
                        const uint32_t *pcDB, uint32_t nDB, uint32_t db_offset, uint32_t N,
                        uint32_t by, uint32_t k, int exclude_self, float *score, uint32_t *idx,
                        void *workspace, size_t workspace_bytes, uint32_t variant,
                        bs_stream_t stream) {
    BS_NVTX_RANGE();
    if ((uint64_t)db_offset + nDB > 0xFFFFFFFFull) return BS_ERR_INVALID_ARG;
    return topk_impl(Q, pcQ, nQ, DB, pcDB, nDB, N, by, k, exclude_self, db_offset, score, idx,
                     workspace, workspace_bytes, variant, (cudaStream_t)stream);
}

bs_status bs_topk_merge(const float *score_parts, const uint32_t *idx_parts, uint32_t parts,
                        uint32_t nQ, uint32_t k, const uint32_t *part_offset, uint32_t by,
                        float *score, uint32_t *idx, bs_stream_t stream) {
    BS_NVTX_RANGE();
    const int m = measure_code(by);
    if (m < 0 || k == 0 || k > BS_TOPK_K_MAX) return BS_ERR_INVALID_ARG;
    if (parts == 0 || parts > BS_TOPK_MERGE_PARTS_MAX) return BS_ERR_INVALID_ARG;
    if (nQ == 0) return BS_OK;
    if (!score_parts || !idx_parts || !score || !idx) return BS_ERR_INVALID_ARG;
    PartOffsets offs = {};
    if (part_offset)
        for (uint32_t i = 0; i < parts; ++i) offs.v[i] = part_offset[i];
    return merge_lists<true>(m, score_parts, idx_parts, nQ, k, parts, score, idx, offs,
                             (cudaStream_t)stream);
}

bs_status bs_topk_plan(uint32_t nQ, uint32_t nDB, uint32_t N, uint32_t k, uint32_t variant,
                       int same_matrix, uint32_t *uses_tc, uint32_t *splits, uint32_t *launches) {
    variant &= 15u;
    if (!valid_N(N) || k == 0 || k > BS_TOPK_K_MAX || variant > BS_VARIANT_TC)
        return BS_ERR_INVALID_ARG;
    bool tc = false;
    if (variant == BS_VARIANT_AUTO && env_variant() == -1) variant = BS_VARIANT_POPC;
    if (variant == BS_VARIANT_TC) {
        if (nDB == 0 || !tc_shape_ok(N, k)) return BS_ERR_UNSUPPORTED;
        tc = true;
    } else if (variant == BS_VARIANT_AUTO) {
        tc = nDB > 0 && tc_shape_ok(N, k);
    }
    uint32_t s = 0, l = 0;
    if (nQ > 0 && tc) {   // the call plan of the default tensor-core configuration
        TcCallPlan pl;
        const int ev = variant == BS_VARIANT_AUTO ? env_variant() : -2;
        const bs_status ps = tc_call_plan(nQ, nDB, N, k, ev >= 0 && tc_cfg_fits(ev, k) ? ev : -1,
                                          same_matrix != 0, KEPT_NONE, pl);
        if (ps != BS_OK) return ps;
        s = pl.splits;
        l = pl.launches;
    } else if (nQ > 0) {
        s = popc_splits(nQ, nDB);
        l = 1 + (s > 1 ? 1 : 0);
    }
    if (uses_tc) *uses_tc = tc ? 1 : 0;
    if (splits) *splits = s;
    if (launches) *launches = l;
    return BS_OK;
}

size_t bs_tiled_bytes(uint32_t n, uint32_t N) {
    if (!valid_N(N) || (N % 128) != 0) return 0;
    return tc_tiled_bytes(n, N, kTcTileRows);
}

bs_status bs_tile_sketches(const uint32_t *sketch, uint32_t n_rows, uint32_t N, void *tiled,
                           bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (!valid_N(N) || (N % 128) != 0) return BS_ERR_INVALID_ARG;
    if (n_rows == 0) return BS_OK;
    if (!sketch || !tiled) return BS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(sketch) & 15u) || (reinterpret_cast<uintptr_t>(tiled) & 15u))
        return BS_ERR_INVALID_ARG;
    return tile_sketches(sketch, n_rows, N, kTcTileRows, tiled, (cudaStream_t)stream);
}

size_t bs_topk_pretiled_workspace_bytes(uint32_t nQ, uint32_t nDB, uint32_t N, uint32_t k) {
    if (nQ == 0 || nDB == 0 || !valid_N(N) || !tc_shape_ok(N, k)) return 0;
    return align256(tc_lists_bytes(nQ, nDB, k)) + align256(tc_tiled_bytes(nQ, N, kTcQueryRows));
}

bs_status bs_topk_pretiled(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ, const void *DB_tiled,
                           const uint32_t *pcDB, uint32_t nDB, uint32_t N, uint32_t by, uint32_t k,
                           float *score, uint32_t *idx, void *workspace, size_t workspace_bytes,
                           bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (!valid_N(N)) return BS_ERR_INVALID_ARG;
    if (k == 0 || k > BS_TOPK_K_MAX) return BS_ERR_INVALID_ARG;
    const int m = measure_code(by);
    if (m < 0) return BS_ERR_INVALID_ARG;
    if (nQ == 0) return BS_OK;
    if (!tc_shape_ok(N, k) || nDB == 0) return BS_ERR_UNSUPPORTED;
    if (!Q || !pcQ || !DB_tiled || !pcDB || !score || !idx) return BS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(Q) & 15u) || (reinterpret_cast<uintptr_t>(DB_tiled) & 15u))
        return BS_ERR_INVALID_ARG;
    unsigned int *err = error_word();
    if (!err) return BS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t lists = tc_lists_bytes(nQ, nDB, k);
    const size_t need = align256(lists) + align256(tc_tiled_bytes(nQ, N, kTcQueryRows));
    if (!workspace || workspace_bytes < need) return BS_ERR_NO_MEMORY;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return BS_ERR_INVALID_ARG;
    uint8_t *w = reinterpret_cast<uint8_t *>(workspace);
    return topk_tc(Q, pcQ, nQ, nullptr, pcDB, nDB, N, m, k, 0, 0, score, idx, w, lists, w + align256(lists),
                   DB_tiled, KEPT_TILED, -1, 0, err, st);
}

size_t bs_fp4_bytes(uint32_t n_rows, uint32_t N) {
    if (!valid_N(N) || (N % 128) != 0) return 0;
    return tc_fp4_bytes(n_rows, N);
}

bs_status bs_fp4_sketches(const uint32_t *sketch, uint32_t n_rows, uint32_t N, void *fp4, bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (!valid_N(N) || (N % 128) != 0) return BS_ERR_INVALID_ARG;
    if (n_rows == 0) return BS_OK;
    if (!sketch || !fp4) return BS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(sketch) & 15u) || (reinterpret_cast<uintptr_t>(fp4) & 15u))
        return BS_ERR_INVALID_ARG;
    return fp4_sketches(sketch, n_rows, N, fp4, (cudaStream_t)stream);
}

size_t bs_topk_prewidened_workspace_bytes(uint32_t nQ, uint32_t nDB, uint32_t N, uint32_t k) {
    if (nQ == 0 || nDB == 0 || !valid_N(N) || !tc_shape_ok(N, k)) return 0;
    const size_t q = std::max(tc_tiled_bytes(nQ, N, kTcQueryRows), tc_fp4_bytes(nQ, N));
    return align256(tc_lists_bytes(nQ, nDB, k)) + align256(q);
}

bs_status bs_topk_prewidened(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ, const void *DB_fp4,
                             const uint32_t *pcDB, uint32_t nDB, uint32_t N, uint32_t by, uint32_t k,
                             float *score, uint32_t *idx, void *workspace, size_t workspace_bytes,
                             bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (!valid_N(N)) return BS_ERR_INVALID_ARG;
    if (k == 0 || k > BS_TOPK_K_MAX) return BS_ERR_INVALID_ARG;
    const int m = measure_code(by);
    if (m < 0) return BS_ERR_INVALID_ARG;
    if (nQ == 0) return BS_OK;
    if (!tc_shape_ok(N, k) || nDB == 0) return BS_ERR_UNSUPPORTED;
    if (!Q || !pcQ || !DB_fp4 || !pcDB || !score || !idx) return BS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(Q) & 15u) || (reinterpret_cast<uintptr_t>(DB_fp4) & 15u))
        return BS_ERR_INVALID_ARG;
    unsigned int *err = error_word();
    if (!err) return BS_ERR_CUDA;
    const size_t lists = tc_lists_bytes(nQ, nDB, k);
    const size_t need = bs_topk_prewidened_workspace_bytes(nQ, nDB, N, k);
    if (!workspace || workspace_bytes < need) return BS_ERR_NO_MEMORY;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return BS_ERR_INVALID_ARG;
    uint8_t *w = reinterpret_cast<uint8_t *>(workspace);
    return topk_tc(Q, pcQ, nQ, nullptr, pcDB, nDB, N, m, k, 0, 0, score, idx, w, lists, w + align256(lists),
                   DB_fp4, KEPT_FP4, -1, 0, err, (cudaStream_t)stream);
}

size_t bs_topk_batched_workspace_bytes(const bs_topk_job *jobs, uint32_t n_jobs, uint32_t k) {
    if (!jobs || n_jobs == 0 || n_jobs > BS_TOPK_BATCH_MAX || k == 0 || k > BS_TOPK_K_MAX) return 0;
    return tc_batched_workspace(jobs, n_jobs, k);
}

bs_status bs_topk_batched_plan(const bs_topk_job *jobs, uint32_t n_jobs, uint32_t k, uint32_t *splits,
                               uint32_t *launches) {
    if (!jobs || n_jobs == 0 || n_jobs > BS_TOPK_BATCH_MAX) return BS_ERR_INVALID_ARG;
    if (k == 0 || k > BS_TOPK_K_MAX) return BS_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < n_jobs; ++i)
        if (!valid_N(jobs[i].N)) return BS_ERR_INVALID_ARG;
    uint32_t s = 1, nj = 0;
    const bs_status st = tc_batched_plan(jobs, n_jobs, k, &s, &nj);
    if (st != BS_OK) return st;
    if (splits) *splits = s;
    if (launches) *launches = nj == 0 ? 0 : 2;
    return BS_OK;
}

bs_status bs_topk_batched(const bs_topk_job *jobs, uint32_t n_jobs, uint32_t by, uint32_t k,
                          void *workspace, size_t workspace_bytes, uint32_t variant,
                          bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (!jobs || n_jobs == 0 || n_jobs > BS_TOPK_BATCH_MAX) return BS_ERR_INVALID_ARG;
    if (k == 0 || k > BS_TOPK_K_MAX) return BS_ERR_INVALID_ARG;
    const int m = measure_code(by);
    const int cfg = (int)((variant >> 4) & 15u) - 1;
    if (m < 0 || (variant >> 8) || cfg >= kTcConfigCount) return BS_ERR_INVALID_ARG;
    if ((variant & 15u) != BS_VARIANT_AUTO && (variant & 15u) != BS_VARIANT_TC) return BS_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < n_jobs; ++i)
        if (!valid_N(jobs[i].N)) return BS_ERR_INVALID_ARG;
    unsigned int *err = error_word();
    if (!err) return BS_ERR_CUDA;
    return topk_tc_batched(jobs, n_jobs, m, k, workspace, workspace_bytes, cfg, err, (cudaStream_t)stream);
}

bs_status bs_topk(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ, const uint32_t *DB,
                  const uint32_t *pcDB, uint32_t nDB, uint32_t N, uint32_t by, uint32_t k,
                  int exclude_self, float *score, uint32_t *idx, void *workspace,
                  size_t workspace_bytes, bs_stream_t stream) {
    return bs_topk_ex(Q, pcQ, nQ, DB, pcDB, nDB, N, by, k, exclude_self, score, idx, workspace,
                      workspace_bytes, BS_VARIANT_AUTO, stream);
}

}  // extern "C"
