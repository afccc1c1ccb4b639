/*
 * binsketch.h -- C ABI of the GB300 BinSketch library (libbinsketch.so).
 *
 * BinSketch (Pratap, Bera, Revanuru, arXiv 1910.04658) compresses a sparse
 * binary vector a in {0,1}^d into an N-bit vector a_s whose bit j is the OR
 * of the bits of a mapped to j by a random mapping pi : [d] -> [N]
 * (Definition "BinSketch", Sec. 3), and estimates inner product, Hamming
 * distance, Jaccard and cosine similarity of two vectors from the counts
 * |a_s|, |b_s| and <a_s, b_s> of their sketches (Alg. 1-4, Sec. 3.1-3.4).
 * Ranking (Experiment 2, Sec. 4) is offered as a per-query top-k.
 *
 * Conventions shared by every call
 *  - All array arguments are DEVICE pointers owned by the caller; the library
 *    allocates nothing on these paths and never frees caller memory.
 *  - Every call is asynchronous on `stream` (NULL = legacy default stream)
 *    and never synchronises.  Argument errors are reported immediately by the
 *    return value and nothing is launched.  Data errors found by the kernels
 *    (column index >= d, malformed row offsets) do not fault: the offending
 *    row is skipped (its sketch and count are written as zero) and a sticky
 *    per-device flag is raised; bs_get_async_error() reads and clears it.
 *  - Errors every call shares: BS_ERR_INVALID_ARG for a size parameter
 *    outside its documented range (N, k, d, thresholds), an unknown measure
 *    or variant, a NULL array that a non-zero count needs, or a pointer
 *    without the alignment the call states; BS_ERR_CUDA when a launch or a
 *    CUDA attribute call fails.  Kernels with bounded waits (tensor-core
 *    top-k, learned inference) raise BS_ERR_TIMEOUT through
 *    bs_get_async_error instead of hanging.  A call with a zero count (no
 *    rows, no queries) returns BS_OK after checking its size parameters,
 *    except bs_mlp_train_step (a step needs a batch).
 *  - Sketch layout: row r of a sketch matrix is N/32 consecutive uint32
 *    words; bucket j is bit (j & 31) of word (j >> 5) (LSB first).  Rows are
 *    contiguous (row stride N/32 words).
 *  - Column indices are 0-based (the paper counts from 1).
 *  - The mapping pi is a seeded multiply-add-shift hash (the paper only
 *    requires a random mapping): (mult, add) are the first two SplitMix64
 *    outputs of `seed` with mult forced odd;
 *    pi(i) = floor(N * hi32(mult * i + add mod 2^64) / 2^32).
 *    Sketches are comparable only when made with the same (seed, N).
 */
#ifndef BINSKETCH_H
#define BINSKETCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t / CUstream. */
typedef struct CUstream_st *bs_stream_t;

typedef enum {
    BS_OK = 0,
    BS_ERR_INVALID_ARG = 1,   /* NULL pointer, bad size or N, k out of range  */
    BS_ERR_INDEX_RANGE = 2,   /* (async) a column index was >= d              */
    BS_ERR_ROWPTR = 3,        /* (async) row offsets decrease or exceed nnz   */
    BS_ERR_CUDA = 4,          /* a CUDA runtime/driver call failed            */
    BS_ERR_NO_MEMORY = 5,     /* workspace too small                          */
    BS_ERR_TIMEOUT = 6,       /* a bounded device wait gave up                */
    BS_ERR_UNSUPPORTED = 7    /* valid request outside what is implemented    */
} bs_status;

/* Similarity measures (bit mask for bs_estimate_pairs, one value for bs_topk). */
enum { BS_IP = 1, BS_HAM = 2, BS_JS = 4, BS_COS = 8 };

/* Limits. */
enum { BS_N_MAX = 65536, BS_TOPK_K_MAX = 128 };

/*
 * bs_sketch -- sketch a CSR batch of binary vectors (Definition "BinSketch",
 * Sec. 3: a_s[j] = OR_{i : pi(i) = j} a[i]) and count |a_s| (Alg. 1 step 1).
 *
 *  row_ptr  uint64[n_rows + 1]  row r lists col[row_ptr[r] .. row_ptr[r+1])
 *  col      uint32[nnz]         column indices, < d; any order, repeats allowed
 *  n_rows   number of vectors (0 is a valid empty batch)
 *  nnz      number of entries of `col` (row_ptr[n_rows] must equal it)
 *  d        original dimension
 *  N        sketch length in bits: a multiple of 32, 32 <= N <= BS_N_MAX
 *  seed     selects the mapping pi (see above)
 *  sketch   uint32[n_rows][N/32] output
 *  popcnt   uint32[n_rows] output |a_s| (may be NULL)
 * Errors: BS_ERR_INVALID_ARG for NULL pointers (with n_rows > 0) or bad N;
 *         asynchronous BS_ERR_INDEX_RANGE / BS_ERR_ROWPTR for bad data.
 */
bs_status bs_sketch(const uint64_t *row_ptr, const uint32_t *col, uint32_t n_rows, uint64_t nnz,
                    uint32_t d, uint32_t N, uint64_t seed, uint32_t *sketch, uint32_t *popcnt,
                    bs_stream_t stream);

/*
 * bs_sketch_batched -- sketch many independent CSR datasets, each with its own
 * d, N and seed, in one persistent launch (one warp per row, grid-stride over
 * all rows of all jobs).  Results are identical to one bs_sketch per job.
 *  jobs    DEVICE array of n_jobs bs_sketch_job (all pointers device memory;
 *          popcnt may be NULL)
 *  max_N   upper bound of every job's N (sizes the per-warp shared buffer)
 * Errors: BS_ERR_INVALID_ARG for a bad max_N; bad jobs (N > max_N, N not a
 * multiple of 32, NULL arrays) and bad data are reported asynchronously.
 */
typedef struct {
    const uint64_t *row_ptr;   /* [n_rows + 1] */
    const uint32_t *col;       /* [nnz] */
    uint64_t nnz;
    uint64_t seed;
    uint32_t n_rows;
    uint32_t d;
    uint32_t N;
    uint32_t pad_;
    uint32_t *sketch;          /* [n_rows][N/32] out */
    uint32_t *popcnt;          /* [n_rows] out, may be NULL */
} bs_sketch_job;
bs_status bs_sketch_batched(const bs_sketch_job *jobs, uint32_t n_jobs, uint32_t max_N,
                            bs_stream_t stream);

/*
 * bs_sketch_parity -- the BCS sketch of the same batch (Definition "BCS",
 * Sec. 2): u_s[j] = sum_{i : pi(i) = j} u[i] mod 2, with the same mapping.
 * Arguments and errors as bs_sketch.  Rows must not repeat a column (a
 * repeat would cancel itself).
 */
bs_status bs_sketch_parity(const uint64_t *row_ptr, const uint32_t *col, uint32_t n_rows,
                           uint64_t nnz, uint32_t d, uint32_t N, uint64_t seed,
                           uint32_t *sketch, uint32_t *popcnt, bs_stream_t stream);

/*
 * bs_popcount_rows -- |a_s| of n_rows packed sketches (Alg. 1 step 1), for
 * callers that hold sketches without their counts.
 *  sketch uint32[n_rows][N/32] in, popcnt uint32[n_rows] out.
 */
bs_status bs_popcount_rows(const uint32_t *sketch, uint32_t n_rows, uint32_t N, uint32_t *popcnt,
                           bs_stream_t stream);

/*
 * bs_estimate_pairs -- every (A row i, B row j) pair: the common-bit count
 * n_{a_s,b_s} = <a_s, b_s> (Alg. 1 step 2) and the requested estimates in
 * FP32: IP (Alg. 1), Ham (Alg. 2, read as n_a + n_b - 2 n_{a,b}), JS (Alg. 3)
 * and Cos (Alg. 4).
 *
 *  A, B       uint32[nA][N/32], uint32[nB][N/32] sketches (same seed and N)
 *  pcA, pcB   uint32[nA], uint32[nB] their |a_s| (from bs_sketch or
 *             bs_popcount_rows)
 *  N          a multiple of 32, 32 <= N <= BS_N_MAX
 *  measures   OR of BS_IP | BS_HAM | BS_JS | BS_COS (0 allowed with counts)
 *  out        float[m][nA][nB], m = number of bits set in `measures`, planes
 *             in the order IP, HAM, JS, COS (may be NULL when measures = 0)
 *  counts     uint32[nA][nB] common-bit counts (may be NULL)
 * Saturated counts are clamped so that N - |a_s|, N - |b_s| and
 * N - |a_s OR b_s| are at least 1; Cos = 0 when an estimated size is 0 and
 * JS = 0 when the estimated union is 0.  Estimates are not clamped.
 * Errors: BS_ERR_INVALID_ARG for measure bits outside the four or out NULL
 * with measures != 0; BS_ERR_UNSUPPORTED for nB > 65535 * 128 rows (call
 * once per slice of B).
 */
bs_status bs_estimate_pairs(const uint32_t *A, const uint32_t *pcA, uint32_t nA,
                            const uint32_t *B, const uint32_t *pcB, uint32_t nB, uint32_t N,
                            uint32_t measures, float *out, uint32_t *counts, bs_stream_t stream);

/*
 * bs_estimate_pairs_ex -- bs_estimate_pairs with an explicit choice of the
 * pair-counting kernel (same results, bit for bit in the counts):
 *   BS_VARIANT_TC    the common-bit counts on the tensor cores (0/1 bits
 *                    widened to E2M1 elements of a block-scaled FP4 MMA with
 *                    unit scales, exact FP32 accumulation), reading the
 *                    row-major sketches directly: N % 128 == 0,
 *                    256 <= N <= 8192, 16-byte aligned A and B
 *                    (BS_ERR_UNSUPPORTED otherwise);
 *   BS_VARIANT_POPC  AND + population count on the CUDA cores, any N;
 *   BS_VARIANT_AUTO  the tensor cores where they apply, else POPC (what
 *                    bs_estimate_pairs does; BS_VARIANT=popc in the
 *                    environment forces POPC).
 */
bs_status bs_estimate_pairs_ex(const uint32_t *A, const uint32_t *pcA, uint32_t nA,
                               const uint32_t *B, const uint32_t *pcB, uint32_t nB, uint32_t N,
                               uint32_t measures, float *out, uint32_t *counts, uint32_t variant,
                               bs_stream_t stream);

/*
 * bs_topk_workspace_bytes -- device workspace bs_topk / bs_topk_ex need for
 * this shape, whichever kernel runs: partial top-k lists when a query row's
 * database is divided between blocks (the CUDA-core kernel splits the
 * database; the tensor-core kernel's persistent blocks cut some row blocks
 * in two), and for the tensor-core kernel k-chunk-tiled copies of Q (rows
 * rounded up to 128) and DB (rows rounded up to 208), N/8 bytes per row --
 * or, for the configurations that read them (c >= 10 below), the FP4
 * copies of Q and DB, N/2 bytes per row; plus partial lists for the plan of
 * every configuration.
 */
size_t bs_topk_workspace_bytes(uint32_t nQ, uint32_t nDB, uint32_t N, uint32_t k);

/*
 * bs_topk -- ranking (Experiment 2, Sec. 4) as a top-k: for every query row
 * q, the k DB rows with the best estimate `by` (one of BS_IP, BS_JS, BS_COS:
 * largest first; BS_HAM: smallest first), ties broken by smaller DB index.
 * The count/estimate matrix is never materialised.  The pair counts run on
 * the tensor cores where bs_topk_ex's BS_VARIANT_TC applies, else on the
 * CUDA cores (BS_VARIANT_POPC).
 *
 *  Q, pcQ       uint32[nQ][N/32] query sketches and their |a_s|
 *  DB, pcDB     uint32[nDB][N/32] database sketches and their |b_s|
 *  k            1 <= k <= BS_TOPK_K_MAX
 *  exclude_self non-zero: skip the pair (q, q) -- for all-pairs use with
 *               Q == DB (query row q is DB row q)
 *  score        float[nQ][k] estimates of the returned pairs, best first;
 *               unused slots (nDB < k) hold -inf (+inf for BS_HAM)
 *  idx          uint32[nQ][k] DB row of each slot; 0xFFFFFFFF when unused
 *  workspace    device memory of at least bs_topk_workspace_bytes(...)
 *               bytes, 256-byte aligned (may be NULL when that is 0);
 *               contents are scratch
 * Errors: BS_ERR_INVALID_ARG for k outside 1..BS_TOPK_K_MAX, `by` not one
 * measure, exclude_self with nQ > nDB, or a workspace not 256-byte aligned;
 * BS_ERR_NO_MEMORY when workspace_bytes is below what the shape needs.
 */
bs_status bs_topk(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ,
                  const uint32_t *DB, const uint32_t *pcDB, uint32_t nDB, uint32_t N,
                  uint32_t by, uint32_t k, int exclude_self, float *score, uint32_t *idx,
                  void *workspace, size_t workspace_bytes, bs_stream_t stream);

/*
 * bs_topk_ex -- bs_topk with an explicit choice of the pair-counting kernel.
 * The ranking and the results are the same; only the way <a_s, b_s> is
 * computed differs:
 *   BS_VARIANT_POPC  AND + population count on 32-bit words (CUDA cores),
 *                    any N and k;
 *   BS_VARIANT_TC    0/1 bits widened to 4-bit E2M1 elements (1.0 / 0) and
 *                    multiplied on the tensor cores (tcgen05.mma block-scaled
 *                    FP4 with unit scales, exact FP32 accumulation), for
 *                    N % 128 == 0, 256 <= N <= 8192 and 16-byte aligned Q
 *                    and DB; BS_ERR_UNSUPPORTED otherwise;
 *   BS_VARIANT_AUTO  the tensor-core kernel where it applies, else POPC
 *                    (this is what bs_topk does).
 * For the tensor-core kernel, BS_VARIANT_TC_CFG(c) OR-ed into `variant` picks
 * its block configuration c (an autotuner's knob): operand slots (widened
 * pieces of K of 256 or 128 sketch bits), epilogue groups, the depth of the
 * ring the bulk copies fill, and whether the two groups share one heap per
 * row:
 *   c = 0: 2 slots x 256 bits, 2 groups, ring 4
 *   c = 1: 2 slots x 256 bits, 2 groups, ring 4, shared heap
 *   c = 2: 4 slots x 128 bits, 2 groups, ring 8
 *   c = 3: 4 slots x 128 bits, 2 groups, ring 8, shared heap
 *   c = 4: 2 slots x 256 bits, 1 group,  ring 4
 *   c = 5: 2 slots x 256 bits, 2 groups, ring 6
 *   c = 6: 2 slots x 256 bits, 2 groups, ring 2
 *   c = 7: 2 slots x 256 bits, 2 groups, ring 6, shared heap
 *   c = 8: 2 slots x 256 bits, 1 group,  ring 2
 *   c = 9: 1 slot  x 256 bits, 1 group,  ring 2 (the smallest: every k up
 *          to BS_TOPK_K_MAX fits)
 *   c = 10: the database operand is not widened in the kernel: the call
 *          writes an FP4 copy of DB (N/2 bytes a row, in the workspace) and
 *          TMA moves each 256-bit slot of a tile from it into shared memory,
 *          3 database slots, 2 query slots, 2 groups
 *   c = 11: as c = 10 with 4 database slots and the shared heap
 *   c = 12: both operands from FP4 copies by TMA (the query block's too; for
 *          Q == DB one copy serves both), no widening warps, database tiles
 *          of 240 rows (208 for every other c), 3 stages, 3 epilogue groups
 *          sharing one heap per row
 *   c = 13: as c = 12 with 2 stages (every k up to BS_TOPK_K_MAX fits)
 *   c = 14: as c = 12 with 208-row tiles and 2 epilogue groups
 * The default, for bs_topk / bs_topk_ex / bs_topk_shard / bs_topk_noalloc,
 * is the first of 12, 13, 14, 10, 11 that fits k, else the first of 0, 1,
 * ..., 9 that fits; calls with a database kept tiled (bs_topk_pretiled) use
 * 0..9 only, a database kept as its FP4 copy (bs_topk_prewidened) 10..14
 * only, and the batched form the first of 12, 13, 14, 0, ..., 9 that fits
 * (c = 10, 11 there return BS_ERR_UNSUPPORTED).
 * With c >= 10 a call whose query rows fill R >= 1 rounds of one 128-row
 * block per SM runs those rounds as one launch (every SM sweeps the
 * database tiles in the same order, so the FP4 copy streams from L2) and
 * the rows left over as a second launch with partial lists; when the
 * database's FP4 copy is over 64 MiB that launch cuts each of its T row
 * blocks into the same min(SMs / T, tiles) parts of the database, one SM per
 * part, so the SMs holding the same part sweep it together.
 * Environment: for calls that pass BS_VARIANT_AUTO (bs_topk among them) the
 * variable BS_VARIANT, read once, overrides the choice: "popc" forces the
 * CUDA-core kernel, "tc<c>" (c = 0..14) selects configuration c wherever the
 * tensor-core kernel applies and c fits k.
 * A configuration whose shared memory does not fit k returns
 * BS_ERR_UNSUPPORTED.  bs_topk_workspace_bytes() covers every variant.
 *
 * BS_VARIANT_INJECT_STALL OR-ed into a tensor-core request is a fault
 * injector for testing failure detection, not for production: the kernel's
 * MMA-issuing thread skips announcing its first finished accumulator (as if
 * it had died), and every bounded wait of that launch gives up after about
 * 2e6 cycles instead of 4e9.  The waiting warps then raise BS_ERR_TIMEOUT
 * (read by bs_get_async_error), every role drains and exits, the kernel
 * frees its tensor memory, and the call's outputs are unspecified.  The GPU
 * context stays usable; the next call on the stream runs normally.
 */
enum { BS_VARIANT_AUTO = 0, BS_VARIANT_POPC = 1, BS_VARIANT_TC = 2 };
#define BS_VARIANT_TC_CFG(c) (((uint32_t)(c) + 1u) << 4)
#define BS_VARIANT_INJECT_STALL 0x100u
bs_status bs_topk_ex(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ,
                     const uint32_t *DB, const uint32_t *pcDB, uint32_t nDB, uint32_t N,
                     uint32_t by, uint32_t k, int exclude_self, float *score, uint32_t *idx,
                     void *workspace, size_t workspace_bytes, uint32_t variant,
                     bs_stream_t stream);

/*
 * bs_topk_batched -- bs_topk for many independent problems (datasets, each
 * with its own sketches, N, rows and self-exclusion; one measure `by` and one
 * k for all) in ONE persistent tensor-core launch.  The work items are the
 * row blocks of all problems (128 queries against the whole database of
 * their problem); the resident blocks claim them at run time from a counter
 * in the workspace, problems in decreasing cost of one row block, so the
 * largest items start first and small problems fill the tail.  A row block
 * is never split, so every list is written once and no merge runs.  The
 * ranking of every problem is that of bs_topk (Experiment 2, Sec. 4), index
 * for index and bit for bit.
 *  jobs        HOST array of n_jobs bs_topk_job (their pointers are device
 *              memory); 1 <= n_jobs <= BS_TOPK_BATCH_MAX.  Every job needs
 *              the tensor-core shape (N % 128 == 0, 256 <= N <= 8192, 16-byte
 *              aligned Q and DB); exclude_self requires Q == DB, nQ == nDB.
 *              A job with nQ == 0 is skipped; one with nDB == 0 and nQ > 0
 *              is refused, as bs_topk_ex refuses it for the tensor-core
 *              variant.
 *  variant     BS_VARIANT_AUTO or BS_VARIANT_TC, optionally with
 *              BS_VARIANT_TC_CFG(c): one block configuration for the launch
 *  workspace   device memory of at least bs_topk_batched_workspace_bytes()
 *              bytes, 256-byte aligned: the claim counter and, per job, its
 *              operand copies (tiled, or FP4 for c = 12..14)
 * Launches: one re-layout (or FP4 widening) kernel for all jobs (it also
 * zeroes the counter) and the persistent ranking kernel.  Calls that share a workspace must run
 * in order (one stream).
 * Errors: BS_ERR_INVALID_ARG for n_jobs outside 1..BS_TOPK_BATCH_MAX, a bad
 * measure or k, NULL arrays; BS_ERR_UNSUPPORTED for a job outside the
 * tensor-core shape or a configuration that does not fit k;
 * BS_ERR_NO_MEMORY for a short workspace.
 */
#define BS_TOPK_BATCH_MAX 64
typedef struct {
    const uint32_t *Q;      /* [nQ][N/32] query sketches */
    const uint32_t *pcQ;    /* [nQ] */
    const uint32_t *DB;     /* [nDB][N/32] database sketches */
    const uint32_t *pcDB;   /* [nDB] */
    float *score;           /* [nQ][k] out */
    uint32_t *idx;          /* [nQ][k] out */
    uint32_t nQ;
    uint32_t nDB;
    uint32_t N;
    int exclude_self;
} bs_topk_job;
size_t bs_topk_batched_workspace_bytes(const bs_topk_job *jobs, uint32_t n_jobs, uint32_t k);
bs_status bs_topk_batched(const bs_topk_job *jobs, uint32_t n_jobs, uint32_t by, uint32_t k,
                          void *workspace, size_t workspace_bytes, uint32_t variant,
                          bs_stream_t stream);
/* bs_topk_batched_plan -- host only: *splits = partial lists per query row
 * (always 1: row blocks are never split), *launches = kernels one bs_topk_batched
 * call launches (0 when every job is empty).  Errors as bs_topk_batched
 * returns them for this table and k; either output may be NULL. */
bs_status bs_topk_batched_plan(const bs_topk_job *jobs, uint32_t n_jobs, uint32_t k, uint32_t *splits,
                               uint32_t *launches);

/*
 * bs_topk_shard -- bs_topk_ex against one contiguous shard of a database that
 * is split across GPUs or calls (rows db_offset .. db_offset + nDB - 1 of
 * the whole database; the ranking of Experiment 2, Sec. 4, is unchanged).
 * DB/pcDB point at the shard's own rows.  The returned indices are LOCAL to
 * the shard (0 .. nDB-1); bs_topk_merge adds the shard offsets.
 *  exclude_self non-zero: skip the pairs with q == db_offset + j, i.e. query
 *               row q is row q of the whole database (all-pairs over a
 *               sharded corpus); nQ may exceed nDB
 * Everything else, including the workspace (bs_topk_workspace_bytes(nQ,
 * nDB, N, k)) and `variant`, is as for bs_topk_ex.
 * Errors: BS_ERR_INVALID_ARG when db_offset + nDB exceeds 2^32 - 1.
 */
bs_status bs_topk_shard(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ,
                        const uint32_t *DB, const uint32_t *pcDB, uint32_t nDB,
                        uint32_t db_offset, uint32_t N, uint32_t by, uint32_t k,
                        int exclude_self, float *score, uint32_t *idx, void *workspace,
                        size_t workspace_bytes, uint32_t variant, bs_stream_t stream);

/*
 * bs_topk_merge -- merge the top-k lists of `parts` database shards into the
 * top-k of the whole database: for every query row, the k best of all the
 * parts' entries in the order of bs_topk (score, then smaller global index).
 * Because each shard's list holds its k best, the result equals bs_topk over
 * the unsharded database, index for index and bit for bit.
 *  score_parts  float[parts][nQ][k], idx_parts uint32[parts][nQ][k]: the
 *               outputs of bs_topk_shard (device memory)
 *  part_offset  HOST uint32[parts]: global index of each part's row 0, added
 *               to its valid indices (NULL: all 0); unused slots (index
 *               0xFFFFFFFF) stay unused
 *  by           the measure the lists were ranked by
 *  score, idx   float[nQ][k], uint32[nQ][k] output (device; must not alias
 *               the inputs)
 * Errors: BS_ERR_INVALID_ARG for parts == 0 or parts > BS_TOPK_MERGE_PARTS_MAX.
 */
#define BS_TOPK_MERGE_PARTS_MAX 256
bs_status bs_topk_merge(const float *score_parts, const uint32_t *idx_parts, uint32_t parts,
                        uint32_t nQ, uint32_t k, const uint32_t *part_offset, uint32_t by,
                        float *score, uint32_t *idx, bs_stream_t stream);

/*
 * bs_topk_plan -- how bs_topk_ex would run this shape with its default
 * configuration, without running it: *uses_tc = 1 when the tensor-core
 * kernel is chosen, *splits = partial lists per query row of the launch that
 * uses them (a merge kernel runs when > 1; with the FP4 copies, the launch
 * over the rows left after the rounds), *launches = kernels launched per
 * call.  same_matrix != 0 when Q and DB will be the same array (the
 * tensor-core path then makes one FP4 copy instead of two).  Any output
 * pointer may be NULL.  Host only; Q/DB alignment is assumed to be 16 bytes.
 */
bs_status bs_topk_plan(uint32_t nQ, uint32_t nDB, uint32_t N, uint32_t k, uint32_t variant,
                       int same_matrix, uint32_t *uses_tc, uint32_t *splits, uint32_t *launches);

/*
 * bs_tiled_bytes / bs_tile_sketches -- keep a sketch database in the layout
 * the tensor-core kernel reads for its database operand, so repeated searches
 * against it skip the re-layout: row blocks of 208, each block's 16-byte
 * k-chunks contiguous ([block][k-chunk][208 rows] x 16 bytes), so one 256-bit
 * operand slot of a database tile is a single contiguous run for the
 * kernel's bulk copies.
 *  sketch  uint32[n_rows][N/32] in (16-byte aligned), N % 128 == 0
 *  tiled   bs_tiled_bytes(n_rows, N) bytes out (16-byte aligned); rows
 *          rounded up to 208 are zero.  Same paper content as the sketches.
 */
size_t bs_tiled_bytes(uint32_t n_rows, uint32_t N);
bs_status bs_tile_sketches(const uint32_t *sketch, uint32_t n_rows, uint32_t N, void *tiled,
                           bs_stream_t stream);

/*
 * bs_topk_pretiled -- bs_topk (tensor-core kernel) of nQ row-major query
 * sketches against a database kept tiled by bs_tile_sketches: the ranking of
 * Experiment 2 (Sec. 4) for a query stream against a resident corpus.
 * Requires N % 128 == 0, 256 <= N <= 8192 (BS_ERR_UNSUPPORTED
 * otherwise); no self-exclusion.  Workspace: bs_topk_pretiled_workspace_bytes.
 */
size_t bs_topk_pretiled_workspace_bytes(uint32_t nQ, uint32_t nDB, uint32_t N, uint32_t k);
bs_status bs_topk_pretiled(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ, const void *DB_tiled,
                           const uint32_t *pcDB, uint32_t nDB, uint32_t N, uint32_t by, uint32_t k,
                           float *score, uint32_t *idx, void *workspace, size_t workspace_bytes,
                           bs_stream_t stream);

/*
 * bs_fp4_bytes / bs_fp4_sketches -- keep a sketch database as the FP4 copy
 * the default tensor-core configurations read by TMA: every sketch bit one
 * 4-bit E2M1 element (set: 1.0, clear: 0), 32-bit word w written as the 16
 * bytes ((w << 1) & M, w & M, (w >> 1) & M, (w >> 2) & M), M = 0x22222222,
 * rows contiguous (N/2 bytes each, 4x the packed sketch).  Same paper
 * content as the sketches (Definition "BinSketch", Sec. 3).
 *  sketch  uint32[n_rows][N/32] in (16-byte aligned), N % 128 == 0
 *  fp4     bs_fp4_bytes(n_rows, N) bytes out (16-byte aligned)
 * Errors: BS_ERR_INVALID_ARG for N outside the tensor-core shapes, NULL or
 * misaligned pointers.  bs_fp4_bytes returns 0 for such N.
 */
size_t bs_fp4_bytes(uint32_t n_rows, uint32_t N);
bs_status bs_fp4_sketches(const uint32_t *sketch, uint32_t n_rows, uint32_t N, void *fp4,
                          bs_stream_t stream);

/*
 * bs_topk_prewidened -- bs_topk_pretiled against a database kept as its FP4
 * copy (bs_fp4_sketches): the default configuration order of bs_topk (both
 * operands by TMA; the queries' FP4 copy is made in the workspace), so a
 * resident corpus is searched with the fastest kernel and no per-call
 * database pass.  Same requirements, results and errors as
 * bs_topk_pretiled (the lists are identical, bit for bit); workspace:
 * bs_topk_prewidened_workspace_bytes.
 */
size_t bs_topk_prewidened_workspace_bytes(uint32_t nQ, uint32_t nDB, uint32_t N, uint32_t k);
bs_status bs_topk_prewidened(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ, const void *DB_fp4,
                             const uint32_t *pcDB, uint32_t nDB, uint32_t N, uint32_t by, uint32_t k,
                             float *score, uint32_t *idx, void *workspace, size_t workspace_bytes,
                             bs_stream_t stream);

/*
 * bs_topk_noalloc -- bs_topk for callers that may not allocate GPU memory
 * (a serving process whose arena owns the whole device, a plugin living in
 * another framework's allocator, a request path that must not pay for an
 * allocation).  The paper has no counterpart: this is a library service.
 * Same arguments, results and errors as bs_topk, minus the workspace: the
 * scratch bs_topk would need lives in a fixed device array of
 * BS_TOPK_NOALLOC_SCRATCH_BYTES inside the library, present on every GPU that
 * loads it until the process exits.  Shapes whose bs_topk_workspace_bytes()
 * exceeds that size are refused with BS_ERR_NO_MEMORY (nothing launched).
 * The array is reserved on a device when the library's module holding it is
 * first loaded there (CUDA loads device code lazily): at the first call made
 * while that device is current, which also looks up its address and may
 * synchronise.  Make that first call before the caller's own memory arena
 * takes the whole device and before any stream capture; if the reservation
 * fails the call returns BS_ERR_CUDA and leaves no CUDA error set for later
 * calls.  Calls share the array: calls whose
 * kernels overlap on the GPU race on it and must be serialised by the caller.
 * Allocates nothing.
 */
enum { BS_TOPK_NOALLOC_SCRATCH_BYTES = 16 << 20 };
bs_status bs_topk_noalloc(const uint32_t *Q, const uint32_t *pcQ, uint32_t nQ,
                          const uint32_t *DB, const uint32_t *pcDB, uint32_t nDB, uint32_t N,
                          uint32_t by, uint32_t k, int exclude_self, float *score, uint32_t *idx,
                          bs_stream_t stream);

/*
 * Learned estimator.  The paper estimates with the closed form of Alg. 1-4;
 * near saturation (|a_s| close to N) that inversion loses accuracy.  These
 * calls train and run a small MLP (4 -> 64 -> 64 -> 4, GELU in its tanh form, weights and
 * activations rounded to BF16, FP32 accumulation) on sketch pairs that
 * BinSketch itself produces, as an alternative estimator for that regime;
 * the closed form stays the reference.
 *
 * bs_dense_pairs -- n_pairs synthetic set pairs and their sketch counts.
 * Pair p draws |a|, |b| uniform in [size_lo, size_hi] and the overlap uniform
 * in [0, min(|a|, |b|)] from pair_seed, takes |a| + |b| - overlap distinct
 * columns of [0, d) from a keyed random permutation, and sketches both sets
 * with the mapping of hash_seed at length N (Definition "BinSketch").
 *  counts  uint32[n_pairs][3] out: |a_s|, |b_s|, <a_s, b_s>
 *  sizes   uint32[n_pairs][3] out (may be NULL): |a|, |b|, |a AND b| (exact)
 *  cols    uint32[n_pairs][max_cols] out (may be NULL): the columns in order
 *          (first the overlap, then a only, then b only), for checking
 * Errors: BS_ERR_INVALID_ARG unless 2 * size_hi <= d and N is valid.
 */
bs_status bs_dense_pairs(uint32_t n_pairs, uint32_t N, uint32_t d, uint32_t size_lo, uint32_t size_hi,
                         uint64_t pair_seed, uint64_t hash_seed, uint32_t *counts, uint32_t *sizes,
                         uint32_t *cols, uint32_t max_cols, bs_stream_t stream);

/* bs_estimate_counts -- closed-form IP, Ham, JS, Cos (Alg. 1-4, as in
 * bs_estimate_pairs) of n count triples counts[n][3]; out float[n][4]. */
bs_status bs_estimate_counts(const uint32_t *counts, uint32_t n, uint32_t N, float *out,
                             bs_stream_t stream);

/*
 * bs_onehot_csr -- categorical front end (Sec. 1, "Extension for
 * categorical data compression"): one-hot encoding of label-encoded rows into
 * the CSR layout bs_sketch reads.
 *  labels    uint32[n][F] (device): labels[i][f] in 0 .. m_f - 1
 *  offsets   uint32[F + 1] (device), non-decreasing: feature f owns columns
 *            offsets[f] .. offsets[f + 1] - 1 (m_f = offsets[f+1] - offsets[f]);
 *            the binary dimension is d = offsets[F]
 *  row_ptr   uint64[n + 1] out: row i starts at i * F
 *  col       uint32[n * F] out: col[i * F + f] = offsets[f] + labels[i][f]
 * The Hamming distance of two encoded rows is twice the number of features
 * on which they differ.  A label >= m_f is written as 0 and reported
 * (BS_ERR_INDEX_RANGE through bs_get_async_error).
 */
bs_status bs_onehot_csr(const uint32_t *labels, uint32_t n, uint32_t F, const uint32_t *offsets,
                        uint64_t *row_ptr, uint32_t *col, bs_stream_t stream);

/*
 * Ranking-quality evaluation (Experiment 2, Sec. 4 "Ranking"): the ground
 * truth of the uncompressed vectors and the retrieval sets at thresholds.
 *
 * bs_exact_counts -- exact |a AND b| for every pair (query row q, database row
 * j) of two CSR batches (same layout as bs_sketch's input):
 *  counts    uint32[nq][ndb] (device)
 *  q_sizes   uint32[nq] distinct indices of each query row (may be NULL)
 *  db_sizes  uint32[ndb] indices of each database row (may be NULL)
 * Database rows must not repeat an index (query rows may).  d <=
 * BS_EXACT_D_MAX: a query row is held as a d-bit bitmap in shared memory.
 * Indices >= d and malformed offsets are reported as by bs_sketch.
 */
#define BS_EXACT_D_MAX 1572864u
bs_status bs_exact_counts(const uint64_t *q_row_ptr, const uint32_t *q_col, uint32_t nq, uint64_t q_nnz,
                          const uint64_t *db_row_ptr, const uint32_t *db_col, uint32_t ndb,
                          uint64_t db_nnz, uint32_t d, uint32_t *counts, uint32_t *q_sizes,
                          uint32_t *db_sizes, bs_stream_t stream);

/*
 * bs_threshold_eval -- for every query row q and threshold thr[t] (host
 * array, 1 <= n_thresholds <= BS_EVAL_THRESHOLDS_MAX):
 *   out[q][t][0] = |O|      database rows whose exact similarity `by` is at
 *                           least thr[t] (BS_HAM: a distance at most thr[t])
 *   out[q][t][1] = |O'|     rows whose estimate est[q][j] passes the same test
 *   out[q][t][2] = |O n O'|
 * The exact similarity is formed in FP64 from counts / q_sizes / db_sizes
 * (IP = c, Ham = a + b - 2c, JS = c / (a + b - c) or 0 for an empty union,
 * Cos = c / sqrt(a b) or 0), the estimate is widened to FP64, and both are
 * compared with thr[t] in FP64.  est float[nq][ndb], counts uint32[nq][ndb]
 * (device), out uint32[nq][n_thresholds][3] (device).
 */
#define BS_EVAL_THRESHOLDS_MAX 16
bs_status bs_threshold_eval(const float *est, const uint32_t *counts, const uint32_t *q_sizes,
                            const uint32_t *db_sizes, uint32_t nq, uint32_t ndb, uint32_t by,
                            const double *thresholds, uint32_t n_thresholds, uint32_t *out,
                            bs_stream_t stream);

/* MLP parameters: BS_MLP_PARAMS floats laid out as W1[64][4], b1[64],
 * W2[64][64], b2[64], W3[4][64], b3[4].  The MLP refines the closed form:
 * inputs are the closed-form (n_a/4N, n_b/4N, IP/4N, log2(N)/16); outputs
 * are corrections added to the closed-form (IP/4N, Ham/8N, JS, Cos), so a
 * zero last layer reproduces Alg. 1-4 exactly. */
enum { BS_MLP_PARAMS = 4740 };

/* bs_mlp_prepare -- inputs x float[n][4] from counts[n][3], and (when sizes is
 * given) the training targets t float[n][4]: scaled exact similarities from
 * sizes[n][3] minus the scaled closed form. */
bs_status bs_mlp_prepare(const uint32_t *counts, const uint32_t *sizes, uint32_t n, uint32_t N, float *x,
                         float *t, bs_stream_t stream);

/* bs_mlp_train_step -- one Adam step (beta 0.9 / 0.999, eps 1e-8) on the mean
 * squared error of a batch: params, adam_m, adam_v, grad are float
 * [BS_MLP_PARAMS] (grad must start at zero and is left at zero); step counts
 * from 1; loss (may be NULL) receives the batch loss added to its value.
 * Errors: BS_ERR_INVALID_ARG for n = 0 or step = 0. */
bs_status bs_mlp_train_step(float *params, float *adam_m, float *adam_v, float *grad, uint32_t step,
                            float lr, const float *x, const float *t, uint32_t n, float *loss,
                            bs_stream_t stream);

/* bs_mlp_estimate -- the MLP's IP, Ham, JS, Cos of counts[n][3]; out float[n][4].
 * The 64 x 64 hidden layer runs on the tensor cores (tcgen05.mma kind::f16,
 * BF16 operands, FP32 accumulation); bs_mlp_estimate_ex with variant
 * BS_VARIANT_POPC runs every layer on the CUDA cores instead (same results up
 * to the order of FP32 sums), BS_VARIANT_AUTO / BS_VARIANT_TC the former. */
bs_status bs_mlp_estimate_ex(const float *params, const uint32_t *counts, uint32_t n, uint32_t N,
                             float *out, uint32_t variant, bs_stream_t stream);
bs_status bs_mlp_estimate(const float *params, const uint32_t *counts, uint32_t n, uint32_t N, float *out,
                          bs_stream_t stream);

/*
 * bs_get_async_error -- synchronise `stream`, return the first data error
 * raised by a kernel on the current device since the last call (BS_OK if
 * none) and clear it.  BS_ERR_CUDA if the synchronisation itself failed.
 */
bs_status bs_get_async_error(bs_stream_t stream);

/* Hash parameters (mult, add) that `seed` selects (host computation). */
void bs_hash_params(uint64_t seed, uint64_t *mult, uint64_t *add);

/* Human-readable name of a status. */
const char *bs_status_string(bs_status s);

/* Library version, major * 10000 + minor * 100 + patch. */
int bs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BINSKETCH_H */
