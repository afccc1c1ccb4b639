// Learned estimator for the saturated regime, and the data it is trained on.
//
// The closed form of Alg. 1-4 inverts E|a_s| = N (1 - (1 - 1/N)^|a|); as
// |a_s| approaches N that inversion loses precision (and is capped at N - 1).
// Here a small MLP learns a correction to the closed form from the
// closed-form estimates themselves.  It is trained on sketch pairs that
// BinSketch itself produces:
//
//  * bs_dense_pairs: one warp per pair draws |a|, |b| uniform in [lo, hi] and
//    the overlap uniform in [0, min(|a|, |b|)], takes |a| + |b| - overlap
//    distinct columns of [0, d) from a keyed random permutation (a 4-round
//    Feistel network on 2^m >= d values with cycle walking), gives the first
//    `overlap` to both sets, then sketches both sets with the seeded mapping
//    (Definition "BinSketch") and counts |a_s|, |b_s|, <a_s, b_s>.  The exact
//    sizes -- and so the exact IP, Ham, JS, Cos -- are known by construction.
//  * bs_mlp_*: a 4 -> 64 -> 64 -> 4 MLP that corrects the closed form (its
//    inputs are the closed-form n_a, n_b and IP, its outputs are added to the
//    closed-form estimates), with GELU (tanh form), weights and activations
//    rounded to BF16, products accumulated in FP32; a fused training step
//    (forward and backward of 128 samples per block in shared memory, block
//    gradient sums added to a global buffer) followed by Adam on FP32 master
//    weights; and a fused inference kernel that goes from counts to the four
//    estimates.
#include <cuda_bf16.h>
#include <math.h>

#include "bs_internal.cuh"

namespace bs {
namespace mlp {

constexpr int IN = 4, H = 64, OUT = 4;
// parameter layout (floats): W1[H][IN], b1[H], W2[H][H], b2[H], W3[OUT][H], b3[OUT]
constexpr int OW1 = 0, OB1 = OW1 + H * IN, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H,
              OB3 = OW3 + OUT * H, NPARAM = OB3 + OUT;
static_assert(NPARAM == BS_MLP_PARAMS, "parameter count");
constexpr int TB = 128;   // samples (threads) per training block

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
// GELU in the tanh form of Hendrycks and Gimpel (2016):
//   gelu(z) = z/2 (1 + tanh(u)),  u = sqrt(2/pi) (z + 0.044715 z^3)
constexpr float kGeluC = 0.7978845608f;   // sqrt(2 / pi)
constexpr float kGeluA = 0.044715f;
__device__ __forceinline__ float gelu(float z) {
    const float u = kGeluC * fmaf(kGeluA * z * z, z, z);
    return 0.5f * z * (1.0f + tanhf(u));
}
// d gelu / dz = (1 + t)/2 + z/2 (1 - t^2) sqrt(2/pi) (1 + 3 a z^2),  t = tanh(u)
__device__ __forceinline__ float gelu_grad(float z) {
    const float u = kGeluC * fmaf(kGeluA * z * z, z, z);
    const float t = tanhf(u);
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * kGeluC * fmaf(3.0f * kGeluA, z * z, 1.0f);
}
// the same with the hardware tanh approximation (tanh.approx.f32); its
// error is far below the BF16 rounding every activation gets
__device__ __forceinline__ float gelu_fast(float z) {
    const float u = kGeluC * fmaf(kGeluA * z * z, z, z);
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
    return 0.5f * z * (1.0f + t);
}

// target scaling: IP / 4N, Ham / 8N, JS, Cos
__device__ __forceinline__ float out_scale(int o, uint32_t N) {
    return o == 0 ? 4.0f * N : (o == 1 ? 8.0f * N : 1.0f);
}

// The MLP refines the closed form: its inputs are the closed-form set sizes
// and inner product (n_a / 4N, n_b / 4N, IP / 4N, log2(N) / 16), and its
// outputs are corrections added to the scaled closed-form estimates (`base`).
__device__ __forceinline__ void features(uint32_t a, uint32_t b, uint32_t c, uint32_t N, float x[IN],
                                         float base[OUT]) {
    const float fN = (float)N;
    const float invL = 1.0f / log1pf(-1.0f / fN);
    const float lnA = row_log(a, N), lnB = row_log(b, N);
    const float ip = estimate_one<M_IP>(a, b, c, N, lnA, lnB, invL);
    x[0] = lnA * invL / (4.0f * fN);
    x[1] = lnB * invL / (4.0f * fN);
    x[2] = ip / (4.0f * fN);
    x[3] = log2f(fN) * (1.0f / 16.0f);
    base[0] = ip / out_scale(0, N);
    base[1] = estimate_one<M_HAM>(a, b, c, N, lnA, lnB, invL) / out_scale(1, N);
    base[2] = estimate_one<M_JS>(a, b, c, N, lnA, lnB, invL);
    base[3] = estimate_one<M_COS>(a, b, c, N, lnA, lnB, invL);
}

// ---------------------------------------------------------------------------
// training step: forward + backward of TB samples per block
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TB)
    train_grad_kernel(const float *__restrict__ params, const float *__restrict__ x,
                      const float *__restrict__ t, uint32_t n, float *__restrict__ grad,
                      float *__restrict__ loss) {
    // shared memory (dynamic): weights, then per-sample columns of
    // pre-activations / activations / deltas, one column per thread
    extern __shared__ float smf[];
    float *W = smf;
    float(*z1)[TB + 1] = reinterpret_cast<float(*)[TB + 1]>(smf + NPARAM);
    float(*z2)[TB + 1] = z1 + H;
    float(*d2)[TB + 1] = z2 + H;
    float(*xs)[TB] = reinterpret_cast<float(*)[TB]>(d2 + H);
    const int tid = threadIdx.x;
    for (int i = tid; i < NPARAM; i += TB) W[i] = bf(params[i]);
    const uint32_t s = blockIdx.x * TB + tid;
    const bool live = s < n;
    float xi[IN], ti[OUT];
#pragma unroll
    for (int i = 0; i < IN; ++i) {
        xi[i] = live ? bf(x[(size_t)s * IN + i]) : 0.f;
        xs[i][tid] = xi[i];
    }
#pragma unroll
    for (int o = 0; o < OUT; ++o) ti[o] = live ? t[(size_t)s * OUT + o] : 0.f;
    __syncthreads();
    // layer 1
    for (int m = 0; m < H; ++m) {
        float acc = W[OB1 + m];
#pragma unroll
        for (int i = 0; i < IN; ++i) acc = fmaf(W[OW1 + m * IN + i], xi[i], acc);
        z1[m][tid] = acc;
    }
    // layer 2
    for (int m = 0; m < H; ++m) {
        float acc = W[OB2 + m];
        for (int k = 0; k < H; ++k) acc = fmaf(W[OW2 + m * H + k], bf(gelu(z1[k][tid])), acc);
        z2[m][tid] = acc;
    }
    // layer 3 and the loss gradient (mean over samples and outputs)
    float dy[OUT], l = 0.f;
#pragma unroll
    for (int o = 0; o < OUT; ++o) {
        float acc = W[OB3 + o];
        for (int k = 0; k < H; ++k) acc = fmaf(W[OW3 + o * H + k], bf(gelu(z2[k][tid])), acc);
        const float e = live ? acc - ti[o] : 0.f;
        l += e * e;
        dy[o] = 2.0f * e / ((float)n * OUT);
    }
    // backward through layer 3 into z2 (kept separate from z2 until used)
    float dh2[H];
#pragma unroll 8
    for (int k = 0; k < H; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int o = 0; o < OUT; ++o) acc = fmaf(W[OW3 + o * H + k], dy[o], acc);
        dh2[k] = acc * gelu_grad(z2[k][tid]);
    }
    __syncthreads();
    // dz1 = W2^T dh2 * gelu'(z1); keep h2 in z2 for the W3 / W2 sums
    float dz1[H];
#pragma unroll 8
    for (int k = 0; k < H; ++k) {
        float acc = 0.f;
        for (int m = 0; m < H; ++m) acc = fmaf(W[OW2 + m * H + k], dh2[m], acc);
        dz1[k] = acc * gelu_grad(z1[k][tid]);
    }
    __syncthreads();
    // overwrite: z2 <- h2 (bf16), z1 <- h1 (bf16) for the weight sums; keep the
    // deltas in d2
    for (int k = 0; k < H; ++k) {
        d2[k][tid] = dh2[k];
        z2[k][tid] = bf(gelu(z2[k][tid]));
    }
    __syncthreads();
    // the W2 sums need h1; dy goes to d2 once those are done (below)
    for (int k = 0; k < H; ++k) {
        const float h1 = bf(gelu(z1[k][tid]));
        z1[k][tid] = h1;
    }
    __syncthreads();
    // W2 and b2: thread pairs (m, k) over the block's samples
    for (int e = tid; e < H * H; e += TB) {
        const int m = e / H, k = e % H;
        float acc = 0.f;
        for (int q = 0; q < TB; ++q) acc = fmaf(d2[m][q], z1[k][q], acc);
        atomicAdd(&grad[OW2 + e], acc);
    }
    if (tid < H) {
        float acc = 0.f;
        for (int q = 0; q < TB; ++q) acc += d2[tid][q];
        atomicAdd(&grad[OB2 + tid], acc);
    }
    __syncthreads();
    // now z1 can hold dz1 (W1 sums) and d2 can hold dy (W3 sums)
    for (int k = 0; k < H; ++k) z1[k][tid] = dz1[k];
#pragma unroll
    for (int o = 0; o < OUT; ++o) d2[o][tid] = dy[o];
    __syncthreads();
    for (int e = tid; e < H * IN; e += TB) {
        const int m = e / IN, i = e % IN;
        float acc = 0.f;
        for (int q = 0; q < TB; ++q) acc = fmaf(z1[m][q], xs[i][q], acc);
        atomicAdd(&grad[OW1 + e], acc);
    }
    if (tid < H) {
        float acc = 0.f;
        for (int q = 0; q < TB; ++q) acc += z1[tid][q];
        atomicAdd(&grad[OB1 + tid], acc);
    }
    for (int e = tid; e < OUT * H; e += TB) {
        const int o = e / H, k = e % H;
        float acc = 0.f;
        for (int q = 0; q < TB; ++q) acc = fmaf(d2[o][q], z2[k][q], acc);
        atomicAdd(&grad[OW3 + e], acc);
    }
    if (tid < OUT) {
        float acc = 0.f;
        for (int q = 0; q < TB; ++q) acc += d2[tid][q];
        atomicAdd(&grad[OB3 + tid], acc);
    }
    // loss sum
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((tid & 31) == 0 && loss) atomicAdd(loss, l / ((float)n * OUT));
}

constexpr size_t train_smem_bytes() {
    return sizeof(float) * ((size_t)NPARAM + 3 * (size_t)H * (TB + 1) + (size_t)IN * TB);
}

__global__ void adam_kernel(float *__restrict__ params, float *__restrict__ m, float *__restrict__ v,
                            float *__restrict__ grad, float lr, float b1c, float b2c) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float g = grad[i];
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / b1c) / (sqrtf(vi / b2c) + 1e-8f);
    grad[i] = 0.f;
}

// counts -> estimates through the MLP (weights rounded to BF16 once per block)
__global__ void __launch_bounds__(256)
    infer_kernel(const float *__restrict__ params, const uint32_t *__restrict__ counts, uint32_t n,
                 uint32_t N, float *__restrict__ out) {
    __shared__ float W[NPARAM];
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) W[i] = bf(params[i]);
    __syncthreads();
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[IN], base[OUT];
    features(counts[3 * s], counts[3 * s + 1], counts[3 * s + 2], N, x, base);
#pragma unroll
    for (int i = 0; i < IN; ++i) x[i] = bf(x[i]);
    float h1[H];
#pragma unroll
    for (int m = 0; m < H; ++m) {
        float acc = W[OB1 + m];
#pragma unroll
        for (int i = 0; i < IN; ++i) acc = fmaf(W[OW1 + m * IN + i], x[i], acc);
        h1[m] = bf(gelu(acc));
    }
    float y[OUT];
#pragma unroll
    for (int o = 0; o < OUT; ++o) y[o] = W[OB3 + o];
    for (int m = 0; m < H; ++m) {
        float acc = W[OB2 + m];
#pragma unroll
        for (int k = 0; k < H; ++k) acc = fmaf(W[OW2 + m * H + k], h1[k], acc);
        const float h2 = bf(gelu(acc));
#pragma unroll
        for (int o = 0; o < OUT; ++o) y[o] = fmaf(W[OW3 + o * H + m], h2, y[o]);
    }
#pragma unroll
    for (int o = 0; o < OUT; ++o) out[(size_t)s * OUT + o] = (base[o] + y[o]) * out_scale(o, N);
}

// ---------------------------------------------------------------------------
// inference with the 64 x 64 hidden layer on the tensor cores
// ---------------------------------------------------------------------------
// A tile of 128 samples per block: each thread computes its sample's first
// layer on the CUDA cores and stores GELU(h1) rounded to BF16 as row `tid` of
// the A operand (K-major, 128-byte swizzle: one 128-byte row of 64 BF16 per
// sample); W2 (BF16, rows = output neurons, K-major) is the B operand, loaded
// once per block.  One thread issues 4 x tcgen05.mma.kind::f16 (M = 128,
// N = 64, K = 16, BF16 x BF16 -> FP32) into 64 TMEM columns; every thread
// then reads its own row (TMEM lane = sample) and finishes b2, GELU and the
// 64 -> 4 output layer on the CUDA cores.  Same arithmetic as infer_kernel up
// to the order of the FP32 sums.
namespace tcm {
constexpr int ROWS = 128;                    // samples per tile (MMA M, TMEM lanes)
constexpr int A_BYTES = ROWS * 128;          // 16 KB
constexpr int B_BYTES = H * 128;             // 8 KB
// D = F32, A = B = BF16, both K-major, N = 64, M = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(H >> 3) << 17) |
                           ((uint32_t)(ROWS >> 4) << 24);
// dynamic shared memory: A, B, small weights, barrier; sized so that at most
// 7 blocks share an SM (7 x 64 TMEM columns <= 512)
constexpr int SMEM_BYTES = 30 * 1024;

__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                 // LBO (ignored for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // SBO: 8-row groups 1024 bytes apart
    d |= (uint64_t)1 << 46;                 // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
    return d;
}
__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}
// 64 values -> one 128-byte swizzled K-major row r (16-byte chunk c at c ^ (r % 8))
__device__ __forceinline__ void store_row_bf16(uint8_t *tile, int r, const float (&v)[H]) {
    uint8_t *row = tile + (r >> 3) * 1024 + (r & 7) * 128;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        uint4 q;
        q.x = pack_bf2(v[8 * c + 0], v[8 * c + 1]);
        q.y = pack_bf2(v[8 * c + 2], v[8 * c + 3]);
        q.z = pack_bf2(v[8 * c + 4], v[8 * c + 5]);
        q.w = pack_bf2(v[8 * c + 6], v[8 * c + 7]);
        *reinterpret_cast<uint4 *>(row + ((c ^ (r & 7)) << 4)) = q;
    }
}
__device__ __forceinline__ void ld32(uint32_t taddr, uint32_t (&r)[32]) {
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
}  // namespace tcm

__global__ void __launch_bounds__(tcm::ROWS)
    infer_tc_kernel(const float *__restrict__ params, const uint32_t *__restrict__ counts, uint32_t n,
                    uint32_t N, float *__restrict__ out, unsigned int *err) {
    using namespace tcm;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *At = base;
    uint8_t *Bt = base + A_BYTES;
    float *Ws = reinterpret_cast<float *>(Bt + B_BYTES);   // W1, b1, b2, W3, b3 (BF16-rounded)
    float *W1s = Ws, *b1s = W1s + H * IN, *b2s = b1s + H, *W3s = b2s + H, *b3s = W3s + OUT * H;
    uint64_t *bar = reinterpret_cast<uint64_t *>(b3s + 4);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;

    // weights: the small layers as FP32 (BF16-rounded), W2 as the BF16 B operand
    for (int i = tid; i < H * IN; i += ROWS) W1s[i] = bf(params[OW1 + i]);
    for (int i = tid; i < H; i += ROWS) {
        b1s[i] = bf(params[OB1 + i]);
        b2s[i] = bf(params[OB2 + i]);
    }
    for (int i = tid; i < OUT * H; i += ROWS) W3s[i] = bf(params[OW3 + i]);
    if (tid < OUT) b3s[tid] = bf(params[OB3 + tid]);
    if (tid < H) {   // row tid of B = output neuron tid's 64 input weights
        float w[H];
#pragma unroll
        for (int k = 0; k < H; ++k) w[k] = params[OW2 + tid * H + k];
        store_row_bf16(Bt, tid, w);
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(64u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t n_tiles = (n + ROWS - 1) / ROWS;
    bool ok = true;
    uint32_t phase = 0;
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, phase ^= 1u) {
        const uint32_t s = tile * ROWS + tid;
        float x[IN] = {0.f, 0.f, 0.f, 0.f}, bsv[OUT] = {0.f, 0.f, 0.f, 0.f};
        if (s < n) features(counts[3 * s], counts[3 * s + 1], counts[3 * s + 2], N, x, bsv);
        float h1[H];
#pragma unroll
        for (int m = 0; m < H; ++m) {
            float acc = b1s[m];
#pragma unroll
            for (int i = 0; i < IN; ++i) acc = fmaf(W1s[m * IN + i], bf(x[i]), acc);
            h1[m] = (s < n) ? gelu_fast(acc) : 0.0f;   // rounded to BF16 by the store
        }
        store_row_bf16(At, tid, h1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0 && ok) {
            const uint32_t a = smem_u32(At), b = smem_u32(Bt);
#pragma unroll
            for (int kk = 0; kk < H / 16; ++kk) {
                const uint64_t ad = sw128_desc(a + kk * 32), bd = sw128_desc(b + kk * 32);
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(IDESC), "r"((uint32_t)kk)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(bar))
                         : "memory");
        }
        if (ok && !mbar_wait(bar, phase)) {
            ok = false;
            raise_error(err, BS_ERR_TIMEOUT);
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t r0[32], r1[32];
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        ld32(trow, r0);
        ld32(trow + 32, r1);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float y[OUT];
#pragma unroll
        for (int o = 0; o < OUT; ++o) y[o] = b3s[o];
#pragma unroll
        for (int m = 0; m < H; ++m) {
            const float acc = __uint_as_float(m < 32 ? r0[m] : r1[m - 32]) + b2s[m];
            const float h2 = bf(gelu_fast(acc));
#pragma unroll
            for (int o = 0; o < OUT; ++o) y[o] = fmaf(W3s[o * H + m], h2, y[o]);
        }
        if (s < n && ok) {
#pragma unroll
            for (int o = 0; o < OUT; ++o) out[(size_t)s * OUT + o] = (bsv[o] + y[o]) * out_scale(o, N);
        }
        // every thread has read its accumulator row and is done with A before
        // the next tile overwrites them
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64u) : "memory");
}

// features x[n][4] and scaled targets t[n][4] from counts and exact sizes
__global__ void prepare_kernel(const uint32_t *__restrict__ counts, const uint32_t *__restrict__ sizes,
                               uint32_t n, uint32_t N, float *__restrict__ x, float *__restrict__ t) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float f[IN], base[OUT];
    features(counts[3 * s], counts[3 * s + 1], counts[3 * s + 2], N, f, base);
#pragma unroll
    for (int i = 0; i < IN; ++i) x[(size_t)s * IN + i] = f[i];
    if (sizes && t) {   // targets: exact minus closed form, both scaled
        const float A = (float)sizes[3 * s], B = (float)sizes[3 * s + 1], I = (float)sizes[3 * s + 2];
        const float U = A + B - I;
        t[(size_t)s * OUT + 0] = I / out_scale(0, N) - base[0];
        t[(size_t)s * OUT + 1] = (A + B - 2.f * I) / out_scale(1, N) - base[1];
        t[(size_t)s * OUT + 2] = (U > 0 ? I / U : 0.f) - base[2];
        t[(size_t)s * OUT + 3] = ((A * B > 0) ? I / sqrtf(A * B) : 0.f) - base[3];
    }
}

}  // namespace mlp

// ---------------------------------------------------------------------------
// training pairs
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint64_t mix64(uint64_t z) {   // SplitMix64 finaliser
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// keyed Feistel permutation of [0, 2^(2h)), cycle-walked into [0, d)
__device__ __forceinline__ uint32_t perm_d(uint32_t x, uint32_t d, uint32_t h, uint64_t key) {
    const uint32_t mask = (1u << h) - 1u;
    do {
        uint32_t L = x >> h, R = x & mask;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint32_t f = (uint32_t)mix64(key + ((uint64_t)r << 32) + R) & mask;
            const uint32_t nl = R;
            R = L ^ f;
            L = nl;
        }
        x = (L << h) | R;
    } while (x >= d);
    return x;
}

__global__ void __launch_bounds__(256)
    dense_pairs_kernel(uint32_t n_pairs, uint32_t N, uint32_t d, uint32_t lo, uint32_t hi,
                       uint64_t seed, uint64_t mult, uint64_t add, uint32_t *__restrict__ counts,
                       uint32_t *__restrict__ sizes, uint32_t *__restrict__ cols, uint32_t max_cols) {
    extern __shared__ uint32_t sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t W = N >> 5;
    uint32_t *sa = sm + (size_t)warp * 2 * W;
    uint32_t *sb = sa + W;
    uint32_t h = 1;
    while ((1u << (2 * h)) < d) ++h;
    const uint32_t nw = gridDim.x * (blockDim.x >> 5);
    for (uint32_t p = blockIdx.x * (blockDim.x >> 5) + warp; p < n_pairs; p += nw) {
        const uint64_t key = mix64(seed * 0x9E3779B97F4A7C15ull + p);
        const uint64_t r0 = mix64(key ^ 0x5bd1e995ull), r1 = mix64(key ^ 0x27d4eb2full),
                       r2 = mix64(key ^ 0x165667b1ull);
        const uint32_t span = hi - lo + 1;
        const uint32_t A = lo + (uint32_t)((r0 >> 32) % span);
        const uint32_t Bz = lo + (uint32_t)((r1 >> 32) % span);
        const uint32_t mn = A < Bz ? A : Bz;
        const uint32_t I = (uint32_t)((r2 >> 32) % (mn + 1));
        const uint32_t tot = A + Bz - I;   // <= d by the caller's check
        for (uint32_t w = lane; w < W; w += 32) { sa[w] = 0u; sb[w] = 0u; }
        __syncwarp();
        for (uint32_t j = lane; j < tot; j += 32) {
            const uint32_t c = perm_d(j, d, h, key);
            const uint32_t bk = bucket_of(c, mult, add, N);
            const uint32_t bit = 1u << (bk & 31);
            // columns [0, I) are common, [I, A) only in a, [A, A+B-I) only in b
            if (j < A) atomicOr(&sa[bk >> 5], bit);
            if (j < I || j >= A) atomicOr(&sb[bk >> 5], bit);
            if (cols && j < max_cols) cols[(size_t)p * max_cols + j] = c;
        }
        __syncwarp();
        uint32_t ca = 0, cb = 0, cc = 0;
        for (uint32_t w = lane; w < W; w += 32) {
            ca += __popc(sa[w]);
            cb += __popc(sb[w]);
            cc += __popc(sa[w] & sb[w]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ca += __shfl_xor_sync(0xffffffffu, ca, o);
            cb += __shfl_xor_sync(0xffffffffu, cb, o);
            cc += __shfl_xor_sync(0xffffffffu, cc, o);
        }
        if (lane == 0) {
            counts[3 * (size_t)p] = ca;
            counts[3 * (size_t)p + 1] = cb;
            counts[3 * (size_t)p + 2] = cc;
            if (sizes) {
                sizes[3 * (size_t)p] = A;
                sizes[3 * (size_t)p + 1] = Bz;
                sizes[3 * (size_t)p + 2] = I;
            }
        }
        __syncwarp();
    }
}

__global__ void estimate_counts_kernel(const uint32_t *__restrict__ counts, uint32_t n, uint32_t N,
                                       float invL, float *__restrict__ out) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t a = counts[3 * s], b = counts[3 * s + 1], c = counts[3 * s + 2];
    const float lnA = row_log(a, N), lnB = row_log(b, N);
    out[4 * (size_t)s + 0] = estimate_one<M_IP>(a, b, c, N, lnA, lnB, invL);
    out[4 * (size_t)s + 1] = estimate_one<M_HAM>(a, b, c, N, lnA, lnB, invL);
    out[4 * (size_t)s + 2] = estimate_one<M_JS>(a, b, c, N, lnA, lnB, invL);
    out[4 * (size_t)s + 3] = estimate_one<M_COS>(a, b, c, N, lnA, lnB, invL);
}

}  // namespace bs

using namespace bs;

static bool valid_N_l(uint32_t N) { return N >= 32 && N <= BS_N_MAX && (N % 32) == 0; }

extern "C" {

bs_status bs_dense_pairs(uint32_t n_pairs, uint32_t N, uint32_t d, uint32_t size_lo, uint32_t size_hi,
                         uint64_t pair_seed, uint64_t hash_seed, uint32_t *counts, uint32_t *sizes,
                         uint32_t *cols, uint32_t max_cols, bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (!valid_N_l(N) || size_lo > size_hi || d == 0 || d > (1u << 30)) return BS_ERR_INVALID_ARG;
    if (2ull * size_hi > d) return BS_ERR_INVALID_ARG;   // a and b together must fit in [0, d)
    if (n_pairs == 0) return BS_OK;
    if (!counts || (cols && max_cols == 0)) return BS_ERR_INVALID_ARG;
    uint64_t mult, add;
    hash_params(hash_seed, &mult, &add);
    const size_t smem = (size_t)8 * 2 * (N / 32) * sizeof(uint32_t);
    if (ensure_smem((const void *)dense_pairs_kernel, smem) != cudaSuccess) return BS_ERR_CUDA;
    const uint32_t want = (n_pairs + 7) / 8, cap = (uint32_t)sm_count() * 16u;
    dense_pairs_kernel<<<want < cap ? want : cap, 256, smem, (cudaStream_t)stream>>>(
        n_pairs, N, d, size_lo, size_hi, pair_seed, mult, add, counts, sizes, cols, max_cols);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

bs_status bs_estimate_counts(const uint32_t *counts, uint32_t n, uint32_t N, float *out,
                             bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (!valid_N_l(N)) return BS_ERR_INVALID_ARG;
    if (n == 0) return BS_OK;
    if (!counts || !out) return BS_ERR_INVALID_ARG;
    const float invL = (float)(1.0 / log1p(-1.0 / (double)N));
    estimate_counts_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(counts, n, N, invL, out);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

bs_status bs_mlp_prepare(const uint32_t *counts, const uint32_t *sizes, uint32_t n, uint32_t N, float *x,
                         float *t, bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (!valid_N_l(N)) return BS_ERR_INVALID_ARG;
    if (n == 0) return BS_OK;
    if (!counts || !x || (sizes && !t)) return BS_ERR_INVALID_ARG;
    mlp::prepare_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(counts, sizes, n, N, x, t);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

bs_status bs_mlp_train_step(float *params, float *adam_m, float *adam_v, float *grad, uint32_t step,
                            float lr, const float *x, const float *t, uint32_t n, float *loss,
                            bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (n == 0 || step == 0) return BS_ERR_INVALID_ARG;
    if (!params || !adam_m || !adam_v || !grad || !x || !t) return BS_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = mlp::train_smem_bytes();
    if (ensure_smem((const void *)mlp::train_grad_kernel, smem) != cudaSuccess) return BS_ERR_CUDA;
    mlp::train_grad_kernel<<<(n + mlp::TB - 1) / mlp::TB, mlp::TB, smem, s>>>(params, x, t, n, grad, loss);
    const float b1c = 1.0f - powf(0.9f, (float)step), b2c = 1.0f - powf(0.999f, (float)step);
    mlp::adam_kernel<<<(mlp::NPARAM + 255) / 256, 256, 0, s>>>(params, adam_m, adam_v, grad, lr, b1c, b2c);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

bs_status bs_mlp_estimate_ex(const float *params, const uint32_t *counts, uint32_t n, uint32_t N,
                             float *out, uint32_t variant, bs_stream_t stream) {
    BS_NVTX_RANGE();
    if (!valid_N_l(N)) return BS_ERR_INVALID_ARG;
    if (variant > BS_VARIANT_TC) return BS_ERR_INVALID_ARG;
    if (n == 0) return BS_OK;
    if (!params || !counts || !out) return BS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (variant == BS_VARIANT_POPC) {   // CUDA cores only
        mlp::infer_kernel<<<(n + 255) / 256, 256, 0, st>>>(params, counts, n, N, out);
        return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
    }
    unsigned int *err = error_word();
    if (!err) return BS_ERR_CUDA;
    const void *kern = (const void *)mlp::infer_tc_kernel;
    if (ensure_smem(kern, mlp::tcm::SMEM_BYTES) != cudaSuccess) return BS_ERR_CUDA;
    const uint32_t tiles = (n + mlp::tcm::ROWS - 1) / mlp::tcm::ROWS;
    const uint32_t cap = (uint32_t)sm_count() * 6u;
    const uint32_t grid = tiles < cap ? tiles : cap;
    mlp::infer_tc_kernel<<<grid, mlp::tcm::ROWS, mlp::tcm::SMEM_BYTES, st>>>(params, counts, n, N, out, err);
    return cudaGetLastError() == cudaSuccess ? BS_OK : BS_ERR_CUDA;
}

bs_status bs_mlp_estimate(const float *params, const uint32_t *counts, uint32_t n, uint32_t N, float *out,
                          bs_stream_t stream) {
    return bs_mlp_estimate_ex(params, counts, n, N, out, BS_VARIANT_AUTO, stream);
}

}  // extern "C"
