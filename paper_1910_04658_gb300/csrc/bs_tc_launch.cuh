// Launch of the tensor-core top-k kernel for one measure, every block
// configuration; included only by the per-measure translation units
// (bs_tc_ip.cu, bs_tc_ham.cu, bs_tc_js.cu, bs_tc_cos.cu), so that their
// kernels compile in parallel and the host code does not instantiate them.
#pragma once

#include "bs_tc_kernel.cuh"

namespace bs {
namespace tc {

template <int M, int NJ>
cudaError_t launch_topk(int cfg, const Args<NJ> &p, uint32_t grid, cudaStream_t stream) {
    cudaError_t ce = cudaErrorInvalidConfiguration;
    auto go = [&](auto kern, size_t smem, int threads) {
        if (smem > kSmemLimit) return;
        ce = ensure_smem((const void *)kern, smem);
        if (ce != cudaSuccess) return;
        kern<<<grid, threads, smem, stream>>>(p);
        ce = cudaGetLastError();
    };
    // a batch's job table is copied to shared memory behind the heaps
    const size_t jobs_smem = NJ > 1 ? (size_t)p.njobs * sizeof(Job) : 0;
    switch (cfg) {
#define X(c, nop, ng, sk, rd, sh, nb, tb)                                                              \
    case c:                                                                                            \
        if constexpr (nb == 0 || NJ == 1 || nop == 0)                                                  \
            go(pair_tc_kernel<MODE_TOPK, M, nop, ng, sk, rd, sh, NJ, nb, tb>,                          \
               smem_bytes<nop, ng, sk, rd, sh, nb, tb>(p.k) + jobs_smem, threads_for(ng, nop > 0));    \
        break;
        BS_TC_CONFIGS(X)
#undef X
    }
    return ce;
}

}  // namespace tc
}  // namespace bs

// one measure's instantiations: a single problem and the batched job table
#define BS_TC_INSTANTIATE(M)                                                                                   \
    namespace bs {                                                                                             \
    namespace tc {                                                                                             \
    template cudaError_t launch_topk<M, 1>(int, const Args<1> &, uint32_t, cudaStream_t);                    \
    template cudaError_t launch_topk<M, MAXJ>(int, const Args<MAXJ> &, uint32_t, cudaStream_t);              \
    }                                                                                                          \
    }
