// Tensor-core kernel storing the full count and estimate matrices
// (bs_estimate_pairs: Alg. 1 step 2 and Alg. 1-4 for every pair).
#include "bs_tc_kernel.cuh"

namespace bs {
namespace tc {

// Two epilogue groups, two 256-bit operand slots, a four-deep raw ring, no heaps.
cudaError_t launch_store(const Args<1> &p, uint32_t grid, cudaStream_t stream) {
    auto kern = pair_tc_kernel<MODE_STORE, M_IP, 2, 2, 128, 4, false, 1>;
    const size_t smem = smem_bytes<2, 2, 128, 4, false>(0);
    cudaError_t ce = ensure_smem((const void *)kern, smem);
    if (ce != cudaSuccess) return ce;
    kern<<<grid, threads_for(2), smem, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace tc
}  // namespace bs
