// Tensor-core top-k kernels ranked by HAM (one translation unit per measure so
// the instantiations compile in parallel).
#include "bs_tc_launch.cuh"

BS_TC_INSTANTIATE(bs::M_HAM)
