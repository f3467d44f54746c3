// mrhs31.cu -- instantiation of the N-right-hand-side Dslash kernels, their
// launch variants and the autotuner for 16-bit fixed-point links with FP32
// vectors (see mrhs_kernels.cuh).
#include "mrhs_kernels.cuh"

namespace stag {
STAG_INSTANTIATE_MRHS_N(31, 2)
STAG_INSTANTIATE_MRHS_N(31, 4)
STAG_INSTANTIATE_MRHS_N(31, 8)
STAG_INSTANTIATE_MRHS_RED3(31, 2)
STAG_INSTANTIATE_MRHS_RED3(31, 4)
STAG_INSTANTIATE_MRHS_RED3(31, 8)
}  // namespace stag
