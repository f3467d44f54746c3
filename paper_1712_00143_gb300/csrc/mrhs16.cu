// mrhs16.cu -- instantiation of the N-right-hand-side Dslash kernels, their
// launch variants and the autotuner for storage format 16 (see mrhs_kernels.cuh).
#include "mrhs_kernels.cuh"

namespace stag {
STAG_INSTANTIATE_MRHS_N(16, 2)
STAG_INSTANTIATE_MRHS_N(16, 4)
STAG_INSTANTIATE_MRHS_N(16, 8)
STAG_INSTANTIATE_MRHS_RED3(16, 2)
STAG_INSTANTIATE_MRHS_RED3(16, 4)
STAG_INSTANTIATE_MRHS_RED3(16, 8)
}  // namespace stag
