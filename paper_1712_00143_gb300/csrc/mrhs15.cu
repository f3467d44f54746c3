// mrhs15.cu -- instantiation of the N-right-hand-side Dslash kernels, their
// launch variants and the autotuner for storage format 15 (see mrhs_kernels.cuh).
#include "mrhs_kernels.cuh"

namespace stag {
STAG_INSTANTIATE_MRHS_N(15, 2)
STAG_INSTANTIATE_MRHS_N(15, 4)
STAG_INSTANTIATE_MRHS_N(15, 8)
STAG_INSTANTIATE_MRHS_RED3(15, 2)
STAG_INSTANTIATE_MRHS_RED3(15, 4)
STAG_INSTANTIATE_MRHS_RED3(15, 8)
}  // namespace stag
