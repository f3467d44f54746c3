// mrhs64.cu -- instantiation of the N-right-hand-side Dslash kernels, their
// launch variants and the autotuner for storage format 64 (see mrhs_kernels.cuh).
#include "mrhs_kernels.cuh"

namespace stag {
STAG_INSTANTIATE_MRHS_N(64, 2)
STAG_INSTANTIATE_MRHS_N(64, 4)
STAG_INSTANTIATE_MRHS_N(64, 8)
// the FP64 true residual of the batched solve: ||b - M y||^2 per system
#define STAG_INSTANTIATE_MRHS_RED2(N)                                                                                \
  template int mdslash_epi<64, N, 2>(const stag_lattice_s*, SpinorM<64>, SpinorM<64>, int, SpinorM<64>, double,     \
                                     SpinorM<64>, double, double, RedScratch, RedTarget, const int*, cudaStream_t);
STAG_INSTANTIATE_MRHS_RED2(2)
STAG_INSTANTIATE_MRHS_RED2(4)
STAG_INSTANTIATE_MRHS_RED2(8)
}  // namespace stag
