// dslash31.cu -- instantiation of the hop kernels for 16-bit fixed-point links
// with FP32 vectors.
#include "dslash_impl.cuh"

namespace stag {
STAG_INSTANTIATE_DSLASH(31)
}  // namespace stag
