// dslash15.cu -- instantiation of the hop kernels for 16-bit fixed-point storage.
#include "dslash_impl.cuh"

namespace stag {
STAG_INSTANTIATE_DSLASH(15)
}  // namespace stag
