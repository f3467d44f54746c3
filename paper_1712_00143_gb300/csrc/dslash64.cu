// dslash64.cu -- instantiation of the hop kernels for 64-bit storage.
#include "dslash_impl.cuh"

namespace stag {
STAG_INSTANTIATE_DSLASH(64)
}  // namespace stag
