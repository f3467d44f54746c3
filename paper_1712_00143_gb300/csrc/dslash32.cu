// dslash32.cu -- instantiation of the hop kernels for 32-bit storage.
#include "dslash_impl.cuh"

namespace stag {
STAG_INSTANTIATE_DSLASH(32)
}  // namespace stag
