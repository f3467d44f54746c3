// dslash16.cu -- instantiation of the hop kernels for binary16 storage.
#include "dslash_impl.cuh"

namespace stag {
STAG_INSTANTIATE_DSLASH(16)
}  // namespace stag
