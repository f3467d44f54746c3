// mrhs32.cu -- instantiation of the N-right-hand-side Dslash kernels, their
// launch variants and the autotuner for storage format 32 (see mrhs_kernels.cuh).
#include "mrhs_kernels.cuh"

namespace stag {
STAG_INSTANTIATE_MRHS_N(32, 2)
STAG_INSTANTIATE_MRHS_N(32, 4)
STAG_INSTANTIATE_MRHS_N(32, 8)
STAG_INSTANTIATE_MRHS_RED3(32, 2)
STAG_INSTANTIATE_MRHS_RED3(32, 4)
STAG_INSTANTIATE_MRHS_RED3(32, 8)
}  // namespace stag

using namespace stag;

namespace {

int tuned_mrhs(stag_lattice_t lat, int prec, int nrhs, bool epi, int* threads_per_site, int* min_blocks, double* us) {
  if (!lat || prec < 0 || prec > STAG_FX16L32 || prec == STAG_DF64 || !lat->links[link_copy_of(prec)].present)
    return STAG_EINVAL;
  if (nrhs != 2 && nrhs != 4 && nrhs != 8) return STAG_EINVAL;
  const auto& slot = lat->mrhs[prec][mrhs_nindex(nrhs)];
  const int p = prec == STAG_FP64 ? 64 : prec == STAG_FP32 ? 32 : prec == STAG_FP16 ? 16 : prec == STAG_FX16L32 ? 31 : 15;
  const int chosen = epi ? slot.variant_epi : slot.variant;
  const int v = chosen >= 0 ? chosen : mrhs_default_variant(p, nrhs);
  if (threads_per_site) *threads_per_site = mvariant(v).sp;
  if (min_blocks) *min_blocks = mvariant(v).minb;
  if (us) *us = chosen >= 0 ? (epi ? slot.us_epi : slot.us) : 0.0;
  return STAG_OK;
}

}  // namespace

extern "C" int stag_tuned_mrhs(stag_lattice_t lat, int prec, int nrhs, int* threads_per_site, int* min_blocks,
                               double* us) {
  return tuned_mrhs(lat, prec, nrhs, false, threads_per_site, min_blocks, us);
}

extern "C" int stag_tuned_mrhs_variant(stag_lattice_t lat, int prec, int nrhs, int epilogue) {
  if (!lat || prec < 0 || prec > STAG_FX16L32 || prec == STAG_DF64 || !lat->links[link_copy_of(prec)].present)
    return STAG_EINVAL;
  if (nrhs != 2 && nrhs != 4 && nrhs != 8) return STAG_EINVAL;
  const auto& slot = lat->mrhs[prec][mrhs_nindex(nrhs)];
  const int p = prec == STAG_FP64 ? 64 : prec == STAG_FP32 ? 32 : prec == STAG_FP16 ? 16 : prec == STAG_FX16L32 ? 31 : 15;
  const int chosen = epilogue ? slot.variant_epi : slot.variant;
  return chosen >= 0 ? chosen : mrhs_default_variant(p, nrhs);
}

extern "C" int stag_tuned_mrhs_epi(stag_lattice_t lat, int prec, int nrhs, int* threads_per_site, int* min_blocks,
                                   double* us) {
  return tuned_mrhs(lat, prec, nrhs, true, threads_per_site, min_blocks, us);
}
