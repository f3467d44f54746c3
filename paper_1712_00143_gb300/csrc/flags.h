// flags.h -- host-side handling of the library's device status words.
//
// Kernels that give up a bounded wait (the tensor-core layers' mbarrier
// waits) record it in a device word instead of trapping, and the host turns
// the word into a status: read it; if it is set, clear it and report the
// status that goes with it, so that the next check starts clean.  The
// reading and clearing are passed in, so that the logic is the same with a
// device word (cudaMemcpyFromSymbol / cudaMemcpyToSymbol) and with a host
// stand-in; plain C++, no CUDA header.
#pragma once

#include "../../include/stag.h"

namespace stag {

// read(ctx, &v) and clear(ctx) return 0 on success.  Returns STAG_OK when
// the word is 0, `status_if_set` after clearing a non-zero word, STAG_ECUDA
// when reading or clearing fails (a failed clear still reports the event).
template <class Read, class Clear>
int take_flag(Read read, Clear clear, int status_if_set) {
  int v = 0;
  if (read(&v) != 0) return STAG_ECUDA;
  if (v == 0) return STAG_OK;
  if (clear() != 0) return STAG_ECUDA;
  return status_if_set;
}

}  // namespace stag
