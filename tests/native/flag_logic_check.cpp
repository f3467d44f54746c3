// Host check of take_flag (paper_1712_00143_gb300/csrc/flags.h): the
// read-and-clear of a device status word, with a host word standing in for
// the device symbol and injectable read/clear failures.  Prints "ok" and
// exits 0 when every case holds.
#include <cstdio>

#include "flags.h"

namespace {
struct FakeWord {
  int value = 0;
  bool fail_read = false, fail_clear = false;
  int reads = 0, clears = 0;
};

int check(bool cond, const char* what) {
  if (!cond) std::printf("FAILED: %s\n", what);
  return cond ? 0 : 1;
}
}  // namespace

int main() {
  int bad = 0;
  FakeWord w;
  auto read = [&w](int* v) {
    ++w.reads;
    if (w.fail_read) return 1;
    *v = w.value;
    return 0;
  };
  auto clear = [&w]() {
    ++w.clears;
    if (w.fail_clear) return 1;
    w.value = 0;
    return 0;
  };
  // nothing recorded: OK, and the word is not written
  bad += check(stag::take_flag(read, clear, STAG_ETIMEOUT) == STAG_OK, "clean word reads OK");
  bad += check(w.clears == 0, "clean word is not cleared");
  // a kernel gave up a wait: reported once, then cleared
  w.value = 1;
  bad += check(stag::take_flag(read, clear, STAG_ETIMEOUT) == STAG_ETIMEOUT, "set word reports the status");
  bad += check(w.value == 0 && w.clears == 1, "set word is cleared");
  bad += check(stag::take_flag(read, clear, STAG_ETIMEOUT) == STAG_OK, "the next check starts clean");
  // any non-zero bit pattern counts (kernels OR their bits in)
  w.value = 6;
  bad += check(stag::take_flag(read, clear, STAG_ETIMEOUT) == STAG_ETIMEOUT, "other bits report too");
  // a failed read is a CUDA error, and nothing is cleared
  w.value = 1;
  w.fail_read = true;
  const int clears = w.clears;
  bad += check(stag::take_flag(read, clear, STAG_ETIMEOUT) == STAG_ECUDA, "failed read -> ECUDA");
  bad += check(w.clears == clears && w.value == 1, "failed read clears nothing");
  // a failed clear is a CUDA error (the word stays set for the next check)
  w.fail_read = false;
  w.fail_clear = true;
  bad += check(stag::take_flag(read, clear, STAG_ETIMEOUT) == STAG_ECUDA, "failed clear -> ECUDA");
  bad += check(w.value == 1, "failed clear leaves the word set");
  w.fail_clear = false;
  bad += check(stag::take_flag(read, clear, STAG_ETIMEOUT) == STAG_ETIMEOUT, "then it is reported");
  if (bad == 0) std::printf("ok\n");
  return bad == 0 ? 0 : 1;
}
