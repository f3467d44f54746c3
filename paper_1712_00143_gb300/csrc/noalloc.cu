// noalloc.cu -- stag_apply_m_noalloc: the FP64 even-odd operator with its
// odd-parity intermediate in a fixed, file-scope device array, so that the
// call performs no device allocation of any kind.
//
// The array is a static __device__ symbol: every GPU that loads libstag
// holds it (3 MiB) until the process exits.  Host code never uses the
// symbol's name as an address; the device address is looked up once per
// device with cudaGetSymbolAddress, with that device current, the first time
// the entry point runs on it.
#include <mutex>

#include "dslash_impl.cuh"

namespace stag {
namespace {

__device__ __align__(256) double2 g_noalloc_t[3 * STAG_NOALLOC_MAX_VH];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_t on the current device (looked up once).
int noalloc_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return STAG_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_t) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return STAG_ECUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return STAG_OK;
}

}  // namespace
}  // namespace stag

using namespace stag;

extern "C" int stag_apply_m_noalloc(stag_lattice_t lat, void* out, const void* in, double mass, double shift,
                                    void* stream) {
  if (!lat || !out || !in) return STAG_EINVAL;
  if (!lat->links[STAG_FP64].present) return STAG_EINVAL;
  if (lat->g.Vh > STAG_NOALLOC_MAX_VH) return STAG_EINVAL;
  // in is read through the read-only path by the kernel that writes out
  const size_t bytes = (size_t)lat->g.Vh * 48;
  const char *pi = (const char*)in, *po = (const char*)out;
  if (pi < po + bytes && po < pi + bytes) return STAG_EINVAL;
  void* scratch = nullptr;
  int s = noalloc_scratch(&scratch);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int Vh = lat->g.Vh;
  // FP64 vectors use the canonical layout internally: in/out need no copies.
  Spinor<64> x{const_cast<void*>(in), Vh};
  Spinor<64> t{scratch, Vh};
  Spinor<64> o{out, Vh};
  Spinor<64> none{nullptr, Vh};
  const int B = 256, G = (Vh + B - 1) / B;
  // t = D_oe in (odd sites): every entry of t is written before it is read
  DslashArgs<64> a1 = make_args<64>(lat, x, 1);
  {
    ProfScope ps("dslash64", st);
    k_dslash<64, 9, 256, 1><<<G, B, 0, st>>>(a1, t, nullptr);
  }
  if ((s = last_launch_status())) return s;
  // out = (m^2 + shift) in - D_eo t (even sites)
  DslashArgs<64> a2 = make_args<64>(lat, t, 0);
  {
    ProfScope ps("dslash64_epi", st);
    k_dslash_epi<64, 9, 0, 256, 1><<<G, B, 0, st>>>(a2, o, x, mass * mass + shift, none, 0.0, -1.0,
                                                    RedBuf{nullptr, nullptr}, RedTarget{RED_STORE, nullptr, nullptr},
                                                    nullptr);
  }
  return last_launch_status();
}
