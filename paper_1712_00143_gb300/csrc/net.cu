// net.cu -- the learned preconditioner: a gauge-covariant network built from
// the staggered operator's own fat-link hops, trained on the GPU with the
// kernels of net_kernels.cuh (forward, backward, Adam), and flexible CG that
// applies it to the residual at every iteration.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "flags.h"
#include "net_tc.cuh"

struct stag_net_s {
  int nl = 0;
  int ch[8] = {0};
  size_t nparam = 0;
  std::vector<size_t> woff, boff;  // offsets of W_l and b_l in the flat arrays (boff = SIZE_MAX: none)
  float* w = nullptr;              // FP32 master parameters
  float* m = nullptr;              // Adam moments
  float* v = nullptr;
  float* grad = nullptr;           // accumulated gradient
  __nv_bfloat16* wb = nullptr;     // bfloat16 copy used by the kernels (weights only; biases stay FP32)
  int step = 0;
  stag::Workspace ws;
};

namespace stag {

namespace netk {

#define TRYN(...)              \
  do {                         \
    int _s = (__VA_ARGS__);    \
    if (_s) return _s;         \
  } while (0)

// SplitMix64 + Box-Muller for the seeded initial weights.
uint64_t sm64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double unif(uint64_t seed, uint64_t i) { return ((sm64(seed * 0x100000001B3ull + i) >> 11) + 1.0) * (1.0 / 9007199254740992.0); }
double normal(uint64_t seed, uint64_t i) {
  const double u1 = unif(seed, 2 * i), u2 = unif(seed, 2 * i + 1);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16_rn(w[i]);
}

// Adam on the FP32 master copy; the kernels then read the bfloat16 rounding.
__global__ void k_adam(float* w, float* m, float* v, const float* __restrict__ g, size_t n, float lr, float b1,
                       float b2, float eps, float c1, float c2, float scale) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i] * scale;
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// One-channel input field: even sites r * scale, odd sites 0 (scale from a
// device norm: sqrt(Vh / ||r||^2)).
__global__ void k_net_embed(Spinor<32> r, const double* __restrict__ rr, float2* __restrict__ h0) {
  const int Vh = r.Vh;
  const float sc = (float)sqrt((double)Vh / fmax(*rr, 1e-300));
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
    float2 v[3];
    SpinorLoad<32>::ld(r, s, v);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      h0[(size_t)s * 3 + c] = make_float2(v[c].x * sc, v[c].y * sc);
      h0[((size_t)Vh + s) * 3 + c] = make_float2(0.f, 0.f);
    }
  }
}

// z = prediction / scale on even sites (the network's output channel).
__global__ void k_net_extract(const float2* __restrict__ hL, const double* __restrict__ rr, Spinor<32> z) {
  const int Vh = z.Vh;
  const float inv = (float)sqrt(fmax(*rr, 0.0) / (double)Vh);
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
    float2 o[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 v = hL[(size_t)s * 3 + c];
      o[c] = make_float2(v.x * inv, v.y * inv);
    }
    SpinorLoad<32>::st(z, s, o);
  }
}

// Loss ||pred - e_hat||^2 / ||e_hat||^2 (e_hat = e * scale) and its gradient
// g = 2 (pred - e_hat) / ||e_hat||^2 on even sites, 0 on odd sites.  ee =
// ||e||^2, rr = ||r||^2.  The numerator is reduced into `tgt`.
__global__ void k_net_loss(const float2* __restrict__ hL, Spinor<32> e, const double* __restrict__ rr,
                           const double* __restrict__ ee, float2* __restrict__ g, RedBuf rb, RedTarget tgt) {
  const int Vh = e.Vh;
  const double sc2 = (double)Vh / fmax(*rr, 1e-300);
  const float sc = (float)sqrt(sc2);
  const float inv = (float)(1.0 / (fmax(*ee, 1e-300) * sc2));
  Acc1<float> acc;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
    float2 ev[3];
    SpinorLoad<32>::ld(e, s, ev);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 pv = hL[(size_t)s * 3 + c];
      const float dx = pv.x - ev[c].x * sc, dy = pv.y - ev[c].y * sc;
      acc.add_prod(dx, dx);
      acc.add_prod(dy, dy);
      g[(size_t)s * 3 + c] = make_float2(2.f * dx * inv, 2.f * dy * inv);
      g[((size_t)Vh + s) * 3 + c] = make_float2(0.f, 0.f);
    }
  }
  double v[1] = {acc.value() * (1.0 / (fmax(*ee, 1e-300) * sc2))};
  grid_reduce<1>(v, rb, tgt);
}

// Residual-space loss, step 1: the scaled prediction z^ (even block of the
// output channel) as an FP32 structure-of-arrays field.
__global__ void k_net_pred_to_spinor(const float2* __restrict__ hL, Spinor<32> z) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < z.Vh; s += gridDim.x * blockDim.x) {
    float2 o[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) o[c] = hL[(size_t)s * 3 + c];
    SpinorLoad<32>::st(z, s, o);
  }
}

// Step 2: diff = M z^ - r^ (mz = M z^, r^ = r * scale), loss numerator
// ||diff||^2 / ||r^||^2 (||r^||^2 = scale^2 ||r||^2) reduced into `tgt`.
__global__ void k_net_resid_loss(Spinor<32> mz, Spinor<32> r, const double* __restrict__ rr, Spinor<32> diff, RedBuf rb,
                                 RedTarget tgt) {
  const int Vh = r.Vh;
  const double sc2 = (double)Vh / fmax(*rr, 1e-300);
  const float sc = (float)sqrt(sc2);
  Acc1<float> acc;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
    float2 a[3], b[3], o[3];
    SpinorLoad<32>::ld(mz, s, a);
    SpinorLoad<32>::ld(r, s, b);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      o[c] = make_float2(a[c].x - b[c].x * sc, a[c].y - b[c].y * sc);
      acc.add_prod(o[c].x, o[c].x);
      acc.add_prod(o[c].y, o[c].y);
    }
    SpinorLoad<32>::st(diff, s, o);
  }
  double v[1] = {acc.value() / (sc2 * fmax(*rr, 1e-300))};
  grid_reduce<1>(v, rb, tgt);
}

// Step 3: the output-channel gradient 2 M diff / ||r^||^2 on even sites, 0 on odd.
__global__ void k_net_resid_grad(Spinor<32> mdiff, float2* __restrict__ g) {
  const int Vh = mdiff.Vh;
  const float k = 2.f / (float)Vh;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < Vh; s += gridDim.x * blockDim.x) {
    float2 a[3];
    SpinorLoad<32>::ld(mdiff, s, a);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      g[(size_t)s * 3 + c] = make_float2(k * a[c].x, k * a[c].y);
      g[((size_t)Vh + s) * 3 + c] = make_float2(0.f, 0.f);
    }
  }
}

int grid_for(int n, int block) {
  int g = (n + block - 1) / block;
  return g < 8192 ? g : 8192;
}

}  // namespace netk
using namespace netk;

// ------------------------------------------------------------ network state on a lattice
struct NetRun {
  stag_net_s* net;
  stag_lattice_s* lat;
  NetGeom ng;
  int Vh;
  std::vector<float2*> h, pre;  // per layer output (h[0] = input)
  float2* U = nullptr;          // [9][2 Vh][3]: per-direction mixes of the one-channel output layer
  float2* g0 = nullptr;         // gradient buffers (ping-pong)
  float2* g1 = nullptr;
  float* part = nullptr;        // per-block partial sums for dW / db
  int part_blocks = 0;
  double* scal = nullptr;       // rr, ee, loss
  RedScratch rs;
};

static int net_run_init(stag_net_s* net, stag_lattice_s* lat, NetRun& R, bool training) {
  if (!lat->links[STAG_FP32].present) return STAG_EINVAL;
  R.net = net;
  R.lat = lat;
  R.Vh = lat->g.Vh;
  R.ng.g = lat->g;
  const LinkCopy& L = lat->links[STAG_FP32];
  R.ng.links[0] = (const uint4*)L.data;
  R.ng.links[1] = (const uint4*)((const char*)L.data + L.parity_stride);
  R.ng.cpm = 18 + 2 * L.nl;
  int s = 0;
  const size_t sites = 2 * (size_t)R.Vh;
  R.h.assign(net->nl + 1, nullptr);
  R.pre.assign(net->nl + 1, nullptr);
  const std::string pre = "net." + std::to_string(R.Vh) + ".";
  for (int l = 0; l <= net->nl; ++l) {
    R.h[l] = (float2*)net->ws.get(pre + "h" + std::to_string(l), sites * net->ch[l] * 3 * sizeof(float2), &s);
    if (l > 0 && l < net->nl)
      R.pre[l] = (float2*)net->ws.get(pre + "p" + std::to_string(l), sites * net->ch[l] * 3 * sizeof(float2), &s);
  }
  int cmax = 1;
  for (int l = 0; l <= net->nl; ++l) cmax = net->ch[l] > cmax ? net->ch[l] : cmax;
  R.U = (float2*)net->ws.get(pre + "U", sites * NET_NDIR * 3 * sizeof(float2), &s);
  if (training) {
    R.g0 = (float2*)net->ws.get(pre + "g0", sites * cmax * 3 * sizeof(float2), &s);
    R.g1 = (float2*)net->ws.get(pre + "g1", sites * cmax * 3 * sizeof(float2), &s);
    R.part_blocks = 2 * 152;
    R.part = (float*)net->ws.get(pre + "part", (size_t)R.part_blocks * NET_NDIR * cmax * cmax * sizeof(float), &s);
  }
  R.scal = (double*)net->ws.get(pre + "scal", 64, &s);
  if (s) return s;
  return get_red_scratch(lat, "net", &R.rs, 2);
}

template <int CIN, int COUT, bool GATE>
static int launch_layer(const NetRun& R, int l, const float2* in, float2* pre, float2* out, const __nv_bfloat16* W,
                        const float* b, int transpose, cudaStream_t st) {
  const int n = 2 * R.Vh;
  count_launch();
  if constexpr (CIN == 16 && COUT == 16) {
    // the channel mixing of a 16 -> 16 layer runs on the tensor cores
    // one CTA per 64-site tile
    static bool attr[2] = {false, false};
    if (!attr[GATE]) {
      cudaFuncSetAttribute(k_net_layer_tc<GATE>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::LAYER_SMEM);
      attr[GATE] = true;
    }
    // the layer's bulk copies need 16-byte aligned input records
    if (((uintptr_t)in & 15u) != 0) return STAG_EINVAL;
    const int tiles = 2 * ((R.Vh + tc::TILE - 1) / tc::TILE);
    k_net_layer_tc<GATE><<<tiles, 128, tc::LAYER_SMEM, st>>>(R.ng, in, pre, out, W, b, transpose);
  } else if constexpr (COUT == 1 && CIN == 16 && !GATE) {
    if (!transpose) {
      // one output channel: site-local mix into the nine directions, then
      // one transport per direction
      k_net_mix_local<CIN><<<grid_for(n, 256), 256, 0, st>>>(n, in, W, R.U);
      count_launch();
      k_net_transport_sum<<<grid_for(n, 256), 256, 0, st>>>(R.ng, R.U, out);
    } else {
      k_net_layer<CIN, COUT, GATE><<<(n + 127) / 128, 128, 0, st>>>(R.ng, in, pre, out, W, b, transpose);
    }
  } else {
    // 16 output channels: the block's outputs are staged in shared memory
    const size_t smem = COUT == 16 ? (size_t)128 * 97 * sizeof(float) : 0;
    static bool attr = false;
    if (COUT == 16 && !attr) {
      cudaFuncSetAttribute(k_net_layer<CIN, COUT, GATE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      attr = true;
    }
    k_net_layer<CIN, COUT, GATE><<<(n + 127) / 128, 128, smem, st>>>(R.ng, in, pre, out, W, b, transpose);
  }
  return STAG_OK;
}

// STAG_ETIMEOUT if a tensor-core layer gave up a bounded wait since the
// last check (the flag is cleared here).  Synchronous.
static int net_tc_status() {
  auto read = [](int* v) {
    const cudaError_t e = cudaMemcpyFromSymbol(v, tc::g_tc_error, sizeof(int));
    if (e != cudaSuccess) cudaGetLastError();
    return e == cudaSuccess ? 0 : 1;
  };
  auto clear = []() {
    const int z = 0;
    const cudaError_t e = cudaMemcpyToSymbol(tc::g_tc_error, &z, sizeof(int));
    if (e != cudaSuccess) cudaGetLastError();
    return e == cudaSuccess ? 0 : 1;
  };
  return take_flag(read, clear, STAG_ETIMEOUT);
}

// Layer l forward (ch[l] -> ch[l+1]); supported widths 1 and 16.
static int layer_fwd(const NetRun& R, int l, cudaStream_t st) {
  stag_net_s* N = R.net;
  const int ci = N->ch[l], co = N->ch[l + 1];
  const bool gate = l + 1 < N->nl;
  const __nv_bfloat16* W = N->wb + N->woff[l];
  const float* b = gate ? N->w + N->boff[l] : nullptr;
  float2 *in = R.h[l], *out = R.h[l + 1], *pre = gate ? R.pre[l + 1] : R.h[l + 1];
  ProfScope ps(ci == 16 && co == 16 ? "net_tc" : "net", st);
  int ls;
  if (ci == 1 && co == 16 && gate) ls = launch_layer<1, 16, true>(R, l, in, pre, out, W, b, 0, st);
  else if (ci == 16 && co == 16 && gate) ls = launch_layer<16, 16, true>(R, l, in, pre, out, W, b, 0, st);
  else if (ci == 16 && co == 1 && !gate) ls = launch_layer<16, 1, false>(R, l, in, pre, out, W, b, 0, st);
  else if (ci == 1 && co == 1 && !gate) ls = launch_layer<1, 1, false>(R, l, in, pre, out, W, b, 0, st);
  else return STAG_EINVAL;
  if (ls) return ls;
  return last_launch_status();
}

// Backward through layer l: g (gradient w.r.t. the layer's output, ch[l+1]
// channels) -> dW, db accumulated into N->grad; gin (gradient w.r.t. its
// input) when want_in.
static int layer_bwd(const NetRun& R, int l, float2* g, float2* gin, bool want_in, cudaStream_t st) {
  stag_net_s* N = R.net;
  const int ci = N->ch[l], co = N->ch[l + 1];
  const bool gate = l + 1 < N->nl;
  const int n2 = 2 * R.Vh;
  if (gate) {
    ProfScope ps("net_bwd", st);
    const int G = R.part_blocks;
    if (co == 16)
      k_net_gate_bwd<16><<<G, 256, 0, st>>>(n2, R.pre[l + 1], g, N->w + N->boff[l], R.part);
    else
      return STAG_EINVAL;
    TRYN(last_launch_status());
    k_net_sum_parts<<<1, 64, 0, st>>>(R.part, G, co, N->grad + N->boff[l]);
    TRYN(last_launch_status());
  }
  {
    ProfScope ps("net_bwd", st);
    constexpr int TS = 16;
    const int G = R.part_blocks;
    const int nw = NET_NDIR * ci * co;
#define STAG_DW(CI, CO)                                                                                  \
  {                                                                                                      \
    const size_t smem = (size_t)(TS * NET_NDIR * CI * 6 + TS * CO * 6) * sizeof(float);                   \
    cudaFuncSetAttribute(k_net_dw<CI, CO, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
    k_net_dw<CI, CO, TS><<<G, 256, smem, st>>>(R.ng, R.h[l], g, R.part);                                  \
  }
    if (ci == 1 && co == 16) STAG_DW(1, 16)
    else if (ci == 16 && co == 16) STAG_DW(16, 16)
    else if (ci == 16 && co == 1) STAG_DW(16, 1)
    else if (ci == 1 && co == 1) STAG_DW(1, 1)
    else return STAG_EINVAL;
#undef STAG_DW
    TRYN(last_launch_status());
    k_net_sum_parts<<<grid_for(nw, 256), 256, 0, st>>>(R.part, G, nw, N->grad + N->woff[l]);
    TRYN(last_launch_status());
  }
  if (want_in) {
    // adjoint layer: co -> ci channels with W' (transposed, partner directions, sign)
    ProfScope ps("net_bwd", st);
    const __nv_bfloat16* W = N->wb + N->woff[l];
    int ls;
    if (ci == 16 && co == 16) ls = launch_layer<16, 16, false>(R, l, g, gin, gin, W, nullptr, 1, st);
    else if (ci == 16 && co == 1) ls = launch_layer<1, 16, false>(R, l, g, gin, gin, W, nullptr, 1, st);
    else if (ci == 1 && co == 16) ls = launch_layer<16, 1, false>(R, l, g, gin, gin, W, nullptr, 1, st);
    else if (ci == 1 && co == 1) ls = launch_layer<1, 1, false>(R, l, g, gin, gin, W, nullptr, 1, st);
    else return STAG_EINVAL;
    TRYN(ls);
    TRYN(last_launch_status());
  }
  return STAG_OK;
}

// Network forward on an even-site residual r (FP32 structure of arrays);
// rr = ||r||^2 on the device.  Leaves the output in R.h[nl].
static int net_forward(const NetRun& R, Spinor<32> r, const double* rr, cudaStream_t st) {
  {
    ProfScope ps("net", st);
    k_net_embed<<<grid_for(R.Vh, 256), 256, 0, st>>>(r, rr, R.h[0]);
  }
  TRYN(last_launch_status());
  for (int l = 0; l < R.net->nl; ++l) TRYN(layer_fwd(R, l, st));
  return STAG_OK;
}

// z = N(r) on even sites.
int net_apply(stag_net_s* net, stag_lattice_s* lat, Spinor<32> z, Spinor<32> r, const double* rr, cudaStream_t st) {
  NetRun R;
  TRYN(net_run_init(net, lat, R, false));
  TRYN(net_forward(R, r, rr, st));
  ProfScope ps("net", st);
  k_net_extract<<<grid_for(R.Vh, 256), 256, 0, st>>>(R.h[net->nl], rr, z);
  return last_launch_status();
}

// M v = m^2 v - D_eo D_oe v in FP32 (t: odd-parity scratch).
static int apply_m32(stag_lattice_s* lat, Spinor<32> out, Spinor<32> v, Spinor<32> t, double m2, RedScratch rs,
                     cudaStream_t st) {
  TRYN(launch_dslash<32>(lat, t, v, 1, nullptr, st));
  return launch_dslash_epi<32>(lat, out, t, 0, v, m2, Spinor<32>{nullptr, v.Vh}, 0.0, -1.0, 0, rs,
                               RedTarget{RED_STORE, nullptr, nullptr}, nullptr, st);
}

// Loss of one (r, e) pair (kind: stag_loss) and its gradient added to net->grad.
static int net_loss_grad(NetRun& R, Spinor<32> r, Spinor<32> e, int kind, double mass, double* loss_dev,
                         cudaStream_t st) {
  stag_net_s* N = R.net;
  TRYN(launch_norm2<32>(r, R.rs, RedTarget{RED_STORE, nullptr, R.scal}, st));
  if (kind == STAG_LOSS_ERROR) TRYN(launch_norm2<32>(e, R.rs, RedTarget{RED_STORE, nullptr, R.scal + 1}, st));
  TRYN(net_forward(R, r, R.scal, st));
  const int G = grid_for(R.Vh, 256) < R.rs.max_grid ? grid_for(R.Vh, 256) : R.rs.max_grid;
  if (kind == STAG_LOSS_ERROR) {
    ProfScope ps("net_bwd", st);
    k_net_loss<<<G, 256, 0, st>>>(R.h[N->nl], e, R.scal, R.scal + 1, R.g0, RedBuf{R.rs.partials, R.rs.counter},
                                  RedTarget{RED_STORE, nullptr, loss_dev});
    TRYN(last_launch_status());
  } else {
    int s = 0;
    Spinor<32> z = ws_spinor<32>(R.lat, "netloss.z", &s);
    Spinor<32> mz = ws_spinor<32>(R.lat, "netloss.mz", &s);
    Spinor<32> t = ws_spinor<32>(R.lat, "netloss.t", &s);
    if (s) return s;
    const double m2 = mass * mass;
    {
      ProfScope ps("net_bwd", st);
      k_net_pred_to_spinor<<<grid_for(R.Vh, 256), 256, 0, st>>>(R.h[N->nl], z);
    }
    TRYN(last_launch_status());
    TRYN(apply_m32(R.lat, mz, z, t, m2, R.rs, st));
    {
      ProfScope ps("net_bwd", st);
      k_net_resid_loss<<<G, 256, 0, st>>>(mz, r, R.scal, z, RedBuf{R.rs.partials, R.rs.counter},
                                          RedTarget{RED_STORE, nullptr, loss_dev});
    }
    TRYN(last_launch_status());
    TRYN(apply_m32(R.lat, mz, z, t, m2, R.rs, st));  // M (M z^ - r^)
    {
      ProfScope ps("net_bwd", st);
      k_net_resid_grad<<<grid_for(R.Vh, 256), 256, 0, st>>>(mz, R.g0);
    }
    TRYN(last_launch_status());
  }
  float2 *g = R.g0, *gin = R.g1;
  for (int l = N->nl - 1; l >= 0; --l) {
    TRYN(layer_bwd(R, l, g, gin, l > 0, st));
    float2* t = g;
    g = gin;
    gin = t;
  }
  return STAG_OK;
}

}  // namespace stag

namespace stag {
namespace netk {
int canon_to_sloppy(stag_lattice_s* lat, Spinor<32> out, const void* in, int in_prec, cudaStream_t st);
}
}  // namespace stag

using namespace stag;

extern "C" {

int stag_net_create(stag_net_t* out, const int* channels, int nlayers, unsigned long long seed) {
  if (!out || !channels || nlayers < 1 || nlayers > 7) return STAG_EINVAL;
  for (int l = 0; l <= nlayers; ++l)
    if (channels[l] != 1 && channels[l] != 16) return STAG_EINVAL;
  if (channels[0] != 1 || channels[nlayers] != 1) return STAG_EINVAL;
  stag_net_s* n = new stag_net_s();
  n->nl = nlayers;
  size_t off = 0;
  for (int l = 0; l <= nlayers; ++l) n->ch[l] = channels[l];
  for (int l = 0; l < nlayers; ++l) {
    n->woff.push_back(off);
    off += (size_t)NET_NDIR * channels[l + 1] * channels[l];
    if (l + 1 < nlayers) {
      n->boff.push_back(off);
      off += channels[l + 1];
    } else {
      n->boff.push_back((size_t)-1);
    }
  }
  n->nparam = off;
  // Near-identity start: the self direction passes channel c to channel c
  // (weight 1), everything else is small noise, and the gates start open
  // (b = -8: sigmoid(|v|^2 + 8) > 0.9996), so N(r) is close to r and flexible
  // CG starts out close to CG; training learns the correction.
  std::vector<float> h(off, 0.f);
  uint64_t k = 0;
  for (int l = 0; l < nlayers; ++l) {
    const int ci = channels[l], co = channels[l + 1];
    const double sd = 0.02 / std::sqrt((double)NET_NDIR * ci);
    for (int d = 0; d < NET_NDIR; ++d)
      for (int c = 0; c < co; ++c)
        for (int cp = 0; cp < ci; ++cp) {
          double w = sd * normal(seed, k++);
          if (d == 0 && c == cp) w += 1.0;
          h[n->woff[l] + ((size_t)d * co + c) * ci + cp] = (float)w;
        }
    if (n->boff[l] != (size_t)-1)
      for (int c = 0; c < co; ++c) h[n->boff[l] + c] = -8.0f;
  }
  bool ok = cudaMalloc(&n->w, off * 4) == cudaSuccess && cudaMalloc(&n->m, off * 4) == cudaSuccess &&
            cudaMalloc(&n->v, off * 4) == cudaSuccess && cudaMalloc(&n->grad, off * 4) == cudaSuccess &&
            cudaMalloc(&n->wb, off * 2) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    stag_net_free(n);
    return STAG_ENOMEM;
  }
  cudaMemcpy(n->w, h.data(), off * 4, cudaMemcpyHostToDevice);
  cudaMemset(n->m, 0, off * 4);
  cudaMemset(n->v, 0, off * 4);
  cudaMemset(n->grad, 0, off * 4);
  k_to_bf16<<<grid_for((int)off, 256), 256, 0, 0>>>(n->w, n->wb, off);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    stag_net_free(n);
    return STAG_ECUDA;
  }
  *out = n;
  return STAG_OK;
}

int stag_net_free(stag_net_t n) {
  if (!n) return STAG_EINVAL;
  cudaDeviceSynchronize();
  cudaFree(n->w);
  cudaFree(n->m);
  cudaFree(n->v);
  cudaFree(n->grad);
  cudaFree(n->wb);
  delete n;
  return STAG_OK;
}

long long stag_net_num_params(stag_net_t n) { return n ? (long long)n->nparam : -1; }

int stag_net_get_params(stag_net_t n, float* host, long long count, int rounded) {
  if (!n || !host || count != (long long)n->nparam) return STAG_EINVAL;
  if (cudaMemcpy(host, n->w, n->nparam * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return STAG_ECUDA;
  if (rounded) {
    // the values the kernels use: weights rounded to bfloat16, biases FP32
    std::vector<__nv_bfloat16> b(n->nparam);
    if (cudaMemcpy(b.data(), n->wb, n->nparam * 2, cudaMemcpyDeviceToHost) != cudaSuccess) return STAG_ECUDA;
    for (int l = 0; l < n->nl; ++l) {
      const size_t nw = (size_t)NET_NDIR * n->ch[l] * n->ch[l + 1];
      for (size_t i = 0; i < nw; ++i) host[n->woff[l] + i] = __bfloat162float(b[n->woff[l] + i]);
    }
  }
  return STAG_OK;
}

int stag_net_set_params(stag_net_t n, const float* host, long long count) {
  if (!n || !host || count != (long long)n->nparam) return STAG_EINVAL;
  if (cudaMemcpy(n->w, host, n->nparam * 4, cudaMemcpyHostToDevice) != cudaSuccess) return STAG_ECUDA;
  k_to_bf16<<<grid_for((int)n->nparam, 256), 256, 0, 0>>>(n->w, n->wb, n->nparam);
  return cuda_status(cudaDeviceSynchronize());
}

int stag_net_apply(stag_net_t n, stag_lattice_t lat, void* z, const void* r, void* stream) {
  if (!n || !lat || !z || !r) return STAG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int s = 0;
  Spinor<32> rs = ws_spinor<32>(lat, "netapply.r", &s);
  Spinor<32> zs = ws_spinor<32>(lat, "netapply.z", &s);
  double* rr = (double*)lat->ws.get("netapply.rr", 64, &s);
  if (s) return s;
  RedScratch red;
  TRYN(get_red_scratch(lat, "netapply", &red));
  TRYN(launch_from_canonical<32>(rs, (const double2*)r, lat->g.Vh, st));
  TRYN(launch_norm2<32>(rs, red, RedTarget{RED_STORE, nullptr, rr}, st));
  TRYN(net_apply(n, lat, zs, rs, rr, st));
  return launch_to_canonical<32>((double2*)z, zs, lat->g.Vh, st);
}

int stag_net_loss_grad(stag_net_t n, stag_lattice_t lat, const void* r, const void* e, int loss_kind, double mass,
                       double* loss, float* grad, long long count, void* stream) {
  if (!n || !lat || !r || !e || !loss || !grad || count != (long long)n->nparam) return STAG_EINVAL;
  if (loss_kind != STAG_LOSS_ERROR && loss_kind != STAG_LOSS_RESIDUAL) return STAG_EINVAL;
  if (loss_kind == STAG_LOSS_RESIDUAL && !(mass >= 0.0)) return STAG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  NetRun R;
  TRYN(net_run_init(n, lat, R, true));
  int s = 0;
  Spinor<32> rs = ws_spinor<32>(lat, "netgrad.r", &s);
  Spinor<32> es = ws_spinor<32>(lat, "netgrad.e", &s);
  if (s) return s;
  TRYN(launch_from_canonical<32>(rs, (const double2*)r, lat->g.Vh, st));
  TRYN(launch_from_canonical<32>(es, (const double2*)e, lat->g.Vh, st));
  TRYN(cuda_status(cudaMemsetAsync(n->grad, 0, n->nparam * 4, st)));
  TRYN(net_loss_grad(R, rs, es, loss_kind, mass, R.scal + 2, st));
  TRYN(cuda_status(cudaMemcpyAsync(loss, R.scal + 2, sizeof(double), cudaMemcpyDeviceToHost, st)));
  TRYN(cuda_status(cudaMemcpyAsync(grad, n->grad, n->nparam * 4, cudaMemcpyDeviceToHost, st)));
  TRYN(cuda_status(cudaStreamSynchronize(st)));
  return net_tc_status();
}

int stag_tc_selftest(double* max_rel_err) {
  if (!max_rel_err) return STAG_EINVAL;
  float* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return STAG_ENOMEM;
  }
  cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
  count_launch();
  k_tc_selftest<<<1, 128, tc::SMEM_BYTES>>>(d);
  int s = last_launch_status();
  float h[2] = {0.f, 0.f};
  if (!s) s = cuda_status(cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost));
  cudaFree(d);
  if (s) return s;
  *max_rel_err = h[0];
  return h[1] == 1.f ? STAG_OK : STAG_ETIMEOUT;
}

int stag_net_train(stag_net_t n, const stag_train_pair* pairs, int npairs, const stag_train_params* tp,
                   double* losses, void* stream) {
  if (!n || !pairs || npairs <= 0 || !tp || tp->epochs <= 0 || tp->batch <= 0) return STAG_EINVAL;
  if (tp->pair_prec != STAG_FP64 && tp->pair_prec != STAG_FP32) return STAG_EINVAL;
  if (tp->loss != STAG_LOSS_ERROR && tp->loss != STAG_LOSS_RESIDUAL) return STAG_EINVAL;
  if (tp->loss == STAG_LOSS_RESIDUAL && !(tp->mass >= 0.0)) return STAG_EINVAL;
  for (int i = 0; i < npairs; ++i)
    if (!pairs[i].lat || !pairs[i].r || !pairs[i].e || pairs[i].lat->g.Vh != pairs[0].lat->g.Vh) return STAG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  stag_lattice_s* lat0 = pairs[0].lat;
  int s = 0;
  Spinor<32> rs = ws_spinor<32>(lat0, "nettrain.r", &s);
  Spinor<32> es = ws_spinor<32>(lat0, "nettrain.e", &s);
  double* lossd = (double*)lat0->ws.get("nettrain.loss", sizeof(double) * (size_t)npairs * tp->epochs, &s);
  if (s) return s;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  // visiting order: a seeded permutation per epoch
  std::vector<int> order(npairs);
  for (int ep = 0; ep < tp->epochs; ++ep) {
    for (int i = 0; i < npairs; ++i) order[i] = i;
    for (int i = npairs - 1; i > 0; --i) {
      const int j = (int)(sm64(tp->seed * 1000003ull + ep * 7919ull + i) % (uint64_t)(i + 1));
      std::swap(order[i], order[j]);
    }
    int inbatch = 0;
    for (int k = 0; k < npairs; ++k) {
      const stag_train_pair& P = pairs[order[k]];
      NetRun R;
      TRYN(net_run_init(n, P.lat, R, true));
      if (tp->pair_prec == STAG_FP64) {
        TRYN(launch_from_canonical<32>(rs, (const double2*)P.r, rs.Vh, st));
        TRYN(launch_from_canonical<32>(es, (const double2*)P.e, es.Vh, st));
      } else {
        TRYN(canon_to_sloppy(P.lat, rs, P.r, STAG_FP32, st));
        TRYN(canon_to_sloppy(P.lat, es, P.e, STAG_FP32, st));
      }
      if (inbatch == 0) TRYN(cuda_status(cudaMemsetAsync(n->grad, 0, n->nparam * 4, st)));
      TRYN(net_loss_grad(R, rs, es, tp->loss, tp->mass, lossd + (size_t)ep * npairs + k, st));
      if (++inbatch == tp->batch || k == npairs - 1) {
        n->step += 1;
        const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
        count_launch();
        k_adam<<<grid_for((int)n->nparam, 256), 256, 0, st>>>(n->w, n->m, n->v, n->grad, n->nparam, (float)tp->lr, b1, b2,
                                                             eps, c1, c2, 1.f / inbatch);
        TRYN(last_launch_status());
        count_launch();
        k_to_bf16<<<grid_for((int)n->nparam, 256), 256, 0, st>>>(n->w, n->wb, n->nparam);
        TRYN(last_launch_status());
        inbatch = 0;
      }
    }
  }
  if (losses)
    TRYN(cuda_status(cudaMemcpyAsync(losses, lossd, sizeof(double) * (size_t)npairs * tp->epochs, cudaMemcpyDeviceToHost, st)));
  TRYN(cuda_status(cudaStreamSynchronize(st)));
  return net_tc_status();
}

}  // extern "C"

namespace stag {
namespace netk {

__global__ void k_from_canonical_c64(Spinor<32> out, const float2* __restrict__ in) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < out.Vh; s += gridDim.x * blockDim.x) {
    float2 o[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) o[c] = in[(size_t)s * 3 + c];
    SpinorLoad<32>::st(out, s, o);
  }
}

int canon_to_sloppy(stag_lattice_s* lat, Spinor<32> out, const void* in, int in_prec, cudaStream_t st) {
  if (in_prec == STAG_FP64) return launch_from_canonical<32>(out, (const double2*)in, lat->g.Vh, st);
  ProfScope ps("convert", st);
  k_from_canonical_c64<<<grid_for(lat->g.Vh, 256), 256, 0, st>>>(out, (const float2*)in);
  return last_launch_status();
}

}  // namespace netk
}  // namespace stag

// ------------------------------------------------------------ flexible CG with the network
namespace stag {

struct FcgState {
  CgState cg;  // rr = ||r||^2 (sloppy), target, flags, iteration count, reliable updates
  double zap_re, zap_im;   // <Ap_prev, z>
  double beta_re, beta_im;
  double pr_re, pr_im;     // <p, r>
  double alpha_re, alpha_im;
  double pap_prev;
  int first;               // 1: no previous direction yet
};

namespace fcgk {

// beta = first ? 0 : <Ap_prev, z> / <p_prev, Ap_prev>
__global__ void k_fcg_beta(Spinor<32> Ap, Spinor<32> z, FcgState* fs, RedBuf rb) {
  if (stopped(&fs->cg.flags)) return;
  Acc1<float> re, im;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < z.Vh; s += gridDim.x * blockDim.x) {
    float2 a[3], b[3];
    SpinorLoad<32>::ld(Ap, s, a);
    SpinorLoad<32>::ld(z, s, b);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      re.add_prod(a[c].x, b[c].x);
      re.add_prod(a[c].y, b[c].y);
      im.add_prod(a[c].x, b[c].y);
      im.add_prod(-a[c].y, b[c].x);
    }
  }
  double v[2] = {re.value(), im.value()};
  grid_reduce<2>(v, rb, RedTarget{RED_STORE, nullptr, &fs->zap_re});
}

// p = z - beta p (beta from the <Ap_prev, z> just reduced), and <p, r>
template <int P>
__global__ void k_fcg_dir(Spinor<P> p, Spinor<32> z, Spinor<32> r, FcgState* fs, RedBuf rb) {
  if (stopped(&fs->cg.flags)) return;
  const bool first = __ldcg(&fs->first) != 0;
  double br = 0.0, bi = 0.0;
  if (!first) {
    const double pp = __ldcg(&fs->pap_prev);
    br = __ldcg(&fs->zap_re) / pp;
    bi = __ldcg(&fs->zap_im) / pp;
  }
  const float fr = (float)br, fi = (float)bi;
  Acc1<float> re, im;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < z.Vh; s += gridDim.x * blockDim.x) {
    float2 pv[3], zv[3], rv[3];
    SpinorLoad<P>::ldw(p, s, pv);
    SpinorLoad<32>::ld(z, s, zv);
    SpinorLoad<32>::ld(r, s, rv);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 o;
      o.x = zv[c].x - (fr * pv[c].x - fi * pv[c].y);
      o.y = zv[c].y - (fr * pv[c].y + fi * pv[c].x);
      if (first) o = zv[c];
      pv[c] = o;
    }
    SpinorLoad<P>::st(p, s, pv);
    SpinorLoad<P>::ldw(p, s, pv);  // the stored (rounded) direction enters the dot
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      re.add_prod(pv[c].x, rv[c].x);
      re.add_prod(pv[c].y, rv[c].y);
      im.add_prod(pv[c].x, rv[c].y);
      im.add_prod(-pv[c].y, rv[c].x);
    }
  }
  double v[2] = {re.value(), im.value()};
  grid_reduce<2>(v, rb, RedTarget{RED_STORE, nullptr, &fs->pr_re});
}

// alpha = <p, r> / <p, Ap> (pAp reduced by the operator epilogue into cg.pAp).
// <p, r> = <z, r> in exact arithmetic (r is orthogonal to the previous
// direction), so Re<p, r> <= 0 means N(r) is no descent direction: the
// network is not acting as a positive preconditioner and the solve is
// handed to the fallback at once.
__global__ void k_fcg_alpha(FcgState* fs) {
  if (stopped(&fs->cg.flags)) return;
  const double pap = fs->cg.pAp;
  if (!(pap > 0.0) || !isfinite(pap) || !(fs->pr_re > 0.0)) {
    fs->cg.flags |= F_BREAKDOWN;
    return;
  }
  fs->alpha_re = fs->pr_re / pap;
  fs->alpha_im = fs->pr_im / pap;
  fs->pap_prev = pap;
}

// x += alpha p; r -= alpha Ap; ||r||^2 -> iteration bookkeeping (RED_CG_BETA)
template <int P>
__global__ void k_fcg_update(Spinor<32> x, Spinor<32> r, Spinor<P> p, Spinor<32> Ap, FcgState* fs, RedBuf rb) {
  if (stopped(&fs->cg.flags)) return;
  const float ar = (float)__ldcg(&fs->alpha_re), ai = (float)__ldcg(&fs->alpha_im);
  Acc1<float> acc;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < x.Vh; s += gridDim.x * blockDim.x) {
    float2 xv[3], rv[3], pv[3], av[3];
    SpinorLoad<32>::ldw(x, s, xv);
    SpinorLoad<32>::ldw(r, s, rv);
    SpinorLoad<P>::ld(p, s, pv);
    SpinorLoad<32>::ld(Ap, s, av);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      xv[c].x += ar * pv[c].x - ai * pv[c].y;
      xv[c].y += ar * pv[c].y + ai * pv[c].x;
      rv[c].x -= ar * av[c].x - ai * av[c].y;
      rv[c].y -= ar * av[c].y + ai * av[c].x;
      acc.add_prod(rv[c].x, rv[c].x);
      acc.add_prod(rv[c].y, rv[c].y);
    }
    SpinorLoad<32>::st(x, s, xv);
    SpinorLoad<32>::st(r, s, rv);
  }
  double v[1] = {acc.value()};
  grid_reduce<1>(v, rb, RedTarget{RED_CG_BETA, &fs->cg, nullptr});
}

__global__ void k_fcg_clear_first(FcgState* fs) { fs->first = 0; }

int red_grid_n(int Vh, int cap) {
  int g = (Vh + 255) / 256;
  g = g < 608 ? g : 608;
  return g < cap ? g : cap;
}

}  // namespace fcgk
using namespace fcgk;

// Flexible CG (one-term truncation: each direction A-orthogonal to the
// previous one, which is what a preconditioner that changes from iteration
// to iteration requires) with z = N(r), sloppy operator of format P, FP32
// vectors, FP64 solution and reliable updates that restart the direction.
template <int P>
static int fcg_solve(stag_lattice_s* lat, stag_net_s* net, double2* x_can, const double2* b_can, double shift,
                     const stag_solve_params& prm, stag_solve_info* info, cudaStream_t st, int* fell_back) {
  const double t0 = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
  const int Vh = lat->g.Vh;
  int s = 0;
  Spinor<64> b64 = ws_spinor<64>(lat, "fcg.b", &s);
  Spinor<64> y64 = ws_spinor<64>(lat, "fcg.y", &s);
  Spinor<64> r64 = ws_spinor<64>(lat, "fcg.r64", &s);
  Spinor<64> t64 = ws_spinor<64>(lat, "fcg.t64", &s);
  Spinor<P> p = ws_spinor<P>(lat, "fcg.p", &s);
  Spinor<P> t = ws_spinor<P>(lat, "fcg.t", &s);
  Spinor<32> Ap = ws_spinor<32>(lat, "fcg.Ap", &s);
  Spinor<32> xh = ws_spinor<32>(lat, "fcg.xh", &s);
  Spinor<32> rh = ws_spinor<32>(lat, "fcg.rh", &s);
  Spinor<32> z = ws_spinor<32>(lat, "fcg.z", &s);
  FcgState* dst = (FcgState*)lat->ws.get("fcg.state", sizeof(FcgState), &s);
  double* dscal = (double*)lat->ws.get("fcg.scal", 64, &s);
  if (s) return s;
  RedScratch rs;
  TRYN(get_red_scratch(lat, "fcg", &rs));
  FcgState* hs = nullptr;
  if (cudaMallocHost(&hs, sizeof(FcgState) + 64) != cudaSuccess) {
    cudaGetLastError();
    return STAG_ENOMEM;
  }
  struct Free {
    void* p;
    ~Free() { cudaFreeHost(p); }
  } freer{hs};
  double* hscal = (double*)(hs + 1);
  NetRun R;
  TRYN(net_run_init(net, lat, R, false));

  auto true_residual = [&](RedTarget tgt) -> int {
    TRYN(launch_dslash<64>(lat, t64, y64, 1, nullptr, st));
    return launch_dslash_epi<64>(lat, r64, t64, 0, y64, -shift, b64, 1.0, 1.0, 2, rs, tgt, nullptr, st);
  };
  TRYN(launch_from_canonical<64>(b64, b_can, Vh, st));
  TRYN(launch_norm2<64>(b64, rs, RedTarget{RED_STORE, nullptr, dscal}, st));
  if (prm.use_initial_guess) {
    TRYN(launch_from_canonical<64>(y64, x_can, Vh, st));
  } else {
    TRYN(cuda_status(cudaMemsetAsync(y64.v, 0, spinor_bytes<64>(Vh), st)));
  }
  TRYN(true_residual(RedTarget{RED_STORE, nullptr, dscal + 1}));
  TRYN(cuda_status(cudaMemcpyAsync(hscal, dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st)));
  TRYN(cuda_status(cudaStreamSynchronize(st)));
  const double bb = hscal[0], rr0 = hscal[1];
  const double target = prm.tol * prm.tol * bb;
  FcgState h{};
  h.cg.rr = h.cg.rr_prev = h.cg.rr_max = h.cg.rr_true = rr0;
  h.cg.target = target;
  h.cg.delta2 = prm.delta * prm.delta;
  h.cg.shift = shift;
  h.cg.max_iter = prm.max_iter;
  h.first = 1;
  int status = STAG_OK;
  if (bb > 0.0 && rr0 > target && prm.max_iter > 0) {
    *hs = h;
    TRYN(cuda_status(cudaMemcpyAsync(dst, hs, sizeof(FcgState), cudaMemcpyHostToDevice, st)));
    TRYN(launch_convert<32, 64>(rh, r64, st));
    TRYN(cuda_status(cudaMemsetAsync(xh.v, 0, spinor_bytes<32>(Vh), st)));
    // short chunks: the network kernels do not read the stop flag
    const int C = prm.check_interval > 0 && prm.check_interval < 4 ? prm.check_interval : 4;
    const int* flags = &dst->cg.flags;
    const int G = red_grid_n(Vh, rs.max_grid);
    RedBuf rb{rs.partials, rs.counter};
    long long chunks = 0, max_chunks = (long long)prm.max_iter / C + 64;
    // stagnation guard: a preconditioner that stops the residual from falling
    // by 10x within 1000 iterations hands the system to the fallback
    double rr_mark = rr0;
    int it_mark = 0;
    for (;;) {
      if (++chunks > max_chunks) {
        status = STAG_ENOTCONV;
        break;
      }
      for (int i = 0; i < C; ++i) {
        TRYN(net_apply(net, lat, z, rh, &dst->cg.rr, st));
        count_launch();
        k_fcg_beta<<<G, 256, 0, st>>>(Ap, z, dst, rb);
        TRYN(last_launch_status());
        count_launch();
        k_fcg_dir<P><<<G, 256, 0, st>>>(p, z, rh, dst, rb);
        TRYN(last_launch_status());
        TRYN(launch_dslash<P>(lat, t, p, 1, flags, st));
        TRYN(launch_dslash_epi<P>(lat, Ap, t, 0, p, shift, Spinor<32>{nullptr, Vh}, 0.0, -1.0, 1, rs,
                                  RedTarget{RED_STORE, nullptr, &dst->cg.pAp}, flags, st));
        count_launch();
        k_fcg_alpha<<<1, 1, 0, st>>>(dst);
        TRYN(last_launch_status());
        count_launch();
        k_fcg_update<P><<<G, 256, 0, st>>>(xh, rh, p, Ap, dst, rb);
        TRYN(last_launch_status());
        count_launch();
        k_fcg_clear_first<<<1, 1, 0, st>>>(dst);
        TRYN(last_launch_status());
      }
      TRYN(cuda_status(cudaMemcpyAsync(hs, dst, sizeof(FcgState), cudaMemcpyDeviceToHost, st)));
      TRYN(cuda_status(cudaStreamSynchronize(st)));
      prof_flush_completed();
      TRYN(net_tc_status());
      if (hs->cg.flags & F_BREAKDOWN) {
        status = STAG_EBREAKDOWN;
        break;
      }
      if (hs->cg.rr < 0.01 * rr_mark) {
        rr_mark = hs->cg.rr;
        it_mark = hs->cg.iter;
      } else if (hs->cg.iter - it_mark > 1000) {
        status = STAG_ENOTCONV;
        break;
      }
      if (hs->cg.flags & (F_CONVERGED | F_NEED_RU | F_ITER_CAP)) {
        TRYN(launch_accumulate<32>(y64, xh, st));
        TRYN(true_residual(RedTarget{RED_RU_RESID, &dst->cg, nullptr}));
        // the direction is kept (as in CG's reliable update): the next one is
        // made A-orthogonal to it whatever the residual
        TRYN(launch_convert<32, 64>(rh, r64, st));
        TRYN(cuda_status(cudaMemcpyAsync(hs, dst, sizeof(FcgState), cudaMemcpyDeviceToHost, st)));
        TRYN(cuda_status(cudaStreamSynchronize(st)));
        if (hs->cg.flags & F_BREAKDOWN) {
          status = STAG_EBREAKDOWN;
          break;
        }
        if (hs->cg.rr_true <= target) break;
        if (hs->cg.iter >= prm.max_iter) {
          status = STAG_ENOTCONV;
          break;
        }
      }
    }
    h = *hs;
  }
  TRYN(launch_to_canonical<64>(x_can, y64, Vh, st));
  TRYN(cuda_status(cudaStreamSynchronize(st)));
  *fell_back = 0;
  if (status != STAG_OK) {
    // fallback: plain mixed CG from the last FCG solution
    stag_solve_params fp = prm;
    fp.mode = P == 15 ? STAG_MIXEDFX16 : STAG_MIXED32;
    fp.use_initial_guess = 1;
    fp.precond = nullptr;
    stag_solve_info fi{};
    const int its = h.cg.iter;
    status = stag_cg(lat, x_can, b_can, std::sqrt(shift), &fp, &fi, st);
    *fell_back = 1;
    if (info) {
      *info = fi;
      info->iters += its;
    }
    return status;
  }
  if (info) {
    info->iters = h.cg.iter;
    info->reliable_updates = h.cg.reliable_updates;
    info->true_rel_resid = bb > 0 ? std::sqrt(h.cg.rr_true / bb) : 0.0;
    info->converged = bb > 0 ? h.cg.rr_true <= target : 1;
    info->status = status;
    info->seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count() - t0;
  }
  return status;
}

int learned_solve(stag_lattice_s* lat, double2* x, const double2* b, double mass, const stag_solve_params& prm,
                  stag_solve_info* info, cudaStream_t st) {
  stag_net_s* net = (stag_net_s*)prm.precond;
  if (!net) return STAG_EINVAL;
  int fell = 0;
  int s;
  if (lat->links[STAG_FX16].present)
    s = fcg_solve<15>(lat, net, x, b, mass * mass, prm, info, st, &fell);
  else
    s = fcg_solve<32>(lat, net, x, b, mass * mass, prm, info, st, &fell);
  if (info) info->precond_fallback = fell;
  return s;
}

}  // namespace stag
