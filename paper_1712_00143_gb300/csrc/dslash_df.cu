// dslash_df.cu -- the FP64-class operator of the reliable updates, computed
// in double-float on the FP32 pipes (df.cuh), and the level-1 kernels around
// it.
//
// The mixed-precision solvers recompute the true residual r = b - M y of
// their FP64 solution y each time the iterated residual has dropped by delta
// (QUDA-style reliable updates; the paper notes QUDA's mixed-precision
// solvers, Sec. 3, and the staggered CG the whole benchmark rests on, Sec. 1
// and Sec. 4.1).  That residual needs FP64-class accuracy, but GB300 runs
// FP64 at about 1.1 TFLOP/s, so the FP64 Dslash pair of an update took
// 2.3 ms per launch at 32^4 with four right-hand sides.  Here the same pair
// runs on FP64-precision data (links split at load time into hi + lo
// floats, 16 bytes per complex like FP64) with double-float products and
// sums: about 48 significant bits, every link read once for up to four
// right-hand sides.
//
// Per output site and right-hand side: 16 hops x 9 complex multiply-adds of
// 48 FP32 operations (four TwoProd + TwoSum pairs, eight cross-term FMAs).
#include "df.cuh"
#include "dslash_mrhs.cuh"

namespace stag {

namespace {

constexpr int DFB = 128;  // threads per block of the hop kernels
constexpr int DFNB = 4;   // right-hand sides per hop launch (registers: 4 x 3 accumulators of 4 floats)

struct DfArgs {
  Geom g;
  int out_parity;
  const float4* links;  // DF link copy, this parity: 144 chunks of one complex, [chunk][site]
  const float4* in;     // NB systems [NB][Vh][3]
  float4* out;
  const float4* x;      // epilogue terms (may be null): out = ad D in + ax x + ay y
  const float4* y;
  float2 ax, ay;        // double-float scalars
  int neg_d;            // ad = -1 (else +1)
};

// SP threads share a site, each taking NB / SP of its right-hand sides (the
// link entries they both read come from L1 for all but the first): fewer
// accumulators per thread, more resident warps for the same work.
template <int NB, bool EPI, int SP>
__global__ void __launch_bounds__(DFB) k_dslash_df(DfArgs a, const int* stop) {
  static_assert(NB % SP == 0, "right-hand sides split evenly");
  if (stopped(stop)) return;
  constexpr int SPB = DFB / SP;  // sites per block
  const int part = threadIdx.x / SPB;
  const int s = blockIdx.x * SPB + (threadIdx.x - part * SPB);
  const int Vh = a.g.Vh;
  if (s >= Vh) return;
  const Coord c = cb_coords(a.g, s, a.out_parity);
  const size_t vs = (size_t)3 * Vh;  // float4 per system
  {
    const size_t off = (size_t)part * (NB / SP) * vs;
    a.in += off;
    a.out += off;
    if (a.x) a.x += off;
    if (a.y) a.y += off;
  }
  constexpr int NT = NB / SP;  // right-hand sides of this thread
  float4 acc[NT][3];
#pragma unroll
  for (int r = 0; r < NT; ++r)
#pragma unroll
    for (int i = 0; i < 3; ++i) acc[r][i] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      // hop order of the link layout: +mu, -mu (fat), +3mu, -3mu (Naik)
      const int k = h == 0 ? 1 : h == 1 ? -1 : h == 2 ? 3 : -3;
      const int nb = cb_neighbour(a.g, s, c, mu, k);
      const float4* L = a.links + (size_t)(mu * 36 + h * 9) * Vh + STAG_BOUND(s, Vh, BOUND_LINK);
      const float4* pin = a.in + 3 * (size_t)nb;
      // column by column: one link column (3 entries) and one colour
      // component of each right-hand side live at a time (register budget)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float4 w0 = __ldg(L + (size_t)j * Vh), w1 = __ldg(L + (size_t)(3 + j) * Vh),
                     w2 = __ldg(L + (size_t)(6 + j) * Vh);
#pragma unroll
        for (int r = 0; r < NT; ++r) {
          const float4 v = __ldg(pin + r * vs + j);
          dfc_mac(acc[r][0], w0, v);
          dfc_mac(acc[r][1], w1, v);
          dfc_mac(acc[r][2], w2, v);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < NT; ++r) {
    const size_t o = r * vs + 3 * (size_t)s;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float4 v = acc[r][i];
      if (EPI) {
        if (a.neg_d) v = make_float4(-v.x, -v.y, -v.z, -v.w);
        if (a.x) dfc_axpy(v, a.ax, __ldg(a.x + o + i));
        if (a.y) dfc_axpy(v, a.ay, __ldg(a.y + o + i));
      }
      a.out[o + i] = dfc_norm(v);
    }
  }
}

float2 df_scalar(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

// Launch variants: threads per site sharing the right-hand sides of a
// launch (SP), chosen per lattice by tune_df.
constexpr int kDfSplits[] = {1, 2, 4};
constexpr int kNumDfVariants = 3;

template <bool EPI, int SP>
void launch_hop(int nb, int G, const DfArgs& a, const int* stop, cudaStream_t st) {
  switch (nb) {
    case 1: k_dslash_df<1, EPI, 1><<<G, DFB, 0, st>>>(a, stop); break;
    case 2: k_dslash_df<2, EPI, SP <= 2 ? SP : 2><<<G, DFB, 0, st>>>(a, stop); break;
    case 3: k_dslash_df<3, EPI, 1><<<G, DFB, 0, st>>>(a, stop); break;
    default: k_dslash_df<4, EPI, SP><<<G, DFB, 0, st>>>(a, stop);
  }
}

template <bool EPI>
int hop_launches(const stag_lattice_s* lat, DfField out, DfField in, int n, int out_parity, DfField x, double ax,
                 DfField y, double ay, double ad, const int* stop, cudaStream_t st, int variant = -1) {
  const LinkCopy& L = lat->links[STAG_DF64];
  if (!L.present || n < 1) return STAG_EINVAL;
  DfArgs a;
  a.g = lat->g;
  a.out_parity = out_parity;
  a.links = (const float4*)((const char*)L.data + (size_t)out_parity * L.parity_stride);
  a.ax = df_scalar(ax);
  a.ay = df_scalar(ay);
  a.neg_d = ad < 0.0;
  const int Vh = lat->g.Vh;
  const size_t vs = (size_t)3 * Vh;
  const int v = variant >= 0 ? variant : L.shape_plain;
  for (int r0 = 0; r0 < n; r0 += DFNB) {
    const int nb = n - r0 < DFNB ? n - r0 : DFNB;
    // threads per site actually used for this many right-hand sides
    const int sp = (nb == 4) ? kDfSplits[v] : (nb == 2 && kDfSplits[v] >= 2) ? 2 : 1;
    const int G = (Vh + DFB / sp - 1) / (DFB / sp);
    a.in = in.v + r0 * vs;
    a.out = out.v + r0 * vs;
    a.x = x.v ? x.v + r0 * vs : nullptr;
    a.y = y.v ? y.v + r0 * vs : nullptr;
    ProfScope ps(EPI ? "dslash_df_epi" : "dslash_df", st);
    switch (kDfSplits[v]) {
      case 4: launch_hop<EPI, 4>(nb, G, a, stop, st); break;
      case 2: launch_hop<EPI, 2>(nb, G, a, stop, st); break;
      default: launch_hop<EPI, 1>(nb, G, a, stop, st);
    }
    const int s = last_launch_status();
    if (s) return s;
  }
  return STAG_OK;
}

// ------------------------------------------------------------ level 1
#define DGRID(s, Vh) for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < (Vh); s += gridDim.x * blockDim.x)

int sm_count_df() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
    else {
      cudaGetLastError();
      n = 152;
    }
  }
  return n;
}
int grid_bw_df(int Vh) {
  const int g = (Vh + 255) / 256, m = 8 * sm_count_df();
  return g < m ? g : m;
}
int grid_red_df(int Vh, int cap) {
  int g = (Vh + 255) / 256, m = 4 * sm_count_df();
  g = g < m ? g : m;
  return g < cap ? g : cap;
}

// DF fields of n systems from FP64 [n][Vh][3] (exact split, df_split)
__global__ void k_df_from_double(float4* __restrict__ out, const double2* __restrict__ in, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = dfc_from_double2(in[i]);
}
__global__ void k_df_to_double(double2* __restrict__ out, const float4* __restrict__ in, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = dfc_to_double2(in[i]);
}

// y_r += xh_r (FP64 accumulation of the solution), xh_r = 0, and the
// double-float distance from the anchor, ydf_r = split(y_r - ya_r) (ya null:
// the anchor is 0)
template <int PV, int N>
__global__ void k_accumulate_df(SpinorM<64> y, SpinorM<PV> xh, float4* __restrict__ ydf,
                                const double2* __restrict__ ya, const int* stop) {
  if (stopped(stop)) return;
  DGRID(s, y.Vh) {
#pragma unroll
    for (int r = 0; r < N; ++r) {
      double2 a[3];
      typename Prec<PV>::A2 b[3], z[3];
      SpinorLoadM<64>::ldw(y, s, r, a);
      SpinorLoadM<PV>::ldw(xh, s, r, b);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        a[c].x += (double)b[c].x;
        a[c].y += (double)b[c].y;
        z[c].x = 0;
        z[c].y = 0;
        const size_t i = ((size_t)r * y.Vh + s) * 3 + c;
        double2 d = a[c];
        if (ya) {
          const double2 q = __ldg(ya + i);
          d.x -= q.x;
          d.y -= q.y;
        }
        ydf[i] = dfc_from_double2(d);
      }
      SpinorLoadM<64>::st(y, s, r, a);
      SpinorLoadM<PV>::st(xh, s, r, z);
    }
  }
}

// The anchor moves to the current solution: ya = y, ra = split(r) (FP64
// fields of n systems, [n][Vh][3]).
__global__ void k_df_anchor(double2* __restrict__ ya, float4* __restrict__ ra, const double2* __restrict__ y,
                            const double2* __restrict__ r, size_t count, const int* stop) {
  if (stopped(stop)) return;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    ya[i] = __ldg(y + i);
    ra[i] = dfc_from_double2(__ldg(r + i));
  }
}

// rh_r = r_r rounded to the Krylov loop's precision; ||r_r||^2 (of the
// double-float r, FP64-class) and <rh_r, p_r> -> RED_RU_BOTH (one system,
// CgState) or RED_MCG_RU_BOTH (a group).
template <int P, int N>
__global__ void k_ru_convert_dot_df(SpinorM<Acc<P>::value> rh, const float4* __restrict__ r, SpinorM<P> p,
                                    RedBuf rb, RedTarget tgt, const int* stop) {
  constexpr int PV = Acc<P>::value;
  using A2 = typename Prec<PV>::A2;
  using A = typename Prec<PV>::A;
  if (stopped(stop)) return;  // every block alike: no partial reduction is left behind
  Acc1<A> nn[N], re[N], im[N];
  DGRID(s, rh.Vh) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      A2 o[3];
      typename Prec<P>::A2 pv[3];
      SpinorLoadM<P>::ld(p, s, k, pv);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4 d = __ldg(r + ((size_t)k * rh.Vh + s) * 3 + c);
        const float2 v = dfc_to_float2(d);
        o[c].x = v.x;
        o[c].y = v.y;
        // ||r||^2 of the double-float residual itself: (h + l)^2 = h^2 (exact
        // product into the accumulator) + 2 h l (l^2 is below its precision)
        nn[k].add_prod(d.x, d.x);
        nn[k].add_prod(d.y, d.y);
        nn[k].v.lo = fmaf(2.f * d.x, d.z, nn[k].v.lo);
        nn[k].v.lo = fmaf(2.f * d.y, d.w, nn[k].v.lo);
      }
      SpinorLoadM<PV>::st(rh, s, k, o);
      // the stored (rounded) rh enters <rh, p>, as it will enter p
      SpinorLoadM<PV>::ldw(rh, s, k, o);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        re[k].add_prod(o[c].x, (A)pv[c].x);
        re[k].add_prod(o[c].y, (A)pv[c].y);
        im[k].add_prod(o[c].x, (A)pv[c].y);
        im[k].add_prod(-o[c].y, (A)pv[c].x);
      }
    }
  }
  Acc1<A> all[3 * N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    all[k] = nn[k];
    all[N + 2 * k] = re[k];
    all[N + 2 * k + 1] = im[k];
  }
  grid_reduce_acc<3 * N>(all, rb, tgt);
}

// ||v_r||^2 of DF fields, FP64-class: (h + l)^2 = h^2 + 2 h l -> tgt
template <int N> __global__ void k_norm2_df(const float4* __restrict__ v, int Vh, RedBuf rb, RedTarget tgt) {
  Acc1<float> acc[N];
  DGRID(s, Vh) {
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4 d = __ldg(v + ((size_t)k * Vh + s) * 3 + c);
        acc[k].add_prod(d.x, d.x);
        acc[k].add_prod(d.y, d.y);
        acc[k].v.lo = fmaf(2.f * d.x, d.z, acc[k].v.lo);
        acc[k].v.lo = fmaf(2.f * d.y, d.w, acc[k].v.lo);
      }
  }
  grid_reduce_acc<N>(acc, rb, tgt);
}

// Krylov-loop fields of n systems from DF fields (rounded to the nearest float)
template <int PV, int N> __global__ void k_convert_from_df(SpinorM<PV> out, const float4* __restrict__ in) {
  DGRID(s, out.Vh) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      typename Prec<PV>::A2 o[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4 v = __ldg(in + ((size_t)k * out.Vh + s) * 3 + c);
        if constexpr (PV == 64) {
          o[c] = dfc_to_double2(v);
        } else {
          const float2 f = dfc_to_float2(v);
          o[c].x = f.x;
          o[c].y = f.y;
        }
      }
      SpinorLoadM<PV>::st(out, s, k, o);
    }
  }
}

#undef DGRID

}  // namespace

int launch_dslash_df(const stag_lattice_s* lat, DfField out, DfField in, int n, int out_parity, const int* stop,
                     cudaStream_t st) {
  return hop_launches<false>(lat, out, in, n, out_parity, DfField{nullptr, in.Vh}, 0.0, DfField{nullptr, in.Vh}, 0.0,
                             1.0, stop, st);
}

int launch_dslash_df_epi(const stag_lattice_s* lat, DfField out, DfField in, int n, int out_parity, DfField x,
                         double ax, DfField y, double ay, double ad, const int* stop, cudaStream_t st) {
  if (!(ad == 1.0 || ad == -1.0)) return STAG_EINVAL;
  return hop_launches<true>(lat, out, in, n, out_parity, x, ax, y, ay, ad, stop, st);
}

// Times the launch variants of the double-float hop kernels (four
// right-hand sides, the plain and the epilogue form) on this lattice and
// keeps the fastest.  Runs once per gauge field, from stag_load_links.
int tune_df(stag_lattice_s* lat, cudaStream_t st) {
  LinkCopy& L = lat->links[STAG_DF64];
  if (!L.present) return STAG_EINVAL;
  const int Vh = lat->g.Vh;
  int s = 0;
  DfField a{(float4*)lat->ws.get("tunedf.a", df_bytes(Vh) * DFNB, &s), Vh};
  DfField b{(float4*)lat->ws.get("tunedf.b", df_bytes(Vh) * DFNB, &s), Vh};
  if (s) return s;
  if ((s = cuda_status(cudaMemsetAsync(a.v, 0, df_bytes(Vh) * DFNB, st)))) return s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return STAG_ECUDA;
  }
  const int reps = 3;
  float best = 1e30f;
  int pick = 0;
  for (int v = 0; v < kNumDfVariants && !s; ++v) {
    for (int it = -1; it < reps && !s; ++it) {
      if (it == 0) s = cuda_status(cudaEventRecord(e0, st));
      if (!s) s = hop_launches<false>(lat, b, a, DFNB, 1, DfField{nullptr, Vh}, 0.0, DfField{nullptr, Vh}, 0.0, 1.0,
                                      nullptr, st, v);
      if (!s) s = hop_launches<true>(lat, a, b, DFNB, 0, b, 1.0, DfField{nullptr, Vh}, 0.0, 1.0, nullptr, st, v);
    }
    float ms = 0.f;
    if (!s) s = cuda_status(cudaEventRecord(e1, st));
    if (!s) s = cuda_status(cudaEventSynchronize(e1));
    if (!s) s = cuda_status(cudaEventElapsedTime(&ms, e0, e1));
    if (!s && ms < best) {
      best = ms;
      pick = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  lat->ws.drop("tunedf.a");
  lat->ws.drop("tunedf.b");
  if (s) return s;
  L.shape_plain = L.shape_epi = pick;
  L.tuned_us[0] = L.tuned_us[1] = best * 1e3f / (2 * reps);
  return STAG_OK;
}

int launch_df_from_double(DfField out, const double2* in, int n, cudaStream_t st) {
  const size_t count = (size_t)3 * out.Vh * n;
  ProfScope ps("convert", st);
  k_df_from_double<<<grid_bw_df(out.Vh * n), 256, 0, st>>>(out.v, in, count);
  return last_launch_status();
}

int launch_df_to_double(double2* out, DfField in, int n, cudaStream_t st) {
  const size_t count = (size_t)3 * in.Vh * n;
  ProfScope ps("convert", st);
  k_df_to_double<<<grid_bw_df(in.Vh * n), 256, 0, st>>>(out, in.v, count);
  return last_launch_status();
}

template <int PV>
int launch_accumulate_df(void* y64, void* xh, DfField ydf, const void* ya, int n, const int* stop, cudaStream_t st) {
  const int Vh = ydf.Vh;
  SpinorM<64> y{y64, Vh, n};
  SpinorM<PV> x{xh, Vh, n};
  const double2* a = (const double2*)ya;
  ProfScope ps("blas", st);
  const int G = grid_bw_df(Vh);
  switch (n) {
    case 1: k_accumulate_df<PV, 1><<<G, 256, 0, st>>>(y, x, ydf.v, a, stop); break;
    case 2: k_accumulate_df<PV, 2><<<G, 256, 0, st>>>(y, x, ydf.v, a, stop); break;
    case 4: k_accumulate_df<PV, 4><<<G, 256, 0, st>>>(y, x, ydf.v, a, stop); break;
    case 8: k_accumulate_df<PV, 8><<<G, 256, 0, st>>>(y, x, ydf.v, a, stop); break;
    default: return STAG_EINVAL;
  }
  return last_launch_status();
}

int launch_df_anchor(void* ya, DfField ra, const void* y, const void* r, int n, const int* stop, cudaStream_t st) {
  const size_t count = (size_t)3 * ra.Vh * n;
  ProfScope ps("blas", st);
  k_df_anchor<<<grid_bw_df(ra.Vh * n), 256, 0, st>>>((double2*)ya, ra.v, (const double2*)y, (const double2*)r, count,
                                                       stop);
  return last_launch_status();
}

template <int P>
int launch_ru_convert_dot_df(void* rh, DfField r, const void* p, int n, RedScratch rs, RedTarget tgt, const int* stop,
                             cudaStream_t st) {
  constexpr int PV = Acc<P>::value;
  const int Vh = r.Vh;
  SpinorM<PV> o{rh, Vh, n};
  SpinorM<P> pp{const_cast<void*>(p), Vh, n};
  RedBuf rb{rs.partials, rs.counter};
  ProfScope ps("reduce", st);
  const int G = grid_red_df(Vh, rs.max_grid);
  switch (n) {
    case 1: k_ru_convert_dot_df<P, 1><<<G, 256, 0, st>>>(o, r.v, pp, rb, tgt, stop); break;
    case 2: k_ru_convert_dot_df<P, 2><<<G, 256, 0, st>>>(o, r.v, pp, rb, tgt, stop); break;
    case 4: k_ru_convert_dot_df<P, 4><<<G, 256, 0, st>>>(o, r.v, pp, rb, tgt, stop); break;
    case 8: k_ru_convert_dot_df<P, 8><<<G, 256, 0, st>>>(o, r.v, pp, rb, tgt, stop); break;
    default: return STAG_EINVAL;
  }
  return last_launch_status();
}

int launch_norm2_df(DfField v, int n, RedScratch rs, RedTarget tgt, cudaStream_t st) {
  RedBuf rb{rs.partials, rs.counter};
  ProfScope ps("reduce", st);
  const int G = grid_red_df(v.Vh, rs.max_grid);
  switch (n) {
    case 1: k_norm2_df<1><<<G, 256, 0, st>>>(v.v, v.Vh, rb, tgt); break;
    case 2: k_norm2_df<2><<<G, 256, 0, st>>>(v.v, v.Vh, rb, tgt); break;
    case 4: k_norm2_df<4><<<G, 256, 0, st>>>(v.v, v.Vh, rb, tgt); break;
    case 8: k_norm2_df<8><<<G, 256, 0, st>>>(v.v, v.Vh, rb, tgt); break;
    default: return STAG_EINVAL;
  }
  return last_launch_status();
}

template <int PV> int launch_convert_from_df(void* out, DfField in, int n, cudaStream_t st) {
  SpinorM<PV> o{out, in.Vh, n};
  ProfScope ps("convert", st);
  const int G = grid_bw_df(in.Vh);
  switch (n) {
    case 1: k_convert_from_df<PV, 1><<<G, 256, 0, st>>>(o, in.v); break;
    case 2: k_convert_from_df<PV, 2><<<G, 256, 0, st>>>(o, in.v); break;
    case 4: k_convert_from_df<PV, 4><<<G, 256, 0, st>>>(o, in.v); break;
    case 8: k_convert_from_df<PV, 8><<<G, 256, 0, st>>>(o, in.v); break;
    default: return STAG_EINVAL;
  }
  return last_launch_status();
}

template int launch_accumulate_df<32>(void*, void*, DfField, const void*, int, const int*, cudaStream_t);
template int launch_ru_convert_dot_df<32>(void*, DfField, const void*, int, RedScratch, RedTarget, const int*,
                                          cudaStream_t);
template int launch_ru_convert_dot_df<16>(void*, DfField, const void*, int, RedScratch, RedTarget, const int*,
                                          cudaStream_t);
template int launch_ru_convert_dot_df<15>(void*, DfField, const void*, int, RedScratch, RedTarget, const int*,
                                          cudaStream_t);
template int launch_ru_convert_dot_df<31>(void*, DfField, const void*, int, RedScratch, RedTarget, const int*,
                                          cudaStream_t);
template int launch_convert_from_df<32>(void*, DfField, int, cudaStream_t);
template int launch_convert_from_df<64>(void*, DfField, int, cudaStream_t);

}  // namespace stag
