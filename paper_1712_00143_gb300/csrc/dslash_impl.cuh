// dslash_impl.cuh -- the improved-staggered hop kernel.
//
// Per output site x (one parity) the kernel sums 16 hops, each a 3x3 complex
// link times a neighbouring colour vector:
//   D psi(x) = sum_mu [ Wf_mu(x) psi(x+mu) + Wb_mu(x) psi(x-mu)
//                     + Nf_mu(x) psi(x+3mu) + Nb_mu(x) psi(x-3mu) ]
// with the staggered phase, the 1/2 and the backward minus sign already in
// W/N (see links.cu).  That is 16 x 66 + 15 x 6 = 1146 flop per site.
//
// Memory: the 16 link matrices of a site are read once per application and
// are the bulk of the traffic (288 reals per site, 240 with two-row Naik
// storage); the neighbour vectors are each re-read by up to 16 sites and
// mostly hit L2.  One thread owns one output site; links arrive as 128-bit
// loads of 16-byte chunks laid out [chunk][site] (coalesced), 16-bit
// neighbour vectors as one 128-bit record each, and neighbour indices are
// computed from the site's coordinates (no index table).
#pragma once
#include "internal.h"

namespace stag {

template <int P> struct DslashArgs {
  Geom g;
  int out_parity;
  const uint4* links;  // this parity's 16-byte chunks, [chunk][site]
  float fat_scale, long_scale;  // long_scale = c3/2 for two-row storage
  Spinor<P> in;
  int s_begin, s_end;  // output sites computed: [s_begin, s_end) (all: 0, Vh)
};

// The complex number k of a group of link chunks held in registers (k is a
// compile-time constant once the hop loops are unrolled).
template <int P, int NCH>
__device__ __forceinline__ typename Prec<P>::A2 cget(const uint4 (&buf)[NCH], int k) {
  return Chunk<P>::get(buf[k / Chunk<P>::PER], k % Chunk<P>::PER);
}

template <int NCH>
__device__ __forceinline__ void load_chunks(uint4 (&buf)[NCH], const uint4* __restrict__ L, int c0, int n, int Vh,
                                            int s) {
  s = STAG_BOUND(s, Vh, BOUND_LINK);
#pragma unroll
  for (int j = 0; j < NCH; ++j)
    if (j < n) buf[j] = __ldg(L + (size_t)(c0 + j) * Vh + s);
}

// acc += W psi, W = the 9 complex entries k0 .. k0+8 (row-major)
template <int P, int NCH, class A2>
__device__ __forceinline__ void hop_full(A2 acc[3], const uint4 (&buf)[NCH], int k0, const A2 psi[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) cmac(acc[i], cget<P>(buf, k0 + 3 * i + j), psi[j]);
}

// acc (+/-)= M psi with M in SU(3) from rows 0, 1 (entries k0 .. k0+5); row 2
// = conj(row0 x row1).
template <int P, int NCH, class A2>
__device__ __forceinline__ void hop_recon12(A2 acc[3], const uint4 (&buf)[NCH], int k0, const A2 psi[3],
                                            bool negate) {
  A2 m[6];
#pragma unroll
  for (int e = 0; e < 6; ++e) m[e] = cget<P>(buf, k0 + e);
  A2 t[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) t[i].x = t[i].y = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int k = (j + 1) % 3, l = (j + 2) % 3;
    A2 r2;
    r2.x = m[k].x * m[3 + l].x - m[k].y * m[3 + l].y - (m[l].x * m[3 + k].x - m[l].y * m[3 + k].y);
    r2.y = -(m[k].x * m[3 + l].y + m[k].y * m[3 + l].x - (m[l].x * m[3 + k].y + m[l].y * m[3 + k].x));
    cmac(t[0], m[j], psi[j]);
    cmac(t[1], m[3 + j], psi[j]);
    cmac(t[2], r2, psi[j]);
  }
  if (fixed_links(P)) {
    // rows hold integers 32767 * entry: row 2 (and so t[2]) comes out 32767 times too large
    t[2].x *= 1.0f / FX_ONE;
    t[2].y *= 1.0f / FX_ONE;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (negate) {
      acc[i].x -= t[i].x;
      acc[i].y -= t[i].y;
    } else {
      acc[i].x += t[i].x;
      acc[i].y += t[i].y;
    }
  }
}

// The four hops of direction mu whose entries start at k0 in buf.
template <int P, int NL, int NCH, class A2>
__device__ __forceinline__ void hops_mu(const DslashArgs<P>& a, int s, const Coord& c, int mu, const uint4 (&buf)[NCH],
                                        int k0, A2 accF[3], A2 accL[3]) {
  const Geom& g = a.g;
  A2 psi[3];
  SpinorLoad<P>::ld(a.in, cb_neighbour(g, s, c, mu, +1), psi);
  hop_full<P>(accF, buf, k0, psi);
  SpinorLoad<P>::ld(a.in, cb_neighbour(g, s, c, mu, -1), psi);
  hop_full<P>(accF, buf, k0 + 9, psi);
  SpinorLoad<P>::ld(a.in, cb_neighbour(g, s, c, mu, +3), psi);
  if (NL == 9) {
    hop_full<P>(accL, buf, k0 + 18, psi);
    SpinorLoad<P>::ld(a.in, cb_neighbour(g, s, c, mu, -3), psi);
    hop_full<P>(accL, buf, k0 + 27, psi);
  } else {
    // +-1/2 eta c3 is applied at the end: sign(eta) here, c3/2 in long_scale
    const bool neg = eta_bit(c, mu);
    hop_recon12<P>(accL, buf, k0 + 18, psi, neg);
    SpinorLoad<P>::ld(a.in, cb_neighbour(g, s, c, mu, -3), psi);
    hop_recon12<P>(accL, buf, k0 + 18 + NL, psi, !neg);
  }
}

// Link chunks are read in groups sized so that a group is a whole number of
// 16-byte chunks: one hop (FP64), one direction mu (FP32: 18 or 15 chunks),
// two directions (16-bit: 18 or 15 chunks).
template <int P, int NL>
__device__ __forceinline__ void dslash_site(const DslashArgs<P>& a, int s, typename Prec<P>::A2 out[3]) {
  using A2 = typename Prec<P>::A2;
  using A = typename Prec<P>::A;
  constexpr int CPM = 18 + 2 * NL;  // complex entries per direction
  const int Vh = a.g.Vh;
  Coord c = cb_coords(a.g, s, a.out_parity);
  A2 accF[3], accL[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    accF[i].x = accF[i].y = 0;
    accL[i].x = accL[i].y = 0;
  }
  if constexpr (P == 64) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const Geom& g = a.g;
      A2 psi[3];
      uint4 buf[9];
      const int cb = mu * CPM;
      load_chunks<9>(buf, a.links, cb, 9, Vh, s);
      SpinorLoad<P>::ld(a.in, cb_neighbour(g, s, c, mu, +1), psi);
      hop_full<P>(accF, buf, 0, psi);
      load_chunks<9>(buf, a.links, cb + 9, 9, Vh, s);
      SpinorLoad<P>::ld(a.in, cb_neighbour(g, s, c, mu, -1), psi);
      hop_full<P>(accF, buf, 0, psi);
      load_chunks<9>(buf, a.links, cb + 18, 9, Vh, s);
      SpinorLoad<P>::ld(a.in, cb_neighbour(g, s, c, mu, +3), psi);
      hop_full<P>(accL, buf, 0, psi);
      load_chunks<9>(buf, a.links, cb + 27, 9, Vh, s);
      SpinorLoad<P>::ld(a.in, cb_neighbour(g, s, c, mu, -3), psi);
      hop_full<P>(accL, buf, 0, psi);
    }
  } else if constexpr (Chunk<P>::PER == 2) {
    constexpr int NCH = CPM / 2;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      uint4 buf[NCH];
      load_chunks<NCH>(buf, a.links, mu * NCH, NCH, Vh, s);
      hops_mu<P, NL>(a, s, c, mu, buf, 0, accF, accL);
    }
  } else {
    constexpr int NCH = CPM / 2;  // two directions, 4 complex per chunk
#pragma unroll
    for (int mp = 0; mp < 2; ++mp) {
      uint4 buf[NCH];
      load_chunks<NCH>(buf, a.links, mp * NCH, NCH, Vh, s);
      hops_mu<P, NL>(a, s, c, 2 * mp, buf, 0, accF, accL);
      hops_mu<P, NL>(a, s, c, 2 * mp + 1, buf, CPM, accF, accL);
    }
  }
  const A fs = (A)a.fat_scale, ls = (A)a.long_scale;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    out[i].x = fs * accF[i].x + ls * accL[i].x;
    out[i].y = fs * accF[i].y + ls * accL[i].y;
  }
}

// Launch shapes the autotuner chooses among: threads per block and the
// minimum number of resident blocks per SM promised to the compiler (which
// caps registers per thread; 1 = no cap).
constexpr int kNumShapes = 4;
__host__ __device__ constexpr int shape_block(int v) { return v < 2 ? 256 : 128; }
__host__ __device__ constexpr int shape_minb(int v) { return v == 1 ? 4 : v == 3 ? 8 : 1; }

template <int P, int NL, int B, int MINB>
__global__ void __launch_bounds__(B, MINB) k_dslash(DslashArgs<P> a, Spinor<P> out, const int* flags) {
  if (stopped(flags)) return;
  int s = a.s_begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.s_end) return;
  typename Prec<P>::A2 d[3];
  dslash_site<P, NL>(a, s, d);
  SpinorLoad<P>::st(out, s, d);
}

// out = ax x + ay y + ad (D in), with an FP64 reduction of Re<x,out> (RED=1)
// or ||out||^2 (RED=2) finalised by the last block.
template <int P, int NL, int RED, int B, int MINB>
__global__ void __launch_bounds__(B, MINB)
    k_dslash_epi(DslashArgs<P> a, Spinor<Acc<P>::value> out, Spinor<P> x, double ax, Spinor<Acc<P>::value> y,
                 double ay, double ad, RedBuf rb, RedTarget tgt, const int* flags) {
  using A2 = typename Prec<P>::A2;
  using A = typename Prec<P>::A;
  if (stopped(flags)) return;
  int s = a.s_begin + blockIdx.x * blockDim.x + threadIdx.x;
  Acc1<A> red[1];
  if (s < a.s_end) {
    prefetch_spinor_l2<P>(x, s);  // read by the epilogue, after the stencil
    A2 d[3], xv[3], o[3];
    dslash_site<P, NL>(a, s, d);
    SpinorLoad<P>::ld(x, s, xv);
    const A cx = (A)ax, cd = (A)ad;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      o[i].x = cx * xv[i].x + cd * d[i].x;
      o[i].y = cx * xv[i].y + cd * d[i].y;
    }
    if (ay != 0.0) {
      A2 yv[3];
      SpinorLoad<Acc<P>::value>::ld(y, s, yv);
      const A cy = (A)ay;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        o[i].x += cy * yv[i].x;
        o[i].y += cy * yv[i].y;
      }
    }
    SpinorLoad<Acc<P>::value>::st(out, s, o);
    if (RED) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        red[0].add_prod(RED == 1 ? xv[i].x : o[i].x, o[i].x);
        red[0].add_prod(RED == 1 ? xv[i].y : o[i].y, o[i].y);
      }
    }
  }
  if (RED) grid_reduce_acc<1>(red, rb, tgt);
}

template <int P>
static DslashArgs<P> make_args(const stag_lattice_s* lat, Spinor<P> in, int out_parity) {
  const LinkCopy& L = lat->links[prec_index<P>()];
  DslashArgs<P> a;
  a.g = lat->g;
  a.out_parity = out_parity;
  a.links = (const uint4*)((const char*)L.data + (size_t)out_parity * L.parity_stride);
  const double fx = fixed_links(P) ? 1.0 / 32767.0 : 1.0;  // fixed point: integers -> entries
  a.fat_scale = (float)(L.fat_scale * fx);
  a.long_scale = (float)((L.nl == 6 ? 0.5 * lat->c3 : (double)L.long_scale) * fx);
  a.in = in;
  a.s_begin = 0;
  a.s_end = lat->g.Vh;
  return a;
}

template <int P, int NL>
static void dispatch_plain(int shape, const DslashArgs<P>& a, Spinor<P> out, const int* flags, cudaStream_t st) {
  const int Vh = a.s_end - a.s_begin;
#define STAG_PL(V)                                                                                \
  k_dslash<P, NL, shape_block(V), shape_minb(V)>                                                  \
      <<<(Vh + shape_block(V) - 1) / shape_block(V), shape_block(V), 0, st>>>(a, out, flags)
  switch (shape) {
    case 1: STAG_PL(1); break;
    case 2: STAG_PL(2); break;
    case 3: STAG_PL(3); break;
    default: STAG_PL(0);
  }
#undef STAG_PL
}

template <int P, int NL, int RED>
static void dispatch_epi(int shape, const DslashArgs<P>& a, Spinor<Acc<P>::value> out, Spinor<P> x, double ax,
                         Spinor<Acc<P>::value> y, double ay, double ad, RedBuf rb, RedTarget tgt, const int* flags,
                         cudaStream_t st) {
  const int Vh = a.s_end - a.s_begin;
#define STAG_EP(V)                                                                                \
  k_dslash_epi<P, NL, RED, shape_block(V), shape_minb(V)>                                         \
      <<<(Vh + shape_block(V) - 1) / shape_block(V), shape_block(V), 0, st>>>(a, out, x, ax, y, ay, ad, rb, tgt, flags)
  switch (shape) {
    case 1: STAG_EP(1); break;
    case 2: STAG_EP(2); break;
    case 3: STAG_EP(3); break;
    default: STAG_EP(0);
  }
#undef STAG_EP
}

template <int P>
static int plain_with_shape(const stag_lattice_s* lat, int shape, Spinor<P> out, Spinor<P> in, int out_parity,
                            const int* flags, cudaStream_t st, int s0 = 0, int s1 = -1) {
  const LinkCopy& L = lat->links[prec_index<P>()];
  DslashArgs<P> a = make_args<P>(lat, in, out_parity);
  if (s1 >= 0) {
    a.s_begin = s0;
    a.s_end = s1;
  }
  constexpr int NL2 = P == 64 ? 9 : 6;
  if (P == 64 || L.nl == 9)
    dispatch_plain<P, 9>(shape, a, out, flags, st);
  else
    dispatch_plain<P, NL2>(shape, a, out, flags, st);
  return last_launch_status();
}

template <int P>
static int epi_with_shape(const stag_lattice_s* lat, int shape, Spinor<Acc<P>::value> out, Spinor<P> in,
                          int out_parity, Spinor<P> x, double ax, Spinor<Acc<P>::value> y, double ay, double ad,
                          int red, RedScratch rs, RedTarget tgt, const int* flags, cudaStream_t st, int s0 = 0,
                          int s1 = -1) {
  const LinkCopy& L = lat->links[prec_index<P>()];
  DslashArgs<P> a = make_args<P>(lat, in, out_parity);
  if (s1 >= 0) {
    a.s_begin = s0;
    a.s_end = s1;
  }
  const int G = (a.s_end - a.s_begin + shape_block(shape) - 1) / shape_block(shape);
  if (red && G > rs.max_grid) return STAG_EINVAL;
  RedBuf rb{rs.partials, rs.counter};
  constexpr int NL2 = P == 64 ? 9 : 6;
  const bool r12 = P != 64 && L.nl == 6;
#define STAG_E(NL, R) dispatch_epi<P, NL, R>(shape, a, out, x, ax, y, ay, ad, rb, tgt, flags, st)
  if (r12) {
    if (red == 0) STAG_E(NL2, 0);
    else if (red == 1) STAG_E(NL2, 1);
    else STAG_E(NL2, 2);
  } else {
    if (red == 0) STAG_E(9, 0);
    else if (red == 1) STAG_E(9, 1);
    else STAG_E(9, 2);
  }
#undef STAG_E
  return last_launch_status();
}

template <int P>
int launch_dslash(const stag_lattice_s* lat, Spinor<P> out, Spinor<P> in, int out_parity, const int* flags,
                  cudaStream_t st) {
  const LinkCopy& L = lat->links[prec_index<P>()];
  if (!L.present) return STAG_EINVAL;
  ProfScope ps(P == 64 ? "dslash64" : "dslash", st);
  return plain_with_shape<P>(lat, L.shape_plain, out, in, out_parity, flags, st);
}

template <int P>
int launch_dslash_epi(const stag_lattice_s* lat, Spinor<Acc<P>::value> out, Spinor<P> in, int out_parity,
                      Spinor<P> x, double ax, Spinor<Acc<P>::value> y, double ay, double ad, int red,
                      RedScratch rs, RedTarget tgt, const int* flags, cudaStream_t st) {
  const LinkCopy& L = lat->links[prec_index<P>()];
  if (!L.present) return STAG_EINVAL;
  ProfScope ps(P == 64 ? "dslash64_epi" : "dslash_epi", st);
  return epi_with_shape<P>(lat, L.shape_epi, out, in, out_parity, x, ax, y, ay, ad, red, rs, tgt, flags, st);
}

// The same two kernels on the output sites [s0, s1) only (the interior of a
// rank's slab in the domain-decomposed operator, dd.cu).
template <int P>
int launch_dslash_range(const stag_lattice_s* lat, Spinor<P> out, Spinor<P> in, int out_parity, int s0, int s1,
                        const int* flags, cudaStream_t st) {
  const LinkCopy& L = lat->links[prec_index<P>()];
  if (!L.present || s0 < 0 || s1 > lat->g.Vh || s1 <= s0) return STAG_EINVAL;
  ProfScope ps(P == 64 ? "dslash64" : "dslash", st);
  return plain_with_shape<P>(lat, L.shape_plain, out, in, out_parity, flags, st, s0, s1);
}

template <int P>
int launch_dslash_epi_range(const stag_lattice_s* lat, Spinor<Acc<P>::value> out, Spinor<P> in, int out_parity,
                            Spinor<P> x, double ax, Spinor<Acc<P>::value> y, double ay, double ad, int red,
                            RedScratch rs, RedTarget tgt, int s0, int s1, const int* flags, cudaStream_t st) {
  const LinkCopy& L = lat->links[prec_index<P>()];
  if (!L.present || s0 < 0 || s1 > lat->g.Vh || s1 <= s0) return STAG_EINVAL;
  ProfScope ps(P == 64 ? "dslash64_epi" : "dslash_epi", st);
  return epi_with_shape<P>(lat, L.shape_epi, out, in, out_parity, x, ax, y, ay, ad, red, rs, tgt, flags, st, s0,
                           s1);
}

// Autotuner: times every launch shape of the plain and the fused-epilogue
// (dot-product) kernel on this lattice and precision, on scratch vectors,
// and keeps the fastest of each in the link copy.  Runs once per gauge field.
template <int P>
int tune_dslash(stag_lattice_s* lat, cudaStream_t st) {
  constexpr int PA = Acc<P>::value;
  LinkCopy& L = lat->links[prec_index<P>()];
  if (!L.present) return STAG_EINVAL;
  int s = 0;
  Spinor<P> in = ws_spinor<P>(lat, "tune.in", &s);
  Spinor<P> out = ws_spinor<P>(lat, "tune.out", &s);
  Spinor<PA> o = ws_spinor<PA>(lat, "tune.o", &s);
  double* scal = (double*)lat->ws.get("tune.scalar", 64, &s);
  if (s) return s;
  RedScratch rs;
  if ((s = get_red_scratch(lat, "tune", &rs))) return s;
  if ((s = cuda_status(cudaMemsetAsync(in.v, 0, spinor_bytes<P>(in.Vh), st)))) return s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return STAG_ECUDA;
  }
  const int reps = 5;
  float best[2] = {1e30f, 1e30f};
  int pick[2] = {0, 0};
  for (int kind = 0; kind < 2 && !s; ++kind) {
    for (int v = 0; v < kNumShapes && !s; ++v) {
      for (int it = -2; it < reps && !s; ++it) {
        if (it == 0) s = cuda_status(cudaEventRecord(e0, st));
        if (s) break;
        count_launch();
        s = kind == 0 ? plain_with_shape<P>(lat, v, out, in, 1, nullptr, st)
                      : epi_with_shape<P>(lat, v, o, out, 0, in, 1.0, Spinor<PA>{nullptr, in.Vh}, 0.0, -1.0, 1, rs,
                                          RedTarget{RED_STORE, nullptr, scal}, nullptr, st);
      }
      if (s) break;
      float ms = 0.f;
      if ((s = cuda_status(cudaEventRecord(e1, st)))) break;
      if ((s = cuda_status(cudaEventSynchronize(e1)))) break;
      if ((s = cuda_status(cudaEventElapsedTime(&ms, e0, e1)))) break;
      if (ms < best[kind]) {
        best[kind] = ms;
        pick[kind] = v;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  lat->ws.drop("tune.in");
  lat->ws.drop("tune.out");
  lat->ws.drop("tune.o");
  if (s) return s;
  L.shape_plain = pick[0];
  L.shape_epi = pick[1];
  L.tuned_us[0] = best[0] * 1e3f / reps;
  L.tuned_us[1] = best[1] * 1e3f / reps;
  return STAG_OK;
}

#define STAG_INSTANTIATE_DSLASH(P)                                                                          \
  template int launch_dslash<P>(const stag_lattice_s*, Spinor<P>, Spinor<P>, int, const int*, cudaStream_t); \
  template int launch_dslash_epi<P>(const stag_lattice_s*, Spinor<Acc<P>::value>, Spinor<P>, int, Spinor<P>, \
                                    double, Spinor<Acc<P>::value>, double, double, int, RedScratch, RedTarget, \
                                    const int*, cudaStream_t);                                              \
  template int tune_dslash<P>(stag_lattice_s*, cudaStream_t);                                                  \
  template int launch_dslash_range<P>(const stag_lattice_s*, Spinor<P>, Spinor<P>, int, int, int, const int*,    \
                                      cudaStream_t);                                                             \
  template int launch_dslash_epi_range<P>(const stag_lattice_s*, Spinor<Acc<P>::value>, Spinor<P>, int, Spinor<P>, \
                                          double, Spinor<Acc<P>::value>, double, double, int, RedScratch,          \
                                          RedTarget, int, int, const int*, cudaStream_t);

}  // namespace stag
