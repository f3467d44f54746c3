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
  } else if constexpr (P == 32) {
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

template <int P, int NL>
__global__ void __launch_bounds__(256) k_dslash(DslashArgs<P> a, Spinor<P> out, const int* flags) {
  if (stopped(flags)) return;
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.g.Vh) return;
  typename Prec<P>::A2 d[3];
  dslash_site<P, NL>(a, s, d);
  SpinorLoad<P>::st(out, s, d);
}

// out = ax x + ay y + ad (D in), with an FP64 reduction of Re<x,out> (RED=1)
// or ||out||^2 (RED=2) finalised by the last block.
template <int P, int NL, int RED>
__global__ void __launch_bounds__(256)
    k_dslash_epi(DslashArgs<P> a, Spinor<Acc<P>::value> out, Spinor<P> x, double ax, Spinor<Acc<P>::value> y,
                 double ay, double ad, RedBuf rb, RedTarget tgt, const int* flags) {
  using A2 = typename Prec<P>::A2;
  using A = typename Prec<P>::A;
  if (stopped(flags)) return;
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  double red[1] = {0.0};
  if (s < a.g.Vh) {
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
    if (RED == 1) {
#pragma unroll
      for (int i = 0; i < 3; ++i) red[0] += (double)xv[i].x * (double)o[i].x + (double)xv[i].y * (double)o[i].y;
    } else if (RED == 2) {
#pragma unroll
      for (int i = 0; i < 3; ++i) red[0] += (double)o[i].x * (double)o[i].x + (double)o[i].y * (double)o[i].y;
    }
  }
  if (RED) grid_reduce<1>(red, rb, tgt);
}

template <int P>
static DslashArgs<P> make_args(const stag_lattice_s* lat, Spinor<P> in, int out_parity) {
  const LinkCopy& L = lat->links[prec_index<P>()];
  DslashArgs<P> a;
  a.g = lat->g;
  a.out_parity = out_parity;
  a.links = (const uint4*)((const char*)L.data + (size_t)out_parity * L.parity_stride);
  a.fat_scale = L.fat_scale;
  a.long_scale = L.nl == 6 ? (float)(0.5 * lat->c3) : L.long_scale;
  a.in = in;
  return a;
}

template <int P>
int launch_dslash(const stag_lattice_s* lat, Spinor<P> out, Spinor<P> in, int out_parity, const int* flags,
                  cudaStream_t st) {
  const int pi = prec_index<P>();
  if (!lat->links[pi].present) return STAG_EINVAL;
  DslashArgs<P> a = make_args<P>(lat, in, out_parity);
  const int B = 256;
  const int G = (lat->g.Vh + B - 1) / B;
  ProfScope ps("dslash", st);
  if (P == 64 || lat->links[pi].nl == 9)
    k_dslash<P, 9><<<G, B, 0, st>>>(a, out, flags);
  else
    k_dslash<P, (P == 64 ? 9 : 6)><<<G, B, 0, st>>>(a, out, flags);
  return last_launch_status();
}

template <int P>
int launch_dslash_epi(const stag_lattice_s* lat, Spinor<Acc<P>::value> out, Spinor<P> in, int out_parity,
                      Spinor<P> x, double ax, Spinor<Acc<P>::value> y, double ay, double ad, int red,
                      RedScratch rs, RedTarget tgt, const int* flags, cudaStream_t st) {
  const int pi = prec_index<P>();
  if (!lat->links[pi].present) return STAG_EINVAL;
  DslashArgs<P> a = make_args<P>(lat, in, out_parity);
  const int B = 256;
  const int G = (lat->g.Vh + B - 1) / B;
  if (red && G > rs.max_grid) return STAG_EINVAL;
  RedBuf rb{rs.partials, rs.counter};
  ProfScope ps("dslash_epi", st);
  const bool r12 = P != 64 && lat->links[pi].nl == 6;
  constexpr int NL2 = P == 64 ? 9 : 6;
#define STAG_EPI(NL, R) k_dslash_epi<P, NL, R><<<G, B, 0, st>>>(a, out, x, ax, y, ay, ad, rb, tgt, flags)
  if (r12) {
    if (red == 0) STAG_EPI(NL2, 0);
    else if (red == 1) STAG_EPI(NL2, 1);
    else STAG_EPI(NL2, 2);
  } else {
    if (red == 0) STAG_EPI(9, 0);
    else if (red == 1) STAG_EPI(9, 1);
    else STAG_EPI(9, 2);
  }
#undef STAG_EPI
  return last_launch_status();
}

#define STAG_INSTANTIATE_DSLASH(P)                                                                          \
  template int launch_dslash<P>(const stag_lattice_s*, Spinor<P>, Spinor<P>, int, const int*, cudaStream_t); \
  template int launch_dslash_epi<P>(const stag_lattice_s*, Spinor<Acc<P>::value>, Spinor<P>, int, Spinor<P>, \
                                    double, Spinor<Acc<P>::value>, double, double, int, RedScratch, RedTarget, \
                                    const int*, cudaStream_t);

}  // namespace stag
