// dslash_mrhs.cuh -- the hop kernel for N right-hand sides at once.
//
// Same operator as dslash_impl.cuh; one thread owns one output site and all N
// right-hand sides, so each link chunk is loaded and decoded once and used N
// times (the links are the bulk of the single-RHS traffic).  Per site and
// right-hand side the algorithmic bytes fall from 16 links + 2 vectors to
// 16 links / N + 2 vectors.
//
// Multi-RHS vector layout ("MRHS"): the N vectors one after the other, each
// in the single-vector layout of its format (FP32: [3][Vh]; 16 bit: [Vh]
// records; FP64: [Vh][3]), so that for a fixed right-hand side a warp's loads
// over 32 consecutive sites stay coalesced.
#pragma once
#include "dslash_impl.cuh"

namespace stag {

template <int P> struct SpinorM {
  void* v;
  int Vh;
  int n;  // right-hand sides per site
};

template <int P> __host__ __device__ inline size_t spinorm_bytes(int Vh, int n) {
  return spinor_bytes<P>(Vh) * (size_t)n;
}

template <int P> struct SpinorLoadM {
  using A2 = typename Prec<P>::A2;
  static __device__ __forceinline__ Spinor<P> one(const SpinorM<P>& f, int r) {
    return Spinor<P>{(char*)f.v + spinor_bytes<P>(f.Vh) * r, f.Vh};
  }
  static __device__ __forceinline__ void ld(const SpinorM<P>& f, int s, int r, A2 o[3]) {
    SpinorLoad<P>::ld(one(f, r), s, o);
  }
  static __device__ __forceinline__ void ldw(const SpinorM<P>& f, int s, int r, A2 o[3]) {
    SpinorLoad<P>::ldw(one(f, r), s, o);
  }
  static __device__ __forceinline__ void st(const SpinorM<P>& f, int s, int r, const A2 o[3]) {
    SpinorLoad<P>::st(one(f, r), s, o);
  }
};

// The N-right-hand-side operator halves (mrhs_kernels.cuh; instantiated in
// mrhs64.cu, mrhs32.cu, mrhs16.cu, mrhs15.cu): out = D in on parity
// out_parity, and out = ax x + ay y + ad D in with an optional per-system
// reduction (RED 1: Re<x, out>, 2: ||out||^2), in the launch variant the
// autotuner chose for (P, N) on this lattice (tune_mrhs).
template <int P, int N>
int mdslash(const stag_lattice_s* lat, SpinorM<P> out, SpinorM<P> in, int out_parity, const int* flags,
            cudaStream_t st);
template <int P, int N, int RED>
int mdslash_epi(const stag_lattice_s* lat, SpinorM<Acc<P>::value> out, SpinorM<P> in, int out_parity, SpinorM<P> x,
                double ax, SpinorM<Acc<P>::value> y, double ay, double ad, RedScratch rs, RedTarget tgt,
                const int* flags, cudaStream_t st);
template <int P, int N> int tune_mrhs(stag_lattice_s* lat, cudaStream_t st);
// <p_r, Ap_r> -> RED_MCG_ALPHA from the per-site values of mdslash_epi<P, N, 3>
template <int P, int N>
int launch_mcg_alpha_pt(const stag_lattice_s* lat, const float* pt, McgState* g, RedScratch rs, cudaStream_t st);

template <int P> struct DslashArgsM {
  Geom g;
  int out_parity;
  const uint4* links;
  float fat_scale, long_scale;
  SpinorM<P> in;
};

// Loads the chunks holding the complex entries [k0, k0 + NE) of one hop and
// only those (never past the hop's last chunk); returns the offset of entry
// k0 inside the first chunk.  k0 is a compile-time constant once the
// direction loop is unrolled, so the bounds fold away.
template <int P, int NE, int NCMAX>
__device__ __forceinline__ int load_hop(uint4 (&b)[NCMAX], const uint4* __restrict__ L, int k0, int Vh, int s) {
  constexpr int PER = Chunk<P>::PER;
  const int c0 = k0 / PER, c1 = (k0 + NE - 1) / PER;
  s = STAG_BOUND(s, Vh, BOUND_LINK);
#pragma unroll
  for (int j = 0; j < NCMAX; ++j)
    if (c0 + j <= c1) b[j] = __ldg(L + (size_t)(c0 + j) * Vh + s);
  return k0 % PER;
}

// acc[r] += k W psi_r for every right-hand side; W = full 3x3 at offset off
// in buf, k the field's scale (applied once per entry, not per right-hand side).
template <int P, int N, int NCH, class A2, class A>
__device__ __forceinline__ void hop_full_m(A2 (&acc)[N][3], const uint4 (&buf)[NCH], int off,
                                           const SpinorM<P>& in, int nb, A k) {
  A2 w[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    w[e] = cget<P>(buf, off + e);
    w[e].x *= k;
    w[e].y *= k;
  }
#pragma unroll
  for (int r = 0; r < N; ++r) {
    A2 psi[3];
    SpinorLoadM<P>::ld(in, nb, r, psi);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) cmac(acc[r][i], w[3 * i + j], psi[j]);
  }
}

template <int P, int N, int NCH, class A2, class A>
__device__ __forceinline__ void hop_recon12_m(A2 (&acc)[N][3], const uint4 (&buf)[NCH], int off,
                                              const SpinorM<P>& in, int nb, bool negate, A k) {
  A2 m[9];
#pragma unroll
  for (int e = 0; e < 6; ++e) m[e] = cget<P>(buf, off + e);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int k = (j + 1) % 3, l = (j + 2) % 3;
    A2 r2;
    r2.x = m[k].x * m[3 + l].x - m[k].y * m[3 + l].y - (m[l].x * m[3 + k].x - m[l].y * m[3 + k].y);
    r2.y = -(m[k].x * m[3 + l].y + m[k].y * m[3 + l].x - (m[l].x * m[3 + k].y + m[l].y * m[3 + k].x));
    if (fixed_links(P)) {
      r2.x *= 1.0f / FX_ONE;
      r2.y *= 1.0f / FX_ONE;
    }
    m[6 + j] = r2;
  }
  const A kk = negate ? -k : k;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    m[e].x *= kk;
    m[e].y *= kk;
  }
#pragma unroll
  for (int r = 0; r < N; ++r) {
    A2 psi[3];
    SpinorLoadM<P>::ld(in, nb, r, psi);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) cmac(acc[r][i], m[3 * i + j], psi[j]);
  }
}

template <int P, int NL, int N>
__device__ __forceinline__ void dslash_site_m(const DslashArgsM<P>& a, int s, typename Prec<P>::A2 (&out)[N][3]) {
  using A2 = typename Prec<P>::A2;
  using A = typename Prec<P>::A;
  constexpr int CPM = 18 + 2 * NL;
  const Geom& g = a.g;
  const int Vh = g.Vh;
  Coord c = cb_coords(g, s, a.out_parity);
  const A fs = (A)a.fat_scale, ls = (A)a.long_scale;
#pragma unroll
  for (int r = 0; r < N; ++r)
#pragma unroll
    for (int i = 0; i < 3; ++i) out[r][i].x = out[r][i].y = 0;
  constexpr int PER = Chunk<P>::PER;
  constexpr int NC9 = (9 + PER - 1) / PER + 1;
  constexpr int NCL = (NL + PER - 1) / PER + 1;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int kb = mu * CPM;
    {
      uint4 b[NC9];
      const int off = load_hop<P, 9>(b, a.links, kb, Vh, s);
      hop_full_m<P, N>(out, b, off, a.in, cb_neighbour(g, s, c, mu, +1), fs);
    }
    {
      uint4 b[NC9];
      const int off = load_hop<P, 9>(b, a.links, kb + 9, Vh, s);
      hop_full_m<P, N>(out, b, off, a.in, cb_neighbour(g, s, c, mu, -1), fs);
    }
    {
      uint4 b[NCL];
      const int off = load_hop<P, NL>(b, a.links, kb + 18, Vh, s);
      if (NL == 9)
        hop_full_m<P, N>(out, b, off, a.in, cb_neighbour(g, s, c, mu, +3), ls);
      else
        hop_recon12_m<P, N>(out, b, off, a.in, cb_neighbour(g, s, c, mu, +3), eta_bit(c, mu), ls);
    }
    {
      uint4 b[NCL];
      const int off = load_hop<P, NL>(b, a.links, kb + 18 + NL, Vh, s);
      if (NL == 9)
        hop_full_m<P, N>(out, b, off, a.in, cb_neighbour(g, s, c, mu, -3), ls);
      else
        hop_recon12_m<P, N>(out, b, off, a.in, cb_neighbour(g, s, c, mu, -3), !eta_bit(c, mu), ls);
    }
  }
}

}  // namespace stag
