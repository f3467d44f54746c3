// mrhs_kernels.cuh -- the N-right-hand-side Dslash kernels (plain, and with
// the fused axpy and per-system FP64 reductions), their launch variants and
// the autotuner that picks among them.  Instantiated per storage format in
// mrhs64.cu, mrhs32.cu, mrhs31.cu, mrhs16.cu and mrhs15.cu.
//
// Launch variants.  A block has MB = 128 threads.  SP threads share a site,
// each taking N / SP of the group's right-hand sides (the link chunks that
// all SP read come from L1 for all but the first); fewer accumulators per
// thread leave more resident warps to hide the loads.  MINB promises the
// compiler that many resident blocks per SM (6: at most 80 registers per
// thread; 4: 128; 1: no cap).  Which variant is fastest depends on the format, N and
// the lattice, so the batched solver and stag_dslash time the variants once
// per (format, Naik storage, N, extents) and keep the fastest (tune_mrhs),
// remembered for the process and, if asked, in a JSON file (tune.cu).
#pragma once
#include <string>

#include "dslash_mrhs.cuh"

namespace stag {

constexpr int MB = 128;  // threads per block of the N-RHS kernels

struct MVariant {
  int sp;    // threads per site
  int minb;  // resident blocks per SM promised to the compiler (1: no cap, 4: 128 registers, 6: 80)
};
// {1,1} {1,6} {2,4} {2,6} {4,4} {4,6}: without a cap the compiler takes
// 140-170 registers (three blocks per SM) whatever the split, so the split
// variants are capped at 128 (4 blocks) or 80 (6 blocks) registers.  Two
// more forms of {1,x} were measured at 32^4, N = 4, and removed: each
// thread's link chunks staged one direction ahead in shared memory with
// asynchronous copies (three blocks per SM; 128 us per launch against 117),
// and a bulk L2 prefetch of the block's next-direction links (130 us).
__host__ __device__ constexpr MVariant mvariant(int v) {
  return MVariant{v < 2 ? 1 : v < 4 ? 2 : 4, (v & 1) ? 6 : v == 0 ? 1 : 4};
}
constexpr int kNumMVariants = 6;

// The variant used without tuning: FP32 with up to four right-hand sides
// fits in 80 registers without spilling (six blocks, 24 warps, measured
// faster than five); the other forms take no cap.
__host__ __device__ constexpr int mrhs_default_variant(int p, int n) {
  return ((p == 32 || p == 31) && n <= 4) ? 1 : 0;
}

// Variants compiled for (format, Naik storage, N): the default always; the
// tuned set for two-row Naik storage with FP32 vectors (N = 2, 4, 8; the 80-register
// cap only for at most four right-hand sides per thread, beyond which it
// spills) and the 16-bit formats (N = 2, 4, the groups the batched solver
// forms for them; their decode needs more than 80 registers).
__host__ __device__ constexpr bool mrhs_variant_built(int p, int nl, int n, int v) {
  return v == mrhs_default_variant(p, n) ||
         (nl == 6 && n % mvariant(v).sp == 0 &&
          (((p == 32 || p == 31) && (mvariant(v).minb != 6 || n / mvariant(v).sp <= 4)) ||
           ((p == 16 || p == 15) && n <= 4 && mvariant(v).minb != 6)));
}

template <int P, int NL, int N, int SP, int MINB>
__global__ void __launch_bounds__(MB, MINB) k_dslash_mv(DslashArgsM<P> a, SpinorM<P> out, const int* flags) {
  static_assert(N % SP == 0, "right-hand sides split evenly");
  constexpr int NT = N / SP, SPB = MB / SP;
  if (stopped(flags)) return;
  const int part = threadIdx.x / SPB;
  const int s = blockIdx.x * SPB + (threadIdx.x - part * SPB);
  if (s >= a.g.Vh) return;
  const size_t off = spinor_bytes<P>(a.g.Vh) * (size_t)(part * NT);
  a.in.v = (char*)a.in.v + off;
  out.v = (char*)out.v + off;
  typename Prec<P>::A2 d[NT][3];
  dslash_site_m<P, NL, NT>(a, s, d);
#pragma unroll
  for (int r = 0; r < NT; ++r) SpinorLoadM<P>::st(out, s, r, d[r]);
}

// out_r = ax x_r + ay y_r + ad (D in)_r; RED = 1: Re<x_r, out_r>, RED = 2:
// ||out_r||^2, one sum per system, finalised by the last block (needs SP = 1:
// the block's threads hold the sums of one system each).  RED = 3: the
// site's Re<x_r, out_r> stored per site, float [N][Vh] in rb.partials (its
// six products summed in FP32: an error of a few units in the last place of
// the sum of their magnitudes, the level of the FP32 operands themselves),
// summed over sites by k_mcg_alpha_pt: the batched CG's <p, Ap> without
// reading p and Ap back (4 bytes per site and system against 48).  No
// barrier, no shuffle and nothing after the site's branch: every form that
// kept a sum live past the stencil (per-warp sums, double-float per-thread
// sums) made the compiler spill at the 80-register cap.
template <int P, int NL, int N, int RED, int SP, int MINB>
__global__ void __launch_bounds__(MB, MINB)
    k_dslash_m_epi_v(DslashArgsM<P> a, SpinorM<Acc<P>::value> out, SpinorM<P> x, double ax,
                     SpinorM<Acc<P>::value> y, double ay, double ad, RedBuf rb, RedTarget tgt, const int* flags) {
  static_assert(N % SP == 0 && (RED == 0 || RED == 3 || SP == 1), "variant");
  using A2 = typename Prec<P>::A2;
  using A = typename Prec<P>::A;
  constexpr int PA = Acc<P>::value;
  constexpr int NT = N / SP, SPB = MB / SP;
  if (stopped(flags)) return;
  const int part = threadIdx.x / SPB;
  const int s = blockIdx.x * SPB + (threadIdx.x - part * SPB);
  {
    const size_t off = spinor_bytes<P>(a.g.Vh) * (size_t)(part * NT);
    const size_t offa = spinor_bytes<PA>(a.g.Vh) * (size_t)(part * NT);
    a.in.v = (char*)a.in.v + off;
    x.v = (char*)x.v + off;
    out.v = (char*)out.v + offa;
    if (y.v) y.v = (char*)y.v + offa;
  }
  Acc1<A> red[NT];
  if (s < a.g.Vh) {
    // the epilogue's x_r are read after the stencil: start them towards L2 now
#pragma unroll
    for (int r = 0; r < NT; ++r) prefetch_spinor_l2<P>(SpinorLoadM<P>::one(x, r), s);
    A2 d[NT][3];
    dslash_site_m<P, NL, NT>(a, s, d);
    const A cx = (A)ax, cd = (A)ad, cy = (A)ay;
#pragma unroll
    for (int r = 0; r < NT; ++r) {
      A2 xv[3], o[3];
      SpinorLoadM<P>::ld(x, s, r, xv);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        o[i].x = cx * xv[i].x + cd * d[r][i].x;
        o[i].y = cx * xv[i].y + cd * d[r][i].y;
      }
      if (ay != 0.0) {
        A2 yv[3];
        SpinorLoadM<PA>::ld(y, s, r, yv);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          o[i].x += cy * yv[i].x;
          o[i].y += cy * yv[i].y;
        }
      }
      SpinorLoadM<PA>::st(out, s, r, o);
      if constexpr (RED == 3) {
        float d3 = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          d3 = fmaf((float)xv[i].x, (float)o[i].x, d3);
          d3 = fmaf((float)xv[i].y, (float)o[i].y, d3);
        }
        ((float*)rb.partials)[(size_t)(part * NT + r) * a.g.Vh + s] = d3;
      } else if constexpr (RED != 0) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          red[r].add_prod(RED == 1 ? xv[i].x : o[i].x, o[i].x);
          red[r].add_prod(RED == 1 ? xv[i].y : o[i].y, o[i].y);
        }
      }
    }
  }
  if constexpr (RED != 0 && RED != 3) {
    grid_reduce_acc<N>(red, rb, tgt);
  }
}

template <int P> DslashArgsM<P> make_args_m(const stag_lattice_s* lat, SpinorM<P> in, int out_parity) {
  const LinkCopy& L = lat->links[prec_index<P>()];
  DslashArgsM<P> a;
  a.g = lat->g;
  a.out_parity = out_parity;
  a.links = (const uint4*)((const char*)L.data + (size_t)out_parity * L.parity_stride);
  const double fx = fixed_links(P) ? 1.0 / 32767.0 : 1.0;
  a.fat_scale = (float)(L.fat_scale * fx);
  a.long_scale = (float)((L.nl == 6 ? 0.5 * lat->c3 : (double)L.long_scale) * fx);
  a.in = in;
  return a;
}

__host__ __device__ constexpr int mrhs_nindex(int n) { return n == 2 ? 0 : n == 4 ? 1 : n == 8 ? 2 : 3; }

// The variants a group of N right-hand sides of format P runs with on this
// lattice: the plain operator half, and the epilogue form.
template <int P, int N> int mrhs_variant(const stag_lattice_s* lat) {
  const int v = lat->mrhs[abi_prec<P>()][mrhs_nindex(N)].variant;
  return v >= 0 ? v : mrhs_default_variant(P, N);
}
template <int P, int N> int mrhs_variant_epi(const stag_lattice_s* lat) {
  const int v = lat->mrhs[abi_prec<P>()][mrhs_nindex(N)].variant_epi;
  return v >= 0 ? v : mrhs_default_variant(P, N);
}

template <int P, int NL, int N, int V>
void launch_plain_v(int G, const DslashArgsM<P>& a, SpinorM<P> out, const int* flags, cudaStream_t st) {
  if constexpr (mrhs_variant_built(P, NL, N, V)) {
    constexpr MVariant mv = mvariant(V);
    k_dslash_mv<P, NL, N, mv.sp, mv.minb><<<G, MB, 0, st>>>(a, out, flags);
  }
}

template <int P, int NL, int N>
void dispatch_plain(int v, const DslashArgsM<P>& a, SpinorM<P> out, const int* flags, cudaStream_t st) {
  if (!mrhs_variant_built(P, NL, N, v)) v = mrhs_default_variant(P, N);
  const int spb = MB / mvariant(v).sp;
  const int G = (a.g.Vh + spb - 1) / spb;
  switch (v) {
    case 0: launch_plain_v<P, NL, N, 0>(G, a, out, flags, st); break;
    case 1: launch_plain_v<P, NL, N, 1>(G, a, out, flags, st); break;
    case 2: launch_plain_v<P, NL, N, 2>(G, a, out, flags, st); break;
    case 3: launch_plain_v<P, NL, N, 3>(G, a, out, flags, st); break;
    case 4: launch_plain_v<P, NL, N, 4>(G, a, out, flags, st); break;
    default: launch_plain_v<P, NL, N, 5>(G, a, out, flags, st);
  }
}

template <int P, int NL, int N, int RED, int V>
void launch_epi_v(int G, const DslashArgsM<P>& a, SpinorM<Acc<P>::value> out, SpinorM<P> x, double ax,
                  SpinorM<Acc<P>::value> y, double ay, double ad, RedBuf rb, RedTarget tgt, const int* flags,
                  cudaStream_t st) {
  if constexpr (mrhs_variant_built(P, NL, N, V) && (RED == 0 || RED == 3 || mvariant(V).sp == 1)) {
    constexpr MVariant mv = mvariant(V);
    k_dslash_m_epi_v<P, NL, N, RED, mv.sp, mv.minb><<<G, MB, 0, st>>>(a, out, x, ax, y, ay, ad, rb, tgt, flags);
  }
}

template <int P, int NL, int N, int RED>
void dispatch_epi(int v, const DslashArgsM<P>& a, SpinorM<Acc<P>::value> out, SpinorM<P> x, double ax,
                  SpinorM<Acc<P>::value> y, double ay, double ad, RedBuf rb, RedTarget tgt, const int* flags,
                  cudaStream_t st) {
  if (!mrhs_variant_built(P, NL, N, v) || (RED != 0 && RED != 3 && mvariant(v).sp != 1))
    v = mrhs_default_variant(P, N);
  const int spb = MB / mvariant(v).sp;
  const int G = (a.g.Vh + spb - 1) / spb;
#define STAG_EPV(V) launch_epi_v<P, NL, N, RED, V>(G, a, out, x, ax, y, ay, ad, rb, tgt, flags, st)
  switch (v) {
    case 0: STAG_EPV(0); break;
    case 1: STAG_EPV(1); break;
    case 2: STAG_EPV(2); break;
    case 3: STAG_EPV(3); break;
    case 4: STAG_EPV(4); break;
    default: STAG_EPV(5);
  }
#undef STAG_EPV
}

template <int P, int N>
int mdslash_v(const stag_lattice_s* lat, int v, SpinorM<P> out, SpinorM<P> in, int out_parity, const int* flags,
              cudaStream_t st) {
  const LinkCopy& L = lat->links[prec_index<P>()];
  if (!L.present) return STAG_EINVAL;
  DslashArgsM<P> a = make_args_m<P>(lat, in, out_parity);
  ProfScope ps(P == 64 ? "dslash_mrhs64" : "dslash_mrhs", st);
  if (P != 64 && L.nl == 6)
    dispatch_plain<P, (P == 64 ? 9 : 6), N>(v, a, out, flags, st);
  else
    dispatch_plain<P, 9, N>(v, a, out, flags, st);
  return last_launch_status();
}

template <int P, int N, int RED>
int mdslash_epi_v(const stag_lattice_s* lat, int v, SpinorM<Acc<P>::value> out, SpinorM<P> in, int out_parity,
                  SpinorM<P> x, double ax, SpinorM<Acc<P>::value> y, double ay, double ad, RedScratch rs,
                  RedTarget tgt, const int* flags, cudaStream_t st) {
  const LinkCopy& L = lat->links[prec_index<P>()];
  if (!L.present) return STAG_EINVAL;
  DslashArgsM<P> a = make_args_m<P>(lat, in, out_parity);
  if (RED && RED != 3 && (a.g.Vh + MB - 1) / MB > rs.max_grid) return STAG_EINVAL;
  ProfScope ps(P == 64 ? "dslash_mrhs64_epi" : "dslash_mrhs_epi", st);
  RedBuf rb{rs.partials, rs.counter};
  if (P != 64 && L.nl == 6)
    dispatch_epi<P, (P == 64 ? 9 : 6), N, RED>(v, a, out, x, ax, y, ay, ad, rb, tgt, flags, st);
  else
    dispatch_epi<P, 9, N, RED>(v, a, out, x, ax, y, ay, ad, rb, tgt, flags, st);
  return last_launch_status();
}

template <int P, int N>
int mdslash(const stag_lattice_s* lat, SpinorM<P> out, SpinorM<P> in, int out_parity, const int* flags,
            cudaStream_t st) {
  return mdslash_v<P, N>(lat, mrhs_variant<P, N>(lat), out, in, out_parity, flags, st);
}

template <int P, int N, int RED>
int mdslash_epi(const stag_lattice_s* lat, SpinorM<Acc<P>::value> out, SpinorM<P> in, int out_parity, SpinorM<P> x,
                double ax, SpinorM<Acc<P>::value> y, double ay, double ad, RedScratch rs, RedTarget tgt,
                const int* flags, cudaStream_t st) {
  return mdslash_epi_v<P, N, RED>(lat, mrhs_variant_epi<P, N>(lat), out, in, out_parity, x, ax, y, ay, ad, rs, tgt,
                                  flags, st);
}

// The autotuner of the N-right-hand-side kernels: on the first group of N
// right-hand sides of format P on a lattice, time every built variant of the
// plain operator half (t = D_oe p) and, separately, of the epilogue form the
// batched CG runs (Ap = m^2 p - D_eo t with the per-site <p, Ap> values for
// the FP32-arithmetic formats), one warm-up and three timed launches each on
// scratch vectors, and keep the fastest of each (a variant's register cap
// can suit one form and not the other).  The choices are looked up first,
// and recorded, in the process-wide cache under the keys ("dslash_mrhs" or
// "dslash_mrhs_epi", format, Naik storage, N, extents).  Must not run while
// a stream is being captured.
template <int P, int N> int tune_mrhs(stag_lattice_s* lat, cudaStream_t st) {
  auto& slot = lat->mrhs[abi_prec<P>()][mrhs_nindex(N)];
  if (slot.variant >= 0 && slot.variant_epi >= 0) return STAG_OK;
  const LinkCopy& L = lat->links[prec_index<P>()];
  if (!L.present) return STAG_EINVAL;
  const int def = mrhs_default_variant(P, N);
  if (!lat->autotune || P == 64) {
    slot.variant = slot.variant_epi = def;
    return STAG_OK;
  }
  const std::string key = tune_key("dslash_mrhs", abi_prec<P>(), L.nl, N, lat->dims);
  const std::string key_epi = tune_key("dslash_mrhs_epi", abi_prec<P>(), L.nl, N, lat->dims);
  auto cached = [&](const std::string& k, int* v, float* us) {
    int c = -1;
    double cu = 0.0;
    if (tune_cache_get(k, &c, &cu) && c >= 0 && c < kNumMVariants && mrhs_variant_built(P, L.nl, N, c)) {
      *v = c;
      *us = (float)cu;
    }
  };
  if (slot.variant < 0) cached(key, &slot.variant, &slot.us);
  if (slot.variant_epi < 0) cached(key_epi, &slot.variant_epi, &slot.us_epi);
  if (slot.variant >= 0 && slot.variant_epi >= 0) return STAG_OK;

  constexpr int PA = Acc<P>::value;
  constexpr int RED = P == 64 ? 0 : 3;
  const int Vh = lat->g.Vh;
  int s = 0;
  SpinorM<P> in{lat->ws.get("tunem.in", spinorm_bytes<P>(Vh, N), &s), Vh, N};
  SpinorM<P> t{lat->ws.get("tunem.t", spinorm_bytes<P>(Vh, N), &s), Vh, N};
  SpinorM<PA> o{lat->ws.get("tunem.o", spinorm_bytes<PA>(Vh, N), &s), Vh, N};
  double* pw = (double*)lat->ws.get("tunem.pw", sizeof(float) * N * (size_t)Vh, &s);
  if (s) return s;
  if ((s = cuda_status(cudaMemsetAsync(in.v, 0, spinorm_bytes<P>(Vh, N), st)))) return s;
  if ((s = cuda_status(cudaMemsetAsync(t.v, 0, spinorm_bytes<P>(Vh, N), st)))) return s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return STAG_ECUDA;
  }
  const int reps = 3;
  SpinorM<PA> none{nullptr, Vh, N};
  RedScratch rs{pw, nullptr, 1 << 30};
  // form 0: plain, form 1: epilogue
  for (int form = 0; form < 2 && !s; ++form) {
    if ((form == 0 ? slot.variant : slot.variant_epi) >= 0) continue;
    float best = 1e30f;
    int pick = def;
    for (int v = 0; v < kNumMVariants && !s; ++v) {
      if (!mrhs_variant_built(P, L.nl, N, v)) continue;
      for (int it = -1; it < reps && !s; ++it) {
        if (it == 0) s = cuda_status(cudaEventRecord(e0, st));
        if (s) break;
        if (form == 0)
          s = mdslash_v<P, N>(lat, v, t, in, 1, nullptr, st);
        else
          s = mdslash_epi_v<P, N, RED>(lat, v, o, t, 0, in, 0.01, none, 0.0, -1.0, rs,
                                       RedTarget{RED_STORE, nullptr, nullptr}, nullptr, st);
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
    if (s) break;
    const float us = best * 1e3f / reps;
    if (form == 0) {
      slot.variant = pick;
      slot.us = us;
      tune_cache_put(key, pick, us);
    } else {
      slot.variant_epi = pick;
      slot.us_epi = us;
      tune_cache_put(key_epi, pick, us);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  lat->ws.drop("tunem.in");
  lat->ws.drop("tunem.t");
  lat->ws.drop("tunem.o");
  lat->ws.drop("tunem.pw");
  return s;
}

// <p_r, Ap_r> of every system from the per-site values of a RED = 3
// operator launch (float [N][Vh]): per-thread double-float sums over a
// grid-stride range of sites, then the library's deterministic grid sum and
// RED_MCG_ALPHA.  Nothing once the group's stop word is set.
template <int N>
__global__ void __launch_bounds__(256) k_mcg_alpha_pt(const float* __restrict__ pt, int Vh, McgState* g, RedBuf rb) {
  if (stopped(&g->flags)) return;
  constexpr int U = 4;  // sites per thread and pass, loaded before they are added
  DF v[N];
#pragma unroll
  for (int r = 0; r < N; ++r) v[r] = DF{0.f, 0.f};
  const int stride = gridDim.x * blockDim.x;
  for (int s0 = blockIdx.x * blockDim.x + threadIdx.x; s0 < Vh; s0 += U * stride) {
    float q[U][N];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < N; ++r) {
        const int s = s0 + u * stride;
        q[u][r] = s < Vh ? __ldcg(pt + (size_t)r * Vh + s) : 0.f;
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < N; ++r) df_add_df(v[r], DF{q[u][r], 0.f});
  }
  grid_reduce_df<N>(v, rb, RedTarget{RED_MCG_ALPHA, g, nullptr});
}

template <int P, int N>
int launch_mcg_alpha_pt(const stag_lattice_s* lat, const float* pt, McgState* g, RedScratch rs, cudaStream_t st) {
  const int Vh = lat->g.Vh;
  int G = (Vh + 4 * 256 - 1) / (4 * 256);  // four sites per thread
  G = G < 1 ? 1 : G > rs.max_grid ? rs.max_grid : G;
  ProfScope ps("reduce", st);
  k_mcg_alpha_pt<N><<<G, 256, 0, st>>>(pt, Vh, g, RedBuf{rs.partials, rs.counter});
  return last_launch_status();
}

#define STAG_INSTANTIATE_MRHS_N(P, N)                                                                               \
  template int mdslash<P, N>(const stag_lattice_s*, SpinorM<P>, SpinorM<P>, int, const int*, cudaStream_t);         \
  template int mdslash_epi<P, N, 0>(const stag_lattice_s*, SpinorM<Acc<P>::value>, SpinorM<P>, int, SpinorM<P>,     \
                                    double, SpinorM<Acc<P>::value>, double, double, RedScratch, RedTarget,          \
                                    const int*, cudaStream_t);                                                      \
  template int tune_mrhs<P, N>(stag_lattice_s*, cudaStream_t);

// the per-warp inner-product form (RED = 3) of the batched CG's operator
#define STAG_INSTANTIATE_MRHS_RED3(P, N)                                                                            \
  template int mdslash_epi<P, N, 3>(const stag_lattice_s*, SpinorM<Acc<P>::value>, SpinorM<P>, int, SpinorM<P>,     \
                                    double, SpinorM<Acc<P>::value>, double, double, RedScratch, RedTarget,          \
                                    const int*, cudaStream_t);                                                      \
  template int launch_mcg_alpha_pt<P, N>(const stag_lattice_s*, const float*, McgState*, RedScratch, cudaStream_t);

}  // namespace stag
