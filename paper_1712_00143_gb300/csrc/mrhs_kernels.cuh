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
// variants are capped at 128 (4 blocks) or 80 (6 blocks) registers
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
// the block's threads hold the sums of one system each).  RED = 3:
// Re<x_r, out_r> as per-warp double-float partials in rb.partials (float2
// [N][W], W warps of site coverage; no block barrier, no last block), summed
// by k_mcg_alpha_pw: the batched CG's <p, Ap> without a pass of its own.
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
      if (RED) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          red[r].add_prod(RED == 2 ? o[i].x : xv[i].x, o[i].x);  // RED 1 and 3: <x, out>
          red[r].add_prod(RED == 2 ? o[i].y : xv[i].y, o[i].y);
        }
      }
    }
  }
  if constexpr (RED == 3) {
    DF v[NT];
#pragma unroll
    for (int r = 0; r < NT; ++r) v[r] = red[r].v;
    warp_sum_df<NT>(v);
    if ((threadIdx.x & 31) == 0) {
      const int W = gridDim.x * (SPB / 32);
      const int w = blockIdx.x * (SPB / 32) + ((threadIdx.x - part * SPB) >> 5);
      float2* pw = (float2*)rb.partials;
#pragma unroll
      for (int r = 0; r < NT; ++r) pw[(size_t)(part * NT + r) * W + w] = make_float2(v[r].hi, v[r].lo);
    }
  } else if constexpr (RED != 0) {
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

// The variant a group of N right-hand sides of format P runs with on this lattice.
template <int P, int N> int mrhs_variant(const stag_lattice_s* lat) {
  const int v = lat->mrhs[abi_prec<P>()][mrhs_nindex(N)].variant;
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
  return mdslash_epi_v<P, N, RED>(lat, mrhs_variant<P, N>(lat), out, in, out_parity, x, ax, y, ay, ad, rs, tgt, flags,
                                  st);
}

// The autotuner of the N-right-hand-side kernels: on the first group of N
// right-hand sides of format P on a lattice, time every built variant of the
// plain and the epilogue kernel (one warm-up and three timed pairs, the
// operator's two halves t = D_oe p, Ap = m^2 p - D_eo t, on scratch vectors)
// and keep the fastest pair.  The choice is looked up first, and recorded,
// in the process-wide cache under the key (kernel, format, Naik storage, N,
// extents).  Must not run while a stream is being captured.
template <int P, int N> int tune_mrhs(stag_lattice_s* lat, cudaStream_t st) {
  auto& slot = lat->mrhs[abi_prec<P>()][mrhs_nindex(N)];
  if (slot.variant >= 0) return STAG_OK;
  const LinkCopy& L = lat->links[prec_index<P>()];
  if (!L.present) return STAG_EINVAL;
  const int def = mrhs_default_variant(P, N);
  if (!lat->autotune || P == 64) {
    slot.variant = def;
    return STAG_OK;
  }
  const std::string key = tune_key("dslash_mrhs", abi_prec<P>(), L.nl, N, lat->dims);
  int cached = -1;
  double cached_us = 0.0;
  if (tune_cache_get(key, &cached, &cached_us) && cached >= 0 && cached < kNumMVariants &&
      mrhs_variant_built(P, L.nl, N, cached)) {
    slot.variant = cached;
    slot.us = (float)cached_us;
    return STAG_OK;
  }
  constexpr int PA = Acc<P>::value;
  const int Vh = lat->g.Vh;
  int s = 0;
  SpinorM<P> in{lat->ws.get("tunem.in", spinorm_bytes<P>(Vh, N), &s), Vh, N};
  SpinorM<P> t{lat->ws.get("tunem.t", spinorm_bytes<P>(Vh, N), &s), Vh, N};
  SpinorM<PA> o{lat->ws.get("tunem.o", spinorm_bytes<PA>(Vh, N), &s), Vh, N};
  if (s) return s;
  if ((s = cuda_status(cudaMemsetAsync(in.v, 0, spinorm_bytes<P>(Vh, N), st)))) return s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return STAG_ECUDA;
  }
  const int reps = 3;
  float best = 1e30f;
  int pick = def;
  SpinorM<PA> none{nullptr, Vh, N};
  RedScratch rs{nullptr, nullptr, 1 << 30};
  for (int v = 0; v < kNumMVariants && !s; ++v) {
    if (!mrhs_variant_built(P, L.nl, N, v)) continue;
    for (int it = -1; it < reps && !s; ++it) {
      if (it == 0) s = cuda_status(cudaEventRecord(e0, st));
      if (!s) s = mdslash_v<P, N>(lat, v, t, in, 1, nullptr, st);
      if (!s)
        s = mdslash_epi_v<P, N, 0>(lat, v, o, t, 0, in, 0.01, none, 0.0, -1.0, rs,
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
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  lat->ws.drop("tunem.in");
  lat->ws.drop("tunem.t");
  lat->ws.drop("tunem.o");
  if (s) return s;
  slot.variant = pick;
  slot.us = best * 1e3f / reps;  // one operator (plain + epilogue launch)
  tune_cache_put(key, pick, slot.us);
  return STAG_OK;
}

// Per-warp partials of a RED = 3 launch for N right-hand sides of format P:
// W = the warps of one part (right-hand-side share) over the grid; at most
// Vh / 32 + 3.
template <int P, int N> int mrhs_partial_warps(const stag_lattice_s* lat) {
  const int spb = MB / mvariant(mrhs_variant<P, N>(lat)).sp;
  return (lat->g.Vh + spb - 1) / spb * (spb / 32);
}

// <p_r, Ap_r> of every system from the per-warp partials of a RED = 3
// operator launch (float2 [N][W]): one block, double-float sums in a fixed
// order, then RED_MCG_ALPHA.  Nothing once the group's stop word is set.
template <int N> __global__ void __launch_bounds__(512) k_mcg_alpha_pw(const float2* pw, int W, McgState* g) {
  if (stopped(&g->flags)) return;
  DF v[N];
#pragma unroll
  for (int r = 0; r < N; ++r) v[r] = DF{0.f, 0.f};
  for (int w = threadIdx.x; w < W; w += blockDim.x)
#pragma unroll
    for (int r = 0; r < N; ++r) {
      const float2 q = __ldcg(pw + (size_t)r * W + w);
      df_add_df(v[r], DF{q.x, q.y});
    }
  block_sum_df<N>(v);
  if (threadIdx.x == 0) {
    double t[N];
#pragma unroll
    for (int r = 0; r < N; ++r) t[r] = df_value(v[r]);
    finalize(RedTarget{RED_MCG_ALPHA, g, nullptr}, t, N);
  }
}

template <int P, int N>
int launch_mcg_alpha_pw(const stag_lattice_s* lat, const float2* pw, McgState* g, cudaStream_t st) {
  ProfScope ps("reduce", st);
  k_mcg_alpha_pw<N><<<1, 512, 0, st>>>(pw, mrhs_partial_warps<P, N>(lat), g);
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
  template int launch_mcg_alpha_pw<P, N>(const stag_lattice_s*, const float2*, McgState*, cudaStream_t);

}  // namespace stag
