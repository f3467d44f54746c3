// blas.cu -- the level-1 kernels of the Krylov solvers, each fused with the
// reduction it feeds (CG is memory-bound, arithmetic intensity about 0.26
// flop/byte in the paper's measurements, Sec. 4.2, so every extra pass over a
// vector costs as much as its bytes).  Grid-stride loops over a grid capped
// at a few blocks per SM, two sites per trip so that each thread has two
// sites' loads in flight; coalesced structure-of-arrays access.  Sums use
// FP64 across threads and, in the FP32 kernels, an error-free FP32 (hi, lo)
// accumulation per thread (see common.cuh).  Scalars (alpha, beta, zeta ...)
// are read from the device-resident solver state, never from the host, so a
// whole iteration is queued without a host round trip.
#include "internal.h"

namespace stag {

static constexpr int BB = 256;  // threads per block of the level-1 kernels

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) {
      n = v;
    } else {
      cudaGetLastError();
      n = 152;
    }
  }
  return n;
}

// Grids: reductions use up to 4 blocks per SM (each block reduces once, at
// the end), streaming kernels up to 8.
static inline int red_grid(int Vh, int cap) {
  int g = (Vh + BB - 1) / BB;
  int m = 4 * sm_count();
  if (g > m) g = m;
  return g < cap ? g : cap;
}
static inline int bw_grid(int Vh) {
  int g = (Vh + BB - 1) / BB;
  int m = 8 * sm_count();
  return g < m ? g : m;
}

#define GRID_STRIDE(s, Vh) for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < (Vh); s += gridDim.x * blockDim.x)

// Two sites per trip: BODY2(s0, s1) handles s0 and s1 = s0 + stride with all
// loads first; BODY1(s) handles a lone last site.
#define GRID_STRIDE2(Vh, BODY2, BODY1)                                      \
  {                                                                         \
    const int stride_ = gridDim.x * blockDim.x;                             \
    int s_ = blockIdx.x * blockDim.x + threadIdx.x;                         \
    for (; s_ + stride_ < (Vh); s_ += 2 * stride_) BODY2(s_, s_ + stride_); \
    if (s_ < (Vh)) BODY1(s_);                                               \
  }

// ------------------------------------------------------------ conversions
template <int P> __global__ void k_from_canonical(Spinor<P> out, const double2* __restrict__ in, int Vh) {
  using A2 = typename Prec<P>::A2;
  GRID_STRIDE(s, Vh) {
    A2 o[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double2 v = in[3 * (size_t)s + c];
      o[c].x = v.x;
      o[c].y = v.y;
    }
    SpinorLoad<P>::st(out, s, o);
  }
}

template <int P> __global__ void k_to_canonical(double2* __restrict__ out, Spinor<P> in, int Vh) {
  using A2 = typename Prec<P>::A2;
  GRID_STRIDE(s, Vh) {
    A2 o[3];
    SpinorLoad<P>::ld(in, s, o);
#pragma unroll
    for (int c = 0; c < 3; ++c) out[3 * (size_t)s + c] = make_double2((double)o[c].x, (double)o[c].y);
  }
}

template <int PO, int PI> __global__ void k_convert(Spinor<PO> out, Spinor<PI> in, int Vh) {
  using AI = typename Prec<PI>::A2;
  using AO = typename Prec<PO>::A2;
  GRID_STRIDE(s, Vh) {
    AI a[3];
    AO o[3];
    SpinorLoad<PI>::ld(in, s, a);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      o[c].x = a[c].x;
      o[c].y = a[c].y;
    }
    SpinorLoad<PO>::st(out, s, o);
  }
}

template <int P> int launch_from_canonical(Spinor<P> out, const double2* in, int Vh, cudaStream_t st) {
  ProfScope ps("convert", st);
  k_from_canonical<P><<<bw_grid(Vh), BB, 0, st>>>(out, in, Vh);
  return last_launch_status();
}
template <int P> int launch_to_canonical(double2* out, Spinor<P> in, int Vh, cudaStream_t st) {
  ProfScope ps("convert", st);
  k_to_canonical<P><<<bw_grid(Vh), BB, 0, st>>>(out, in, Vh);
  return last_launch_status();
}
template <int PO, int PI> int launch_convert(Spinor<PO> out, Spinor<PI> in, cudaStream_t st) {
  ProfScope ps("convert", st);
  k_convert<PO, PI><<<bw_grid(in.Vh), BB, 0, st>>>(out, in, in.Vh);
  return last_launch_status();
}

int launch_zero(void* p, size_t bytes, cudaStream_t st) { return cuda_status(cudaMemsetAsync(p, 0, bytes, st)); }

// ------------------------------------------------------------ reductions
template <int P> __global__ void k_norm2(Spinor<P> v, RedBuf rb, RedTarget tgt) {
  using A2 = typename Prec<P>::A2;
  using A = typename Prec<P>::A;
  Acc1<A> acc;
  GRID_STRIDE(s, v.Vh) {
    A2 a[3];
    SpinorLoad<P>::ld(v, s, a);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc.add_prod(a[c].x, a[c].x);
      acc.add_prod(a[c].y, a[c].y);
    }
  }
  Acc1<A> tot[1] = {acc};
  grid_reduce_acc<1>(tot, rb, tgt);
}

template <int P> int launch_norm2(Spinor<P> v, RedScratch rs, RedTarget tgt, cudaStream_t st) {
  ProfScope ps("reduce", st);
  k_norm2<P><<<red_grid(v.Vh, rs.max_grid), BB, 0, st>>>(v, RedBuf{rs.partials, rs.counter}, tgt);
  return last_launch_status();
}

// ------------------------------------------------------------ CG kernels
// xh += alpha p; rh -= alpha Ap; ||rh||^2 -> beta (RED_CG_BETA)
template <int P, int PV> struct CgUpdate {
  using A2 = typename Prec<PV>::A2;
  using A = typename Prec<PV>::A;
  Spinor<PV> xh, rh, Ap;
  Spinor<P> p;
  A alpha;
  struct Site {
    A2 x[3], r[3], ap[3];
    typename Prec<P>::A2 pv[3];
  };
  __device__ __forceinline__ void load(int s, Site& t) const {
    SpinorLoad<PV>::ldw(xh, s, t.x);
    SpinorLoad<PV>::ldw(rh, s, t.r);
    SpinorLoad<P>::ld(p, s, t.pv);
    SpinorLoad<PV>::ld(Ap, s, t.ap);
  }
  __device__ __forceinline__ void update(int s, Site& t, Acc1<A>& acc) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      t.x[c].x += alpha * (A)t.pv[c].x;
      t.x[c].y += alpha * (A)t.pv[c].y;
      t.r[c].x -= alpha * t.ap[c].x;
      t.r[c].y -= alpha * t.ap[c].y;
      acc.add_prod(t.r[c].x, t.r[c].x);
      acc.add_prod(t.r[c].y, t.r[c].y);
    }
    SpinorLoad<PV>::st(xh, s, t.x);
    SpinorLoad<PV>::st(rh, s, t.r);
  }
};

template <int P, int PV>
__global__ void __launch_bounds__(BB) k_cg_update(Spinor<PV> xh, Spinor<PV> rh, Spinor<P> p, Spinor<PV> Ap,
                                                   CgState* st, RedBuf rb) {
  using A = typename Prec<PV>::A;
  if (stopped(&st->flags)) return;
  CgUpdate<P, PV> u{xh, rh, Ap, p, (A)__ldcg(&st->alpha)};
  Acc1<A> acc;
  typename CgUpdate<P, PV>::Site t0, t1;
#define CGU2(a, b) { u.load(a, t0); u.load(b, t1); u.update(a, t0, acc); u.update(b, t1, acc); }
#define CGU1(a) { u.load(a, t0); u.update(a, t0, acc); }
  GRID_STRIDE2(xh.Vh, CGU2, CGU1)
#undef CGU2
#undef CGU1
  Acc1<A> tot[1] = {acc};
  grid_reduce_acc<1>(tot, rb, RedTarget{RED_CG_BETA, st, nullptr});
}

template <int P>
int launch_cg_update(Spinor<Acc<P>::value> xh, Spinor<Acc<P>::value> rh, Spinor<P> p, Spinor<Acc<P>::value> Ap,
                     CgState* state, RedScratch rs, cudaStream_t st) {
  ProfScope ps("blas", st);
  k_cg_update<P, Acc<P>::value>
      <<<red_grid(xh.Vh, rs.max_grid), BB, 0, st>>>(xh, rh, p, Ap, state, RedBuf{rs.partials, rs.counter});
  return last_launch_status();
}

// p = rh + beta p
template <int P, int PV> __global__ void __launch_bounds__(BB) k_cg_xpay(Spinor<P> p, Spinor<PV> rh, CgState* st) {
  using A2 = typename Prec<P>::A2;
  using A = typename Prec<P>::A;
  if (stopped(&st->flags)) return;
  const A beta = (A)__ldcg(&st->beta);
  A2 p0[3], p1[3];
  typename Prec<PV>::A2 r0[3], r1[3];
  auto upd = [&](int s, A2(&pv)[3], const typename Prec<PV>::A2(&r)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pv[c].x = (A)r[c].x + beta * pv[c].x;
      pv[c].y = (A)r[c].y + beta * pv[c].y;
    }
    SpinorLoad<P>::st(p, s, pv);
  };
#define XPAY2(a, b)                                                         \
  {                                                                         \
    SpinorLoad<P>::ldw(p, a, p0);                                           \
    SpinorLoad<PV>::ld(rh, a, r0);                                          \
    SpinorLoad<P>::ldw(p, b, p1);                                           \
    SpinorLoad<PV>::ld(rh, b, r1);                                          \
    upd(a, p0, r0);                                                         \
    upd(b, p1, r1);                                                         \
  }
#define XPAY1(a) { SpinorLoad<P>::ldw(p, a, p0); SpinorLoad<PV>::ld(rh, a, r0); upd(a, p0, r0); }
  GRID_STRIDE2(p.Vh, XPAY2, XPAY1)
#undef XPAY2
#undef XPAY1
}

template <int P> int launch_cg_xpay(Spinor<P> p, Spinor<Acc<P>::value> rh, CgState* state, cudaStream_t st) {
  ProfScope ps("blas", st);
  k_cg_xpay<P, Acc<P>::value><<<bw_grid(p.Vh), BB, 0, st>>>(p, rh, state);
  return last_launch_status();
}

// y += xh; xh = 0
template <int PV> __global__ void k_accumulate(Spinor<64> y, Spinor<PV> xh) {
  GRID_STRIDE(s, y.Vh) {
    double2 a[3];
    typename Prec<PV>::A2 b[3], z[3];
    SpinorLoad<64>::ldw(y, s, a);
    SpinorLoad<PV>::ldw(xh, s, b);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a[c].x += (double)b[c].x;
      a[c].y += (double)b[c].y;
      z[c].x = 0;
      z[c].y = 0;
    }
    SpinorLoad<64>::st(y, s, a);
    SpinorLoad<PV>::st(xh, s, z);
  }
}

template <int PV> int launch_accumulate(Spinor<64> y, Spinor<PV> xh, cudaStream_t st) {
  ProfScope ps("blas", st);
  k_accumulate<PV><<<bw_grid(y.Vh), BB, 0, st>>>(y, xh);
  return last_launch_status();
}

// rh = r (converted), <rh, p> (complex) -> RED_RU_ORTHO
template <int P, int PV>
__global__ void k_ru_convert_dot(Spinor<PV> rh, Spinor<64> r, Spinor<P> p, CgState* st, RedBuf rb) {
  using A2 = typename Prec<PV>::A2;
  using A = typename Prec<PV>::A;
  Acc1<A> re, im;
  GRID_STRIDE(s, r.Vh) {
    double2 a[3];
    A2 o[3];
    typename Prec<P>::A2 pv[3];
    SpinorLoad<64>::ld(r, s, a);
    SpinorLoad<P>::ld(p, s, pv);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      o[c].x = a[c].x;
      o[c].y = a[c].y;
    }
    SpinorLoad<PV>::st(rh, s, o);
    // the stored (rounded) rh enters the dot, as it will enter p below
    SpinorLoad<PV>::ldw(rh, s, o);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      re.add_prod(o[c].x, (A)pv[c].x);
      re.add_prod(o[c].y, (A)pv[c].y);
      im.add_prod(o[c].x, (A)pv[c].y);
      im.add_prod(-o[c].y, (A)pv[c].x);
    }
  }
  Acc1<A> tot[2] = {re, im};
  grid_reduce_acc<2>(tot, rb, RedTarget{RED_RU_ORTHO, st, nullptr});
}

template <int P>
int launch_ru_convert_dot(Spinor<Acc<P>::value> rh, Spinor<64> r, Spinor<P> p, CgState* state, RedScratch rs,
                          cudaStream_t st) {
  ProfScope ps("reduce", st);
  k_ru_convert_dot<P, Acc<P>::value>
      <<<red_grid(r.Vh, rs.max_grid), BB, 0, st>>>(rh, r, p, state, RedBuf{rs.partials, rs.counter});
  return last_launch_status();
}

// p = rh + beta (p - c rh), c = <rh,p>/||rh||^2: restores r-orthogonality of
// the search direction after a reliable update.
template <int P, int PV> __global__ void k_ru_p(Spinor<P> p, Spinor<PV> rh, CgState* st) {
  using A2 = typename Prec<P>::A2;
  using A = typename Prec<P>::A;
  const A beta = (A)__ldcg(&st->beta);
  const A cr = (A)__ldcg(&st->ortho_re), ci = (A)__ldcg(&st->ortho_im);
  GRID_STRIDE(s, p.Vh) {
    A2 pv[3];
    typename Prec<PV>::A2 r[3];
    SpinorLoad<P>::ldw(p, s, pv);
    SpinorLoad<PV>::ld(rh, s, r);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      A rx = (A)r[c].x, ry = (A)r[c].y;
      A qx = pv[c].x - (cr * rx - ci * ry);
      A qy = pv[c].y - (cr * ry + ci * rx);
      pv[c].x = rx + beta * qx;
      pv[c].y = ry + beta * qy;
    }
    SpinorLoad<P>::st(p, s, pv);
  }
}

template <int P> int launch_ru_p(Spinor<P> p, Spinor<Acc<P>::value> rh, CgState* state, cudaStream_t st) {
  ProfScope ps("blas", st);
  k_ru_p<P, Acc<P>::value><<<bw_grid(p.Vh), BB, 0, st>>>(p, rh, state);
  return last_launch_status();
}

// ------------------------------------------------------------ multi-shift
template <int PV>
__global__ void __launch_bounds__(BB) k_ms_r_update(Spinor<PV> r, Spinor<PV> Ap, MsState* ms, RedBuf rb) {
  using A2 = typename Prec<PV>::A2;
  using A = typename Prec<PV>::A;
  if (stopped(&ms->cg.flags)) return;
  const A alpha = (A)__ldcg(&ms->cg.alpha);
  Acc1<A> acc;
  A2 r0[3], a0[3], r1[3], a1[3];
  auto upd = [&](int s, A2(&rv)[3], const A2(&ap)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      rv[c].x -= alpha * ap[c].x;
      rv[c].y -= alpha * ap[c].y;
      acc.add_prod(rv[c].x, rv[c].x);
      acc.add_prod(rv[c].y, rv[c].y);
    }
    SpinorLoad<PV>::st(r, s, rv);
  };
#define MSR2(a, b)                                                          \
  {                                                                         \
    SpinorLoad<PV>::ldw(r, a, r0);                                          \
    SpinorLoad<PV>::ld(Ap, a, a0);                                          \
    SpinorLoad<PV>::ldw(r, b, r1);                                          \
    SpinorLoad<PV>::ld(Ap, b, a1);                                          \
    upd(a, r0, a0);                                                         \
    upd(b, r1, a1);                                                         \
  }
#define MSR1(a) { SpinorLoad<PV>::ldw(r, a, r0); SpinorLoad<PV>::ld(Ap, a, a0); upd(a, r0, a0); }
  GRID_STRIDE2(r.Vh, MSR2, MSR1)
#undef MSR2
#undef MSR1
  Acc1<A> tot[1] = {acc};
  grid_reduce_acc<1>(tot, rb, RedTarget{RED_MS_BETA, ms, nullptr});
}

template <int P>
int launch_ms_r_update(Spinor<Acc<P>::value> r, Spinor<Acc<P>::value> Ap, MsState* state, RedScratch rs,
                       cudaStream_t st) {
  ProfScope ps("blas", st);
  k_ms_r_update<Acc<P>::value>
      <<<red_grid(r.Vh, rs.max_grid), BB, 0, st>>>(r, Ap, state, RedBuf{rs.partials, rs.counter});
  return last_launch_status();
}

template <int P, int PX> struct ShiftPtrs {
  Spinor<PX> x[MAX_SHIFTS];
  Spinor<P> p[MAX_SHIFTS];
};

// For every shift still iterating: x_s += alpha_s p_s; p_s = zeta_s r + beta_s p_s.
// The base shift's direction (index `base`) is always updated: it drives the
// shared Krylov space.  The solution vectors x_s have the Krylov loop's
// vector precision (FP32 in the mixed modes; FP64 refinement follows).
template <int P, int PV>
__global__ void __launch_bounds__(BB) k_ms_shift_update(ShiftPtrs<P, PV> sp, int nshift, int base, Spinor<PV> r,
                                                         MsState* ms, int expect_iter) {
  using A2 = typename Prec<P>::A2;
  using A = typename Prec<P>::A;
  using AV = typename Prec<PV>::A;
  // runs only if this iteration's residual update ran (it advanced the
  // iteration count to expect_iter); it also runs in the iteration that set
  // F_CONVERGED, so the retiring shifts take their last step
  if (__ldcg(&ms->cg.iter) != expect_iter || (__ldcg(&ms->cg.flags) & F_BREAKDOWN)) return;
  const int mask = __ldcg(&ms->active_mask);
  GRID_STRIDE(s, r.Vh) {
    typename Prec<PV>::A2 rv[3];
    SpinorLoad<PV>::ld(r, s, rv);
    for (int k = 0; k < nshift; ++k) {
      const bool act = (mask >> k) & 1;
      if (!act && k != base) continue;
      const AV as = (AV)__ldcg(&ms->alpha_s[k]);
      const A bs = (A)__ldcg(&ms->beta_s[k]), z = (A)__ldcg(&ms->zeta_next[k]);
      A2 pv[3];
      SpinorLoad<P>::ldw(sp.p[k], s, pv);
      if (act) {
        typename Prec<PV>::A2 xv[3];
        SpinorLoad<PV>::ldw(sp.x[k], s, xv);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          xv[c].x += as * (AV)pv[c].x;
          xv[c].y += as * (AV)pv[c].y;
        }
        SpinorLoad<PV>::st(sp.x[k], s, xv);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pv[c].x = z * (A)rv[c].x + bs * pv[c].x;
        pv[c].y = z * (A)rv[c].y + bs * pv[c].y;
      }
      SpinorLoad<P>::st(sp.p[k], s, pv);
    }
  }
}

template <int P>
int launch_ms_shift_update(Spinor<Acc<P>::value>* xs, Spinor<P>* ps, int nshift, int base, Spinor<Acc<P>::value> r,
                           MsState* state, int expect_iter, cudaStream_t st) {
  if (nshift > MAX_SHIFTS) return STAG_EINVAL;
  ShiftPtrs<P, Acc<P>::value> sp;
  for (int k = 0; k < nshift; ++k) {
    sp.x[k] = xs[k];
    sp.p[k] = ps[k];
  }
  ProfScope pscope("blas", st);
  k_ms_shift_update<P, Acc<P>::value><<<bw_grid(r.Vh), BB, 0, st>>>(sp, nshift, base, r, state, expect_iter);
  return last_launch_status();
}

// ------------------------------------------------------------ instantiations
#define STAG_BLAS_P(P)                                                                                              \
  template int launch_from_canonical<P>(Spinor<P>, const double2*, int, cudaStream_t);                            \
  template int launch_to_canonical<P>(double2*, Spinor<P>, int, cudaStream_t);                                    \
  template int launch_norm2<P>(Spinor<P>, RedScratch, RedTarget, cudaStream_t);                                   \
  template int launch_cg_update<P>(Spinor<Acc<P>::value>, Spinor<Acc<P>::value>, Spinor<P>, Spinor<Acc<P>::value>, \
                                   CgState*, RedScratch, cudaStream_t);                                           \
  template int launch_cg_xpay<P>(Spinor<P>, Spinor<Acc<P>::value>, CgState*, cudaStream_t);                       \
  template int launch_ru_convert_dot<P>(Spinor<Acc<P>::value>, Spinor<64>, Spinor<P>, CgState*, RedScratch,       \
                                        cudaStream_t);                                                            \
  template int launch_ru_p<P>(Spinor<P>, Spinor<Acc<P>::value>, CgState*, cudaStream_t);                          \
  template int launch_ms_r_update<P>(Spinor<Acc<P>::value>, Spinor<Acc<P>::value>, MsState*, RedScratch,          \
                                     cudaStream_t);                                                               \
  template int launch_ms_shift_update<P>(Spinor<Acc<P>::value>*, Spinor<P>*, int, int, Spinor<Acc<P>::value>,    \
                                         MsState*, int, cudaStream_t);
STAG_BLAS_P(64)
STAG_BLAS_P(32)
STAG_BLAS_P(16)
STAG_BLAS_P(15)
STAG_BLAS_P(31)
template int launch_convert<31, 64>(Spinor<31>, Spinor<64>, cudaStream_t);
template int launch_convert<31, 32>(Spinor<31>, Spinor<32>, cudaStream_t);
template int launch_accumulate<64>(Spinor<64>, Spinor<64>, cudaStream_t);
template int launch_accumulate<32>(Spinor<64>, Spinor<32>, cudaStream_t);
template int launch_convert<32, 64>(Spinor<32>, Spinor<64>, cudaStream_t);
template int launch_convert<16, 64>(Spinor<16>, Spinor<64>, cudaStream_t);
template int launch_convert<16, 32>(Spinor<16>, Spinor<32>, cudaStream_t);
template int launch_convert<15, 64>(Spinor<15>, Spinor<64>, cudaStream_t);
template int launch_convert<15, 32>(Spinor<15>, Spinor<32>, cudaStream_t);
template int launch_convert<64, 32>(Spinor<64>, Spinor<32>, cudaStream_t);
template int launch_convert<64, 16>(Spinor<64>, Spinor<16>, cudaStream_t);
template int launch_convert<32, 16>(Spinor<32>, Spinor<16>, cudaStream_t);
template int launch_convert<64, 64>(Spinor<64>, Spinor<64>, cudaStream_t);
template int launch_convert<32, 32>(Spinor<32>, Spinor<32>, cudaStream_t);

}  // namespace stag
