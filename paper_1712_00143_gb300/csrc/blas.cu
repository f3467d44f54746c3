// blas.cu -- the level-1 kernels of the Krylov solvers, each fused with the
// FP64 reduction it feeds (CG is memory-bound, arithmetic intensity about
// 0.26 flop/byte in the paper's measurements, Sec. 4.2, so every extra pass
// over a vector costs as much as its bytes).  One thread per site and colour
// triple, grid-stride, coalesced structure-of-arrays access.  Scalars (alpha,
// beta, zeta ...) are read from the device-resident solver state, never from
// the host, so a whole iteration is queued without a host round trip.
#include "internal.h"

namespace stag {

static constexpr int BB = 256;  // threads per block of the level-1 kernels

static inline int blas_grid(int Vh, int cap) {
  int g = (Vh + BB - 1) / BB;
  return g < cap ? g : cap;
}
static constexpr int NONRED_CAP = 1 << 20;

#define GRID_STRIDE(s, Vh) for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < (Vh); s += gridDim.x * blockDim.x)

// ------------------------------------------------------------ conversions
template <int P> __global__ void k_from_canonical(Spinor<P> out, const double2* __restrict__ in, int Vh) {
  using A2 = typename Prec<P>::A2;
  GRID_STRIDE(s, Vh) {
    A2 o[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double2 v = in[3 * s + c];
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
    for (int c = 0; c < 3; ++c) out[3 * s + c] = make_double2((double)o[c].x, (double)o[c].y);
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
  k_from_canonical<P><<<blas_grid(Vh, NONRED_CAP), BB, 0, st>>>(out, in, Vh);
  return last_launch_status();
}
template <int P> int launch_to_canonical(double2* out, Spinor<P> in, int Vh, cudaStream_t st) {
  ProfScope ps("convert", st);
  k_to_canonical<P><<<blas_grid(Vh, NONRED_CAP), BB, 0, st>>>(out, in, Vh);
  return last_launch_status();
}
template <int PO, int PI> int launch_convert(Spinor<PO> out, Spinor<PI> in, cudaStream_t st) {
  ProfScope ps("convert", st);
  k_convert<PO, PI><<<blas_grid(in.Vh, NONRED_CAP), BB, 0, st>>>(out, in, in.Vh);
  return last_launch_status();
}

int launch_zero(void* p, size_t bytes, cudaStream_t st) { return cuda_status(cudaMemsetAsync(p, 0, bytes, st)); }

// ------------------------------------------------------------ reductions
template <int P> __global__ void k_norm2(Spinor<P> v, RedBuf rb, RedTarget tgt) {
  using A2 = typename Prec<P>::A2;
  double acc[1] = {0.0};
  GRID_STRIDE(s, v.Vh) {
    A2 a[3];
    SpinorLoad<P>::ld(v, s, a);
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[0] += (double)a[c].x * (double)a[c].x + (double)a[c].y * (double)a[c].y;
  }
  grid_reduce<1>(acc, rb, tgt);
}

template <int P> int launch_norm2(Spinor<P> v, RedScratch rs, RedTarget tgt, cudaStream_t st) {
  ProfScope ps("reduce", st);
  k_norm2<P><<<blas_grid(v.Vh, rs.max_grid), BB, 0, st>>>(v, RedBuf{rs.partials, rs.counter}, tgt);
  return last_launch_status();
}

// ------------------------------------------------------------ CG kernels
// xh += alpha p; rh -= alpha Ap; ||rh||^2 -> beta (RED_CG_BETA)
template <int P, int PV>
__global__ void k_cg_update(Spinor<PV> xh, Spinor<PV> rh, Spinor<P> p, Spinor<PV> Ap, CgState* st, RedBuf rb) {
  using A2 = typename Prec<PV>::A2;
  using A = typename Prec<PV>::A;
  if (stopped(&st->flags)) return;
  const A alpha = (A)__ldcg(&st->alpha);
  double acc[1] = {0.0};
  GRID_STRIDE(s, xh.Vh) {
    A2 x[3], r[3], pv[3], ap[3];
    SpinorLoad<PV>::ldw(xh, s, x);
    SpinorLoad<PV>::ldw(rh, s, r);
    SpinorLoad<P>::ld(p, s, pv);
    SpinorLoad<PV>::ld(Ap, s, ap);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      x[c].x += alpha * pv[c].x;
      x[c].y += alpha * pv[c].y;
      r[c].x -= alpha * ap[c].x;
      r[c].y -= alpha * ap[c].y;
      acc[0] += (double)r[c].x * (double)r[c].x + (double)r[c].y * (double)r[c].y;
    }
    SpinorLoad<PV>::st(xh, s, x);
    SpinorLoad<PV>::st(rh, s, r);
  }
  grid_reduce<1>(acc, rb, RedTarget{RED_CG_BETA, st, nullptr});
}

template <int P>
int launch_cg_update(Spinor<Acc<P>::value> xh, Spinor<Acc<P>::value> rh, Spinor<P> p, Spinor<Acc<P>::value> Ap,
                     CgState* state, RedScratch rs, cudaStream_t st) {
  ProfScope ps("blas", st);
  k_cg_update<P, Acc<P>::value>
      <<<blas_grid(xh.Vh, rs.max_grid), BB, 0, st>>>(xh, rh, p, Ap, state, RedBuf{rs.partials, rs.counter});
  return last_launch_status();
}

// p = rh + beta p
template <int P, int PV> __global__ void k_cg_xpay(Spinor<P> p, Spinor<PV> rh, CgState* st) {
  using A2 = typename Prec<P>::A2;
  using A = typename Prec<P>::A;
  if (stopped(&st->flags)) return;
  const A beta = (A)__ldcg(&st->beta);
  GRID_STRIDE(s, p.Vh) {
    A2 pv[3];
    typename Prec<PV>::A2 r[3];
    SpinorLoad<P>::ldw(p, s, pv);
    SpinorLoad<PV>::ld(rh, s, r);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pv[c].x = (A)r[c].x + beta * pv[c].x;
      pv[c].y = (A)r[c].y + beta * pv[c].y;
    }
    SpinorLoad<P>::st(p, s, pv);
  }
}

template <int P> int launch_cg_xpay(Spinor<P> p, Spinor<Acc<P>::value> rh, CgState* state, cudaStream_t st) {
  ProfScope ps("blas", st);
  k_cg_xpay<P, Acc<P>::value><<<blas_grid(p.Vh, NONRED_CAP), BB, 0, st>>>(p, rh, state);
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
  k_accumulate<PV><<<blas_grid(y.Vh, NONRED_CAP), BB, 0, st>>>(y, xh);
  return last_launch_status();
}

// rh = r (converted), <rh, p> (complex) -> RED_RU_ORTHO
template <int P, int PV> __global__ void k_ru_convert_dot(Spinor<PV> rh, Spinor<64> r, Spinor<P> p, CgState* st, RedBuf rb) {
  using A2 = typename Prec<PV>::A2;
  double acc[2] = {0.0, 0.0};
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
      acc[0] += (double)o[c].x * (double)pv[c].x + (double)o[c].y * (double)pv[c].y;
      acc[1] += (double)o[c].x * (double)pv[c].y - (double)o[c].y * (double)pv[c].x;
    }
  }
  grid_reduce<2>(acc, rb, RedTarget{RED_RU_ORTHO, st, nullptr});
}

template <int P>
int launch_ru_convert_dot(Spinor<Acc<P>::value> rh, Spinor<64> r, Spinor<P> p, CgState* state, RedScratch rs,
                          cudaStream_t st) {
  ProfScope ps("reduce", st);
  k_ru_convert_dot<P, Acc<P>::value>
      <<<blas_grid(r.Vh, rs.max_grid), BB, 0, st>>>(rh, r, p, state, RedBuf{rs.partials, rs.counter});
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
  k_ru_p<P, Acc<P>::value><<<blas_grid(p.Vh, NONRED_CAP), BB, 0, st>>>(p, rh, state);
  return last_launch_status();
}

// ------------------------------------------------------------ multi-shift
template <int PV> __global__ void k_ms_r_update(Spinor<PV> r, Spinor<PV> Ap, MsState* ms, RedBuf rb) {
  using A2 = typename Prec<PV>::A2;
  using A = typename Prec<PV>::A;
  if (stopped(&ms->cg.flags)) return;
  const A alpha = (A)__ldcg(&ms->cg.alpha);
  double acc[1] = {0.0};
  GRID_STRIDE(s, r.Vh) {
    A2 rv[3], ap[3];
    SpinorLoad<PV>::ldw(r, s, rv);
    SpinorLoad<PV>::ld(Ap, s, ap);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      rv[c].x -= alpha * ap[c].x;
      rv[c].y -= alpha * ap[c].y;
      acc[0] += (double)rv[c].x * (double)rv[c].x + (double)rv[c].y * (double)rv[c].y;
    }
    SpinorLoad<PV>::st(r, s, rv);
  }
  grid_reduce<1>(acc, rb, RedTarget{RED_MS_BETA, ms, nullptr});
}

template <int P>
int launch_ms_r_update(Spinor<Acc<P>::value> r, Spinor<Acc<P>::value> Ap, MsState* state, RedScratch rs,
                       cudaStream_t st) {
  ProfScope ps("blas", st);
  k_ms_r_update<Acc<P>::value>
      <<<blas_grid(r.Vh, rs.max_grid), BB, 0, st>>>(r, Ap, state, RedBuf{rs.partials, rs.counter});
  return last_launch_status();
}

template <int P> struct ShiftPtrs {
  Spinor<64> x[MAX_SHIFTS];
  Spinor<P> p[MAX_SHIFTS];
};

// For every shift still iterating: x_s += alpha_s p_s; p_s = zeta_s r + beta_s p_s.
// The base shift's direction (index `base`) is always updated: it drives the
// shared Krylov space.
template <int P, int PV>
__global__ void k_ms_shift_update(ShiftPtrs<P> sp, int nshift, int base, Spinor<PV> r, MsState* ms, int expect_iter) {
  using A2 = typename Prec<P>::A2;
  using A = typename Prec<P>::A;
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
      const double as = __ldcg(&ms->alpha_s[k]), bs = __ldcg(&ms->beta_s[k]), zn = __ldcg(&ms->zeta_next[k]);
      A2 pv[3];
      SpinorLoad<P>::ldw(sp.p[k], s, pv);
      if (act) {
        double2 xv[3];
        SpinorLoad<64>::ldw(sp.x[k], s, xv);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          xv[c].x += as * (double)pv[c].x;
          xv[c].y += as * (double)pv[c].y;
        }
        SpinorLoad<64>::st(sp.x[k], s, xv);
      }
      const A z = (A)zn, b = (A)bs;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pv[c].x = z * (A)rv[c].x + b * pv[c].x;
        pv[c].y = z * (A)rv[c].y + b * pv[c].y;
      }
      SpinorLoad<P>::st(sp.p[k], s, pv);
    }
  }
}

template <int P>
int launch_ms_shift_update(Spinor<64>* xs, Spinor<P>* ps, int nshift, int base, Spinor<Acc<P>::value> r,
                           MsState* state, int expect_iter, cudaStream_t st) {
  if (nshift > MAX_SHIFTS) return STAG_EINVAL;
  ShiftPtrs<P> sp;
  for (int k = 0; k < nshift; ++k) {
    sp.x[k] = xs[k];
    sp.p[k] = ps[k];
  }
  ProfScope pscope("blas", st);
  k_ms_shift_update<P, Acc<P>::value><<<blas_grid(r.Vh, NONRED_CAP), BB, 0, st>>>(sp, nshift, base, r, state, expect_iter);
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
  template int launch_ms_shift_update<P>(Spinor<64>*, Spinor<P>*, int, int, Spinor<Acc<P>::value>, MsState*,     \
                                         int, cudaStream_t);
STAG_BLAS_P(64)
STAG_BLAS_P(32)
STAG_BLAS_P(16)
STAG_BLAS_P(15)
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
