// batch_kernels.cuh -- kernels of the multi-right-hand-side CG: the
// per-system level-1 kernels and the control kernels of the graph-resident
// loop, all on the MRHS layout of dslash_mrhs.cuh (the N-RHS Dslash kernels
// are in mrhs_kernels.cuh).  Each system i of a group reads its own scalars
// (alpha_i, beta_i ...) from the group's McgState.
#pragma once
#include "dslash_mrhs.cuh"

namespace stag {

// ------------------------------------------------------------ level 1
// grid-stride over sites, all N systems of a site per trip
#define MGRID(s, Vh) for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < (Vh); s += gridDim.x * blockDim.x)

// xh_r += alpha_r p_r; rh_r -= alpha_r Ap_r; ||rh_r||^2 -> RED_MCG_BETA
template <int P, int N>
__global__ void __launch_bounds__(256) k_mcg_update(SpinorM<Acc<P>::value> xh, SpinorM<Acc<P>::value> rh,
                                                     SpinorM<P> p, SpinorM<Acc<P>::value> Ap, McgState* g,
                                                     RedBuf rb) {
  constexpr int PV = Acc<P>::value;
  using A2 = typename Prec<PV>::A2;
  using A = typename Prec<PV>::A;
  if (stopped(&g->flags)) return;
  A alpha[N];
#pragma unroll
  for (int r = 0; r < N; ++r) alpha[r] = (A)__ldcg(&g->sys[r].alpha);
  Acc1<A> acc[N];
  MGRID(s, xh.Vh) {
#pragma unroll
    for (int r = 0; r < N; ++r) {
      A2 x[3], rv[3], ap[3];
      typename Prec<P>::A2 pv[3];
      SpinorLoadM<PV>::ldw(xh, s, r, x);
      SpinorLoadM<PV>::ldw(rh, s, r, rv);
      SpinorLoadM<P>::ld(p, s, r, pv);
      SpinorLoadM<PV>::ld(Ap, s, r, ap);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        x[c].x += alpha[r] * (A)pv[c].x;
        x[c].y += alpha[r] * (A)pv[c].y;
        rv[c].x -= alpha[r] * ap[c].x;
        rv[c].y -= alpha[r] * ap[c].y;
        acc[r].add_prod(rv[c].x, rv[c].x);
        acc[r].add_prod(rv[c].y, rv[c].y);
      }
      SpinorLoadM<PV>::st(xh, s, r, x);
      SpinorLoadM<PV>::st(rh, s, r, rv);
    }
  }
  grid_reduce_acc<N>(acc, rb, RedTarget{RED_MCG_BETA, g, nullptr});
}

// Re<p_r, Ap_r> -> alpha_r (RED_MCG_ALPHA): the CG dot product read back
// from the operator's stored output, in a level-1 pass of its own (see the
// group's iteration for why it is not fused into the operator kernel).
template <int P, int N>
__global__ void __launch_bounds__(256) k_mcg_pap(SpinorM<P> p, SpinorM<Acc<P>::value> Ap, McgState* g, RedBuf rb) {
  constexpr int PV = Acc<P>::value;
  using A = typename Prec<PV>::A;
  if (stopped(&g->flags)) return;
  Acc1<A> acc[N];
  MGRID(s, p.Vh) {
#pragma unroll
    for (int r = 0; r < N; ++r) {
      typename Prec<P>::A2 pv[3];
      typename Prec<PV>::A2 ap[3];
      SpinorLoadM<P>::ld(p, s, r, pv);
      SpinorLoadM<PV>::ld(Ap, s, r, ap);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc[r].add_prod((A)pv[c].x, ap[c].x);
        acc[r].add_prod((A)pv[c].y, ap[c].y);
      }
    }
  }
  grid_reduce_acc<N>(acc, rb, RedTarget{RED_MCG_ALPHA, g, nullptr});
}

// p_r = rh_r + beta_r p_r
template <int P, int N>
__global__ void __launch_bounds__(256) k_mcg_xpay(SpinorM<P> p, SpinorM<Acc<P>::value> rh, McgState* g,
                                                   const int* skip) {
  using A2 = typename Prec<P>::A2;
  using A = typename Prec<P>::A;
  if (stopped(&g->flags) || (skip && __ldcg(skip))) return;
  A beta[N];
#pragma unroll
  for (int r = 0; r < N; ++r) beta[r] = (A)__ldcg(&g->sys[r].beta);
  MGRID(s, p.Vh) {
#pragma unroll
    for (int r = 0; r < N; ++r) {
      A2 pv[3];
      typename Prec<Acc<P>::value>::A2 rv[3];
      SpinorLoadM<P>::ldw(p, s, r, pv);
      SpinorLoadM<Acc<P>::value>::ld(rh, s, r, rv);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pv[c].x = (A)rv[c].x + beta[r] * pv[c].x;
        pv[c].y = (A)rv[c].y + beta[r] * pv[c].y;
      }
      SpinorLoadM<P>::st(p, s, r, pv);
    }
  }
}

// y_r += xh_r; xh_r = 0
template <int PV, int N> __global__ void k_maccumulate(SpinorM<64> y, SpinorM<PV> xh, const int* stop) {
  if (stopped(stop)) return;
  MGRID(s, y.Vh) {
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
      }
      SpinorLoadM<64>::st(y, s, r, a);
      SpinorLoadM<PV>::st(xh, s, r, z);
    }
  }
}

// rh_r = r64_r (rounded); <rh_r, p_r> -> RED_MCG_RU_ORTHO (2N values)
template <int P, int N>
__global__ void k_mru_convert_dot(SpinorM<Acc<P>::value> rh, SpinorM<64> r64, SpinorM<P> p, McgState* g, RedBuf rb,
                                  const int* stop) {
  constexpr int PV = Acc<P>::value;
  using A2 = typename Prec<PV>::A2;
  using A = typename Prec<PV>::A;
  if (stopped(stop)) return;  // every block alike: no partial reduction is left behind
  Acc1<A> re[N], im[N];
  MGRID(s, r64.Vh) {
#pragma unroll
    for (int r = 0; r < N; ++r) {
      double2 a[3];
      A2 o[3];
      typename Prec<P>::A2 pv[3];
      SpinorLoadM<64>::ld(r64, s, r, a);
      SpinorLoadM<P>::ld(p, s, r, pv);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        o[c].x = a[c].x;
        o[c].y = a[c].y;
      }
      SpinorLoadM<PV>::st(rh, s, r, o);
      SpinorLoadM<PV>::ldw(rh, s, r, o);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        re[r].add_prod(o[c].x, (A)pv[c].x);
        re[r].add_prod(o[c].y, (A)pv[c].y);
        im[r].add_prod(o[c].x, (A)pv[c].y);
        im[r].add_prod(-o[c].y, (A)pv[c].x);
      }
    }
  }
  Acc1<A> all[2 * N];
#pragma unroll
  for (int r = 0; r < N; ++r) {
    all[2 * r] = re[r];
    all[2 * r + 1] = im[r];
  }
  grid_reduce_acc<2 * N>(all, rb, RedTarget{RED_MCG_RU_ORTHO, g, nullptr});
}

// p_r = rh_r + beta_r (p_r - c_r rh_r)
template <int P, int N>
__global__ void k_mru_p(SpinorM<P> p, SpinorM<Acc<P>::value> rh, McgState* g, const int* stop) {
  using A2 = typename Prec<P>::A2;
  using A = typename Prec<P>::A;
  if (stopped(stop)) return;
  A beta[N], cr[N], ci[N];
#pragma unroll
  for (int r = 0; r < N; ++r) {
    beta[r] = (A)__ldcg(&g->sys[r].beta);
    cr[r] = (A)__ldcg(&g->sys[r].ortho_re);
    ci[r] = (A)__ldcg(&g->sys[r].ortho_im);
  }
  MGRID(s, p.Vh) {
#pragma unroll
    for (int r = 0; r < N; ++r) {
      A2 pv[3];
      typename Prec<Acc<P>::value>::A2 rv[3];
      SpinorLoadM<P>::ldw(p, s, r, pv);
      SpinorLoadM<Acc<P>::value>::ld(rh, s, r, rv);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        A rx = (A)rv[c].x, ry = (A)rv[c].y;
        A qx = pv[c].x - (cr[r] * rx - ci[r] * ry);
        A qy = pv[c].y - (cr[r] * ry + ci[r] * rx);
        pv[c].x = rx + beta[r] * qx;
        pv[c].y = ry + beta[r] * qy;
      }
      SpinorLoadM<P>::st(p, s, r, pv);
    }
  }
}

// MRHS out (systems 0..N-1) <- canonical in[r] for r < nreal, zero for the rest
template <int P, int N> __global__ void k_mfrom_canonical(SpinorM<P> out, const double2* __restrict__ in, int nreal) {
  using A2 = typename Prec<P>::A2;
  MGRID(s, out.Vh) {
#pragma unroll
    for (int r = 0; r < N; ++r) {
      A2 o[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double2 v = r < nreal ? in[((size_t)r * out.Vh + s) * 3 + c] : make_double2(0.0, 0.0);
        o[c].x = v.x;
        o[c].y = v.y;
      }
      SpinorLoadM<P>::st(out, s, r, o);
    }
  }
}

// canonical out[r] <- MRHS in, r < nreal
template <int P, int N> __global__ void k_mto_canonical(double2* __restrict__ out, SpinorM<P> in, int nreal) {
  using A2 = typename Prec<P>::A2;
  MGRID(s, in.Vh) {
#pragma unroll
    for (int r = 0; r < N; ++r) {
      if (r >= nreal) break;
      A2 o[3];
      SpinorLoadM<P>::ld(in, s, r, o);
#pragma unroll
      for (int c = 0; c < 3; ++c) out[((size_t)r * in.Vh + s) * 3 + c] = make_double2((double)o[c].x, (double)o[c].y);
    }
  }
}

template <int PO, int PI, int N> __global__ void k_mconvert(SpinorM<PO> out, SpinorM<PI> in) {
  MGRID(s, in.Vh) {
#pragma unroll
    for (int r = 0; r < N; ++r) {
      typename Prec<PI>::A2 a[3];
      typename Prec<PO>::A2 o[3];
      SpinorLoadM<PI>::ld(in, s, r, a);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        o[c].x = a[c].x;
        o[c].y = a[c].y;
      }
      SpinorLoadM<PO>::st(out, s, r, o);
    }
  }
}

// ||v_r||^2 for every system -> RED_STORE (N values)
template <int P, int N> __global__ void k_mnorm2(SpinorM<P> v, RedBuf rb, RedTarget tgt) {
  using A = typename Prec<P>::A;
  Acc1<A> acc[N];
  MGRID(s, v.Vh) {
#pragma unroll
    for (int r = 0; r < N; ++r) {
      typename Prec<P>::A2 a[3];
      SpinorLoadM<P>::ld(v, s, r, a);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        acc[r].add_prod(a[c].x, a[c].x);
        acc[r].add_prod(a[c].y, a[c].y);
      }
    }
  }
  grid_reduce_acc<N>(acc, rb, tgt);
}

#undef MGRID

// ------------------------------------------------------------ graph-resident loop control
// Before a group's reliable-update kernels in each round of the loop: is an
// update due (a flag set by the last chunk)?  ru_skip = 0 lets the update's
// kernels run, F_CONVERGED makes them return at once.
// With double-float updates the gate also picks between them and the one
// FP64 update that moves the anchor (see McgState): ru_skip gates the
// double-float kernels, ru_skip64 the FP64 ones.
__device__ inline bool mcg_anchor_due(const McgState* g) {
  if (!g->use_df || g->anchored) return false;
  for (int i = 0; i < g->n; ++i)
    if (((g->active >> i) & 1) && !(g->sys[i].rr < g->anchor_rr[i])) return false;
  return true;
}

__global__ void k_mcg_ru_gate(McgState* g) {
  g->ru_skip = F_CONVERGED;
  g->ru_skip64 = F_CONVERGED;
  if (g->done) return;
  if (g->flags & F_BREAKDOWN) {
    g->done = 1;
    g->status = STAG_EBREAKDOWN;
    return;
  }
  if (!(g->flags & (F_CONVERGED | F_NEED_RU | F_ITER_CAP))) return;
  if (mcg_anchor_due(g)) {
    g->ru_skip64 = 0;
    g->anchored = 1;
  } else if (g->use_df) {
    g->ru_skip = 0;
  } else {
    g->ru_skip64 = 0;
  }
}

// After them: retire the group (every system at its target, an error, the
// iteration cap) or let it iterate on from the new direction.
__global__ void k_mcg_ru_decide(McgState* g) {
  if (g->ru_skip && g->ru_skip64) return;
  g->ru_skip = F_CONVERGED;
  g->ru_skip64 = F_CONVERGED;
  if (g->flags & F_BREAKDOWN) {
    g->done = 1;
    g->status = STAG_EBREAKDOWN;
  } else if (g->active == 0) {
    g->done = 1;
    g->flags |= F_CONVERGED;
  } else if (g->iter >= g->max_iter) {
    g->done = 1;
    g->status = STAG_ENOTCONV;
    g->flags |= F_ITER_CAP;
  } else {
    g->skip_xpay = 1;  // the update formed the direction already
  }
}

__global__ void k_mcg_clear_skip(McgState* g) { g->skip_xpay = 0; }

// End of a round: another one while any group is live and the budget of
// rounds lasts (the budget bounds the loop whatever the solver state).
__global__ void k_mcg_loop_cond(McgState* const* gs, int ng, int* budget, cudaGraphConditionalHandle h) {
  int live = 0;
  for (int k = 0; k < ng; ++k) live |= !__ldcg(&gs[k]->done);
  const int b = *budget - 1;
  *budget = b;
  cudaGraphSetConditional(h, (live && b > 0) ? 1u : 0u);
}

}  // namespace stag
