// solvers.cu -- host drivers of the even-odd CG solvers.
//
// Single-mass CG on M = m^2 - D_eo D_oe (Sec. 1: the staggered QPhiX library
// provides single-mass and multi-shift CG; Sec. 4: about 90% of the run time
// of the paper's benchmark application is spent there) and the multi-shift
// CG of Sec. 4.1.  Mixed precision follows the paper's note that QUDA
// supports mixed-precision solves and that single precision runs about twice
// as fast as double (Sec. 3, Sec. 4): the Krylov loop runs on the FP32 or
// FP16 operator and vectors, while the solution is accumulated in FP64 and
// the true residual b - M y is recomputed in FP64 ("reliable update") each
// time the iterated residual has dropped by a factor delta, and at the end.
//
// Every scalar of the recurrences lives in device memory (CgState / MsState)
// and is produced by the last block of a fused reduction kernel, so the host
// queues `check_interval` iterations at a time and synchronises only to look
// at the state between such chunks.  Kernels of a chunk that follow
// convergence see the stop flag and return immediately.
#include <chrono>
#include <cmath>
#include <vector>

#include "internal.h"

namespace stag {

namespace {

struct PinnedState {
  void* h = nullptr;
  PinnedState(size_t n) {
    if (cudaMallocHost(&h, n) != cudaSuccess) {
      cudaGetLastError();
      h = nullptr;
    }
  }
  ~PinnedState() {
    if (h) cudaFreeHost(h);
  }
};

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

#define TRY(...)               \
  do {                         \
    int _s = (__VA_ARGS__);    \
    if (_s) return _s;         \
  } while (0)

template <int P> Spinor<P> none_spinor(int Vh) { return Spinor<P>{nullptr, Vh}; }

}  // namespace

// FP64: r = b - shift y + D_eo D_oe y  (the true residual), ||r||^2 -> tgt
static int true_residual(stag_lattice_s* lat, Spinor<64> r, Spinor<64> b, Spinor<64> y, Spinor<64> t64, double shift,
                         RedScratch rs, RedTarget tgt, cudaStream_t st) {
  TRY(launch_dslash<64>(lat, t64, y, 1, nullptr, st));
  return launch_dslash_epi<64>(lat, r, t64, 0, y, -shift, b, 1.0, 1.0, 2, rs, tgt, nullptr, st);
}

// Solve (m^2 + sigma - D_eo D_oe) x = b with sloppy precision P (P = 64: plain
// FP64 CG).  x_can/b_can: canonical device fields.
template <int P>
static int cg_solve(stag_lattice_s* lat, double2* x_can, const double2* b_can, double shift,
                    const stag_solve_params& prm, stag_solve_info* info, cudaStream_t st) {
  constexpr int PV = Acc<P>::value;
  const double t0 = now_s();
  const int Vh = lat->g.Vh;
  int s = 0;
  Spinor<64> b64 = ws_spinor<64>(lat, "cg.b", &s);
  Spinor<64> y64 = ws_spinor<64>(lat, "cg.y", &s);
  Spinor<64> r64 = ws_spinor<64>(lat, "cg.r64", &s);
  Spinor<64> t64 = ws_spinor<64>(lat, "cg.t64", &s);
  Spinor<P> p = ws_spinor<P>(lat, "cg.p", &s);
  Spinor<P> t = ws_spinor<P>(lat, "cg.t", &s);
  Spinor<PV> Ap = ws_spinor<PV>(lat, "cg.Ap", &s);
  Spinor<PV> xh = ws_spinor<PV>(lat, "cg.xh", &s);
  Spinor<PV> rh = ws_spinor<PV>(lat, "cg.rh", &s);
  CgState* dst = (CgState*)lat->ws.get("cg.state", sizeof(CgState), &s);
  double* dscal = (double*)lat->ws.get("cg.scalars", 64, &s);
  // reliable updates in double-float when the handle holds that link copy,
  // measured from an anchor (ya64, its residual radf): r = r_a - M (y - y_a)
  const bool use_df = P != 64 && lat->links[STAG_DF64].present;
  DfField radf{nullptr, Vh}, ydf{nullptr, Vh}, tdf{nullptr, Vh}, rdf{nullptr, Vh};
  Spinor<64> ya64{nullptr, Vh};
  if (use_df) {
    ya64 = ws_spinor<64>(lat, "cg.ya", &s);
    radf.v = (float4*)lat->ws.get("cg.radf", df_bytes(Vh), &s);
    ydf.v = (float4*)lat->ws.get("cg.ydf", df_bytes(Vh), &s);
    tdf.v = (float4*)lat->ws.get("cg.tdf", df_bytes(Vh), &s);
    rdf.v = (float4*)lat->ws.get("cg.rdf", df_bytes(Vh), &s);
  }
  if (s) return s;
  RedScratch rs;
  TRY(get_red_scratch(lat, "cg", &rs, 3));
  auto true_residual_df = [&]() -> int {
    TRY(launch_dslash_df(lat, tdf, ydf, 1, 1, nullptr, st));
    return launch_dslash_df_epi(lat, rdf, tdf, 1, 0, ydf, -shift, radf, 1.0, 1.0, nullptr, st);
  };
  PinnedState pin(sizeof(CgState) + 64);
  if (!pin.h) return STAG_ENOMEM;
  CgState* hs = (CgState*)pin.h;
  double* hscal = (double*)((char*)pin.h + sizeof(CgState));

  // ||b||^2 and the initial residual
  TRY(launch_from_canonical<64>(b64, b_can, Vh, st));
  TRY(launch_norm2<64>(b64, rs, RedTarget{RED_STORE, nullptr, dscal}, st));
  if (use_df) {
    // the anchor starts at (0, b)
    TRY(launch_df_from_double(radf, (const double2*)b64.v, 1, st));
    TRY(launch_zero(ya64.v, spinor_bytes<64>(Vh), st));
  }
  bool anchored = false;
  if (prm.use_initial_guess) {
    TRY(launch_from_canonical<64>(y64, x_can, Vh, st));
    if (use_df) {
      TRY(launch_df_from_double(ydf, (const double2*)y64.v, 1, st));
      TRY(true_residual_df());
      TRY(launch_norm2_df(rdf, 1, rs, RedTarget{RED_STORE, nullptr, dscal + 1}, st));
    } else {
      TRY(true_residual(lat, r64, b64, y64, t64, shift, rs, RedTarget{RED_STORE, nullptr, dscal + 1}, st));
    }
  } else {
    TRY(launch_zero(y64.v, spinor_bytes<64>(Vh), st));
    TRY(cuda_status(cudaMemcpyAsync(r64.v, b64.v, spinor_bytes<64>(Vh), cudaMemcpyDeviceToDevice, st)));
    TRY(cuda_status(cudaMemcpyAsync(dscal + 1, dscal, sizeof(double), cudaMemcpyDeviceToDevice, st)));
  }
  TRY(cuda_status(cudaMemcpyAsync(hscal, dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost, st)));
  TRY(cuda_status(cudaStreamSynchronize(st)));
  const double bb = hscal[0], rr0 = hscal[1];
  if (info) {
    info->iters = 0;
    info->reliable_updates = 0;
    info->converged = 0;
    info->status = STAG_OK;
    info->true_rel_resid = bb > 0 ? std::sqrt(rr0 / bb) : 0.0;
  }
  if (!(bb > 0.0)) {  // b = 0: x = 0 solves it exactly
    TRY(launch_zero(x_can, sizeof(double2) * 3 * (size_t)Vh, st));
    TRY(cuda_status(cudaStreamSynchronize(st)));
    if (info) {
      info->converged = 1;
      info->true_rel_resid = 0.0;
      info->seconds = now_s() - t0;
    }
    return STAG_OK;
  }
  const double target = prm.tol * prm.tol * bb;
  int status = STAG_OK;
  CgState h{};
  h.rr = rr0;
  h.rr_prev = rr0;
  h.target = target;
  h.rr_max = rr0;
  h.delta2 = (P == 64) ? 0.0 : prm.delta * prm.delta;
  h.rr_true = rr0;
  h.shift = shift;
  h.iter = 0;
  h.max_iter = prm.max_iter;
  h.flags = 0;
  *hs = h;
  if (rr0 > target && prm.max_iter > 0) {
    TRY(cuda_status(cudaMemcpyAsync(dst, hs, sizeof(CgState), cudaMemcpyHostToDevice, st)));
    // sloppy copies: rh = r, xh = 0, p = rh
    if (use_df && prm.use_initial_guess)
      TRY(launch_convert_from_df<PV>(rh.v, rdf, 1, st));
    else
      TRY(launch_convert<PV, 64>(rh, r64, st));
    TRY(launch_zero(xh.v, spinor_bytes<PV>(Vh), st));
    TRY(launch_convert<P, PV>(p, rh, st));
    const int* flags = &dst->flags;
    const int C = prm.check_interval > 0 ? prm.check_interval : 16;
    bool pending_p = false;
    // the device caps the iterations (F_ITER_CAP); the host bound on chunks
    // is a second, independent guard
    long long chunks = 0, max_chunks = (long long)prm.max_iter / C + 64;
    for (;;) {
      if (++chunks > max_chunks) {
        status = STAG_ENOTCONV;
        break;
      }
      const long long mark = prof_mark();
      for (int i = 0; i < C; ++i) {
        if (pending_p) TRY(launch_cg_xpay<P>(p, rh, dst, st));
        TRY(launch_dslash<P>(lat, t, p, 1, flags, st));
        TRY(launch_dslash_epi<P>(lat, Ap, t, 0, p, shift, none_spinor<PV>(Vh), 0.0, -1.0, 1, rs,
                                 RedTarget{RED_CG_ALPHA, dst, nullptr}, flags, st));
        TRY(launch_cg_update<P>(xh, rh, p, Ap, dst, rs, st));
        pending_p = true;
      }
      TRY(cuda_status(cudaMemcpyAsync(hs, dst, sizeof(CgState), cudaMemcpyDeviceToHost, st)));
      TRY(cuda_status(cudaStreamSynchronize(st)));
      if (hs->flags & F_STOP) prof_discard_since(mark);  // launches after the flag returned at once
      prof_flush_completed();
      if (hs->flags & F_BREAKDOWN) {
        status = STAG_EBREAKDOWN;
        break;
      }
      if (hs->flags & (F_CONVERGED | F_NEED_RU | F_ITER_CAP)) {
        // reliable update: y += xh, r = b - M y (FP64-class), rh = r, and
        // the search direction re-orthogonalised against the new residual
        auto update = [&](bool df) -> int {
          if constexpr (P != 64) {
            if (df) {
              TRY(launch_accumulate_df<PV>(y64.v, xh.v, ydf, ya64.v, 1, nullptr, st));
              TRY(true_residual_df());
              TRY(launch_ru_convert_dot_df<P>(rh.v, rdf, p.v, 1, rs, RedTarget{RED_RU_BOTH, dst, nullptr}, nullptr,
                                              st));
            }
          }
          if (!df) {
            TRY(launch_accumulate<PV>(y64, xh, st));
            TRY(true_residual(lat, r64, b64, y64, t64, shift, rs, RedTarget{RED_RU_RESID, dst, nullptr}, st));
            TRY(launch_ru_convert_dot<P>(rh, r64, p, dst, rs, st));
          }
          TRY(launch_ru_p<P>(p, rh, dst, st));
          if (!df && use_df) {
            // an FP64 update moves the anchor of the double-float ones
            TRY(launch_df_anchor(ya64.v, radf, y64.v, r64.v, 1, nullptr, st));
            anchored = true;
          }
          TRY(cuda_status(cudaMemcpyAsync(hs, dst, sizeof(CgState), cudaMemcpyDeviceToHost, st)));
          return cuda_status(cudaStreamSynchronize(st));
        };
        // double-float, except the one FP64 update that moves the anchor once
        // the iterated residual is small
        TRY(update(use_df && (anchored || !(hs->rr < kDfAnchorRel2 * bb))));
        pending_p = false;
        // a double-float residual at the target is judged once more in FP64
        // (one FP64 operator pair per solve): the final verdict is FP64's
        if (use_df && !(hs->flags & F_BREAKDOWN) && hs->rr_true <= target) TRY(update(false));
        if (hs->flags & F_BREAKDOWN) {
          status = STAG_EBREAKDOWN;
          break;
        }
        if (hs->rr_true <= target) break;
        if (hs->iter >= prm.max_iter) {
          status = STAG_ENOTCONV;
          break;
        }
      }
    }
    h = *hs;
  }
  TRY(launch_to_canonical<64>(x_can, y64, Vh, st));
  TRY(cuda_status(cudaStreamSynchronize(st)));
  if (info) {
    info->iters = h.iter;
    info->reliable_updates = h.reliable_updates;
    info->true_rel_resid = std::sqrt(h.rr_true / bb);
    info->converged = h.rr_true <= target;
    info->status = status;
    info->seconds = now_s() - t0;
  }
  return status;
}

// Multi-shift CG in sloppy precision P (solution vectors in the loop's vector
// precision: FP64 for P = 64, FP32 otherwise), followed by a per-shift CG
// refinement, accumulated in FP64, of every shift whose FP64 true residual
// misses the target.
template <int P>
static int ms_solve(stag_lattice_s* lat, double2* const* x_can, const double2* b_can, double mass,
                    const double* shifts, int ns, const stag_solve_params& prm, stag_solve_info* infos,
                    cudaStream_t st) {
  constexpr int PV = Acc<P>::value;
  const double t0 = now_s();
  const int Vh = lat->g.Vh;
  int s = 0;
  int base = 0;
  for (int k = 1; k < ns; ++k)
    if (shifts[k] < shifts[base]) base = k;
  Spinor<64> b64 = ws_spinor<64>(lat, "ms.b", &s);
  Spinor<PV> r = ws_spinor<PV>(lat, "ms.r", &s);
  Spinor<PV> Ap = ws_spinor<PV>(lat, "ms.Ap", &s);
  Spinor<P> t = ws_spinor<P>(lat, "ms.t", &s);
  std::vector<Spinor<PV>> xs(ns);
  std::vector<Spinor<P>> ps(ns);
  for (int k = 0; k < ns; ++k) {
    xs[k] = ws_spinor<PV>(lat, "ms.x" + std::to_string(k), &s);
    ps[k] = ws_spinor<P>(lat, "ms.p" + std::to_string(k), &s);
  }
  MsState* dst = (MsState*)lat->ws.get("ms.state", sizeof(MsState), &s);
  double* dscal = (double*)lat->ws.get("ms.scalars", 64, &s);
  if (s) return s;
  RedScratch rs;
  TRY(get_red_scratch(lat, "ms", &rs));
  PinnedState pin(sizeof(MsState) + 64);
  if (!pin.h) return STAG_ENOMEM;
  MsState* hs = (MsState*)pin.h;
  double* hscal = (double*)((char*)pin.h + sizeof(MsState));

  TRY(launch_from_canonical<64>(b64, b_can, Vh, st));
  TRY(launch_norm2<64>(b64, rs, RedTarget{RED_STORE, nullptr, dscal}, st));
  TRY(cuda_status(cudaMemcpyAsync(hscal, dscal, sizeof(double), cudaMemcpyDeviceToHost, st)));
  TRY(cuda_status(cudaStreamSynchronize(st)));
  const double bb = hscal[0];
  for (int k = 0; k < ns && infos; ++k) infos[k] = stag_solve_info{0, 0, 0, STAG_OK, 1.0, 0.0, 0};
  if (!(bb > 0.0)) {
    for (int k = 0; k < ns; ++k) TRY(launch_zero(x_can[k], sizeof(double2) * 3 * (size_t)Vh, st));
    TRY(cuda_status(cudaStreamSynchronize(st)));
    for (int k = 0; k < ns && infos; ++k) infos[k].converged = 1, infos[k].true_rel_resid = 0.0;
    return STAG_OK;
  }
  const double ms_tol = (P == 64 || prm.ms_tol <= 0.0) ? prm.tol : std::max(prm.ms_tol, prm.tol);
  const double shift0 = mass * mass + shifts[base];
  MsState h{};
  h.cg.rr = bb;
  h.cg.rr_prev = bb;
  h.cg.target = 0.0;  // shifts stop individually (stop mask)
  h.cg.rr_max = bb;
  h.cg.delta2 = 0.0;
  h.cg.shift = shift0;
  h.cg.max_iter = prm.max_iter;
  h.nshift = ns;
  h.active_mask = (int)((ns >= 31) ? 0x7fffffff : ((1u << ns) - 1));
  h.stop_mask = 0;
  h.sqrt_target_bb = ms_tol * std::sqrt(bb);
  h.alpha_prev = 1.0;
  h.beta_prev = 0.0;
  for (int k = 0; k < ns; ++k) {
    h.delta[k] = shifts[k] - shifts[base];
    h.zeta_prev[k] = h.zeta[k] = h.zeta_next[k] = 1.0;
    h.alpha_s[k] = h.beta_s[k] = 0.0;
    h.iters[k] = 0;
  }
  *hs = h;
  TRY(cuda_status(cudaMemcpyAsync(dst, hs, sizeof(MsState), cudaMemcpyHostToDevice, st)));
  TRY(launch_convert<PV, 64>(r, b64, st));
  for (int k = 0; k < ns; ++k) {
    TRY(launch_zero(xs[k].v, spinor_bytes<PV>(Vh), st));
    TRY(launch_convert<P, 64>(ps[k], b64, st));
  }
  int status = STAG_OK;
  const int* flags = &dst->cg.flags;
  const int C = prm.check_interval > 0 ? prm.check_interval : 16;
  int iter0 = 0;
  long long chunks = 0, max_chunks = (long long)prm.max_iter / C + 64;
  for (;;) {
    if (++chunks > max_chunks) {
      status = STAG_ENOTCONV;
      break;
    }
    const long long mark = prof_mark();
    for (int i = 0; i < C; ++i) {
      TRY(launch_dslash<P>(lat, t, ps[base], 1, flags, st));
      TRY(launch_dslash_epi<P>(lat, Ap, t, 0, ps[base], shift0, none_spinor<PV>(Vh), 0.0, -1.0, 1, rs,
                               RedTarget{RED_MS_ALPHA, dst, nullptr}, flags, st));
      TRY(launch_ms_r_update<P>(r, Ap, dst, rs, st));
      TRY(launch_ms_shift_update<P>(xs.data(), ps.data(), ns, base, r, dst, iter0 + i + 1, st));
    }
    TRY(cuda_status(cudaMemcpyAsync(hs, dst, sizeof(MsState), cudaMemcpyDeviceToHost, st)));
    TRY(cuda_status(cudaStreamSynchronize(st)));
    if (hs->cg.flags & F_STOP) prof_discard_since(mark);
    prof_flush_completed();
    iter0 = hs->cg.iter;
    if (hs->cg.flags & F_BREAKDOWN) {
      status = STAG_EBREAKDOWN;
      break;
    }
    if (hs->cg.flags & (F_CONVERGED | F_ITER_CAP)) break;
  }
  h = *hs;
  // per-shift verification and refinement from x_s
  int worst = status;
  for (int k = 0; k < ns; ++k) TRY(launch_to_canonical<PV>(x_can[k], xs[k], Vh, st));
  if (status == STAG_OK) {
    stag_solve_params rp = prm;
    rp.use_initial_guess = 1;
    for (int k = 0; k < ns; ++k) {
      stag_solve_info ri{};
      int rsx = cg_solve<P>(lat, x_can[k], b_can, mass * mass + shifts[k], rp, &ri, st);
      if (infos) {
        infos[k].iters = h.iters[k] + ri.iters;
        infos[k].reliable_updates = ri.reliable_updates;
        infos[k].converged = ri.converged;
        infos[k].true_rel_resid = ri.true_rel_resid;
        infos[k].status = rsx;
      }
      if (rsx && !worst) worst = rsx;
    }
  } else if (infos) {
    for (int k = 0; k < ns; ++k) infos[k].status = status, infos[k].iters = h.iters[k];
  }
  TRY(cuda_status(cudaStreamSynchronize(st)));
  const double t1 = now_s();
  for (int k = 0; k < ns && infos; ++k) infos[k].seconds = t1 - t0;
  return worst;
}

}  // namespace stag

using namespace stag;

namespace stag {
int learned_solve(stag_lattice_s* lat, double2* x, const double2* b, double mass, const stag_solve_params& prm,
                  stag_solve_info* info, cudaStream_t st);
}

static int check_params(const stag_solve_params* p) {
  if (!p) return STAG_EINVAL;
  if (!(p->tol > 0.0) || p->max_iter < 0 || p->mode < 0 || p->mode > STAG_MIXED16L) return STAG_EINVAL;
  if (p->mode == STAG_LEARNED && !p->precond) return STAG_EINVAL;
  if (p->mode != STAG_PLAIN64 && !(p->delta > 0.0 && p->delta < 1.0)) return STAG_EINVAL;
  return STAG_OK;
}

// the link copy a mode's Krylov loop reads
static int mode_prec(int mode) {
  return mode == STAG_PLAIN64 ? STAG_FP64 : mode == STAG_MIXED16 ? STAG_FP16
       : (mode == STAG_MIXEDFX16 || mode == STAG_MIXED16L) ? STAG_FX16 : STAG_FP32;
}

extern "C" {

int stag_cg(stag_lattice_t lat, void* x, const void* b, double mass, const stag_solve_params* params,
            stag_solve_info* info, void* stream) {
  if (!lat || !x || !b) return STAG_EINVAL;
  stag_solve_params prm;
  stag_default_params(&prm);
  if (params) prm = *params;
  int s = check_params(&prm);
  if (s) return s;
  if (!lat->links[STAG_FP64].present || !lat->links[mode_prec(prm.mode)].present) return STAG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const double shift = mass * mass;
  if (info) info->precond_fallback = 0;
  if (prm.mode == STAG_LEARNED) return learned_solve(lat, (double2*)x, (const double2*)b, mass, prm, info, st);
  switch (prm.mode) {
    case STAG_PLAIN64: return cg_solve<64>(lat, (double2*)x, (const double2*)b, shift, prm, info, st);
    case STAG_MIXED32: return cg_solve<32>(lat, (double2*)x, (const double2*)b, shift, prm, info, st);
    case STAG_MIXED16: return cg_solve<16>(lat, (double2*)x, (const double2*)b, shift, prm, info, st);
    case STAG_MIXED16L: return cg_solve<31>(lat, (double2*)x, (const double2*)b, shift, prm, info, st);
    default: return cg_solve<15>(lat, (double2*)x, (const double2*)b, shift, prm, info, st);
  }
}

int stag_multishift_cg(stag_lattice_t lat, void* const* x, const void* b, double mass, const double* shifts,
                       int nshift, const stag_solve_params* params, stag_solve_info* infos, void* stream) {
  if (!lat || !x || !b || !shifts || nshift <= 0 || nshift > MAX_SHIFTS) return STAG_EINVAL;
  if (params && params->mode == STAG_LEARNED) return STAG_EINVAL;
  for (int k = 0; k < nshift; ++k)
    if (!x[k] || !(shifts[k] >= 0.0)) return STAG_EINVAL;
  stag_solve_params prm;
  stag_default_params(&prm);
  if (params) prm = *params;
  int s = check_params(&prm);
  if (s) return s;
  if (!lat->links[STAG_FP64].present || !lat->links[mode_prec(prm.mode)].present) return STAG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  double2* const* xs = (double2* const*)x;
  switch (prm.mode) {
    case STAG_PLAIN64: return ms_solve<64>(lat, xs, (const double2*)b, mass, shifts, nshift, prm, infos, st);
    case STAG_MIXED32: return ms_solve<32>(lat, xs, (const double2*)b, mass, shifts, nshift, prm, infos, st);
    case STAG_MIXED16: return ms_solve<16>(lat, xs, (const double2*)b, mass, shifts, nshift, prm, infos, st);
    case STAG_MIXED16L: return ms_solve<31>(lat, xs, (const double2*)b, mass, shifts, nshift, prm, infos, st);
    default: return ms_solve<15>(lat, xs, (const double2*)b, mass, shifts, nshift, prm, infos, st);
  }
}

}  // extern "C"
