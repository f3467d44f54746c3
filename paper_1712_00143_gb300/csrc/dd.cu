// dd.cu -- one lattice split across ranks along t: the halo-exchange form
// of the operator and of FP64 CG (the paper's multi-node weak-scaling study
// of the staggered CG, Sec. 4.1 and Figs. 2-3, where MILC moves the
// neighbouring sites' fields with gathers, Sec. 2; network-bound below about
// L = 30 per node).
//
// Rank r of R owns the time slices [r T, (r + 1) T), T = Lt / R (even, >= 4).
// It holds an extended slab of T + 2 H slices, H = STAG_DD_HALO = 4, local
// slice t' = global t - r T + H: its own slices in [H, H + T) and halo
// slices below and above.  The Naik hops reach three slices, so the
// operator reads the halo slices [1, 4) and [T + 4, T + 7); the outermost
// slice on each side is never read (H = 4 rather than 3 keeps the local
// parity of a site equal to its global parity).  Links are given for the
// whole extended slab (the caller's slab of the global field); vectors of
// the interface are the rank's own sites only.
//
// Since t is the slowest index of the checkerboard order, every slice is a
// contiguous range of S = Lx/2 Ly Lz sites of a single-parity field: the
// three slices a neighbour needs are one contiguous block of 3 S sites, and
// the exchange hands the communicator device pointers straight into the
// field (no packing).  The operator then runs the library's FP64 Dslash on
// the rank's own output sites only; the CG's inner products are summed
// over ranks by the communicator before the (device-resident) solver
// scalars are updated.
#include <chrono>
#include <cmath>

#include "internal.h"

struct stag_dd_s {
  stag_lattice_s* lat = nullptr;  // the extended slab (FP64 link copy)
  int gdims[4];
  int rank = 0, nranks = 1;
  int T = 0;         // own slices
  int S = 0;         // checkerboard sites per slice
  long long Vloc = 0;  // own sites per parity, T S
};

namespace stag {
namespace {

constexpr int H = STAG_DD_HALO;

double now_dd() { return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count(); }

#define TRYD(...)              \
  do {                         \
    int _s = (__VA_ARGS__);    \
    if (_s) return _s;         \
  } while (0)

// The own sites of an extended field.
Spinor<64> own(const stag_dd_s* d, void* ext) {
  return Spinor<64>{(char*)ext + (size_t)H * d->S * 48, (int)d->Vloc};
}

// Sends the three lowest and the three highest own slices to the ranks below
// and above and receives theirs into the halo slices [1, 4) and [T+4, T+7).
int exchange(const stag_dd_s* d, void* ext, const stag_comm* comm, cudaStream_t st) {
  char* f = (char*)ext;
  const size_t slice = (size_t)d->S * 48, bytes = 3 * slice;
  const int T = d->T;
  const int rc = comm->exchange(comm->ctx, f + (size_t)H * slice, f + (size_t)(H + T - 3) * slice, f + 1 * slice,
                                f + (size_t)(H + T) * slice, (unsigned long long)bytes, st);
  return rc == 0 ? STAG_OK : STAG_ECUDA;
}

int allreduce(const stag_comm* comm, double* v, int n, cudaStream_t st) {
  return comm->allreduce_sum(comm->ctx, v, n, st) == 0 ? STAG_OK : STAG_ECUDA;
}

// out (own sites, parity out_parity) = D in; in's halos are exchanged first.
// flags: the CG's stop word (the kernels return at once once it is set; the
// exchanges still run, so that every rank makes the same calls), or null.
int dd_dslash(stag_dd_s* d, void* out_ext, void* in_ext, int out_parity, const stag_comm* comm, cudaStream_t st,
              const int* flags = nullptr) {
  TRYD(exchange(d, in_ext, comm, st));
  const int Vh = d->lat->g.Vh;
  return launch_dslash_range<64>(d->lat, Spinor<64>{out_ext, Vh}, Spinor<64>{in_ext, Vh}, out_parity, H * d->S,
                                 (H + d->T) * d->S, flags, st);
}

// out = ax in + ay y + ad D_eo D_oe in on own even sites (ax = m^2, ad = -1:
// out = M in; ax = -m^2, y = b, ay = 1, ad = +1: out = b - M in); red = 1:
// <in, out>, 2: ||out||^2 into tgt (local sums)
int dd_apply(stag_dd_s* d, void* out_ext, void* in_ext, void* t_ext, double ax, void* y_ext, double ay, double ad,
             int red, RedScratch rs, RedTarget tgt, const stag_comm* comm, cudaStream_t st,
             const int* flags = nullptr) {
  TRYD(dd_dslash(d, t_ext, in_ext, 1, comm, st, flags));
  TRYD(exchange(d, t_ext, comm, st));
  const int Vh = d->lat->g.Vh;
  return launch_dslash_epi_range<64>(d->lat, Spinor<64>{out_ext, Vh}, Spinor<64>{t_ext, Vh}, 0,
                                     Spinor<64>{in_ext, Vh}, ax, Spinor<64>{y_ext, Vh}, ay, ad, red, rs, tgt,
                                     H * d->S, (H + d->T) * d->S, flags, st);
}

// x += alpha p; r -= alpha Ap; local ||r||^2 -> out (alpha from the state);
// nothing once the state's stop word is set
__global__ void k_dd_update(Spinor<64> x, Spinor<64> r, Spinor<64> p, Spinor<64> Ap, const CgState* st, RedBuf rb,
                            double* out) {
  if (stopped(&st->flags)) return;  // every block alike: no partial sum is left behind
  const double a = __ldcg(&st->alpha);
  double acc[1] = {0.0};
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < x.Vh; s += gridDim.x * blockDim.x) {
    double2 xv[3], rv[3], pv[3], av[3];
    SpinorLoad<64>::ldw(x, s, xv);
    SpinorLoad<64>::ldw(r, s, rv);
    SpinorLoad<64>::ld(p, s, pv);
    SpinorLoad<64>::ld(Ap, s, av);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      xv[c].x = fma(a, pv[c].x, xv[c].x);
      xv[c].y = fma(a, pv[c].y, xv[c].y);
      rv[c].x = fma(-a, av[c].x, rv[c].x);
      rv[c].y = fma(-a, av[c].y, rv[c].y);
      acc[0] = fma(rv[c].x, rv[c].x, fma(rv[c].y, rv[c].y, acc[0]));
    }
    SpinorLoad<64>::st(x, s, xv);
    SpinorLoad<64>::st(r, s, rv);
  }
  grid_reduce<1>(acc, rb, RedTarget{RED_STORE, nullptr, out});
}

// The solver-state update of a reduction, from the sums over ranks (none
// once the solve's stop word is set: the iterations queued after the
// iterated residual reached the target, or the cap, do nothing).
__global__ void k_dd_finalize(RedTarget tgt, const double* v, int nv) {
  if (stopped(&((const CgState*)tgt.state)->flags)) return;
  double w[4];
  for (int i = 0; i < nv && i < 4; ++i) w[i] = v[i];
  finalize(tgt, w, nv);
}

int finalize_on_device(RedTarget tgt, const double* v, int nv, cudaStream_t st) {
  count_launch();
  k_dd_finalize<<<1, 1, 0, st>>>(tgt, v, nv);
  return last_launch_status();
}

int grid_dd(long long n) {
  const long long g = (n + 255) / 256;
  return (int)(g < 1024 ? (g > 0 ? g : 1) : 1024);
}

}  // namespace
}  // namespace stag

using namespace stag;

extern "C" {

int stag_dd_create(stag_dd_t* out, const int gdims[4], int rank, int nranks, const void* fat_ext, const void* lng_ext,
                   const stag_link_opts* opts, void* stream) {
  if (!out || !gdims || !fat_ext || !lng_ext || nranks < 1 || rank < 0 || rank >= nranks) return STAG_EINVAL;
  *out = nullptr;
  for (int i = 0; i < 4; ++i)
    if (gdims[i] < 4 || gdims[i] % 2) return STAG_EINVAL;
  if (gdims[3] % nranks) return STAG_EINVAL;
  const int T = gdims[3] / nranks;
  if (T < 4 || T % 2) return STAG_EINVAL;
  const int ext[4] = {gdims[0], gdims[1], gdims[2], T + 2 * STAG_DD_HALO};
  stag_link_opts o;
  o.recon_long = 18;
  o.long_coeff = -1.0 / 24.0;
  o.autotune = 1;
  if (opts) o = *opts;
  o.prec_mask = 1u << STAG_FP64;
  stag_lattice_t lat = nullptr;
  const int s = stag_load_links(&lat, ext, fat_ext, lng_ext, &o, stream);
  if (s) return s;
  stag_dd_s* d = new stag_dd_s();
  d->lat = lat;
  for (int i = 0; i < 4; ++i) d->gdims[i] = gdims[i];
  d->rank = rank;
  d->nranks = nranks;
  d->T = T;
  d->S = gdims[0] / 2 * gdims[1] * gdims[2];
  d->Vloc = (long long)d->S * T;
  *out = d;
  return STAG_OK;
}

int stag_dd_free(stag_dd_t d) {
  if (!d) return STAG_EINVAL;
  stag_free_lattice(d->lat);
  delete d;
  return STAG_OK;
}

int stag_dd_info(stag_dd_t d, int local_dims[4], long long* vh_local, int* t_offset) {
  if (!d) return STAG_EINVAL;
  if (local_dims) {
    for (int i = 0; i < 3; ++i) local_dims[i] = d->gdims[i];
    local_dims[3] = d->T;
  }
  if (vh_local) *vh_local = d->Vloc;
  if (t_offset) *t_offset = d->rank * d->T;
  return STAG_OK;
}

static bool comm_ok(const stag_comm* c) { return c && c->exchange && c->allreduce_sum; }

int stag_dd_dslash(stag_dd_t d, void* out, const void* in, int out_parity, const stag_comm* comm, void* stream) {
  if (!d || !out || !in || (out_parity != 0 && out_parity != 1) || !comm_ok(comm)) return STAG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  stag_lattice_s* lat = d->lat;
  int s = 0;
  void* a = lat->ws.get("dd.in", (size_t)lat->g.Vh * 48, &s);
  void* b = lat->ws.get("dd.out", (size_t)lat->g.Vh * 48, &s);
  if (s) return s;
  const size_t bytes = (size_t)d->Vloc * 48;
  TRYD(cuda_status(cudaMemcpyAsync(own(d, a).v, in, bytes, cudaMemcpyDeviceToDevice, st)));
  TRYD(dd_dslash(d, b, a, out_parity, comm, st));
  return cuda_status(cudaMemcpyAsync(out, own(d, b).v, bytes, cudaMemcpyDeviceToDevice, st));
}

int stag_dd_apply_m(stag_dd_t d, void* out, const void* in, double mass, const stag_comm* comm, void* stream) {
  if (!d || !out || !in || !comm_ok(comm)) return STAG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  stag_lattice_s* lat = d->lat;
  int s = 0;
  void* a = lat->ws.get("dd.in", (size_t)lat->g.Vh * 48, &s);
  void* t = lat->ws.get("dd.t", (size_t)lat->g.Vh * 48, &s);
  void* b = lat->ws.get("dd.out", (size_t)lat->g.Vh * 48, &s);
  if (s) return s;
  const size_t bytes = (size_t)d->Vloc * 48;
  TRYD(cuda_status(cudaMemcpyAsync(own(d, a).v, in, bytes, cudaMemcpyDeviceToDevice, st)));
  RedScratch rs{nullptr, nullptr, 1 << 30};
  TRYD(dd_apply(d, b, a, t, mass * mass, nullptr, 0.0, -1.0, 0, rs, RedTarget{RED_STORE, nullptr, nullptr}, comm,
                st));
  return cuda_status(cudaMemcpyAsync(out, own(d, b).v, bytes, cudaMemcpyDeviceToDevice, st));
}

int stag_dd_cg(stag_dd_t d, void* x, const void* b, double mass, const stag_solve_params* params,
               stag_solve_info* info, const stag_comm* comm, void* stream) {
  if (!d || !x || !b || !comm_ok(comm)) return STAG_EINVAL;
  stag_solve_params prm;
  stag_default_params(&prm);
  if (params) prm = *params;
  if (!(prm.tol > 0.0) || prm.max_iter < 0 || prm.mode != STAG_PLAIN64) return STAG_EINVAL;
  const double t0 = now_dd();
  cudaStream_t st = (cudaStream_t)stream;
  stag_lattice_s* lat = d->lat;
  const size_t ext_bytes = (size_t)lat->g.Vh * 48, bytes = (size_t)d->Vloc * 48;
  int s = 0;
  void* xe = lat->ws.get("ddcg.x", ext_bytes, &s);
  void* be = lat->ws.get("ddcg.b", ext_bytes, &s);
  void* re = lat->ws.get("ddcg.r", ext_bytes, &s);
  void* pe = lat->ws.get("ddcg.p", ext_bytes, &s);
  void* te = lat->ws.get("ddcg.t", ext_bytes, &s);
  void* ae = lat->ws.get("ddcg.Ap", ext_bytes, &s);
  CgState* dst = (CgState*)lat->ws.get("ddcg.state", sizeof(CgState), &s);
  double* dsum = (double*)lat->ws.get("ddcg.sums", 64, &s);
  if (s) return s;
  RedScratch rs;
  TRYD(get_red_scratch(lat, "ddcg", &rs, 1));
  RedBuf rb{rs.partials, rs.counter};
  const double shift = mass * mass;
  Spinor<64> xo = own(d, xe), bo = own(d, be), ro = own(d, re), po = own(d, pe), ao = own(d, ae);
  // the fields' halo slices start at zero (the outermost slice is never written)
  TRYD(cuda_status(cudaMemsetAsync(xe, 0, ext_bytes, st)));
  TRYD(cuda_status(cudaMemsetAsync(pe, 0, ext_bytes, st)));
  TRYD(cuda_status(cudaMemsetAsync(te, 0, ext_bytes, st)));
  TRYD(cuda_status(cudaMemcpyAsync(bo.v, b, bytes, cudaMemcpyDeviceToDevice, st)));
  if (prm.use_initial_guess) TRYD(cuda_status(cudaMemcpyAsync(xo.v, x, bytes, cudaMemcpyDeviceToDevice, st)));
  // ||b||^2 over all ranks
  TRYD(launch_norm2<64>(bo, rs, RedTarget{RED_STORE, nullptr, dsum}, st));
  TRYD(allreduce(comm, dsum, 1, st));
  double bb = 0.0;
  TRYD(cuda_status(cudaMemcpyAsync(&bb, dsum, sizeof(double), cudaMemcpyDeviceToHost, st)));
  TRYD(cuda_status(cudaStreamSynchronize(st)));
  const double target = prm.tol * prm.tol * bb;
  CgState h{};
  int status = STAG_OK, iters = 0, restarts = 0;
  double rr_true = bb;
  if (bb > 0.0) {
    // (re)start: r = b - M x (true residual over all ranks), p = r
    auto restart = [&]() -> int {
      TRYD(dd_apply(d, re, xe, te, -shift, be, 1.0, 1.0, 2, rs, RedTarget{RED_STORE, nullptr, dsum}, comm, st));
      TRYD(allreduce(comm, dsum, 1, st));
      TRYD(cuda_status(cudaMemcpyAsync(&rr_true, dsum, sizeof(double), cudaMemcpyDeviceToHost, st)));
      TRYD(cuda_status(cudaMemcpyAsync(po.v, ro.v, bytes, cudaMemcpyDeviceToDevice, st)));
      return cuda_status(cudaStreamSynchronize(st));
    };
    TRYD(restart());
    h.rr = h.rr_prev = h.rr_max = h.rr_true = rr_true;
    h.target = target;
    h.shift = shift;
    h.max_iter = prm.max_iter;
    TRYD(cuda_status(cudaMemcpyAsync(dst, &h, sizeof(CgState), cudaMemcpyHostToDevice, st)));
    const int C = prm.check_interval > 0 ? prm.check_interval : 16;
    bool first = true;
    while (rr_true > target) {
      if (iters >= prm.max_iter) {
        status = STAG_ENOTCONV;
        break;
      }
      for (int i = 0; i < C && iters < prm.max_iter; ++i, ++iters) {
        if (!first) TRYD(launch_cg_xpay<64>(po, ro, dst, st));
        first = false;
        // Ap = shift p - D_eo D_oe p and <p, Ap> (local, then over ranks)
        TRYD(dd_apply(d, ae, pe, te, shift, nullptr, 0.0, -1.0, 1, rs, RedTarget{RED_STORE, nullptr, dsum}, comm,
                      st, &dst->flags));
        TRYD(allreduce(comm, dsum, 1, st));
        TRYD(finalize_on_device(RedTarget{RED_CG_ALPHA, dst, nullptr}, dsum, 1, st));
        {
          ProfScope ps("blas", st);
          k_dd_update<<<grid_dd(d->Vloc), 256, 0, st>>>(xo, ro, po, ao, dst, rb, dsum + 1);
        }
        TRYD(last_launch_status());
        TRYD(allreduce(comm, dsum + 1, 1, st));
        TRYD(finalize_on_device(RedTarget{RED_CG_BETA, dst, nullptr}, dsum + 1, 1, st));
      }
      TRYD(cuda_status(cudaMemcpyAsync(&h, dst, sizeof(CgState), cudaMemcpyDeviceToHost, st)));
      TRYD(cuda_status(cudaStreamSynchronize(st)));
      // the iterations that did work: after a stop flag the rest of the chunk
      // returned at once and left the device's count where it was
      iters = h.iter;
      if (h.flags & F_BREAKDOWN) {
        status = STAG_EBREAKDOWN;
        break;
      }
      if (h.flags & (F_CONVERGED | F_ITER_CAP)) {
        // the iterated residual reached the target: judge with the true
        // residual, and restart CG from there if it misses
        TRYD(restart());
        ++restarts;
        if (rr_true <= target) break;
        h.rr = h.rr_prev = h.rr_max = rr_true;
        h.flags = 0;
        h.iter = iters;
        TRYD(cuda_status(cudaMemcpyAsync(dst, &h, sizeof(CgState), cudaMemcpyHostToDevice, st)));
        first = true;
      }
    }
  }
  TRYD(cuda_status(cudaMemcpyAsync(x, xo.v, bytes, cudaMemcpyDeviceToDevice, st)));
  TRYD(cuda_status(cudaStreamSynchronize(st)));
  if (info) {
    info->iters = iters;
    info->reliable_updates = restarts;
    info->converged = bb > 0.0 ? rr_true <= target : 1;
    info->status = status;
    info->true_rel_resid = bb > 0.0 ? std::sqrt(rr_true / bb) : 0.0;
    info->seconds = now_dd() - t0;
    info->precond_fallback = 0;
  }
  return status;
}

}  // extern "C"
