// batch.cu -- many CG systems at once: the N-right-hand-side Dslash behind
// stag_dslash(nrhs > 1), and stag_batch_solve, which runs the systems of
// several lattices together.
//
// A lattice's right-hand sides are solved in groups of N = 8, 4 or 2 systems
// that share one N-RHS Dslash per application (links read once for N
// vectors); every system keeps its own CG scalars (McgState) and leaves the
// iteration when its residual reaches the target.  The groups of all
// lattices advance together: each group owns a stream, and the chunk of
// `check_interval` iterations of every group is captured once into one CUDA
// graph (fork from the caller's stream, one branch per group, join) that is
// replayed until the groups finish, so independent lattices of uneven sizes
// fill the GPU side by side and a chunk costs one graph launch.  Reliable
// updates (FP64 true residual of every system of a group) run between chunks
// for the groups that ask for them.
#include <chrono>
#include <cmath>
#include <memory>
#include <vector>

#include "batch_kernels.cuh"

namespace stag {

namespace {

#define TRYB(...)              \
  do {                         \
    int _s = (__VA_ARGS__);    \
    if (_s) return _s;         \
  } while (0)

int sm_count_b() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
    else {
      cudaGetLastError();
      n = 152;
    }
  }
  return n;
}
int grid_red(int Vh, int cap) {
  int g = (Vh + 255) / 256, m = 4 * sm_count_b();
  g = g < m ? g : m;
  return g < cap ? g : cap;
}
int grid_bw(int Vh) {
  int g = (Vh + 255) / 256, m = 8 * sm_count_b();
  return g < m ? g : m;
}

}  // namespace

template <int P> SpinorM<P> ws_spinorm(stag_lattice_s* lat, const std::string& name, int n, int* status) {
  SpinorM<P> f;
  f.Vh = lat->g.Vh;
  f.n = n;
  f.v = lat->ws.get(name, spinorm_bytes<P>(f.Vh, n), status);
  return f;
}

// ------------------------------------------------------------ stag_dslash, nrhs > 1
template <int P, int N>
static int dslash_group(stag_lattice_s* lat, double2* out, const double2* in, int out_parity, cudaStream_t st) {
  int s = tune_mrhs<P, N>(lat, st);
  if (s) return s;
  SpinorM<P> a = ws_spinorm<P>(lat, "mdslash.in", N, &s);
  SpinorM<P> b = ws_spinorm<P>(lat, "mdslash.out", N, &s);
  if (s) return s;
  {
    ProfScope ps("convert", st);
    k_mfrom_canonical<P, N><<<grid_bw(lat->g.Vh), 256, 0, st>>>(a, in, N);
  }
  TRYB(last_launch_status());
  TRYB((mdslash<P, N>(lat, b, a, out_parity, nullptr, st)));
  {
    ProfScope ps("convert", st);
    k_mto_canonical<P, N><<<grid_bw(lat->g.Vh), 256, 0, st>>>(out, b, N);
  }
  return last_launch_status();
}

template <int P>
static int dslash_multi_p(stag_lattice_s* lat, double2* out, const double2* in, int out_parity, int nrhs,
                          cudaStream_t st) {
  const size_t n = (size_t)lat->g.Vh * 3;
  int r = 0;
  while (r < nrhs) {
    const int left = nrhs - r;
    int s;
    if (left >= 8) s = dslash_group<P, 8>(lat, out + r * n, in + r * n, out_parity, st), r += 8;
    else if (left >= 4) s = dslash_group<P, 4>(lat, out + r * n, in + r * n, out_parity, st), r += 4;
    else if (left >= 2) s = dslash_group<P, 2>(lat, out + r * n, in + r * n, out_parity, st), r += 2;
    else break;
    if (s) return s;
  }
  if (r < nrhs) return stag_dslash(lat, out + r * n, in + r * n, out_parity, P == 31 ? STAG_FX16L32 : prec_index<P>(), 1, st);
  return STAG_OK;
}

int dslash_multi(stag_lattice_s* lat, double2* out, const double2* in, int out_parity, int prec, int nrhs,
                 cudaStream_t st) {
  switch (prec) {
    case STAG_FP64: return dslash_multi_p<64>(lat, out, in, out_parity, nrhs, st);
    case STAG_FP32: return dslash_multi_p<32>(lat, out, in, out_parity, nrhs, st);
    case STAG_FP16: return dslash_multi_p<16>(lat, out, in, out_parity, nrhs, st);
    case STAG_FX16L32: return dslash_multi_p<31>(lat, out, in, out_parity, nrhs, st);
    default: return dslash_multi_p<15>(lat, out, in, out_parity, nrhs, st);
  }
}

// ------------------------------------------------------------ batched CG
struct GroupBase {
  stag_lattice_s* lat = nullptr;
  double shift = 0.0;  // m^2
  double2* x = nullptr;        // canonical, first system of the group
  const double2* b = nullptr;
  int nreal = 0;               // systems of the item in this group (<= N)
  int item = 0, first = 0;     // item index and first right-hand side
  cudaStream_t st = nullptr;
  McgState* dst = nullptr;
  McgState* hst = nullptr;     // pinned host copy
  double* dscal = nullptr;     // device: bb[N], rr0[N]
  double* hscal = nullptr;     // pinned
  bool pending_p = false, done = false;
  int status = STAG_OK;
  double bb[MAX_RHS] = {0};
  virtual ~GroupBase() {}
  virtual int n() const = 0;
  virtual int setup(const stag_solve_params& prm) = 0;
  virtual int start(const stag_solve_params& prm) = 0;
  virtual int iterations(int C) = 0;
  virtual int reliable_update() = 0;
  // the same update with the FP64 operator: the final verdict on a group
  // whose double-float residual reached the target
  virtual int reliable_update_fp64() = 0;
  virtual bool uses_df() const = 0;
  virtual int round_dev(int C) = 0;
  virtual int finish() = 0;
};

template <int P, int N> struct Group : GroupBase {
  static constexpr int PV = Acc<P>::value;
  SpinorM<64> b64, y64, r64, t64;
  SpinorM<P> p, t;
  SpinorM<PV> Ap, xh, rh;
  // reliable updates in double-float (when the handle holds that link copy):
  // the anchor (ya64, its residual radf; see McgState), y - ya, the odd
  // intermediate and the residual
  bool use_df = false;
  float* pt = nullptr;  // per-site values of <p, Ap> (FP32-arithmetic formats)
  SpinorM<64> ya64;
  DfField radf, ydf, tdf, rdf;
  RedScratch rs;
  int n() const override { return N; }
  bool uses_df() const override { return use_df; }

  int alloc(int gid) {
    // the launch variant of this group's operator kernels (timed once per
    // format, N and lattice shape)
    int s = tune_mrhs<P, N>(lat, st);
    if (s) return s;
    const std::string pre = "batch" + std::to_string(gid) + ".";
    b64 = ws_spinorm<64>(lat, pre + "b", N, &s);
    y64 = ws_spinorm<64>(lat, pre + "y", N, &s);
    p = ws_spinorm<P>(lat, pre + "p", N, &s);
    t = ws_spinorm<P>(lat, pre + "t", N, &s);
    Ap = ws_spinorm<PV>(lat, pre + "Ap", N, &s);
    xh = ws_spinorm<PV>(lat, pre + "xh", N, &s);
    rh = ws_spinorm<PV>(lat, pre + "rh", N, &s);
    use_df = P != 64 && lat->links[STAG_DF64].present;
    const int Vh = lat->g.Vh;
    if (use_df) {
      ya64 = ws_spinorm<64>(lat, pre + "ya", N, &s);
      radf = DfField{(float4*)lat->ws.get(pre + "radf", df_bytes(Vh) * N, &s), Vh};
      ydf = DfField{(float4*)lat->ws.get(pre + "ydf", df_bytes(Vh) * N, &s), Vh};
      tdf = DfField{(float4*)lat->ws.get(pre + "tdf", df_bytes(Vh) * N, &s), Vh};
      rdf = DfField{(float4*)lat->ws.get(pre + "rdf", df_bytes(Vh) * N, &s), Vh};
    }
    t64 = ws_spinorm<64>(lat, pre + "t64", N, &s);
    r64 = ws_spinorm<64>(lat, pre + "r64", N, &s);
    pt = (float*)lat->ws.get(pre + "pt", sizeof(float) * N * (size_t)Vh, &s);
    dst = (McgState*)lat->ws.get(pre + "state", sizeof(McgState), &s);
    dscal = (double*)lat->ws.get(pre + "scal", sizeof(double) * 2 * MAX_RHS, &s);
    if (s) return s;
    return get_red_scratch(lat, (pre + "red").c_str(), &rs, 3 * N);
  }

  // FP64: r = b - shift y + D_eo D_oe y, ||r_i||^2 -> tgt (stop: a stop word, or nullptr)
  int true_residual(RedTarget tgt, const int* stop = nullptr) {
    TRYB((mdslash<64, N>(lat, t64, y64, 1, stop, st)));
    return mdslash_epi<64, N, 2>(lat, r64, t64, 0, y64, -shift, b64, 1.0, 1.0, rs, tgt, stop, st);
  }

  // Double-float: rdf = r_a - M (y - y_a) = radf - shift ydf + D_eo D_oe ydf
  // (ydf = y - y_a), no reduction
  int true_residual_df(const int* stop) {
    TRYB(launch_dslash_df(lat, tdf, ydf, N, 1, stop, st));
    return launch_dslash_df_epi(lat, rdf, tdf, N, 0, ydf, -shift, radf, 1.0, 1.0, stop, st);
  }

  int setup(const stag_solve_params& prm) override {
    {
      ProfScope ps("convert", st);
      k_mfrom_canonical<64, N><<<grid_bw(lat->g.Vh), 256, 0, st>>>(b64, b, nreal);
    }
    TRYB(last_launch_status());
    {
      ProfScope ps("reduce", st);
      k_mnorm2<64, N><<<grid_red(lat->g.Vh, rs.max_grid), 256, 0, st>>>(b64, RedBuf{rs.partials, rs.counter},
                                                                         RedTarget{RED_STORE, nullptr, dscal});
    }
    TRYB(last_launch_status());
    if (use_df) {
      // the anchor starts at (0, b)
      TRYB(launch_df_from_double(radf, (const double2*)b64.v, N, st));
      TRYB(cuda_status(cudaMemsetAsync(ya64.v, 0, spinorm_bytes<64>(lat->g.Vh, N), st)));
    }
    if (prm.use_initial_guess) {
      {
        ProfScope ps("convert", st);
        k_mfrom_canonical<64, N><<<grid_bw(lat->g.Vh), 256, 0, st>>>(y64, x, nreal);
      }
      TRYB(last_launch_status());
      if (use_df) {
        TRYB(launch_df_from_double(ydf, (const double2*)y64.v, N, st));
        TRYB(true_residual_df(nullptr));
        TRYB(launch_norm2_df(rdf, N, rs, RedTarget{RED_STORE, nullptr, dscal + MAX_RHS}, st));
      } else {
        TRYB(true_residual(RedTarget{RED_STORE, nullptr, dscal + MAX_RHS}));
      }
    } else {
      TRYB(cuda_status(cudaMemsetAsync(y64.v, 0, spinorm_bytes<64>(lat->g.Vh, N), st)));
      TRYB(cuda_status(cudaMemcpyAsync(r64.v, b64.v, spinorm_bytes<64>(lat->g.Vh, N), cudaMemcpyDeviceToDevice, st)));
      TRYB(cuda_status(cudaMemcpyAsync(dscal + MAX_RHS, dscal, sizeof(double) * N, cudaMemcpyDeviceToDevice, st)));
    }
    return cuda_status(cudaMemcpyAsync(hscal, dscal, sizeof(double) * 2 * MAX_RHS, cudaMemcpyDeviceToHost, st));
  }

  // host state from the norms; sloppy copies rh = r, xh = 0, p = rh
  int start(const stag_solve_params& prm) override {
    McgState h{};
    h.n = N;
    h.max_iter = prm.max_iter;
    int active = 0;
    for (int i = 0; i < N; ++i) {
      CgState& c = h.sys[i];
      bb[i] = hscal[i];
      const double rr0 = hscal[MAX_RHS + i];
      c.rr = c.rr_prev = c.rr_max = c.rr_true = rr0;
      c.target = prm.tol * prm.tol * bb[i];
      c.delta2 = (P == 64) ? 0.0 : prm.delta * prm.delta;
      c.shift = shift;
      c.max_iter = prm.max_iter;
      if (i < nreal && bb[i] > 0.0 && rr0 > c.target) active |= 1 << i;
    }
    h.active = active;
    if (active == 0 || prm.max_iter <= 0) h.flags = F_CONVERGED;
    h.done = active == 0 ? 1 : 0;
    h.status = STAG_OK;
    h.ru_skip = F_CONVERGED;
    h.skip_xpay = 1;
    h.use_df = use_df ? 1 : 0;
    h.anchored = 0;
    h.ru_skip64 = F_CONVERGED;
    for (int i = 0; i < N; ++i) h.anchor_rr[i] = kDfAnchorRel2 * bb[i];
    *hst = h;
    TRYB(cuda_status(cudaMemcpyAsync(dst, hst, sizeof(McgState), cudaMemcpyHostToDevice, st)));
    const int G = grid_bw(lat->g.Vh);
    if (use_df && prm.use_initial_guess) {
      TRYB(launch_convert_from_df<PV>(rh.v, rdf, N, st));
    } else {
      {
        ProfScope ps("convert", st);
        k_mconvert<PV, 64, N><<<G, 256, 0, st>>>(rh, r64);
      }
      TRYB(last_launch_status());
    }
    TRYB(cuda_status(cudaMemsetAsync(xh.v, 0, spinorm_bytes<PV>(lat->g.Vh, N), st)));
    {
      ProfScope ps("convert", st);
      k_mconvert<P, PV, N><<<G, 256, 0, st>>>(p, rh);
    }
    TRYB(last_launch_status());
    pending_p = false;
    done = (active == 0);
    return STAG_OK;
  }

  int iterations(int C) override {
    const int* flags = &dst->flags;
    const int Vh = lat->g.Vh;
    SpinorM<PV> none{nullptr, Vh, N};
    for (int i = 0; i < C; ++i) {
      if (pending_p) {
        ProfScope ps("blas", st);
        k_mcg_xpay<P, N><<<grid_bw(Vh), 256, 0, st>>>(p, rh, dst, nullptr);
        TRYB(last_launch_status());
      }
      TRYB((mdslash<P, N>(lat, t, p, 1, flags, st)));
      TRYB(operator_epilogue(none, flags));
      {
        ProfScope ps("blas", st);
        k_mcg_update<P, N><<<grid_red(Vh, rs.max_grid), 256, 0, st>>>(xh, rh, p, Ap, dst,
                                                                        RedBuf{rs.partials, rs.counter});
      }
      TRYB(last_launch_status());
      pending_p = true;
    }
    return STAG_OK;
  }

  // Ap = shift p - D_eo t and <p_r, Ap_r> -> alpha_r.  FP32-arithmetic
  // formats: the operator kernel also stores each site's <p_r, Ap_r> (4
  // bytes per site and system) and a small grid sum reads those instead of
  // p and Ap; FP64: the operator without a reduction, then <p, Ap> in a
  // level-1 pass.  (A block-tree reduction fused into the operator grid,
  // 4096 blocks at 32^4, held every block until its slowest warp was done:
  // measured slower than either.)
  int operator_epilogue(SpinorM<PV> none, const int* flags) {
    const int Vh = lat->g.Vh;
    if constexpr (P != 64) {
      TRYB((mdslash_epi<P, N, 3>(lat, Ap, t, 0, p, shift, none, 0.0, -1.0, RedScratch{(double*)pt, nullptr, 0},
                                 RedTarget{RED_STORE, nullptr, nullptr}, flags, st)));
      return launch_mcg_alpha_pt<P, N>(lat, pt, dst, rs, st);
    } else {
      TRYB((mdslash_epi<P, N, 0>(lat, Ap, t, 0, p, shift, none, 0.0, -1.0, rs, RedTarget{RED_STORE, nullptr, nullptr},
                                 flags, st)));
      ProfScope ps("reduce", st);
      k_mcg_pap<P, N><<<grid_red(Vh, rs.max_grid), 256, 0, st>>>(p, Ap, dst, RedBuf{rs.partials, rs.counter});
      return last_launch_status();
    }
  }

  // Host-driven update: double-float, or the FP64 update that moves the
  // anchor when every active system's residual has fallen below its level.
  int reliable_update() override {
    bool anchor = use_df && !hst->anchored;
    for (int i = 0; i < N && anchor; ++i)
      if (((hst->active >> i) & 1) && !(hst->sys[i].rr < hst->anchor_rr[i])) anchor = false;
    if (use_df && !anchor) return ru_kernels(nullptr, true);
    return reliable_update_fp64();
  }
  int reliable_update_fp64() override {
    TRYB(ru_kernels(nullptr, false));
    if (!use_df) return STAG_OK;
    TRYB(launch_df_anchor(ya64.v, radf, y64.v, r64.v, N, nullptr, st));
    hst->anchored = 1;
    return cuda_status(cudaMemcpyAsync(&dst->anchored, &hst->anchored, sizeof(int), cudaMemcpyHostToDevice, st));
  }

  // the update's kernels (df: double-float operator, else FP64); with
  // stop = &dst->ru_skip they run only when a reliable update is due
  // (graph-resident loop)
  int ru_kernels(const int* stop, bool df) {
    const int Vh = lat->g.Vh;
    if constexpr (P != 64) {
      if (df) {
        // y += xh in FP64 (and its DF copy), r = b - M y in double-float,
        // rh = r with ||rh||^2 and <rh, p> in one pass
        TRYB(launch_accumulate_df<PV>(y64.v, xh.v, ydf, ya64.v, N, stop, st));
        TRYB(true_residual_df(stop));
        TRYB(launch_ru_convert_dot_df<P>(rh.v, rdf, p.v, N, rs, RedTarget{RED_MCG_RU_BOTH, dst, nullptr}, stop, st));
      }
    }
    if (!df) {
      {
        ProfScope ps("blas", st);
        k_maccumulate<PV, N><<<grid_bw(Vh), 256, 0, st>>>(y64, xh, stop);
      }
      TRYB(last_launch_status());
      TRYB(true_residual(RedTarget{RED_MCG_RU_RESID, dst, nullptr}, stop));
      {
        ProfScope ps("reduce", st);
        k_mru_convert_dot<P, N><<<grid_red(Vh, rs.max_grid), 256, 0, st>>>(rh, r64, p, dst,
                                                                            RedBuf{rs.partials, rs.counter}, stop);
      }
      TRYB(last_launch_status());
    }
    {
      ProfScope ps("blas", st);
      k_mru_p<P, N><<<grid_bw(Vh), 256, 0, st>>>(p, rh, dst, stop);
    }
    TRYB(last_launch_status());
    pending_p = false;
    return STAG_OK;
  }

  // One round of the graph-resident loop for this group: a reliable update
  // if one is due (gate, the update's kernels, decide), then C iterations
  // whose first direction update is skipped after a start or an update.
  int round_dev(int C) override {
    const int* flags = &dst->flags;
    const int Vh = lat->g.Vh;
    SpinorM<PV> none{nullptr, Vh, N};
    count_launch();
    k_mcg_ru_gate<<<1, 1, 0, st>>>(dst);
    TRYB(last_launch_status());
    if (use_df) {
      TRYB(ru_kernels(&dst->ru_skip, true));
      TRYB(ru_kernels(&dst->ru_skip64, false));
      TRYB(launch_df_anchor(ya64.v, radf, y64.v, r64.v, N, &dst->ru_skip64, st));
    } else {
      TRYB(ru_kernels(&dst->ru_skip64, false));
    }
    count_launch();
    k_mcg_ru_decide<<<1, 1, 0, st>>>(dst);
    TRYB(last_launch_status());
    for (int i = 0; i < C; ++i) {
      {
        ProfScope ps("blas", st);
        k_mcg_xpay<P, N><<<grid_bw(Vh), 256, 0, st>>>(p, rh, dst, &dst->skip_xpay);
      }
      TRYB(last_launch_status());
      count_launch();
      k_mcg_clear_skip<<<1, 1, 0, st>>>(dst);
      TRYB(last_launch_status());
      TRYB((mdslash<P, N>(lat, t, p, 1, flags, st)));
      TRYB(operator_epilogue(none, flags));
      {
        ProfScope ps("blas", st);
        k_mcg_update<P, N><<<grid_red(Vh, rs.max_grid), 256, 0, st>>>(xh, rh, p, Ap, dst,
                                                                        RedBuf{rs.partials, rs.counter});
      }
      TRYB(last_launch_status());
    }
    return STAG_OK;
  }

  int finish() override {
    {
      ProfScope ps("convert", st);
      k_mto_canonical<64, N><<<grid_bw(lat->g.Vh), 256, 0, st>>>(x, y64, nreal);
    }
    return last_launch_status();
  }
};

template <int P> static std::unique_ptr<GroupBase> make_group(int N) {
  if (N == 8) return std::unique_ptr<GroupBase>(new Group<P, 8>());
  if (N == 4) return std::unique_ptr<GroupBase>(new Group<P, 4>());
  return std::unique_ptr<GroupBase>(new Group<P, 2>());
}

template <int P>
static int alloc_group(GroupBase* g, int gid) {
  const int N = g->n();
  if (N == 8) return static_cast<Group<P, 8>*>(g)->alloc(gid);
  if (N == 4) return static_cast<Group<P, 4>*>(g)->alloc(gid);
  return static_cast<Group<P, 2>*>(g)->alloc(gid);
}

namespace {
struct Streams {
  std::vector<cudaStream_t> s;
  std::vector<cudaEvent_t> ev;
  ~Streams() {
    for (auto x : s) cudaStreamDestroy(x);
    for (auto e : ev) cudaEventDestroy(e);
  }
};
struct Pinned {
  void* p = nullptr;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};
struct GraphExec {
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  ~GraphExec() { reset(); }
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
};
double now_b() { return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count(); }
}  // namespace

// The graph-resident loop over all groups (see batch_solve_p).
static int dev_loop(std::vector<std::unique_ptr<GroupBase>>& groups, cudaStream_t cap, Streams& streams, int C,
                    int budget) {
  const int ng = (int)groups.size();
  McgState** gs_dev = nullptr;
  int* budget_dev = nullptr;
  if (cudaMalloc(&gs_dev, sizeof(McgState*) * ng) != cudaSuccess || cudaMalloc(&budget_dev, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    if (gs_dev) cudaFree(gs_dev);
    return STAG_ENOMEM;
  }
  struct Free {
    void* a;
    void* b;
    ~Free() {
      cudaFree(a);
      cudaFree(b);
    }
  } freer{gs_dev, budget_dev};
  std::vector<McgState*> gs(ng);
  for (int k = 0; k < ng; ++k) gs[k] = groups[k]->dst;
  TRYB(cuda_status(cudaMemcpyAsync(gs_dev, gs.data(), sizeof(McgState*) * ng, cudaMemcpyHostToDevice, cap)));
  TRYB(cuda_status(cudaMemcpyAsync(budget_dev, &budget, sizeof(int), cudaMemcpyHostToDevice, cap)));
  TRYB(cuda_status(cudaStreamSynchronize(cap)));

  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  struct GFree {
    cudaGraph_t* g;
    cudaGraphExec_t* e;
    ~GFree() {
      if (*e) cudaGraphExecDestroy(*e);
      if (*g) cudaGraphDestroy(*g);
    }
  } gfree{&graph, &exec};
  TRYB(cuda_status(cudaGraphCreate(&graph, 0)));
  cudaGraphConditionalHandle handle;
  TRYB(cuda_status(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault)));
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = handle;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  TRYB(cuda_status(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np)));
  cudaGraph_t body = np.conditional.phGraph_out[0];

  set_capturing(true);
  int s = cuda_status(cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  if (!s) s = cuda_status(cudaEventRecord(streams.ev[1], cap));
  for (int k = 0; k < ng && !s; ++k) s = cuda_status(cudaStreamWaitEvent(groups[k]->st, streams.ev[1], 0));
  for (int k = 0; k < ng && !s; ++k) s = groups[k]->round_dev(C);
  for (int k = 0; k < ng && !s; ++k) {
    s = cuda_status(cudaEventRecord(streams.ev[2 + k], groups[k]->st));
    if (!s) s = cuda_status(cudaStreamWaitEvent(cap, streams.ev[2 + k], 0));
  }
  if (!s) {
    count_launch();
    k_mcg_loop_cond<<<1, 1, 0, cap>>>(gs_dev, ng, budget_dev, handle);
    s = last_launch_status();
  }
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cap, &out);
  const long long per_round = set_capturing(false);
  if (s || e != cudaSuccess) {
    cudaGetLastError();
    return s ? s : STAG_ECUDA;
  }
  TRYB(cuda_status(cudaGraphInstantiate(&exec, graph, 0)));
  TRYB(cuda_status(cudaGraphLaunch(exec, cap)));
  TRYB(cuda_status(cudaStreamSynchronize(cap)));
  int left = 0;
  TRYB(cuda_status(cudaMemcpy(&left, budget_dev, sizeof(int), cudaMemcpyDeviceToHost)));
  for (long long i = 0; i < per_round * (long long)(budget - left); ++i) count_launch();
  return STAG_OK;
}

template <int P>
static int batch_solve_p(const stag_batch_item* items, int nitems, const stag_solve_params& prm,
                         stag_solve_info* infos, cudaStream_t origin) {
  const double t0 = now_b();
  // groups of 8, 4, 2 right-hand sides per item (a last single one pads to 2)
  std::vector<std::unique_ptr<GroupBase>> groups;
  for (int it = 0; it < nitems; ++it) {
    const stag_batch_item& I = items[it];
    const size_t n = (size_t)I.lat->g.Vh * 3;
    int r = 0;
    // 16-bit storage: groups of at most 4 (measured: the 8-vector kernel
    // is slower per vector than the 4-vector one); FP32/FP64: up to 8
    const int nmax = (P == 16 || P == 15) ? 4 : 8;
    while (r < I.nrhs) {
      const int left = I.nrhs - r;
      const int N = left >= 8 && nmax >= 8 ? 8 : left >= 4 ? 4 : 2;
      std::unique_ptr<GroupBase> g = make_group<P>(N);
      g->lat = I.lat;
      g->shift = I.mass * I.mass;
      g->x = (double2*)I.x + r * n;
      g->b = (const double2*)I.b + r * n;
      g->nreal = left < N ? left : N;
      g->item = it;
      g->first = r;
      r += g->nreal;
      groups.push_back(std::move(g));
    }
  }
  const int ng = (int)groups.size();
  Streams streams;
  for (int k = 0; k < ng; ++k) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return STAG_ECUDA;
    }
    streams.s.push_back(s);
    groups[k]->st = s;
  }
  for (int k = 0; k < 2 * ng + 2; ++k) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return STAG_ECUDA;
    }
    streams.ev.push_back(e);
  }
  Pinned pin;
  const size_t per = sizeof(McgState) + sizeof(double) * 2 * MAX_RHS;
  if (cudaMallocHost(&pin.p, per * ng) != cudaSuccess) {
    cudaGetLastError();
    return STAG_ENOMEM;
  }
  for (int k = 0; k < ng; ++k) {
    groups[k]->hst = (McgState*)((char*)pin.p + per * k);
    groups[k]->hscal = (double*)((char*)pin.p + per * k + sizeof(McgState));
    TRYB(alloc_group<P>(groups[k].get(), k));
  }
  // fork: the group streams start after the work already queued on `origin`
  TRYB(cuda_status(cudaEventRecord(streams.ev[0], origin)));
  for (int k = 0; k < ng; ++k) TRYB(cuda_status(cudaStreamWaitEvent(groups[k]->st, streams.ev[0], 0)));
  for (auto& g : groups) TRYB(g->setup(prm));
  for (auto& g : groups) TRYB(cuda_status(cudaStreamSynchronize(g->st)));
  for (auto& g : groups) TRYB(g->start(prm));

  const int C = prm.check_interval > 0 ? prm.check_interval : 16;
  GraphExec graph;
  std::vector<int> graph_set;  // groups captured in the current graph
  long long graph_kernels = 0;  // kernels per replay
  cudaStream_t cap = nullptr;   // capture / launch stream of the graph
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return STAG_ECUDA;
  }
  streams.s.push_back(cap);
  long long chunks = 0, max_chunks = (long long)prm.max_iter / C + 64 * ng + 64;
  if (ng > 1) {
    // Several groups: the whole solve is one graph launch.  A WHILE node's
    // body runs one round for every group side by side (its reliable update
    // if due, then C iterations) and a last kernel sets the loop condition:
    // another round while any group is live, at most max_chunks rounds.
    TRYB(dev_loop(groups, cap, streams, C, (int)std::min<long long>(max_chunks, 1 << 30)));
    for (auto& g : groups) {
      TRYB(cuda_status(cudaMemcpyAsync(g->hst, g->dst, sizeof(McgState), cudaMemcpyDeviceToHost, cap)));
    }
    TRYB(cuda_status(cudaStreamSynchronize(cap)));
    for (auto& g : groups) {
      g->done = true;
      if (g->hst->done == 0) g->status = STAG_ENOTCONV;  // the round budget ran out
      else g->status = g->hst->status;
    }
    // the FP64 verdict on the groups retired by their double-float residual;
    // a group it finds short of the target iterates on in the host loop
    std::vector<GroupBase*> verdict;
    for (auto& g : groups)
      if (g->uses_df() && g->status == STAG_OK && g->hst->active == 0) verdict.push_back(g.get());
    for (GroupBase* g : verdict) TRYB(g->reliable_update_fp64());
    for (GroupBase* g : verdict)
      TRYB(cuda_status(cudaMemcpyAsync(g->hst, g->dst, sizeof(McgState), cudaMemcpyDeviceToHost, g->st)));
    for (GroupBase* g : verdict) {
      TRYB(cuda_status(cudaStreamSynchronize(g->st)));
      if (g->hst->flags & F_BREAKDOWN) {
        g->status = STAG_EBREAKDOWN;
      } else if (g->hst->active != 0) {
        g->done = false;
        g->pending_p = false;
      }
    }
  }
  for (;;) {
    std::vector<int> live;
    for (int k = 0; k < ng; ++k)
      if (!groups[k]->done) live.push_back(k);
    if (live.empty()) break;
    if (++chunks > max_chunks) {
      for (int k : live) groups[k]->status = STAG_ENOTCONV, groups[k]->done = true;
      break;
    }
    bool steady = true;  // every live group begins with its direction update
    for (int k : live) steady = steady && groups[k]->pending_p;
    // one group on one stream: its kernels are long enough that the host
    // stays ahead of the GPU, so the chunk is queued directly (and the
    // library's per-launch profiler can time it); graphs pay off when
    // several groups run side by side
    const long long mark = prof_mark();
    if (!steady || ng == 1) {
      // first chunk after a start or a reliable update: queue directly
      for (int k : live) TRYB(groups[k]->iterations(C));
      for (int k : live) TRYB(cuda_status(cudaStreamSynchronize(groups[k]->st)));
    } else {
      if (graph_set != live || graph.exec == nullptr) {
        // capture one chunk of every live group: cap forks to the group
        // streams and joins back; recorded, not run
        graph.reset();
        graph_set.clear();
        set_capturing(true);
        int s = cuda_status(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        if (!s) s = cuda_status(cudaEventRecord(streams.ev[1], cap));
        for (size_t j = 0; j < live.size() && !s; ++j) s = cuda_status(cudaStreamWaitEvent(groups[live[j]]->st, streams.ev[1], 0));
        for (size_t j = 0; j < live.size() && !s; ++j) s = groups[live[j]]->iterations(C);
        for (size_t j = 0; j < live.size() && !s; ++j) {
          s = cuda_status(cudaEventRecord(streams.ev[2 + j], groups[live[j]]->st));
          if (!s) s = cuda_status(cudaStreamWaitEvent(cap, streams.ev[2 + j], 0));
        }
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamEndCapture(cap, &gr);
        graph_kernels = set_capturing(false);
        if (s || e != cudaSuccess || gr == nullptr) {
          cudaGetLastError();
          if (gr) cudaGraphDestroy(gr);
          return s ? s : STAG_ECUDA;
        }
        graph.graph = gr;
        if (cudaGraphInstantiate(&graph.exec, gr, 0) != cudaSuccess) {
          cudaGetLastError();
          graph.reset();
          return STAG_ECUDA;
        }
        graph_set = live;
      }
      TRYB(cuda_status(cudaGraphLaunch(graph.exec, cap)));
      for (long long i = 0; i < graph_kernels; ++i) count_launch();
      TRYB(cuda_status(cudaStreamSynchronize(cap)));
    }
    // read every live group's state
    for (int k : live) {
      GroupBase& g = *groups[k];
      TRYB(cuda_status(cudaMemcpyAsync(g.hst, g.dst, sizeof(McgState), cudaMemcpyDeviceToHost, g.st)));
    }
    for (int k : live) TRYB(cuda_status(cudaStreamSynchronize(groups[k]->st)));
    // a chunk in which a stop flag was raised holds launches that returned at
    // once: its profiling records would not time the kernels' work
    bool cut = false;
    for (int k : live) cut = cut || (groups[k]->hst->flags & F_STOP);
    if (cut) prof_discard_since(mark);
    prof_flush_completed();
    std::vector<int> ru;
    for (int k : live) {
      GroupBase& g = *groups[k];
      if (g.hst->flags & F_BREAKDOWN) {
        g.status = STAG_EBREAKDOWN;
        g.done = true;
      } else if (g.hst->flags & (F_CONVERGED | F_NEED_RU | F_ITER_CAP)) {
        ru.push_back(k);
      }
    }
    for (int k : ru) TRYB(groups[k]->reliable_update());
    for (int k : ru) {
      GroupBase& g = *groups[k];
      TRYB(cuda_status(cudaMemcpyAsync(g.hst, g.dst, sizeof(McgState), cudaMemcpyDeviceToHost, g.st)));
    }
    // a double-float residual at the target is judged once more in FP64
    std::vector<int> verdict;
    for (int k : ru) {
      GroupBase& g = *groups[k];
      TRYB(cuda_status(cudaStreamSynchronize(g.st)));
      if (g.uses_df() && !(g.hst->flags & F_BREAKDOWN) && g.hst->active == 0) verdict.push_back(k);
    }
    for (int k : verdict) TRYB(groups[k]->reliable_update_fp64());
    for (int k : verdict) {
      GroupBase& g = *groups[k];
      TRYB(cuda_status(cudaMemcpyAsync(g.hst, g.dst, sizeof(McgState), cudaMemcpyDeviceToHost, g.st)));
    }
    for (int k : ru) {
      GroupBase& g = *groups[k];
      TRYB(cuda_status(cudaStreamSynchronize(g.st)));
      if (g.hst->flags & F_BREAKDOWN) {
        g.status = STAG_EBREAKDOWN;
        g.done = true;
      } else if (g.hst->active == 0) {
        g.done = true;
      } else if (g.hst->iter >= prm.max_iter) {
        g.status = STAG_ENOTCONV;
        g.done = true;
      }
    }
  }
  for (auto& g : groups) TRYB(g->finish());
  // join: `origin` continues after every group's last kernel
  for (int k = 0; k < ng; ++k) {
    TRYB(cuda_status(cudaEventRecord(streams.ev[2 + k], groups[k]->st)));
    TRYB(cuda_status(cudaStreamWaitEvent(origin, streams.ev[2 + k], 0)));
  }
  TRYB(cuda_status(cudaStreamSynchronize(origin)));
  const double t1 = now_b();
  int worst = STAG_OK;
  for (auto& g : groups) {
    if (g->status && !worst) worst = g->status;
    if (!infos) continue;
    // info order: item by item, right-hand side by right-hand side
    int off = 0;
    for (int it = 0; it < g->item; ++it) off += items[it].nrhs;
    for (int i = 0; i < g->nreal; ++i) {
      stag_solve_info& inf = infos[off + g->first + i];
      const CgState& c = g->hst->sys[i];
      inf.iters = c.iter;
      inf.reliable_updates = g->hst->reliable_updates;
      inf.true_rel_resid = g->bb[i] > 0.0 ? std::sqrt(c.rr_true / g->bb[i]) : 0.0;
      inf.converged = g->bb[i] > 0.0 ? (c.rr_true <= c.target) : 1;
      inf.status = g->status ? g->status : (inf.converged ? STAG_OK : STAG_ENOTCONV);
      inf.seconds = t1 - t0;
      inf.precond_fallback = 0;
      if (!inf.converged && !worst) worst = STAG_ENOTCONV;
    }
  }
  return worst;
}

}  // namespace stag

using namespace stag;

extern "C" int stag_batch_solve(const stag_batch_item* items, int nitems, const stag_solve_params* params,
                                stag_solve_info* infos, void* stream) {
  if (!items || nitems <= 0) return STAG_EINVAL;
  stag_solve_params prm;
  stag_default_params(&prm);
  if (params) prm = *params;
  if (!(prm.tol > 0.0) || prm.max_iter < 0 || prm.mode < 0 || prm.mode > STAG_MIXED16L || prm.mode == STAG_LEARNED)
    return STAG_EINVAL;  // no learned mode
  if (prm.mode != STAG_PLAIN64 && !(prm.delta > 0.0 && prm.delta < 1.0)) return STAG_EINVAL;
  const int pi = prm.mode == STAG_PLAIN64 ? STAG_FP64 : prm.mode == STAG_MIXED32 ? STAG_FP32
               : prm.mode == STAG_MIXED16 ? STAG_FP16 : STAG_FX16;
  for (int i = 0; i < nitems; ++i) {
    const stag_batch_item& I = items[i];
    if (!I.lat || !I.x || !I.b || I.nrhs <= 0) return STAG_EINVAL;
    if (!I.lat->links[STAG_FP64].present || !I.lat->links[pi].present) return STAG_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  switch (prm.mode) {
    case STAG_PLAIN64: return batch_solve_p<64>(items, nitems, prm, infos, st);
    case STAG_MIXED32: return batch_solve_p<32>(items, nitems, prm, infos, st);
    case STAG_MIXED16: return batch_solve_p<16>(items, nitems, prm, infos, st);
    case STAG_MIXED16L: return batch_solve_p<31>(items, nitems, prm, infos, st);
    default: return batch_solve_p<15>(items, nitems, prm, infos, st);
  }
}
