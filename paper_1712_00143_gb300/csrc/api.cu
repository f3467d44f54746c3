// api.cu -- C ABI entry points of libstag (handles, Dslash, operator apply),
// device workspaces and the event-pair kernel profiler.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace stag {

// ------------------------------------------------------------ workspace
Workspace::~Workspace() { release(); }

void Workspace::release() {
  for (auto& kv : bufs)
    if (kv.second.first) cudaFree(kv.second.first);
  bufs.clear();
}

void* Workspace::get(const std::string& name, size_t bytes, int* status, bool* fresh) {
  if (fresh) *fresh = false;
  auto it = bufs.find(name);
  if (it != bufs.end() && it->second.second >= bytes) return it->second.first;
  if (it != bufs.end()) {
    cudaFree(it->second.first);
    bufs.erase(it);
  }
  void* p = nullptr;
  size_t n = bytes ? bytes : 16;
  if (cudaMalloc(&p, n) != cudaSuccess) {
    cudaGetLastError();
    *status = STAG_ENOMEM;
    return nullptr;
  }
  bufs[name] = {p, n};
  if (fresh) *fresh = true;
  return p;
}

void Workspace::drop(const std::string& name) {
  auto it = bufs.find(name);
  if (it == bufs.end()) return;
  cudaFree(it->second.first);
  bufs.erase(it);
}

int get_red_scratch(stag_lattice_s* lat, const char* name, RedScratch* out, int nv_max) {
  int st = 0;
  int max_grid = (lat->g.Vh + 127) / 128;  // one block per 128 sites at most
  if (max_grid < 1024) max_grid = 1024;
  std::string n(name);
  double* p = (double*)lat->ws.get(n + ".partials", sizeof(double) * (size_t)nv_max * (size_t)max_grid, &st);
  if (st) return st;
  bool fresh = false;
  unsigned* c = (unsigned*)lat->ws.get(n + ".counter", 256, &st, &fresh);
  if (st) return st;
  if (fresh && cudaMemset(c, 0, 256) != cudaSuccess) return STAG_ECUDA;
  out->partials = p;
  out->counter = c;
  out->max_grid = max_grid;
  return STAG_OK;
}

int last_launch_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? STAG_OK : STAG_ECUDA;
}

// ------------------------------------------------------------ profiler
namespace {
struct Rec {
  const char* family;
  cudaEvent_t a, b;
  long long seq;  // creation order (see prof_discard_since)
};
std::mutex g_mu;
bool g_prof = false;
std::string g_filter;  // comma-separated families to time; empty = all
long long g_every = 1;  // time one launch in g_every of each selected family
std::map<std::string, long long> g_seen;
std::atomic<long long> g_launches{0};
std::vector<Rec> g_open;
std::vector<cudaEvent_t> g_pool;
struct Tot {
  long long n = 0;
  double ms = 0.0;
};
std::map<std::string, Tot> g_tot;
long long g_seq = 0;
thread_local int t_pending = -1;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Accumulates finished records; with `wait`, waits for every record.
void flush_locked(bool wait) {
  size_t keep = 0;
  for (size_t i = 0; i < g_open.size(); ++i) {
    Rec& r = g_open[i];
    bool done = r.b != nullptr;
    if (done) {
      if (wait)
        done = cudaEventSynchronize(r.b) == cudaSuccess;
      else
        done = cudaEventQuery(r.b) == cudaSuccess;
      cudaGetLastError();
    }
    if (done) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
        Tot& t = g_tot[r.family];
        t.n += 1;
        t.ms += ms;
      }
      cudaGetLastError();
      g_pool.push_back(r.a);
      g_pool.push_back(r.b);
    } else {
      g_open[keep++] = r;
    }
  }
  g_open.resize(keep);
}
}  // namespace

thread_local bool t_capturing = false;
thread_local long long t_captured = 0;

void count_launch() {
  if (t_capturing)
    ++t_captured;
  else
    g_launches.fetch_add(1, std::memory_order_relaxed);
}

long long set_capturing(bool on) {
  long long n = t_captured;
  t_capturing = on;
  t_captured = 0;
  return n;
}

bool family_selected(const char* family) {
  if (g_filter.empty()) return true;
  const std::string f(family);
  size_t pos = 0;
  while (pos <= g_filter.size()) {
    size_t end = g_filter.find(',', pos);
    if (end == std::string::npos) end = g_filter.size();
    if (g_filter.compare(pos, end - pos, f) == 0) return true;
    pos = end + 1;
  }
  return false;
}

void prof_begin(const char* family, cudaStream_t s) {
  t_pending = -1;
  if (!g_prof || t_capturing) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!family_selected(family)) return;
  if (g_every > 1 && (g_seen[family]++ % g_every) != 0) return;
  if (g_open.size() > 8192) flush_locked(false);
  cudaEvent_t a = take_event();
  if (!a) return;
  cudaEventRecord(a, s);
  g_open.push_back(Rec{family, a, nullptr, g_seq++});
  t_pending = (int)g_open.size() - 1;
}

void prof_end(cudaStream_t s) {
  if (t_pending < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  if (b) {
    cudaEventRecord(b, s);
    g_open[t_pending].b = b;
  }
  t_pending = -1;
}

void prof_flush_completed() {
  if (!g_prof) return;
  std::lock_guard<std::mutex> lk(g_mu);
  flush_locked(false);
}

long long prof_mark() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_seq;
}

// Drops the records created since `mark` that have not been accumulated yet,
// when launches are sampled (every > 1; with every launch timed the totals
// stay complete).  The solvers call it, before their next
// prof_flush_completed, for a chunk of queued iterations that a stop flag
// cut short: the launches queued after the flag returned at once and would
// otherwise enter the sampled averages as near-empty launches.  (Records are
// accumulated only by an explicit flush, or when more than 8192 are open,
// far above the records of one chunk.)
void prof_discard_since(long long mark) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_every <= 1) return;
  size_t keep = 0;
  for (size_t i = 0; i < g_open.size(); ++i) {
    Rec& r = g_open[i];
    if (r.seq >= mark) {
      if (r.b) cudaEventSynchronize(r.b);
      cudaGetLastError();
      g_pool.push_back(r.a);
      if (r.b) g_pool.push_back(r.b);
    } else {
      g_open[keep++] = r;
    }
  }
  g_open.resize(keep);
}

// ------------------------------------------------------------ bounds records
#ifdef STAG_DEBUG_BOUNDS
namespace {
struct BoundsTU {
  int (*read)(unsigned long long*);
  int (*clear)();
};
std::vector<BoundsTU>& bounds_registry() {
  static std::vector<BoundsTU> r;
  return r;
}
}  // namespace
void bounds_register(int (*read)(unsigned long long*), int (*clear)()) { bounds_registry().push_back({read, clear}); }
#endif

}  // namespace stag

using namespace stag;

// ------------------------------------------------------------ ABI
extern "C" {

const char* stag_strerror(int s) {
  switch (s) {
    case STAG_OK: return "ok";
    case STAG_EINVAL: return "invalid argument";
    case STAG_ENOMEM: return "device allocation failed";
    case STAG_ECUDA: return "CUDA runtime error";
    case STAG_ENOTCONV: return "solver did not converge within max_iter";
    case STAG_EBREAKDOWN: return "solver breakdown (NaN/Inf or non-positive <p,Ap>)";
    case STAG_ENOTUNITARY: return "long links are not c3 times an SU(3) matrix";
    case STAG_ETIMEOUT: return "bounded device wait gave up";
    default: return "unknown status";
  }
}

void stag_default_params(stag_solve_params* p) {
  if (!p) return;
  p->tol = 1e-10;
  p->max_iter = 100000;
  p->mode = STAG_MIXED32;
  p->delta = 0.1;
  p->use_initial_guess = 0;
  p->check_interval = 16;
  p->ms_tol = 1e-6;
  p->precond = nullptr;
}

int stag_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_prof = on != 0;
  return STAG_OK;
}

int stag_profile_select(const char* families, int every) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_filter = families ? families : "";
  g_every = every > 1 ? every : 1;
  g_seen.clear();
  return STAG_OK;
}

int stag_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  flush_locked(true);
  g_tot.clear();
  g_launches.store(0);
  return STAG_OK;
}

int stag_profile_read(const char* family, long long* launches, double* total_ms) {
  if (!family) return STAG_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  flush_locked(true);
  auto it = g_tot.find(family);
  if (launches) *launches = it == g_tot.end() ? 0 : it->second.n;
  if (total_ms) *total_ms = it == g_tot.end() ? 0.0 : it->second.ms;
  return STAG_OK;
}

long long stag_launch_count(void) { return g_launches.load(); }

int stag_bounds_violations(long long* count, int* first_code, long long* first_index, int clear) {
  if (!count) return STAG_EINVAL;
#ifdef STAG_DEBUG_BOUNDS
  long long n = 0;
  int code = 0;
  long long index = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return STAG_ECUDA;
  }
  for (const auto& tu : bounds_registry()) {
    unsigned long long v[3] = {0ull, 0ull, 0ull};
    if (tu.read(v)) {
      cudaGetLastError();
      return STAG_ECUDA;
    }
    if (v[0] && !n) {
      code = (int)v[1];
      index = (long long)v[2];
    }
    n += (long long)v[0];
    if (clear && v[0] && tu.clear()) {
      cudaGetLastError();
      return STAG_ECUDA;
    }
  }
  *count = n;
  if (first_code) *first_code = code;
  if (first_index) *first_index = index;
#else
  (void)clear;
  *count = -1;
  if (first_code) *first_code = 0;
  if (first_index) *first_index = 0;
#endif
  return STAG_OK;
}

int stag_load_links(stag_lattice_t* out, const int dims[4], const void* fat, const void* lng,
                    const stag_link_opts* opts, void* stream) {
  if (!out || !dims || !fat || !lng) return STAG_EINVAL;
  *out = nullptr;
  long long V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 4 || dims[i] % 2) return STAG_EINVAL;
    V *= dims[i];
  }
  if (V / 2 > (1LL << 30)) return STAG_EINVAL;
  stag_link_opts o;
  o.recon_long = 18;
  o.long_coeff = -1.0 / 24.0;
  o.prec_mask = 0;
  o.autotune = 1;
  if (opts) o = *opts;
  if (o.recon_long != 18 && o.recon_long != 12) return STAG_EINVAL;
  if (o.recon_long == 12 && !(o.long_coeff != 0.0)) return STAG_EINVAL;
  unsigned mask = o.prec_mask ? o.prec_mask : 31u;
  if (mask & ~31u) return STAG_EINVAL;
  stag_lattice_s* lat = new stag_lattice_s();
  for (int i = 0; i < 4; ++i) lat->dims[i] = dims[i];
  lat->g = make_geom(dims);
  lat->c3 = o.long_coeff;
  lat->autotune = o.autotune ? 1 : 0;
  cudaStream_t st = (cudaStream_t)stream;
  for (int p = 0; p < 5; ++p) {
    if (!((mask >> p) & 1)) continue;
    int s = build_link_copy(lat, p, o.recon_long, (const double2*)fat, (const double2*)lng, st);
    if (!s && o.autotune && p == STAG_DF64) s = tune_df(lat, st);
    if (!s && o.autotune && p != STAG_DF64) {
      switch (p) {
        case STAG_FP64: s = tune_dslash<64>(lat, st); break;
        case STAG_FP32: s = tune_dslash<32>(lat, st); break;
        case STAG_FP16: s = tune_dslash<16>(lat, st); break;
        default: s = tune_dslash<15>(lat, st);
      }
    }
    if (s) {
      stag_free_lattice(lat);
      return s;
    }
  }
  *out = lat;
  return STAG_OK;
}

int stag_free_lattice(stag_lattice_t lat) {
  if (!lat) return STAG_EINVAL;
  cudaDeviceSynchronize();
  for (auto& L : lat->links)
    if (L.data) cudaFree(L.data);
  delete lat;
  return STAG_OK;
}

int stag_tuned_shape(stag_lattice_t lat, int prec, int kernel, int* block, int* min_blocks, double* us) {
  if (!lat || prec < 0 || prec > STAG_FX16L32 || kernel < 0 || kernel > 1) return STAG_EINVAL;
  prec = link_copy_of(prec);  // the single-RHS STAG_FX16L32 kernels run in the shapes tuned for STAG_FX16
  if (!lat->links[prec].present) return STAG_EINVAL;
  const LinkCopy& L = lat->links[prec];
  int v = kernel == 0 ? L.shape_plain : L.shape_epi;
  if (prec == STAG_DF64) {
    // double-float: 128 threads per block; min_blocks reports the threads
    // that share one site's four right-hand sides (1, 2 or 4)
    if (block) *block = 128;
    if (min_blocks) *min_blocks = v == 0 ? 1 : v == 1 ? 2 : 4;
    if (us) *us = L.tuned_us[kernel];
    return STAG_OK;
  }
  if (block) *block = v < 2 ? 256 : 128;
  if (min_blocks) *min_blocks = v == 1 ? 4 : v == 3 ? 8 : 1;
  if (us) *us = L.tuned_us[kernel];
  return STAG_OK;
}

int stag_lattice_info(stag_lattice_t lat, int dims[4], long long* vh) {
  if (!lat) return STAG_EINVAL;
  if (dims)
    for (int i = 0; i < 4; ++i) dims[i] = lat->dims[i];
  if (vh) *vh = lat->g.Vh;
  return STAG_OK;
}

}  // extern "C"

namespace stag {

// A Spinor<P> in workspace buffer `name` (FP16: scales after the vectors).
template <int P> Spinor<P> ws_spinor(stag_lattice_s* lat, const std::string& name, int* status) {
  Spinor<P> f;
  f.Vh = lat->g.Vh;
  f.v = lat->ws.get(name, spinor_bytes<P>(f.Vh), status);
  return f;
}
template Spinor<64> ws_spinor<64>(stag_lattice_s*, const std::string&, int*);
template Spinor<32> ws_spinor<32>(stag_lattice_s*, const std::string&, int*);
template Spinor<16> ws_spinor<16>(stag_lattice_s*, const std::string&, int*);
template Spinor<15> ws_spinor<15>(stag_lattice_s*, const std::string&, int*);
template Spinor<31> ws_spinor<31>(stag_lattice_s*, const std::string&, int*);

template <int P>
static int dslash_p(stag_lattice_s* lat, double2* out, const double2* in, int out_parity, int nrhs, cudaStream_t st) {
  int s = 0;
  Spinor<P> a = ws_spinor<P>(lat, "dslash.in", &s);
  if (s) return s;
  Spinor<P> b = ws_spinor<P>(lat, "dslash.out", &s);
  if (s) return s;
  const size_t n = (size_t)lat->g.Vh * 3;
  for (int r = 0; r < nrhs; ++r) {
    if ((s = launch_from_canonical<P>(a, in + r * n, lat->g.Vh, st))) return s;
    if ((s = launch_dslash<P>(lat, b, a, out_parity, nullptr, st))) return s;
    if ((s = launch_to_canonical<P>(out + r * n, b, lat->g.Vh, st))) return s;
  }
  return STAG_OK;
}

template <int P>
static int apply_m_p(stag_lattice_s* lat, double2* out, const double2* in, double shift, cudaStream_t st) {
  constexpr int PA = Acc<P>::value;
  int s = 0;
  Spinor<P> a = ws_spinor<P>(lat, "applym.in", &s);
  if (s) return s;
  Spinor<P> t = ws_spinor<P>(lat, "applym.t", &s);
  if (s) return s;
  Spinor<PA> o = ws_spinor<PA>(lat, "applym.out", &s);
  if (s) return s;
  if ((s = launch_from_canonical<P>(a, in, lat->g.Vh, st))) return s;
  if ((s = launch_dslash<P>(lat, t, a, 1, nullptr, st))) return s;
  RedScratch rs{nullptr, nullptr, 0};
  Spinor<PA> none{nullptr, lat->g.Vh};
  if ((s = launch_dslash_epi<P>(lat, o, t, 0, a, shift, none, 0.0, -1.0, 0, rs, RedTarget{RED_STORE, nullptr, nullptr},
                                nullptr, st)))
    return s;
  return launch_to_canonical<PA>(out, o, lat->g.Vh, st);
}

// Double-float: canonical FP64 in, split exactly, DF hops, DF out widened to FP64.
static int dslash_df_canonical(stag_lattice_s* lat, double2* out, const double2* in, int out_parity, int nrhs,
                               cudaStream_t st) {
  int s = 0;
  const int Vh = lat->g.Vh;
  DfField a{(float4*)lat->ws.get("dslashdf.in", df_bytes(Vh) * nrhs, &s), Vh};
  DfField b{(float4*)lat->ws.get("dslashdf.out", df_bytes(Vh) * nrhs, &s), Vh};
  if (s) return s;
  if ((s = launch_df_from_double(a, in, nrhs, st))) return s;
  if ((s = launch_dslash_df(lat, b, a, nrhs, out_parity, nullptr, st))) return s;
  return launch_df_to_double(out, b, nrhs, st);
}

static int apply_m_df(stag_lattice_s* lat, double2* out, const double2* in, double shift, cudaStream_t st) {
  int s = 0;
  const int Vh = lat->g.Vh;
  DfField a{(float4*)lat->ws.get("applymdf.in", df_bytes(Vh), &s), Vh};
  DfField t{(float4*)lat->ws.get("applymdf.t", df_bytes(Vh), &s), Vh};
  DfField o{(float4*)lat->ws.get("applymdf.out", df_bytes(Vh), &s), Vh};
  if (s) return s;
  if ((s = launch_df_from_double(a, in, 1, st))) return s;
  if ((s = launch_dslash_df(lat, t, a, 1, 1, nullptr, st))) return s;
  if ((s = launch_dslash_df_epi(lat, o, t, 1, 0, a, shift, DfField{nullptr, Vh}, 0.0, -1.0, nullptr, st))) return s;
  return launch_df_to_double(out, o, 1, st);
}

}  // namespace stag

extern "C" {

int stag_dslash(stag_lattice_t lat, void* out, const void* in, int out_parity, int prec, int nrhs, void* stream) {
  if (!lat || !out || !in || (out_parity != 0 && out_parity != 1) || nrhs < 1) return STAG_EINVAL;
  if (prec < 0 || prec > STAG_FX16L32 || !lat->links[link_copy_of(prec)].present) return STAG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == STAG_DF64) return dslash_df_canonical(lat, (double2*)out, (const double2*)in, out_parity, nrhs, st);
  if (nrhs > 1) return dslash_multi(lat, (double2*)out, (const double2*)in, out_parity, prec, nrhs, st);
  switch (prec) {
    case STAG_FX16L32: return dslash_p<31>(lat, (double2*)out, (const double2*)in, out_parity, nrhs, st);
    case STAG_FP64: return dslash_p<64>(lat, (double2*)out, (const double2*)in, out_parity, nrhs, st);
    case STAG_FP32: return dslash_p<32>(lat, (double2*)out, (const double2*)in, out_parity, nrhs, st);
    case STAG_FP16: return dslash_p<16>(lat, (double2*)out, (const double2*)in, out_parity, nrhs, st);
    default: return dslash_p<15>(lat, (double2*)out, (const double2*)in, out_parity, nrhs, st);
  }
}

int stag_apply_m(stag_lattice_t lat, void* out, const void* in, double mass, double shift, int prec, void* stream) {
  if (!lat || !out || !in) return STAG_EINVAL;
  if (prec < 0 || prec > STAG_FX16L32 || !lat->links[link_copy_of(prec)].present) return STAG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  double a = mass * mass + shift;
  if (prec == STAG_DF64) return apply_m_df(lat, (double2*)out, (const double2*)in, a, st);
  switch (prec) {
    case STAG_FX16L32: return apply_m_p<31>(lat, (double2*)out, (const double2*)in, a, st);
    case STAG_FP64: return apply_m_p<64>(lat, (double2*)out, (const double2*)in, a, st);
    case STAG_FP32: return apply_m_p<32>(lat, (double2*)out, (const double2*)in, a, st);
    case STAG_FP16: return apply_m_p<16>(lat, (double2*)out, (const double2*)in, a, st);
    default: return apply_m_p<15>(lat, (double2*)out, (const double2*)in, a, st);
  }
}

}  // extern "C"
