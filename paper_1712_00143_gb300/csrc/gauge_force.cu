// gauge_force.cu -- the Symanzik one-loop improved gauge force in FP64.
//
// The paper benchmarks the gauge force of the HISQ RHMC/RHMD algorithm next
// to the CG (Sec. 4.2, Figs. 6-8: matrix-matrix products, arithmetic
// intensity 1.1 in MILC's baseline code and above 2.0 with reuse of
// three-link staples).  The action is the Luscher-Weisz form
//   S = beta sum_loops c (1 - Re Tr W / 3)
// over plaquettes (c_pl), 1x2 rectangles (c_rt) and parallelograms (the
// six-link loop a, b, c, -a, -b, -c over three directions; c_pg).  For the
// link U_mu(x), Sigma_mu(x) sums c times the product of the other links of
// every loop through it, each loop oriented to traverse U_mu(x) forward and
// started right after it:
//   plaquettes    [nu s, mu -, nu -s]                            6
//   rectangles    [mu +, nu s, mu -, mu -, nu -s]                6
//                 [nu s, mu -, mu -, nu -s, mu +]                6
//                 [nu s, nu s, mu -, nu -s, nu -s]               6
//   parallelograms [nu s, rho r, mu -, nu -s, rho -r]            24
// (nu, rho distinct and != mu, s, r = +-1), and the force is
//   F_mu(x) = (beta/3) TA[U_mu(x) Sigma_mu(x)],  TA(M) = (M - M^dag)/2 - Tr(M - M^dag)/6,
// so that moving the link as exp(eps X) U changes S by -eps Re Tr(X F).
// FP64 throughout; bound by the FP64 pipe on GB300.  The staples are built
// from a stored table of three-link staples (below).
#include "su3.cuh"

namespace stag {
namespace gf {
using namespace su3;

__device__ __forceinline__ M3 dagger(const M3& a) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) r.e[3 * i + j] = make_double2(a.e[3 * j + i].x, -a.e[3 * j + i].y);
  return r;
}

// The link of one step from p (forward: U_dir(p), then p += dir; backward:
// p -= dir, then U_dir(p)^dag).
__device__ __forceinline__ M3 hop_link(const double2* __restrict__ U, const Dims& d, Pos& p, int dir, int sgn) {
  if (sgn > 0) {
    const M3 l = ld(U, p.lex, dir);
    p = step(d, p, dir, 1);
    return l;
  }
  p = step(d, p, dir, -1);
  return dagger(ld(U, p.lex, dir));
}

// ------------------------------------------------------------ staple reuse
// The paper's QOPQDP and QPhiX versions reuse three-link staples (60 % fewer
// flops than MILC's baseline, Sec. 4.2).  Here: one pass stores, for every
// link (y, mu) and plane (nu, s), its plaquette staple
//   T_{mu nu s}(y) = h(y+mu, nu, s) U_mu(y+s nu)^dag h(y+s nu, nu, -s)
// (the path [nu s, mu -, nu -s] from y + mu; h(z, nu, +1) = U_nu(z),
// h(z, nu, -1) = U_nu(z-nu)^dag), 24 per site; the force pass then closes
// every loop through U_mu(x) from at most three factors, the hops next to
// x + mu and x + s nu cancelling between adjacent staples:
//   plaquette        T(x; mu nu s)
//   rectangle 1      U_mu(x+mu) T(x+mu; mu nu s) T(x; mu nu s)
//   rectangle 2      T(x; mu nu s) T(x-mu; mu nu s) U_mu(x-mu)
//   rectangle 3      h(x+mu, nu, s) T(x+s nu; mu nu s) h(x+s nu, nu, -s)
//   parallelogram    h(x+mu, nu, s) T(x+s nu; mu rho r) Q,  Q = T(x; nu rho r) (s = +1)
//                                                          or T(x-nu; nu rho r)^dag (s = -1)
// with the left factor h(x+mu, nu, s) shared by rectangle 3 and the four
// parallelograms of (nu, s): 12 products per link for the table and 60 for
// the force, against 181 when every staple is walked link by link.

// slot of T(y; mu nu s) in the table: [site][mu][nu][s], 9 complex each
__device__ __forceinline__ long long tslot(long long y, int mu, int nu, int s) {
  return (((y * 4 + mu) * 4 + nu) * 2 + (s < 0 ? 1 : 0)) * 9;
}

__device__ __forceinline__ M3 ldT(const double2* __restrict__ T, long long y, int mu, int nu, int s) {
  M3 m;
  const double2* p = T + tslot(y, mu, nu, s);
#pragma unroll
  for (int i = 0; i < 9; ++i) m.e[i] = __ldg(p + i);
  return m;
}

// h(p, dir, sgn) without moving p
__device__ __forceinline__ M3 hop_at(const double2* __restrict__ U, const Dims& d, Pos p, int dir, int sgn) {
  return hop_link(U, d, p, dir, sgn);
}

__global__ void __launch_bounds__(128) k_gf_staples(Dims d, long long V, const double2* __restrict__ U,
                                                    double2* __restrict__ T) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= 24 * V) return;
  const int k = (int)(idx / V);  // mu * 6 + (other direction index) * 2 + sign
  const long long x = idx - (long long)k * V;
  const int mu = k / 6, o = (k % 6) >> 1, s = (k & 1) ? -1 : 1;
  const int nu = o < mu ? o : o + 1;
  Pos p0;
  p0.lex = x;
  {
    long long r = x;
    p0.c.x = (int)(r % d.L0);
    r /= d.L0;
    p0.c.y = (int)(r % d.L1);
    r /= d.L1;
    p0.c.z = (int)(r % d.L2);
    p0.c.t = (int)(r / d.L2);
  }
  Pos p = step(d, p0, mu, 1);  // walk [nu s, mu -, nu -s] from x + mu
  M3 m = hop_link(U, d, p, nu, s);
  m = mul(m, hop_link(U, d, p, mu, -1));
  m = mul(m, hop_link(U, d, p, nu, -s));
  double2* out = T + tslot(x, mu, nu, s);
#pragma unroll
  for (int i = 0; i < 9; ++i) out[i] = m.e[i];
}

// acc += c m
__device__ __forceinline__ void axpy3(M3& acc, double c, const M3& m) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    acc.e[i].x = fma(c, m.e[i].x, acc.e[i].x);
    acc.e[i].y = fma(c, m.e[i].y, acc.e[i].y);
  }
}

__global__ void __launch_bounds__(128) k_gauge_force_reuse(Dims d, long long V, const double2* __restrict__ U,
                                                           const double2* __restrict__ T, double2* __restrict__ F,
                                                           double beta, double cpl, double crt, double cpg) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= 4 * V) return;
  const int mu = (int)(idx / V);
  const long long x = idx - (long long)mu * V;
  Pos p0;
  p0.lex = x;
  {
    long long r = x;
    p0.c.x = (int)(r % d.L0);
    r /= d.L0;
    p0.c.y = (int)(r % d.L1);
    r /= d.L1;
    p0.c.z = (int)(r % d.L2);
    p0.c.t = (int)(r / d.L2);
  }
  const Pos pp = step(d, p0, mu, 1), pm = step(d, p0, mu, -1);  // x + mu, x - mu
  const M3 u_pm = ld(U, pp.lex, mu), u_mm = ld(U, pm.lex, mu);  // U_mu(x+mu), U_mu(x-mu)
  M3 S;
#pragma unroll
  for (int i = 0; i < 9; ++i) S.e[i] = make_double2(0.0, 0.0);
#pragma unroll 1
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
#pragma unroll 1
    for (int s = -1; s <= 1; s += 2) {
      const M3 t0 = ldT(T, x, mu, nu, s);
      axpy3(S, cpl, t0);                                          // plaquette
      axpy3(S, crt, mul(u_pm, mul(ldT(T, pp.lex, mu, nu, s), t0)));  // rectangle 1
      axpy3(S, crt, mul(mul(t0, ldT(T, pm.lex, mu, nu, s)), u_mm));  // rectangle 2
      // rectangle 3 and the parallelograms share the left factor h(x+mu, nu, s)
      const Pos ps = step(d, p0, nu, s);  // x + s nu
      M3 R = mul(ldT(T, ps.lex, mu, nu, s), hop_at(U, d, ps, nu, -s));
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        R.e[i].x *= crt;
        R.e[i].y *= crt;
      }
      const Pos pmn = step(d, p0, nu, -1);  // x - nu (for s = -1)
#pragma unroll 1
      for (int rho = 0; rho < 4; ++rho) {
        if (rho == mu || rho == nu) continue;
#pragma unroll 1
        for (int r = -1; r <= 1; r += 2) {
          const M3 a = ldT(T, ps.lex, mu, rho, r);
          M3 q = s > 0 ? ldT(T, x, nu, rho, r) : dagger(ldT(T, pmn.lex, nu, rho, r));
          const M3 aq = mul(a, q);
          axpy3(R, cpg, aq);
        }
      }
      const M3 hl = hop_at(U, d, pp, nu, s);
      const M3 hr = mul(hl, R);
      axpy3(S, 1.0, hr);
    }
  }
  const M3 us = mul(ld(U, x, mu), S);
  M3 a;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      a.e[3 * i + j] = make_double2(0.5 * (us.e[3 * i + j].x - us.e[3 * j + i].x),
                                    0.5 * (us.e[3 * i + j].y + us.e[3 * j + i].y));
  const double tr3 = (a.e[0].y + a.e[4].y + a.e[8].y) / 3.0;
  const double k = beta / 3.0;
  double2* f = F + (x * 4 + mu) * 9;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      f[3 * i + j] = make_double2(k * a.e[3 * i + j].x, k * (a.e[3 * i + j].y - (i == j ? tr3 : 0.0)));
}

}  // namespace gf
}  // namespace stag

using namespace stag;

extern "C" int stag_gauge_force(const int dims[4], const void* thin, void* force, double beta, double c_pl,
                                double c_rt, double c_pg, void* stream) {
  if (!dims || !thin || !force) return STAG_EINVAL;
  long long V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 4 || dims[i] % 2) return STAG_EINVAL;
    V *= dims[i];
  }
  if (V > (1LL << 31)) return STAG_EINVAL;
  const size_t bytes = (size_t)V * 4 * 9 * sizeof(double2);
  const char *p = (const char*)thin, *q = (const char*)force;
  if (p < q + bytes && q < p + bytes) return STAG_EINVAL;
  const su3::Dims d{dims[0], dims[1], dims[2], dims[3]};
  cudaStream_t st = (cudaStream_t)stream;
  // the staple table (24 matrices per site, 3456 B) in stream-ordered scratch
  double2* T = nullptr;
  if (cudaMallocAsync((void**)&T, (size_t)V * 32 * 9 * sizeof(double2), st) != cudaSuccess) {
    cudaGetLastError();
    return STAG_ENOMEM;
  }
  int s = STAG_OK;
  {
    ProfScope ps("gauge_force", st);
    const long long n = 24 * V;
    gf::k_gf_staples<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(d, V, (const double2*)thin, T);
    s = last_launch_status();
  }
  if (!s) {
    ProfScope ps("gauge_force", st);
    const long long n = 4 * V;
    gf::k_gauge_force_reuse<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(d, V, (const double2*)thin, T,
                                                                          (double2*)force, beta, c_pl, c_rt, c_pg);
    s = last_launch_status();
  }
  const int f = cuda_status(cudaFreeAsync(T, st));
  return s ? s : f;
}
