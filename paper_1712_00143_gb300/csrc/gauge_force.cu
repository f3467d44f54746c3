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
// One thread per (site, direction), each staple walked link by link (the
// baseline algorithm, about 41 kflop per link), FP64 throughout: bound by
// the FP64 pipe on GB300.
#include "su3.cuh"

namespace stag {
namespace gf {
using namespace su3;

struct Pos {
  long long lex;
  C4 c;
};

__device__ __forceinline__ Pos step(const Dims& d, Pos p, int dir, int k) {
  Pos q;
  q.lex = shifted(d, p.lex, p.c, dir, k);
  const int L = extent(d, dir);
  int w = p.c.get(dir) + k;
  w = w >= L ? w - L : (w < 0 ? w + L : w);
  q.c = p.c;
  q.c.x = dir == 0 ? w : q.c.x;
  q.c.y = dir == 1 ? w : q.c.y;
  q.c.z = dir == 2 ? w : q.c.z;
  q.c.t = dir == 3 ? w : q.c.t;
  return q;
}

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

// acc += coef * (product of the links along the n steps from p)
template <int N>
__device__ __forceinline__ void staple(M3& acc, double coef, const double2* __restrict__ U, const Dims& d, Pos p,
                                       const int (&dir)[N], const int (&sgn)[N]) {
  M3 m = hop_link(U, d, p, dir[0], sgn[0]);
#pragma unroll
  for (int k = 1; k < N; ++k) m = mul(m, hop_link(U, d, p, dir[k], sgn[k]));
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    acc.e[i].x = fma(coef, m.e[i].x, acc.e[i].x);
    acc.e[i].y = fma(coef, m.e[i].y, acc.e[i].y);
  }
}

__global__ void __launch_bounds__(128) k_gauge_force(Dims d, long long V, const double2* __restrict__ U,
                                                     double2* __restrict__ F, double beta, double cpl, double crt,
                                                     double cpg) {
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
  const Pos p1 = step(d, p0, mu, 1);  // the staples start at x + mu
  M3 S;
#pragma unroll
  for (int i = 0; i < 9; ++i) S.e[i] = make_double2(0.0, 0.0);
#pragma unroll 1
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
#pragma unroll 1
    for (int s = -1; s <= 1; s += 2) {
      {
        const int dr[3] = {nu, mu, nu}, sg[3] = {s, -1, -s};
        staple<3>(S, cpl, U, d, p1, dr, sg);
      }
      {
        const int dr[5] = {mu, nu, mu, mu, nu}, sg[5] = {1, s, -1, -1, -s};
        staple<5>(S, crt, U, d, p1, dr, sg);
      }
      {
        const int dr[5] = {nu, mu, mu, nu, mu}, sg[5] = {s, -1, -1, -s, 1};
        staple<5>(S, crt, U, d, p1, dr, sg);
      }
      {
        const int dr[5] = {nu, nu, mu, nu, nu}, sg[5] = {s, s, -1, -s, -s};
        staple<5>(S, crt, U, d, p1, dr, sg);
      }
#pragma unroll 1
      for (int rho = 0; rho < 4; ++rho) {
        if (rho == mu || rho == nu) continue;
#pragma unroll 1
        for (int r = -1; r <= 1; r += 2) {
          const int dr[5] = {nu, rho, mu, nu, rho}, sg[5] = {s, r, -1, -s, -r};
          staple<5>(S, cpg, U, d, p1, dr, sg);
        }
      }
    }
  }
  const M3 us = mul(ld(U, x, mu), S);
  // TA: anti-Hermitian part minus a third of its trace, times beta / 3
  M3 a;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      a.e[3 * i + j] = make_double2(0.5 * (us.e[3 * i + j].x - us.e[3 * j + i].x),
                                    0.5 * (us.e[3 * i + j].y + us.e[3 * j + i].y));
  const double tr3 = (a.e[0].y + a.e[4].y + a.e[8].y) / 3.0;  // the trace is imaginary
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
  ProfScope ps("gauge_force", st);
  const long long n = 4 * V;
  gf::k_gauge_force<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(d, V, (const double2*)thin, (double2*)force, beta,
                                                                  c_pl, c_rt, c_pg);
  return last_launch_status();
}
