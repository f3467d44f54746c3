// fermion_force.cu -- the staggered fermion force through the link
// construction, FP64.
//
// The paper benchmarks the HISQ fermion force of the RHMC/RHMD algorithm as
// its third routine (Sec. 4.2).  For the pseudofermion action of a rational
// approximation in partial fractions,
//   S = sum_i alpha_i phi^dag (M + sigma_i)^{-1} phi,   M = m^2 - D_eo D_oe,
// with X_i = (M + sigma_i)^{-1} phi (even sites) and Y_i = D_oe X_i (odd
// sites), a change of the links changes S by sum_i alpha_i 2 Re X_i^dag dD_eo Y_i
//   = sum_{x,mu} Re Tr[dF_mu(x) G^F_mu(x) + dL_mu(x) G^L_mu(x)],
// with the outer products (summed over i, weight alpha_i)
//   x even: G^F_mu(x) =  eta_mu(x) Y(x+mu) X(x)^dag,   G^L: Y(x+3mu) in place of Y(x+mu)
//   x odd:  G^F_mu(x) = -eta_mu(x) X(x+mu) Y(x)^dag,   G^L: X(x+3mu) in place of X(x+mu)
// Pass 1 (k_ff_outer) stores G^F and G^L.  Pass 2 (k_ff_chain) takes the
// chain rule through the fat link F = c1 U + c_st (upper + lower staples) and
// the Naik link L = c3 U U U: for the thin link U_r(y) it gathers
//   Z = c1 G^F_r(y)
//     + c3 [ U_r(y+r) (U_r(y+2r) G^L_r(y) + G^L_r(y-r) U_r(y-r))
//            + G^L_r(y-2r) U_r(y-2r) U_r(y-r) ]
//     + c_st sum_{n != r} [ U_n(y+r) (G^F_r(y+n) U_n(y)^dag + U_r(y+n)^dag G^F_n(y))
//                           + G^F_n(y+r)^dag (U_n(y) U_r(y+n))^dag
//                           + U_n(y-n+r)^dag (G^F_r(y-n) U_n(y-n) + U_r(y-n)^dag G^F_n(y-n)^dag)
//                           + G^F_n(y-n+r) U_r(y-n)^dag U_n(y-n) ]
// (the six places a thin link takes in the staples: middle link of an upper
// and of a lower staple of F_r, first and last link of an upper and of a
// lower staple of F_n), so that dS = sum Re Tr[dU Z], and writes
//   force_r(y) = -TA[U_r(y) Z],  TA(A) = (A - A^dag)/2 - Tr(A - A^dag)/6,
// the convention of the gauge force: U -> exp(eps X) U changes S by
// -eps Re Tr(X force).  36 products of 3x3 complex matrices per link; bound
// by the FP64 pipe on GB300.
#include "su3.cuh"

namespace stag {
namespace ffc {
using namespace su3;

constexpr int MAX_TERMS = 32;
struct Alphas {
  double a[MAX_TERMS];
};

__device__ __forceinline__ void ld3(const double2* __restrict__ f, long long cb, double2 v[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c] = __ldg(f + cb * 3 + c);
}

// acc += w a b^dag (colour vectors a, b)
__device__ __forceinline__ void outer_acc(M3& acc, double w, const double2 a[3], const double2 b[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double re = a[i].x * b[j].x + a[i].y * b[j].y, im = a[i].y * b[j].x - a[i].x * b[j].y;
      acc.e[3 * i + j].x = fma(w, re, acc.e[3 * i + j].x);
      acc.e[3 * i + j].y = fma(w, im, acc.e[3 * i + j].y);
    }
}

__device__ __forceinline__ void st3x3(double2* __restrict__ p, const M3& m) {
#pragma unroll
  for (int i = 0; i < 9; ++i) p[i] = m.e[i];
}

// One thread per (site x, direction mu), idx = x * 4 + mu: consecutive threads
// write consecutive matrices.  X, Y: [n][V/2][3], checkerboard index lex / 2.
__global__ void __launch_bounds__(128) k_ff_outer(Dims d, long long V, long long Vh, int n, Alphas al,
                                                  const double2* __restrict__ X, const double2* __restrict__ Y,
                                                  double2* __restrict__ GF, double2* __restrict__ GL) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= 4 * V) return;
  const int mu = (int)(idx & 3);
  const long long x = idx >> 2;
  const Pos p = pos_of(d, x);
  const int par = (p.c.x + p.c.y + p.c.z + p.c.t) & 1;
  const int below = mu == 0 ? 0 : mu == 1 ? p.c.x : mu == 2 ? p.c.x + p.c.y : p.c.x + p.c.y + p.c.z;
  // eta_mu(x), and the sign of the odd-site terms
  const double sgn = ((below & 1) ? -1.0 : 1.0) * (par ? -1.0 : 1.0);
  const long long n1 = shifted(d, x, p.c, mu, 1) >> 1, n3 = shifted(d, x, p.c, mu, 3) >> 1, here = x >> 1;
  // even x: left field Y at the neighbour, right field X here; odd x: the reverse
  const double2* Fl = par ? X : Y;
  const double2* Fr = par ? Y : X;
  M3 gf = zero3(), gl = zero3();
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    const double w = sgn * al.a[i];
    double2 r[3], l1[3], l3[3];
    ld3(Fr + (long long)i * Vh * 3, here, r);
    ld3(Fl + (long long)i * Vh * 3, n1, l1);
    ld3(Fl + (long long)i * Vh * 3, n3, l3);
    outer_acc(gf, w, l1, r);
    outer_acc(gl, w, l3, r);
  }
  st3x3(GF + idx * 9, gf);
  st3x3(GL + idx * 9, gl);
}

__device__ __forceinline__ M3 ldG(const double2* __restrict__ G, long long site, int mu) { return ld(G, site, mu); }

// One thread per thin link, idx = r * V + y (a warp shares r).
__global__ void __launch_bounds__(128) k_ff_chain(Dims d, long long V, const double2* __restrict__ U,
                                                  const double2* __restrict__ GF, const double2* __restrict__ GL,
                                                  double2* __restrict__ force, double c1, double cst, double c3) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= 4 * V) return;
  const int r = (int)(idx / V);
  const long long y = idx - (long long)r * V;
  const Pos py = pos_of(d, y);
  const Pos pr = step(d, py, r, 1);   // y + r
  const Pos pmr = step(d, py, r, -1);  // y - r
  M3 Z = ldG(GF, y, r);
  scale3(Z, c1);
  // Naik: the link as first, middle and last factor of L_r(y), L_r(y-r), L_r(y-2r)
  {
    const M3 u_mr = ld(U, pmr.lex, r);  // U_r(y-r)
    M3 t = zero3();
    mac_mul(t, ld(U, step(d, pr, r, 1).lex, r), ldG(GL, y, r));  // U_r(y+2r) G^L_r(y)
    mac_mul(t, ldG(GL, pmr.lex, r), u_mr);                        // G^L_r(y-r) U_r(y-r)
    scale3(t, c3);
    mac_mul(Z, ld(U, pr.lex, r), t);
    const Pos pm2 = step(d, pmr, r, -1);  // y - 2r
    M3 w = mul(ldG(GL, pm2.lex, r), ld(U, pm2.lex, r));
    scale3(w, c3);
    mac_mul(Z, w, u_mr);
  }
#pragma unroll 1
  for (int n = 0; n < 4; ++n) {
    if (n == r) continue;
    {
      // staples through y + n and y: A = U_n(y+r), B = U_n(y), C = U_r(y+n)
      const Pos pn = step(d, py, n, 1);
      const M3 B = ld(U, y, n), C = ld(U, pn.lex, r);
      M3 t = zero3();
      mac_mul_dag(t, ldG(GF, pn.lex, r), B);  // G^F_r(y+n) U_n(y)^dag
      mac_dag_mul(t, C, ldG(GF, y, n));       // U_r(y+n)^dag G^F_n(y)
      scale3(t, cst);
      mac_mul(Z, ld(U, pr.lex, n), t);
      M3 w = mul(B, C);
      scale3(w, cst);
      mac_dag_mul_dag(Z, ldG(GF, pr.lex, n), w);  // G^F_n(y+r)^dag (U_n(y) U_r(y+n))^dag
    }
    {
      // staples through y - n: D = U_n(y-n+r), E = U_n(y-n), H = U_r(y-n)
      const Pos pmn = step(d, py, n, -1);
      const Pos pmnr = step(d, pmn, r, 1);
      const M3 E = ld(U, pmn.lex, n), H = ld(U, pmn.lex, r);
      M3 t = zero3();
      mac_mul(t, ldG(GF, pmn.lex, r), E);           // G^F_r(y-n) U_n(y-n)
      mac_dag_mul_dag(t, H, ldG(GF, pmn.lex, n));   // U_r(y-n)^dag G^F_n(y-n)^dag
      scale3(t, cst);
      mac_dag_mul(Z, ld(U, pmnr.lex, n), t);
      M3 w = zero3();
      mac_dag_mul(w, H, E);  // U_r(y-n)^dag U_n(y-n)
      scale3(w, cst);
      mac_mul(Z, ldG(GF, pmnr.lex, n), w);
    }
  }
  const M3 uz = mul(ld(U, y, r), Z);
  M3 a;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      a.e[3 * i + j] = make_double2(0.5 * (uz.e[3 * i + j].x - uz.e[3 * j + i].x),
                                    0.5 * (uz.e[3 * i + j].y + uz.e[3 * j + i].y));
  const double tr3 = (a.e[0].y + a.e[4].y + a.e[8].y) / 3.0;
  double2* f = force + (y * 4 + r) * 9;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      f[3 * i + j] = make_double2(-a.e[3 * i + j].x, -(a.e[3 * i + j].y - (i == j ? tr3 : 0.0)));
}

}  // namespace ffc
}  // namespace stag

using namespace stag;

extern "C" int stag_fermion_force(const int dims[4], const void* thin, int n_terms, const void* x_even,
                                  const void* y_odd, const double* alpha, double c1, double c_staple, double c3,
                                  void* force, void* stream) {
  if (!dims || !thin || !x_even || !y_odd || !alpha || !force) return STAG_EINVAL;
  if (n_terms < 1 || n_terms > ffc::MAX_TERMS) return STAG_EINVAL;
  long long V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 4 || dims[i] % 2) return STAG_EINVAL;
    V *= dims[i];
  }
  if (V > (1LL << 31)) return STAG_EINVAL;
  const long long Vh = V / 2;
  const size_t lbytes = (size_t)V * 4 * 9 * sizeof(double2), fbytes = (size_t)n_terms * Vh * 3 * sizeof(double2);
  auto overlap = [](const void* a, size_t na, const void* b, size_t nb) {
    const char *p = (const char*)a, *q = (const char*)b;
    return p < q + nb && q < p + na;
  };
  if (overlap(force, lbytes, thin, lbytes) || overlap(force, lbytes, x_even, fbytes) ||
      overlap(force, lbytes, y_odd, fbytes))
    return STAG_EINVAL;
  ffc::Alphas al{};
  for (int i = 0; i < n_terms; ++i) al.a[i] = alpha[i];
  const su3::Dims d{dims[0], dims[1], dims[2], dims[3]};
  cudaStream_t st = (cudaStream_t)stream;
  // G^F and G^L, one matrix per link each, in stream-ordered scratch
  double2* G = nullptr;
  if (cudaMallocAsync((void**)&G, 2 * lbytes, st) != cudaSuccess) {
    cudaGetLastError();
    return STAG_ENOMEM;
  }
  double2* GF = G;
  double2* GL = G + (size_t)V * 4 * 9;
  int s = STAG_OK;
  const long long n = 4 * V;
  const unsigned grid = (unsigned)((n + 127) / 128);
  {
    ProfScope ps("fermion_force", st);
    ffc::k_ff_outer<<<grid, 128, 0, st>>>(d, V, Vh, n_terms, al, (const double2*)x_even, (const double2*)y_odd, GF,
                                          GL);
    s = last_launch_status();
  }
  if (!s) {
    ProfScope ps("fermion_force", st);
    ffc::k_ff_chain<<<grid, 128, 0, st>>>(d, V, (const double2*)thin, GF, GL, (double2*)force, c1, c_staple, c3);
    s = last_launch_status();
  }
  const int f = cuda_status(cudaFreeAsync(G, st));
  return s ? s : f;
}
