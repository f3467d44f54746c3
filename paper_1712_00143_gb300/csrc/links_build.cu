// links_build.cu -- the link construction that precedes the operator: fat
// (three-staple) and Naik links from thin links, in FP64 on the GPU.
//
// The paper's production code smears the thin gauge links before the CG
// (HISQ-link smearing, Sec. 1, and its share of the run time in Sec. 2,
// Fig. 1); the workload here uses the three-staple fat link and the Naik
// link:
//   F_mu(x) = c1 U_mu(x) + c_st sum_{nu != mu} [ U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
//                                               + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ]
//   L_mu(x) = c3 U_mu(x) U_mu(x+mu) U_mu(x+2mu)
// One thread per (site, direction): 12 staple products and 2 Naik products
// of 3x3 complex matrices (about 1500 FP64 FMA), inputs from L2 (each thin
// link is read by up to 19 threads), outputs written once in the canonical
// layout.  Bound by the FP64 pipe on GB300 (about 1.2 TFLOP/s).
#include "su3.cuh"

namespace stag {
namespace lb {
using namespace su3;

__global__ void __launch_bounds__(128) k_build_links(Dims d, long long V, const double2* __restrict__ U,
                                                     double2* __restrict__ F, double2* __restrict__ Lk, double c1,
                                                     double cst, double c3) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= 4 * V) return;
  const int mu = (int)(idx / V);
  const long long x = idx - (long long)mu * V;
  C4 c;
  {
    long long r = x;
    c.x = (int)(r % d.L0);
    r /= d.L0;
    c.y = (int)(r % d.L1);
    r /= d.L1;
    c.z = (int)(r % d.L2);
    c.t = (int)(r / d.L2);
  }
  const long long x_pmu = shifted(d, x, c, mu, 1);
  M3 S;
#pragma unroll
  for (int i = 0; i < 9; ++i) S.e[i] = make_double2(0.0, 0.0);
#pragma unroll 1
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    // upper staple U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
    {
      const M3 ab = mul(ld(U, x, nu), ld(U, shifted(d, x, c, nu, 1), mu));
      mac_mul_dag(S, ab, ld(U, x_pmu, nu));
    }
    // lower staple U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu): x - nu + mu is
    // x + mu moved by -nu (mu != nu)
    {
      const long long x_mnu = shifted(d, x, c, nu, -1);
      C4 cp = c;  // coordinates of x + mu
      const int Lm = extent(d, mu), vm = c.get(mu) + 1 == Lm ? 0 : c.get(mu) + 1;
      cp.x = mu == 0 ? vm : cp.x;
      cp.y = mu == 1 ? vm : cp.y;
      cp.z = mu == 2 ? vm : cp.z;
      cp.t = mu == 3 ? vm : cp.t;
      const M3 ab = dag_mul(ld(U, x_mnu, nu), ld(U, x_mnu, mu));
      mac_mul(S, ab, ld(U, shifted(d, x_pmu, cp, nu, -1), nu));
    }
  }
  const M3 u = ld(U, x, mu);
  double2* f = F + (x * 4 + mu) * 9;
#pragma unroll
  for (int i = 0; i < 9; ++i) f[i] = make_double2(c1 * u.e[i].x + cst * S.e[i].x, c1 * u.e[i].y + cst * S.e[i].y);
  // Naik: c3 U_mu(x) U_mu(x+mu) U_mu(x+2mu)
  const M3 uu = mul(u, ld(U, x_pmu, mu));
  const M3 l3 = mul(uu, ld(U, shifted(d, x, c, mu, 2), mu));
  double2* l = Lk + (x * 4 + mu) * 9;
#pragma unroll
  for (int i = 0; i < 9; ++i) l[i] = make_double2(c3 * l3.e[i].x, c3 * l3.e[i].y);
}

}  // namespace lb
}  // namespace stag

using namespace stag;

extern "C" int stag_build_links(const int dims[4], const void* thin, void* fat, void* lng, double c1, double c_staple,
                                double c3, void* stream) {
  if (!dims || !thin || !fat || !lng) return STAG_EINVAL;
  long long V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 4 || dims[i] % 2) return STAG_EINVAL;
    V *= dims[i];
  }
  const su3::Dims d{dims[0], dims[1], dims[2], dims[3]};
  if (V > (1LL << 31)) return STAG_EINVAL;
  const size_t bytes = (size_t)V * 4 * 9 * sizeof(double2);
  // the outputs may not overlap the input or each other
  auto overlap = [bytes](const void* a, const void* b) {
    const char *p = (const char*)a, *q = (const char*)b;
    return p < q + bytes && q < p + bytes;
  };
  if (overlap(thin, fat) || overlap(thin, lng) || overlap(fat, lng)) return STAG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  ProfScope ps("links", st);
  const long long n = 4 * V;
  lb::k_build_links<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(d, V, (const double2*)thin, (double2*)fat,
                                                                  (double2*)lng, c1, c_staple, c3);
  return last_launch_status();
}
