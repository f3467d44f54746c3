// links.cu -- gauge-field remap: canonical [V][4][3][3] complex double links
// (no phases) -> the internal per-parity hop layout in FP64, double-float
// (FP64 as hi + lo floats), FP32, FP16 or 16-bit fixed point, with the
// staggered phase eta_mu(x), the 1/2 and the sign of the backward hops
// folded in.  The paper notes that remapping from
// the host code's layout to the library's costs about as much as one call of
// the routine and keeps it out of its timings (Sec. 4.2; caption of Fig. 9);
// here it runs once per gauge field, on the GPU.
//
// Layout (per output parity): for each site the 16 hop matrices in the order
//   for mu = 0..3: Wf_mu (9), Wb_mu (9), Nf_mu (NL), Nb_mu (NL)
// (W = fat hops at distance 1, N = Naik hops at distance 3; NL = 9, or 6 for
// two-row storage of the SU(3) part) form one list of complex numbers,
// packed PER to a 16-byte chunk; chunk j of all sites is contiguous,
// [chunk][site], so a warp's 128-bit loads of one chunk are coalesced.
#include <cstring>

#include "internal.h"

namespace stag {

__device__ __forceinline__ void store_c(double2* p, double re, double im) { *p = make_double2(re, im); }
__device__ __forceinline__ void store_c(float2* p, double re, double im) {
  *p = make_float2((float)re, (float)im);
}
__device__ __forceinline__ void store_c(__half2* p, double re, double im) {
  *p = __halves2half2(__double2half(re), __double2half(im));
}
// double-float: {hi.re, hi.im, lo.re, lo.im}, hi the nearest float, lo the
// nearest float to the remainder (about 48 significant bits in all)
__device__ __forceinline__ void store_c(float4* p, double re, double im) {
  const float hre = (float)re, him = (float)im;
  *p = make_float4(hre, him, (float)(re - (double)hre), (float)(im - (double)him));
}
__device__ __forceinline__ void store_c(short2* p, double re, double im) {
  // re, im are normalised to [-1, 1]
  double a = fmin(fmax(rint(re * 32767.0), -32767.0), 32767.0);
  double b = fmin(fmax(rint(im * 32767.0), -32767.0), 32767.0);
  *p = make_short2((short)a, (short)b);
}

__device__ __forceinline__ int lex_of(const Geom& g, int x, int y, int z, int t) {
  return x + g.L[0] * (y + g.L[1] * (z + g.L[2] * t));
}

// Max |re|, |im| over a canonical link array, as the bit pattern of a
// non-negative double (order-preserving as an unsigned integer).
__global__ void k_maxabs(const double* a, long long n, unsigned long long* out) {
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(a[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

template <class S2, int PER, int NL> struct LinkWriter {
  S2* base;  // this parity's array
  int Vh, s;
  __device__ void put(int k, double re, double im) const {
    store_c(base + ((size_t)(k / PER) * Vh + s) * PER + (k % PER), re, im);
  }
};

// One thread per (output parity, checkerboard site).
template <class S2, int PER, int NL>
__global__ void k_load_links(const double2* __restrict__ fat, const double2* __restrict__ lng, Geom g,
                             S2* __restrict__ out, double inv_fat_scale, double inv_long_scale, double inv_c3,
                             int* err) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 2 * g.Vh) return;
  constexpr int CPM = 18 + 2 * NL;
  int p = idx / g.Vh;
  int s = idx - p * g.Vh;
  Coord c = cb_coords(g, s, p);
  int here = lex_of(g, c.x, c.y, c.z, c.t);
  LinkWriter<S2, PER, NL> w{out + (size_t)p * 4 * CPM * g.Vh, g.Vh, s};
  double worst = 0.0;
  for (int mu = 0; mu < 4; ++mu) {
    const int k0 = mu * CPM;
    double h = eta_bit(c, mu) ? -0.5 : 0.5;
    int cm1[4] = {c.x, c.y, c.z, c.t};
    int cm3[4] = {c.x, c.y, c.z, c.t};
    cm1[mu] = wrapc(cm1[mu] - 1, g.L[mu]);
    cm3[mu] = wrapc(cm3[mu] - 3, g.L[mu]);
    int back1 = lex_of(g, cm1[0], cm1[1], cm1[2], cm1[3]);
    int back3 = lex_of(g, cm3[0], cm3[1], cm3[2], cm3[3]);
    const double2* Ff = fat + ((size_t)here * 4 + mu) * 9;
    const double2* Fb = fat + ((size_t)back1 * 4 + mu) * 9;
    const double2* Lf = lng + ((size_t)here * 4 + mu) * 9;
    const double2* Lb = lng + ((size_t)back3 * 4 + mu) * 9;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double2 f = Ff[3 * i + j];
        double2 b = Fb[3 * j + i];  // (F^dag)_ij = conj(F_ji)
        w.put(k0 + 3 * i + j, h * f.x * inv_fat_scale, h * f.y * inv_fat_scale);
        w.put(k0 + 9 + 3 * i + j, -h * b.x * inv_fat_scale, h * b.y * inv_fat_scale);
      }
    if (NL == 9) {
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double2 f = Lf[3 * i + j];
          double2 b = Lb[3 * j + i];
          w.put(k0 + 18 + 3 * i + j, h * f.x * inv_long_scale, h * f.y * inv_long_scale);
          w.put(k0 + 27 + 3 * i + j, -h * b.x * inv_long_scale, h * b.y * inv_long_scale);
        }
    } else {
      // SU(3) parts: Mf = L(x)/c3, Mb = (L(x-3mu)/c3)^dag; rows 0, 1 stored
      double2 mf[9], mb[9];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double2 f = Lf[3 * i + j], b = Lb[3 * j + i];
          mf[3 * i + j] = make_double2(f.x * inv_c3, f.y * inv_c3);
          mb[3 * i + j] = make_double2(b.x * inv_c3, -b.y * inv_c3);
        }
      for (int which = 0; which < 2; ++which) {
        double2* m = which ? mb : mf;
        // row 2 must equal conj(row0 x row1)
        for (int j = 0; j < 3; ++j) {
          int k = (j + 1) % 3, l = (j + 2) % 3;
          double2 a0 = m[k], a1 = m[l], b0 = m[3 + k], b1 = m[3 + l];
          double re = a0.x * b1.x - a0.y * b1.y - (a1.x * b0.x - a1.y * b0.y);
          double im = a0.x * b1.y + a0.y * b1.x - (a1.x * b0.y + a1.y * b0.x);
          worst = fmax(worst, fabs(m[6 + j].x - re));
          worst = fmax(worst, fabs(m[6 + j].y + im));
        }
      }
      for (int e = 0; e < 6; ++e) {
        w.put(k0 + 18 + e, mf[e].x, mf[e].y);
        w.put(k0 + 18 + NL + e, mb[e].x, mb[e].y);
      }
    }
  }
  if (!(worst <= 1e-10)) atomicExch(err, 1);
}

template <class S2, int PER, int NL>
static int run_load(const double2* fat, const double2* lng, const Geom& g, void* out, double ifs, double ils,
                    double ic3, int* err, cudaStream_t st) {
  int n = 2 * g.Vh;
  ProfScope ps("links", st);
  k_load_links<S2, PER, NL><<<(n + 127) / 128, 128, 0, st>>>(fat, lng, g, (S2*)out, ifs, ils, ic3, err);
  return last_launch_status();
}

static double max_abs(const double2* a, long long n_complex, unsigned long long* scratch, cudaStream_t st,
                      int* status) {
  *status = cuda_status(cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), st));
  if (*status) return 0.0;
  {
    ProfScope ps("links", st);
    k_maxabs<<<1216, 256, 0, st>>>((const double*)a, 2 * n_complex, scratch);
  }
  *status = last_launch_status();
  if (*status) return 0.0;
  unsigned long long bits = 0;
  *status = cuda_status(cudaMemcpyAsync(&bits, scratch, sizeof(bits), cudaMemcpyDeviceToHost, st));
  if (!*status) *status = cuda_status(cudaStreamSynchronize(st));
  double v;
  memcpy(&v, &bits, sizeof(v));
  return v;
}

int build_link_copy(stag_lattice_s* lat, int prec, int recon, const double2* fat, const double2* lng,
                    cudaStream_t st) {
  const Geom& g = lat->g;
  LinkCopy& L = lat->links[prec];
  int nl = (prec == STAG_FP64 || prec == STAG_DF64 || recon != 12) ? 9 : 6;
  size_t eb = (prec == STAG_FP64 || prec == STAG_DF64) ? 16 : prec == STAG_FP32 ? 8 : 4;
  size_t bytes = (size_t)2 * 4 * (18 + 2 * nl) * g.Vh * eb;
  if (L.data) cudaFree(L.data);
  L = LinkCopy();
  if (cudaMalloc(&L.data, bytes) != cudaSuccess) {
    cudaGetLastError();
    L.data = nullptr;
    return STAG_ENOMEM;
  }
  L.nl = nl;
  L.elem_bytes = eb;
  L.parity_stride = (size_t)4 * (18 + 2 * nl) * g.Vh * eb;
  int status = 0;
  int* err = (int*)lat->ws.get("links_err", 64, &status);
  if (status) return status;
  if ((status = cuda_status(cudaMemsetAsync(err, 0, 64, st)))) return status;
  double ifs = 1.0, ils = 1.0;
  if (prec == STAG_FP16 || prec == STAG_FX16) {
    // per-field scales so that every stored entry lies in [-1, 1]; the two
    // rows kept for two-row storage are SU(3) entries and need none
    long long nlinks = (long long)2 * g.Vh * 4 * 9;
    double mf = max_abs(fat, nlinks, (unsigned long long*)(err + 4), st, &status);
    if (status) return status;
    double ml = max_abs(lng, nlinks, (unsigned long long*)(err + 4), st, &status);
    if (status) return status;
    L.fat_scale = mf > 0 ? (float)(0.5 * mf) : 1.f;
    L.long_scale = (nl == 9 && ml > 0) ? (float)(0.5 * ml) : 1.f;
    ifs = 1.0 / (double)L.fat_scale;
    ils = 1.0 / (double)L.long_scale;
  }
  double ic3 = 1.0 / lat->c3;
  switch (prec) {
    case STAG_FP64: status = run_load<double2, 1, 9>(fat, lng, g, L.data, ifs, ils, ic3, err, st); break;
    case STAG_DF64: status = run_load<float4, 1, 9>(fat, lng, g, L.data, ifs, ils, ic3, err, st); break;
    case STAG_FP32:
      status = nl == 9 ? run_load<float2, 2, 9>(fat, lng, g, L.data, ifs, ils, ic3, err, st)
                       : run_load<float2, 2, 6>(fat, lng, g, L.data, ifs, ils, ic3, err, st);
      break;
    case STAG_FP16:
      status = nl == 9 ? run_load<__half2, 4, 9>(fat, lng, g, L.data, ifs, ils, ic3, err, st)
                       : run_load<__half2, 4, 6>(fat, lng, g, L.data, ifs, ils, ic3, err, st);
      break;
    default:
      status = nl == 9 ? run_load<short2, 4, 9>(fat, lng, g, L.data, ifs, ils, ic3, err, st)
                       : run_load<short2, 4, 6>(fat, lng, g, L.data, ifs, ils, ic3, err, st);
  }
  if (status) return status;
  int herr = 0;
  if ((status = cuda_status(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st)))) return status;
  if ((status = cuda_status(cudaStreamSynchronize(st)))) return status;
  if (herr) return STAG_ENOTUNITARY;
  L.present = true;
  return STAG_OK;
}

}  // namespace stag
