// su3.cuh -- FP64 3x3 complex matrix products and periodic site stepping on
// the canonical lex layout, shared by the link construction, the gauge force
// and the fermion force kernels.
#pragma once
#include "internal.h"

namespace stag {
namespace su3 {

struct M3 {
  double2 e[9];
};

__device__ __forceinline__ M3 ld(const double2* __restrict__ U, long long site, int mu) {
  M3 m;
  const double2* p = U + (site * 4 + mu) * 9;
#pragma unroll
  for (int i = 0; i < 9; ++i) m.e[i] = __ldg(p + i);
  return m;
}

// a b
__device__ __forceinline__ M3 mul(const M3& a, const M3& b) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac(s, a.e[3 * i + k], b.e[3 * k + j]);
      r.e[3 * i + j] = s;
    }
  return r;
}

// acc += a b^dag
__device__ __forceinline__ void mac_mul_dag(M3& acc, const M3& a, const M3& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        // a_ik conj(b_jk)
        const double2 x = a.e[3 * i + k], y = b.e[3 * j + k];
        acc.e[3 * i + j].x = fma(x.x, y.x, fma(x.y, y.y, acc.e[3 * i + j].x));
        acc.e[3 * i + j].y = fma(x.y, y.x, fma(-x.x, y.y, acc.e[3 * i + j].y));
      }
}

// a^dag b
__device__ __forceinline__ M3 dag_mul(const M3& a, const M3& b) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double2 s = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        // conj(a_ki) b_kj
        const double2 x = a.e[3 * k + i], y = b.e[3 * k + j];
        s.x = fma(x.x, y.x, fma(x.y, y.y, s.x));
        s.y = fma(x.x, y.y, fma(-x.y, y.x, s.y));
      }
      r.e[3 * i + j] = s;
    }
  return r;
}

// acc += a b
__device__ __forceinline__ void mac_mul(M3& acc, const M3& a, const M3& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac(acc.e[3 * i + j], a.e[3 * i + k], b.e[3 * k + j]);
}

// acc += a^dag b
__device__ __forceinline__ void mac_dag_mul(M3& acc, const M3& a, const M3& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        // conj(a_ki) b_kj
        const double2 x = a.e[3 * k + i], y = b.e[3 * k + j];
        acc.e[3 * i + j].x = fma(x.x, y.x, fma(x.y, y.y, acc.e[3 * i + j].x));
        acc.e[3 * i + j].y = fma(x.x, y.y, fma(-x.y, y.x, acc.e[3 * i + j].y));
      }
}

// acc += a^dag b^dag = acc + (b a)^dag
__device__ __forceinline__ void mac_dag_mul_dag(M3& acc, const M3& a, const M3& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        // conj(a_ki) conj(b_jk) = conj(a_ki b_jk)
        const double2 x = a.e[3 * k + i], y = b.e[3 * j + k];
        acc.e[3 * i + j].x = fma(x.x, y.x, fma(-x.y, y.y, acc.e[3 * i + j].x));
        acc.e[3 * i + j].y = fma(-x.x, y.y, fma(-x.y, y.x, acc.e[3 * i + j].y));
      }
}

__device__ __forceinline__ M3 zero3() {
  M3 r;
#pragma unroll
  for (int i = 0; i < 9; ++i) r.e[i] = make_double2(0.0, 0.0);
  return r;
}

__device__ __forceinline__ void scale3(M3& a, double c) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    a.e[i].x *= c;
    a.e[i].y *= c;
  }
}

struct Dims {
  int L0, L1, L2, L3;
};

// Site coordinates as four scalars; component mu selected without an array
// (a runtime-indexed local array would live in local memory).
struct C4 {
  int x, y, z, t;
  __device__ __forceinline__ int get(int mu) const { return mu == 0 ? x : mu == 1 ? y : mu == 2 ? z : t; }
};

__device__ __forceinline__ int extent(const Dims& d, int mu) {
  return mu == 0 ? d.L0 : mu == 1 ? d.L1 : mu == 2 ? d.L2 : d.L3;
}
__device__ __forceinline__ long long stride(const Dims& d, int mu) {
  return mu == 0 ? 1LL : mu == 1 ? (long long)d.L0 : mu == 2 ? (long long)d.L0 * d.L1 : (long long)d.L0 * d.L1 * d.L2;
}

// lex index of the site with coordinates c (lex index x) moved by k along mu (periodic)
__device__ __forceinline__ long long shifted(const Dims& d, long long x, const C4& c, int mu, int k) {
  const int L = extent(d, mu), v = c.get(mu);
  int w = v + k;
  w = w >= L ? w - L : (w < 0 ? w + L : w);
  return x + stride(d, mu) * (long long)(w - v);
}

// A site as its lex index and coordinates, moved along one direction at a time.
struct Pos {
  long long lex;
  C4 c;
};

__device__ __forceinline__ Pos pos_of(const Dims& d, long long x) {
  Pos p;
  p.lex = x;
  long long r = x;
  p.c.x = (int)(r % d.L0);
  r /= d.L0;
  p.c.y = (int)(r % d.L1);
  r /= d.L1;
  p.c.z = (int)(r % d.L2);
  p.c.t = (int)(r / d.L2);
  return p;
}

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

}  // namespace su3
}  // namespace stag
