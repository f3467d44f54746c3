// df.cuh -- FP64-class arithmetic on the FP32 pipes ("double-float").
//
// A real number is carried as the unevaluated sum hi + lo of two floats
// (about 48 significant bits); a complex number as a float4 {hi.re, hi.im,
// lo.re, lo.im}, 16 bytes like a complex double.  GB300 runs FP64 at a small
// fraction of its FP32 rate (about 1.1 TFLOP/s against some 80), so the
// FP64-accurate operator of the reliable updates (the true residual
// b - M y of the mixed-precision solvers) computes in this format:
// every product of two hi parts is split exactly into p + e with one FMA
// (TwoProd) and added to the accumulator's hi part with Knuth's TwoSum, whose
// exact rounding error joins the lo part together with e and the cross
// products hi*lo + lo*hi (the lo*lo product lies below the format's
// precision).  These are the error-free transformations of Ogita, Rump and
// Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005),
// the same ones the FP64-class reductions of common.cuh use.  The _rn
// intrinsics keep the compiler from contracting the sums into FMAs, which
// would break the transformations.
#pragma once
#include "common.cuh"

namespace stag {

// Split of a double into hi + lo floats with integer operations only (no
// FP64 instruction): hi keeps the sign, the exponent and the leading 23
// fraction bits (truncated), lo the remaining 29 fraction bits rounded to a
// float, so |d - (hi + lo)| <= 2^-48 |d|.  |d| < 2^-126 becomes 0 (absolute
// error below 1e-38); non-finite input gives a NaN hi, so that the solvers'
// finiteness checks still see it.
__device__ __forceinline__ float2 df_split(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned h = (unsigned)(u >> 32);
  const unsigned sign = h & 0x80000000u;
  const int e = (int)((h >> 20) & 0x7ffu);  // biased by 1023
  if (e >= 1151) return make_float2(__int_as_float(0x7fc00000), 0.f);  // |d| >= 2^128, Inf, NaN
  if (e <= 896) return make_float2(0.f, 0.f);
  const unsigned top = (unsigned)(u >> 29) & 0x7fffffu;  // fraction bits 51..29
  const unsigned low = (unsigned)u & 0x1fffffffu;        // fraction bits 28..0
  const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | top);
  float lo = 0.f;
  if (e > 948) {  // low * 2^(e - 1075), a normal float scale 2^(e - 1075)
    lo = __fmul_rn(__uint2float_rn(low), __uint_as_float((unsigned)(e - 948) << 23));
    lo = __uint_as_float(__float_as_uint(lo) | sign);
  }
  return make_float2(hi, lo);
}

// hi + lo += a * b: TwoProd by FMA, TwoSum into hi, both errors into lo.
__device__ __forceinline__ void df_mac(float& hi, float& lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float v = __fadd_rn(s, -hi);
  const float err = __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -v)), __fadd_rn(p, -v));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}

// hi + lo += a (a float): TwoSum.
__device__ __forceinline__ void df_add(float& hi, float& lo, float a) {
  const float s = __fadd_rn(hi, a);
  const float v = __fadd_rn(s, -hi);
  const float err = __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -v)), __fadd_rn(a, -v));
  hi = s;
  lo = __fadd_rn(lo, err);
}

// acc += w * v, complex double-float.
__device__ __forceinline__ void dfc_mac(float4& acc, const float4& w, const float4& v) {
  df_mac(acc.x, acc.z, w.x, v.x);
  df_mac(acc.x, acc.z, -w.y, v.y);
  df_mac(acc.y, acc.w, w.x, v.y);
  df_mac(acc.y, acc.w, w.y, v.x);
  acc.z = fmaf(w.x, v.z, acc.z);
  acc.z = fmaf(w.z, v.x, acc.z);
  acc.z = fmaf(-w.y, v.w, acc.z);
  acc.z = fmaf(-w.w, v.y, acc.z);
  acc.w = fmaf(w.x, v.w, acc.w);
  acc.w = fmaf(w.z, v.y, acc.w);
  acc.w = fmaf(w.y, v.z, acc.w);
  acc.w = fmaf(w.w, v.x, acc.w);
}

// acc += a * v, a a real double-float scalar (a.x = hi, a.y = lo).
__device__ __forceinline__ void dfc_axpy(float4& acc, float2 a, const float4& v) {
  df_mac(acc.x, acc.z, a.x, v.x);
  df_mac(acc.y, acc.w, a.x, v.y);
  acc.z = fmaf(a.x, v.z, acc.z);
  acc.z = fmaf(a.y, v.x, acc.z);
  acc.w = fmaf(a.x, v.w, acc.w);
  acc.w = fmaf(a.y, v.y, acc.w);
}

// acc += v (exact sign change for s = -1).
__device__ __forceinline__ void dfc_add(float4& acc, const float4& v, bool negate) {
  const float sx = negate ? -v.x : v.x, sy = negate ? -v.y : v.y;
  df_add(acc.x, acc.z, sx);
  df_add(acc.y, acc.w, sy);
  acc.z = __fadd_rn(acc.z, negate ? -v.z : v.z);
  acc.w = __fadd_rn(acc.w, negate ? -v.w : v.w);
}

// Renormalised form (|lo| at most half an ulp of hi) of hi + lo.
__device__ __forceinline__ float4 dfc_norm(const float4& a) {
  float4 r;
  r.x = __fadd_rn(a.x, a.z);
  r.z = __fadd_rn(a.z, -__fadd_rn(r.x, -a.x));
  r.y = __fadd_rn(a.y, a.w);
  r.w = __fadd_rn(a.w, -__fadd_rn(r.y, -a.y));
  // Fast2Sum above needs |hi| >= |lo|; where the lo part dominates (heavy
  // cancellation in the hi part) fall back to the exact TwoSum
  if (fabsf(a.z) > fabsf(a.x)) {
    float h = a.z, l = 0.f;
    df_add(h, l, a.x);
    r.x = h;
    r.z = l;
  }
  if (fabsf(a.w) > fabsf(a.y)) {
    float h = a.w, l = 0.f;
    df_add(h, l, a.y);
    r.y = h;
    r.w = l;
  }
  return r;
}

__device__ __forceinline__ float4 dfc_from_double2(double2 v) {
  const float2 a = df_split(v.x), b = df_split(v.y);
  return make_float4(a.x, b.x, a.y, b.y);
}

// The double nearest hi + lo (two exact widenings and one FP64 addition:
// used only when results leave the library).
__device__ __forceinline__ double2 dfc_to_double2(const float4& v) {
  return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}

// The float nearest hi + lo.
__device__ __forceinline__ float2 dfc_to_float2(const float4& v) {
  return make_float2(__fadd_rn(v.x, v.z), __fadd_rn(v.y, v.w));
}

// A single-parity field in double-float: [Vh][3] float4, n systems one after
// the other (the layout of the FP64 fields, 48 bytes per site and system).
struct DfField {
  float4* v;
  int Vh;
};
__host__ __device__ inline size_t df_bytes(int Vh) { return (size_t)Vh * 48; }

}  // namespace stag
