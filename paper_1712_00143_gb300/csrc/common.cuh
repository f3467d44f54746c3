// common.cuh -- shared device definitions of libstag: lattice geometry on a
// checkerboard, complex helpers, storage precisions, deterministic FP64 grid
// reductions and the solver scalar state they finalise.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace stag {

// ------------------------------------------------------------------ bounds-checked build
// Built with -DSTAG_DEBUG_BOUNDS (libstag_debug.so), the index computations
// that address global memory -- every neighbour index of the stencil, every
// site index of a vector load or store, the site index of every link load --
// are checked against their extent; a violation is counted in a device word
// (with the first one's code and index) and the access goes to index 0
// instead, so the kernel completes and the host reads the record
// (stag_bounds_violations).  Every translation unit has its own record,
// registered with the host at load time.  The normal build compiles the
// checks away.
#ifdef STAG_DEBUG_BOUNDS
void bounds_register(int (*read)(unsigned long long*), int (*clear)());
namespace {
__device__ unsigned long long g_bounds[3];  // violations, first code, first index
__device__ __forceinline__ long long bounds_check(long long idx, long long n, int code) {
  if (idx >= 0 && idx < n) return idx;
  if (atomicAdd(&g_bounds[0], 1ull) == 0ull) {
    g_bounds[1] = (unsigned long long)code;
    g_bounds[2] = (unsigned long long)idx;
  }
  return 0;
}
inline int bounds_read_tu(unsigned long long* v) {
  return cudaMemcpyFromSymbol(v, g_bounds, sizeof(g_bounds)) == cudaSuccess ? 0 : 1;
}
inline int bounds_clear_tu() {
  const unsigned long long z[3] = {0ull, 0ull, 0ull};
  return cudaMemcpyToSymbol(g_bounds, z, sizeof(z)) == cudaSuccess ? 0 : 1;
}
struct BoundsReg {
  BoundsReg() { bounds_register(&bounds_read_tu, &bounds_clear_tu); }
} g_bounds_reg;
}  // namespace
#define STAG_BOUND(idx, n, code) ((int)::stag::bounds_check((long long)(idx), (long long)(n), (code)))
#else
#define STAG_BOUND(idx, n, code) (idx)
#endif
// codes of the checked index kinds
enum BoundCode : int { BOUND_NEIGHBOUR = 1, BOUND_VECTOR = 2, BOUND_LINK = 3 };

// ------------------------------------------------------------------ geometry
// Checkerboard (single-parity) index s of a site = lex/2, lex = x + Lx*(y +
// Ly*(z + Lz*t)).  With Lx even, s = x/2 + Lxh*(y + Ly*(z + Lz*t)), so a
// step along y, z, t moves s by a fixed stride and x is rebuilt from the
// parity of the site.
struct Geom {
  int L[4];  // Lx, Ly, Lz, Lt (even, >= 4)
  int Lxh;   // Lx / 2
  int Vh;    // sites per parity
  int sy, sz, st;  // checkerboard strides of y, z, t
  // exact division by Lxh, Ly, Lz as a multiply and a shift:
  // n / d = (n * m) >> s for 0 <= n <= 2^30 (see magic_div)
  unsigned long long m_xh, m_y, m_z;
  int s_xh, s_y, s_z;
};

// Multiplier and shift for division by d >= 1: with l = ceil(log2 d),
// s = 31 + l and m = ceil(2^s / d), m d = 2^s + e (0 <= e < d), so
// n m / 2^s = n / d + n e / (d 2^s) and the second term is below 1/d for
// n < 2^31: the floor is exact.  n m < 2^30 (2^32 + 1) fits in 64 bits.
__host__ __device__ inline void magic_div(int d, unsigned long long& m, int& s) {
  int l = 0;
  while ((1 << l) < d) ++l;
  s = 31 + l;
  m = ((1ull << s) + (unsigned long long)d - 1) / (unsigned long long)d;
}

__host__ __device__ __forceinline__ int mdiv(int n, unsigned long long m, int s) {
  return (int)(((unsigned long long)(unsigned)n * m) >> s);
}

struct Coord {
  int x, y, z, t;
};

__host__ __device__ inline Geom make_geom(const int d[4]) {
  Geom g;
  for (int i = 0; i < 4; ++i) g.L[i] = d[i];
  g.Lxh = d[0] / 2;
  g.sy = g.Lxh;
  g.sz = g.Lxh * d[1];
  g.st = g.Lxh * d[1] * d[2];
  g.Vh = g.st * d[3];
  magic_div(g.Lxh, g.m_xh, g.s_xh);
  magic_div(d[1], g.m_y, g.s_y);
  magic_div(d[2], g.m_z, g.s_z);
  return g;
}

__device__ __forceinline__ Coord cb_coords(const Geom& g, int s, int parity) {
  const int q1 = mdiv(s, g.m_xh, g.s_xh);  // s / Lxh
  const int xh = s - q1 * g.Lxh;
  const int q2 = mdiv(q1, g.m_y, g.s_y);   // / Ly
  Coord c;
  c.y = q1 - q2 * g.L[1];
  c.t = mdiv(q2, g.m_z, g.s_z);            // / Lz
  c.z = q2 - c.t * g.L[2];
  c.x = 2 * xh + ((parity + c.y + c.z + c.t) & 1);
  return c;
}

__device__ __forceinline__ int wrapc(int v, int L) { return v < 0 ? v + L : (v >= L ? v - L : v); }

// Checkerboard index of the site c + k*mu (k in {-3,-1,1,3}); s is c's own index.
__device__ __forceinline__ int cb_neighbour_raw(const Geom& g, int s, const Coord& c, int mu, int k) {
  switch (mu) {
    case 0: return s - (c.x >> 1) + (wrapc(c.x + k, g.L[0]) >> 1);
    case 1: return s + (wrapc(c.y + k, g.L[1]) - c.y) * g.sy;
    case 2: return s + (wrapc(c.z + k, g.L[2]) - c.z) * g.sz;
    default: return s + (wrapc(c.t + k, g.L[3]) - c.t) * g.st;
  }
}
__device__ __forceinline__ int cb_neighbour(const Geom& g, int s, const Coord& c, int mu, int k) {
  return STAG_BOUND(cb_neighbour_raw(g, s, c, mu, k), g.Vh, BOUND_NEIGHBOUR);
}

// Staggered phase eta_mu(x) as a sign bit: 1 means -1.
__device__ __forceinline__ int eta_bit(const Coord& c, int mu) {
  int e = (mu == 0) ? 0 : (mu == 1) ? c.x : (mu == 2) ? c.x + c.y : c.x + c.y + c.z;
  return e & 1;
}

// ------------------------------------------------------------------ complex
template <class R> struct C2;
template <> struct C2<double> { using T = double2; };
template <> struct C2<float> { using T = float2; };

template <class T2> __device__ __forceinline__ T2 mk(decltype(T2::x) a, decltype(T2::x) b) {
  T2 r;
  r.x = a;
  r.y = b;
  return r;
}

// acc += a * b
template <class T2> __device__ __forceinline__ void cmac(T2& acc, T2 a, T2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <class T2> __device__ __forceinline__ void cmac_conj(T2& acc, T2 a, T2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

// ------------------------------------------------------------------ precision
// Storage formats, by tag P:
//   64: FP64 (double2 per complex)          32: FP32 (float2)
//   16: IEEE binary16 (__half2)             15: 16-bit fixed point (short2,
//       15 fraction bits), values in units of a per-site or per-field scale.
// Arithmetic is FP64 for P = 64 and FP32 otherwise.
template <int P> struct Prec;
template <> struct Prec<64> {
  using S2 = double2;
  using A = double;
  using A2 = double2;
};
template <> struct Prec<32> {
  using S2 = float2;
  using A = float;
  using A2 = float2;
};
template <> struct Prec<16> {
  using S2 = __half2;
  using A = float;
  using A2 = float2;
};
template <> struct Prec<15> {
  using S2 = short2;
  using A = float;
  using A2 = float2;
};

// Tag 31: 16-bit fixed-point links (the storage of tag 15) with FP32 vectors
// and arithmetic (those of tag 32): the link bytes, the bulk of a multi-RHS
// operator's traffic, halve while the vectors keep single precision.
template <> struct Prec<31> : Prec<32> {};

// Links stored as 16-bit fixed point (integers in units of a per-field scale).
__host__ __device__ constexpr bool fixed_links(int p) { return p == 15 || p == 31; }

constexpr float FX_ONE = 32767.0f;  // fixed-point full scale

// ---- 16-byte link chunks: complex numbers packed PER to a 16-byte word so
// that every link load is a 128-bit load.  get() returns the stored value as
// a normalised number (binary16: in [-1, 1]; fixed point: the integer), to be
// multiplied by the field's scale.
template <int P> struct Chunk;
template <> struct Chunk<64> {
  static constexpr int PER = 1;
  static __device__ __forceinline__ double2 get(const uint4& c, int) {
    return make_double2(__hiloint2double(c.y, c.x), __hiloint2double(c.w, c.z));
  }
};
template <> struct Chunk<32> {
  static constexpr int PER = 2;
  static __device__ __forceinline__ float2 get(const uint4& c, int lane) {
    return lane == 0 ? make_float2(__uint_as_float(c.x), __uint_as_float(c.y))
                     : make_float2(__uint_as_float(c.z), __uint_as_float(c.w));
  }
};
__device__ __forceinline__ unsigned word_of(const uint4& c, int lane) {
  return lane == 0 ? c.x : lane == 1 ? c.y : lane == 2 ? c.z : c.w;
}
__device__ __forceinline__ float2 half2_bits_to_float2(unsigned w) {
  __half2_raw r;
  r.x = (unsigned short)(w & 0xffffu);
  r.y = (unsigned short)(w >> 16);
  return __half22float2(__half2(r));
}
// Two signed 16-bit integers (one 32-bit word) to floats without the
// quarter-rate integer-to-float conversion: each half, biased by 2^15 (the
// XOR), is placed in the low mantissa bits of 1.5 * 2^23, giving the exact
// float 1.5 * 2^23 + 2^15 + q; one FP32 subtraction then yields q.
__device__ __forceinline__ float2 short2_bits_to_float2(unsigned w) {
  const unsigned b = w ^ 0x80008000u;
  const float lo = __uint_as_float(__byte_perm(b, 0x4B40u, 0x5410));
  const float hi = __uint_as_float(__byte_perm(b, 0x4B40u, 0x5432));
  return make_float2(__fadd_rn(lo, -12615680.0f), __fadd_rn(hi, -12615680.0f));
}
template <> struct Chunk<16> {
  static constexpr int PER = 4;
  static __device__ __forceinline__ float2 get(const uint4& c, int lane) {
    return half2_bits_to_float2(word_of(c, lane));
  }
};
// Fixed point: get() returns the stored integer (as an exact float); the
// 1/32767 joins the per-field scale applied after the hop sums.
template <> struct Chunk<15> {
  static constexpr int PER = 4;
  static __device__ __forceinline__ float2 get(const uint4& c, int lane) {
    return short2_bits_to_float2(word_of(c, lane));
  }
};
template <> struct Chunk<31> : Chunk<15> {};

// A single-parity colour-vector field in the internal layout:
//   P = 64: [Vh][3] double2 (array of structures, the canonical layout)
//   P = 32: [3][Vh] float2  (structure of arrays)
//   P = 16, 15: [Vh] 16-byte records {c0, c1, c2, scale}: three complex in
//           16-bit storage and one FP32 per-site scale, so that a
//           neighbour gather is a single 128-bit load.
// ld() uses the read-only path (fields not written by the same kernel),
// ldw() plain loads (fields the kernel also writes).
template <int P> struct Spinor {
  void* v;
  int Vh;
};

template <int P> __host__ __device__ inline size_t spinor_bytes(int Vh) {
  return P == 64 ? (size_t)Vh * 48 : (P == 32 || P == 31) ? (size_t)Vh * 24 : (size_t)Vh * 16;
}

template <int P> struct SpinorLoad;
template <> struct SpinorLoad<64> {
  static __device__ __forceinline__ void ld(const Spinor<64>& f, int s, double2 o[3]) {
    s = STAG_BOUND(s, f.Vh, BOUND_VECTOR);
    const double2* p = (const double2*)f.v + 3 * (size_t)s;
#pragma unroll
    for (int c = 0; c < 3; ++c) o[c] = __ldg(p + c);
  }
  static __device__ __forceinline__ void ldw(const Spinor<64>& f, int s, double2 o[3]) {
    s = STAG_BOUND(s, f.Vh, BOUND_VECTOR);
    const double2* p = (const double2*)f.v + 3 * (size_t)s;
#pragma unroll
    for (int c = 0; c < 3; ++c) o[c] = p[c];
  }
  static __device__ __forceinline__ void st(const Spinor<64>& f, int s, const double2 o[3]) {
    s = STAG_BOUND(s, f.Vh, BOUND_VECTOR);
    double2* p = (double2*)f.v + 3 * (size_t)s;
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c] = o[c];
  }
};
template <> struct SpinorLoad<32> {
  static __device__ __forceinline__ void ld(const Spinor<32>& f, int s, float2 o[3]) {
    s = STAG_BOUND(s, f.Vh, BOUND_VECTOR);
    const float2* p = (const float2*)f.v;
#pragma unroll
    for (int c = 0; c < 3; ++c) o[c] = __ldg(p + c * (size_t)f.Vh + s);
  }
  static __device__ __forceinline__ void ldw(const Spinor<32>& f, int s, float2 o[3]) {
    s = STAG_BOUND(s, f.Vh, BOUND_VECTOR);
    const float2* p = (const float2*)f.v;
#pragma unroll
    for (int c = 0; c < 3; ++c) o[c] = p[c * (size_t)f.Vh + s];
  }
  static __device__ __forceinline__ void st(const Spinor<32>& f, int s, const float2 o[3]) {
    s = STAG_BOUND(s, f.Vh, BOUND_VECTOR);
    float2* p = (float2*)f.v;
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c * (size_t)f.Vh + s] = o[c];
  }
};

// FP32 vectors of the fixed-point-link format (tag 31)
template <> struct SpinorLoad<31> {
  static __device__ __forceinline__ Spinor<32> as32(const Spinor<31>& f) { return Spinor<32>{f.v, f.Vh}; }
  static __device__ __forceinline__ void ld(const Spinor<31>& f, int s, float2 o[3]) { SpinorLoad<32>::ld(as32(f), s, o); }
  static __device__ __forceinline__ void ldw(const Spinor<31>& f, int s, float2 o[3]) {
    SpinorLoad<32>::ldw(as32(f), s, o);
  }
  static __device__ __forceinline__ void st(const Spinor<31>& f, int s, const float2 o[3]) {
    SpinorLoad<32>::st(as32(f), s, o);
  }
};

// L2 prefetch of one site's vector (no registers): issued at the start of a
// kernel whose epilogue reads the vector only after a long computation.
template <int P> __device__ __forceinline__ void prefetch_spinor_l2(const Spinor<P>& f, int s) {
  if constexpr (P == 32 || P == 31) {
    const float2* p = (const float2*)f.v;
#pragma unroll
    for (int c = 0; c < 3; ++c) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + c * (size_t)f.Vh + s));
  } else if constexpr (P == 64) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"((const double2*)f.v + 3 * (size_t)s));
  } else {
    asm volatile("prefetch.global.L2 [%0];" ::"l"((const uint4*)f.v + s));
  }
}

// 16-bit records.  FP16: components stored as value/max (round to nearest
// even), scale = max.  Fixed point: components stored as round(value/max *
// 32767), scale = max/32767.  max = largest |re|, |im| of the site.
template <int P> struct SpinorLoad16 {
  static __device__ __forceinline__ void unpack(const uint4& r, float2 o[3]) {
    const float k = __uint_as_float(r.w);
    float2 a = P == 16 ? half2_bits_to_float2(r.x) : short2_bits_to_float2(r.x);
    float2 b = P == 16 ? half2_bits_to_float2(r.y) : short2_bits_to_float2(r.y);
    float2 c = P == 16 ? half2_bits_to_float2(r.z) : short2_bits_to_float2(r.z);
    o[0] = make_float2(a.x * k, a.y * k);
    o[1] = make_float2(b.x * k, b.y * k);
    o[2] = make_float2(c.x * k, c.y * k);
  }
  static __device__ __forceinline__ void ld(const Spinor<P>& f, int s, float2 o[3]) {
    unpack(__ldg((const uint4*)f.v + STAG_BOUND(s, f.Vh, BOUND_VECTOR)), o);
  }
  static __device__ __forceinline__ void ldw(const Spinor<P>& f, int s, float2 o[3]) {
    unpack(((const uint4*)f.v)[STAG_BOUND(s, f.Vh, BOUND_VECTOR)], o);
  }
  static __device__ __forceinline__ unsigned pack2(float x, float y) {
    if (P == 16) {
      __half2_raw r = (__half2_raw)__floats2half2_rn(x, y);
      return (unsigned)r.x | ((unsigned)r.y << 16);
    } else {
      int a = __float2int_rn(x), b = __float2int_rn(y);
      a = max(-32767, min(32767, a));
      b = max(-32767, min(32767, b));
      return (unsigned)(unsigned short)(short)a | ((unsigned)(unsigned short)(short)b << 16);
    }
  }
  static __device__ __forceinline__ void st(const Spinor<P>& f, int s, const float2 o[3]) {
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) m = fmaxf(m, fmaxf(fabsf(o[c].x), fabsf(o[c].y)));
    const float full = P == 16 ? 1.0f : FX_ONE;
    const float inv = m > 0.f ? full / m : 0.f;
    uint4 r;
    r.x = pack2(o[0].x * inv, o[0].y * inv);
    r.y = pack2(o[1].x * inv, o[1].y * inv);
    r.z = pack2(o[2].x * inv, o[2].y * inv);
    r.w = __float_as_uint(m / full);
    ((uint4*)f.v)[STAG_BOUND(s, f.Vh, BOUND_VECTOR)] = r;
  }
};
template <> struct SpinorLoad<16> : SpinorLoad16<16> {};
template <> struct SpinorLoad<15> : SpinorLoad16<15> {};

// ------------------------------------------------------------------ solver state
enum StateFlags : int {
  F_CONVERGED = 1,  // iterated residual reached the target
  F_BREAKDOWN = 2,  // NaN/Inf or <p,Ap> <= 0
  F_NEED_RU = 4,    // reliable-update trigger
  F_ITER_CAP = 8,   // max_iter reached
  // Krylov-loop kernels queued after any of these return at once; the host
  // then performs the reliable update (or stops) at the end of the chunk, so
  // an update happens at the iteration that triggered it
  F_STOP = F_CONVERGED | F_BREAKDOWN | F_ITER_CAP | F_NEED_RU,
};

// Scalars of one CG solve, resident in device memory and updated by the
// last block of each reduction (no host round trip per iteration).
struct CgState {
  double rr;       // iterated ||r||^2
  double rr_prev;  // ||r||^2 of the previous iteration
  double pAp, alpha, beta;
  double target;   // tol^2 ||b||^2
  double rr_max;   // max ||r||^2 since the last reliable update
  double delta2;   // delta^2; 0 disables the reliable-update trigger
  double rr_true;  // last FP64 true ||r||^2
  double ortho_re, ortho_im;  // <r,p>/||r||^2 used to re-orthogonalise p
  double shift;    // m^2 + sigma of this system
  int iter, max_iter;
  int flags;
  int reliable_updates;
};

constexpr int MAX_SHIFTS = 32;
// Scalars of a multi-shift solve: the base system's CG scalars plus the
// per-shift zeta / alpha / beta recurrences.
struct MsState {
  CgState cg;       // base system (smallest shift)
  int nshift;
  int active_mask;  // bit s set while shift s still iterates
  int stop_mask;    // shifts that reached their target in the last iteration
  double sqrt_target_bb;  // tol * ||b||
  double alpha_prev, beta_prev;
  double delta[MAX_SHIFTS];      // sigma_s - sigma_0
  double zeta_prev[MAX_SHIFTS];  // zeta_s(k-1)
  double zeta[MAX_SHIFTS];       // zeta_s(k)
  double zeta_next[MAX_SHIFTS];  // zeta_s(k+1)
  double alpha_s[MAX_SHIFTS];
  double beta_s[MAX_SHIFTS];
  int iters[MAX_SHIFTS];
};

constexpr int MAX_RHS = 8;
// Scalars of a group of up to MAX_RHS CG systems that share one lattice (and
// one multi-right-hand-side Dslash): per-system recurrences plus group flags.
// A system whose iterated residual reaches its target leaves the active set
// (its alpha and beta become 0, so its vectors stop changing); the group stops
// for a reliable update when any active system triggers one.
struct McgState {
  int n;
  int active;  // bit i: system i still iterates
  int flags;   // group flags (F_*): CONVERGED = no active system left
  int iter, max_iter;
  int reliable_updates;
  CgState sys[MAX_RHS];
  // control of the graph-resident solve loop (several groups)
  int done;       // 1: the group needs no more work (converged, or ended by an error)
  int status;     // STAG_OK or the error that ended the group
  int ru_skip;    // F_CONVERGED while no reliable update is due (a stop word for its kernels), else 0
  int skip_xpay;  // 1: the next direction update must not run (after the start or an update)
  // double-float reliable updates measure r = r_a - M (y - y_a) from an
  // anchor (y_a, r_a = b - M y_a); the anchor starts at (0, b) and is moved
  // once, by an FP64 update, when every active system's iterated ||r||^2
  // has fallen below anchor_rr[i] (the FP64-class accuracy of the residual
  // then no longer depends on the size of y)
  int use_df;     // 1: updates in double-float (ru_skip gates them), FP64 anchor gated by ru_skip64
  int anchored;   // the anchor has been moved
  int ru_skip64;  // stop word of the FP64 anchor update (graph-resident loop)
  double anchor_rr[MAX_RHS];
};

enum RedOp : int {
  RED_STORE = 0,      // out[0..NV) = totals
  RED_CG_ALPHA = 1,   // pAp -> alpha
  RED_CG_BETA = 2,    // ||r||^2 -> beta, flags
  RED_RU_RESID = 3,   // true ||r||^2 after a reliable update
  RED_RU_ORTHO = 4,   // <r,p> (re, im) -> ortho coefficient
  RED_MS_ALPHA = 5,   // base pAp -> alpha and per-shift zeta, alpha_s
  RED_MS_BETA = 6,    // ||r||^2 -> beta, per-shift beta_s, shift stopping
  RED_MCG_ALPHA = 7,  // per-system pAp -> alpha (McgState)
  RED_MCG_BETA = 8,   // per-system ||r||^2 -> beta, activity, group flags
  RED_MCG_RU_RESID = 9,  // per-system true ||r||^2 after a reliable update
  RED_MCG_RU_ORTHO = 10, // per-system <r,p> (re, im pairs)
  RED_RU_BOTH = 11,      // true ||r||^2, then <r,p> (re, im): RU_RESID followed by RU_ORTHO
  RED_MCG_RU_BOTH = 12,  // per-system true ||r||^2 (n values), then <r,p> pairs (2n values)
};

struct RedTarget {
  int op;
  void* state;   // CgState* or MsState*
  double* out;   // RED_STORE destination
};

struct RedBuf {
  double* partials;   // [NV][gridDim.x]
  unsigned* counter;  // zero between reductions
};

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

__device__ inline void cg_beta_update(CgState* st, double rr_new) {
  if (!finite_d(rr_new)) {
    st->flags |= F_BREAKDOWN;
    return;
  }
  st->beta = rr_new / st->rr;
  st->rr_prev = st->rr;
  st->rr = rr_new;
  st->iter += 1;
  if (rr_new > st->rr_max) st->rr_max = rr_new;
  if (rr_new <= st->target) st->flags |= F_CONVERGED;
  if (st->delta2 > 0.0 && rr_new < st->delta2 * st->rr_max) st->flags |= F_NEED_RU;
  if (st->iter >= st->max_iter) st->flags |= F_ITER_CAP;
}

// Reliable update, single system: the FP64-class true ||r||^2 restarts the
// recurrence (beta, rr, rr_max) ...
__device__ inline void fin_ru_resid(CgState* st, double rr) {
  st->rr_true = rr;
  if (!finite_d(rr)) {
    st->flags |= F_BREAKDOWN;
    return;
  }
  st->beta = rr / st->rr_prev;
  st->rr = rr;
  st->rr_max = rr;
  st->reliable_updates += 1;
  st->flags &= ~(F_CONVERGED | F_NEED_RU);
}
// ... and <r,p>/||r||^2 (v = re, im) re-orthogonalises the search direction.
__device__ inline void fin_ru_ortho(CgState* st, const double* v) {
  st->ortho_re = st->rr > 0.0 ? v[0] / st->rr : 0.0;
  st->ortho_im = st->rr > 0.0 ? v[1] / st->rr : 0.0;
}
// The same for every system of a group (v: n norms; then n (re, im) pairs).
__device__ inline void fin_mcg_ru_resid(McgState* g, const double* v) {
  int active = 0;
  for (int i = 0; i < g->n; ++i) {
    CgState* st = &g->sys[i];
    const double rr = v[i];
    st->rr_true = rr;
    if (!finite_d(rr)) {
      g->flags |= F_BREAKDOWN;
      continue;
    }
    st->beta = st->rr_prev > 0.0 ? rr / st->rr_prev : 0.0;
    st->rr = rr;
    st->rr_max = rr;
    if (rr > st->target) active |= 1 << i;
  }
  g->active = active;
  g->reliable_updates += 1;
  g->flags &= ~(F_CONVERGED | F_NEED_RU);
  if (active == 0) g->flags |= F_CONVERGED;
}
__device__ inline void fin_mcg_ru_ortho(McgState* g, const double* v) {
  for (int i = 0; i < g->n; ++i) {
    CgState* st = &g->sys[i];
    st->ortho_re = st->rr > 0.0 ? v[2 * i] / st->rr : 0.0;
    st->ortho_im = st->rr > 0.0 ? v[2 * i + 1] / st->rr : 0.0;
    if (!((g->active >> i) & 1)) st->beta = 0.0;
  }
}

__device__ inline void finalize(const RedTarget& t, const double* v, int nv) {
  switch (t.op) {
    case RED_STORE:
      for (int i = 0; i < nv; ++i) t.out[i] = v[i];
      break;
    case RED_CG_ALPHA: {
      CgState* st = (CgState*)t.state;
      st->pAp = v[0];
      if (!(v[0] > 0.0) || !finite_d(v[0])) st->flags |= F_BREAKDOWN;
      else st->alpha = st->rr / v[0];
      break;
    }
    case RED_CG_BETA:
      cg_beta_update((CgState*)t.state, v[0]);
      break;
    case RED_RU_RESID:
      fin_ru_resid((CgState*)t.state, v[0]);
      break;
    case RED_RU_ORTHO:
      fin_ru_ortho((CgState*)t.state, v);
      break;
    case RED_RU_BOTH:
      fin_ru_resid((CgState*)t.state, v[0]);
      fin_ru_ortho((CgState*)t.state, v + 1);
      break;
    case RED_MS_ALPHA: {
      MsState* ms = (MsState*)t.state;
      CgState* st = &ms->cg;
      st->pAp = v[0];
      if (!(v[0] > 0.0) || !finite_d(v[0])) {
        st->flags |= F_BREAKDOWN;
        break;
      }
      double a = st->rr / v[0];
      st->alpha = a;
      // the previous iteration's shift update has consumed zeta(k+1): rotate,
      // and retire the shifts that reached their target
      for (int s = 0; s < ms->nshift; ++s) {
        ms->zeta_prev[s] = ms->zeta[s];
        ms->zeta[s] = ms->zeta_next[s];
      }
      ms->active_mask &= ~ms->stop_mask;
      ms->stop_mask = 0;
      for (int s = 0; s < ms->nshift; ++s) {
        if (!((ms->active_mask >> s) & 1)) continue;
        double zp = ms->zeta_prev[s], z = ms->zeta[s];
        double den = ms->alpha_prev * zp * (1.0 + a * ms->delta[s]) + a * ms->beta_prev * (zp - z);
        double zn = z * zp * ms->alpha_prev / den;
        ms->zeta_next[s] = zn;
        ms->alpha_s[s] = a * zn / z;
      }
      break;
    }
    case RED_MS_BETA: {
      MsState* ms = (MsState*)t.state;
      CgState* st = &ms->cg;
      double rr_new = v[0];
      if (!finite_d(rr_new)) {
        st->flags |= F_BREAKDOWN;
        break;
      }
      double b = rr_new / st->rr;
      st->beta = b;
      st->rr_prev = st->rr;
      st->rr = rr_new;
      st->iter += 1;
      double rn = sqrt(rr_new);
      int mask = ms->active_mask;
      for (int s = 0; s < ms->nshift; ++s) {
        if (!((mask >> s) & 1)) continue;
        double ratio = ms->zeta_next[s] / ms->zeta[s];
        ms->beta_s[s] = b * ratio * ratio;
        ms->iters[s] = st->iter;
      }
      ms->alpha_prev = st->alpha;
      ms->beta_prev = b;
      // shifts whose residual |zeta_s| ||r|| reached the target still take
      // this iteration's update; they are retired at the next alpha step
      int stop = 0;
      for (int s = 0; s < ms->nshift; ++s)
        if (((mask >> s) & 1) && fabs(ms->zeta_next[s]) * rn <= ms->sqrt_target_bb) stop |= 1 << s;
      ms->stop_mask = stop;
      if ((mask & ~stop) == 0) st->flags |= F_CONVERGED;
      if (st->iter >= st->max_iter) st->flags |= F_ITER_CAP;
      break;
    }
    case RED_MCG_ALPHA: {
      McgState* g = (McgState*)t.state;
      for (int i = 0; i < g->n; ++i) {
        CgState* st = &g->sys[i];
        if (!((g->active >> i) & 1)) {
          st->alpha = 0.0;
          continue;
        }
        st->pAp = v[i];
        if (!(v[i] > 0.0) || !finite_d(v[i])) {
          st->flags |= F_BREAKDOWN;
          g->flags |= F_BREAKDOWN;
        } else {
          st->alpha = st->rr / v[i];
        }
      }
      break;
    }
    case RED_MCG_BETA: {
      McgState* g = (McgState*)t.state;
      g->iter += 1;
      int active = g->active;
      for (int i = 0; i < g->n; ++i) {
        CgState* st = &g->sys[i];
        if (!((active >> i) & 1)) {
          st->beta = 0.0;
          continue;
        }
        const double rr_new = v[i];
        if (!finite_d(rr_new)) {
          st->flags |= F_BREAKDOWN;
          g->flags |= F_BREAKDOWN;
          continue;
        }
        st->beta = rr_new / st->rr;
        st->rr_prev = st->rr;
        st->rr = rr_new;
        st->iter = g->iter;
        if (rr_new > st->rr_max) st->rr_max = rr_new;
        if (rr_new <= st->target) active &= ~(1 << i);
        if (st->delta2 > 0.0 && rr_new < st->delta2 * st->rr_max) g->flags |= F_NEED_RU;
      }
      g->active = active;
      if (active == 0) g->flags |= F_CONVERGED;
      if (g->iter >= g->max_iter) g->flags |= F_ITER_CAP;
      break;
    }
    case RED_MCG_RU_RESID:
      fin_mcg_ru_resid((McgState*)t.state, v);
      break;
    case RED_MCG_RU_ORTHO:
      fin_mcg_ru_ortho((McgState*)t.state, v);
      break;
    case RED_MCG_RU_BOTH: {
      McgState* g = (McgState*)t.state;
      fin_mcg_ru_resid(g, v);
      fin_mcg_ru_ortho(g, v + g->n);
      break;
    }
  }
}

// ------------------------------------------------------------------ accurate sums
// Per-thread dot-product accumulation in FP32 arithmetic with FP64-class
// accuracy: each product is split exactly into p + e (e = fma(a, b, -p)) and
// added to a (hi, lo) pair with Knuth's TwoSum, the error-free
// transformations of Ogita, Rump and Oishi ("Accurate sum and dot product",
// 2005).  GB300 executes FP64 at a small fraction of its FP32 rate, so the
// per-element work stays on the FP32 pipes and only the per-thread result
// enters the FP64 cross-thread tree.  The _rn intrinsics keep the compiler
// from contracting the sums into FMAs, which would break the transformation.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ void df_add_prod(DF& acc, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);
  const float s = __fadd_rn(acc.hi, p);
  const float bb = __fadd_rn(s, -acc.hi);
  const float err = __fadd_rn(__fadd_rn(acc.hi, -__fadd_rn(s, -bb)), __fadd_rn(p, -bb));
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}
__device__ __forceinline__ double df_value(const DF& d) { return (double)d.hi + (double)d.lo; }

// Accumulator selected by arithmetic type: FP64 sums for double, DF for float.
template <class A> struct Acc1;
template <> struct Acc1<double> {
  double v = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ double value() const { return v; }
};
template <> struct Acc1<float> {
  DF v{0.f, 0.f};
  __device__ __forceinline__ void add_prod(float a, float b) { df_add_prod(v, a, b); }
  __device__ __forceinline__ double value() const { return df_value(v); }
};

// Deterministic block sum of NV doubles; the total is valid in thread 0.
template <int NV> __device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sm[NV][32];
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sm[i][w] = v[i];
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      v[i] = (l < nw) ? sm[i][l] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
  }
  __syncthreads();
}

// Grid-wide sum: each block stores its partial, the last block to finish
// (atomic ticket) adds the partials in block order and finalises.  Every
// thread of every block must call this (no early return before it).
template <int NV> __device__ __forceinline__ void grid_reduce(double (&v)[NV], RedBuf rb, RedTarget tgt) {
  block_sum<NV>(v);
  __shared__ int is_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) rb.partials[i * gridDim.x + blockIdx.x] = v[i];
    __threadfence();
    unsigned t = atomicAdd(rb.counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double w[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) w[i] = 0.0;
  // unrolled so that the loads of several partials are in flight together;
  // each thread still adds its partials in block order (deterministic)
#pragma unroll 8
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int i = 0; i < NV; ++i) w[i] += __ldcg(rb.partials + i * gridDim.x + b);
  block_sum<NV>(w);
  if (threadIdx.x == 0) {
    finalize(tgt, w, NV);
    *rb.counter = 0u;
    __threadfence();
  }
}

// ---- the same sums in double-float: GB300's FP64 pipe is so narrow (about
// 1.75 results per clock per SM) that even the FP64 additions of a block
// tree are visible in a memory-bound kernel, so the FP32-arithmetic kernels
// keep their per-thread (hi, lo) sums and add them across threads and
// blocks with TwoSum on the FP32 pipes; only the final totals become
// doubles.  Same fixed order as the FP64 tree (deterministic).

// a += b, both double-float
__device__ __forceinline__ void df_add_df(DF& a, const DF& b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fadd_rn(s, -a.hi);
  const float err = __fadd_rn(__fadd_rn(a.hi, -__fadd_rn(s, -v)), __fadd_rn(b.hi, -v));
  a.hi = s;
  a.lo = __fadd_rn(__fadd_rn(a.lo, b.lo), err);
}

template <int NV> __device__ __forceinline__ void warp_sum_df(DF (&v)[NV]) {
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      DF w;
      w.hi = __shfl_xor_sync(0xffffffffu, v[i].hi, o);
      w.lo = __shfl_xor_sync(0xffffffffu, v[i].lo, o);
      df_add_df(v[i], w);
    }
}

// Deterministic block sum of NV double-float values; valid in thread 0.
template <int NV> __device__ __forceinline__ void block_sum_df(DF (&v)[NV]) {
  __shared__ float2 sm[NV][32];
  warp_sum_df<NV>(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sm[i][w] = make_float2(v[i].hi, v[i].lo);
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const float2 q = l < nw ? sm[i][l] : make_float2(0.f, 0.f);
      v[i].hi = q.x;
      v[i].lo = q.y;
    }
    warp_sum_df<NV>(v);
  }
  __syncthreads();
}

// grid_reduce for per-thread double-float sums (the partials buffer holds
// (hi, lo) float pairs in its 8-byte slots); the last block converts the
// totals to double and finalises.
template <int NV> __device__ __forceinline__ void grid_reduce_df(DF (&v)[NV], RedBuf rb, RedTarget tgt) {
  block_sum_df<NV>(v);
  float2* part = (float2*)rb.partials;
  __shared__ int is_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) part[i * gridDim.x + blockIdx.x] = make_float2(v[i].hi, v[i].lo);
    __threadfence();
    unsigned t = atomicAdd(rb.counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  DF w[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) w[i] = DF{0.f, 0.f};
#pragma unroll 8
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const float2 q = __ldcg(part + i * gridDim.x + b);
      df_add_df(w[i], DF{q.x, q.y});
    }
  block_sum_df<NV>(w);
  if (threadIdx.x == 0) {
    double t[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) t[i] = df_value(w[i]);
    finalize(tgt, t, NV);
    *rb.counter = 0u;
    __threadfence();
  }
}

// The reduction of an array of per-thread accumulators: double-float sums
// for FP32 arithmetic, the FP64 tree for FP64 arithmetic.
template <int NV> __device__ __forceinline__ void grid_reduce_acc(Acc1<float> (&a)[NV], RedBuf rb, RedTarget tgt) {
  DF v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = a[i].v;
  grid_reduce_df<NV>(v, rb, tgt);
}
template <int NV> __device__ __forceinline__ void grid_reduce_acc(Acc1<double> (&a)[NV], RedBuf rb, RedTarget tgt) {
  double v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = a[i].value();
  grid_reduce<NV>(v, rb, tgt);
}

// Early-exit test shared by the Krylov-loop kernels.
__device__ __forceinline__ bool stopped(const int* flags) { return flags != nullptr && (__ldcg(flags) & F_STOP); }

}  // namespace stag
