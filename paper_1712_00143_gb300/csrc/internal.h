// internal.h -- host-side internals of libstag shared by its translation units.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>

#include "../../include/stag.h"
#include "common.cuh"
#include "df.cuh"

namespace stag {

// One precision copy of the gauge field in the internal layout (see
// links.cu): per output parity, the 16 hop matrices of every site with the
// staggered phase, the 1/2 and the backward sign folded in, packed into
// 16-byte chunks stored [chunk][site].  With NL = 6 only rows 0, 1 of the
// SU(3) part of each Naik hop are kept and the factor +-1/2 eta c3 is applied
// in-kernel.
struct LinkCopy {
  bool present = false;
  void* data = nullptr;     // [2 parities][chunks][Vh] 16-byte chunks
  size_t parity_stride = 0; // bytes per parity
  int nl = 9;
  float fat_scale = 1.f;    // 16-bit formats: stored (normalised) value * scale
  float long_scale = 1.f;   //   = matrix entry
  size_t elem_bytes = 0;    // bytes of one stored complex
  int shape_plain = 1;      // launch shapes chosen by the autotuner
  int shape_epi = 1;        // (default: 256 threads, 4 blocks per SM)
  float tuned_us[2] = {0.f, 0.f};  // their timings (us per launch)
};

struct Workspace {
  std::map<std::string, std::pair<void*, size_t>> bufs;
  ~Workspace();
  // Device buffer of at least `bytes` bytes under `name` (contents kept only
  // while the size does not grow; *fresh set when newly allocated).
  void* get(const std::string& name, size_t bytes, int* status, bool* fresh = nullptr);
  void drop(const std::string& name);
  void release();
};

}  // namespace stag

struct stag_lattice_s {
  stag::Geom g;
  int dims[4];
  double c3 = -1.0 / 24.0;
  int autotune = 1;  // time launch variants on this lattice (stag_link_opts.autotune)
  // launch variants of the N-right-hand-side kernels per (format, N = 2, 4,
  // 8): the plain operator half and the epilogue form the batched CG runs
  // (-1: not chosen yet), each with its time per launch (us)
  struct MrhsTune {
    int variant = -1;
    float us = 0.f;
    int variant_epi = -1;
    float us_epi = 0.f;
  } mrhs[6][4];  // by the ABI precision (stag_prec), tuned per format
  stag::LinkCopy links[5];  // by stag_prec (STAG_DF64 = 4: FP64 split into hi + lo floats)
  stag::Workspace ws;
};

namespace stag {

// ------------------------------------------------------------ instrumentation
void prof_begin(const char* family, cudaStream_t s);
void prof_end(cudaStream_t s);
void prof_flush_completed();
// Sequence mark of the next profiling record, and the discard of the records
// made since a mark (a chunk of iterations cut short by a stop flag).
long long prof_mark();
void prof_discard_since(long long mark);
void count_launch();
// While capturing a CUDA graph: no profiling events, and kernel launches are
// counted aside; set_capturing(false) returns how many were captured.
long long set_capturing(bool on);
// stag_dslash for nrhs > 1 (N-right-hand-side kernels)
int dslash_multi(stag_lattice_s* lat, double2* out, const double2* in, int out_parity, int prec, int nrhs,
                 cudaStream_t st);

struct ProfScope {
  cudaStream_t s;
  ProfScope(const char* family, cudaStream_t st) : s(st) {
    count_launch();
    prof_begin(family, st);
  }
  ~ProfScope() { prof_end(s); }
};

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? STAG_OK : STAG_ECUDA; }
int last_launch_status();

// Reduction scratch: [nv_max][max_grid] partial sums and a ticket counter.
struct RedScratch {
  double* partials;
  unsigned* counter;
  int max_grid;
};
int get_red_scratch(stag_lattice_s* lat, const char* name, RedScratch* out, int nv_max = 2);

// A Spinor<P> living in the handle's workspace buffer `name`.
template <int P> Spinor<P> ws_spinor(stag_lattice_s* lat, const std::string& name, int* status);

// ------------------------------------------------------------------- autotuner cache (tune.cu)
// Key of a tuned launch: kernel family, storage format, Naik entries per
// hop, right-hand sides, lattice extents.
std::string tune_key(const char* kernel, int prec, int nl, int nrhs, const int dims[4]);
// Process-wide cache of tuned variants (loaded on first use from the JSON
// file named by STAG_TUNE_CACHE, if set; rewritten there on every put).
bool tune_cache_get(const std::string& key, int* variant, double* us);
void tune_cache_put(const std::string& key, int variant, double us);

// ------------------------------------------------------------------- links
int build_link_copy(stag_lattice_s* lat, int prec, int recon, const double2* fat, const double2* lng,
                    cudaStream_t st);

// ------------------------------------------------------------------- dslash
// Storage format P of the links and spinors (64, 32, 16 = binary16, 15 =
// 16-bit fixed point, 31 = 16-bit fixed-point links with FP32 vectors);
// accumulation precision PA = 64 for P = 64, else 32.
template <int P> struct Acc { static constexpr int value = (P == 64) ? 64 : 32; };
// The link copy an operator precision of the ABI reads (STAG_FX16L32 reads
// the 16-bit fixed-point copy).
inline int link_copy_of(int prec) { return prec == STAG_FX16L32 ? STAG_FX16 : prec; }
// The ABI precision (stag_prec) of a format tag.
template <int P> constexpr int abi_prec() {
  return P == 64 ? STAG_FP64 : P == 32 ? STAG_FP32 : P == 16 ? STAG_FP16 : P == 31 ? STAG_FX16L32 : STAG_FX16;
}
// The link copy a format reads (tag 31 reads the 16-bit fixed-point copy).
template <int P> constexpr int prec_index() {
  return P == 64 ? STAG_FP64 : P == 32 ? STAG_FP32 : P == 16 ? STAG_FP16 : STAG_FX16;
}

template <int P>
int launch_dslash(const stag_lattice_s* lat, Spinor<P> out, Spinor<P> in, int out_parity, const int* flags,
                  cudaStream_t st);

// Times the launch shapes of the Dslash kernels and keeps the fastest.
template <int P> int tune_dslash(stag_lattice_s* lat, cudaStream_t st);

// out = ax * x + ay * y + ad * (D in) on parity out_parity, and optionally a
// reduction: red = 1: Re <x, out>; red = 2: ||out||^2.
template <int P>
int launch_dslash_epi(const stag_lattice_s* lat, Spinor<Acc<P>::value> out, Spinor<P> in, int out_parity,
                      Spinor<P> x, double ax, Spinor<Acc<P>::value> y, double ay, double ad, int red,
                      RedScratch rs, RedTarget tgt, const int* flags, cudaStream_t st);

// The plain and the fused-epilogue kernel on the output sites [s0, s1) only
// (flags: a solver's stop word, or null).
template <int P>
int launch_dslash_range(const stag_lattice_s* lat, Spinor<P> out, Spinor<P> in, int out_parity, int s0, int s1,
                        const int* flags, cudaStream_t st);
template <int P>
int launch_dslash_epi_range(const stag_lattice_s* lat, Spinor<Acc<P>::value> out, Spinor<P> in, int out_parity,
                            Spinor<P> x, double ax, Spinor<Acc<P>::value> y, double ay, double ad, int red,
                            RedScratch rs, RedTarget tgt, int s0, int s1, const int* flags, cudaStream_t st);

// ------------------------------------------------------------------- blas
// canonical [Vh][3] complex double <-> internal Spinor<P>
template <int P> int launch_from_canonical(Spinor<P> out, const double2* in, int Vh, cudaStream_t st);
template <int P> int launch_to_canonical(double2* out, Spinor<P> in, int Vh, cudaStream_t st);
// out (precision PO) = in (precision PI)
template <int PO, int PI> int launch_convert(Spinor<PO> out, Spinor<PI> in, cudaStream_t st);
int launch_zero(void* p, size_t bytes, cudaStream_t st);

// ||v||^2 (FP64) or Re<a,b>, Im<a,b> into a RedTarget.
template <int P> int launch_norm2(Spinor<P> v, RedScratch rs, RedTarget tgt, cudaStream_t st);

// CG update: xh += alpha p; rh -= alpha Ap; ||rh||^2 -> RED_CG_BETA.
template <int P>
int launch_cg_update(Spinor<Acc<P>::value> xh, Spinor<Acc<P>::value> rh, Spinor<P> p, Spinor<Acc<P>::value> Ap,
                     CgState* state, RedScratch rs, cudaStream_t st);
// p = rh + beta p
template <int P> int launch_cg_xpay(Spinor<P> p, Spinor<Acc<P>::value> rh, CgState* state, cudaStream_t st);
// y += xh; xh = 0   (y FP64)
template <int PV> int launch_accumulate(Spinor<64> y, Spinor<PV> xh, cudaStream_t st);
// rh = convert(r64) and <rh, p> -> RED_RU_ORTHO
template <int P>
int launch_ru_convert_dot(Spinor<Acc<P>::value> rh, Spinor<64> r, Spinor<P> p, CgState* state, RedScratch rs,
                          cudaStream_t st);
// p = rh + beta (p - ortho rh)
template <int P> int launch_ru_p(Spinor<P> p, Spinor<Acc<P>::value> rh, CgState* state, cudaStream_t st);

// Multi-shift: r -= alpha Ap; ||r||^2 -> RED_MS_BETA
template <int P>
int launch_ms_r_update(Spinor<Acc<P>::value> r, Spinor<Acc<P>::value> Ap, MsState* state, RedScratch rs,
                       cudaStream_t st);
// for every active shift s: x_s += alpha_s p_s; p_s = zeta_s r + beta_s p_s
// Runs only when the state's iteration count equals expect_iter (the residual
// update of this iteration ran); `base` is the smallest shift.
template <int P>
int launch_ms_shift_update(Spinor<Acc<P>::value>* xs, Spinor<P>* ps, int nshift, int base, Spinor<Acc<P>::value> r,
                           MsState* state, int expect_iter, cudaStream_t st);


// ------------------------------------------------------------------- double-float (dslash_df.cu)
// t = D in on parity out_parity for n systems of DF fields ([n][Vh][3] float4),
// with the handle's DF link copy; up to four systems per launch.
int launch_dslash_df(const stag_lattice_s* lat, DfField out, DfField in, int n, int out_parity, const int* stop,
                     cudaStream_t st);
// out_r = ad (D in)_r + ax x_r + ay y_r (ad = +1 or -1; x, y DF fields or null)
int launch_dslash_df_epi(const stag_lattice_s* lat, DfField out, DfField in, int n, int out_parity, DfField x,
                         double ax, DfField y, double ay, double ad, const int* stop, cudaStream_t st);
// times the double-float hop kernel's launch variants on this lattice
int tune_df(stag_lattice_s* lat, cudaStream_t st);
// FP64 [n][Vh][3] <-> DF
int launch_df_from_double(DfField out, const double2* in, int n, cudaStream_t st);
int launch_df_to_double(double2* out, DfField in, int n, cudaStream_t st);
// y_r += xh_r (FP64), xh_r = 0, ydf_r = split(y_r - ya_r) (ya: the anchor,
// null = 0); n in {1, 2, 4, 8}; MRHS layouts
template <int PV>
int launch_accumulate_df(void* y64, void* xh, DfField ydf, const void* ya, int n, const int* stop, cudaStream_t st);
// the anchor moves to (y, r): ya = y, ra = split(r) (FP64 fields, n systems)
int launch_df_anchor(void* ya, DfField ra, const void* y, const void* r, int n, const int* stop, cudaStream_t st);
// Reliable updates in double-float are measured from an anchor (y_a, r_a =
// b - M y_a), which starts at (0, b) and is moved once, by an FP64 update,
// when the iterated residual has fallen below this fraction of ||b|| (squared):
// from then on the update's rounding error is relative to y - y_a, not to y.
constexpr double kDfAnchorRel2 = 1e-10;
// rh_r = r_r (rounded), ||rh_r||^2 and <rh_r, p_r> -> tgt (RED_RU_BOTH for one
// system, RED_MCG_RU_BOTH for a group)
template <int P>
int launch_ru_convert_dot_df(void* rh, DfField r, const void* p, int n, RedScratch rs, RedTarget tgt, const int* stop,
                             cudaStream_t st);
// ||v_r||^2 -> tgt (n values)
int launch_norm2_df(DfField v, int n, RedScratch rs, RedTarget tgt, cudaStream_t st);
// Krylov-loop (PV) fields from DF fields
template <int PV> int launch_convert_from_df(void* out, DfField in, int n, cudaStream_t st);

}  // namespace stag
