/*
 * stag.h -- C ABI of libstag, a single-GPU (GB300, sm_103a) library for the
 * even-odd improved-staggered conjugate-gradient solve.
 *
 * What it computes (the paper benchmarks the staggered single-mass and
 * multi-shift CG, Sec. 1 and Sec. 4.1, but prints no operator; the standard
 * improved-staggered form it refers to is written out here):
 *
 *   (D psi)(x) = 1/2 sum_mu eta_mu(x) [ F_mu(x) psi(x+mu) - F_mu(x-mu)^+ psi(x-mu)
 *                                      + L_mu(x) psi(x+3mu) - L_mu(x-3mu)^+ psi(x-3mu) ]
 *
 *   eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y), eta_t = (-1)^(x+y+z),
 *   periodic wrap in all directions, F = fat links, L = Naik (long) links,
 *   M = m^2 - D_eo D_oe on even sites (Hermitian positive definite).
 *
 * Canonical layout (the only layout callers see):
 *   - extents dims[4] = {Lx, Ly, Lz, Lt}, each even and >= 4;
 *   - sites lexicographic, x fastest: lex = x + Lx*(y + Ly*(z + Lz*t));
 *   - links: [V][4][3][3] interleaved complex double (re, im), mu = x,y,z,t,
 *     row-major colour matrices, WITHOUT staggered phases or the 1/2 (the
 *     library folds both in);
 *   - single-parity colour-vector fields: [V/2][3] complex double indexed by
 *     lex/2; an even field lives on sites with (x+y+z+t) even.
 *   - several right-hand sides: [nrhs][V/2][3], each system contiguous.
 *
 * Pointers: every field/link pointer is a DEVICE pointer (cudaMalloc or a
 * PyTorch CUDA tensor) unless stated otherwise.  The caller owns them.
 * stream: a cudaStream_t passed as void*; NULL means the legacy default
 * stream.  Solvers synchronise `stream` before returning; stag_dslash and
 * stag_apply_m are asynchronous.
 *
 * Errors: every call returns an int status (0 = STAG_OK, negative = error);
 * no exception crosses the ABI.  A handle is not thread-safe: use one handle
 * per host thread, or serialise calls on it.
 */
#ifndef STAG_H
#define STAG_H

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define STAG_OK 0
#define STAG_EINVAL (-1)      /* null pointer, odd or too small extent, bad enum */
#define STAG_ENOMEM (-2)      /* device allocation failed */
#define STAG_ECUDA (-3)       /* a CUDA runtime call or kernel launch failed */
#define STAG_ENOTCONV (-4)    /* max_iter reached; x holds the last iterate */
#define STAG_EBREAKDOWN (-5)  /* NaN/Inf or <p,Ap> <= 0 in a solver */
#define STAG_ENOTUNITARY (-6) /* recon-12 asked for links with L/c3 not in SU(3) */
#define STAG_ETIMEOUT (-7)    /* a bounded device wait gave up */

/* --------------------------------------------------------------- precision */
/* STAG_FP16: IEEE binary16 storage.  STAG_FX16: 16-bit fixed point (15
 * fraction bits) in units of a per-site (vectors) or per-field (links) scale.
 * Both keep one FP32 scale per site for vectors and compute in FP32.
 * STAG_DF64: FP64-class "double-float": links and vectors carried as the sum
 * hi + lo of two floats (about 48 significant bits; links split once at load,
 * 16 bytes per complex like FP64), products and sums by error-free
 * transformations on the FP32 pipes (GB300 runs FP64 arithmetic at a small
 * fraction of its FP32 rate).  Relative error of the operator about 1e-14.
 * The mixed-precision solvers compute their reliable updates (the true
 * residual b - M y) in this format when the handle holds its link copy, and
 * in FP64 otherwise.
 * STAG_FX16L32: the 16-bit fixed-point links of the STAG_FX16 copy with FP32
 * vectors and FP32 arithmetic (no copy of its own; the link bytes, the bulk
 * of a multi-right-hand-side operator's traffic, halve while the vectors keep
 * single precision).  Accepted by stag_dslash and stag_apply_m; the Krylov
 * operator of STAG_MIXED16L. */
typedef enum {
  STAG_FP64 = 0,
  STAG_FP32 = 1,
  STAG_FP16 = 2,
  STAG_FX16 = 3,
  STAG_DF64 = 4,
  STAG_FX16L32 = 5
} stag_prec;

/* Solver modes (the paper: QUDA's mixed-precision solvers, Sec. 3; single
 * precision about twice as fast as double, Sec. 4).  PLAIN64: every
 * operation in FP64.  MIXED32 / MIXED16 / MIXEDFX16: the Krylov iteration
 * uses the FP32 / binary16 / 16-bit fixed-point Dslash and search direction,
 * FP32 residual and iterate, FP64-class reductions, FP64 solution
 * accumulation and "reliable updates": the true residual b - M y recomputed
 * with an FP64-class operator (STAG_DF64 if the handle holds that copy,
 * else FP64) whenever the iterated residual has dropped by `delta` since the
 * last update, and at the end. */
typedef enum {
  STAG_PLAIN64 = 0,
  STAG_MIXED32 = 1,
  STAG_MIXED16 = 2,
  STAG_MIXEDFX16 = 3,
  STAG_LEARNED = 4,  /* flexible CG preconditioned by a trained network (params->precond);
                        sloppy operator in 16-bit fixed point if the handle holds that
                        copy, else FP32; falls back to mixed CG if FCG breaks down or
                        reaches max_iter */
  STAG_MIXED16L = 5  /* as MIXED32 with the STAG_FX16L32 operator: 16-bit fixed-point
                        links, FP32 vectors (needs the STAG_FX16 copy) */
} stag_mode;

typedef struct stag_lattice_s* stag_lattice_t; /* opaque, library-owned */

typedef struct {
  int recon_long;    /* 18: long links stored in full; 12: two rows stored, the
                        third rebuilt as conj(row0 x row1) (FP32 and 16-bit
                        copies; needs L/long_coeff in SU(3), else ENOTUNITARY) */
  double long_coeff; /* c3 with L = c3 * (product of SU(3) links); -1/24 */
  unsigned prec_mask; /* bit (1 << stag_prec) per copy to build; 0 = all five */
  int autotune;      /* 1: time the Dslash launch shapes of each copy on this
                        lattice and keep the fastest (a few ms); 0: defaults */
} stag_link_opts;

typedef struct {
  double tol;          /* target ||b - M x|| / ||b|| (FP64 true residual) */
  int max_iter;        /* cap on Krylov iterations (per solve / per shift) */
  int mode;            /* stag_mode */
  double delta;        /* reliable-update trigger: ||r|| < delta * max||r|| */
  int use_initial_guess; /* 1: start from the x passed in; 0: from zero */
  int check_interval;  /* iterations between host convergence checks (>=1) */
  double ms_tol;       /* multi-shift: relative residual at which the shared
                          Krylov loop hands each shift to refinement (<=0: tol) */
  void* precond;       /* stag_net_t for STAG_LEARNED, else ignored */
} stag_solve_params;

typedef struct {
  int iters;            /* Krylov iterations (multi-shift: shared + refinement) */
  int reliable_updates; /* FP64-class true-residual recomputations */
  int converged;        /* 1 if true_rel_resid <= tol */
  int status;           /* STAG_OK or the error for this system */
  double true_rel_resid; /* ||b - M x|| / ||b|| recomputed on the GPU with the
                            FP64-class operator of the reliable updates */
  double seconds;       /* wall time of the solve on the host */
  int precond_fallback; /* STAG_LEARNED: 1 if the mixed-CG fallback ran */
} stag_solve_info;

/* Default parameters: tol 1e-10, max_iter 100000, MIXED32, delta 0.1,
 * check_interval 16, ms_tol 1e-6. */
void stag_default_params(stag_solve_params* p);

/* Load a gauge field (the operator's fat and long links) into a new handle.
 * Builds, on the GPU, the library's internal site-blocked structure-of-arrays
 * copies (the paper's QPhiX uses an SOA layout, Sec. 3) with the staggered
 * phases and the 1/2 folded in, in each precision of opts->prec_mask.
 *   out  : receives the handle (release with stag_free_lattice).
 *   dims : host array {Lx, Ly, Lz, Lt}, even, each >= 4.
 *   fat, lng : device, canonical [V][4][3][3] complex double.  Copied; the
 *          caller may free them after the call returns.
 *   opts : may be NULL (recon 18, c3 = -1/24, all precisions, autotune).
 * Errors: EINVAL, ENOMEM, ECUDA, ENOTUNITARY.  Synchronises `stream`. */
int stag_load_links(stag_lattice_t* out, const int dims[4], const void* fat, const void* lng,
                    const stag_link_opts* opts, void* stream);

/* Release a handle from stag_load_links: waits for all device work
 * (cudaDeviceSynchronize), then frees every device buffer the handle owns.
 * The handle must not be used afterwards.  NULL: EINVAL. */
int stag_free_lattice(stag_lattice_t lat);

/* The launch shape the autotuner kept for a copy's Dslash kernel
 * (kernel 0: plain, 1: fused epilogue with dot product): threads per block,
 * minimum resident blocks per SM given to the compiler, and its timing in us
 * per launch (0 when not tuned).  For STAG_DF64 (four right-hand sides per
 * launch) min_blocks reports the threads that share a site's right-hand
 * sides (1, 2 or 4).  STAG_FX16L32 reports the shape tuned for STAG_FX16,
 * which its single-right-hand-side kernels share.  Any output pointer may be
 * NULL. */
int stag_tuned_shape(stag_lattice_t lat, int prec, int kernel, int* block, int* min_blocks, double* us);

/* The launch variant of the N-right-hand-side Dslash kernel (the operator
 * of stag_batch_solve and of stag_dslash with nrhs > 1) for groups of nrhs
 * = 2, 4 or 8 right-hand sides of format prec on this lattice: the threads
 * that share one site's right-hand sides (1, 2 or 4), the resident blocks
 * per SM promised to the compiler (1: no register cap; 4: at most 128
 * registers; 6: at most 80), and the timed cost of one launch in us (0 when
 * the variant was not timed: before the first such group, or with
 * autotune off).  stag_tuned_mrhs reports the plain kernel (t = D_oe p),
 * stag_tuned_mrhs_epi the epilogue form the batched CG runs (Ap = m^2 p -
 * D_eo t with its <p, Ap> partials); each is chosen, the first time a group
 * of that size runs on a lattice of these extents, by timing every compiled
 * variant (the autotuner; the paper tunes nothing at run time, its QPhiX
 * and QUDA builds fix their blocking at compile time or tune it inside
 * QUDA, Sec. 3).  EINVAL for another nrhs or a missing copy.  Any output
 * may be NULL. */
int stag_tuned_mrhs(stag_lattice_t lat, int prec, int nrhs, int* threads_per_site, int* min_blocks, double* us);
int stag_tuned_mrhs_epi(stag_lattice_t lat, int prec, int nrhs, int* threads_per_site, int* min_blocks, double* us);
/* The same choice as a variant index (epilogue != 0: the epilogue form):
 * 0..5 = (threads per site, min blocks) (1,1) (1,6) (2,4) (2,6) (4,4)
 * (4,6).  Returns the index (>= 0) or STAG_EINVAL. */
int stag_tuned_mrhs_variant(stag_lattice_t lat, int prec, int nrhs, int epilogue);

/* The autotuner's cache (host only, no GPU call).  Tuned launches are kept
 * for the life of the process under a key naming the kernel family, the
 * storage format, the Naik entries per hop, the right-hand sides per launch
 * and the extents, e.g. "dslash_mrhs/fp32/nl6/n4/32x32x32x32"; a later
 * lattice with the same key reuses the choice without timing.  If the
 * environment variable STAG_TUNE_CACHE names a file, the cache is loaded
 * from it on first use and the file is rewritten after every new entry.
 * File format (JSON): {"version": 1, "entries": {"<key>": {"variant": v,
 * "us": t}, ...}}.
 *   stag_tune_key   : writes the key for (kernel, prec, nl, nrhs, dims) into
 *                     buf (len bytes, NUL included); EINVAL if it does not fit
 *   stag_tune_cache_get   : *variant = the stored variant, or -1 if the key
 *                     is absent (*us likewise, 0)
 *   stag_tune_cache_put   : stores (variant >= 0), replacing an entry
 *   stag_tune_cache_load  : merges a file's entries; EINVAL if the file is
 *                     missing or malformed (the cache is then unchanged)
 *   stag_tune_cache_save  : writes every entry (via a temporary file)
 *   stag_tune_cache_clear : forgets every entry (and the STAG_TUNE_CACHE file
 *                     for the rest of the process)
 *   stag_tune_cache_size  : number of entries */
int stag_tune_key(char* buf, int len, const char* kernel, int prec, int nl, int nrhs, const int dims[4]);
int stag_tune_cache_get(const char* key, int* variant, double* us);
int stag_tune_cache_put(const char* key, int variant, double us);
int stag_tune_cache_load(const char* path);
int stag_tune_cache_save(const char* path);
int stag_tune_cache_clear(void);
long long stag_tune_cache_size(void);

/* Lattice extents and the per-parity site count V/2 of a handle. */
int stag_lattice_info(stag_lattice_t lat, int dims[4], long long* vh);

/* out = D psi restricted to sites of parity out_parity (0 even, 1 odd); in
 * lives on the other parity.  D is the operator written at the top of this
 * header: the kernel of every CG iteration the paper benchmarks (Sec. 1,
 * Sec. 4.1, its single-GPU L^4 sweep in Fig. 9), applied twice per
 * iteration; the paper itself prints no formula for it.  Computed with the
 * links and arithmetic of `prec` (FP64: FP64 throughout; DF64: double-float,
 * see stag_prec; FP32: FP32 storage and accumulation; FP16 and FX16: 16-bit
 * storage with a per-site vector scale and a per-field link scale, FP32
 * accumulation).  nrhs > 1 right-hand sides share each link read (groups of
 * 8, 4, 2; DF64: 4).  in/out: device, canonical [nrhs][V/2][3] complex
 * double (converted to and from the internal layout around the kernel).
 * Asynchronous on `stream`.  Errors: EINVAL, ENOMEM, ECUDA. */
int stag_dslash(stag_lattice_t lat, void* out, const void* in, int out_parity, int prec, int nrhs,
                void* stream);

/* out = (m^2 + shift) in - D_eo D_oe in on even sites, arithmetic of `prec`
 * (the even-odd operator M whose solves the paper benchmarks, Sec. 4.1).
 * in/out: device canonical [V/2][3] complex double.  Asynchronous. */
int stag_apply_m(stag_lattice_t lat, void* out, const void* in, double mass, double shift, int prec,
                 void* stream);

/* ------------------------------------------------- allocation-free operator
 * stag_apply_m_noalloc computes exactly what stag_apply_m computes with
 * prec = STAG_FP64 (out = (m^2 + shift) in - D_eo D_oe in, even sites), but
 * never allocates device memory.  It exists for callers that cannot call
 * cudaMalloc at the point where they apply the operator: applications whose
 * own pool allocator owns all device memory and forbids other allocations,
 * and real-time or certified code paths that allow no allocation (and none
 * of the device-wide synchronisation cudaFree implies) after start-up.
 * There is no counterpart in the paper.
 *
 * Scratch: the odd-parity intermediate D_oe in lives in a file-scope static
 * device array of STAG_NOALLOC_MAX_VH sites x 3 complex doubles (3 MiB),
 * which every GPU that loads libstag holds until the process exits.  The
 * lattice must have V/2 <= STAG_NOALLOC_MAX_VH (e.g. 16^4, 16^3 x 32);
 * larger lattices are rejected with STAG_EINVAL before any GPU work.
 * The handle must hold an FP64 link copy (prec_mask bit 0).
 *
 * The first call on a device looks up the array's device address for that
 * device (one-time set-up, with that device current); make that first call
 * before any stream capture.  The address is kept for the life of the
 * device's context: do not use this call after cudaDeviceReset (or any
 * other reset of the primary context) in the same process.  in and out
 * must not overlap (STAG_EINVAL).  Profiler families "dslash64" and
 * "dslash64_epi" (one launch each).  All calls share the one array: calls whose
 * kernels can overlap on the GPU (different streams, or several host
 * threads) race on it and must be serialised by the caller.  The array
 * keeps the last call's contents; nothing in it needs to start at zero, as
 * every entry is written before it is read.
 * in/out: device, canonical [V/2][3] complex double.  Asynchronous on
 * `stream`.  Errors: EINVAL, ECUDA. */
#define STAG_NOALLOC_MAX_VH 65536
int stag_apply_m_noalloc(stag_lattice_t lat, void* out, const void* in, double mass, double shift,
                         void* stream);

/* Solve M x = b (even sites) to params->tol in FP64-class true residual:
 * the single-mass CG of the paper (Sec. 1: the staggered QPhiX library
 * provides single-mass and multi-shift CG; Sec. 4 and Fig. 1: CG takes
 * about 90 % of the RHMD run time), with the precision modes of stag_mode.
 * x, b: device canonical [V/2][3] complex double; x is read as the initial
 * guess when params->use_initial_guess, and always written.
 * info: host, may be NULL.  Returns STAG_OK, ENOTCONV (x = last iterate),
 * EBREAKDOWN, EINVAL, ENOMEM, ECUDA.  Synchronises `stream`. */
int stag_cg(stag_lattice_t lat, void* x, const void* b, double mass, const stag_solve_params* params,
            stag_solve_info* info, void* stream);

/* Solve (M + shifts[s]) x_s = b for nshift shifts from one shared Krylov
 * space (multi-shift CG, the production workhorse of Sec. 4.1), then refine
 * each shift whose FP64 true residual misses tol with single-shift CG from
 * x_s in the same mode.  x: host array of nshift device pointers
 * (canonical [V/2][3] complex double); shifts: host array, each >= 0.
 * infos: host array of nshift, may be NULL.  Synchronises `stream`. */
int stag_multishift_cg(stag_lattice_t lat, void* const* x, const void* b, double mass,
                       const double* shifts, int nshift, const stag_solve_params* params,
                       stag_solve_info* infos, void* stream);

/* One lattice's share of a batched solve: nrhs systems M x_i = b_i with the
 * same mass.  x, b: device, canonical [nrhs][V/2][3] complex double. */
typedef struct {
  stag_lattice_t lat;
  void* x;
  const void* b;
  int nrhs;
  double mass;
} stag_batch_item;

/* Solve every system of every item to params->tol (FP64-class true
 * residual), all items together.  The paper solves one system at a time
 * (Sec. 4.1) and says nothing of batching; this call is the library's
 * extension for the many independent solves of a configuration (several
 * sources, several gauge fields of uneven sizes).
 * Each item's right-hand sides are solved in groups of up to 8 (16-bit
 * modes: 4) that share one multi-right-hand-side Dslash per operator
 * application (links read once for the whole group), each system with its
 * own CG scalars and its own stopping point; a group takes a reliable update
 * for all its systems when any of them triggers one.
 *   - One group: chunks of check_interval iterations queued directly on the
 *     group's stream, the host reading the group's state between chunks.
 *   - Several groups: the whole solve is one launch of a CUDA graph whose
 *     conditional WHILE node repeats a round over all groups side by side
 *     (each group's reliable update when one is due, then check_interval
 *     iterations whose kernels return at once once the group is done) until
 *     every group is done or a fixed budget of rounds runs out; the host
 *     waits once.
 * Modes as for stag_cg except STAG_LEARNED (use_initial_guess reads x).
 * infos: host array with one entry per system, item by item, may be NULL.
 * Returns STAG_OK, or the first error (ENOTCONV, EBREAKDOWN ...) met by a
 * system.  Synchronises `stream`. */
int stag_batch_solve(const stag_batch_item* items, int nitems, const stag_solve_params* params,
                     stag_solve_info* infos, void* stream);

/* ------------------------------------------------------------ learned part
 * The paper has no learned component: it benchmarks plain and multi-shift CG
 * (Sec. 4.1).  These calls are the library's extension: a gauge-covariant
 * network used as a preconditioner z = N(r) inside flexible CG (Notay's FCG
 * with one-term truncation; STAG_LEARNED), trained on the GPU on (residual,
 * error) pairs from the unpreconditioned solver.  Fields are full-lattice,
 * channels of colour vectors; a layer with real weights W[d][c][c'] (stored
 * as bfloat16, FP32 accumulation)
 * computes pre_c = sum_d sum_c' W[d][c][c'] T_d h_c', d = 0 the identity and
 * d = 1 + 2mu, 2 + 2mu the fat-link hops of the staggered operator from +mu
 * and -mu (the +-1/2 eta F parts of D); hidden layers apply the covariant
 * gate v * sigmoid(|v|^2 - b_c).  The residual is scaled to unit mean square
 * per site and placed on the even sites; the output's even sites, scaled
 * back, are z.  Parameters, flat FP32 array: for each layer W[9][Cout][Cin]
 * then (hidden layers) b[Cout].  Widths 1 and 16 are supported, first and
 * last width 1.  The network needs the handle's FP32 link copy. */
typedef struct stag_net_s* stag_net_t;

typedef struct {
  stag_lattice_t lat; /* gauge field of the pair (FP32 copy required) */
  const void* r;      /* device, canonical [V/2][3] residual */
  const void* e;      /* device, canonical [V/2][3] error x* - x of that residual */
} stag_train_pair;

typedef struct {
  int epochs;
  int batch;               /* pairs per Adam step (gradients averaged) */
  double lr;               /* Adam step size (beta1 0.9, beta2 0.999) */
  unsigned long long seed; /* visiting-order permutations */
  int pair_prec;           /* STAG_FP64: complex double pairs; STAG_FP32: complex float */
  int loss;                /* stag_loss */
  double mass;             /* the pairs' mass m (STAG_LOSS_RESIDUAL) */
} stag_train_params;

/* Training losses, both on the scaled fields r^ = r sqrt(V/2)/||r||, e^, z^ = N^(r^):
 *   STAG_LOSS_RESIDUAL  ||M z^ - r^||^2 / ||r^||^2, M = m^2 - D_eo D_oe of the
 *                       pair's field in FP32 (= ||M (z^ - e^)||^2 / ||M e^||^2
 *                       since r = M e: the error weighted by M^2, i.e. by the
 *                       high modes a short-range network can represent)
 *   STAG_LOSS_ERROR     ||z^ - e^||^2 / ||e^||^2 (dominated by the low modes
 *                       that make up most of e at small mass; at m = 0.01 it
 *                       barely falls below 1) */
enum stag_loss { STAG_LOSS_ERROR = 0, STAG_LOSS_RESIDUAL = 1 };

/* channels: nlayers + 1 widths (e.g. {1, 16, 16, 16, 1}); seed: the small
 * normal noise of the initial weights.  The network starts near the
 * identity (self direction maps channel c to c with weight 1, gates open),
 * so an untrained network makes flexible CG behave like CG. */
int stag_net_create(stag_net_t* out, const int* channels, int nlayers, unsigned long long seed);
/* Release a network: waits for all device work, then frees its weights,
 * optimiser moments and gradient buffers.  NULL: EINVAL. */
int stag_net_free(stag_net_t net);
/* Number of parameters in the flat host layout of get/set params: for each
 * layer l, W[9][C_out][C_in] (direction 0 = the site itself; 1 + 2 mu and
 * 2 + 2 mu = the forward and backward fat-link hops of direction mu)
 * followed, except after the last layer, by the gate biases b[C_out].
 * -1 for a NULL handle. */
long long stag_net_num_params(stag_net_t net);
/* host copies of the parameters; rounded = 1 returns the weights as the
 * kernels use them (bfloat16 values), 0 the FP32 master copy */
int stag_net_get_params(stag_net_t net, float* host, long long count, int rounded);
int stag_net_set_params(stag_net_t net, const float* host, long long count);
/* z = N(r), r and z device canonical [V/2][3] complex double: the
 * preconditioner application inside STAG_LEARNED flexible CG (no
 * counterpart in the paper).  Asynchronous. */
int stag_net_apply(stag_net_t net, stag_lattice_t lat, void* z, const void* r, void* stream);
/* Loss of one pair (loss_kind: stag_loss; mass: the pair's m, used by
 * STAG_LOSS_RESIDUAL) and its gradient w.r.t. the parameters (host array of
 * count floats); no counterpart in the paper.  r, e: device canonical
 * [V/2][3] complex double.  Synchronises `stream`. */
int stag_net_loss_grad(stag_net_t net, stag_lattice_t lat, const void* r, const void* e, int loss_kind, double mass,
                       double* loss, float* grad, long long count, void* stream);
/* Adam training on the pairs (all on lattices of one size; no counterpart in
 * the paper); losses: host, epochs * npairs values in visiting order, may be
 * NULL.  Synchronises. */
int stag_net_train(stag_net_t net, const stag_train_pair* pairs, int npairs, const stag_train_params* tp,
                   double* losses, void* stream);

/* ------------------------------------------- one lattice over several ranks
 * The paper's multi-node study (Sec. 4.1, Figs. 2-3: weak scaling of the
 * staggered CG on KNL clusters, network-bound below about L = 30 per node;
 * MILC moves neighbouring fields with gathers, Sec. 2) splits one lattice
 * across nodes.  Here the lattice is split along t: rank r of R owns the
 * global time slices [r T, (r + 1) T), T = Lt / R, which must be even and
 * >= 4.  Each rank's handle holds the links of an extended slab of T + 2 H
 * slices (H = STAG_DD_HALO): global slices r T - H .. r T + T + H - 1,
 * periodic in t, local slice t' = t - r T + H (canonical [V_ext][4][3][3]
 * complex double, V_ext = Lx Ly Lz (T + 2 H)).  Vectors are the rank's own
 * sites: [Lx Ly Lz T / 2][3] complex double, local index lex_local / 2 with
 * lex_local = x + Lx (y + Ly (z + Lz (t - r T))); a rank's even sites are
 * the global even sites.  Each application of D first exchanges the three
 * outermost own slices with the ranks above and below (the reach of the
 * Naik hops) through the caller's communicator; CG sums its inner products
 * over ranks through it.  FP64 (PLAIN64) only. */
#define STAG_DD_HALO 4

/* The caller's communicator.  Both calls get `stream`, the library's stream;
 * they must finish (or queue on `stream`) their transfers before any work
 * queued on `stream` after they return runs, and must wait for the work
 * already queued on `stream` before reading device memory (e.g.
 * cudaStreamSynchronize).  Return 0 on success.
 *   exchange     : send `bytes` from send_lo to the rank below (r - 1 mod R)
 *                  and from send_hi to the rank above (r + 1 mod R); receive
 *                  the rank below's send_hi into recv_lo and the rank above's
 *                  send_lo into recv_hi.  All four are device pointers into
 *                  the library's fields (contiguous).  With R = 1 the rank is
 *                  its own neighbour (periodic wrap).
 *   allreduce_sum: replace the n doubles at `values` (device) by their sum
 *                  over all ranks. */
typedef struct {
  void* ctx;
  int (*exchange)(void* ctx, const void* send_lo, const void* send_hi, void* recv_lo, void* recv_hi,
                  unsigned long long bytes, void* stream);
  int (*allreduce_sum)(void* ctx, double* values, int n, void* stream);
} stag_comm;

typedef struct stag_dd_s* stag_dd_t;

/* A rank's handle: gdims the global extents (even, >= 4), fat_ext/lng_ext
 * the extended slab's links (device, copied), opts as for stag_load_links
 * (an FP64 copy is built whatever prec_mask says).  EINVAL if Lt is not a
 * multiple of nranks or T = Lt / nranks is odd or below 4.  Synchronises. */
int stag_dd_create(stag_dd_t* out, const int gdims[4], int rank, int nranks, const void* fat_ext, const void* lng_ext,
                   const stag_link_opts* opts, void* stream);
int stag_dd_free(stag_dd_t d);
/* The rank's own extents {Lx, Ly, Lz, T}, its sites per parity and the
 * global t of its first slice.  Any output may be NULL. */
int stag_dd_info(stag_dd_t d, int local_dims[4], long long* vh_local, int* t_offset);
/* out = D in on the rank's own sites of parity out_parity (in: own sites of
 * the other parity).  Every rank must call it (it exchanges).  Synchronous
 * as far as the communicator is. */
int stag_dd_dslash(stag_dd_t d, void* out, const void* in, int out_parity, const stag_comm* comm, void* stream);
/* out = m^2 in - D_eo D_oe in on the rank's own even sites (two exchanges). */
int stag_dd_apply_m(stag_dd_t d, void* out, const void* in, double mass, const stag_comm* comm, void* stream);
/* FP64 CG on the split lattice (params->mode must be STAG_PLAIN64; tol,
 * max_iter, use_initial_guess, check_interval as for stag_cg): per
 * iteration two exchanges and two sums over ranks; when the iterated
 * residual reaches the target the true residual b - M x (summed over ranks)
 * decides, and CG restarts from it if it misses (info->reliable_updates
 * counts these checks).  x, b: the rank's own even sites.  Every rank must
 * call it with the same params; all ranks return the same status.
 * Synchronises `stream`. */
int stag_dd_cg(stag_dd_t d, void* x, const void* b, double mass, const stag_solve_params* params,
               stag_solve_info* info, const stag_comm* comm, void* stream);

/* Link construction before the operator (the paper's production code smears
 * the thin links before the solver: HISQ-link smearing, Sec. 1 and Sec. 2,
 * Fig. 1; the workload uses the three-staple fat link and the Naik link):
 *   F_mu(x) = c1 U_mu(x) + c_staple sum_{nu != mu} [ U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
 *                                                   + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ]
 *   L_mu(x) = c3 U_mu(x) U_mu(x+mu) U_mu(x+2mu)
 * (the benchmark workload: c1 = 1, c_staple = 1/8, c3 = -1/24), in FP64 on
 * the GPU, periodic boundaries, no staggered phases (stag_load_links folds
 * them in).  thin, fat, lng: device, canonical [V][4][3][3] complex double,
 * caller-owned; fat and lng must not overlap thin or each other
 * (STAG_EINVAL).  dims: even extents >= 4.  Asynchronous on `stream`. */
int stag_build_links(const int dims[4], const void* thin, void* fat, void* lng, double c1, double c_staple,
                     double c3, void* stream);

/* Symanzik one-loop improved gauge force (the paper's second benchmark
 * routine, Sec. 4.2, Figs. 6-8; the paper gives no formula, this is the
 * Luscher-Weisz form).  Action S = beta sum_loops c (1 - Re Tr W / 3) over
 * plaquettes (c_pl), 1x2 rectangles (c_rt) and parallelograms a, b, c, -a,
 * -b, -c over three directions (c_pg), each geometric loop once.  Output:
 *   force[x][mu] = (beta/3) TA[U_mu(x) Sigma_mu(x)],
 *   TA(M) = (M - M^dag)/2 - Tr(M - M^dag)/6,
 * Sigma_mu(x) = sum over the 6 + 18 + 24 loops through U_mu(x) of c times
 * the product of their other links (each loop traversing U_mu(x) forward),
 * so that U_mu(x) -> exp(eps X) U_mu(x) changes S by -eps Re Tr(X force).
 * FP64.  thin, force: device, canonical [V][4][3][3] complex double,
 * caller-owned, not overlapping (STAG_EINVAL).  dims: even extents >= 4.
 * Asynchronous on `stream`. */
int stag_gauge_force(const int dims[4], const void* thin, void* force, double beta, double c_pl, double c_rt,
                     double c_pg, void* stream);

/* Fermion force of the pseudofermion action of a rational approximation,
 *   S = sum_i alpha_i phi^dag (M + sigma_i)^{-1} phi,   M = m^2 - D_eo D_oe,
 * taken through the link construction of stag_build_links (fat link
 * c1 U + c_staple (staples), Naik link c3 U U U): the paper's third benchmark
 * routine, the HISQ fermion force (Sec. 4.2; the paper gives no formula).
 * With X_i = (M + sigma_i)^{-1} phi on even sites and Y_i = D_oe X_i on odd
 * sites (the caller solves, e.g. with stag_multishift_cg, and applies
 * stag_dslash), the output is
 *   force[y][nu] = -TA[U_nu(y) Z_nu(y)],  TA(A) = (A - A^dag)/2 - Tr(A - A^dag)/6,
 * with dS = sum Re Tr[dU_nu(y) Z_nu(y)], so that U_nu(y) -> exp(eps X)
 * U_nu(y) changes S by -eps Re Tr(X force) (the convention of
 * stag_gauge_force).  FP64.
 *   thin    : device, canonical [V][4][3][3] complex double, caller-owned.
 *   x_even  : device, [n_terms][V/2][3] complex double, X_i (checkerboard
 *             index lex / 2, the layout of every field of this API).
 *   y_odd   : device, [n_terms][V/2][3] complex double, Y_i.
 *   alpha   : host, n_terms weights; 1 <= n_terms <= 32.
 *   force   : device, canonical [V][4][3][3] complex double, caller-owned,
 *             not overlapping thin, x_even or y_odd (STAG_EINVAL).
 * dims: even extents >= 4.  Scratch: 2 V x 4 x 9 complex doubles
 * (1152 B per site), stream-ordered (STAG_ENOMEM if unavailable).
 * Asynchronous on `stream`; profiler family "fermion_force". */
int stag_fermion_force(const int dims[4], const void* thin, int n_terms, const void* x_even, const void* y_odd,
                       const double* alpha, double c1, double c_staple, double c3, void* force, void* stream);

/* Check of this build's tensor-core path on the current GPU (the path the
 * network's 16 -> 16 layers take): one tile of tcgen05 bfloat16 products
 * with FP32 accumulation in tensor memory, 9 accumulated steps, compared
 * with the same sums on the CUDA cores.  *max_rel_err: max |difference| /
 * max |reference| (0 expected: the test values are exact in both).
 * STAG_ETIMEOUT if a bounded wait gave up.  Synchronous.  No counterpart in
 * the paper, which predates these tensor cores. */
int stag_tc_selftest(double* max_rel_err);

/* Human-readable text of a status code (static storage). */
const char* stag_strerror(int status);

/* ---------------------------------------------------------- instrumentation
 * When enabled, every kernel the library launches is bracketed by a pair of
 * CUDA events recorded on its launch stream; stag_profile_read returns, for
 * a kernel family name, the number of launches and their summed device
 * time (ms).  Families: "dslash", "dslash_epi" (FP32 and 16-bit operator,
 * plain and with the fused axpy/reduction epilogue), "dslash64",
 * "dslash64_epi" (FP64), "dslash_mrhs", "dslash_mrhs_epi", "dslash_mrhs64",
 * "dslash_mrhs64_epi" (multi-right-hand-side forms), "dslash_df",
 * "dslash_df_epi" (double-float), "blas", "reduce",
 * "convert", "links", "net" (network forward layers), "net_tc" (the
 * 16 -> 16 tensor-core layers of the forward), "net_bwd", "gauge_force",
 * "fermion_force".  stag_launch_count
 * counts all library kernel launches since the last reset, whether or not
 * profiling is on. */
int stag_profile_enable(int on);
/* Restrict the event pairs to the listed families (comma-separated, e.g.
 * "dslash,dslash_epi"; NULL or "" times every family) and to one launch in
 * `every` of each family (every <= 1: all), which keeps the events' own cost
 * out of the measured workload.  With every > 1 the solvers drop the samples
 * of a chunk of queued iterations that a stop flag (a reliable-update
 * trigger, convergence) cut short, whose later launches return at once: the
 * sampled averages then time launches that did their work.  With every <= 1
 * all launches count. */
int stag_profile_select(const char* families, int every);
/* Zero every family's launch count and time, and the launch counter. */
int stag_profile_reset(void);
/* Launches and summed device time (ms) of one family since the last reset
 * (waits for the pending events).  Unknown family: 0 launches; NULL family:
 * EINVAL. */
int stag_profile_read(const char* family, long long* launches, double* total_ms);
/* All library kernel launches since the last reset. */
long long stag_launch_count(void);

/* The bounds-checked build (libstag_debug.so, compiled with
 * -DSTAG_DEBUG_BOUNDS; compute-sanitizer is not available to this library's
 * tests) checks every neighbour index of the stencil, every site index of a
 * vector load or store and the site index of every link load against its
 * extent; an out-of-range index is counted, the access redirected to index
 * 0, and the kernel completes.  *count: violations since the last clear
 * (waits for the device first), *first_code the kind of the first one (1:
 * neighbour, 2: vector site, 3: link site) and *first_index its index;
 * clear != 0 resets the records.  The normal build reports *count = -1.
 * No counterpart in the paper. */
int stag_bounds_violations(long long* count, int* first_code, long long* first_index, int clear);

#ifdef __cplusplus
}
#endif
#endif /* STAG_H */
