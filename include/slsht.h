/*
 * slsht.h -- C ABI of libslsht, a GB300 (sm_103a) implementation of the
 * directional spatially localised spherical harmonic transform (directional
 * SLSHT) of Khalid, Kennedy, Durrani, Sadeghi, Wiaux and McEwen,
 * arXiv:1207.5558.
 *
 * What is computed (Sec. III-A, Definition 1, Eq. stft_spatial): for a signal
 * f and a window h on the sphere, given by spherical-harmonic coefficients,
 *     g(rho; l, m) = int_{S^2} f(x) (D_rho h)(x) conj(Y_l^m(x)) ds(x),
 * sampled on an equiangular grid of rotations rho = (alpha, beta, gamma)
 * (Sec. II-D, the tessellation E_L, generalised to independent sizes):
 *     alpha_a = 2 pi a / n_alpha,  beta_b = 2 pi b / (2 n_beta - 1),
 *     gamma_c = 2 pi c / n_gamma.
 * Rotations are zyz Euler angles acting as (D_rho h)(x) = h(R^{-1} x) with
 * R = R_z(alpha) R_y(beta) R_z(gamma) (Sec. II-B, Eq. rotation_non_symm,
 * Eq. Dlm).  The inverse recovers f_lm = fhat_lm / (sqrt(16 pi^3) h_0^0) with
 * fhat_lm = int_SO(3) g(rho; l, m) drho (Sec. III-C, Eq. inversion_1,
 * Eq. inversion_2, Eq. sig_reconstruction_discrete).
 *
 * Conventions shared by every entry point
 *  - Band limits are EXCLUSIVE: f_lm = 0 for l >= L_f, h_pq = 0 for p >= L_h
 *    (the paper's inclusive band limit is L - 1).  g(rho; l, m) is non-zero
 *    only for l <= L_f + L_h - 2.
 *  - Spherical harmonics carry the Condon-Shortley phase
 *    (Y_l^{-m} = (-1)^m conj Y_l^m), Eq. Sph_harmonics.
 *  - Coefficient vectors are complex128 stored as interleaved (re, im)
 *    doubles, flat index l*l + l + m: f_lm has L_f*L_f entries, h_lm L_h*L_h.
 *  - Pair lists are int32 [n_pairs][2] = (l, m), 0 <= l <= L_f + L_h - 2,
 *    |m| <= l.
 *  - g is laid out [pair][a][b][c] (gamma fastest, then beta, then alpha),
 *    interleaved complex: complex128 for SLSHT_FP64, complex64 for
 *    SLSHT_FP32_BULK.  One pair occupies n_alpha*n_beta*n_gamma samples.
 *  - Memory spaces: every pointer argument may be host or device memory of
 *    the context's device unless stated otherwise; the library detects which
 *    (cudaPointerGetAttributes).  Host outputs are filled by stream-ordered
 *    copies: synchronise the stream before reading them.
 *  - The caller owns every buffer it passes; the context owns its cached
 *    device tables and scratch.  Nothing is retained after a call returns.
 *  - All work is issued on the caller's CUDA stream (cudaStream_t passed as
 *    void*; NULL = legacy default stream) and is asynchronous: argument
 *    validation happens before anything is enqueued and is synchronous.
 *  - Errors: every int-returning call returns SLSHT_OK (0) or a negative
 *    SLSHT_E_* code; slsht_strerror() describes it.  No exception crosses the
 *    ABI.  On an error nothing has been enqueued unless the code is
 *    SLSHT_E_CUDA (a CUDA call failed; the message of the last failure is
 *    available from slsht_last_error()).
 *  - There is no CPU fallback: every step of the transform runs in this
 *    library's CUDA kernels.
 */
#ifndef SLSHT_H
#define SLSHT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define SLSHT_OK          0
#define SLSHT_PENDING     1   /* slsht_poll: request admitted, not finished   */
#define SLSHT_E_ARG      -1   /* invalid argument (sizes, indices, null)      */
#define SLSHT_E_H00      -2   /* inverse with h_0^0 == 0 (Eq. inversion_2)    */
#define SLSHT_E_NOMEM    -3   /* allocation failed or over the memory budget  */
#define SLSHT_E_BUSY     -4   /* serving queue full; retry later              */
#define SLSHT_E_TIMEOUT  -5   /* a bounded device-side wait gave up           */
#define SLSHT_E_CUDA     -6   /* a CUDA runtime/driver call failed            */
#define SLSHT_E_STATE    -7   /* unknown ticket / context misuse              */

/* ---------------------------------------------------------------- types */
typedef struct slsht_ctx slsht_ctx;   /* opaque; one device, owns tables */

typedef enum {
  SLSHT_FP64 = 0,       /* FP64 accuracy (relative error <= 1e-12): 3j,
                           Delta, coupling and rotated window in FP64, X and
                           the alpha sum in FP64, double-float or exact
                           digit-product tensor-core arithmetic
                           (SLSHT_OPT_FP64_ARITH); g is complex128           */
  SLSHT_FP32_BULK = 1   /* 3j, Delta, phases in FP64; coupling in FP64;
                           beta/gamma sums in FP32; alpha stage on tcgen05
                           tensor cores (split-FP16 operands, FP32
                           accumulate); g is complex64                      */
} slsht_prec;

typedef struct {
  int32_t L_f;        /* signal band limit (exclusive), >= 1              */
  int32_t L_h;        /* window band limit (exclusive), 1 <= L_h <= 64    */
  int32_t n_alpha;    /* grid sizes, each >= 1                            */
  int32_t n_beta;
  int32_t n_gamma;
  int32_t prec;       /* slsht_prec                                       */
} slsht_desc;

/* Per-stage device timings, filled when profiling is on (slsht_profile). */
#define SLSHT_NSTAGES 8
enum {
  SLSHT_STAGE_TABLES = 0,  /* Delta recursion, d(beta) tables, phase tables */
  SLSHT_STAGE_COUPLE = 1,  /* 3j chains + Gaunt coupling k_lm(p, q)         */
  SLSHT_STAGE_CTENSOR = 2, /* C_{q,q',q''} tensor (factoring-of-rotations)  */
  SLSHT_STAGE_BETA = 3,    /* beta and gamma sums                           */
  SLSHT_STAGE_ALPHA = 4,   /* alpha sum and store of g                      */
  SLSHT_STAGE_INVERSE = 5, /* SO(3) quadrature reduction                    */
  SLSHT_STAGE_COPY = 6,    /* host<->device copies issued by the library    */
  SLSHT_STAGE_OTHER = 7
};
typedef struct {
  uint64_t launches[SLSHT_NSTAGES];  /* kernel launches (copies for COPY)   */
  double   ms[SLSHT_NSTAGES];        /* summed device time, milliseconds    */
  uint64_t samples_written;          /* g samples written by forward calls  */
} slsht_stats;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  `mem_budget_bytes` caps the
 * device memory the context may hold for tables and scratch (0 = 8 GiB).
 * Returns SLSHT_E_ARG (ctx NULL / bad device), SLSHT_E_CUDA. */
int slsht_create(slsht_ctx** ctx, int device, size_t mem_budget_bytes);

/* Synchronise the context's own streams and free everything it owns.
 * NULL is a no-op. */
void slsht_destroy(slsht_ctx* ctx);

/* ---------------------------------------------------------------- window */

/* The band-limited window of maximal energy concentration in the elliptical
 * region R(theta_c, a) of Sec. III-D (Eq. region_def: points whose
 * great-circle distances to the foci (theta_c, 0) and (theta_c, pi) add up
 * to at most 2a), computed on the device: the concentration matrix over the
 * real even harmonics (the region is symmetric under phi -> -phi) by
 * quadrature ring by ring, then its top eigenpair by block subspace
 * iteration.
 *   L            exclusive band limit, 1..256
 *   theta_c, a   focal colatitude and semi-major arc, radians,
 *                0 <= theta_c <= a < pi/2
 *   n_phi, n_theta  quadrature longitudes / Gauss-Legendre nodes per ring
 *                (0: 8L+64 and 2L+24)
 *   h_out        complex128 [L*L] (host or device), flat index l*l+l+m:
 *                unit energy, real-valued, symmetric under phi -> -phi,
 *                h_0^0 > 0
 *   concentration  optional host double: the eigenvalue (fraction of the
 *                window's energy inside R)
 * Synchronous.  Errors: SLSHT_E_ARG, SLSHT_E_NOMEM (context budget: the
 * quadrature matrix is n_phi*n_theta*L(L+1)/2 doubles), SLSHT_E_TIMEOUT (the
 * iteration did not converge), SLSHT_E_CUDA. */
int slsht_window_ellipse(slsht_ctx* ctx, int32_t L, double theta_c, double a, int32_t n_phi, int32_t n_theta,
                         double* h_out, double* concentration, void* stream);

/* ---------------------------------------------------------------- forward */

/* g(rho; l, m) for every listed pair on the desc's grid (Definition 1,
 * evaluated through the convolution form Eq. alternative_harmonic_formulation
 * with Gaunt coupling, Wigner-d from the Delta = d(pi/2) recursion of
 * Sec. IV-B and separable beta / gamma / alpha sums).
 *   f_lm  complex128 [L_f*L_f]        (host or device)
 *   h_lm  complex128 [L_h*L_h]        (host or device)
 *   lm    int32 [n_pairs][2]          (host or device)
 *   g_out [n_pairs][n_alpha][n_beta][n_gamma] complex128 (FP64) or complex64
 *         (FP32_BULK), device or host, 8-byte aligned, caller-owned.
 * n_pairs == 0 is valid and does nothing.  Errors: SLSHT_E_ARG (null ctx /
 * desc / pointers, L_f < 1, L_h < 1 or > 64, a grid size < 1, unknown prec,
 * l outside [0, L_f+L_h-2], |m| > l), SLSHT_E_NOMEM, SLSHT_E_CUDA. */
int slsht_forward(slsht_ctx* ctx, const slsht_desc* desc,
                  const double* f_lm, const double* h_lm,
                  const int32_t* lm, int32_t n_pairs,
                  void* g_out, void* stream);

/* g for n_windows windows over the same signal and pair list (Sec. IV-B,
 * the remark on analysing one signal with several windows): the coupling
 * k_lm (window independent) is formed once; everything per window (the
 * rotated window H and the alpha stage) runs for each.  Equal to n_windows
 * slsht_forward calls with the same f and lm.
 *   h_lms  complex128 [n_windows][L_h*L_h]          (host or device)
 *   g_out  [n_windows][n_pairs][n_alpha][n_beta][n_gamma], as slsht_forward.
 * Other arguments and errors as slsht_forward; n_windows < 0 is SLSHT_E_ARG,
 * 0 does nothing. */
int slsht_forward_windows(slsht_ctx* ctx, const slsht_desc* desc, const double* f_lm, int32_t n_windows,
                          const double* h_lms, const int32_t* lm, int32_t n_pairs, void* g_out, void* stream);

/* ---------------------------------------------------------------- inverse */

/* f_lm for every listed pair from sampled g (Eq. inversion_1, inversion_2,
 * with the exact SO(3) quadrature of Eq. sig_reconstruction_discrete
 * generalised to the desc's grid):
 *   f_lm = (2 pi/n_alpha)(2 pi/n_gamma) sum_{a,b,c} q_b g[a][b][c]
 *          / (sqrt(16 pi^3) h_0^0),
 * with q_b the beta weights of the printed w(m) rule.  Exact when the grid
 * resolves the window: n_alpha, n_beta, n_gamma >= L_h.
 *   g_in   device buffer laid out as slsht_forward's g_out (desc->prec
 *          selects complex128 / complex64)
 *   h00    host double[2], the window's (re, im) h_0^0
 *   lm     int32 [n_pairs][2] (host or device; only used for validation)
 *   f_out  complex128 [n_pairs] (host or device)
 * Errors: SLSHT_E_ARG (as forward, plus a grid size < L_h, or g_in not in
 * device memory), SLSHT_E_H00 (h_0^0 == 0), SLSHT_E_NOMEM, SLSHT_E_CUDA.
 * The reduction order is fixed: results are bitwise reproducible. */
int slsht_inverse(slsht_ctx* ctx, const slsht_desc* desc,
                  const void* g_in, const double h00[2],
                  const int32_t* lm, int32_t n_pairs,
                  double* f_out, void* stream);

/* f_lm without the condition h_0^0 != 0: the reconstruction of the remark
 * after Eq. inversion_2 (Sec. III-C).  The projection of g(.; l, m) on
 * conj(D^p_{q,q'}) over SO(3) is 8 pi^2/(2p+1) k_lm(p, q) h_p^q'
 * (Eq. WignerD_ortho); summing it against conj(h_p^q') leaves the window's
 * energy at degree p, E_p = sum_q' |h_p^q'|^2, times k_lm(p, q); and the
 * Wigner-3j orthogonality over q decouples the signal:
 *   f_LM = (2L+1)/c^2 sum_q T(L, M; p, q; L+p, M+q) khat_{L+p, M+q}(q),
 * c^2 = (2L+1)(2p+1)(2L+2p+1)/(4 pi) (L p L+p; 0 0 0)^2.
 *   g_in   device buffer laid out as slsht_forward's g_out for the pairs
 *          lm_in (desc->prec selects complex128 / complex64)
 *   h_lm   complex128 [L_h*L_h] (host or device): the window of g_in
 *   lm_in  int32 [n_in][2] (host or device): the pairs of g_in's rows
 *   p      the window degree used, 0 <= p < L_h, with E_p > 0; the
 *          distribution must hold, for each output (L, M), every pair
 *          (L + p, M + q) with |q| <= p
 *   lm_out int32 [n_out][2] (host or device): the (L, M) to recover,
 *          0 <= L < L_f, |M| <= L
 *   f_out  complex128 [n_out] (host or device)
 * Exact (to rounding) when n_alpha, n_beta, n_gamma >= L_h + p.  Device
 * argument arrays are read on `stream` after the work queued there; the call
 * returns when its work is done.  Errors: SLSHT_E_ARG (as slsht_inverse,
 * plus p out of range, a grid size < L_h + p, an output outside the signal
 * band, or a missing pair), SLSHT_E_H00 (E_p == 0), SLSHT_E_NOMEM,
 * SLSHT_E_CUDA.  Fixed reduction order: bitwise reproducible. */
int slsht_inverse_alt(slsht_ctx* ctx, const slsht_desc* desc, const void* g_in, const double* h_lm,
                      const int32_t* lm_in, int32_t n_in, int32_t p, const int32_t* lm_out, int32_t n_out,
                      double* f_out, void* stream);

/* g at arbitrary orientations gamma from the grid's gamma samples (Sec. IV-B,
 * the remark on steerable windows: by linearity the distribution at any
 * gamma follows from a few basis orientations).  g depends on gamma only
 * through e^{-i q' gamma} for the window's orders |q'| <= Q, so with
 * n_gamma >= 2Q + 1 samples it is recovered exactly at any gamma by the
 * trigonometric interpolation of that band:
 *   g(gamma) = sum_c g(gamma_c) (1 + 2 sum_{q'=1..Q} cos(q' (gamma - gamma_c))) / n_gamma.
 * Q = L_h - 1 serves any window; a steerable window (h_p^q' = 0 for |q'| >= N)
 * needs only Q = N - 1, i.e. 2N - 1 basis orientations.
 *   g_in    device, laid out as slsht_forward's g_out for n_pairs pairs
 *   gammas  double [n_g] angles in radians (host or device)
 *   g_out   device [n_pairs][n_alpha][n_beta][n_g], same precision as g_in
 * Errors: SLSHT_E_ARG (bad desc, Q outside [0, L_h - 1], n_gamma < 2Q + 1,
 * g_in or g_out not in device memory), SLSHT_E_NOMEM, SLSHT_E_CUDA.  The
 * weights and sums are FP64. */
int slsht_steer_gamma(slsht_ctx* ctx, const slsht_desc* desc, const void* g_in, int32_t n_pairs,
                      const double* gammas, int32_t n_g, int32_t Q, void* g_out, void* stream);

/* ---------------------------------------------------------------- no-alloc */

/* Size of the static device scratch array behind slsht_forward_noalloc. */
#define SLSHT_NOALLOC_SCRATCH_BYTES (32u << 20)

/* The forward transform for callers that cannot allocate device memory when
 * they need it: real-time sections where cudaMalloc's implicit
 * synchronisation is not allowed, plug-ins whose host application owns the
 * device allocator, and processes that have given the whole device to a
 * fixed pool.  Call it from ordinary host code: it calls the CUDA runtime,
 * which a function queued with cudaLaunchHostFunc (or a stream callback) may
 * not do.  The paper has no counterpart to this call.
 * It needs no context and allocates nothing: it works in one static device
 * array of SLSHT_NOALLOC_SCRATCH_BYTES that every GPU loading this library
 * holds until the process exits.  Arguments, layouts and results are those of
 * slsht_forward, except that g_out must be device memory; FP32_BULK runs its
 * alpha stage on CUDA cores here.  Tables are rebuilt on every call; pairs are
 * processed in chunks that fit the array.
 *  - Requests whose tables plus one pair exceed the array are rejected with
 *    SLSHT_E_NOMEM before anything is enqueued (slsht_last_error explains).
 *  - A pair list in device memory is validated by reading it on `stream`
 *    (after the work queued there before the call) and synchronising that
 *    stream, so such a call blocks until the stream's earlier work is done;
 *    pass lm in host memory for a call that must not block.  The kernels read
 *    the device list again later in stream order: leave it unchanged until
 *    the call's work has completed.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current: make that first call
 *    before any stream capture.
 *  - Calls share the array and it keeps the last call's contents: calls whose
 *    work can overlap on the GPU race with each other; order them on one
 *    stream (or with events). */
int slsht_forward_noalloc(const slsht_desc* desc, const double* f_lm, const double* h_lm,
                          const int32_t* lm, int32_t n_pairs, void* g_out, void* stream);

/* ---------------------------------------------------------------- batches */

/* One analysis of a batch plan: a signal, a window, a pair list and a grid,
 * each with its own band limits, sizes and precision.  f_lm, h_lm and g_out
 * are DEVICE pointers bound to the plan: every slsht_batch_launch reads the
 * coefficients they hold at that time and writes g_out (layout and size as for
 * slsht_forward; g_out 16-byte aligned).  lm may be host or device memory and
 * is copied when the plan is created. */
typedef struct {
  slsht_desc desc;
  const double* f_lm;   /* device, L_f*L_f complex128 */
  const double* h_lm;   /* device, L_h*L_h complex128 */
  const int32_t* lm;    /* n_pairs x (l, m) */
  int32_t n_pairs;      /* >= 1 */
  void* g_out;          /* device */
} slsht_batch_item;

typedef struct slsht_batch slsht_batch;   /* opaque plan */

/* Flags of slsht_batch_create. */
#define SLSHT_BATCH_NO_GRAPH 1   /* enqueue the kernels one by one at each launch
                                    instead of replaying a captured CUDA graph */
#define SLSHT_BATCH_NO_TUNE  2   /* tile shapes from the built-in rule instead of
                                    timing the candidates */
#define SLSHT_BATCH_NO_TC    4   /* keep FP32_BULK items on CUDA cores */
#define SLSHT_BATCH_NO_DD    8   /* FP64 items in FP64 arithmetic only */
#define SLSHT_BATCH_FP64_DD 16   /* FP64 items in double-float arithmetic only */

/* Plan many analyses (maps, windows, requests of uneven band limits and grids)
 * as one unit.  Per launch the plan runs: the Gaunt gather-sum of every pair
 * of every item (one kernel); every distinct rotated window (one kernel); the
 * alpha stage of every CUDA-core item as ONE persistent kernel per precision,
 * whose CTAs take (item, pair, column block) tiles from a shared counter; and
 * one fused tensor-core launch per FP32_BULK item that the tuner gave to the
 * tensor cores.  These launches are captured once into a CUDA graph that each
 * slsht_batch_launch replays.
 *  - Signal-independent work is done here, once: the Gaunt coefficient table
 *    of every distinct (L_f, L_h, pair list) (Sec. III-B), the Delta and
 *    d(beta) tables and the phase tables (shared with the context's cache).
 *  - Tile shapes: for every distinct (precision, L_h, N_alpha, N_beta,
 *    N_gamma) the autotuner times each candidate (columns per tile 32/64/128;
 *    direct alpha sum or split DFT with each odd factor 3/5/7/9 of N_alpha;
 *    for FP32_BULK the fused tensor-core kernel; for FP64 the X and alpha
 *    sums in FP64 or in double-float arithmetic) on the item's own data into
 *    plan scratch, and keeps the fastest per sample.  The choice is cached in
 *    the context for later plans of the same shape.
 *  - Double-float engine (FP64 items): X and the alpha sum carried as pairs of
 *    floats (about 48 significant bits, from exact TwoProd/TwoSum steps on the
 *    FP32 pipe, which GB300 issues at 64 times its FP64 rate), k and the
 *    rotated window scaled by powers of two into the float range, every g
 *    sample assembled as a double with its scale: relative L2 error about
 *    1e-14, inside the FP64 path's 1e-12.
 *  - Memory: tables, k, the rotated windows and the tile lists are plan-owned
 *    and counted against the context's budget.
 *  - Creation is synchronous: it waits for `stream` (so f and h may be
 *    written on it just before), builds the tables, tunes, runs the plan once
 *    (so every g_out holds its result when the call returns) and captures the
 *    graph, all on its own stream, and returns when they are complete.
 * Errors: SLSHT_E_ARG (null ctx/items/out, n_items < 1, a bad descriptor or
 * pair list, an f/h/g_out not in device memory, g_out misaligned),
 * SLSHT_E_NOMEM, SLSHT_E_CUDA.  On error *out is NULL and nothing is kept. */
int slsht_batch_create(slsht_ctx* ctx, int32_t n_items, const slsht_batch_item* items, int32_t flags,
                       void* stream, slsht_batch** out);

/* Enqueue one evaluation of every item of the plan on `stream`.  Launches of
 * one plan share its scratch (k, rotated windows, tile counter): order them
 * (one stream or events) and do not launch one plan from two threads at once. */
int slsht_batch_launch(slsht_batch* batch, void* stream);

/* Facts about a plan (item ignored where it says so):
 *  SLSHT_BQ_TILE_COLS  item's columns per tile (0 on the tensor cores)
 *  SLSHT_BQ_ALPHA_FORM item's alpha form: 0 direct sum, 3/5/7/9 split DFT with
 *                      that factor, -1 fused tensor-core kernel
 *  SLSHT_BQ_TUNED      item's shape: 1 timed by this plan, 2 taken from the
 *                      context's cache, 0 built-in rule (SLSHT_BATCH_NO_TUNE)
 *  SLSHT_BQ_TILES      CUDA-core tiles per launch (item ignored)
 *  SLSHT_BQ_KERNELS    kernels per launch (item ignored)
 *  SLSHT_BQ_GRAPH      1 if launches replay a CUDA graph (item ignored)
 *  SLSHT_BQ_BYTES      device memory the plan holds (item ignored)
 *  SLSHT_BQ_SAMPLES    g samples per launch (item ignored)
 *  SLSHT_BQ_ENGINE     item's arithmetic: 0 its precision on CUDA cores, 1
 *                      double-float on CUDA cores (FP64 items), 2 tensor cores
 * Returns SLSHT_OK or SLSHT_E_ARG. */
#define SLSHT_BQ_TILE_COLS  1
#define SLSHT_BQ_ALPHA_FORM 2
#define SLSHT_BQ_TUNED      3
#define SLSHT_BQ_TILES      4
#define SLSHT_BQ_KERNELS    5
#define SLSHT_BQ_GRAPH      6
#define SLSHT_BQ_BYTES      7
#define SLSHT_BQ_SAMPLES    8
#define SLSHT_BQ_ENGINE     9
int slsht_batch_query(const slsht_batch* batch, int32_t item, int32_t what, int64_t* value);

/* Measure the tile shapes of one grid shape now: the same autotuner as
 * slsht_batch_create (every candidate timed on seeded synthetic
 * coefficients of that shape, a few pairs of degree L_f - 1), its choice
 * cached in the context (for FP32_BULK also the shape on CUDA cores alone).
 * slsht_forward reads the cache for the CUDA-core alpha kernels of FP64 calls
 * (double-float engine) and slsht_submit for every request's alpha tiles;
 * without an entry they use a built-in rule.  Synchronous; returns SLSHT_OK,
 * SLSHT_E_ARG, SLSHT_E_NOMEM or SLSHT_E_CUDA. */
int slsht_tune(slsht_ctx* ctx, const slsht_desc* desc);

/* Wait for the plan's last launch and free everything it holds.  NULL is a
 * no-op.  slsht_destroy frees the plans of its context that are still alive;
 * a plan must not be used (or destroyed) after its context. */
void slsht_batch_destroy(slsht_batch* batch);

/* ---------------------------------------------------------------- serving */

/* Non-blocking forward request for a continuous-batching server.  The
 * library copies f_lm, h_lm and lm before returning (host or device input);
 * g_out must be DEVICE memory and stay valid until the request completes.
 * A worker thread evaluates the requests in ticks: each tick takes a chunk of
 * pairs from every started request (oldest first; a large request is spread
 * over several ticks, so requests that arrive behind it are not held up) and
 * from newly arrived ones while its arena has room (admission by memory), and
 * runs them as ONE set of persistent batched kernels -- the 3j-chain
 * coupling, the rotated windows, and one alpha kernel per arithmetic whose
 * blocks take tiles from a counter -- replayed from a captured CUDA graph.
 * Two ticks can be on the device at once.  The alpha stage runs on CUDA
 * cores (FP64 requests in double-float arithmetic unless the tuner cache of
 * the context says otherwise; slsht_tune fills it), with the tile shape of
 * the request's grid shape, so a request's g does not depend on the requests
 * it shares ticks with.  *ticket receives the request id.  Returns SLSHT_OK,
 * SLSHT_E_BUSY (more than 4096 requests unfinished), SLSHT_E_NOMEM (one pair
 * exceeds a tick's arena), or the errors of slsht_forward (validation is
 * synchronous). */
int slsht_submit(slsht_ctx* ctx, const slsht_desc* desc,
                 const double* f_lm, const double* h_lm,
                 const int32_t* lm, int32_t n_pairs,
                 void* g_out, uint64_t* ticket);

/* SLSHT_OK if the request's g_out is complete (and device-visible),
 * SLSHT_PENDING if not yet, or the request's error code.  A ticket can be
 * polled until it has returned a final status once; then it is forgotten
 * (SLSHT_E_STATE afterwards). */
int slsht_poll(slsht_ctx* ctx, uint64_t ticket);

/* slsht_poll that also reports, once the request has finished, its times
 * in milliseconds: times[0] queue (submission to its first tick), times[1]
 * host issue (building and launching its first tick), times[2] device (start
 * of its first tick to the end of its last, device clock), times[3] total
 * (submission to the completion seen by the worker).  times may be NULL. */
int slsht_poll_times(slsht_ctx* ctx, uint64_t ticket, double* times);

/* Block until every submitted request has finished (bounded by timeout_ms;
 * SLSHT_E_TIMEOUT if it expires). */
int slsht_drain(slsht_ctx* ctx, int64_t timeout_ms);

/* ---------------------------------------------------------------- tools */

/* Human-readable text for a status code (static storage). */
const char* slsht_strerror(int code);

/* Text of the most recent SLSHT_E_CUDA failure in this process. */
const char* slsht_last_error(void);

/* Validate a descriptor and pair list without touching the GPU (host memory
 * only).  Returns SLSHT_OK or SLSHT_E_ARG. */
int slsht_check_args(const slsht_desc* desc, const int32_t* lm_host, int32_t n_pairs);

/* Turn per-stage device timing on (1) or off (0).  While on, every kernel
 * launch and library copy is bracketed by CUDA events on its stream. */
int slsht_profile(slsht_ctx* ctx, int enable);

/* Read (and with reset != 0 clear) the per-stage statistics.  Synchronises
 * on the recorded events. */
int slsht_get_stats(slsht_ctx* ctx, slsht_stats* out, int reset);

/* Execution options of a context (defaults 0 = automatic):
 *  SLSHT_OPT_BETA_ROUTE   1: beta sum from a table of d^p(beta_b) built from
 *                            Delta (separation of variables, Sec. IV-B remark);
 *                         2: factoring of rotations: C tensor
 *                            (Eq. constant_alternative_formulation) + DFT in q''.
 *  SLSHT_OPT_ALPHA_ENGINE 1: CUDA cores (the alpha index split as
 *                            a = Q s + t with a small odd factor P of n_alpha
 *                            when that saves work, else the direct sum);
 *                            2: tcgen05 tensor cores fed by a separate
 *                            producer kernel; 3: one fused kernel (producer
 *                            warps build the tensor-core operand in shared
 *                            memory; route 1 only); 4: CUDA cores, direct sum
 *                            only.  Tensor cores: FP32_BULK with L_h <= 16
 *                            (2 and 3), and the wide engine for
 *                            16 < L_h <= 64 (orders +-q paired, producer in
 *                            two passes), which 0 and 2 select there.
 *                            0 (default): 3 where it applies, else 2, else 1.
 *  SLSHT_OPT_CHUNK_PAIRS  pairs per launch chunk (scratch size).
 *  SLSHT_OPT_GAUNT_TABLE  the 3j part of the coupling (Sec. III-B: T through
 *                            Wigner-3j symbols) depends only on (L_f, L_h, the
 *                            pair list): 0 (default): each workspace keeps
 *                            the table of the last pair list it saw when it
 *                            fits in 256 MB, and a call with the same list
 *                            only gathers k = sum T f; 1: always keep it;
 *                            2: never (3j chains recomputed in every call).
 *  SLSHT_OPT_WAIT_TEST    1: the next forward call that runs a tensor-core
 *                            kernel (the fused, two-kernel, wide or FP64
 *                            digit-product alpha engine, or the rotated window
 *                            of SLSHT_OPT_ROTWIN_ENGINE 2, which takes it
 *                            first) withholds one internal
 *                            hand-off in its first launch, so the kernel's
 *                            bounded waits expire, it exits cleanly and the
 *                            next slsht_get_stats returns SLSHT_E_TIMEOUT;
 *                            that call's g is not computed.  Resets itself.
 *                            For testing the timeout path; the context stays
 *                            usable.
 *  SLSHT_OPT_REAL_FIELDS  1: the caller guarantees that f and h are real
 *                            fields (f_{l,-m} = (-1)^m conj f_lm, and the same
 *                            for h).  Then g(rho; l, -m) = (-1)^m conj
 *                            g(rho; l, m), and of every pair whose mirror
 *                            (l, -m) is also listed only one is computed:
 *                            the alpha stage stores both outputs (device g_out
 *                            only; host g_out is computed in full).  0: off.
 *  SLSHT_OPT_COUPLING     1 (default 0 = 1): k by Gaunt coefficients (3j
 *                            recurrences, Sec. III-B); 2: k by the spherical
 *                            harmonic transform of the modulated signal
 *                            (Appendix A: Gauss-Legendre quadrature of the
 *                            band-limited triple products), cheaper when the
 *                            window band is wide and the signal band narrow;
 *                            rounding limits it to ~1e-11 relative near
 *                            l = 255.
 *  SLSHT_OPT_FP64_ARITH   FP64 calls on the rotated-window route (tables,
 *                            3j, coupling and the rotated window in FP64
 *                            throughout): 0 (default) = 2 where it applies,
 *                            else 3; 1: X and the alpha sum in FP64
 *                            arithmetic; 2 (L_h <= 16, alpha engine not held
 *                            to CUDA cores): X in double-float, the alpha
 *                            sum on the tensor cores from base-256 digits of
 *                            X and of the cos/sin tables (7 digits each, 28
 *                            digit products whose FP32 sums are exact),
 *                            combined by TwoSum into a double-float and
 *                            assembled as a double; 3: X and the alpha sum
 *                            in double-float arithmetic on CUDA cores (pairs
 *                            of floats from exact TwoProd/TwoSum steps, about
 *                            48 significant bits).  Relative error about
 *                            1e-14 for 0, 2 and 3.
 *  SLSHT_OPT_WINDOW_ORDERS 1: the rotated window (the window turned to every
 *                            (beta, gamma) sample) sums only over the orders
 *                            q' at which the window has a non-zero
 *                            coefficient at some degree (found on the device
 *                            from h in every call).  A steerable window --
 *                            azimuthally band-limited, h_p^q' = 0 for
 *                            |q'| >= N < L_h (Sec. IV-B) -- then costs
 *                            (2N-1)/(2p+1) of the full sum at degree p; the
 *                            terms left out are zero, so g is unchanged.
 *                            2: as 1, also leaving out orders whose
 *                            coefficients are at most 2^-40 (FP32_BULK) or
 *                            2^-52 (FP64) of the largest one: windows whose
 *                            vanishing orders carry rounding noise only (the
 *                            concentration window of an ellipse centred on
 *                            the pole has its odd orders at that level).
 *                            0 (default): every order.
 *  SLSHT_OPT_ROTWIN_ENGINE FP32_BULK calls: the rotated window on 1 the
 *                            CUDA cores, or 2 the tensor cores where they
 *                            apply (n_gamma <= 128); 0, the default: the
 *                            tensor cores for L_h > 16 where they apply and
 *                            the context's budget holds their d(beta) image
 *                            with a quarter of the budget to spare, else the
 *                            CUDA cores.  On the tensor cores: split-FP16
 *                            products with FP32 accumulation, each MMA tile
 *                            the gamma samples (128 rows) by 128 (beta, q)
 *                            rows of one degree, Re and Im in two
 *                            accumulators.  The d(beta) operand's split parts
 *                            are built once per (L_h, n_beta) and kept by the
 *                            context: about 4 bytes per element of the d(beta)
 *                            table (3.8 GB at L_h = 64, n_beta = 2048).
 * Returns SLSHT_OK or SLSHT_E_ARG. */
#define SLSHT_OPT_BETA_ROUTE   1
#define SLSHT_OPT_ALPHA_ENGINE 2
#define SLSHT_OPT_CHUNK_PAIRS  3
#define SLSHT_OPT_GAUNT_TABLE  4
#define SLSHT_OPT_WAIT_TEST    5
#define SLSHT_OPT_REAL_FIELDS  6
#define SLSHT_OPT_COUPLING     7
#define SLSHT_OPT_FP64_ARITH   8
#define SLSHT_OPT_WINDOW_ORDERS 9
#define SLSHT_OPT_ROTWIN_ENGINE 10
int slsht_set_option(slsht_ctx* ctx, int option, int64_t value);

/* Bytes of device memory the context currently holds. */
size_t slsht_mem_used(slsht_ctx* ctx);

/* Library version string. */
const char* slsht_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SLSHT_H */
