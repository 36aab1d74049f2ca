/*
 * exa.h -- C ABI of the GB300 exact Matérn Gaussian log-likelihood library.
 *
 * The library evaluates, on one GPU, the log-likelihood of zero-mean Gaussian
 * data z observed at n two-dimensional locations s_1..s_n (Section I, Eq. 2
 * with mu = 0):
 *
 *     l(theta) = -n/2 log(2 pi) - 1/2 log|Sigma(theta)| - 1/2 z^T Sigma(theta)^-1 z
 *
 * where Sigma is the isotropic Matérn covariance of Section I, Eq. 3,
 *
 *     Sigma_ij = sigma^2 / (2^(nu-1) Gamma(nu)) (r_ij/beta)^nu K_nu(r_ij/beta),
 *     r_ij = ||s_i - s_j|| (Euclidean),  Sigma_ii = sigma^2,
 *
 * theta = (sigma^2, beta, nu), all > 0.  As Section I states, log|Sigma| and
 * Sigma^-1 z come from the Cholesky factor Sigma = L L^T, which dominates the
 * cost (O(n^3) flops, O(n^2) memory).  The mixed-precision form follows the
 * MP variant of Section II-A (Fig. 1(d)): diagonal tiles stay FP64, off-diagonal
 * updates run in reduced precision.  The gradient and the batched form are
 * extensions of the same evaluation (the paper's optimiser, BOBYQA of Section
 * II-B, needs no derivatives).
 *
 * The steps of an evaluation, by the names the sources use for them:
 *   a1  covariance generation (Eq. 3);
 *   a2  tiled Cholesky factorisation Sigma = L L^T;
 *   a3  log|Sigma| = 2 sum log L_ii;
 *   a4  y = L^-1 z and the quadratic form q = y^T y;
 *   a5  assembly of l (Eq. 2);
 *   a6  mixed precision: iterative refinement of Sigma^-1 z against the FP64 Sigma;
 *   a7  the gradient of l with respect to theta;
 *   a8  a1-a6 for many replicate fields in one batched launch.
 *
 * Conventions for every entry point:
 *   - Pointers prefixed d_ are DEVICE pointers on the context's device; h_
 *     or unprefixed pointers are HOST pointers.  The caller owns all inputs
 *     and outputs; the library never frees them.
 *   - Locations are n x 2 FP64, interleaved (x_0, y_0, x_1, y_1, ...).
 *     Observations z are n FP64.  Both must be 8-byte aligned.
 *   - Work is issued on the context's CUDA stream.  Entry points returning a
 *     host value synchronise that stream before returning; the batched form
 *     is stream-asynchronous.
 *   - Every entry point returns an exa_status.  On any error other than
 *     EXA_ERR_NOT_SPD the outputs are left unspecified; exa_last_error()
 *     gives a message.  A non-positive or non-finite Cholesky pivot gives
 *     EXA_ERR_NOT_SPD with loglik = NaN and the 0-based failing row in
 *     exa_last_pivot() (Section III, Example 2: Sigma is numerically singular
 *     when two locations nearly coincide).
 *   - Functions are not thread-safe on one context; use one context per
 *     host thread.
 */
#ifndef EXA_H
#define EXA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EXA_OK = 0,
  EXA_ERR_ARG = 1,        /* bad argument: n < 1, null pointer, theta <= 0 or non-finite, bad enum,
                             z with a non-finite entry (single-field log-likelihood, gradient, prediction) */
  EXA_ERR_NOT_SPD = 2,    /* Cholesky pivot <= 0 or non-finite: Sigma(theta) not numerically SPD */
  EXA_ERR_NOMEM = 3,      /* workspace would exceed the context limit, or cudaMalloc failed */
  EXA_ERR_CUDA = 4,       /* a CUDA runtime or driver call failed */
  EXA_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up (batched scheduler) */
  EXA_ERR_IR_NOCONV = 6   /* mixed precision: iterative refinement did not reach its tolerance */
} exa_status;

/* Arithmetic of the Cholesky updates.  In every mode the covariance
 * generation, the diagonal-tile factorisation (POTRF), the log-determinant
 * and the triangular solves are FP64.                                      */
typedef enum {
  EXA_FP64 = 0,          /* all tiles FP64 (the exact variant, Fig. 1(a)) */
  EXA_MIXED_FP32 = 1,    /* batched form only: off-diagonal tile products in FP32 (FFMA), FP32 accumulate per
                            tile; exa_loglik refuses it (EXA_ERR_ARG): on one large field FP32 FFMA runs at a
                            third of the TF32x3 tensor-core rate with fewer significant bits */
  EXA_MIXED_BF16X3 = 2,  /* refused (EXA_ERR_ARG): 3 BF16 products keep 16 significant bits, |dl|/|l| ~ 3e-4 */
  EXA_MIXED_TF32X3 = 3   /* off-diagonal TRSM/GEMM/SYRK products as 3 TF32 tensor-core products, FP32 accumulate */
} exa_prec;

typedef struct exa_ctx exa_ctx;

/* Detailed result of one evaluation (exa_loglik_ex).                       */
typedef struct {
  double loglik;      /* l(theta) */
  double logdet;      /* log|Sigma| = 2 sum log L_ii */
  double quad;        /* z^T Sigma^-1 z */
  double ir_resid;    /* mixed: last computed ||z - Sigma x||_2 / ||z||_2 (taken before the final
                         correction when the quadratic form settled first); FP64: 0 */
  int32_t ir_iters;   /* mixed: refinement steps taken; FP64: 0 */
  int32_t tile_nb;    /* tile size used by the factorisation */
  int32_t exact_band; /* mixed: tile rows next to the diagonal with exact products (all tiles when = T) */
  int32_t n_tiles;    /* number of tile rows T of the factorisation */
  float ms_gen;       /* device time of the covariance generation (ms) */
  float ms_chol;      /* device time of the Cholesky factorisation (ms) */
  float ms_solve;     /* device time of log-det + solve (+ refinement) (ms) */
  float ms_total;     /* device time of the whole evaluation (ms) */
  double quad_err;    /* mixed: estimated relative error of quad (see exa_ctx_set_refinement_quad);
                         FP64: 0 */
} exa_result;

/* Create a context on the current CUDA device.
 *   cuda_stream      cudaStream_t to issue work on (NULL: the legacy default stream).
 *   workspace_bytes  upper bound on device memory the context may hold (0: no bound).
 *   tile_nb          FP64 tile size, a multiple of 64 and <= 128 (0: library default).
 * Returns EXA_ERR_ARG on a bad tile size, EXA_ERR_CUDA if no device is usable. */
exa_status exa_ctx_create(exa_ctx** ctx, void* cuda_stream, size_t workspace_bytes, int tile_nb);

/* Free every device buffer the context holds and the context itself.       */
void exa_ctx_destroy(exa_ctx* ctx);

/* Replace the stream work is issued on.                                    */
exa_status exa_ctx_set_stream(exa_ctx* ctx, void* cuda_stream);

/* Mixed precision: number of 512-wide panel rows next to the diagonal whose
 * products use the exact digit-slice arithmetic (the rest use TF32x3).
 * band >= 1 fixes it; a negative value makes every tile exact; 0 (the
 * default) picks it per evaluation from Sigma itself: the widest tile-row
 * offset d whose tiles hold some |Sigma_ij| >= 0.8 sigma^2 (where the Schur
 * complement cancels most), one panel more when nu >= 0.75, and every tile
 * when nu > 1.2 (smooth fields cancel everywhere).  If the reduced-precision factor loses positive
 * definiteness the evaluation is repeated with every tile exact.           */
exa_status exa_ctx_set_mixed_band(exa_ctx* ctx, int band);

/* Mixed precision: SMs left to the look-ahead stream (which factors the next
 * diagonal block and runs the next panel solve) while the trailing update
 * runs on the others.  0 restores the default (20).                        */
exa_status exa_ctx_set_lookahead(exa_ctx* ctx, int sms);

/* Mixed precision, one-panel phase: once the trailing matrix has fewer than `rows`
 * rows, the look-ahead stream's SM share grows linearly from exa_ctx_set_lookahead's
 * to `sms` (reached at rows / 3) and the trailing update's shrinks by as much, since
 * the look-ahead stream's panel then sets the pace.  rows = 0 turns the ramp off;
 * rows < 0 and sms = 0 restore the defaults (61440 rows, 48 SMs).            */
exa_status exa_ctx_set_lookahead_late(exa_ctx* ctx, int64_t rows, int sms);

/* Mixed precision: while the trailing matrix still has at least min_rows rows,
 * panels are applied in pairs (the off-band TF32x3 update of the two panels
 * accumulates in one pass, K = 1024, so each FP64 tile is read and written once
 * per pair; band tiles keep one exact pass per panel) while the look-ahead
 * stream factors the next two panels.  Needs CTA pairs (exa_ctx_set_tc_pairs)
 * and at least four panels.  0 turns it off; a negative value restores the
 * default (40960).  Results differ from the one-panel order only by rounding. */
exa_status exa_ctx_set_panel_fusion(exa_ctx* ctx, int64_t min_rows);

/* Mixed precision: refinement stopping rule.  resid_target > 0: refine
 * x = Sigma^-1 z until ||z - Sigma x||_2 / ||z||_2 <= resid_target (or the
 * residual stops halving, or 10 steps); 0 (the default): stop once q is final
 * to the tolerance of exa_ctx_set_refinement_quad.  exa_result.ir_resid reports
 * the last residual computed.
 * EXA_ERR_ARG for a negative or non-finite target.                          */
exa_status exa_ctx_set_refinement(exa_ctx* ctx, double resid_target);

/* Mixed precision: relative accuracy to which the quadratic form is refined
 * when exa_ctx_set_refinement's target is 0 (default 1e-8, far below the
 * log-determinant's error of the mixed factor; 0 restores it).  With
 * r = z - Sigma x and d = (L L^T)^-1 r, the variational estimate
 * q = z^T x + x^T r + r^T d is off by r^T (Sigma^-1 - (L L^T)^-1) r, estimated
 * as 100 rho |r^T d| with rho = ||r|| / ||r_prev|| the contraction of the last
 * step (||r_prev|| = ||z|| at the first; the factor 100 covers the 3 to 40 times
 * by which rho |r^T d| fell short of the true error on smooth fields); the
 * refinement stops once that estimate, or 100 rho |z^T d| for the plain
 * q = z^T (x + d), is at most tol |q|, and reports it relative to q in
 * exa_result.quad_err.  EXA_ERR_ARG for tol < 0, tol >= 1e-3 or NaN.        */
exa_status exa_ctx_set_refinement_quad(exa_ctx* ctx, double tol);

/* Message describing the last error on this context ("" if none).  The
 * string is owned by the context and valid until its next call.           */
const char* exa_last_error(const exa_ctx* ctx);

/* 0-based row of the failing pivot of the last EXA_ERR_NOT_SPD, else -1.   */
int64_t exa_last_pivot(const exa_ctx* ctx);

/* Device memory currently held by the context, in bytes.                   */
size_t exa_workspace_bytes(const exa_ctx* ctx);

/* Step a1 alone: write the lower triangle (diagonal included) of the n x n
 * Matérn covariance Sigma(theta) (Eq. 3) into the caller's column-major
 * device matrix d_sigma with leading dimension ld >= n: entry (i, j), i >= j,
 * lands at d_sigma[i + j * ld].  The strict upper triangle is not written.
 * theta is a host array {sigma^2, beta, nu}.                               */
exa_status exa_covariance(exa_ctx* ctx, const double* d_locs, int64_t n, const double theta[3], double* d_sigma,
                          int64_t ld);

/* Step a2 alone: in-place FP64 Cholesky of the caller's column-major SPD
 * matrix (lower triangle read, factor L written to the lower triangle; the
 * strict upper triangle is left untouched).  ld >= n.  Returns
 * EXA_ERR_NOT_SPD on a non-positive or non-finite pivot.                    */
exa_status exa_potrf(exa_ctx* ctx, double* d_a, int64_t n, int64_t ld);

/* Steps a1-a5: log-likelihood l(theta) (Eq. 2) at host theta {sigma^2, beta, nu}.
 * *loglik (host) receives l, or NaN with EXA_ERR_NOT_SPD.  A z holding a
 * non-finite entry gives EXA_ERR_ARG with loglik = NaN; it is found from
 * z^T Sigma^-1 z (FP64) or ||z||^2 (mixed, before any refinement step), at
 * no extra pass over z.  z = 0 is valid: q = 0 exactly.                     */
exa_status exa_loglik(exa_ctx* ctx, const double* d_locs, const double* d_z, const double theta[3], int64_t n,
                      exa_prec prec, double* loglik);

/* As exa_loglik, with the log-determinant, the quadratic form, refinement
 * statistics and per-phase device timings in *out (host).                  */
exa_status exa_loglik_ex(exa_ctx* ctx, const double* d_locs, const double* d_z, const double theta[3], int64_t n,
                         exa_prec prec, exa_result* out);

/* Log-likelihood and its gradient dl/d(sigma^2, beta, nu) (Eq. 2 differentiated
 * through the Matern covariance of Eq. 3):
 *   dl/dtheta_k = 1/2 a^T (dSigma/dtheta_k) a - 1/2 tr(Sigma^-1 dSigma/dtheta_k),  a = Sigma^-1 z.
 * grad (host, 3 doubles).  dSigma/dtheta_k is regenerated entry by entry (never stored).
 *   EXA_FP64          FP64 factor, a, and Sigma^-1 = L^-T L^-1 on FP64 DMMA.  Holds two
 *                     n_pad^2 FP64 buffers (n_pad = n rounded up to the tile) when the
 *                     context can hold them; otherwise (workspace bound or cudaMalloc
 *                     failure) it holds one: L^-1 overwrites the factor and each tile of
 *                     L^-T L^-1 is reduced as it is formed.  Same result to rounding.
 *   EXA_MIXED_TF32X3  l from the mixed evaluation (exa_loglik), a refined in FP64 to
 *                     rounding level, Sigma^-1 of the mixed factor with every product on
 *                     the tensor cores in exact 7-bit digit slices (35-bit operands), or on
 *                     FP64 DMMA after exa_ctx_set_gradient_inverse(ctx, 1).  Holds two
 *                     n_pad^2 FP64 buffers (n_pad = n rounded up to 512) plus about 5 n^2
 *                     bytes of digit planes.  Stated accuracy against the FP64 oracle:
 *                     each component within 5e-5 of max|grad| (2.4e-5 measured on the
 *                     smoothest field tested, nu = 1.5, beta = 0.2; <= 2e-6 for nu <= 1).
 * Other precisions return EXA_ERR_ARG.                                       */
exa_status exa_loglik_grad(exa_ctx* ctx, const double* d_locs, const double* d_z, const double theta[3], int64_t n,
                           exa_prec prec, double* loglik, double grad[3]);

/* Mixed-precision gradient: compute Sigma^-1 of the mixed factor on FP64 DMMA
 * (fp64 != 0: about 2 n^3 / 3 FP64 flops, for ill-conditioned fields) or on the
 * tensor cores (0, the default).                                             */
exa_status exa_ctx_set_gradient_inverse(exa_ctx* ctx, int fp64);

/* Batched evaluation of nrep independent replicate fields of uneven sizes
 * (one persistent launch walks the tile tasks of every replicate; the
 * replicate studies of Section III, Example 2).
 *   prec      EXA_FP64: every tile task in FP64.  EXA_MIXED_FP32 (the MP
 *             variant of Section II-A): diagonal tiles factored in FP64, the
 *             off-diagonal TRSM and update tiles computed from FP32-rounded
 *             operands with FP32 accumulation over the tile and added to the
 *             FP64 tile (tiles within the band set by exa_ctx_set_batched_mixed
 *             stay FP64), then x = Sigma^-1 z refined in FP64 against an FP64
 *             copy of Sigma until q is final to 1e-8 relative by the rule of
 *             exa_ctx_set_refinement_quad (variational estimate, error taken as
 *             100 x the last step's contraction x |r^T d|), else to rounding
 *             level with q = z^T x; a replicate whose refinement stalls above a
 *             1e-8 relative residual before that reports EXA_ERR_IR_NOCONV.
 *             EXA_MIXED_TF32X3: the same precision pattern on the tensor cores,
 *             step-synchronous over 128-wide tile columns: per step one launch
 *             factors every replicate's FP64 diagonal tile, then grouped tcgen05
 *             launches run every replicate's panel solve and trailing update as
 *             TF32x3 128 x 128 tiles (FP32 accumulation, FP64 tiles); the same
 *             FP64 refinement.  exa_ctx_set_batched's tile and CTA options and
 *             the FP64 band of exa_ctx_set_batched_mixed apply to the persistent
 *             forms only.  EXA_MIXED_BF16X3 returns EXA_ERR_ARG.
 *   h_n       host array of nrep sizes (each >= 1).
 *   d_locs    host array of nrep DEVICE pointers, replicate r has h_n[r] x 2 locations.
 *   d_z       host array of nrep DEVICE pointers, h_n[r] observations each.
 *   d_theta   DEVICE array nrep x 3 (sigma^2, beta, nu per replicate), read at execution time,
 *             so a captured graph can be replayed with new parameters.
 *   d_loglik  DEVICE output, nrep values (NaN where the replicate's status is not EXA_OK).
 *   d_status  DEVICE output, nrep exa_status codes.  z is not inspected: a
 *             replicate whose z holds a non-finite entry gets loglik = NaN
 *             without a status of its own; z = 0 gives q = 0.
 * Stream-asynchronous: returns once the work is enqueued; device memory is
 * allocated on the first call for a shape set, so make that call before any
 * CUDA-graph capture, after which the sequence can be captured and replayed
 * with new d_theta.  Calls that overlap on the GPU share the context's
 * buffers and must not run concurrently.                                     */
exa_status exa_loglik_batched(exa_ctx* ctx, int32_t nrep, const int64_t* h_n, const double* const* d_locs,
                              const double* const* d_z, const double* d_theta, exa_prec prec, double* d_loglik,
                              int32_t* d_status);

/* Spatial prediction (kriging) at m new locations from n observations, FP64:
 * the conditional mean and variance of the zero-mean field (the prediction of
 * the sea-surface-temperature tutorial, Section IV):
 *   mean_i = c_i^T Sigma^-1 z,  var_i = sigma^2 - c_i^T Sigma^-1 c_i,
 *   c_i = (Sigma(new_i, obs_j))_j from Eq. 3.
 *   d_locs      DEVICE n x 2 observed locations; d_z DEVICE n observations.
 *   d_new_locs  DEVICE m x 2 new locations (m >= 0).
 *   d_mean      DEVICE output, m values.
 *   d_var       DEVICE output, m values, or NULL to skip the variances (they cost
 *               n^2 m FP64 flops; the means cost n m covariance evaluations).
 * Uses the context's factor workspace (like exa_loglik) and synchronises the
 * context stream.  EXA_ERR_NOT_SPD if Sigma(theta) of the observations is not
 * positive definite.                                                          */
exa_status exa_predict(exa_ctx* ctx, const double* d_locs, const double* d_z, const double theta[3], int64_t n,
                       const double* d_new_locs, int64_t m, double* d_mean, double* d_var);

/* Fisher information of theta = (sigma^2, beta, nu) at the observed locations, FP64
 * (the package's exact_fisher):  I_kl = 1/2 tr(Sigma^-1 D_k Sigma^-1 D_l),
 * D_k = dSigma/dtheta_k (Eq. 3 differentiated as for exa_loglik_grad).
 *   fisher   HOST output, 3 x 3 row-major (symmetric).
 * Holds five n_pad^2 FP64 buffers (the matrix, Sigma^-1 and the three products
 * Sigma^-1 D_k, n_pad = n rounded up to 128) and costs ~7 n^3 FP64 flops.
 * Synchronises the context stream; EXA_ERR_NOT_SPD if Sigma(theta) is not
 * positive definite.                                                          */
exa_status exa_fisher(exa_ctx* ctx, const double* d_locs, const double theta[3], int64_t n, double fisher[9]);

/* Products of step a2 on their own (component check of the tensor-core
 * contractions used by the mixed-precision factorisation):
 *   C = A B^T (store != 0)  or  C -= A B^T (store == 0)
 * A is m x k and B is n x k, row-major FP64 device matrices; C is a column-
 * major FP64 device matrix with leading dimension ldc >= m.  kind selects
 * the arithmetic: EXA_GEMM_T3 (three TF32 products, FP32 accumulation) or
 * EXA_GEMM_OZ (five exact 7-bit BF16 digit slices per row, exact FP32
 * accumulation, FP64 combination), or EXA_GEMM_T3_PAIR (T3 on pairs of SMs
 * with 256 x 256 tiles, tcgen05 .cta_group::2).  Shapes: m % 128 == 0 (256 for
 * T3_PAIR), k % 64 == 0, n % 128 == 0 (T3), n % 32 == 0 (OZ) or n % 256 == 0
 * (T3_PAIR), and k <= 512 (the digit sums of OZ stay below 2^24 up to
 * k = 512, so its accumulation is exact); T3_PAIR takes k <= 1024, reducing
 * columns 512.. as a second operand pair into the same accumulator (the
 * two-panel pass of the factorisation).                                      */
typedef enum { EXA_GEMM_T3 = 0, EXA_GEMM_OZ = 1, EXA_GEMM_T3_PAIR = 2 } exa_gemm_kind;
exa_status exa_gemm_update(exa_ctx* ctx, exa_gemm_kind kind, int64_t m, int64_t n, int64_t k, const double* d_a,
                           const double* d_b, double* d_c, int64_t ldc, int store);

/* Model options (the paper's dmetric and a nugget), applied by every later call
 * on the context except exa_loglik_noalloc (always Euclidean, no nugget):
 *   nugget  tau^2 >= 0 added to every diagonal entry: Sigma + tau^2 I (a fixed
 *           value, not estimated; the gradient and Fisher information are those of
 *           theta with tau^2 held fixed; predictions are of the noise-free field);
 *   metric  0: Euclidean distance between (x, y); 1: great-circle distance
 *           between (longitude, latitude) in degrees, haversine form, on a sphere
 *           of the given radius (beta is then in the radius's units);
 *   radius  > 0, or 0 for 6371 (the Earth's mean radius in km).
 * EXA_ERR_ARG for a negative or non-finite nugget/radius or another metric.   */
exa_status exa_ctx_set_model(exa_ctx* ctx, double nugget, int metric, double radius);

/* Off-band trailing updates of the mixed factorisation on pairs of SMs
 * (256 x 256 tiles, tcgen05 .cta_group::2; default on) or on single SMs
 * (128 x 128 tiles).  Both compute the same products.                       */
exa_status exa_ctx_set_tc_pairs(exa_ctx* ctx, int on);

/* Far tiles of the mixed factorisation (the MP variant's precision map, taken
 * per tile from the data): an off-band 256 x 256 trailing-update tile whose two
 * operand blocks have largest magnitudes 2^eA and 2^eB with eA + eB at least
 * `bits` binades below sigma^2 is computed with the single TF32 product hi*hi
 * (relative error ~2^-10, absolute error below that of the three-product form
 * on entries of size sigma^2 when bits >= 12).  bits = 0 turns it off; the
 * default is 16 (at n = 90,000, theta = (1, 0.03, 1): |dl|/|l| vs FP64 5.1e-8
 * with 16 or with the feature off, 1.2e-7 with 12, 5.7e-6 with 8).
 * Ignored when exa_ctx_set_tc_pairs is off.                                 */
exa_status exa_ctx_set_far_tile_margin(exa_ctx* ctx, int bits);

/* Kernel accounting.  Launch counts and the algorithmic flops / bytes of every
 * kernel class are always accumulated; with profiling enabled each launch is
 * also bracketed by CUDA events on the stream it runs on (adds ~2 us per
 * launch).  The rate of a class is timed_flops / ms (or timed_bytes / ms):
 * both count the same timed launch groups.                                  */
typedef struct {
  char name[32];          /* kernel class */
  int64_t launches;       /* kernels launched */
  int64_t timed_launches; /* launch groups timed with events */
  double ms;              /* summed device time of the timed launch groups */
  double flops;           /* algorithmic flops of every launch (useful multiply-adds x 2) */
  double bytes;           /* algorithmic DRAM bytes of every launch (compulsory reads + writes) */
  double timed_flops;     /* algorithmic flops of the timed launch groups only */
  double timed_bytes;     /* algorithmic bytes of the timed launch groups only */
} exa_kernel_stat;
exa_status exa_profile_enable(exa_ctx* ctx, int on);

/* Launch timeline (with profiling enabled): start and end of every timed launch
 * group, in ms from the first timed group of each evaluation (one evaluation per
 * batch of records), and the stream it ran on (0: the context stream, 1: the
 * mixed factorisation's look-ahead stream).  exa_profile_timeline_enable clears
 * the records and turns recording on (1) or off (0); exa_profile_timeline copies
 * up to max records into out (host), oldest first, and returns how many
 * (reset != 0 clears them).  At most 2^20 records are kept.                  */
typedef struct {
  char name[32];    /* kernel class (as exa_kernel_stat) */
  int32_t stream;   /* 0 context stream, 1 look-ahead stream */
  float start_ms;
  float end_ms;
} exa_timeline_rec;
exa_status exa_profile_timeline_enable(exa_ctx* ctx, int on);
int exa_profile_timeline(exa_ctx* ctx, exa_timeline_rec* out, int max, int reset);
/* Copy up to max per-class records into out (host); returns how many.  Waits
 * for pending timed launches.  reset != 0 zeroes the accumulators.         */
int exa_profile_read(exa_ctx* ctx, exa_kernel_stat* out, int max, int reset);

/* Options of the batched form:
 *   tile_nb      tile of the persistent factorisation, 32 or 64 (0: 64);
 *   ctas_per_sm  persistent CTAs per SM, capped at what fits resident (0: all that fit);
 *   spin_cycles  bound of one dependency wait in SM clock cycles (0: 2e9, about 1 s);
 *   inject_stall test hook: non-zero adds to the work list a task whose dependency is
 *                never met, so its wait runs out and the affected replicates report
 *                EXA_ERR_TIMEOUT (the path a real stall would take).                 */
exa_status exa_ctx_set_batched(exa_ctx* ctx, int tile_nb, int ctas_per_sm, long long spin_cycles, int inject_stall);

/* Tile autotuner of the batched form.  Runs the batch (same arguments as
 * exa_loglik_batched) with every candidate configuration -- tile 64 and 32,
 * each with the largest and the next-largest number of resident CTAs per SM --
 * twice (plan + buffers, then a run timed with CUDA events on the context
 * stream), keeps the fastest in the context and returns it (tile_nb,
 * ctas_per_sm, best_ms: host outputs).  Synchronises the stream.  d_loglik /
 * d_status hold the last candidate's results.  On any failure the previous
 * configuration is kept and the error returned.  EXA_MIXED_TF32X3 (the
 * tensor-core form, one configuration: 128-wide tiles) is run twice the same
 * way and reported as tile_nb = 128, ctas_per_sm = 0; the context's options
 * of the persistent forms stay as they were.                               */
exa_status exa_batched_autotune(exa_ctx* ctx, int32_t nrep, const int64_t* h_n, const double* const* d_locs,
                                const double* const* d_z, const double* d_theta, exa_prec prec, double* d_loglik,
                                int32_t* d_status, int* tile_nb, int* ctas_per_sm, float* best_ms);

/* Options of the mixed-precision batched form:
 *   band      TRSM / update tiles fewer than `band` tile diagonals away from the
 *             diagonal stay FP64 (0: every off-diagonal product on tensor cores);
 *   max_iter  refinement steps per replicate at most (0: 10).                    */
exa_status exa_ctx_set_batched_mixed(exa_ctx* ctx, int band, int max_iter);

/* Exact synthetic realisation (Section III, Example 1, simulate_obs_exact):
 * d_z = L d_eps with L L^T = Sigma(theta), both n FP64 device vectors.       */
exa_status exa_simulate(exa_ctx* ctx, const double* d_locs, const double* d_eps, const double theta[3], int64_t n,
                        exa_prec prec, double* d_z);

/* Issue-rate probe of the FP64 pipes (measurement only; no counterpart in the
 * paper): kind 0 times FP64 fused multiply-adds, kind 1 the FP64 tensor-core MMA
 * (mma.sync m8n8k4), each with eight independent chains per thread or warp and
 * every resident CTA, best of three timed launches after a warm-up, on
 * cuda_stream (NULL: the legacy default stream).  *tflops (host) receives the
 * rate in TFLOP/s (2 flops per multiply-add).  Synchronises the stream.
 * EXA_ERR_ARG for another kind or a NULL tflops, EXA_ERR_CUDA on a failed call. */
exa_status exa_probe_fp64_rate(void* cuda_stream, int kind, double* tflops);

/* Allocation-free FP64 log-likelihood (no counterpart in the paper; an
 * interface for callers that cannot allocate device memory).
 *
 * Some callers cannot call cudaMalloc: a host application whose memory pool
 * owns all device memory, or a latency-critical path that cannot afford the
 * device-wide synchronisation cudaMalloc and cudaFree imply.  This entry point
 * computes the same l(theta) as exa_loglik with EXA_FP64 but allocates
 * nothing: it needs no context, and its workspace is one fixed array in the
 * library's device memory, about 36 MiB, held by every GPU that loads the
 * library until the process exits.
 *   cuda_stream  stream to run on (NULL: the legacy default stream).
 *   d_locs, d_z  device inputs as for exa_loglik; theta on the host.
 *   n            1 <= n <= 2048; larger n returns EXA_ERR_ARG.
 *   loglik       host output (NaN on any error).
 * The call synchronises the stream.  On the first call on a device it looks
 * up the device address of the array (cudaGetSymbolAddress); make that first
 * call before any stream capture.  All calls on a device share the one array:
 * calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.  Returns EXA_ERR_NOT_SPD for a
 * non-positive pivot (no pivot index is kept), EXA_ERR_ARG for a z holding a
 * non-finite entry, and EXA_ERR_CUDA if a CUDA call fails.                   */
exa_status exa_loglik_noalloc(void* cuda_stream, const double* d_locs, const double* d_z, const double theta[3],
                              int64_t n, double* loglik);

#ifdef __cplusplus
}
#endif

#endif /* EXA_H */
