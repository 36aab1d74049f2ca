// The opaque exa_ctx and the host-side helpers shared by the driver files.
#pragma once

#include <stddef.h>

#include "exa_internal.cuh"
#include "gemm_tc.cuh"
#include "prof.cuh"

namespace exa {

struct BatchPlan;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

constexpr int kNumEvents = 8;
constexpr int kMixPanel = 512;     // panel width of the mixed-precision factorisation
constexpr int kRedPartials = 512;  // partial sums of one two-stage reduction

inline int64_t kPartialDoubles(int64_t npad, int nb) { return 2 * kRedPartials + (npad / 1024 + 2) * (int64_t)nb; }

}  // namespace exa

struct exa_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t ws_limit = 0;   // 0: unbounded
  size_t held_bytes = 0;
  int tile_nb = 128;     // FP64 tile
  int lookahead_sms = 0;  // SMs reserved for the look-ahead stream (0: default)
  int64_t late_rows = -1; // one-panel phase: below this many trailing rows the look-ahead share grows (-1: default)
  int late_sms = 0;       // ... linearly up to this many SMs at late_rows / 3 (0: default)
  int64_t fuse_min_rows = -1;  // two-panel trailing passes down to this many rows (0: off, < 0: default)
  int mixed_band = 0;    // exact-product band (256-wide tiles); 0: from Sigma; < 0: all tiles
  int64_t last_pivot = -1;
  char err[512];
  // workspace
  exa::DevBuf mat;          // padded n x n FP64 matrix (column-major, ld = npad)
  exa::DevBuf w_all;        // inverted diagonal tiles, T x nb x nb
  exa::DevBuf panel;        // row-major panel copy, npad x nb
  exa::DevBuf logdet_part;  // per-tile log-det sums
  exa::DevBuf vec;          // n-vectors
  exa::DevBuf partial;      // reduction partials
  exa::DevBuf table;        // per-theta Matérn interpolation table + its node values
  // mixed precision
  exa::DevBuf mx_sigma;     // FP64 copy of Sigma for the refinement residual
  exa::DevBuf mx_split;     // split-precision panel operands (A role), four buffers by panel index mod 4
  exa::DevBuf mx_split2;
  exa::DevBuf mx_split3;
  exa::DevBuf mx_split4;
  exa::DevBuf mx_split_b;   // split-precision operands (B role: inverse diagonal block / test B)
  exa::SplitOperand sp_a, sp_a2, sp_a3, sp_a4, sp_b;
  exa::DevBuf mx_vec;       // refinement vectors
  exa::DevBuf mx_w2;        // inverse of the panel-wide diagonal block (row-major)
  exa::DevBuf mx_wall;      // every panel's diagonal-block inverse, T x 512 x 512 (kept for the gradient)
  exa::DevBuf mx_dscr;      // scratch of the cooperative diagonal-block factorisation
  int keep_block_inverses = 0;  // mixed factorisation: write block k's inverse to mx_wall + k 512^2
  int ir_tight = 0;         // mixed refinement: iterate to rounding level (the gradient needs Sigma^-1 z)
  double ir_target = 0.0;   // mixed refinement: relative residual to reach (0: quadratic-form rule)
  double ir_quad_tol = 0.0; // mixed refinement: relative accuracy of q (0: the default)
  int grad_inverse_fp64 = 0;  // mixed gradient: Sigma^-1 of the mixed factor on FP64 DMMA instead of the tensor cores
  exa::DevBuf mx_offmax;    // per tile-row offset max |Sigma_ij| (precision map)
  exa::DevBuf mx_symv;      // partial sums of the tiled symmetric product
  // gradient
  exa::DevBuf gr_part;      // second n x n buffer: Sigma^-1 for the gradient trace term
  exa::DevBuf gr_xsplit;    // mixed gradient: digit planes of every 512-row block of X = L^-1
  exa::DevBuf gr_lsplit;    // mixed gradient: digit planes of one 512-row block of L
  exa::DevBuf gr_t;         // mixed gradient: 512 x n product of one row block
  exa::DevBuf gr_blocks;    // per-block gradient partial sums
  exa::DevBuf pr_c, pr_y;   // prediction: cross-covariance block and its solve block
  exa::DevBuf fs_m;         // Fisher information: Sigma^-1 D_k for k = 0, 1, 2
  // batched
  exa::DevBuf bt_mat, bt_meta, bt_vec, bt_work, bt_mat2;
  exa::DevBuf bt_tasks, bt_ps, bt_ws;  // tensor-core batched form: task lists, panel and inverse split operands
  exa::BatchPlan* bplan = nullptr;  // cached work list of the last shape set
  void* bt_stage = nullptr;         // pinned host staging for the work list / metadata
  size_t bt_stage_bytes = 0;
  int batched_nb = 64;              // tile of the batched factorisation (32 or 64)
  int batched_ctas_per_sm = 0;      // 0: as many as fit
  long long batched_spin = 2000000000LL;  // bound of one dependency wait (SM cycles)
  int batched_stall = 0;            // test hook: add a task whose dependency is never met
  int tc_pairs = 1;                 // mixed trailing update on CTA pairs (tcgen05 .cta_group::2)
  double nugget = 0.0;              // tau^2 on the diagonal
  int metric = 0;                   // 0 Euclidean, 1 great circle (longitude, latitude in degrees)
  double radius = 6371.0;           // sphere radius of the great-circle metric
  int far_tile_margin = 16;         // single-product far tiles below sigma^2 by this many binades (0: off)
  int batched_band = 0;             // mixed: tile updates within this many tile diagonals stay FP64
  int batched_max_iter = 10;        // mixed: refinement steps per replicate at most
  // status and small results
  exa::DevStatus* d_status = nullptr;
  exa::DevStatus* h_status = nullptr;  // pinned
  double* d_scalars = nullptr;
  double* h_scalars = nullptr;          // pinned
  cudaEvent_t ev[exa::kNumEvents] = {};
  cudaStream_t side = nullptr;          // look-ahead stream of the mixed factorisation
  cudaEvent_t la_ev[2] = {};            // look-ahead hand-off events
  exa::Prof prof;
};

namespace exa {

exa_status set_err(exa_ctx* c, exa_status st, const char* fmt, ...);
exa_status cuda_err(exa_ctx* c, cudaError_t e, const char* what);
exa_status ensure(exa_ctx* c, DevBuf& b, size_t bytes, const char* name);
exa_status check_theta(exa_ctx* c, const double theta[3]);
exa_status reset_status(exa_ctx* c);
exa_status read_status(exa_ctx* c);
exa_status factor_fp64(exa_ctx* c, double* a, int64_t ld, int64_t npad, int nb);
exa_status factor_mixed(exa_ctx* c, double* a, int64_t ld, int64_t npad, exa_prec prec, int band, int far_thr);
// Generate Sigma into `sigma_keep` (or straight into the factor buffer) and factor it in mixed precision.
exa_status mixed_generate_factor(exa_ctx* c, const double* d_locs, int64_t n, const double theta[3], int64_t npad,
                                 exa_prec prec, double* sigma_keep, int* band_used);
exa_status loglik_fp64(exa_ctx* c, const double* d_locs, const double* d_z, const double theta[3], int64_t n,
                       exa_result* out, double** keep_y);
exa_status loglik_mixed(exa_ctx* c, const double* d_locs, const double* d_z, const double theta[3], int64_t n,
                        exa_prec prec, exa_result* out);
void release_extra(exa_ctx* c);
// Build the interpolation table for theta on the context stream; returns its device address.
exa_status matern_table(exa_ctx* c, const MaternParams& P, const MaternTable** tab);
// matern_params plus the context's model options (nugget, metric, radius).
void model_params(const exa_ctx* c, const double theta[3], MaternParams* P);
void release_batched(exa_ctx* c);
// Lay out a split operand of `rows` x K in `buf` (T3 planes and/or OZ digits) and build its TMA maps.
exa_status ensure_split(exa_ctx* c, SplitOperand& op, DevBuf& buf, int64_t rows, int K, bool t3, bool oz);
// Bytes of one split operand (a multiple of 1024), and its layout at `base` (1024-byte aligned)
// with its TMA maps.
size_t split_bytes(int64_t rows, int K, bool t3, bool oz);
cudaError_t split_layout(SplitOperand& op, void* base, int64_t rows, int K, bool t3, bool oz);

}  // namespace exa
