// Mixed-precision driver (Section II-A, Fig. 1(d): diagonal tiles in double
// precision, off-diagonal tiles in reduced precision) and the component entry
// point for the tensor-core products.
#include <math.h>
#include <string.h>

#include <climits>

#include "ctx.cuh"
#include "gemm_tc.cuh"
#include "util.cuh"

namespace exa {

constexpr int kMixNB = kMixPanel;  // panel width = K of every tensor-core product
constexpr int kMixSub = 128;     // FP64 sub-tile of the diagonal block
constexpr double kIrFailTol = 1e-8;
constexpr double kIrQuadTol = 1e-8;   // refinement stops once q is final to this (relative), by default
// The error estimates below use the contraction of the last step, which measured 3 to 40 times
// below the true error of the quadratic form on smooth fields (the residual of a preconditioned
// step gathers in the directions where Sigma^-1 is large); they are taken 100 times over.
constexpr double kIrQuadSafety = 100.0;
constexpr int kLookaheadSMs = 20;         // SMs left to the look-ahead stream during a trailing update
constexpr int64_t kFuseMinRows = 40960;   // two panels per trailing pass down to this many rows
constexpr int64_t kLateRows = 61440;      // one-panel phase: the look-ahead share grows below this many rows
constexpr int kLateSMs = 48;              // ... up to this many SMs
constexpr int kDiagMaxCtas = 64;          // CTAs of one diagonal-block launch at most
constexpr double kExactThreshold = 0.8;  // tiles holding |Sigma_ij| >= 0.8 sigma^2 get exact products
constexpr double kSmoothNu = 1.2;        // above this smoothness every tile gets exact products
constexpr double kWideBandNu = 0.75;     // from this smoothness one more panel of the band is exact

size_t split_bytes(int64_t rows, int K, bool t3, bool oz) {
  const size_t t3_bytes = t3 ? (size_t)rows * K * 4 : 0;
  const size_t dig_bytes = oz ? (size_t)kOzSlices * rows * K * 2 : 0;
  const size_t ex_bytes = oz ? (size_t)round_up(rows, 64) * 4 : 0;
  const size_t exb_bytes = oz ? (size_t)round_up((rows + 255) / 256, 64) * 4 : 0;
  return (2 * t3_bytes + dig_bytes + ex_bytes + exb_bytes + 1023) / 1024 * 1024;
}

cudaError_t split_layout(SplitOperand& op, void* base_p, int64_t rows, int K, bool t3, bool oz) {
  const size_t t3_bytes = t3 ? (size_t)rows * K * 4 : 0;
  const size_t dig_bytes = oz ? (size_t)kOzSlices * rows * K * 2 : 0;
  const size_t ex_bytes = oz ? (size_t)round_up(rows, 64) * 4 : 0;
  uint8_t* base = (uint8_t*)base_p;
  op.rows = rows;
  op.K = K;
  op.hi = t3 ? (float*)base : nullptr;
  op.lo = t3 ? (float*)(base + t3_bytes) : nullptr;
  op.dig = oz ? (void*)(base + 2 * t3_bytes) : nullptr;
  op.ex = oz ? (int*)(base + 2 * t3_bytes + dig_bytes) : nullptr;
  op.exb = oz ? (int*)(base + 2 * t3_bytes + dig_bytes + ex_bytes) : nullptr;
  const cudaError_t e = make_split_maps(op);
  if (e != cudaSuccess) op.rows = 0;
  return e;
}

exa_status ensure_split(exa_ctx* c, SplitOperand& op, DevBuf& buf, int64_t rows, int K, bool t3, bool oz) {
  void* old = buf.p;
  exa_status st = ensure(c, buf, split_bytes(rows, K, t3, oz) + 1024, "split operands");
  if (st != EXA_OK) return st;
  const bool same = (old == buf.p) && op.rows == rows && op.K == K && ((op.hi != nullptr) == t3) &&
                    ((op.dig != nullptr) == oz);
  if (same) return EXA_OK;
  const cudaError_t e = split_layout(op, buf.p, rows, K, t3, oz);
  if (e != cudaSuccess) return cuda_err(c, e, "tensor map encode");
  return EXA_OK;
}

// ---------------------------------------------------------------------------
// Mixed-precision tiled Cholesky (panel width kMixNB = 512).  For tile column k:
//   1. FP64 factorisation of the 512 x 512 diagonal block as four 128 sub-tiles
//      (POTRF with the sub-tile inverse, TRSM and SYRK within the block on DMMA),
//      then its inverse W, block row by block row from the sub-tile inverses:
//      W_ij = -W_ii sum_{l=j}^{i-1} L_il W_lj (small DMMA products).
//   2. Panel TRSM  L_ik = A_ik W^T on the tensor cores: the first `band` tile
//      rows with the exact OZ products, the rest with T3.
//   3. Trailing update A_ij -= L_ik L_jk^T: tiles with I - J <= band (the
//      diagonal tile and its neighbours, where the Schur complement cancels
//      most) with OZ, all others with T3 (far tiles with one product).  Storage
//      stays FP64 throughout.
// ---------------------------------------------------------------------------
struct MixStep {
  exa_ctx* c;
  double* a;
  int64_t ld, npad;
  int band, T;
  int far_thr;  // single-product far tiles when eA + eB <= far_thr (INT_MIN: never)
};

// FP64 diagonal block k, its inverse, the panel splits and the tensor-core TRSM
// L_ik = A_ik W^T, all on stream s; the split of panel k lands in `sp`.
// `ctas` caps the persistent grids of the TRSM (0: all SMs).
static exa_status panel_factor(const MixStep& M, cudaStream_t s, int k, SplitOperand& sp, int ctas) {
  exa_ctx* c = M.c;
  double* a = M.a;
  const int64_t ld = M.ld, npad = M.npad;
  const int NB = kMixNB, nb = kMixSub;
  double* W = (double*)c->w_all.p;
  double* LD = (double*)c->logdet_part.p;
  // NB x NB inverse of the diagonal block (row-major); every block's is kept when asked
  double* W2 = c->keep_block_inverses ? (double*)c->mx_wall.p + (size_t)k * kMixNB * kMixNB : (double*)c->mx_w2.p;
  const int64_t k0 = (int64_t)k * NB;
  cudaError_t e = cudaSuccess;
  // 1. FP64 Cholesky of the diagonal block, its 128 sub-tile inverses and log sums, and
  // 2. its inverse W = L_kk^-1: one cooperative launch (diag_block.cu)
  {
    // one CTA per SM of the look-ahead share, 64 at most (the block's parallel phases gain
    // little beyond: 1.45 ms on 32 CTAs, 1.33 ms on 64)
    const int grid = ctas > 0 ? (ctas < kDiagMaxCtas ? ctas : kDiagMaxCtas) : kDiagMaxCtas;
    const double nb3 = (double)NB * NB * NB;
    ProfScope ps(c, PK_POTRF, 2.0 * nb3 / 3.0, 8.0 * (3.0 * NB * NB + 4.0 * nb * nb), 1, s, true);
    e = launch_diag_block(s, a, ld, k0, W + (k0 / nb) * (int64_t)nb * nb, LD + k0 / nb, W2, (double*)c->mx_dscr.p,
                          c->d_status, grid);
  }
  if (e != cudaSuccess) return cuda_err(c, e, "diagonal block launch");
  if (k == M.T - 1) return EXA_OK;  // the last block has no panel below it
  const int64_t r0 = k0 + NB;
  const int64_t m = npad - r0;
  double* panel_src = a + r0 + k0 * ld;  // element (r, t) at panel_src[r + t*ld]
  {
    ProfScope ps(c, PK_SPLIT, 0.0, 26.0 * (double)(m + NB) * NB, 2, s, true);
    e = launch_split_rows(s, W2, NB, 1, NB, NB, c->sp_b, 0);
    if (e == cudaSuccess) e = launch_split_rows(s, panel_src, 1, ld, (int)m, NB, sp, 0);
  }
  if (e != cudaSuccess) return cuda_err(c, e, "split launch");
  // 3. panel TRSM on the tensor cores: the first `band` tile rows exact, the rest TF32x3
  const int64_t rb = m < (int64_t)M.band * NB ? m : (int64_t)M.band * NB;
  GemmArgs g;
  memset(&g, 0, sizeof(g));
  g.C = a;
  g.ldc = ld;
  g.K = NB;
  g.panel = NB;
  g.st = c->d_status;
  g.store = 1;
  g.enum_mode = kEnumFull;
  g.c_col0 = k0;
  g.c_row0 = r0;
  g.nt = NB / 32;
  g.ntiles = (rb / 128) * g.nt;
  {
    ProfScope ps(c, PK_GEMM_OZ, 2.0 * (double)rb * NB * NB, 8.0 * (double)rb * NB, 1, s, true);
    e = launch_gemm_oz(s, sp, c->sp_b, g, ctas);
  }
  if (e == cudaSuccess && m > rb) {
    g.c_row0 = r0 + rb;
    g.a_row0 = (int)rb;
    g.nt = NB / 128;
    g.ntiles = ((m - rb) / 128) * g.nt;
    ProfScope ps(c, PK_GEMM_T3, 2.0 * (double)(m - rb) * NB * NB, 8.0 * (double)(m - rb) * NB, 1, s, true);
    e = launch_gemm_t3(s, sp, c->sp_b, g, ctas);
  }
  if (e == cudaSuccess) {
    ProfScope ps(c, PK_SPLIT, 0.0, 26.0 * (double)m * NB, 2, s, true);
    e = launch_split_rows(s, panel_src, 1, ld, (int)m, NB, sp, 0);
    if (e == cudaSuccess) e = launch_row_exp_blockmax(s, sp, m);
  }
  if (e != cudaSuccess) return cuda_err(c, e, "panel trsm launch");
  return EXA_OK;
}

// Block column j (> p) from panel p, whose split `sp` holds rows from (p + 1) NB: the
// first band+1 tile rows from the diagonal exact (OZ), the rest TF32x3.  `ctas` caps
// the persistent grids.
static exa_status column_update(const MixStep& M, cudaStream_t s, int p, int j, const SplitOperand& sp, int ctas) {
  exa_ctx* c = M.c;
  const int NB = kMixNB;
  const int64_t cj = (int64_t)j * NB;
  const int off = (int)(cj - (int64_t)(p + 1) * NB);  // operand row of global row cj
  const int64_t m = M.npad - cj;
  if (m <= 0) return EXA_OK;
  GemmArgs g;
  memset(&g, 0, sizeof(g));
  g.C = M.a;
  g.ldc = M.ld;
  g.K = NB;
  g.panel = NB;
  g.st = c->d_status;
  g.store = 0;
  g.band = M.band;
  g.enum_mode = kEnumFull;
  const int64_t rb = m < (int64_t)(M.band + 1) * NB ? m : (int64_t)(M.band + 1) * NB;
  g.lower_mask = 1;
  g.c_row0 = cj;
  g.c_col0 = cj;
  g.a_row0 = off;
  g.b_row0 = off;
  g.nt = NB / 32;
  g.ntiles = (rb / 128) * g.nt;
  cudaError_t e;
  {
    ProfScope ps(c, PK_GEMM_OZ, 2.0 * (double)rb * NB * NB, 16.0 * (double)rb * NB, 1, s, true);
    e = launch_gemm_oz(s, sp, sp, g, ctas);
  }
  if (e == cudaSuccess && m > rb) {
    g.lower_mask = 0;
    g.c_row0 = cj + rb;
    g.a_row0 = off + (int)rb;
    g.nt = NB / 128;
    g.ntiles = ((m - rb) / 128) * g.nt;
    // far tiles (one TF32 product) by the same test as the trailing update's, when CTA pairs
    // (and so far tiles) are on
    g.ea_blk = g.eb_blk = c->tc_pairs ? sp.exb : nullptr;
    g.far_thr = c->tc_pairs ? M.far_thr : INT_MIN;
    ProfScope ps(c, PK_GEMM_T3, 2.0 * (double)(m - rb) * NB * NB, 16.0 * (double)(m - rb) * NB, 1, s, true);
    e = launch_gemm_t3(s, sp, sp, g, ctas);
  }
  if (e != cudaSuccess) return cuda_err(c, e, "column update launch");
  return EXA_OK;
}

// The trailing lower triangle from row/column j0 NB on, from panel p (split `sp`, rows
// from (p + 1) NB) and, when sp2 is given, panel p + 1 as well (rows from (p + 2) NB).
// Band tiles (I - J <= band) take the exact OZ products, one pass per panel (its digit
// sums stay exact only up to K = 512); the others take TF32x3 on CTA pairs with both
// panels reduced into one accumulator (K = 2 NB), so every such tile of the FP64
// matrix is read and written once for the two panels.
static exa_status region_update(const MixStep& M, cudaStream_t s, int p, int j0, const SplitOperand& sp,
                                const SplitOperand* sp2, int ctas) {
  exa_ctx* c = M.c;
  const int NB = kMixNB, SUB = kMixNB / kMixSub;
  const int64_t cs = (int64_t)j0 * NB;
  const int64_t m2 = M.npad - cs;
  if (m2 <= 0) return EXA_OK;
  const int off1 = (int)(cs - (int64_t)(p + 1) * NB), off2 = (int)(cs - (int64_t)(p + 2) * NB);
  const int band = M.band;
  const double npan = sp2 ? 2.0 : 1.0;
  GemmArgs g;
  memset(&g, 0, sizeof(g));
  g.C = M.a;
  g.ldc = M.ld;
  g.K = NB;
  g.panel = NB;
  g.st = c->d_status;
  g.store = 0;
  g.band = band;
  g.lower_mask = 1;
  g.c_row0 = g.c_col0 = cs;
  g.a_row0 = g.b_row0 = off1;
  const long long t128 = m2 / 128;
  g.enum_mode = kEnumLowerOffBand;
  cudaError_t e = cudaSuccess;
  long long t3_tiles = 0;
  for (long long bi = 0; bi < t128; ++bi) {
    const long long lim = (long long)SUB * (bi / SUB - band);
    if (lim > 0) t3_tiles += lim;
  }
  if (t3_tiles > 0) {
    ProfScope ps(c, c->tc_pairs ? PK_GEMM_T3_PAIR : PK_GEMM_T3, npan * 2.0 * 128.0 * 128.0 * NB * (double)t3_tiles,
                 16.0 * 128.0 * 128.0 * (double)t3_tiles + npan * 8.0 * (double)m2 * NB, 1, s, true);
    if (c->tc_pairs) {  // 256-tiles on CTA pairs (m2 is a multiple of the 512 panel)
      const long long t256 = m2 / 256, sp2s = kPairSuper;
      const long long ts = (t256 + sp2s - 1) / sp2s;
      g.nt = (int)t256;
      g.ntiles = ts * (ts + 1) / 2 * sp2s * sp2s;
      g.ea_blk = g.eb_blk = sp.exb;
      g.far_thr = M.far_thr;
      if (sp2) {
        g.K2 = NB;
        g.a2_row0 = g.b2_row0 = off2;
        g.ea2_blk = g.eb2_blk = sp2->exb;
      }
      e = launch_gemm_t3_pair(s, sp, sp, g, ctas, sp2, sp2);
      g.K2 = 0;
      g.ea_blk = g.eb_blk = g.ea2_blk = g.eb2_blk = nullptr;
      g.far_thr = INT_MIN;
    } else {
      const long long ts = (t128 + kRasterSuper - 1) / kRasterSuper;  // supertile rows
      g.nt = (int)t128;
      g.ntiles = ts * (ts + 1) / 2 * kRasterSuper * kRasterSuper;
      e = launch_gemm_t3(s, sp, sp, g, ctas);
      if (e == cudaSuccess && sp2) {
        g.a_row0 = g.b_row0 = off2;
        e = launch_gemm_t3(s, *sp2, *sp2, g, ctas);
      }
    }
  }
  // band tiles, one exact pass per panel
  const long long tr = m2 / NB;
  long long pairs = 0;
  for (long long I = 0; I < tr; ++I) pairs += (I < band ? I : band) + 1;
  const long long per_pair = (long long)(NB / 128) * (NB / 32);
  long long skipped = 0;
  for (int h = 0; h < NB / 128; ++h)
    for (int q = 0; q < NB / 32; ++q)
      if ((long long)q * 32 > (long long)h * 128 + 127) ++skipped;
  const double oz_tiles = (double)pairs * per_pair - (double)skipped * (double)tr;
  g.enum_mode = kEnumBand;
  g.ntiles = pairs * per_pair;
  for (int q = 0; q < (sp2 ? 2 : 1) && e == cudaSuccess; ++q) {
    g.a_row0 = g.b_row0 = q ? off2 : off1;
    ProfScope ps(c, PK_GEMM_OZ, 2.0 * 128.0 * 32.0 * NB * oz_tiles, 16.0 * 128.0 * 32.0 * oz_tiles, 1, s, true);
    e = launch_gemm_oz(s, q ? *sp2 : sp, q ? *sp2 : sp, g, ctas);
  }
  if (e != cudaSuccess) return cuda_err(c, e, "trailing update launch");
  return EXA_OK;
}

// Mixed-precision tiled Cholesky with look-ahead on a side stream (kLookaheadSMs SMs
// reserved for it during the big trailing updates).  Panel splits rotate through four
// buffers (panel k in buffer k mod 4), so the side stream never overwrites operands
// still in use.
//
// While the trailing matrix is large (at least c->fuse_min_rows rows), panels go in
// pairs: with panels k and k+1 factored and every column >= k+2 holding the updates
// of the panels before k, the main stream brings columns k+2 and k+3 up to date
// (what the side stream needs next), the side stream factors panel k+2, applies it
// to column k+3 and factors panel k+3, and meanwhile the main stream applies panels
// k and k+1 together to every column >= k+4 (one read and write of each FP64 tile for
// the two panels).  Then, and for every panel when fusion is off, one panel at a
// time: column k+1 first, the side stream factors panel k+1 while the main stream
// applies panel k to the columns >= k+2.
exa_status factor_mixed(exa_ctx* c, double* a, int64_t ld, int64_t npad, exa_prec prec, int band, int far_thr) {
  const int NB = kMixNB, nb = kMixSub;
  const int T = (int)(npad / NB);
  const int T128 = (int)(npad / nb);
  if (band < 1) band = 1;
  exa_status st;
  if (prec != EXA_MIXED_TF32X3) return set_err(c, EXA_ERR_ARG, "precision %d has no mixed kernel", (int)prec);
  if ((st = ensure(c, c->w_all, (size_t)T128 * nb * nb * sizeof(double), "inverted diagonal tiles")) != EXA_OK)
    return st;
  if ((st = ensure(c, c->panel, (size_t)(NB * nb + nb * nb) * sizeof(double), "panel")) != EXA_OK) return st;
  if ((st = ensure(c, c->logdet_part, (size_t)T128 * sizeof(double), "log-det partials")) != EXA_OK) return st;
  const int64_t fuse_rows = c->fuse_min_rows < 0 ? kFuseMinRows : c->fuse_min_rows;
  // the fused phase runs while rows (k + 4) NB .. npad number at least fuse_rows, from k = 0
  const bool fuse = fuse_rows > 0 && c->tc_pairs && T >= 4 && npad - 4 * (int64_t)NB >= fuse_rows;
  SplitOperand* buf[4] = {&c->sp_a, &c->sp_a2, &c->sp_a3, &c->sp_a4};
  DevBuf* mem[4] = {&c->mx_split, &c->mx_split2, &c->mx_split3, &c->mx_split4};
  for (int i = 0; i < (fuse ? 4 : 2); ++i)
    if ((st = ensure_split(c, *buf[i], *mem[i], npad, NB, true, true)) != EXA_OK) return st;
  const int nbuf = fuse ? 4 : 2;
  if ((st = ensure_split(c, c->sp_b, c->mx_split_b, NB, NB, true, true)) != EXA_OK) return st;
  if ((st = ensure(c, c->mx_w2, (size_t)NB * NB * sizeof(double), "diagonal block inverse")) != EXA_OK) return st;
  if ((st = ensure(c, c->mx_dscr, diag_block_scratch_doubles() * sizeof(double), "diagonal block scratch")) != EXA_OK)
    return st;
  if (c->keep_block_inverses &&
      (st = ensure(c, c->mx_wall, (size_t)T * NB * NB * sizeof(double), "diagonal block inverses")) != EXA_OK)
    return st;
  if (!c->side) {
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->la_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->la_ev[1], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return set_err(c, EXA_ERR_CUDA, "look-ahead stream creation failed");
    }
  }
  MixStep M{c, a, ld, npad, band, T, far_thr};
  cudaStream_t ms = c->stream, ss = c->side;
  const int sms = tc_num_sms();
  const int side_ctas = c->lookahead_sms > 0 ? c->lookahead_sms : kLookaheadSMs;
  const int main_ctas = sms - side_ctas;
  auto B = [&](int p) -> SplitOperand& { return *buf[p % nbuf]; };
  // panel 0 on the main stream
  if ((st = panel_factor(M, ms, 0, B(0), 0)) != EXA_OK) return st;
  int k = 0;
  if (fuse) {
    // panel 1 on the main stream as well
    if ((st = column_update(M, ms, 0, 1, B(0), 0)) != EXA_OK) return st;
    if ((st = panel_factor(M, ms, 1, B(1), 0)) != EXA_OK) return st;
    for (; k + 3 < T && npad - (int64_t)(k + 4) * NB >= fuse_rows; k += 2) {
      for (int j = k + 2; j <= k + 3; ++j)
        for (int p = k; p <= k + 1; ++p)
          if ((st = column_update(M, ms, p, j, B(p), 0)) != EXA_OK) return st;
      cudaEventRecord(c->la_ev[0], ms);
      cudaStreamWaitEvent(ss, c->la_ev[0], 0);
      if ((st = panel_factor(M, ss, k + 2, B(k + 2), side_ctas)) != EXA_OK) return st;
      if ((st = column_update(M, ss, k + 2, k + 3, B(k + 2), side_ctas)) != EXA_OK) return st;
      if ((st = panel_factor(M, ss, k + 3, B(k + 3), side_ctas)) != EXA_OK) return st;
      cudaEventRecord(c->la_ev[1], ss);
      if ((st = region_update(M, ms, k, k + 4, B(k), &B(k + 1), main_ctas)) != EXA_OK) return st;
      cudaStreamWaitEvent(ms, c->la_ev[1], 0);
    }
    // hand over to the one-panel loop: panel k applied to every column >= k+2 leaves
    // panel k+1 factored and the columns >= k+2 holding every panel before k+1
    if ((st = region_update(M, ms, k, k + 2, B(k), nullptr, 0)) != EXA_OK) return st;
    ++k;
  }
  // As the trailing matrix shrinks, the main stream's update of it gets shorter than the
  // look-ahead stream's panel (FP64 diagonal block, panel solve, splits), which then sets
  // the pace: below late_rows trailing rows the look-ahead stream's SM share grows linearly
  // to late_sms (reached at late_rows / 3) and the main stream's shrinks by as much.
  const int64_t late_rows = c->late_rows < 0 ? kLateRows : c->late_rows;
  const int late_sms = c->late_sms > 0 ? c->late_sms : kLateSMs;
  for (; k + 1 < T; ++k) {
    const int64_t rows = npad - (int64_t)(k + 2) * NB;  // rows of the main stream's region update
    int side_k = side_ctas;
    if (late_rows > 0 && rows < late_rows && late_sms > side_ctas) {
      const double f = fmin(1.0, (double)(late_rows - rows) / (double)(late_rows - late_rows / 3));
      side_k = side_ctas + (int)(f * (late_sms - side_ctas));
      side_k = side_k < sms - 2 ? side_k & ~1 : (sms - 2) & ~1;
    }
    // block column k+1 first (everything the side stream needs), on the whole GPU
    if ((st = column_update(M, ms, k, k + 1, B(k), 0)) != EXA_OK) return st;
    cudaEventRecord(c->la_ev[0], ms);
    cudaStreamWaitEvent(ss, c->la_ev[0], 0);
    if ((st = panel_factor(M, ss, k + 1, B(k + 1), side_k)) != EXA_OK) return st;
    cudaEventRecord(c->la_ev[1], ss);
    // the rest of the trailing matrix on the remaining SMs
    if ((st = region_update(M, ms, k, k + 2, B(k), nullptr, sms - side_k)) != EXA_OK) return st;
    cudaStreamWaitEvent(ms, c->la_ev[1], 0);
  }
  return EXA_OK;
}

// x = (L L^T)^-1 rhs with the FP64-stored factor, on 128-wide tiles with the
// stored inverses of the diagonal sub-tiles.
// x = (L L^T)^-1 rhs; the upper tiles of a hold L^T.  flags: scratch for the solves' flags.
static cudaError_t solve_llt(exa_ctx* c, const double* a, int64_t ld, int64_t npad, const double* rhs, double* x,
                             double* work, int* flags) {
  cudaError_t e = cudaMemcpyAsync(work, rhs, npad * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return e;
  ProfScope ps(c, PK_TRSV, 2.0 * (double)npad * (double)npad, 8.0 * (double)npad * (double)npad, 2);
  return launch_llt_solve_persistent(c->stream, a, ld, npad, (const double*)c->w_all.p, work, x, flags,
                                     c->d_status);
}

// Generation (FP64, with the per-offset maxima for the precision map), the
// band choice and the mixed factorisation, retried with every tile exact if
// the reduced-precision factor is not positive definite.
exa_status mixed_generate_factor(exa_ctx* c, const double* d_locs, int64_t n, const double theta[3], int64_t npad,
                                 exa_prec prec, double* sigma_keep, int* band_used) {
  const int T = (int)(npad / kMixNB);
  exa_status st;
  if ((st = ensure(c, c->mat, (size_t)npad * npad * sizeof(double), "matrix")) != EXA_OK) return st;
  if ((st = ensure(c, c->mx_offmax, (size_t)(T + 1) * sizeof(unsigned long long), "precision map")) != EXA_OK)
    return st;
  double* A = (double*)c->mat.p;
  double* G = sigma_keep ? sigma_keep : A;
  unsigned long long* offmax = (unsigned long long*)c->mx_offmax.p;
  MaternParams Pm;
  model_params(c, theta, &Pm);
  cudaStream_t s = c->stream;
  const MaternTable* tab = nullptr;
  if ((st = matern_table(c, Pm, &tab)) != EXA_OK) return st;
  cudaError_t e = cudaMemsetAsync(offmax, 0, (size_t)(T + 1) * sizeof(unsigned long long), s);
  if (e == cudaSuccess) {
    ProfScope ps(c, PK_GEN, 0.0, 4.0 * (double)npad * (double)(npad + 1));
    e = launch_matern_gen(s, d_locs, n, npad, Pm, G, npad, offmax, tab, kMixNB, sigma_keep ? A : nullptr);
  }
  if (e != cudaSuccess) return cuda_err(c, e, "generation");
  cudaEventRecord(c->ev[1], s);
  int band = c->mixed_band;
  if (band == 0 && theta[2] > kSmoothNu) band = -1;  // smooth fields: exact products everywhere
  if (band == 0) {
    static thread_local unsigned long long h[1 << 14];
    const int cnt = T < (1 << 14) ? T : (1 << 14);
    e = cudaMemcpyAsync(h, offmax, (size_t)cnt * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(c, e, "precision map read");
    band = 1;
    for (int d = cnt - 1; d >= 1; --d) {
      double v;
      memcpy(&v, &h[d], sizeof(v));
      if (v >= kExactThreshold * theta[0]) {
        band = d;
        break;
      }
    }
    // smoother fields cancel farther from the diagonal: at n = 22,500, theta = (1, 0.1, 1) the
    // rule above gives 3 panels and |dl|/|l| = 1.2e-6, one panel more 8.8e-7; at n = 90,000,
    // theta = (1, 0.03, 1) one more panel also saves a refinement step
    if (theta[2] >= kWideBandNu) band += 1;
    if (band > T) band = T;
  } else if (band < 0) {
    band = T;
  }
  // far tiles: operand blocks bounded by 2^eA and 2^eB with eA + eB at least far_tile_margin
  // below the exponent of sigma^2 (the largest |Sigma_ij|) take one TF32 product
  int es = 0;
  frexp(theta[0], &es);
  const int far_thr = c->far_tile_margin > 0 ? es - c->far_tile_margin : INT_MIN;
  st = factor_mixed(c, A, npad, npad, prec, band, far_thr);
  if (st != EXA_OK) return st;
  st = read_status(c);
  if (st == EXA_ERR_NOT_SPD && band < T && sigma_keep) {
    // the reduced-precision updates broke positive definiteness: redo with exact products everywhere
    if ((st = reset_status(c)) != EXA_OK) return st;
    e = cudaMemcpyAsync(A, G, (size_t)npad * npad * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_err(c, e, "refactor copy");
    band = T;
    st = factor_mixed(c, A, npad, npad, prec, band, INT_MIN);
    if (st == EXA_OK) st = read_status(c);
  }
  if (band_used) *band_used = band;
  return st;
}

exa_status loglik_mixed(exa_ctx* c, const double* d_locs, const double* d_z, const double theta[3], int64_t n,
                        exa_prec prec, exa_result* out) {
  if (prec != EXA_MIXED_TF32X3)
    return set_err(c, EXA_ERR_ARG,
                   "EXA_MIXED_BF16X3 is not offered: three BF16 products (16 significant bits) leave "
                   "|dl|/|l| near 3e-4 on smooth Matern fields; use EXA_MIXED_TF32X3");
  const int64_t npad = round_up(n, kMixNB);
  const int T128 = (int)(npad / kMixSub);
  exa_status st;
  if ((st = ensure(c, c->mx_sigma, (size_t)npad * npad * sizeof(double), "FP64 covariance copy")) != EXA_OK)
    return st;
  if ((st = ensure(c, c->mx_vec, (size_t)6 * npad * sizeof(double), "refinement vectors")) != EXA_OK) return st;
  if ((st = ensure(c, c->partial, (size_t)(2 * kRedPartials + 2 * npad + 64) * sizeof(double), "partials")) != EXA_OK)
    return st;
  if ((st = reset_status(c)) != EXA_OK) return st;
  double* S = (double*)c->mx_sigma.p;
  double* zp = (double*)c->mx_vec.p;
  double* x = zp + npad;
  double* r = x + npad;
  double* d = r + npad;
  double* y = d + npad;
  double* work = y + npad;
  double* part = (double*)c->partial.p;
  double* red = part + 2 * kRedPartials;  // the solves' flags live after the reduction partials
  cudaStream_t s = c->stream;
  cudaEventRecord(c->ev[0], s);
  int band = 0;
  if ((st = mixed_generate_factor(c, d_locs, n, theta, npad, prec, S, &band)) != EXA_OK) return st;
  cudaEventRecord(c->ev[2], s);
  cudaError_t e;
  e = launch_sum(s, (const double*)c->logdet_part.p, T128, part, c->d_scalars + 1);
  if (e == cudaSuccess) e = launch_pad_vector(s, d_z, n, npad, zp);
  if (e == cudaSuccess) e = launch_sumsq(s, zp, npad, part, c->d_scalars + 2);
  double* A = (double*)c->mat.p;
  if (e == cudaSuccess) {
    // L^T into the unused upper triangle: the backward solves stream contiguous columns
    ProfScope ps(c, PK_OTHER, 0.0, 8.0 * (double)npad * (double)npad);
    e = launch_transpose_lower_to_upper(s, A, npad, npad);
  }
  if (e == cudaSuccess) e = solve_llt(c, A, npad, npad, zp, x, work, (int*)red);
  if (e != cudaSuccess) return cuda_err(c, e, "solve launch");
  // iterative refinement of x = Sigma^-1 z with the FP64 residual.  It stops when the
  // residual no longer halves or reaches rounding level, or once the quadratic form is final
  // to kIrQuadTol relative: a correction d changes z^T x by less than that, or the
  // second-order term r^T d of the variational estimate is below it (q is then that estimate).
  if ((st = ensure(c, c->mx_symv, (size_t)symv_tiled_partials(npad) * sizeof(double), "symmetric product partials")) !=
      EXA_OK)
    return st;
  double* sp = (double*)c->mx_symv.p;
  double rel = 0.0, prev = 1e300;
  double rel_prev = 1.0;  // ||r|| / ||z|| of the step before (the residual of x = 0 is z itself)
  double rho = 1.0;       // contraction of the last step, ||r_k|| / ||r_k-1||
  double q_var = NAN;     // the variational estimate, when it ended the refinement
  double q_err = NAN;     // estimated relative error of the q returned
  const double qtol = c->ir_quad_tol > 0.0 ? c->ir_quad_tol : kIrQuadTol;
  bool q_done = false;
  // stopping rule: a caller's residual target (exa_ctx_set_refinement), rounding level for the
  // gradient (which needs Sigma^-1 z itself), else the quadratic-form rule (target < 0)
  const double target = c->ir_target > 0.0 ? c->ir_target : (c->ir_tight ? 0.0 : -1.0);
  int it = 0;
  const int kMaxIt = 10;
  for (;; ++it) {
    {
      ProfScope ps(c, PK_SYMV, 2.0 * (double)npad * (double)npad, 8.0 * (double)npad * (double)(npad + 1) / 2.0, 2);
      e = launch_symv_lower_tiled(s, S, npad, npad, x, y, sp);
    }
    if (e == cudaSuccess) e = launch_residual(s, zp, y, r, npad);
    if (e == cudaSuccess) e = launch_sumsq(s, r, npad, part, c->d_scalars + 3);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_scalars, c->d_scalars, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_err(c, e, "refinement launch");
    if ((st = read_status(c)) != EXA_OK) return st;  // synchronises
    if (!isfinite(c->h_scalars[2]))
      return set_err(c, EXA_ERR_ARG, "||z||^2 = %g: z holds a non-finite entry (or its squares overflow)",
                     c->h_scalars[2]);
    // z = 0: x = 0 and q = 0 are exact, nothing to refine
    rel = c->h_scalars[2] > 0.0 ? sqrt(c->h_scalars[3]) / sqrt(c->h_scalars[2]) : 0.0;
    rho = rel_prev > 0.0 ? rel / rel_prev : 1.0;
    rel_prev = rel;
    if (!(rel > (target > 0.0 ? target : 1e-15)) || it >= kMaxIt || rel > 0.5 * prev) break;
    prev = rel;
    e = solve_llt(c, A, npad, npad, r, d, work, (int*)red);
    // the variational estimate of q before x moves: with r = z - Sigma x and d = (L L^T)^-1 r,
    // q = z^T x + x^T r + r^T Sigma^-1 r, so q_hat = z^T x + x^T r + r^T d is off by
    // r^T (Sigma^-1 - (L L^T)^-1) r, second order in the residual (about the contraction
    // factor of the refinement times r^T d), where z^T (x + d) is off to first order
    if (e == cudaSuccess) e = launch_dot(s, x, r, npad, part, c->d_scalars + 6);
    if (e == cudaSuccess) e = launch_dot(s, r, d, npad, part, c->d_scalars + 7);
    if (e == cudaSuccess) e = launch_dot(s, zp, x, npad, part, c->d_scalars + 8);
    if (e == cudaSuccess) e = launch_axpy(s, 1.0, d, x, npad);
    if (e == cudaSuccess) e = launch_dot(s, zp, d, npad, part, c->d_scalars + 4);
    if (e == cudaSuccess) e = launch_dot(s, zp, x, npad, part, c->d_scalars + 5);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->h_scalars + 4, c->d_scalars + 4, 5 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_err(c, e, "refinement solve");
    if ((st = read_status(c)) != EXA_OK) return st;
    if (target < 0.0) {
      // q_hat is off by r^T (Sigma^-1 - (L L^T)^-1) r: about the step's contraction times r^T d
      const double q_hat = c->h_scalars[8] + c->h_scalars[6] + c->h_scalars[7];
      const double e_var = kIrQuadSafety * rho * fabs(c->h_scalars[7]);
      const double e_plain = kIrQuadSafety * rho * fabs(c->h_scalars[4]);
      if (e_var <= qtol * fabs(q_hat)) {
        q_var = q_hat;
        q_err = e_var / fabs(q_hat);
        q_done = true;
        ++it;
        break;
      }
      if (e_plain <= qtol * fabs(c->h_scalars[5])) {  // z^T (x + d) is off by about rho |z^T d|
        q_err = e_plain / fabs(c->h_scalars[5]);
        q_done = true;
        ++it;
        break;
      }
    }
  }
  e = launch_dot(s, zp, x, npad, part, c->d_scalars + 0);
  // x^T r for the error estimate of a refinement that stopped on its residual (r then belongs to x)
  if (e == cudaSuccess && isnan(q_err)) e = launch_dot(s, x, r, npad, part, c->d_scalars + 9);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_scalars, c->d_scalars, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && isnan(q_err))
    e = cudaMemcpyAsync(c->h_scalars + 9, c->d_scalars + 9, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_err(c, e, "quadratic form");
  cudaEventRecord(c->ev[3], s);
  if ((st = read_status(c)) != EXA_OK) return st;
  cudaEventElapsedTime(&out->ms_gen, c->ev[0], c->ev[1]);
  cudaEventElapsedTime(&out->ms_chol, c->ev[1], c->ev[2]);
  cudaEventElapsedTime(&out->ms_solve, c->ev[2], c->ev[3]);
  cudaEventElapsedTime(&out->ms_total, c->ev[0], c->ev[3]);
  out->tile_nb = kMixNB;
  out->exact_band = band;
  out->n_tiles = (int)(npad / kMixNB);
  out->ir_iters = it;
  out->ir_resid = rel;
  out->quad = isnan(q_var) ? c->h_scalars[0] : q_var;
  // stopped on the residual (a caller's target, rounding level or stalling): x^T r, the first-order
  // term q lacks, measured against q
  const double xr = fabs(c->h_scalars[9]);
  out->quad_err = !isnan(q_err) ? q_err : (xr == 0.0 ? 0.0 : xr / fabs(out->quad));
  out->logdet = 2.0 * c->h_scalars[1];
  out->loglik = -0.5 * (double)n * 1.8378770664093454836 - 0.5 * out->logdet - 0.5 * out->quad;
  if (!q_done && !(rel <= kIrFailTol))
    return set_err(c, EXA_ERR_IR_NOCONV, "refinement stalled at relative residual %.3e", rel);
  return EXA_OK;
}

}  // namespace exa

using namespace exa;

extern "C" exa_status exa_ctx_set_far_tile_margin(exa_ctx* c, int bits) {
  if (!c || bits < 0) return c ? set_err(c, EXA_ERR_ARG, "far-tile margin must be >= 0") : EXA_ERR_ARG;
  c->far_tile_margin = bits;
  return EXA_OK;
}

extern "C" exa_status exa_ctx_set_refinement_quad(exa_ctx* c, double tol) {
  if (!c) return EXA_ERR_ARG;
  if (!(tol >= 0.0) || !(tol < 1e-3)) return set_err(c, EXA_ERR_ARG, "quadratic-form tolerance must be in [0, 1e-3)");
  c->ir_quad_tol = tol;
  return EXA_OK;
}

extern "C" exa_status exa_ctx_set_refinement(exa_ctx* c, double resid_target) {
  if (!c) return EXA_ERR_ARG;
  if (!(resid_target >= 0.0) || !isfinite(resid_target))
    return set_err(c, EXA_ERR_ARG, "refinement target must be finite and >= 0");
  c->ir_target = resid_target;
  return EXA_OK;
}

extern "C" exa_status exa_ctx_set_lookahead_late(exa_ctx* c, int64_t rows, int sms) {
  if (!c || sms < 0 || sms > 150) return c ? set_err(c, EXA_ERR_ARG, "bad late look-ahead share") : EXA_ERR_ARG;
  c->late_rows = rows < 0 ? -1 : rows;
  c->late_sms = sms;
  return EXA_OK;
}

extern "C" exa_status exa_ctx_set_tc_pairs(exa_ctx* c, int on) {
  if (!c) return EXA_ERR_ARG;
  c->tc_pairs = on ? 1 : 0;
  return EXA_OK;
}

extern "C" exa_status exa_gemm_update(exa_ctx* c, exa_gemm_kind kind, int64_t m, int64_t n, int64_t k,
                                      const double* d_a, const double* d_b, double* d_c, int64_t ldc, int store) {
  if (!c) return EXA_ERR_ARG;
  c->err[0] = 0;
  if (!d_a || !d_b || !d_c || m <= 0 || n <= 0 || k <= 0 || ldc < m)
    return set_err(c, EXA_ERR_ARG, "bad gemm arguments");
  const bool oz = (kind == EXA_GEMM_OZ);
  const bool pair = (kind == EXA_GEMM_T3_PAIR);
  if (kind != EXA_GEMM_T3 && kind != EXA_GEMM_OZ && !pair) return set_err(c, EXA_ERR_ARG, "unknown gemm kind");
  // T3 on pairs reduces up to two operand pairs per pass: k up to 2 kSplitMaxK
  const int64_t kmax = pair ? 2 * (int64_t)kSplitMaxK : kSplitMaxK;
  if (m % (pair ? 256 : 128) || k % 64 || k > kmax || (oz ? (n % 32) : (n % (pair ? 256 : 128))))
    return set_err(c, EXA_ERR_ARG, "gemm shape m=%lld n=%lld k=%lld not supported", (long long)m, (long long)n,
                   (long long)k);
  const int k1 = (int)(k < kSplitMaxK ? k : kSplitMaxK), k2 = (int)(k - k1);
  exa_status st;
  if ((st = ensure_split(c, c->sp_a, c->mx_split, m, k1, !oz, oz)) != EXA_OK) return st;
  if ((st = ensure_split(c, c->sp_b, c->mx_split_b, n, k1, !oz, oz)) != EXA_OK) return st;
  if (k2 > 0) {
    if ((st = ensure_split(c, c->sp_a2, c->mx_split2, m, k2, true, false)) != EXA_OK) return st;
    if ((st = ensure_split(c, c->sp_a3, c->mx_split3, n, k2, true, false)) != EXA_OK) return st;
  }
  if ((st = reset_status(c)) != EXA_OK) return st;
  cudaError_t e = launch_split_rows(c->stream, d_a, k, 1, (int)m, k1, c->sp_a, 0);
  if (e == cudaSuccess) e = launch_split_rows(c->stream, d_b, k, 1, (int)n, k1, c->sp_b, 0);
  if (e == cudaSuccess && k2 > 0) e = launch_split_rows(c->stream, d_a + k1, k, 1, (int)m, k2, c->sp_a2, 0);
  if (e == cudaSuccess && k2 > 0) e = launch_split_rows(c->stream, d_b + k1, k, 1, (int)n, k2, c->sp_a3, 0);
  if (e != cudaSuccess) return cuda_err(c, e, "split launch");
  GemmArgs g;
  memset(&g, 0, sizeof(g));
  g.C = d_c;
  g.ldc = ldc;
  g.K = k1;
  g.enum_mode = kEnumFull;
  g.store = store ? 1 : 0;
  g.st = c->d_status;
  if (oz) {
    g.nt = (int)(n / 32);
    g.ntiles = (m / 128) * (n / 32);
    e = launch_gemm_oz(c->stream, c->sp_a, c->sp_b, g);
  } else if (pair) {
    g.nt = (int)(n / 256);
    g.ntiles = (m / 256) * (n / 256);
    g.K2 = k2;
    e = launch_gemm_t3_pair(c->stream, c->sp_a, c->sp_b, g, 0, k2 > 0 ? &c->sp_a2 : nullptr,
                            k2 > 0 ? &c->sp_a3 : nullptr);
  } else {
    g.nt = (int)(n / 128);
    g.ntiles = (m / 128) * (n / 128);
    e = launch_gemm_t3(c->stream, c->sp_a, c->sp_b, g);
  }
  if (e != cudaSuccess) return cuda_err(c, e, "gemm launch");
  return read_status(c);
}
