// Step a2 (mixed precision): the Cholesky's dense contractions on the fifth-
// generation tensor cores (tcgen05.mma, TMEM accumulators, TMA-staged tiles).
//
// The MP variant of Section II-A (Fig. 1(d)) keeps the tiles next to the
// diagonal in double precision and lowers the precision of the rest.  Here
// every operand is stored in FP64 and each product C -= A B^T runs as one of:
//
//  * T3 (off-band tiles): A = A_hi + A_lo with A_hi = tf32(A), A_lo = tf32(A - A_hi)
//    (both rounded to nearest), C -= A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T,
//    accumulated in FP32 in TMEM (~22 significant bits per product).
//  * OZ (band tiles, where the Schur complement cancels most): each row is scaled
//    by a power of two 2^e_r so that |a| <= 1 and cut into S = 5 signed 7-bit
//    integer digits held exactly in BF16, a = 2^e_r sum_s d_s 2^{-7(s+1)}
//    (|d_0| <= 128, |d_s| <= 64 after it).  A group g = s + t sums at most two
//    products with a leading digit (<= 2^13, or 2^14 for g = 0) and g - 1 others
//    (<= 2^12), at most 7 * 2^12 per k; with K <= 512 every partial sum stays
//    below 2^24, so FP32 accumulation in TMEM is exact.  The 15 products with g <= 4 go to five accumulators that
//    the epilogue combines in FP64 (error ~2^-35 of the row maxima).
//
// Both kernels are persistent and warp-specialised: warp 0 issues TMA loads,
// warp 1 owns TMEM and issues tcgen05.mma from one thread, warps 2-5 drain the
// accumulators into the FP64 matrix.  Every wait is bounded; on time-out the
// CTA records EXA_ERR_TIMEOUT, drains its in-flight copies, frees TMEM and exits.
#include <cuda.h>
#include <math.h>

#include <climits>

#include "ctx.cuh"
#include "gemm_tc.cuh"
#include "tc_common.cuh"

namespace exa {

using namespace tc;

__device__ __forceinline__ void tile_tri_decode(long long b, int& ti, int& tj) {
  long long t = (long long)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while (t * (t + 1) / 2 > b) --t;
  while ((t + 1) * (t + 2) / 2 <= b) ++t;
  ti = (int)t;
  tj = (int)(b - t * (t + 1) / 2);
}

// Output-tile enumeration shared by all roles of a CTA.  Returns false if the
// tile is to be skipped.  (bi, bj) are tile indices in units of (TM, TN).
template <int TM, int TN>
__device__ __forceinline__ bool decode_tile(const GemmArgs& g, long long t, int& bi, int& bj) {
  if (g.enum_mode == kEnumFull) {
    bi = (int)(t / g.nt);
    bj = (int)(t % g.nt);
    return true;
  }
  if (g.enum_mode == kEnumLowerOffBand) {
    // TM == TN == 128, g.nt tile rows, band measured in panel-wide tiles.  Tiles are
    // taken in supertiles of kSuper x kSuper (lower-triangle order of supertiles,
    // row-major inside), so the CTAs of one wave share a few operand row blocks
    // in L2 instead of streaming a different B row block each from DRAM.
    constexpr int kSuper = kRasterSuper;
    const long long sidx = t / (kSuper * kSuper);
    const int loc = (int)(t % (kSuper * kSuper));
    int SI, SJ;
    tile_tri_decode(sidx, SI, SJ);
    bi = SI * kSuper + loc / kSuper;
    bj = SJ * kSuper + loc % kSuper;
    if (bi >= g.nt || bj > bi) return false;
    const int per = g.panel / 128;
    return (bi / per - bj / per) > g.band;
  }
  // kEnumBand: pairs (I, J) of panel-wide tiles with 0 <= I - J <= band, each split in
  // (panel/TM) x (panel/TN) sub-tiles
  const int SI = g.panel / TM, SJ = g.panel / TN;
  const long long pair = t / (SI * SJ);
  const int sub = (int)(t % (SI * SJ));
  const int b = g.band;
  const long long head = (long long)b * (b + 1) / 2;
  int I, J;
  if (pair < head) {
    tile_tri_decode(pair, I, J);
  } else {
    I = b + (int)((pair - head) / (b + 1));
    J = I - b + (int)((pair - head) % (b + 1));
  }
  bi = I * SI + sub / SJ;
  bj = J * SJ + sub % SJ;
  // skip sub-tiles strictly above the diagonal
  return (long long)bj * TN <= (long long)bi * TM + TM - 1;
}

// T3 (128 x 128 tiles): operand rows and output origin of tile t, from the enumeration or the
// launch's task list.  Returns false if the tile is to be skipped.
struct T3Tile {
  int ya, yb;
  double* C;
  int64_t ldc;
  bool diag;
};
__device__ __forceinline__ bool t3_tile(const GemmArgs& g, long long t, T3Tile& o) {
  if (g.enum_mode == kEnumTasks) {
    const TcTask tk = g.tasks[t];
    o.ya = tk.a_row;
    o.yb = tk.b_row;
    o.C = tk.C;
    o.ldc = tk.ldc;
    o.diag = tk.lower != 0;
    return true;
  }
  int bi, bj;
  if (!decode_tile<128, 128>(g, t, bi, bj)) return false;
  o.ya = g.a_row0 + bi * 128;
  o.yb = g.b_row0 + bj * 128;
  o.C = g.C + (g.c_row0 + (int64_t)bi * 128) + (g.c_col0 + (int64_t)bj * 128) * g.ldc;
  o.ldc = g.ldc;
  o.diag = g.lower_mask && (bi == bj);
  return true;
}

// Far 128 x 128 tiles of the single-CTA kernel: the same test as the pair kernel's far tiles,
// on the 256-row block exponents of the two operand row blocks (never in task mode).
__device__ __forceinline__ bool far_t3(const GemmArgs& g, const T3Tile& tl) {
  if (g.enum_mode == kEnumTasks || g.far_thr == INT_MIN || !g.ea_blk || !g.eb_blk) return false;
  return (long long)g.ea_blk[tl.ya / 256] + (long long)g.eb_blk[tl.yb / 256] <= (long long)g.far_thr;
}

__device__ __forceinline__ void record_timeout(DevStatus* st, int site) {
  if (atomicExch(&st->timeout, 1) == 0) st->timeout_where = site;
}

// ===========================================================================
// T3 kernel: tile 128 x 128, K chunks of 32 FP32 (TF32) values, 3 stages.
// ===========================================================================
constexpr int kEpiThreads = 256;                 // 8 epilogue warps
constexpr int kGemmThreads = 64 + kEpiThreads;   // + TMA producer warp + MMA warp

namespace t3 {
constexpr int TM = 128, TN = 128, KC = 32, STAGES = 3;
constexpr int OP_BYTES = TM * KC * 4;           // 16 KB per operand tile
constexpr int STAGE_BYTES = 4 * OP_BYTES;       // A_hi, A_lo, B_hi, B_lo
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t IDESC = idesc(kFmtTF32, TM, TN);
constexpr int TMEM_COLS = 256;                  // 2 accumulator buffers x 128 columns
}  // namespace t3

__global__ void __launch_bounds__(kGemmThreads)
    gemm_t3_kernel(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
                   const __grid_constant__ CUtensorMap tB_hi, const __grid_constant__ CUtensorMap tB_lo,
                   const __grid_constant__ GemmArgs g) {
  using namespace t3;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accfull = empty + STAGES;
  uint64_t* accempty = accfull + 2;
  uint32_t* tmem_slot = (uint32_t*)(accempty + 2);
  volatile int* abort = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], kEpiThreads);
    }
    *abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const int kchunks = g.K / KC;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    const uint64_t pol = l2_evict_last_policy();
    prefetch_tmap(&tA_hi);
    prefetch_tmap(&tA_lo);
    prefetch_tmap(&tB_hi);
    prefetch_tmap(&tB_lo);
    int stage = 0;
    uint32_t phase = 0;
    int last_par[STAGES];
    for (int s = 0; s < STAGES; ++s) last_par[s] = -1;
    for (long long t = blockIdx.x; t < g.ntiles && !*abort; t += gridDim.x) {
      T3Tile tl;
      if (!t3_tile(g, t, tl)) continue;
      const int ya = tl.ya, yb = tl.yb;
      const bool one = far_t3(g, tl);  // far tile: the hi halves only
      for (int kc = 0; kc < kchunks; ++kc) {
        if (!mbar_wait(&empty[stage], phase ^ 1, abort)) {
          *abort = 1;
          record_timeout(g.st, 11);
          break;
        }
        uint8_t* sb = smem + stage * STAGE_BYTES;
        mbar_expect_tx(&full[stage], one ? 2 * OP_BYTES : STAGE_BYTES);
        tma_load_2d_hint(sb, &tA_hi, &full[stage], kc * KC, ya, pol);
        tma_load_2d_hint(sb + 2 * OP_BYTES, &tB_hi, &full[stage], kc * KC, yb, pol);
        if (!one) {
          tma_load_2d_hint(sb + OP_BYTES, &tA_lo, &full[stage], kc * KC, ya, pol);
          tma_load_2d_hint(sb + 3 * OP_BYTES, &tB_lo, &full[stage], kc * KC, yb, pol);
        }
        last_par[stage] = (int)phase;
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
    if (*abort) {  // let every copy this thread issued land before the CTA exits
      for (int s = 0; s < STAGES; ++s)
        if (last_par[s] >= 0) {
          volatile int never = 0;
          mbar_wait(&full[s], (uint32_t)last_par[s], &never);
        }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    int stage = 0;
    uint32_t phase = 0;
    int it = 0;
    for (long long t = blockIdx.x; t < g.ntiles && !*abort; t += gridDim.x) {
      T3Tile tl;
      if (!t3_tile(g, t, tl)) continue;
      const int b = it & 1;
      const uint32_t ap = (it >> 1) & 1;
      if (!mbar_wait(&accempty[b], ap ^ 1, abort)) {
        *abort = 1;
        record_timeout(g.st, 12);
        break;
      }
      fence_after();
      const uint32_t d = tmem + b * TN;
      const bool one = far_t3(g, tl);
      bool ok = true;
      for (int kc = 0; kc < kchunks; ++kc) {
        if (!mbar_wait(&full[stage], phase, abort)) {
          *abort = 1;
          record_timeout(g.st, 13);
          ok = false;
          break;
        }
        fence_after();
        const uint32_t sb = smem_u32(smem + stage * STAGE_BYTES);
        const uint64_t ahi = sdesc_sw128(sb), alo = sdesc_sw128(sb + OP_BYTES);
        const uint64_t bhi = sdesc_sw128(sb + 2 * OP_BYTES), blo = sdesc_sw128(sb + 3 * OP_BYTES);
#pragma unroll
        for (int kk = 0; kk < KC / 8; ++kk) {  // K = 8 per instruction: advance 32 bytes
          const uint64_t o = (uint64_t)(kk * 2);
          mma_tf32(d, ahi + o, bhi + o, IDESC, (kc | kk) ? 1u : 0u);
          if (!one) {
            mma_tf32(d, ahi + o, blo + o, IDESC, 1u);
            mma_tf32(d, alo + o, bhi + o, IDESC, 1u);
          }
        }
        mma_commit(&empty[stage]);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!ok) break;
      mma_commit(&accfull[b]);
      ++it;
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: TMEM -> FP64 C ----------------
    // 8 warps: warp w drains TMEM lanes 32*(w%4).. (its row quarter) and column half (w-2)/4
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;
    const int r = quad * 32 + lane;
    int it = 0;
    for (long long t = blockIdx.x; t < g.ntiles && !*abort; t += gridDim.x) {
      T3Tile tl;
      if (!t3_tile(g, t, tl)) continue;
      const int b = it & 1;
      const uint32_t ap = (it >> 1) & 1;
      if (!mbar_wait(&accfull[b], ap, abort)) {
        *abort = 1;
        record_timeout(g.st, 14);
        break;
      }
      fence_after();
      const bool diag = tl.diag;
      const int64_t ldc = tl.ldc;
      double* cp = tl.C + r;
      // two batches of 32 C loads in flight per thread (64 KB per SM), then drain TMEM
#pragma unroll 1
      for (int h2 = 0; h2 < 2; ++h2) {
        const int cb = half * 64 + h2 * 32;
        double cv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) cv[j] = g.store ? 0.0 : __ldcs(cp + (int64_t)(cb + j) * ldc);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          uint32_t acc[16];
          tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + b * TN + cb + c * 16, acc);
          tmem_ld_wait();
          if (h2 == 1 && c == 1) {
            fence_before();
            mbar_arrive(&accempty[b]);
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int cc = cb + c * 16 + j;
            if (diag && cc > r) continue;
            const double v = f32_bits_to_f64(acc[j]);
            __stcs(cp + (int64_t)cc * ldc, g.store ? v : cv[c * 16 + j] - v);
          }
        }
      }
      ++it;
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ===========================================================================
// T3 on CTA pairs: a 256 x 256 output tile per cluster of two CTAs.  Each CTA
// stages its 128 rows of A and its 128 rows of B (TF32 halves); the leader's
// tcgen05.mma.cta_group::2 (M = N = 256) reads both CTAs' stages, so every
// staged byte feeds twice the products of the single-CTA kernel.  Each CTA's
// TMEM receives its own 128 rows x 256 columns; both epilogues drain their own.
// Barriers: full[] lives in the leader (both CTAs' TMA loads complete on it,
// the leader expects both byte counts); empty[] and accfull[] in both (the
// leader's commits multicast to the pair); accempty[] in the leader (every
// epilogue warp of both CTAs arrives on it).
// ===========================================================================
namespace t3p {
constexpr int KC = 32, STAGES = 3;
constexpr int HALF_ROWS = 128;                  // rows of A (and of B) staged by one CTA
constexpr int OP_BYTES = HALF_ROWS * KC * 4;    // 16 KB
constexpr int STAGE_BYTES = 4 * OP_BYTES;       // A_hi, A_lo, B_hi, B_lo halves
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int TILE = 256;
constexpr uint32_t IDESC = idesc(kFmtTF32, TILE, TILE);
constexpr int TMEM_COLS = 512;                  // 2 accumulator buffers x 256 columns
constexpr int kSuper = kPairSuper;              // supertile edge in 256-tiles
}  // namespace t3p

// Pair tiles (units of 256): kEnumFull (bi = t / nt) or kEnumLowerOffBand (supertiles of the
// lower triangle, g.nt tile rows, band in panel-wide tiles).
__device__ __forceinline__ bool decode_pair_tile(const GemmArgs& g, long long t, int& bi, int& bj) {
  if (g.enum_mode == kEnumFull) {
    bi = (int)(t / g.nt);
    bj = (int)(t % g.nt);
    return true;
  }
  constexpr int S = t3p::kSuper;
  const long long sidx = t / (S * S);
  const int loc = (int)(t % (S * S));
  int SI, SJ;
  tile_tri_decode(sidx, SI, SJ);
  bi = SI * S + loc / S;
  bj = SJ * S + loc % S;
  if (bi >= g.nt || bj > bi) return false;
  const int per = g.panel / t3p::TILE;
  return (bi / per - bj / per) > g.band;
}

// Far tiles: when the largest |entries| of the two operand blocks are at most 2^eA and 2^eB
// with eA + eB <= far_thr, the single product hi * hi (relative error ~2^-10 per term) has
// an absolute error no larger than the three-product form makes on blocks of size 1; the
// caller sets far_thr from the scale of Sigma.  Producer and MMA issuer decide alike.
// src 1 asks about the second operand pair (g.K2 > 0), whose rows start at a2_row0 / b2_row0.
__device__ __forceinline__ bool far_tile(const GemmArgs& g, int bi, int bj, int src) {
  const int* eab = src ? g.ea2_blk : g.ea_blk;
  const int* ebb = src ? g.eb2_blk : g.eb_blk;
  if (g.far_thr == INT_MIN || !eab || !ebb) return false;
  const int ea = eab[(src ? g.a2_row0 : g.a_row0) / t3p::TILE + bi];
  const int eb = ebb[(src ? g.b2_row0 : g.b_row0) / t3p::TILE + bj];
  return (long long)ea + (long long)eb <= (long long)g.far_thr;
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kGemmThreads, 1)
    gemm_t3_pair_kernel(const __grid_constant__ CUtensorMap tA_hi, const __grid_constant__ CUtensorMap tA_lo,
                        const __grid_constant__ CUtensorMap tB_hi, const __grid_constant__ CUtensorMap tB_lo,
                        const __grid_constant__ CUtensorMap tA2_hi, const __grid_constant__ CUtensorMap tA2_lo,
                        const __grid_constant__ CUtensorMap tB2_hi, const __grid_constant__ CUtensorMap tB2_lo,
                        const __grid_constant__ GemmArgs g) {
  using namespace t3p;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accfull = empty + STAGES;
  uint64_t* accempty = accfull + 2;
  uint64_t* drain = accempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = (rank == 0);
  const long long pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], 2 * (kEpiThreads / 32));
    }
    mbar_init(drain, 1);
    *abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc_pair(tmem_slot, TMEM_COLS);
  fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs' barriers are initialised before any remote arrival or copy
  fence_after();
  const uint32_t tmem = *tmem_slot;
  // chunks [0, kc1) reduce over the first operand pair, [kc1, kchunks) over the second
  const int kc1 = g.K / KC;
  const int kchunks = kc1 + g.K2 / KC;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer (both CTAs) ----------------
    const uint64_t pol = l2_evict_last_policy();
    prefetch_tmap(&tA_hi);
    prefetch_tmap(&tA_lo);
    prefetch_tmap(&tB_hi);
    prefetch_tmap(&tB_lo);
    if (g.K2 > 0) {
      prefetch_tmap(&tA2_hi);
      prefetch_tmap(&tA2_lo);
      prefetch_tmap(&tB2_hi);
      prefetch_tmap(&tB2_lo);
    }
    int stage = 0;
    uint32_t phase = 0;
    int last_par[STAGES];
    for (int s = 0; s < STAGES; ++s) last_par[s] = -1;
    for (long long t = pair; t < g.ntiles && !*abort; t += npairs) {
      int bi, bj;
      if (!decode_pair_tile(g, t, bi, bj)) continue;
      const int ya1 = g.a_row0 + bi * TILE + (int)rank * HALF_ROWS;
      const int yb1 = g.b_row0 + bj * TILE + (int)rank * HALF_ROWS;
      const int ya2 = g.a2_row0 + bi * TILE + (int)rank * HALF_ROWS;
      const int yb2 = g.b2_row0 + bj * TILE + (int)rank * HALF_ROWS;
      const bool one1 = far_tile(g, bi, bj, 0);
      const bool one2 = g.K2 > 0 && far_tile(g, bi, bj, 1);
      for (int kc = 0; kc < kchunks; ++kc) {
        if (!mbar_wait(&empty[stage], phase ^ 1, abort)) {
          *abort = 1;
          record_timeout(g.st, 51);
          break;
        }
        const bool second = kc >= kc1;
        const bool one = second ? one2 : one1;
        const int kx = (second ? kc - kc1 : kc) * KC;
        const int ya = second ? ya2 : ya1, yb = second ? yb2 : yb1;
        uint8_t* sb = smem + stage * STAGE_BYTES;
        if (leader) mbar_expect_tx(&full[stage], (one ? 1 : 2) * STAGE_BYTES);
        const uint32_t fl = map_to_rank(smem_u32(&full[stage]), 0);
        tma_load_2d_pair_hint(sb, second ? &tA2_hi : &tA_hi, fl, kx, ya, pol);
        if (!one) tma_load_2d_pair_hint(sb + OP_BYTES, second ? &tA2_lo : &tA_lo, fl, kx, ya, pol);
        tma_load_2d_pair_hint(sb + 2 * OP_BYTES, second ? &tB2_hi : &tB_hi, fl, kx, yb, pol);
        if (!one) tma_load_2d_pair_hint(sb + 3 * OP_BYTES, second ? &tB2_lo : &tB_lo, fl, kx, yb, pol);
        last_par[stage] = (int)phase;
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
    if (*abort && leader) {  // the leader's full barriers also count the peer's bytes
      for (int s = 0; s < STAGES; ++s)
        if (last_par[s] >= 0) {
          volatile int never = 0;
          mbar_wait(&full[s], (uint32_t)last_par[s], &never);
        }
    }
  } else if (warp == 1 && lane == 0 && leader) {
    // ---------------- MMA issuer (leader only) ----------------
    int stage = 0;
    uint32_t phase = 0;
    int it = 0;
    for (long long t = pair; t < g.ntiles && !*abort; t += npairs) {
      int bi, bj;
      if (!decode_pair_tile(g, t, bi, bj)) continue;
      const int b = it & 1;
      const uint32_t ap = (it >> 1) & 1;
      if (!mbar_wait(&accempty[b], ap ^ 1, abort)) {
        *abort = 1;
        record_timeout(g.st, 52);
        break;
      }
      fence_after();
      const uint32_t d = tmem + b * TILE;
      const bool one1 = far_tile(g, bi, bj, 0);
      const bool one2 = g.K2 > 0 && far_tile(g, bi, bj, 1);
      bool ok = true;
      for (int kc = 0; kc < kchunks; ++kc) {
        if (!mbar_wait(&full[stage], phase, abort)) {
          *abort = 1;
          record_timeout(g.st, 53);
          ok = false;
          break;
        }
        fence_after();
        const bool one = kc >= kc1 ? one2 : one1;
        const uint32_t sb = smem_u32(smem + stage * STAGE_BYTES);
        const uint64_t ahi = sdesc_sw128(sb), alo = sdesc_sw128(sb + OP_BYTES);
        const uint64_t bhi = sdesc_sw128(sb + 2 * OP_BYTES), blo = sdesc_sw128(sb + 3 * OP_BYTES);
#pragma unroll
        for (int kk = 0; kk < KC / 8; ++kk) {  // K = 8 per instruction: advance 32 bytes
          const uint64_t o = (uint64_t)(kk * 2);
          mma_tf32_pair(d, ahi + o, bhi + o, IDESC, (kc | kk) ? 1u : 0u);
          if (!one) {
            mma_tf32_pair(d, ahi + o, blo + o, IDESC, 1u);
            mma_tf32_pair(d, alo + o, bhi + o, IDESC, 1u);
          }
        }
        mma_commit_pair(&empty[stage], (uint16_t)0x3);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!ok) break;
      mma_commit_pair(&accfull[b], (uint16_t)0x3);
      ++it;
    }
    // every MMA issued has finished before the pair leaves (matters after a time-out)
    mma_commit_pair(drain, (uint16_t)0x1);
    volatile int never = 0;
    mbar_wait(drain, 0, &never);
  } else if (warp >= 2) {
    // ---------------- epilogue (both CTAs): own TMEM -> FP64 C ----------------
    // warp w drains TMEM lanes 32*(w%4).. and the 128-column half (w-2)/4 of the 256 columns
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;
    const int r = quad * 32 + lane;
    const uint32_t accempty_l[2] = {map_to_rank(smem_u32(&accempty[0]), 0), map_to_rank(smem_u32(&accempty[1]), 0)};
    int it = 0;
    for (long long t = pair; t < g.ntiles && !*abort; t += npairs) {
      int bi, bj;
      if (!decode_pair_tile(g, t, bi, bj)) continue;
      const int b = it & 1;
      const uint32_t ap = (it >> 1) & 1;
      if (!mbar_wait(&accfull[b], ap, abort)) {
        *abort = 1;
        record_timeout(g.st, 54);
        break;
      }
      fence_after();
      const int64_t row = g.c_row0 + (int64_t)bi * TILE + (int64_t)rank * HALF_ROWS + r;
      const int64_t col0 = g.c_col0 + (int64_t)bj * TILE + half * 128;
      double* cp = g.C + row + col0 * g.ldc;
      // L2 prefetch two chunks ahead (lane l: column l / 2 of the chunk, rows 16 (l % 2) .. of
      // this warp's 32), and in the last two chunks the first two of this pair's next tile: the
      // loads below then wait on L2 rather than DRAM, and each SM keeps more C lines in flight
      // than its registers hold
      const double* pf = g.C + (row - lane + 16 * (lane & 1)) + (col0 + (lane >> 1)) * g.ldc;
      const double* pf_next = nullptr;
      if (!g.store) {
        for (long long t2 = t + npairs; t2 < g.ntiles; t2 += npairs) {
          int bi2, bj2;
          if (!decode_pair_tile(g, t2, bi2, bj2)) continue;
          pf_next = g.C + (g.c_row0 + (int64_t)bi2 * TILE + (int64_t)rank * HALF_ROWS + quad * 32 + 16 * (lane & 1)) +
                    (g.c_col0 + (int64_t)bj2 * TILE + half * 128 + (lane >> 1)) * g.ldc;
          break;
        }
      }
      // eight 16-column chunks of this warp's 128 columns, the C loads of chunk q + 1 issued
      // before chunk q is drained from TMEM, so their latency hides behind its conversion and stores
      double cbuf[2][16];
#pragma unroll
      for (int j = 0; j < 16; ++j) cbuf[0][j] = g.store ? 0.0 : __ldcs(cp + (int64_t)j * g.ldc);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (!g.store) {
          if (q + 2 < 8)
            prefetch_l2(pf + (int64_t)((q + 2) * 16) * g.ldc);
          else if (pf_next)
            prefetch_l2(pf_next + (int64_t)((q - 6) * 16) * g.ldc);
        }
        if (q + 1 < 8) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            cbuf[(q + 1) & 1][j] = g.store ? 0.0 : __ldcs(cp + (int64_t)((q + 1) * 16 + j) * g.ldc);
        }
        uint32_t acc[16];
        tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + b * TILE + half * 128 + q * 16, acc);
        tmem_ld_wait();
        if (q == 7) {
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive_cluster(accempty_l[b]);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const double v = f32_bits_to_f64(acc[j]);
          __stcs(cp + (int64_t)(q * 16 + j) * g.ldc, g.store ? v : cbuf[q & 1][j] - v);
        }
      }
      ++it;
    }
  }
  fence_before();
  __syncthreads();
  cluster_sync();  // the leader's MMAs read this CTA's shared memory: both stay until both are done
  if (warp == 1) {
    fence_after();
    tmem_dealloc_pair(tmem, TMEM_COLS);
  }
}

// ===========================================================================
// OZ kernel: tile 128 x 32, K chunks of 64 BF16 digits, S = 5 slices, 2 stages.
// ===========================================================================
namespace oz {
constexpr int TM = 128, KC = 64, STAGES = 2, S = kOzSlices;
constexpr int A_BYTES = TM * KC * 2;   // 16 KB per slice
constexpr int TMEM_COLS = 512;         // 2 accumulator buffers of S groups x TN columns
// Per tile width TN (32, or 48 for the band of the trailing update: 27% fewer operand bytes per
// output, and 2 x 5 x 48 = 480 TMEM columns still hold two accumulator buffers)
template <int TN>
struct Cfg {
  static constexpr int B_BYTES = TN * KC * 2;  // per slice
  static constexpr int STAGE_BYTES = S * (A_BYTES + B_BYTES);
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
  static constexpr int GROUP_COLS = TN;        // one accumulator per slice-sum group
  static constexpr int BUF_COLS = S * GROUP_COLS;
  static constexpr int CH = TN / 2;            // columns drained by one epilogue warp
};
static_assert(Cfg<48>::SMEM_BYTES <= 232448, "two 48-wide stages fit in shared memory");
static_assert(2 * Cfg<48>::BUF_COLS <= TMEM_COLS, "two 48-wide accumulator buffers fit in TMEM");

// Tile t of a launch: row block bi (128 rows), column offset cofs (from c_col0 / b_row0) and
// the number of its TN columns inside the output (band tiles of width 48 end ragged at each
// panel boundary: 512 = 10 x 48 + 32).  False: skip the tile.
template <int TN>
__device__ __forceinline__ bool oz_tile(const GemmArgs& g, long long t, int& bi, int& cofs, int& cvalid) {
  if (g.enum_mode != kEnumBand) {  // kEnumFull (TN = 32)
    bi = (int)(t / g.nt);
    cofs = (int)(t % g.nt) * TN;
    cvalid = TN;
    return true;
  }
  const int SI = g.panel / TM, SJ = (g.panel + TN - 1) / TN;
  const long long pair = t / (SI * SJ);
  const int sub = (int)(t % (SI * SJ));
  const int b = g.band;
  const long long head = (long long)b * (b + 1) / 2;
  int I, J;
  if (pair < head) {
    tile_tri_decode(pair, I, J);
  } else {
    I = b + (int)((pair - head) / (b + 1));
    J = I - b + (int)((pair - head) % (b + 1));
  }
  bi = I * SI + sub / SJ;
  const int sj = sub % SJ;
  cofs = J * g.panel + sj * TN;
  cvalid = g.panel - sj * TN < TN ? g.panel - sj * TN : TN;
  // skip tiles strictly above the diagonal
  return (long long)cofs <= (long long)bi * TM + TM - 1;
}
}  // namespace oz

// CL = 2: the CTAs of a cluster pair take adjacent column tiles (bj even, bj + 1) of one row
// block, so they need the same A digits: each loads half of the 128 A rows (map `ta`, 64-row
// boxes) and multicasts it to both, halving the A bytes each CTA pulls through L2 (A is four
// fifths of a tile's operand bytes).  Each CTA's MMA commit releases the stage in both CTAs
// (empty[] counts CL arrivals), since both write into both.  Band and full enumerations list
// the two tiles of a pair consecutively and skip them together; tile counts are even.
template <int CL, int TN>
__global__ void __launch_bounds__(kGemmThreads, 1) gemm_oz_kernel(const __grid_constant__ OzMaps ta,
                                                         const __grid_constant__ OzMaps tb,
                                                         const __grid_constant__ GemmArgs g) {
  using namespace oz;
  using C_ = Cfg<TN>;
  constexpr int B_BYTES = C_::B_BYTES, STAGE_BYTES = C_::STAGE_BYTES, GROUP_COLS = C_::GROUP_COLS,
                BUF_COLS = C_::BUF_COLS, CH = C_::CH;
  static_assert(CL == 1 || TN == 32, "CTA pairs take 32-wide tiles");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accfull = empty + STAGES;
  uint64_t* accempty = accfull + 2;
  uint64_t* drain = accempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = CL > 1 ? (int)cluster_rank() : 0;
  const long long first = CL > 1 ? (long long)(blockIdx.x / CL) : (long long)blockIdx.x;
  const long long step = CL > 1 ? (long long)(gridDim.x / CL) : (long long)gridDim.x;
  const long long nunits = g.ntiles / CL;  // tiles, or tile pairs
  constexpr uint16_t kAll = (uint16_t)((1u << CL) - 1u);
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], CL);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], kEpiThreads);
    }
    mbar_init(drain, 1);
    *abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
  fence_before();
  __syncthreads();
  if (CL > 1) cluster_sync();  // the peer's barriers exist before anything is multicast to them
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const int kchunks = g.K / KC;

  if (warp == 0 && lane == 0) {
    const uint64_t pol = l2_evict_last_policy();
    for (int s = 0; s < S; ++s) {
      prefetch_tmap(&ta.m[s]);
      prefetch_tmap(&tb.m[s]);
    }
    int stage = 0;
    uint32_t phase = 0;
    int last_par[STAGES];
    for (int s = 0; s < STAGES; ++s) last_par[s] = -1;
    for (long long u = first; u < nunits && !*abort; u += step) {
      const long long t = u * CL + rank;
      int bi, cofs, cvalid;
      if (!oz_tile<TN>(g, t, bi, cofs, cvalid)) continue;
      const int ya = g.a_row0 + bi * TM, yb = g.b_row0 + cofs;
      for (int kc = 0; kc < kchunks; ++kc) {
        if (!mbar_wait(&empty[stage], phase ^ 1, abort)) {
          *abort = 1;
          record_timeout(g.st, 21);
          break;
        }
        uint8_t* sb = smem + stage * STAGE_BYTES;
        mbar_expect_tx(&full[stage], STAGE_BYTES);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          if (CL > 1)
            tma_load_2d_mc_hint(sb + s * A_BYTES + rank * (A_BYTES / CL), &ta.m[s], &full[stage], kc * KC,
                                ya + rank * (TM / CL), kAll, pol);
          else
            tma_load_2d_hint(sb + s * A_BYTES, &ta.m[s], &full[stage], kc * KC, ya, pol);
          tma_load_2d_hint(sb + S * A_BYTES + s * B_BYTES, &tb.m[s], &full[stage], kc * KC, yb, pol);
        }
        last_par[stage] = (int)phase;
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
    if (*abort) {
      for (int s = 0; s < STAGES; ++s)
        if (last_par[s] >= 0) {
          volatile int never = 0;
          mbar_wait(&full[s], (uint32_t)last_par[s], &never);
        }
    }
  } else if (warp == 1 && lane == 0) {
    int stage = 0;
    uint32_t phase = 0;
    int it = 0;
    for (long long u = first; u < nunits && !*abort; u += step) {
      const long long t = u * CL + rank;
      int bi, cofs, cvalid;
      if (!oz_tile<TN>(g, t, bi, cofs, cvalid)) continue;
      const int b = it & 1;
      const uint32_t ap = (it >> 1) & 1;
      if (!mbar_wait(&accempty[b], ap ^ 1, abort)) {
        *abort = 1;
        record_timeout(g.st, 22);
        break;
      }
      fence_after();
      const uint32_t d0 = tmem + b * BUF_COLS;
      bool ok = true;
      for (int kc = 0; kc < kchunks; ++kc) {
        if (!mbar_wait(&full[stage], phase, abort)) {
          *abort = 1;
          record_timeout(g.st, 23);
          ok = false;
          break;
        }
        fence_after();
        const uint32_t sb = smem_u32(smem + stage * STAGE_BYTES);
#pragma unroll
        for (int kk = 0; kk < KC / 16; ++kk) {  // K = 16 per instruction: advance 32 bytes
          const uint64_t o = (uint64_t)(kk * 2);
          // The B slices lie one after another (slice t = rows [TN t, TN t + TN) of one
          // SW128 tile) and group g = s + t sits at columns [TN g, TN g + TN), so one
          // MMA of A slice s against B slices 0 .. S-1-s (N = TN (S - s)) adds every
          // product of that slice to its group.  The first (s = 0, N = S TN) writes all
          // groups; sums stay exact integers, so the order changes no bit.
          const uint64_t bb = sdesc_sw128(sb + S * A_BYTES) + o;
#pragma unroll
          for (int s = 0; s < S; ++s) {
            const uint64_t a = sdesc_sw128(sb + s * A_BYTES) + o;
            mma_bf16(d0 + s * GROUP_COLS, a, bb, idesc(kFmtBF16, TM, TN * (S - s)), (kc | kk | s) ? 1u : 0u);
          }
        }
        if (CL > 1)
          mma_commit_mc(&empty[stage], kAll);
        else
          mma_commit(&empty[stage]);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!ok) break;
      mma_commit(&accfull[b]);
      ++it;
    }
    if (CL > 1) {  // every MMA (and so every commit to the peer) has finished before the pair leaves
      mma_commit(drain);
      volatile int never = 0;
      mbar_wait(drain, 0, &never);
    }
  } else if (warp >= 2) {
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;  // columns [CH half, CH half + CH) of the tile
    const int r = quad * 32 + lane;
    int it = 0;
    for (long long u = first; u < nunits && !*abort; u += step) {
      const long long t = u * CL + rank;
      int bi, cofs, cvalid;
      if (!oz_tile<TN>(g, t, bi, cofs, cvalid)) continue;
      const int b = it & 1;
      const uint32_t ap = (it >> 1) & 1;
      if (!mbar_wait(&accfull[b], ap, abort)) {
        *abort = 1;
        record_timeout(g.st, 24);
        break;
      }
      fence_after();
      const int64_t row = g.c_row0 + (int64_t)bi * TM + r;
      const int lc0 = CH * half;  // first tile column of this warp
      const int64_t col0 = g.c_col0 + (int64_t)cofs + lc0;
      double* cp = g.C + row + col0 * g.ldc;
      const bool lower = g.lower_mask != 0;
      // columns of this warp inside the output (ragged tiles end early) and on or below the diagonal
      bool live[CH];
#pragma unroll
      for (int j = 0; j < CH; ++j) live[j] = lc0 + j < cvalid && !(lower && col0 + j > row);
      double cv[CH];
#pragma unroll
      for (int j = 0; j < CH; ++j) cv[j] = (g.store || !live[j]) ? 0.0 : __ldcs(cp + (int64_t)j * g.ldc);
      // group g holds an exact integer a_g (|a_g| < 2^24) of weight 2^(-7(g+2)):
      // V = sum_g a_g 2^(7(4-g)) is an integer below 2^53, combined exactly in int64
      long long V[CH];
#pragma unroll
      for (int j = 0; j < CH; ++j) V[j] = 0;
#pragma unroll
      for (int gs = 0; gs < S; ++gs) {
        uint32_t acc[CH];
        const uint32_t ta0 = tmem + ((uint32_t)(quad * 32) << 16) + b * BUF_COLS + gs * GROUP_COLS + lc0;
        if constexpr (CH == 16) {
          tmem_ld16(ta0, *reinterpret_cast<uint32_t(*)[16]>(acc));
        } else {  // CH = 24: 16 + 8 columns (half 0) or 8 + 16 (half 1), each load aligned to its width
          if (half == 0) {
            tmem_ld16(ta0, *reinterpret_cast<uint32_t(*)[16]>(acc));
            tmem_ld8(ta0 + 16, *reinterpret_cast<uint32_t(*)[8]>(acc + 16));
          } else {
            tmem_ld8(ta0, *reinterpret_cast<uint32_t(*)[8]>(acc));
            tmem_ld16(ta0 + 8, *reinterpret_cast<uint32_t(*)[16]>(acc + 8));
          }
        }
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < CH; ++j) V[j] = V[j] * 128 + (long long)__float2int_rn(__uint_as_float(acc[j]));
      }
      fence_before();
      mbar_arrive(&accempty[b]);
      const int er = g.ea[g.a_row0 + bi * TM + r];
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        if (!live[j]) continue;
        const int ec = g.eb[g.b_row0 + cofs + lc0 + j];
        const double x = i53_to_f64_scaled(V[j], er + ec - 7 * (S + 1));
        __stcs(cp + (int64_t)j * g.ldc, g.store ? x : cv[j] - x);
      }
      ++it;
    }
  }
  fence_before();
  __syncthreads();
  if (CL > 1) cluster_sync();  // the peer's copies into this CTA and commits to its barriers are done
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ===========================================================================
// Split kernel: FP64 rows -> T3 (tf32 hi/lo, row-major) and OZ digits.
// One CTA per kSplitRows rows; K <= kSplitMaxK.  src element (r, k) at src[r*rs + k*cs].
// ===========================================================================
// TF32 rounding (11 significant bits, half away from zero in magnitude) of the
// double with bit pattern D, as FP32 bits; |a| below the FP32 normal range -> 0.
// Integer instructions only (FP64 instructions are the scarce resource here).
__device__ __forceinline__ uint32_t tf32_bits_of(unsigned long long D, unsigned long long* rounded) {
  const unsigned long long sign = D & 0x8000000000000000ull;
  unsigned long long mag = (D & 0x7FFFFFFFFFFFFFFFull) + (1ull << 41);
  mag &= ~((1ull << 42) - 1);
  const int fe = (int)(mag >> 52) - 896;  // FP64 bias 1023 -> FP32 bias 127
  if (fe <= 0) {
    *rounded = sign;
    return (uint32_t)(sign >> 32);
  }
  *rounded = sign | mag;
  return (uint32_t)(sign >> 32) | ((uint32_t)fe << 23) | (uint32_t)((mag >> 29) & 0x7FFFFFu);
}

// Rows [r0, r0 + kSplitRows) of the split (one CTA).
__device__ __forceinline__ void split_rows_body(const double* __restrict__ src, int64_t rs, int64_t cs, int rows,
                                                int K, float* __restrict__ hi, float* __restrict__ lo,
                                                __nv_bfloat16_raw* __restrict__ dig, int64_t dig_stride,
                                                int* __restrict__ ex, int out_row0, int r0) {
  extern __shared__ double tile[];  // kSplitRows x (K + 1)
  const int tid = threadIdx.x;
  const int ld = K + 1;
  // coalesced along whichever source dimension is contiguous; 16 loads in flight per thread
  constexpr int CH = 16;
  const int total = kSplitRows * K;
  for (int base = 0; base < total; base += CH * 256) {
    double v[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int idx = base + u * 256 + tid;
      v[u] = 0.0;
      if (idx < total) {
        const int rr = (cs == 1) ? idx / K : idx % kSplitRows;
        const int k = (cs == 1) ? idx % K : idx / kSplitRows;
        if (r0 + rr < rows) v[u] = src[(int64_t)(r0 + rr) * rs + (int64_t)k * cs];
      }
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int idx = base + u * 256 + tid;
      if (idx < total) {
        const int rr = (cs == 1) ? idx / K : idx % kSplitRows;
        const int k = (cs == 1) ? idx % K : idx / kSplitRows;
        tile[rr * ld + k] = v[u];
      }
    }
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  for (int rr = warp; rr < kSplitRows; rr += blockDim.x / 32) {
    const int row = r0 + rr;
    if (row >= rows) break;
    const int64_t orow = (int64_t)(out_row0 + row);
    // row maximum of |a| on the bit patterns (non-negative doubles order like their bits)
    unsigned long long mxb = 0;
    for (int k = lane; k < K; k += 32) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(tile[rr * ld + k]) & 0x7FFFFFFFFFFFFFFFull;
      mxb = b > mxb ? b : mxb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, mxb, o);
      mxb = ob > mxb ? ob : mxb;
    }
    // max = f 2^e with f in [0.5, 1): e = biased exponent - 1022 (0 for an all-zero row)
    const int e = mxb ? (int)(mxb >> 52) - 1022 : 0;
    if (lane == 0 && ex) ex[orow] = e;
    for (int k = lane; k < K; k += 32) {
      const double a = tile[rr * ld + k];
      const unsigned long long D = (unsigned long long)__double_as_longlong(a);
      if (hi) {
        unsigned long long hd, ld2;
        const uint32_t h = tf32_bits_of(D, &hd);
        const double rem = a - __longlong_as_double((long long)hd);  // exact: a's bits below the rounding point
        const uint32_t l = tf32_bits_of((unsigned long long)__double_as_longlong(rem), &ld2);
        hi[orow * K + k] = __uint_as_float(h);
        lo[orow * K + k] = __uint_as_float(l);
      }
      if (dig) {
        // N = round(a 2^(35-e)) from the bits: a = M 2^(E-1075) with M the 53-bit significand,
        // so a 2^(35-e) = M 2^-(1040+e-E); |a| < 2^e makes the shift >= 18 and |N| <= 2^35.
        long long N = 0;
        const int E = (int)((D >> 52) & 0x7FF);
        if (E != 0) {
          const unsigned long long M = (D & 0xFFFFFFFFFFFFFull) | (1ull << 52);
          const int sh = 1040 + e - E;
          if (sh >= 64) N = 0;
          else if (sh > 0) N = (long long)((M + (1ull << (sh - 1))) >> sh);
          else N = (long long)(M << (-sh));
          if (D >> 63) N = -N;
        }
        // balanced base-128 digits from the least significant end: d = ((N + 64) mod 128) - 64,
        // N = (N - d) / 128.  The leading digit keeps the rest (|d_0| <= 128, |d_s| <= 64
        // otherwise); all are exact in BF16.
        short d[kOzSlices];
#pragma unroll
        for (int s2 = kOzSlices - 1; s2 >= 1; --s2) {
          const long long q = ((N + 64) & 127) - 64;
          d[s2] = (short)q;
          N = (N - q) >> 7;
        }
        d[0] = (short)N;
#pragma unroll
        for (int s2 = 0; s2 < kOzSlices; ++s2) {
          __nv_bfloat16_raw raw;
          raw.x = (unsigned short)(__float_as_uint((float)d[s2]) >> 16);
          dig[(int64_t)s2 * dig_stride + orow * K + k] = raw;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(256) split_rows_kernel(const double* __restrict__ src, int64_t rs, int64_t cs,
                                                         int rows, int K, float* __restrict__ hi,
                                                         float* __restrict__ lo, __nv_bfloat16_raw* __restrict__ dig,
                                                         int64_t dig_stride, int* __restrict__ ex, int out_row0) {
  split_rows_body(src, rs, cs, rows, K, hi, lo, dig, dig_stride, ex, out_row0, blockIdx.x * kSplitRows);
}

// Many pieces in one launch: blockIdx.y = piece, blockIdx.x = 16-row chunk of it.
__global__ void __launch_bounds__(256) split_rows_tasks_kernel(const SplitTask* __restrict__ tasks, int K,
                                                               float* __restrict__ hi, float* __restrict__ lo,
                                                               __nv_bfloat16_raw* __restrict__ dig,
                                                               int64_t dig_stride, int* __restrict__ ex) {
  const SplitTask t = tasks[blockIdx.y];
  const int r0 = blockIdx.x * kSplitRows;
  if (r0 >= t.rows) return;  // uniform over the CTA, before any barrier
  split_rows_body(t.src, t.rs, t.cs, t.rows, K, hi, lo, dig, dig_stride, ex, t.out_row0, r0);
}

// Per 256-row block maximum of the row exponents (rows past the end count as -infinity).
__global__ void __launch_bounds__(256) row_exp_blockmax_kernel(const int* __restrict__ ex, int64_t rows,
                                                               int* __restrict__ exb) {
  const int64_t r = (int64_t)blockIdx.x * 256 + threadIdx.x;
  int v = r < rows ? ex[r] : INT_MIN;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ int w[8];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = w[0];
    for (int i = 1; i < 8; ++i) m = max(m, w[i]);
    exb[blockIdx.x] = m;
  }
}

// ===========================================================================
// host side
// ===========================================================================
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2-D row-major tensor [rows][K] of 4-byte (fp32) or 2-byte (bf16) elements,
// box = (box_k, box_rows), 128-byte swizzle.
cudaError_t make_tmap(CUtensorMap* m, const void* base, int64_t rows, int K, int elem_bytes, int box_k, int box_rows) {
  auto enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  if (((uintptr_t)base & 15) != 0 || ((int64_t)K * elem_bytes) % 16 != 0 || box_k * elem_bytes != 128)
    return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)K * elem_bytes};
  cuuint32_t box[2] = {(cuuint32_t)box_k, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_split_maps(SplitOperand& op) {
  cudaError_t e = cudaSuccess;
  if (op.hi) {
    if ((e = make_tmap(&op.t_hi, op.hi, op.rows, op.K, 4, 32, 128)) != cudaSuccess) return e;
    if ((e = make_tmap(&op.t_lo, op.lo, op.rows, op.K, 4, 32, 128)) != cudaSuccess) return e;
  }
  if (op.dig) {
    for (int s = 0; s < kOzSlices; ++s) {
      const void* base = (const uint8_t*)op.dig + (size_t)s * op.rows * op.K * 2;
      if ((e = make_tmap(&op.oz_a.m[s], base, op.rows, op.K, 2, 64, 128)) != cudaSuccess) return e;
      if ((e = make_tmap(&op.oz_b.m[s], base, op.rows, op.K, 2, 64, 32)) != cudaSuccess) return e;
      if ((e = make_tmap(&op.oz_ah.m[s], base, op.rows, op.K, 2, 64, 64)) != cudaSuccess) return e;
      if ((e = make_tmap(&op.oz_b48.m[s], base, op.rows, op.K, 2, 64, 48)) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_split_rows(cudaStream_t s, const double* src, int64_t rs, int64_t cs, int rows, int K,
                              SplitOperand& op, int out_row0) {
  if (rows <= 0) return cudaSuccess;
  if (K > kSplitMaxK) return cudaErrorInvalidValue;
  const size_t smem = (size_t)kSplitRows * (K + 1) * sizeof(double);
  static PerDeviceOnce attr_once;
  cudaError_t e = attr_once([] {
    return cudaFuncSetAttribute(split_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kSplitRows * (kSplitMaxK + 1) * (int)sizeof(double));
  });
  if (e != cudaSuccess) return e;
  split_rows_kernel<<<(rows + kSplitRows - 1) / kSplitRows, 256, smem, s>>>(src, rs, cs, rows, K, op.hi, op.lo,
                                                        (__nv_bfloat16_raw*)op.dig, (int64_t)op.rows * op.K, op.ex,
                                                        out_row0);
  return cudaGetLastError();
}

cudaError_t launch_split_rows_tasks(cudaStream_t s, const SplitTask* d_tasks, int ntasks, int max_rows, int K,
                                    SplitOperand& op) {
  if (ntasks <= 0 || max_rows <= 0) return cudaSuccess;
  if (K > kSplitMaxK) return cudaErrorInvalidValue;
  const size_t smem = (size_t)kSplitRows * (K + 1) * sizeof(double);
  static PerDeviceOnce attr_once;
  cudaError_t e = attr_once([] {
    return cudaFuncSetAttribute(split_rows_tasks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kSplitRows * (kSplitMaxK + 1) * (int)sizeof(double));
  });
  if (e != cudaSuccess) return e;
  split_rows_tasks_kernel<<<dim3((unsigned)((max_rows + kSplitRows - 1) / kSplitRows), (unsigned)ntasks), 256, smem,
                            s>>>(d_tasks, K, op.hi, op.lo, (__nv_bfloat16_raw*)op.dig, (int64_t)op.rows * op.K, op.ex);
  return cudaGetLastError();
}

static int num_sms() {
  static std::atomic<int> cache[64];
  const int n = per_device_int(cache, [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v;
  });
  return n > 0 ? n : 148;
}

int tc_num_sms() { return num_sms(); }

cudaError_t launch_gemm_t3(cudaStream_t s, const SplitOperand& A, const SplitOperand& B, const GemmArgs& g,
                           int max_ctas) {
  if (g.ntiles <= 0) return cudaSuccess;
  static PerDeviceOnce attr_once;
  {
    const cudaError_t e =
        attr_once([] { return cudaFuncSetAttribute(gemm_t3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, t3::SMEM_BYTES); });
    if (e != cudaSuccess) return e;
  }
  int cap = num_sms();
  if (max_ctas > 0 && max_ctas < cap) cap = max_ctas;
  const int grid = (int)(g.ntiles < cap ? g.ntiles : cap);
  gemm_t3_kernel<<<grid, kGemmThreads, t3::SMEM_BYTES, s>>>(A.t_hi, A.t_lo, B.t_hi, B.t_lo, g);
  return cudaGetLastError();
}

cudaError_t launch_row_exp_blockmax(cudaStream_t s, SplitOperand& op, int64_t rows) {
  if (!op.ex || !op.exb || rows <= 0) return cudaSuccess;
  row_exp_blockmax_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(op.ex, rows, op.exb);
  return cudaGetLastError();
}

cudaError_t launch_gemm_t3_pair(cudaStream_t s, const SplitOperand& A, const SplitOperand& B, const GemmArgs& g,
                                int max_ctas, const SplitOperand* A2, const SplitOperand* B2) {
  if (g.K2 > 0 && (!A2 || !B2)) return cudaErrorInvalidValue;
  if (g.K2 <= 0) A2 = &A, B2 = &B;
  if (g.ntiles <= 0) return cudaSuccess;
  static PerDeviceOnce attr_once;
  {
    const cudaError_t e =
        attr_once([] { return cudaFuncSetAttribute(gemm_t3_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, t3p::SMEM_BYTES); });
    if (e != cudaSuccess) return e;
  }
  int cap = num_sms();
  if (max_ctas > 0 && max_ctas < cap) cap = max_ctas;
  const long long pairs = g.ntiles < cap / 2 ? g.ntiles : cap / 2;
  if (pairs < 1) return cudaErrorInvalidValue;
  gemm_t3_pair_kernel<<<(unsigned)(2 * pairs), kGemmThreads, t3p::SMEM_BYTES, s>>>(
      A.t_hi, A.t_lo, B.t_hi, B.t_lo, A2->t_hi, A2->t_lo, B2->t_hi, B2->t_lo, g);
  return cudaGetLastError();
}

cudaError_t launch_gemm_oz(cudaStream_t s, const SplitOperand& A, const SplitOperand& B, const GemmArgs& g,
                           int max_ctas) {
  if (g.ntiles <= 0) return cudaSuccess;
  static PerDeviceOnce attr_once;
  {
    const cudaError_t e = attr_once([] {
      cudaError_t r = cudaFuncSetAttribute(gemm_oz_kernel<1, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           oz::Cfg<32>::SMEM_BYTES);
      if (r == cudaSuccess)
        r = cudaFuncSetAttribute(gemm_oz_kernel<2, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 oz::Cfg<32>::SMEM_BYTES);
      if (r == cudaSuccess)
        r = cudaFuncSetAttribute(gemm_oz_kernel<1, 48>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 oz::Cfg<48>::SMEM_BYTES);
      return r;
    });
    if (e != cudaSuccess) return e;
  }
  int cap = num_sms();
  if (max_ctas > 0 && max_ctas < cap) cap = max_ctas;
  GemmArgs g2 = g;
  g2.ea = A.ex;
  g2.eb = B.ex;
  if (g.enum_mode == kEnumBand && g.panel % 128 == 0) {
    // band tiles 128 x 48 (the caller counts 128 x 32 sub-tiles per panel pair)
    const long long per32 = (long long)(g.panel / 128) * (g.panel / 32);
    const long long per48 = (long long)(g.panel / 128) * ((g.panel + 47) / 48);
    g2.ntiles = g.ntiles / per32 * per48;
    const int grid = (int)(g2.ntiles < cap ? g2.ntiles : cap);
    gemm_oz_kernel<1, 48><<<grid, kGemmThreads, oz::Cfg<48>::SMEM_BYTES, s>>>(A.oz_a, B.oz_b48, g2);
    return cudaGetLastError();
  }
  // CTA pairs sharing the A digits when the tiles pair up (even counts) and the launch may use
  // most of the GPU: a cluster needs two free SMs of one GPC at once, which a small SM share
  // beside other running kernels may not offer (the launch would then wait for them)
  if (g.ntiles % 2 == 0 && cap >= 64 && g.enum_mode == kEnumFull && g.nt % 2 == 0) {
    const long long pairs = g.ntiles / 2;
    const int grid = 2 * (int)(pairs < cap / 2 ? pairs : cap / 2);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kGemmThreads);
    cfg.dynamicSmemBytes = oz::Cfg<32>::SMEM_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, gemm_oz_kernel<2, 32>, A.oz_ah, B.oz_b, g2);
  }
  const int grid = (int)(g.ntiles < cap ? g.ntiles : cap);
  gemm_oz_kernel<1, 32><<<grid, kGemmThreads, oz::Cfg<32>::SMEM_BYTES, s>>>(A.oz_a, B.oz_b, g2);
  return cudaGetLastError();
}

}  // namespace exa
