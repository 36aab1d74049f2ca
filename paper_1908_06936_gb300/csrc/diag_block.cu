// FP64 factorisation and inversion of one 512 x 512 diagonal block of the mixed-precision
// Cholesky (the diagonal tiles that the MP variant of Section II-A, Fig. 1(d), keeps in double
// precision), as ONE cooperative launch on a few SMs.
//
// On this part FP64 issues at ~4 flops per clock per SM, so the block's ~90 MFLOP (Cholesky
// 512^3/3 and inverse 512^3/3) need ~0.7 ms on 16 SMs; chained as ~30 small launches they took
// ~4.8 ms, the pace-setter of the look-ahead stream.  Here every CTA of a cooperative grid works
// through the same steps, separated by grid-wide barriers (bounded waits; every CTA reaches every
// barrier; a failed pivot only turns values into NaN and is recorded in the status):
//
//   Cholesky, right-looking in 64-wide steps j (c0 = 64 j):
//     (a) CTA 0: D = chol(A_jj) and V_j = D^-1 in shared memory (unblocked, column by column)
//     (b) L_rj = A_rj V_j^T for the 32-row strips r below, into a scratch panel P (one task per
//         strip and 32-column half)
//     (c) A_rc -= L_rj L_cj^T over the 32 x 32 lower tiles of the trailing block, from P, while P
//         is copied into the matrix; CTA 0 updates the next leaf first and runs its (a) meanwhile
//   Inverse W = L^-1 by doubling: the 64-inverses V_j are the leaves; a 2b block
//   [[X_A, 0], [L_BA, X_B]] has inverse [[W_A, 0], [-W_B (L_BA W_A), W_B]], formed for
//   b = 64, 128, 256 as two steps of 32 x 32 product tasks each.
//
// Outputs: L in the block's lower triangle (upper triangle untouched), log L_ii summed in row
// order per 128 sub-tile, the four 128 x 128 sub-tile inverses (row-major, zero above the
// diagonal) and the 512 x 512 inverse (row-major, zero above the diagonal).
#include <math.h>

#include "exa_internal.cuh"

namespace exa {

constexpr int kDB = 512;        // block size
constexpr int kDW = 64;         // Cholesky step / inverse leaf
constexpr int kDT = 32;         // product task tile
constexpr int kDThreads = 256;
constexpr int kDSteps = kDB / kDW;
// scratch (doubles): the eight 64-inverses, the 256 x 256 product of the widest inverse step,
// then the current Cholesky step's panel (448 x 64)
constexpr int64_t kDiagT = (int64_t)kDSteps * kDW * kDW;
constexpr int64_t kDiagP = kDiagT + 256 * 256;
constexpr int64_t kDiagBar = kDiagP + (int64_t)(kDB - kDW) * kDW;  // barrier counter, abort flag, lead counter
constexpr int64_t kDiagScratch = kDiagBar + 2;
constexpr long long kDiagSpin = 2000000000LL;  // bound of one barrier wait, SM clock cycles (~1 s)

struct DiagArgs {
  double* a;            // column-major matrix, element (i, j) at a[i + j * ld]
  int64_t ld, k0;       // block origin (k0, k0)
  double* w_sub;        // four 128 x 128 row-major sub-tile inverses (w_all + (k0 / 128) 128^2)
  double* logdet;       // four sub-tile log sums (logdet_part + k0 / 128)
  double* w2;           // 512 x 512 row-major inverse
  double* scr;          // kDiagScratch doubles
  DevStatus* st;
};

// Grid-wide barrier of the cooperative launch (all CTAs co-resident): CTA leader arrives on a
// monotone counter and waits, bounded, until all G CTAs of barrier number `n` (1, 2, ...) have
// arrived.  On time-out the status records it, the abort flag releases every later wait, and the
// (then meaningless) results are discarded by the caller through the status.
__device__ __forceinline__ void grid_barrier(unsigned int* count, volatile int* abort, unsigned int target,
                                             DevStatus* st) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    const long long t0 = clock64();
    while (*(volatile unsigned int*)count < target && !*abort) {
      if (clock64() - t0 > kDiagSpin) {
        if (atomicExch((int*)abort, 1) == 0 && atomicExch(&st->timeout, 1) == 0) st->timeout_where = 71;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
}

// acc[u][v] (u, v in {0, 1}) += sum_k A(r, k) B(c, k) over k in [0, K) for the 32 x 32 tile
// rows r = 2 ty + u, columns c = 2 tx + v (ty, tx in [0, 16)), with
// A(r, k) = pa[r * ars + k * acs] and B(c, k) = pb[c * brs + k * bcs]; K a multiple of 32.
__device__ __forceinline__ void tile_gemm(double acc[2][2], const double* pa, int64_t ars, int64_t acs,
                                          const double* pb, int64_t brs, int64_t bcs, int K, double* sA,
                                          double* sB) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int k0 = 0; k0 < K; k0 += kDT) {
    __syncthreads();  // the previous chunk (or the caller's use of sA / sB) is finished
    for (int idx = tid; idx < kDT * kDT; idx += kDThreads) {
      // consecutive threads walk the dimension with the smaller stride
      const int p = idx & 31, q = idx >> 5;
      const int ra = (acs == 1) ? q : p, ka = (acs == 1) ? p : q;
      const int rb = (bcs == 1) ? q : p, kb = (bcs == 1) ? p : q;
      // L2 loads (ld.global.cg): the operands were written by other CTAs since the last barrier
      sA[ra * (kDT + 1) + ka] = __ldcg(pa + (int64_t)ra * ars + (int64_t)(k0 + ka) * acs);
      sB[rb * (kDT + 1) + kb] = __ldcg(pb + (int64_t)rb * brs + (int64_t)(k0 + kb) * bcs);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kDT; ++k) {
      const double a0 = sA[(2 * ty) * (kDT + 1) + k], a1 = sA[(2 * ty + 1) * (kDT + 1) + k];
      const double b0 = sB[(2 * tx) * (kDT + 1) + k], b1 = sB[(2 * tx + 1) * (kDT + 1) + k];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
  }
}

__device__ __forceinline__ void zero_acc(double acc[2][2]) { acc[0][0] = acc[0][1] = acc[1][0] = acc[1][1] = 0.0; }

// (a) of step j on one CTA: chol of the 64 x 64 diagonal block and its inverse, in shared memory
// (S: 64 x 65 factor, V: 64 x 65 inverse, T: 32 x 33 products, R: 64 reciprocal square roots).
//
// Cost model (measured on this part with dependent-chain probes): a dependent FP64 operation
// costs ~64 SM cycles whatever the number of active lanes, a division ~430, a square root ~675,
// a reciprocal square root ~430; FP32 ~5.  So the leaf keeps its sequential chain short in
// FP64 instructions and spreads independent ones over the four SM sub-partitions:
//   * one reciprocal square root per column, r_c = 1 / sqrt(d_c), which gives the pivot
//     (d_c r_c), the column scale and the inverse's diagonal (V_cc = r_c): no divisions;
//   * 16-column panels over all rows of the leaf, factored right-looking by four groups of 64
//     threads: thread t of group q holds row p0 + t of the panel columns p0 + q + 4u (u < 4)
//     in registers, the group owning column c scales it, every group updates its own columns;
//   * the trailing part of the leaf after each panel as one product over all threads;
//   * the four 16 x 16 diagonal inverses on four warps (one per sub-partition), then doubling.
constexpr int kLeafPW = 16;
constexpr int kLeafSmem = 2 * kDW * (kDW + 1) + 32 * 33 + kDW;  // doubles

__device__ void diag_leaf(const DiagArgs& g, int j, double* S) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t c0 = g.k0 + (int64_t)j * kDW;
  double* A = g.a + c0 + c0 * g.ld;
  constexpr int sd = kDW + 1;
  double* V = S + kDW * sd;    // inverse, 64 x 65
  double* T = V + kDW * sd;    // 32 x 33 products
  double* R = T + 32 * 33;     // r_c = 1 / L_cc
  for (int idx = tid; idx < kDW * kDW; idx += kDThreads) {
    const int i = idx & (kDW - 1), c = idx / kDW;
    S[i * sd + c] = (i >= c) ? __ldcg(A + i + (int64_t)c * g.ld) : 0.0;
    V[(idx / kDW) * sd + (idx & (kDW - 1))] = 0.0;
  }
  __syncthreads();
  const int grp = tid >> 6, t64 = tid & 63;
  for (int p0 = 0; p0 < kDW; p0 += kLeafPW) {
    const int i = p0 + t64;  // this thread's row of the panel
    const bool own = i < kDW;
    double a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] = own ? S[i * sd + p0 + grp + 4 * u] : 0.0;
#pragma unroll
    for (int cc = 0; cc < kLeafPW; ++cc) {
      const int c = p0 + cc;
      if (grp == (cc & 3)) {  // the group owning column c: pivot, scale (d_c was published in S)
        double d = S[c * sd + c];
        if (!(d > 0.0) || !isfinite(d)) {  // uniform across the group
          if (t64 == 0) {
            atomicMin(&g.st->pivot, (long long)(c0 + c));
            atomicExch(&g.st->info, 1);
          }
          d = NAN;  // the rest becomes NaN; every barrier is still reached
        }
        const double r = rsqrt(d);
        if (own && i >= c) {
          double v = 0.0;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (u == (cc >> 2)) v = (i == c) ? d * r : a[u] * r;
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (u == (cc >> 2)) a[u] = v;
          S[i * sd + c] = v;
        }
        if (t64 == 0) R[c] = r;
      }
      __syncthreads();
      // a_il -= L_ic L_lc for this group's columns l > c (rows i >= l)
      if (own && i > c) {
        const double lic = S[i * sd + c];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int l = p0 + grp + 4 * u;
          if (l > c && i >= l) a[u] = fma(-lic, S[l * sd + c], a[u]);
        }
      }
      // publish the next pivot d_{c+1} from its owner's registers
      if (cc + 1 < kLeafPW && grp == ((cc + 1) & 3) && i == c + 1) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u == ((cc + 1) >> 2)) S[i * sd + c + 1] = a[u];
      }
      __syncthreads();
    }
    const int m = kDW - p0 - kLeafPW;  // rows below the panel within the leaf
    if (m > 0) {
      // trailing update of the leaf: S_il -= sum_k L_ik L_lk over the panel's 16 columns
      for (int idx = tid; idx < m * m; idx += kDThreads) {
        const int ii = p0 + kLeafPW + idx / m, l = p0 + kLeafPW + idx % m;
        if (ii < l) continue;
        double t0 = S[ii * sd + l], t1 = 0.0;
#pragma unroll
        for (int k = 0; k < kLeafPW; k += 2) {
          t0 = fma(-S[ii * sd + p0 + k], S[l * sd + p0 + k], t0);
          t1 = fma(-S[ii * sd + p0 + k + 1], S[l * sd + p0 + k + 1], t1);
        }
        S[ii * sd + l] = t0 + t1;
      }
      __syncthreads();
    }
  }
  // L back to the matrix (lower triangle)
  for (int idx = tid; idx < kDW * kDW; idx += kDThreads) {
    const int ii = idx & (kDW - 1), c = idx / kDW;
    if (ii >= c) A[ii + (int64_t)c * g.ld] = S[ii * sd + c];
  }
  // the four 16 x 16 diagonal inverses, warp w < 4 taking block w (lane = row), column by column
  // from the last: V_cc = r_c, V_ic = -r_c sum_{l = c+1..i} V_il L_lc (two partial sums)
  if (warp < 4 && lane < kLeafPW) {
    const int q0 = warp * kLeafPW, ii = q0 + lane;
    for (int c = kLeafPW - 1; c >= 0; --c) {
      const double rc = R[q0 + c];
      if (lane > c) {
        double s0 = 0.0, s1 = 0.0;
        int l = c + 1;
        for (; l + 1 <= lane; l += 2) {
          s0 = fma(V[ii * sd + q0 + l], S[(q0 + l) * sd + q0 + c], s0);
          s1 = fma(V[ii * sd + q0 + l + 1], S[(q0 + l + 1) * sd + q0 + c], s1);
        }
        if (l <= lane) s0 = fma(V[ii * sd + q0 + l], S[(q0 + l) * sd + q0 + c], s0);
        V[ii * sd + q0 + c] = -(s0 + s1) * rc;
      } else if (lane == c) {
        V[ii * sd + q0 + c] = rc;
      }
      __syncwarp(0x0000FFFFu);
    }
  }
  __syncthreads();
  // V = L^-1 by doubling: [[V_A, 0], [L_BA, V_B]]^-1 has off-diagonal block -V_B (L_BA V_A)
  for (int h = kLeafPW; h < kDW; h *= 2) {
    const int pairs = kDW / (2 * h);
    for (int idx = tid; idx < pairs * h * h; idx += kDThreads) {
      const int p = idx / (h * h), r = (idx / h) % h, c = idx % h, o = p * 2 * h;
      double t0 = 0.0, t1 = 0.0;
      int k = c;
      for (; k + 1 < h; k += 2) {
        t0 = fma(S[(o + h + r) * sd + o + k], V[(o + k) * sd + o + c], t0);
        t1 = fma(S[(o + h + r) * sd + o + k + 1], V[(o + k + 1) * sd + o + c], t1);
      }
      if (k < h) t0 = fma(S[(o + h + r) * sd + o + k], V[(o + k) * sd + o + c], t0);
      T[p * 16 * 33 * (h == kLeafPW) + r * 33 + c] = t0 + t1;  // h = 16: pairs at rows 0 and 16
    }
    __syncthreads();
    for (int idx = tid; idx < pairs * h * h; idx += kDThreads) {
      const int p = idx / (h * h), r = (idx / h) % h, c = idx % h, o = p * 2 * h;
      const double* Tp = T + p * 16 * 33 * (h == kLeafPW);
      double t0 = 0.0, t1 = 0.0;
      int k = 0;
      for (; k + 1 <= r; k += 2) {
        t0 = fma(V[(o + h + r) * sd + o + h + k], Tp[k * 33 + c], t0);
        t1 = fma(V[(o + h + r) * sd + o + h + k + 1], Tp[(k + 1) * 33 + c], t1);
      }
      if (k <= r) t0 = fma(V[(o + h + r) * sd + o + h + k], Tp[k * 33 + c], t0);
      V[(o + h + r) * sd + o + c] = -(t0 + t1);
    }
    __syncthreads();
  }
  double* Vg = g.scr + (int64_t)j * kDW * kDW;  // row-major, zero above the diagonal
  for (int idx = tid; idx < kDW * kDW; idx += kDThreads) {
    const int r = idx / kDW, c = idx & (kDW - 1);
    Vg[idx] = (c <= r) ? V[r * sd + c] : 0.0;
  }
}

__global__ void __launch_bounds__(kDThreads) diag_block_kernel(const __grid_constant__ DiagArgs g) {
  extern __shared__ double smem[];
  double* S = smem;                          // leaf workspace (CTA 0), kLeafSmem doubles
  double* sA = smem + kLeafSmem;             // 32 x 33 staging
  double* sB = sA + kDT * (kDT + 1);
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  unsigned int* bar = (unsigned int*)(g.scr + kDiagBar);
  volatile int* abort = (volatile int*)(bar + 1);
  unsigned int* leadcnt = bar + 2;  // lead tiles finished by CTAs other than 0 (monotone)
  unsigned int nbar = 0, lead_target = 0;
  auto sync_all = [&]() { grid_barrier(bar, abort, (++nbar) * (unsigned int)G, g.st); };
  const int64_t ld = g.ld, k0 = g.k0;
  double* a = g.a;
  double* P = g.scr + kDiagP;  // the current step's panel below the leaf, 448 x 64 row-major

  // ---------------- Cholesky in 64-wide steps ----------------
  // Per step j: (b) the panel below the leaf into P, then (c) the trailing update from P while
  // P is copied into the matrix; CTA 0 takes the three tiles of the next leaf first and factors
  // it during the rest of (c) (look-ahead), so the serial leaves overlap the updates.
  if (b == 0) diag_leaf(g, 0, S);
  sync_all();
  for (int j = 0; j < kDSteps; ++j) {
    const int64_t c0 = k0 + (int64_t)j * kDW;
    const int below = kDB - (j + 1) * kDW;  // rows of the block below step j
    const int ns = below / kDT;             // 32-row strips
    const double* V = g.scr + (int64_t)j * kDW * kDW;
    // (b) P(r, c) = sum_k A(c0 + 64 + r, c0 + k) V(c, k): one task per strip and 32-column half
    //     (V is lower triangular, so the first half needs only the first 32 columns of A)
    for (int t = b; t < 2 * ns; t += G) {
      const int strip = t >> 1, half = t & 1;
      const int64_t r0 = c0 + kDW + (int64_t)strip * kDT;
      double acc[2][2];
      zero_acc(acc);
      tile_gemm(acc, a + r0 + c0 * ld, 1, ld, V + half * kDT * kDW, kDW, 1, (half + 1) * kDT, sA, sB);
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) P[(strip * kDT + 2 * ty + u) * kDW + half * kDT + 2 * tx + v] = acc[u][v];
    }
    sync_all();
    // (c) A_rc -= L_r L_c^T over the 32 x 32 lower tiles (R >= C) of the rows below step j, from P;
    //     tiles 0..2 (the next leaf) on CTA 0, which then factors that leaf; the others, and the copy
    //     of P into the matrix, on CTAs 1..G-1
    const int nt = ns * (ns + 1) / 2;
    auto update_tile = [&](int t) {
      int R = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
      while (R * (R + 1) / 2 > t) --R;
      while ((R + 1) * (R + 2) / 2 <= t) ++R;
      const int C = t - R * (R + 1) / 2;
      const int64_t rr = c0 + kDW + (int64_t)R * kDT, cc = c0 + kDW + (int64_t)C * kDT;
      double acc[2][2];
      zero_acc(acc);
      tile_gemm(acc, P + (int64_t)R * kDT * kDW, kDW, 1, P + (int64_t)C * kDT * kDW, kDW, 1, kDW, sA, sB);
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const int i = 2 * ty + u, c = 2 * tx + v;
          if (R == C && c > i) continue;
          double* pc = a + (rr + i) + (cc + c) * ld;
          *pc = __ldcg(pc) - acc[u][v];
        }
    };
    // the three tiles of the next leaf on CTAs 0, 1, 2 (CTA 0 where the grid is smaller); the
    // others count their tile on a monotone counter that CTA 0 waits for before the leaf
    const int lead = nt < 3 ? nt : 3;
    int foreign = 0;  // lead tiles of this step on CTAs other than 0
    for (int t = 0; t < lead; ++t) {
      const int owner = t < G ? t : 0;
      foreign += owner != 0;
      if (owner == b) update_tile(t);
    }
    if (b != 0 && b < lead) {
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        atomicAdd(leadcnt, 1u);
      }
    }
    lead_target += (unsigned int)foreign;
    if (b == 0) {
      if (j + 1 < kDSteps) {
        if (tid == 0) {
          const long long t0 = clock64();
          while (*(volatile unsigned int*)leadcnt < lead_target && !*abort) {
            if (clock64() - t0 > kDiagSpin) {
              if (atomicExch((int*)abort, 1) == 0 && atomicExch(&g.st->timeout, 1) == 0) g.st->timeout_where = 72;
              break;
            }
            __nanosleep(32);
          }
          __threadfence();
        }
        __syncthreads();  // the leaf's tiles are written
        diag_leaf(g, j + 1, S);
      }
    } else {
      for (int t = lead + (b - 1); t < nt; t += G - 1) update_tile(t);
      for (int64_t idx = (int64_t)(b - 1) * kDThreads + tid; idx < (int64_t)below * kDW;
           idx += (int64_t)(G - 1) * kDThreads) {
        const int r = (int)(idx % below), c = (int)(idx / below);
        a[(c0 + kDW + r) + (c0 + c) * ld] = __ldcg(P + (int64_t)r * kDW + c);
      }
    }
    sync_all();
  }

  // ---------------- log-determinant parts, leaves of the inverse ----------------
  for (int s4 = b; s4 < 4 && tid == 0; s4 += G) {
    double s = 0.0;
    for (int i = 0; i < 128; ++i) {
      const int64_t r = k0 + 128 * s4 + i;
      s += log(__ldcg(a + r + r * ld));
    }
    g.logdet[s4] = s;
  }
  double* w2 = g.w2;
  // W2 <- zero above the diagonal, the 64-inverses on the diagonal (other lower entries later)
  for (int64_t idx = (int64_t)b * kDThreads + tid; idx < (int64_t)kDB * kDB; idx += (int64_t)G * kDThreads) {
    const int r = (int)(idx / kDB), c = (int)(idx % kDB);
    if (c > r) {
      w2[idx] = 0.0;
    } else if (r / kDW == c / kDW) {
      const double* V = g.scr + (int64_t)(r / kDW) * kDW * kDW;
      w2[idx] = __ldcg(V + (r % kDW) * kDW + (c % kDW));
    }
  }
  sync_all();

  // ---------------- inverse by doubling: widths h = 64, 128, 256 ----------------
  double* T = g.scr + kDiagT;  // h x h product, row-major
  for (int h = kDW; h < kDB; h *= 2) {
    const int pairs = kDB / (2 * h);             // blocks of width 2h
    const int tiles = (h / kDT) * (h / kDT);     // 32 x 32 tiles of one h x h product
    // first product: T_p = L_BA W_A  (L_BA: rows p 2h + h .., columns p 2h ..; W_A lower, row-major in w2)
    for (int t = b; t < pairs * tiles; t += G) {
      const int p = t / tiles, q = t % tiles, ti = q / (h / kDT), tj = q % (h / kDT);
      const int64_t o = (int64_t)p * 2 * h;  // block origin within the 512 block
      double acc[2][2];
      zero_acc(acc);
      // T(r, c) = sum_k L(o + h + r, o + k) W(o + k, o + c): W_A(k, c) = 0 for k < c
      const int kstart = tj * kDT;
      tile_gemm(acc, a + (k0 + o + h + ti * kDT) + (k0 + o + kstart) * ld, 1, ld,
                w2 + (o + kstart) * kDB + (o + tj * kDT), 1, kDB, h - kstart, sA, sB);
      double* Tp = T + (int64_t)p * h * h;
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) Tp[(ti * kDT + 2 * ty + u) * h + tj * kDT + 2 * tx + v] = acc[u][v];
    }
    sync_all();
    // second product: W_BA = -W_B T_p  (W_B lower, row-major in w2 at (o + h, o + h))
    for (int t = b; t < pairs * tiles; t += G) {
      const int p = t / tiles, q = t % tiles, ti = q / (h / kDT), tj = q % (h / kDT);
      const int64_t o = (int64_t)p * 2 * h;
      const double* Tp = T + (int64_t)p * h * h;
      double acc[2][2];
      zero_acc(acc);
      // W_BA(r, c) = -sum_k W_B(r, k) T(k, c): W_B(r, k) = 0 for k > r
      const int kend = (ti + 1) * kDT;
      tile_gemm(acc, w2 + (o + h + ti * kDT) * kDB + (o + h), kDB, 1, Tp + tj * kDT, 1, h, kend, sA, sB);
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) w2[(o + h + ti * kDT + 2 * ty + u) * kDB + o + tj * kDT + 2 * tx + v] = -acc[u][v];
    }
    sync_all();
  }

  // ---------------- the four 128 sub-tile inverses (diagonal blocks of W2) ----------------
  for (int64_t idx = (int64_t)b * kDThreads + tid; idx < 4 * 128 * 128; idx += (int64_t)G * kDThreads) {
    const int s = (int)(idx / (128 * 128)), rc = (int)(idx % (128 * 128)), r = rc / 128, c = rc % 128;
    g.w_sub[idx] = __ldcg(w2 + (int64_t)(128 * s + r) * kDB + 128 * s + c);
  }
}

size_t diag_block_scratch_doubles() { return (size_t)kDiagScratch; }

cudaError_t launch_diag_block(cudaStream_t s, double* a, int64_t ld, int64_t k0, double* w_sub, double* logdet_part,
                              double* w2, double* scratch, DevStatus* st, int grid) {
  // at least 116 KB of shared memory, so that no SM holds two CTAs (the FP64 pipe of an SM is
  // the resource: two CTAs on one SM would leave another idle)
  size_t smem = (size_t)(kLeafSmem + 2 * kDT * (kDT + 1)) * sizeof(double);
  if (smem < (size_t)116 * 1024) smem = (size_t)116 * 1024;
  static PerDeviceOnce attr_once;
  cudaError_t e = attr_once([&] {
    return cudaFuncSetAttribute(diag_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  if (grid < 2) grid = 2;  // CTA 0 runs the leaves; the updates need at least one more CTA
  e = cudaMemsetAsync(scratch + kDiagBar, 0, 2 * sizeof(double), s);
  if (e != cudaSuccess) return e;
  DiagArgs g{a, ld, k0, w_sub, logdet_part, w2, scratch, st};
  void* args[] = {&g};
  // cooperative launch: every CTA is resident at once, so the grid barriers cannot wait on an
  // unscheduled CTA
  return cudaLaunchCooperativeKernel((const void*)diag_block_kernel, grid, kDThreads, args, smem, s);
}

}  // namespace exa
