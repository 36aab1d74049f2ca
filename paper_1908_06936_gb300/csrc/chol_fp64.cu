// Step a2 (FP64): right-looking tiled Cholesky, Sigma = L L^T (Section I;
// the tile decomposition of Section II-A, Fig. 1(a)).
//
// For tile column k (k0 = k nb):
//   potrf_diag  : L_kk = chol(A_kk) in shared memory (one CTA), then W_k = L_kk^-1
//                 by independent row substitutions spread over several CTAs.
//   trsm_panel  : L_ik = A_ik L_kk^-T = A_ik W_k^T for all rows below (DMMA GEMM),
//                 written in place and to a row-major panel copy P.
//   syrk_update : A_ij -= L_ik L_jk^T over the trailing lower triangle (DMMA GEMM).
// The matrix is column-major with leading dimension ld, padded to a multiple
// of nb with an identity block, so every tile is full.
//
// FP64 tensor-core MMA on sm_103a is the warp-level mma.sync .f64 (DMMA): the
// chip's FP64 rate (~1.05 TFLOP/s measured, all DMMA shapes alike) is so low
// that a shared-memory-staged m8n8k4 kernel keeps the pipe busy.
#include <math.h>

#include "exa_internal.cuh"

namespace exa {

// D (8x8) += A (8x4, row) * B (4x8, col).  Fragments (g = lane/4, q = lane%4):
//   a = A[g][q], b = B[q][g], d = {D[g][2q], D[g][2q+1]}.
__device__ __forceinline__ void dmma_884(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__device__ __forceinline__ bool failed(const DevStatus* st) { return *(volatile const int32_t*)&st->info != 0; }

// ---------------------------------------------------------------------------
// potrf_diag: one CTA of 256 threads, the nb x nb diagonal tile in shared memory
// (row stride nb + 1).  Unblocked right-looking Cholesky, then in-place
// triangular inversion (column by column from the last), W written row-major.
// logdet_part[k] = sum_i log L_ii over the tile, summed in row order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) potrf_diag_kernel(double* __restrict__ a, int64_t ld, int64_t k0, int nb,
                                                         double* __restrict__ w_out, double* __restrict__ logdet_part,
                                                         DevStatus* st) {
  extern __shared__ double sm[];
  const int sd = nb + 1;
  double* S = sm;               // nb x sd
  double* tmp = sm + nb * sd;   // nb
  const int tid = threadIdx.x;
  const int k = (int)(k0 / nb);
  if (failed(st)) return;
  double* A = a + k0 + k0 * ld;
  for (int idx = tid; idx < nb * nb; idx += blockDim.x) {
    const int i = idx % nb, j = idx / nb;
    S[i * sd + j] = (i >= j) ? A[i + (int64_t)j * ld] : 0.0;
  }
  __syncthreads();
  int bad = -1;
  for (int j = 0; j < nb; ++j) {
    const double d = S[j * sd + j];
    if (!(d > 0.0) || !isfinite(d)) {  // uniform: every thread reads the same value
      bad = j;
      break;
    }
    const double lj = sqrt(d);
    const double inv = 1.0 / lj;
    for (int i = j + 1 + tid; i < nb; i += blockDim.x) S[i * sd + j] *= inv;
    __syncthreads();
    if (tid == 0) S[j * sd + j] = lj;
    // rank-1 update of the trailing lower triangle: thread -> column l, rows i >= l
    // split between the blockDim / nb threads sharing that column
    {
      const int per = blockDim.x / nb;          // threads per column (2 for nb = 128)
      const int l = tid % nb, i0 = tid / nb;
      if (l > j) {
        const double slj = S[l * sd + j];
        for (int i = l + i0; i < nb; i += per) S[i * sd + l] = fma(-S[i * sd + j], slj, S[i * sd + l]);
      }
    }
    __syncthreads();
  }
  if (bad >= 0) {
    if (tid == 0) {
      atomicMin(&st->pivot, (long long)(k0 + bad));
      atomicExch(&st->info, 1);
    }
    return;
  }
  // write L back (lower triangle of the tile)
  for (int idx = tid; idx < nb * nb; idx += blockDim.x) {
    const int i = idx % nb, j = idx / nb;
    if (i >= j) A[i + (int64_t)j * ld] = S[i * sd + j];
  }
  if (tid == 0) {
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += log(S[i * sd + i]);
    logdet_part[k] = s;
  }
  __syncthreads();
  // in-place inversion: column j of W from the already-inverted trailing block
  //   W_jj = 1 / L_jj,  W_ij = -W_jj * sum_{l=j+1..i} W_il L_lj  (i > j)
  for (int j = nb - 1; j >= 0; --j) {
    const double wjj = 1.0 / S[j * sd + j];  // read before anyone overwrites it below
    for (int i = j + 1 + tid; i < nb; i += blockDim.x) {
      double t = 0.0;
      for (int l = j + 1; l <= i; ++l) t = fma(S[i * sd + l], S[l * sd + j], t);
      tmp[i] = t;
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < nb; i += blockDim.x) S[i * sd + j] = -tmp[i] * wjj;
    if (tid == 0) S[j * sd + j] = wjj;
    __syncthreads();
  }
  double* W = w_out + (int64_t)k * nb * nb;
  for (int idx = tid; idx < nb * nb; idx += blockDim.x) {
    const int r = idx / nb, c = idx % nb;
    W[idx] = (c <= r) ? S[r * sd + c] : 0.0;
  }
}

// Blocked variant for nb = 64 / 128 (the factor and log-determinant part of
// potrf_diag_kernel; the inverse follows in trtri_rows_kernel).  On this part FP64
// instructions issue at ~1.6 per clock per SM, so one SM needs ~0.2 ms for the
// nb^3/3 multiply-adds of a 128 tile: the aim is to keep its FP64 pipe busy with few
// block-wide barriers.  16-wide panels are factored by warp 0 (warp-level syncs
// only), then a rank-16 update of the trailing triangle by all warps (one barrier per
// panel).
constexpr int kPotrfPW = 16;

// The tile's log sum goes to *logdet_out.  Returns true (on every thread) when the tile was
// factored; L then also sits in the first NB x (NB + 1) doubles of shared memory.
template <int NB>
__device__ __forceinline__ bool potrf_blocked_body(double* __restrict__ a, int64_t ld, int64_t k0,
                                                   double* __restrict__ logdet_out, DevStatus* st) {
  constexpr int PW = kPotrfPW, sd = NB + 1;
  extern __shared__ double sm[];
  double* S = sm;                // NB x sd, element (i, j) at S[i * sd + j]
  double* lg = sm + NB * sd;     // NB logs
  __shared__ int s_bad, s_skip;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) s_skip = failed(st) ? 1 : 0;  // one read, so that every thread takes the same path
  __syncthreads();
  if (s_skip) return false;
  double* A = a + k0 + k0 * ld;
  if (tid == 0) s_bad = -1;
  // load the lower triangle (column-major source, consecutive threads on consecutive rows)
  constexpr int PER = NB * NB / 256, CH = PER < 16 ? PER : 16;
#pragma unroll
  for (int c0 = 0; c0 < PER; c0 += CH) {
    double v[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int idx = tid + (c0 + u) * 256, i = idx % NB, j = idx / NB;
      v[u] = (i >= j) ? A[i + (int64_t)j * ld] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int idx = tid + (c0 + u) * 256;
      S[(idx % NB) * sd + idx / NB] = v[u];
    }
  }
  __syncthreads();
  // ---- factorisation ----
  for (int p = 0; p < NB; p += PW) {
    if (warp == 0) {
      for (int j = p; j < p + PW; ++j) {
        const double d = S[j * sd + j];
        if (!(d > 0.0) || !isfinite(d)) {  // warp-uniform
          if (lane == 0) s_bad = j;
          break;
        }
        const double lj = sqrt(d), inv = 1.0 / lj;
        for (int i = j + 1 + lane; i < NB; i += 32) S[i * sd + j] *= inv;
        __syncwarp();
        if (lane == 0) S[j * sd + j] = lj;
        for (int c = j + 1; c < p + PW; ++c) {
          const double scj = S[c * sd + j];
          for (int i = c + lane; i < NB; i += 32) S[i * sd + c] = fma(-S[i * sd + j], scj, S[i * sd + c]);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (s_bad >= 0) break;
    // trailing triangle (i >= l >= p + PW): S_il -= sum_{t in panel} S_it S_lt
    const int q0 = p + PW, m = NB - q0;
    for (int e = tid; e < m * m; e += 256) {
      const int i = q0 + e % m, l = q0 + e / m;
      if (i < l) continue;
      const double* ri = S + i * sd + p;
      const double* rl = S + l * sd + p;
      double s0 = 0.0, s1 = 0.0;
#pragma unroll
      for (int t = 0; t < PW; t += 2) {
        s0 = fma(ri[t], rl[t], s0);
        s1 = fma(ri[t + 1], rl[t + 1], s1);
      }
      S[i * sd + l] -= s0 + s1;
    }
    __syncthreads();
  }
  if (s_bad >= 0) {
    if (tid == 0) {
      atomicMin(&st->pivot, (long long)(k0 + s_bad));
      atomicExch(&st->info, 1);
    }
    return false;
  }
  // write L back (lower triangle) and the log-determinant part (fixed-order sum)
  for (int idx = tid; idx < NB * NB; idx += 256) {
    const int i = idx % NB, j = idx / NB;
    if (i >= j) A[i + (int64_t)j * ld] = S[i * sd + j];
  }
  if (tid < NB) lg[tid] = log(S[tid * sd + tid]);
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int i = 0; i < NB; ++i) s += lg[i];
    *logdet_out = s;
  }
  return true;
}

template <int NB>
__global__ void __launch_bounds__(256) potrf_diag_blocked_kernel(double* __restrict__ a, int64_t ld, int64_t k0,
                                                                 double* __restrict__ logdet_part, DevStatus* st) {
  potrf_blocked_body<NB>(a, ld, k0, logdet_part + k0 / NB, st);
}

// W_k = L_kk^-1 (row-major, zeros above the diagonal) for the NB x NB diagonal tile that
// potrf_diag_blocked_kernel has just factored in place.  Row i of W solves x L = e_i
// (the left-inverse equations W L = I that LAPACK's trtri satisfies) by substitution
// from the right: x_i = 1 / L_ii, then for l = i-1 .. 0,
// x_l = -(sum_{m > l} x_m L_ml) / L_ll.  Rows are independent, so warp w of CTA c takes
// row c + gridDim.x w (short and long rows mix within every CTA).  The lane holding
// column l broadcasts x_l, then every column j < l accumulates x_l L_lj (columns at
// or above l read the zeros stored above the diagonal, or L_ll once x_l is final).
// The sums are compensated (each product split exactly with an FMA, each addition
// with Knuth's TwoSum, the errors carried in a second word: the Dot2 scheme of Ogita,
// Rump and Oishi, SIAM J. Sci. Comput. 26, 2005), so W is as accurate as if the sums
// were formed in twice the precision: its rounding errors, which the condition number
// of an ill-conditioned tile would magnify, stay out of the panel solve A W^T.
// CTA `cta` of `nctas` takes rows cta + nctas w of W (the tile's inverse, row-major at W).
template <int NB>
__device__ __forceinline__ void trtri_rows_body(const double* __restrict__ a, int64_t ld, int64_t k0,
                                                double* __restrict__ W, const DevStatus* st, int cta, int nctas) {
  constexpr int sd = NB + 1, Q = NB / 32;
  extern __shared__ double sm[];
  double* S = sm;  // S[l * sd + j] = L(l, j) for l >= j, 0 above
  if (failed(st)) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const double* A = a + k0 + k0 * ld;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int l = idx % NB, j = idx / NB;
    S[l * sd + j] = (l >= j) ? A[l + (int64_t)j * ld] : 0.0;
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  for (int i = cta + nctas * warp; i < NB; i += nctas * nw) {
    // hi[q] + lo[q] = sum_{m > l} x_m L_mj for column j = lane + 32 q
    double hi[Q], lo[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) hi[q] = lo[q] = 0.0;
    for (int j = i + 1 + lane; j < NB; j += 32) W[(int64_t)i * NB + j] = 0.0;
    for (int l = i; l >= 0; --l) {
      const int ql = l >> 5;
      double h = hi[0], e = lo[0];
#pragma unroll
      for (int q = 1; q < Q; ++q)
        if (q == ql) h = hi[q], e = lo[q];
      const double sum = __shfl_sync(0xffffffffu, h + e, l & 31);
      const double xl = (l == i) ? 1.0 / S[l * sd + l] : -sum / S[l * sd + l];
      if (lane == (l & 31)) W[(int64_t)i * NB + l] = xl;
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (q <= ql) {
          const double lv = S[l * sd + lane + 32 * q];
          const double p = xl * lv, pe = fma(xl, lv, -p);  // p + pe = xl lv exactly
          const double t = hi[q] + p, bv = t - hi[q];      // TwoSum(hi, p)
          const double te = (hi[q] - (t - bv)) + (p - bv);
          hi[q] = t;
          lo[q] += te + pe;
        }
    }
  }
}

template <int NB>
__global__ void __launch_bounds__(256) trtri_rows_kernel(const double* __restrict__ a, int64_t ld, int64_t k0,
                                                         double* __restrict__ w_out, const DevStatus* st) {
  trtri_rows_body<NB>(a, ld, k0, w_out + (k0 / NB) * (int64_t)NB * NB, st, blockIdx.x, gridDim.x);
}

// Batched diagonal tiles (NB = 128), one CTA per task: the blocked Cholesky above, then the
// inverse W = L^-1 (row-major, zeros above the diagonal) from L in shared memory: the eight
// 16 x 16 diagonal blocks inverted by the eight warps (column by column), then by doubling,
// [[W_A, 0], [L_BA, W_B]]^-1 = [[W_A, 0], [-W_B (L_BA W_A), W_B]] for widths 16, 32, 64, with
// the products in shared memory.  Plain FP64 sums: W preconditions the FP64 refinement and
// feeds TF32 panel solves, so the compensated row inverse of the single-field FP64 path (16
// CTAs per tile) is not needed here, and one CTA per tile keeps a batch of hundreds of tiles
// at one wave or two.
constexpr int kInvSmem = 128 * 129 + 128 + 64 * 64;  // doubles: L, logs, one product

__global__ void __launch_bounds__(256) potrf_inv128_tasks_kernel(const DiagTileTask* __restrict__ tasks) {
  constexpr int NB = 128, sd = NB + 1, PW = 16;
  const DiagTileTask t = tasks[blockIdx.x];
  if (!potrf_blocked_body<NB>(t.a, t.ld, t.k0, t.logdet, t.st)) return;  // uniform over the CTA
  extern __shared__ double sm[];
  const double* S = sm;            // L(i, j) at S[i * sd + j]
  double* T = sm + NB * sd + NB;   // products, at most 64 x 64
  double* W = t.w;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int idx = tid; idx < NB * NB; idx += 256) {
    const int r = idx / NB, c = idx % NB;
    if (c > r) W[idx] = 0.0;  // the strict upper triangle
  }
  __syncthreads();
  {
    const int p0 = warp * PW;  // warp w inverts diagonal block w
    for (int c = PW - 1; c >= 0; --c) {
      const double vcc = 1.0 / S[(p0 + c) * sd + p0 + c];
      if (lane > c && lane < PW) {
        double acc = 0.0;
        for (int l = c + 1; l <= lane; ++l) acc = fma(W[(p0 + lane) * NB + p0 + l], S[(p0 + l) * sd + p0 + c], acc);
        W[(p0 + lane) * NB + p0 + c] = -acc * vcc;
      }
      if (lane == c) W[(p0 + c) * NB + p0 + c] = vcc;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int h = PW; h < NB; h *= 2) {
    const int pairs = NB / (2 * h);
    for (int idx = tid; idx < pairs * h * h; idx += 256) {
      const int p = idx / (h * h), r = (idx / h) % h, c = idx % h, o = p * 2 * h;
      double acc = 0.0;
      for (int k = c; k < h; ++k) acc = fma(S[(o + h + r) * sd + o + k], W[(o + k) * NB + o + c], acc);
      T[idx] = acc;
    }
    __syncthreads();
    for (int idx = tid; idx < pairs * h * h; idx += 256) {
      const int p = idx / (h * h), r = (idx / h) % h, c = idx % h, o = p * 2 * h;
      double acc = 0.0;
      for (int k = 0; k <= r; ++k) acc = fma(W[(o + h + r) * NB + o + h + k], T[p * h * h + k * h + c], acc);
      W[(o + h + r) * NB + o + c] = -acc;
    }
    __syncthreads();
  }
}

cudaError_t launch_potrf128_tasks(cudaStream_t s, const DiagTileTask* d_tasks, int ntasks) {
  if (ntasks <= 0) return cudaSuccess;
  const size_t smem = (size_t)kInvSmem * sizeof(double);
  static PerDeviceOnce attr_once;
  cudaError_t e = attr_once([&] {
    return cudaFuncSetAttribute(potrf_inv128_tasks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  potrf_inv128_tasks_kernel<<<(unsigned)ntasks, 256, smem, s>>>(d_tasks);
  return cudaGetLastError();
}

template <int NB>
static cudaError_t launch_potrf_blocked(cudaStream_t s, double* a, int64_t ld, int64_t k0, double* w_out,
                                        double* logdet_part, DevStatus* st) {
  const size_t smem = (size_t)(NB * (NB + 1) + NB) * sizeof(double);  // potrf: S and the logs; trtri: S
  static PerDeviceOnce attr_once;
  cudaError_t e = attr_once([&] {
    cudaError_t r = cudaFuncSetAttribute(potrf_diag_blocked_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(trtri_rows_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return r;
  });
  if (e != cudaSuccess) return e;
  potrf_diag_blocked_kernel<NB><<<1, 256, smem, s>>>(a, ld, k0, logdet_part, st);
  // one row per warp: NB / 8 CTAs of 8 warps
  trtri_rows_kernel<NB><<<NB / 8, 256, smem, s>>>(a, ld, k0, w_out, st);
  return cudaGetLastError();
}

cudaError_t launch_potrf_diag(cudaStream_t s, double* a, int64_t ld, int64_t k0, int nb, double* w_out,
                              double* logdet_part, DevStatus* st) {
  if (nb == 128) return launch_potrf_blocked<128>(s, a, ld, k0, w_out, logdet_part, st);
  if (nb == 64) return launch_potrf_blocked<64>(s, a, ld, k0, w_out, logdet_part, st);
  const size_t smem = (size_t)(nb * (nb + 1) + nb) * sizeof(double);
  static PerDeviceOnce attr_once;
  cudaError_t e = attr_once([] {
    return cudaFuncSetAttribute(potrf_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)((128 * 129 + 128) * sizeof(double)));
  });
  if (e != cudaSuccess) return e;
  potrf_diag_kernel<<<1, 256, smem, s>>>(a, ld, k0, nb, w_out, logdet_part, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// trsm_panel: rows [k0+nb, k0+nb+m), one CTA per 32-row strip, nb/32 warps,
// warp w owns output columns [32w, 32w+32).  out = A_strip * W^T with K = nb,
// staged through shared memory in K-chunks of 32 (row stride 36 doubles).
// ---------------------------------------------------------------------------
constexpr int kKC = 32;      // K chunk
constexpr int kSS = kKC + 4; // padded row stride (doubles) of staged chunks

__global__ void __launch_bounds__(128) trsm_panel_kernel(double* __restrict__ a, int64_t ld, int64_t k0, int nb,
                                                         const double* __restrict__ w, double* __restrict__ p,
                                                         const DevStatus* st) {
  __shared__ double As[32 * kSS];
  __shared__ double Ws[128 * kSS];
  if (failed(st)) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int64_t r0 = k0 + nb + (int64_t)blockIdx.x * 32;
  const double* Wk = w + (int64_t)(k0 / nb) * nb * nb;
  double acc[4][4][2];
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) acc[mi][ni][0] = acc[mi][ni][1] = 0.0;
  for (int t0 = 0; t0 < nb; t0 += kKC) {
    for (int idx = tid; idx < 32 * kKC; idx += blockDim.x) {
      const int r = idx & 31, t = idx >> 5;
      As[r * kSS + t] = a[(r0 + r) + (k0 + t0 + t) * ld];
    }
    for (int idx = tid; idx < nb * kKC; idx += blockDim.x) {
      const int c = idx / kKC, t = idx % kKC;
      Ws[c * kSS + t] = Wk[(int64_t)c * nb + t0 + t];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kKC; kk += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) af[mi] = As[(mi * 8 + g) * kSS + kk + q];
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) bf[ni] = Ws[(warp * 32 + ni * 8 + g) * kSS + kk + q];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) dmma_884(acc[mi][ni][0], acc[mi][ni][1], af[mi], bf[ni]);
    }
    __syncthreads();
  }
  // every read of this strip is done: write L_ik in place and to P (row-major, nb wide)
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int64_t row = r0 + mi * 8 + g;
        const int col = warp * 32 + ni * 8 + 2 * q + e;
        const double v = acc[mi][ni][e];
        a[row + (k0 + col) * ld] = v;
        p[(row - (k0 + nb)) * nb + col] = v;
      }
}

cudaError_t launch_trsm_panel(cudaStream_t s, double* a, int64_t ld, int64_t k0, int nb, int64_t m,
                              const double* w, double* p, const DevStatus* st) {
  if (m <= 0) return cudaSuccess;
  trsm_panel_kernel<<<(unsigned)(m / 32), nb, 0, s>>>(a, ld, k0, nb, w, p, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// syrk_update: trailing matrix rows/cols [r0, r0+m), m a multiple of 64.  One
// CTA per 64 x 64 lower tile (ti >= tj), 4 warps in a 2 x 2 arrangement of
// 32 x 32 warp tiles:  C -= P_i P_j^T with K = nb.  Diagonal tiles store only
// their lower triangle.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tri_decode_u(long long b, int& ti, int& tj) {
  long long t = (long long)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while (t * (t + 1) / 2 > b) --t;
  while ((t + 1) * (t + 2) / 2 <= b) ++t;
  ti = (int)t;
  tj = (int)(b - t * (t + 1) / 2);
}

__global__ void __launch_bounds__(128) syrk_update_kernel(double* __restrict__ a, int64_t ld, int64_t r0, int nb,
                                                          const double* __restrict__ p, const DevStatus* st) {
  __shared__ double Pi[64 * kSS];
  __shared__ double Pj[64 * kSS];
  if (failed(st)) return;
  int ti, tj;
  tri_decode_u(blockIdx.x, ti, tj);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int wm = warp >> 1, wn = warp & 1;
  const double* pi = p + (int64_t)ti * 64 * nb;
  const double* pj = p + (int64_t)tj * 64 * nb;
  double acc[4][4][2];
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) acc[mi][ni][0] = acc[mi][ni][1] = 0.0;
  for (int t0 = 0; t0 < nb; t0 += kKC) {
    for (int idx = tid; idx < 64 * kKC; idx += blockDim.x) {
      const int r = idx / kKC, t = idx % kKC;
      Pi[r * kSS + t] = pi[(int64_t)r * nb + t0 + t];
      Pj[r * kSS + t] = pj[(int64_t)r * nb + t0 + t];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kKC; kk += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) af[mi] = Pi[(wm * 32 + mi * 8 + g) * kSS + kk + q];
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) bf[ni] = Pj[(wn * 32 + ni * 8 + g) * kSS + kk + q];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) dmma_884(acc[mi][ni][0], acc[mi][ni][1], af[mi], bf[ni]);
    }
    __syncthreads();
  }
  const bool diag = (ti == tj);
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int li = wm * 32 + mi * 8 + g;
        const int lj = wn * 32 + ni * 8 + 2 * q + e;
        if (diag && lj > li) continue;
        const int64_t row = r0 + (int64_t)ti * 64 + li;
        const int64_t col = r0 + (int64_t)tj * 64 + lj;
        double* c = a + row + col * ld;
        *c -= acc[mi][ni][e];
      }
}

cudaError_t launch_syrk_update(cudaStream_t s, double* a, int64_t ld, int64_t r0, int64_t m, int nb,
                               const double* p, const DevStatus* st) {
  if (m <= 0) return cudaSuccess;
  const long long t = m / 64;
  syrk_update_kernel<<<(unsigned)(t * (t + 1) / 2), 128, 0, s>>>(a, ld, r0, nb, p, st);
  return cudaGetLastError();
}

}  // namespace exa

namespace exa {

// ---------------------------------------------------------------------------
// Small strided FP64 product on DMMA:  C = alpha A B^T + beta C, element
// accessors A(i,k) = a[i*ar + k*ac], B(j,k) = b[j*br + k*bc], C(i,j) = c[i*cr + j*cc].
// M, N multiples of 32, K a multiple of 32.  One CTA (4 warps, 2 x 2 warp tiles
// of 16 x 16) per 32 x 32 output tile.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) dgemm_nt_small_kernel(int K, double alpha, const double* __restrict__ a,
                                                             int64_t ar, int64_t ac, const double* __restrict__ b,
                                                             int64_t br, int64_t bc, double beta, double* c,
                                                             int64_t cr, int64_t cc, const DevStatus* st) {
  __shared__ double As[32 * kSS];
  __shared__ double Bs[32 * kSS];
  if (failed(st)) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3;
  const int wm = warp >> 1, wn = warp & 1;
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  double acc[2][2][2];
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 2; ++ni) acc[mi][ni][0] = acc[mi][ni][1] = 0.0;
  for (int t0 = 0; t0 < K; t0 += kKC) {
    for (int idx = tid; idx < 32 * kKC; idx += blockDim.x) {
      const int r = idx & 31, t = idx >> 5;
      As[r * kSS + t] = a[(i0 + r) * ar + (int64_t)(t0 + t) * ac];
      Bs[r * kSS + t] = b[(j0 + r) * br + (int64_t)(t0 + t) * bc];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kKC; kk += 4) {
      double af[2], bf[2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) af[mi] = As[(wm * 16 + mi * 8 + g) * kSS + kk + q];
#pragma unroll
      for (int ni = 0; ni < 2; ++ni) bf[ni] = Bs[(wn * 16 + ni * 8 + g) * kSS + kk + q];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) dmma_884(acc[mi][ni][0], acc[mi][ni][1], af[mi], bf[ni]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 2; ++ni)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int64_t i = i0 + wm * 16 + mi * 8 + g;
        const int64_t j = j0 + wn * 16 + ni * 8 + 2 * q + e;
        double* p = c + i * cr + j * cc;
        *p = alpha * acc[mi][ni][e] + (beta != 0.0 ? beta * *p : 0.0);
      }
}

cudaError_t launch_dgemm_nt_small(cudaStream_t s, int M, int N, int K, double alpha, const double* a, int64_t ar,
                                  int64_t ac, const double* b, int64_t br, int64_t bc, double beta, double* c,
                                  int64_t cr, int64_t cc, const DevStatus* st) {
  dim3 grid(N / 32, M / 32);
  dgemm_nt_small_kernel<<<grid, 128, 0, s>>>(K, alpha, a, ar, ac, b, br, bc, beta, c, cr, cc, st);
  return cudaGetLastError();
}

}  // namespace exa
