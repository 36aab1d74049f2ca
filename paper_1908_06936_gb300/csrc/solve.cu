// Steps a3-a4: log-determinant and the triangular solve for the quadratic
// form (Section I: |Sigma| and Sigma^-1 Z from the Cholesky factor),
//   log|Sigma| = 2 sum_i log L_ii,   y = L^-1 z,   z^T Sigma^-1 z = y^T y.
// Both are HBM-bound: the solve streams the lower triangle once.  All
// reductions run in a fixed order, so FP64 results are bitwise reproducible.
#include "exa_internal.cuh"

namespace exa {

__device__ __forceinline__ bool failed_s(const DevStatus* st) { return *(volatile const int32_t*)&st->info != 0; }

// Forward block step k (right-looking):
//   y_k = W_k z_k                        (W_k = L_kk^-1, row-major)
//   z_r -= sum_t L[r][k0+t] y_k[t]       for every row r >= k0 + nb
// Every block recomputes y_k from the (not yet overwritten) z_k; block 0 stores it.
__global__ void __launch_bounds__(256) trsv_fwd_kernel(const double* __restrict__ a, int64_t ld, int64_t npad, int nb,
                                                       int k, const double* __restrict__ w_all, double* __restrict__ z,
                                                       double* __restrict__ y, const DevStatus* st) {
  __shared__ double zk[256];
  __shared__ double yk[256];
  if (failed_s(st)) return;
  const int tid = threadIdx.x;
  const int64_t k0 = (int64_t)k * nb;
  if (tid < nb) zk[tid] = z[k0 + tid];
  __syncthreads();
  const double* W = w_all + (int64_t)k * nb * nb;
  if (tid < nb) {
    double s = 0.0;
    for (int t = 0; t <= tid; ++t) s = fma(W[(int64_t)tid * nb + t], zk[t], s);
    yk[tid] = s;
    if (blockIdx.x == 0) y[k0 + tid] = s;
  }
  __syncthreads();
  const int64_t r = k0 + nb + (int64_t)blockIdx.x * blockDim.x + tid;
  if (r < npad) {
    double s = z[r];
    const double* col = a + r + k0 * ld;
    for (int t = 0; t < nb; ++t) s = fma(-col[(int64_t)t * ld], yk[t], s);
    z[r] = s;
  }
}

cudaError_t launch_trsv_fwd_step(cudaStream_t s, const double* a, int64_t ld, int64_t npad, int nb, int k,
                                 const double* w_all, double* y, double* tmp, const DevStatus* st) {
  // tmp holds the working right-hand side z (updated in place), y receives L^-1 z
  const int64_t m = npad - (int64_t)(k + 1) * nb;
  const unsigned blocks = (unsigned)(m > 0 ? (m + 255) / 256 : 1);
  trsv_fwd_kernel<<<blocks, 256, 0, s>>>(a, ld, npad, nb, k, w_all, tmp, y, st);
  return cudaGetLastError();
}

// Backward block step k (left-looking), a = L^-T y:
//   s_t = sum_{r >= k0+nb} L[r][k0+t] a_r   (t < nb; partial sums per block)
//   a_k = W_k^T (y_k - s)
// Two kernels: column-panel reduction into fixed per-block partials, then one
// block that finishes the sum in order and applies W_k^T.
constexpr int kBwdRows = 1024;  // rows per partial

__global__ void __launch_bounds__(256) trsv_bwd_partial_kernel(const double* __restrict__ a, int64_t ld, int64_t npad,
                                                               int nb, int k, const double* __restrict__ y,
                                                               double* __restrict__ part, const DevStatus* st) {
  // block b: rows [k0+nb + b*kBwdRows, ...); warp w: panel columns w, w+8, ...; lanes stride the
  // rows so every load of a column is one coalesced 256-byte access
  if (failed_s(st)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k0 = (int64_t)k * nb;
  const int64_t rs = k0 + nb + (int64_t)blockIdx.x * kBwdRows;
  int64_t re = rs + kBwdRows;
  if (re > npad) re = npad;
  for (int t = warp; t < nb; t += 8) {
    const double* col = a + (k0 + t) * ld;
    double s = 0.0;
    for (int64_t r = rs + lane; r < re; r += 32) s = fma(col[r], y[r], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) part[(int64_t)blockIdx.x * nb + t] = s;
  }
}

__global__ void __launch_bounds__(256) trsv_bwd_finish_kernel(int64_t npad, int nb, int k, int nparts,
                                                              const double* __restrict__ w_all,
                                                              const double* __restrict__ part, double* __restrict__ y,
                                                              const DevStatus* st) {
  __shared__ double v[256];
  if (failed_s(st)) return;
  const int t = threadIdx.x;
  const int64_t k0 = (int64_t)k * nb;
  if (t < nb) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += part[(int64_t)b * nb + t];
    v[t] = y[k0 + t] - s;
  }
  __syncthreads();
  const double* W = w_all + (int64_t)k * nb * nb;
  if (t < nb) {
    // (W^T v)_t = sum_{c >= t} W[c][t] v_c
    double s = 0.0;
    for (int c = t; c < nb; ++c) s = fma(W[(int64_t)c * nb + t], v[c], s);
    y[k0 + t] = s;
  }
}

cudaError_t launch_trsv_bwd_step(cudaStream_t s, const double* a, int64_t ld, int64_t npad, int nb, int k,
                                 const double* w_all, double* y, double* tmp, const DevStatus* st) {
  const int64_t m = npad - (int64_t)(k + 1) * nb;
  int nparts = 0;
  if (m > 0) {
    nparts = (int)((m + kBwdRows - 1) / kBwdRows);
    trsv_bwd_partial_kernel<<<nparts, 256, 0, s>>>(a, ld, npad, nb, k, y, tmp, st);
  }
  trsv_bwd_finish_kernel<<<1, 256, 0, s>>>(npad, nb, k, nparts, w_all, tmp, y, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Deterministic two-stage reductions.
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kRedMaxBlocks = 512;

__device__ __forceinline__ double block_reduce(double v, double* sh) {
  const int tid = threadIdx.x;
  sh[tid] = v;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (tid < w) sh[tid] += sh[tid + w];
    __syncthreads();
  }
  return sh[0];
}

template <bool SQ>
__global__ void __launch_bounds__(kRedThreads) reduce_stage1(const double* __restrict__ v, int64_t n, int64_t chunk,
                                                             double* __restrict__ partial) {
  __shared__ double sh[kRedThreads];
  const int64_t start = (int64_t)blockIdx.x * chunk;
  int64_t end = start + chunk;
  if (end > n) end = n;
  double s = 0.0;
  for (int64_t i = start + threadIdx.x; i < end; i += kRedThreads) {
    const double x = v[i];
    s += SQ ? x * x : x;
  }
  const double r = block_reduce(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

__global__ void __launch_bounds__(kRedThreads) reduce_stage2(const double* __restrict__ partial, int nb,
                                                             double* __restrict__ out) {
  __shared__ double sh[kRedThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += kRedThreads) s += partial[i];
  const double r = block_reduce(s, sh);
  if (threadIdx.x == 0) *out = r;
}

template <bool SQ>
static cudaError_t launch_reduce(cudaStream_t s, const double* v, int64_t n, double* partial, double* out) {
  int64_t chunk = 4096;
  int64_t blocks = (n + chunk - 1) / chunk;
  if (blocks > kRedMaxBlocks) {
    chunk = (n + kRedMaxBlocks - 1) / kRedMaxBlocks;
    blocks = (n + chunk - 1) / chunk;
  }
  if (blocks < 1) blocks = 1;
  reduce_stage1<SQ><<<(unsigned)blocks, kRedThreads, 0, s>>>(v, n, chunk, partial);
  reduce_stage2<<<1, kRedThreads, 0, s>>>(partial, (int)blocks, out);
  return cudaGetLastError();
}

cudaError_t launch_sumsq(cudaStream_t s, const double* v, int64_t n, double* partial, double* out) {
  return launch_reduce<true>(s, v, n, partial, out);
}
cudaError_t launch_sum(cudaStream_t s, const double* v, int64_t n, double* partial, double* out) {
  return launch_reduce<false>(s, v, n, partial, out);
}

}  // namespace exa

namespace exa {

// y = S x for symmetric S stored as its lower triangle (column-major, ld), in
// two deterministic passes that each stream the triangle once:
//   pass 1 (thread per row i):  y_i  = sum_{j <= i} S_ij x_j
//   pass 2 (warp per column i): y_i += sum_{j > i}  S_ji x_j
// One pass over the lower triangle in 128 x 128 tiles: tile (I, J), I >= J, is read
// once and gives both of its contributions,
//   rowpart[I][J][r] = sum_c S_IJ(r, c) x_J(c)          (to y_I)
//   colpart[J][I][c] = sum_r S_IJ(r, c) x_I(r)          (to y_J, I > J)
// A diagonal tile uses only its lower half: rows take c <= r, columns r > c.
// Each warp takes 16 columns, four at a time (16 loads in flight per lane); the
// row partials of the 8 warps are summed in a fixed order.
constexpr int kSymvNB = 128;

__global__ void __launch_bounds__(256) symv_tile_kernel(const double* __restrict__ S, int64_t ld, int T,
                                                        const double* __restrict__ x, double* __restrict__ rowpart,
                                                        double* __restrict__ colpart) {
  __shared__ double xi[kSymvNB], xj[kSymvNB];
  __shared__ double racc[8][kSymvNB];
  // tiles column block by column block (J outer, I = J..T-1 inner): CTAs running at the
  // same time stream neighbouring rows of the same 128 columns
  const long long b = blockIdx.x, TT = T;
  // first tile of column block J: S(J) = J T - J (J - 1) / 2
  long long J = (long long)(((2.0 * TT + 1.0) - sqrt((2.0 * TT + 1.0) * (2.0 * TT + 1.0) - 8.0 * (double)b)) * 0.5);
  if (J < 0) J = 0;
  while (J > 0 && J * TT - J * (J - 1) / 2 > b) --J;
  while ((J + 1) * TT - (J + 1) * J / 2 <= b) ++J;
  const long long I = J + (b - (J * TT - J * (J - 1) / 2));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid < kSymvNB) xj[tid] = x[J * kSymvNB + tid];
  else xi[tid - kSymvNB] = x[I * kSymvNB + tid - kSymvNB];
  __syncthreads();
  const bool diag = (I == J);
  const double* base = S + I * kSymvNB + J * kSymvNB * ld;
  double ra[4] = {0.0, 0.0, 0.0, 0.0};
  for (int c0 = warp * 16; c0 < warp * 16 + 16; c0 += 4) {
    double v[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double* col = base + (int64_t)(c0 + u) * ld;
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) v[u][rr] = __ldcs(col + lane + 32 * rr);
    }
    double cs[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + u;
      cs[u] = 0.0;
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const int r = lane + 32 * rr;
        const double e = v[u][rr];
        const double er = (!diag || c <= r) ? e : 0.0;  // the upper half of a diagonal tile is not data
        const double ec = (!diag || r > c) ? e : 0.0;
        ra[rr] = fma(er, xj[c], ra[rr]);
        cs[u] = fma(ec, xi[r], cs[u]);
      }
    }
    // the four column sums over the warp's 32 lanes, reduced together: halves of the set are
    // exchanged at the first two levels (lanes 0-15 keep columns 0-1, 16-31 columns 2-3; then
    // lanes with bit 3 clear keep the first), so 6 FP64 additions per lane instead of 20
    const bool up16 = (lane & 16) != 0, up8 = (lane & 8) != 0;
    const double k0 = up16 ? cs[2] : cs[0], k1 = up16 ? cs[3] : cs[1];
    const double s0 = up16 ? cs[0] : cs[2], s1 = up16 ? cs[1] : cs[3];
    const double h0 = k0 + __shfl_xor_sync(0xffffffffu, s0, 16);
    const double h1 = k1 + __shfl_xor_sync(0xffffffffu, s1, 16);
    double q = (up8 ? h1 : h0) + __shfl_xor_sync(0xffffffffu, up8 ? h0 : h1, 8);
    q += __shfl_xor_sync(0xffffffffu, q, 4);
    q += __shfl_xor_sync(0xffffffffu, q, 2);
    q += __shfl_xor_sync(0xffffffffu, q, 1);
    if ((lane & 7) == 0) colpart[(J * T + I) * kSymvNB + c0 + (up16 ? 2 : 0) + (up8 ? 1 : 0)] = q;
  }
#pragma unroll
  for (int rr = 0; rr < 4; ++rr) racc[warp][lane + 32 * rr] = ra[rr];
  __syncthreads();
  if (tid < kSymvNB) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += racc[w][tid];
    rowpart[(I * T + J) * kSymvNB + tid] = t;
  }
}

// y_I = sum_{J <= I} rowpart[I][J] + sum_{I' >= I} colpart[I][I'], in that order.
__global__ void __launch_bounds__(kSymvNB) symv_tile_reduce_kernel(int T, const double* __restrict__ rowpart,
                                                                    const double* __restrict__ colpart,
                                                                    double* __restrict__ y) {
  const int64_t I = blockIdx.x;
  const int r = threadIdx.x;
  double t = 0.0;
  for (int64_t J = 0; J <= I; ++J) t += rowpart[(I * T + J) * kSymvNB + r];
  for (int64_t I2 = I; I2 < T; ++I2) t += colpart[(I * T + I2) * kSymvNB + r];
  y[I * kSymvNB + r] = t;
}

int64_t symv_tiled_partials(int64_t npad) {
  const int64_t T = npad / kSymvNB;
  return 2 * T * T * kSymvNB;
}

cudaError_t launch_symv_lower_tiled(cudaStream_t s, const double* a, int64_t ld, int64_t npad, const double* x,
                                    double* y, double* partials) {
  if (npad % kSymvNB) return cudaErrorInvalidValue;
  const int64_t T = npad / kSymvNB;
  if (T < 1) return cudaSuccess;
  double* rowpart = partials;
  double* colpart = partials + T * T * kSymvNB;
  symv_tile_kernel<<<(unsigned)(T * (T + 1) / 2), 256, 0, s>>>(a, ld, (int)T, x, rowpart, colpart);
  symv_tile_reduce_kernel<<<(unsigned)T, kSymvNB, 0, s>>>((int)T, rowpart, colpart, y);
  return cudaGetLastError();
}

// r = z - y ; elementwise helpers
__global__ void residual_kernel(const double* __restrict__ z, const double* __restrict__ y, double* __restrict__ r,
                                int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = z[i] - y[i];
}

__global__ void axpy_kernel(double a, const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = fma(a, x[i], y[i]);
}

__global__ void __launch_bounds__(kRedThreads) dot_stage1(const double* __restrict__ a, const double* __restrict__ b,
                                                          int64_t n, int64_t chunk, double* __restrict__ partial) {
  __shared__ double sh[kRedThreads];
  const int64_t start = (int64_t)blockIdx.x * chunk;
  int64_t end = start + chunk;
  if (end > n) end = n;
  double s = 0.0;
  for (int64_t i = start + threadIdx.x; i < end; i += kRedThreads) s = fma(a[i], b[i], s);
  const double r = block_reduce(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = r;
}


cudaError_t launch_residual(cudaStream_t s, const double* z, const double* y, double* r, int64_t n) {
  residual_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(z, y, r, n);
  return cudaGetLastError();
}

cudaError_t launch_axpy(cudaStream_t s, double a, const double* x, double* y, int64_t n) {
  axpy_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_dot(cudaStream_t s, const double* a, const double* b, int64_t n, double* partial, double* out) {
  int64_t chunk = 4096;
  int64_t blocks = (n + chunk - 1) / chunk;
  if (blocks > kRedMaxBlocks) {
    chunk = (n + kRedMaxBlocks - 1) / kRedMaxBlocks;
    blocks = (n + chunk - 1) / chunk;
  }
  if (blocks < 1) blocks = 1;
  dot_stage1<<<(unsigned)blocks, kRedThreads, 0, s>>>(a, b, n, chunk, partial);
  reduce_stage2<<<1, kRedThreads, 0, s>>>(partial, (int)blocks, out);
  return cudaGetLastError();
}

}  // namespace exa

namespace exa {

// ---------------------------------------------------------------------------
// Persistent block triangular solves (one cooperative launch per solve).
// 128-row blocks with stored row-major inverses W_k of the diagonal tiles.
// CTA c owns the blocks b with b % gridDim.x == c and is the only writer of
// their right-hand side / partial sums, so every sum runs in a fixed order.
// Block k's result is published with a flag (release); readers wait on it with
// a bounded spin (acquire) and read it from L2.
// ---------------------------------------------------------------------------
constexpr int kPNB = 128;

struct PTrsvArgs {
  const double* a;
  int64_t ld, npad;
  int T;
  const double* w;
  double* z;     // forward: working right-hand side (in: rhs);  backward: partial sums s (zeroed)
  double* y;     // forward: output L^-1 rhs;  backward: in y, out L^-T y (in place)
  int* flags;    // T flags, zeroed
  int* abort;
  DevStatus* st;
  long long spin;
};

__device__ __forceinline__ bool ptrsv_wait(const int* f, volatile int* abort, long long spin) {
  if (*(volatile const int*)f) return true;
  const long long t0 = clock64();
  while (!*(volatile const int*)f) {
    if (*abort) return false;
    if (clock64() - t0 > spin) return false;
    __nanosleep(100);
  }
  return true;
}

// Warm L2 with what the next step of a CTA reads first, while it waits for the step's
// input block: the 128 x 128 tile at rows r0.. and columns c0.. (column-major, ld), and
// with w != nullptr the 128 x 128 inverse w (row-major, contiguous).  prefetch.global.L2
// takes one 128-byte line per instruction and never faults on these in-bounds lines.
__device__ __forceinline__ void ptrsv_prefetch(const PTrsvArgs& g, int64_t r0, int64_t c0, const double* w) {
  const double* tile = g.a + r0 + c0 * g.ld;
  for (int li = threadIdx.x; li < kPNB * 8; li += blockDim.x) {  // 8 lines per 128-row column
    const double* p = tile + (li & 7) * 16 + (int64_t)(li >> 3) * g.ld;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
  }
  if (w)
    for (int li = threadIdx.x; li < kPNB * kPNB / 16; li += blockDim.x) {
      const double* p = w + li * 16;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
    }
}

__device__ __forceinline__ void ptrsv_fail(const PTrsvArgs& g, int site) {
  if (atomicExch(g.abort, 1) == 0 && atomicExch(&g.st->timeout, 1) == 0) g.st->timeout_where = site;
}

// Forward: y = L^-1 z.  The owner of block k+1 finalises y_{k+1} = W_{k+1} z_{k+1}
// right after applying column k to z_{k+1} (its first block of that column), so the
// chain of diagonal blocks advances one block GEMV per step; the rest of column k
// is applied afterwards.  y_k is double-buffered in shared memory by parity.
__device__ __forceinline__ void ptrsv_fwd_finalize(const PTrsvArgs& g, int k, double (*red)[kPNB], double* ybuf) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t k0 = (int64_t)k * kPNB;
  const double* W = g.w + (int64_t)k * kPNB * kPNB;
  double* zk = red[0];  // the final right-hand side of block k
  if (tid < kPNB) zk[tid] = __ldcg(&g.z[k0 + tid]);
  __syncthreads();
  // warp per row of W (row-major, lower), four rows at a time, lanes along the row
  for (int r0 = warp * 16; r0 < warp * 16 + 16; r0 += 4) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int t = lane + 32 * q;
        const double w = W[(r0 + u) * kPNB + t];
        s[u] = fma(t <= r0 + u ? w : 0.0, zk[t], s[u]);
      }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s[u] += __shfl_xor_sync(0xffffffffu, s[u], o);
    }
    if (lane < 4) {
      const double v = lane == 0 ? s[0] : lane == 1 ? s[1] : lane == 2 ? s[2] : s[3];
      ybuf[r0 + lane] = v;
      g.y[k0 + r0 + lane] = v;
    }
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    atomicExch(&g.flags[k], 1);
  }
}

__global__ void __launch_bounds__(256) trsv_fwd_persistent_kernel(PTrsvArgs g) {
  __shared__ double ybuf[2][kPNB];
  __shared__ double red[2][kPNB];
  __shared__ int ok;
  const int tid = threadIdx.x, row = tid & (kPNB - 1), half = tid >> 7;
  const int G = gridDim.x, me = blockIdx.x;
  if (*(volatile const int*)&g.st->info) return;
  if (me == 0) ptrsv_fwd_finalize(g, 0, red, ybuf[0]);
  for (int k = 0; k < g.T; ++k) {
    const int64_t k0 = (int64_t)k * kPNB;
    // this CTA's first block below k (blocks b with b % G == me); none now means none later
    int b = k + 1 + ((me - (k + 1)) % G + G) % G;
    if (b >= g.T) break;
    ptrsv_prefetch(g, (int64_t)b * kPNB, k0, b == k + 1 ? g.w + (int64_t)(k + 1) * kPNB * kPNB : nullptr);
    if (k % G != me) {
      if (tid == 0) {
        ok = ptrsv_wait(&g.flags[k], g.abort, g.spin);
        if (!ok) ptrsv_fail(g, 41);
        __threadfence();
      }
      __syncthreads();
      if (!ok) return;
      if (tid < kPNB) ybuf[k & 1][tid] = __ldcg(&g.y[k0 + tid]);
    }
    __syncthreads();
    const double* yk = ybuf[k & 1];
    // z_b -= L_bk y_k for this CTA's blocks b > k, nearest first
    for (; b < g.T; b += G) {
      const int64_t r = (int64_t)b * kPNB + row;
      const double* col = g.a + r + (k0 + half * 64) * g.ld;
      const double* yh = yk + half * 64;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll 4
      for (int t = 0; t < 64; t += 4) {
        s0 = fma(__ldcg(col + (int64_t)t * g.ld), yh[t], s0);
        s1 = fma(__ldcg(col + (int64_t)(t + 1) * g.ld), yh[t + 1], s1);
        s2 = fma(__ldcg(col + (int64_t)(t + 2) * g.ld), yh[t + 2], s2);
        s3 = fma(__ldcg(col + (int64_t)(t + 3) * g.ld), yh[t + 3], s3);
      }
      red[half][row] = (s0 + s1) + (s2 + s3);
      __syncthreads();
      if (tid < kPNB) g.z[r] = g.z[r] - (red[0][tid] + red[1][tid]);
      __syncthreads();
      if (b == k + 1) ptrsv_fwd_finalize(g, k + 1, red, ybuf[(k + 1) & 1]);
    }
  }
}

// Backward: x = L^-T y with U = L^T held in the strictly upper off-diagonal tiles of
// the same matrix (launch_transpose_lower_to_upper), in place on y.  Mirror of the
// forward solve: blocks from the bottom, x_k = W_k^T z_k; once x_k is known,
// z_i -= U_ik x_k for i < k, where U_ik is column block k above the diagonal
// (contiguous in memory).  The owner of block k-1 finalises it right after
// applying x_k to it.
__device__ __forceinline__ void ptrsv_bwd_finalize(const PTrsvArgs& g, int k, double* zk, double* xbuf) {
  const int tid = threadIdx.x, t = tid & (kPNB - 1), h = tid >> 7;
  const int64_t k0 = (int64_t)k * kPNB;
  __shared__ double part[2][kPNB];
  if (tid < kPNB) zk[tid] = __ldcg(&g.y[k0 + tid]);
  __syncthreads();
  // x_k[t] = sum_{u >= t} W_k[u][t] z_k[u]; W row-major: consecutive t are contiguous
  const double* W = g.w + (int64_t)k * kPNB * kPNB;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll 4
  for (int u = h * 64; u < h * 64 + 64; u += 4) {
    s0 = fma(u >= t ? W[u * kPNB + t] : 0.0, zk[u], s0);
    s1 = fma(u + 1 >= t ? W[(u + 1) * kPNB + t] : 0.0, zk[u + 1], s1);
    s2 = fma(u + 2 >= t ? W[(u + 2) * kPNB + t] : 0.0, zk[u + 2], s2);
    s3 = fma(u + 3 >= t ? W[(u + 3) * kPNB + t] : 0.0, zk[u + 3], s3);
  }
  part[h][t] = (s0 + s1) + (s2 + s3);
  __syncthreads();
  if (tid < kPNB) {
    const double v = part[0][tid] + part[1][tid];
    xbuf[tid] = v;
    g.y[k0 + tid] = v;
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    atomicExch(&g.flags[k], 1);
  }
}

__global__ void __launch_bounds__(256) trsv_bwd_persistent_kernel(PTrsvArgs g) {
  __shared__ double xbuf[2][kPNB];
  __shared__ double zk[kPNB];
  __shared__ double red[2][kPNB];
  __shared__ int ok;
  const int tid = threadIdx.x, row = tid & (kPNB - 1), half = tid >> 7;
  const int G = gridDim.x, me = blockIdx.x;
  if (*(volatile const int*)&g.st->info) return;
  if ((g.T - 1) % G == me) ptrsv_bwd_finalize(g, g.T - 1, zk, xbuf[(g.T - 1) & 1]);
  for (int k = g.T - 1; k >= 1; --k) {
    const int64_t k0 = (int64_t)k * kPNB;
    // this CTA's first block above k, nearest first; none now means none later
    int i = k - 1 - ((k - 1 - me) % G + G) % G;
    if (i < 0) break;
    ptrsv_prefetch(g, (int64_t)i * kPNB, k0, i == k - 1 ? g.w + (int64_t)(k - 1) * kPNB * kPNB : nullptr);
    if (k % G != me) {
      if (tid == 0) {
        ok = ptrsv_wait(&g.flags[k], g.abort, g.spin);
        if (!ok) ptrsv_fail(g, 42);
        __threadfence();
      }
      __syncthreads();
      if (!ok) return;
      if (tid < kPNB) xbuf[k & 1][tid] = __ldcg(&g.y[k0 + tid]);
    }
    __syncthreads();
    const double* xk = xbuf[k & 1];
    for (; i >= 0; i -= G) {
      // z_i -= U_ik x_k, U_ik(row, t) = a[i*128 + row + (k0 + t) ld]
      const int64_t r = (int64_t)i * kPNB + row;
      const double* col = g.a + r + (k0 + half * 64) * g.ld;
      const double* xh = xk + half * 64;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll 4
      for (int t = 0; t < 64; t += 4) {
        s0 = fma(__ldcg(col + (int64_t)t * g.ld), xh[t], s0);
        s1 = fma(__ldcg(col + (int64_t)(t + 1) * g.ld), xh[t + 1], s1);
        s2 = fma(__ldcg(col + (int64_t)(t + 2) * g.ld), xh[t + 2], s2);
        s3 = fma(__ldcg(col + (int64_t)(t + 3) * g.ld), xh[t + 3], s3);
      }
      red[half][row] = (s0 + s1) + (s2 + s3);
      __syncthreads();
      if (tid < kPNB) g.y[r] = g.y[r] - (red[0][tid] + red[1][tid]);
      __syncthreads();
      if (i == k - 1) ptrsv_bwd_finalize(g, k - 1, zk, xbuf[(k - 1) & 1]);
    }
  }
}

// Strictly upper off-diagonal tiles <- L^T: tile (I, J), I > J, of the lower
// triangle is written transposed to tile (J, I), in 32 x 32 pieces through
// shared memory (both the reads and the writes run along columns).
__global__ void __launch_bounds__(256) transpose_lower_to_upper_kernel(double* __restrict__ a, int64_t ld, int T) {
  __shared__ double t[32][33];
  // strictly lower tiles, column block by column block: column J holds T - 1 - J tiles
  const long long b = blockIdx.x, TT = T;
  long long J = (long long)(((2.0 * TT - 1.0) - sqrt((2.0 * TT - 1.0) * (2.0 * TT - 1.0) - 8.0 * (double)b)) * 0.5);
  if (J < 0) J = 0;
  while (J > 0 && J * (TT - 1) - J * (J - 1) / 2 > b) --J;
  while ((J + 1) * (TT - 1) - (J + 1) * J / 2 <= b) ++J;
  const long long I = J + 1 + (b - (J * (TT - 1) - J * (J - 1) / 2));
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int sj = 0; sj < 4; ++sj)
    for (int si = 0; si < 4; ++si) {
      const int64_t r0 = I * kPNB + si * 32, c0 = J * kPNB + sj * 32;
#pragma unroll
      for (int q = 0; q < 4; ++q) t[ty + 8 * q][tx] = a[(r0 + tx) + (c0 + ty + 8 * q) * ld];  // t[c][r] = L(r, c)
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 4; ++q) a[(c0 + tx) + (r0 + ty + 8 * q) * ld] = t[tx][ty + 8 * q];  // U(c, r) = L(r, c)
      __syncthreads();
    }
}

cudaError_t launch_transpose_lower_to_upper(cudaStream_t s, double* a, int64_t ld, int64_t npad) {
  const int64_t T = npad / kPNB;
  if (npad % kPNB) return cudaErrorInvalidValue;
  if (T < 2) return cudaSuccess;
  transpose_lower_to_upper_kernel<<<(unsigned)(T * (T - 1) / 2), 256, 0, s>>>(a, ld, (int)T);
  return cudaGetLastError();
}

static int ptrsv_grid() {
  static std::atomic<int> cache[64];
  return per_device_int(cache, [] {
    int dev = 0, sms = 0, per = 0, per2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, trsv_fwd_persistent_kernel, 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, trsv_bwd_persistent_kernel, 256, 0);
    if (per2 < per) per = per2;
    // two CTAs per SM: the off-chain updates need the loads in flight (one per SM, which would
    // give the chain's CTA its SM's FP64 pipe to itself, measured 40 -> 54 ms per solve pair)
    if (per > 2) per = 2;
    return (per < 1 ? 1 : per) * (sms > 0 ? sms : 1);
  });
}

// Forward (x = L^-1 rhs, rhs overwritten) then backward (x = L^-T x) solve.  The
// strictly upper off-diagonal 128-tiles of a must hold L^T.  flags: 2 T + 1 ints
// (zeroed here).
cudaError_t launch_llt_solve_persistent(cudaStream_t s, const double* a, int64_t ld, int64_t npad, const double* w,
                                        double* rhs_work, double* x, int* flags, DevStatus* st) {
  const int T = (int)(npad / kPNB);
  cudaError_t e = cudaMemsetAsync(flags, 0, (size_t)(2 * T + 1) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int grid = ptrsv_grid() < T ? ptrsv_grid() : T;
  PTrsvArgs g{a, ld, npad, T, w, rhs_work, x, flags, flags + 2 * T, st, 2000000000LL};
  void* args[] = {&g};
  e = cudaLaunchCooperativeKernel((const void*)trsv_fwd_persistent_kernel, grid, 256, args, 0, s);
  if (e != cudaSuccess) return e;
  PTrsvArgs g2{a, ld, npad, T, w, nullptr, x, flags + T, flags + 2 * T, st, 2000000000LL};
  void* args2[] = {&g2};
  return cudaLaunchCooperativeKernel((const void*)trsv_bwd_persistent_kernel, grid, 256, args2, 0, s);
}

}  // namespace exa
