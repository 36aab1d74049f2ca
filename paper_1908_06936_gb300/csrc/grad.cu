// Gradient of the log-likelihood (Eq. 2) with respect to theta = (sigma^2, beta, nu):
//
//   dl/dtheta_k = 1/2 a^T D_k a - 1/2 tr(Sigma^-1 D_k),   a = Sigma^-1 z,  D_k = dSigma/dtheta_k,
//
// with D_k regenerated entry by entry from Eq. 3 (never stored):
//   D_sigma2 = Sigma / sigma^2
//   D_beta   = sigma^2 c x^nu K_{nu-1}(x) x / beta            (d[x^nu K_nu]/dx = -x^nu K_{nu-1}, DLMF 10.29.4)
//   D_nu     = Sigma (-ln 2 - psi(nu) + ln x) + sigma^2 c x^nu dK_nu/dnu,   c = 2^(1-nu) / Gamma(nu)
// and all three vanishing on the diagonal except D_sigma2 = 1.
//
// Steps after the FP64 factorisation Sigma = L L^T (DMMA):
//   a  = L^-T (L^-1 z)                     backward block solve
//   X  = L^-1 in place                      block columns right to left:
//                                           T = X22 L_panel, X_panel = -T W_j, X_jj = W_j
//   S  = X^T X = Sigma^-1 (lower tiles)     into a second n x n buffer
//   g  = 1/2 sum_ij w_ij (a_i a_j - S_ij) D_k,ij   (w = 1 on the diagonal, 2 below), fused
//                                           with the regeneration of D_k, fixed-order reduction.
#include <math.h>
#include <string.h>

#include <vector>

#include "bessel.cuh"
#include "ctx.cuh"
#include "util.cuh"

namespace exa {

__device__ __forceinline__ void dmma884(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

constexpr int gKC = 32, gSS = 36;

// T(i, c) = sum_{l = l0}^{min(i, tile end)} X(i, l) L(l, j0 + c) for rows i in [l0, npad),
// X lower triangular (entries above its diagonal read as 0).  Output T row-major, nb wide.
// CTA: 64 x 64 output tile, 4 warps of 32 x 32.
__global__ void __launch_bounds__(128) trmm_lower_panel_kernel(const double* __restrict__ a, int64_t ld, int64_t l0,
                                                               int64_t j0, int nb, double* __restrict__ tout,
                                                               const DevStatus* st) {
  __shared__ double As[64 * gSS];
  __shared__ double Bs[64 * gSS];
  if (*(volatile const int32_t*)&st->info) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3, wm = warp >> 1, wn = warp & 1;
  const int64_t i0 = l0 + (int64_t)blockIdx.y * 64;  // output rows [i0, i0 + 64)
  const int c0 = blockIdx.x * 64;                      // output cols [c0, c0 + 64)
  double acc[4][4][2];
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) acc[mi][ni][0] = acc[mi][ni][1] = 0.0;
  for (int64_t k0 = l0; k0 < i0 + 64; k0 += gKC) {
    for (int idx = tid; idx < 64 * gKC; idx += blockDim.x) {
      const int r = idx & 63, t = idx >> 6;
      const int64_t i = i0 + r, l = k0 + t;
      As[r * gSS + t] = (l <= i) ? a[i + l * ld] : 0.0;
      const int tb = idx & 31, cb = idx >> 5;  // k fastest: the panel column is contiguous in l
      Bs[cb * gSS + tb] = a[(k0 + tb) + (j0 + c0 + cb) * ld];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < gKC; kk += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) af[mi] = As[(wm * 32 + mi * 8 + g) * gSS + kk + q];
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) bf[ni] = Bs[(wn * 32 + ni * 8 + g) * gSS + kk + q];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) dmma884(acc[mi][ni][0], acc[mi][ni][1], af[mi], bf[ni]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int64_t row = i0 + wm * 32 + mi * 8 + g - l0;
        const int col = c0 + wn * 32 + ni * 8 + 2 * q + e;
        tout[row * nb + col] = acc[mi][ni][e];
      }
}

// Diagonal tile of X: lower triangle <- W_j (row-major), strict upper left untouched.
__global__ void put_diag_inverse_kernel(double* __restrict__ a, int64_t ld, int64_t j0, int nb,
                                        const double* __restrict__ w) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nb * nb; idx += gridDim.x * blockDim.x) {
    const int r = idx % nb, c = idx / nb;
    if (r >= c) a[(j0 + r) + (j0 + c) * ld] = w[r * nb + c];
  }
}

// S = X^T X on 64 x 64 lower tiles (I >= J):  S(i, j) = sum_{k >= I*64} X(k, i) X(k, j),
// X lower triangular (X(k, i) = 0 for k < i).  Output column-major into s (ld_s).
__device__ __forceinline__ void tri_dec(long long b, int& ti, int& tj) {
  long long t = (long long)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while (t * (t + 1) / 2 > b) --t;
  while ((t + 1) * (t + 2) / 2 <= b) ++t;
  ti = (int)t;
  tj = (int)(b - t * (t + 1) / 2);
}

__global__ void __launch_bounds__(128) lauum_tiles_kernel(const double* __restrict__ a, int64_t ld, int64_t npad,
                                                          double* __restrict__ s, int64_t lds, const DevStatus* st) {
  __shared__ double As[64 * gSS];
  __shared__ double Bs[64 * gSS];
  if (*(volatile const int32_t*)&st->info) return;
  int ti, tj;
  tri_dec(blockIdx.x, ti, tj);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3, wm = warp >> 1, wn = warp & 1;
  const int64_t i0 = (int64_t)ti * 64, j0 = (int64_t)tj * 64;
  double acc[4][4][2];
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) acc[mi][ni][0] = acc[mi][ni][1] = 0.0;
  for (int64_t k0 = i0; k0 < npad; k0 += gKC) {
    for (int idx = tid; idx < 64 * gKC; idx += blockDim.x) {
      const int t = idx & 31, r = idx >> 5;  // k fastest: X(k, col) contiguous in k
      const int64_t k = k0 + t;
      const int64_t ci = i0 + r, cj = j0 + r;
      As[r * gSS + t] = (k >= ci) ? a[k + ci * ld] : 0.0;
      Bs[r * gSS + t] = (k >= cj) ? a[k + cj * ld] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < gKC; kk += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) af[mi] = As[(wm * 32 + mi * 8 + g) * gSS + kk + q];
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) bf[ni] = Bs[(wn * 32 + ni * 8 + g) * gSS + kk + q];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) dmma884(acc[mi][ni][0], acc[mi][ni][1], af[mi], bf[ni]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int64_t i = i0 + wm * 32 + mi * 8 + g;
        const int64_t j = j0 + wn * 32 + ni * 8 + 2 * q + e;
        if (ti == tj && j > i) continue;
        s[i + j * lds] = acc[mi][ni][e];
      }
}

// sinh and cosh of x (series below 0.1 so that small steps keep full relative accuracy)
__device__ __forceinline__ void sincosh_pair(double x, double& sh, double& ch) {
  if (fabs(x) < 0.1) {
    const double x2 = x * x;
    sh = x * (1.0 + x2 * (1.0 / 6.0 + x2 * (1.0 / 120.0 + x2 * (1.0 / 5040.0 + x2 / 362880.0))));
    ch = 1.0 + x2 * (0.5 + x2 * (1.0 / 24.0 + x2 * (1.0 / 720.0 + x2 * (1.0 / 40320.0 + x2 / 3628800.0))));
  } else {
    const double e = exp(x), ie = 1.0 / e;
    sh = 0.5 * (e - ie);
    ch = 0.5 * (e + ie);
  }
}

// e^x dK_nu(x)/dnu = int_0^inf t sinh(nu t) exp(-x (cosh t - 1)) dt  (DLMF 10.32.9
// differentiated in nu) by the trapezoid rule with step h = min(0.2, 0.6/sqrt(x)):
// the integrand is entire, so the error falls like exp(-2 pi d / h) with d the
// usable half-width of the strip around the real axis (~pi/2 for small x,
// ~1/sqrt(x) for large x).  sinh(t/2) and sinh/cosh(nu t) advance by exact
// hyperbolic rotations, so cosh t - 1 = 2 sinh^2(t/2) carries no cancellation.
__device__ __forceinline__ double dknu_dnu_scaled(double nu, double x) {
  if (nu == 0.0) return 0.0;
  const double h = fmin(0.2, 0.6 / sqrt(x));
  double sh_h, ch_h, snu_h, cnu_h;
  sincosh_pair(0.5 * h, sh_h, ch_h);
  sincosh_pair(nu * h, snu_h, cnu_h);
  double s = 0.0, c = 1.0;    // sinh(t/2), cosh(t/2) at t = 0
  double sn = 0.0, cn = 1.0;  // sinh(nu t), cosh(nu t)
  double sum = 0.0;
  const double anu = fabs(nu);
  for (int k = 1; k < 4000; ++k) {
    const double s2 = s * ch_h + c * sh_h;
    const double c2 = c * ch_h + s * sh_h;
    s = s2;
    c = c2;
    const double sn2 = sn * cnu_h + cn * snu_h;
    const double cn2 = cn * cnu_h + sn * snu_h;
    sn = sn2;
    cn = cn2;
    const double t = k * h;
    const double f = t * sn * exp(-2.0 * x * s * s);
    sum += f;
    // past the peak (log-derivative 1/t + nu coth(nu t) - x sinh t < 0) and negligible
    const double sinh_t = 2.0 * s * c;
    if (x * sinh_t > 1.0 / t + anu * cn / fabs(sn) && fabs(f) <= 1e-18 * fabs(sum)) break;
  }
  return h * sum;
}

struct GradParams {
  MaternParams m;
  double psi_nu;  // digamma(nu)
};

// D_sigma2, D_beta, D_nu at distance r (the formulas of the header; the diagonal r = 0
// gives (1, 0, 0)).
__device__ __forceinline__ void matern_derivs(const GradParams& G, double r, double& d0, double& d1, double& d2) {
  const MaternParams& P = G.m;
  if (r == 0.0) {
    d0 = 1.0;
    d1 = d2 = 0.0;
    return;
  }
  const double x = r / P.beta;
  if (x > 800.0) {
    d0 = d1 = d2 = 0.0;
    return;
  }
  const double lnx = log(x);
  double knu, knum1;
  const bool scaled = bessel_k_nu(P, x, lnx, knu, knum1);
  const double base = P.logc + P.nu * lnx;
  const double pre = P.sigma2 * exp(base - (scaled ? x : 0.0));  // sigma^2 c x^nu (e^-x if scaled)
  const double sig = pre * knu;
  d0 = sig / P.sigma2;
  d1 = pre * knum1 * x / P.beta;
  d2 = sig * (lnx - 0.69314718055994530942 - G.psi_nu) + P.sigma2 * exp(base - x) * dknu_dnu_scaled(P.nu, x);
}

// One 64 x 64 lower tile per block (as the generator), 256 threads; per-block partial
// sums of w (a_i a_j - S_ij) D_k for k = sigma^2, beta, nu in a fixed order.
__global__ void __launch_bounds__(256) grad_reduce_kernel(const double* __restrict__ locs, int64_t n,
                                                          const __grid_constant__ GradParams G,
                                                          const double* __restrict__ alpha,
                                                          const double* __restrict__ sinv, int64_t lds,
                                                          double ssign, double* __restrict__ partial) {
  __shared__ double red[3][256];
  int ti, tj;
  tri_dec(blockIdx.x, ti, tj);
  const int64_t i = (int64_t)ti * 64 + (threadIdx.x & 63);
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
  if (i < n) {
    const double xi = locs[2 * i], yi = locs[2 * i + 1], ai = alpha[i];
    for (int s = 0; s < 16; ++s) {
      const int64_t j = (int64_t)tj * 64 + (threadIdx.x >> 6) + 4 * s;
      if (j > i) continue;
      const double w = (i == j) ? 1.0 : 2.0;
      const double cij = w * (ai * alpha[j] - ssign * sinv[i + j * lds]);
      double d0, d1, d2;
      matern_derivs(G, sqrt(model_dist2(G.m, xi, yi, locs[2 * j], locs[2 * j + 1])), d0, d1, d2);
      acc0 = fma(cij, d0, acc0);
      acc1 = fma(cij, d1, acc1);
      acc2 = fma(cij, d2, acc2);
    }
  }
  const int tid = threadIdx.x;
  red[0][tid] = acc0;
  red[1][tid] = acc1;
  red[2][tid] = acc2;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) {
      red[0][tid] += red[0][tid + w];
      red[1][tid] += red[1][tid + w];
      red[2][tid] += red[2][tid + w];
    }
    __syncthreads();
  }
  if (tid < 3) partial[(int64_t)blockIdx.x * 3 + tid] = red[tid][0];
}

// One-buffer form of the two steps above, for when Sigma^-1 and the factor cannot both
// be held: the 64 x 64 lower tile (I, J) of S = X^T X (X = L^-1, in place of the
// factor) is accumulated on DMMA exactly as lauum_tiles_kernel does, parked in shared
// memory instead of a second n x n buffer, and reduced at once with the regenerated
// D_k into the tile's partial sums (same layout as grad_reduce_kernel's, over the
// npad / 64 tile grid).  Entries with i or j >= n are padding and skipped.
__global__ void __launch_bounds__(128) lauum_grad_fused_kernel(const double* __restrict__ a, int64_t ld,
                                                               int64_t npad, int64_t n,
                                                               const double* __restrict__ locs,
                                                               const __grid_constant__ GradParams G,
                                                               const double* __restrict__ alpha,
                                                               double* __restrict__ partial, const DevStatus* st) {
  __shared__ double As[64 * gSS];
  __shared__ double Bs[64 * gSS];
  __shared__ double red[3][128];
  if (*(volatile const int32_t*)&st->info) return;
  int ti, tj;
  tri_dec(blockIdx.x, ti, tj);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3, wm = warp >> 1, wn = warp & 1;
  const int64_t i0 = (int64_t)ti * 64, j0 = (int64_t)tj * 64;
  double acc[4][4][2];
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) acc[mi][ni][0] = acc[mi][ni][1] = 0.0;
  for (int64_t k0 = i0; k0 < npad; k0 += gKC) {
    for (int idx = tid; idx < 64 * gKC; idx += blockDim.x) {
      const int t = idx & 31, r = idx >> 5;
      const int64_t k = k0 + t;
      const int64_t ci = i0 + r, cj = j0 + r;
      As[r * gSS + t] = (k >= ci) ? a[k + ci * ld] : 0.0;
      Bs[r * gSS + t] = (k >= cj) ? a[k + cj * ld] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < gKC; kk += 4) {
      double af[4], bf[4];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) af[mi] = As[(wm * 32 + mi * 8 + g) * gSS + kk + q];
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) bf[ni] = Bs[(wn * 32 + ni * 8 + g) * gSS + kk + q];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) dmma884(acc[mi][ni][0], acc[mi][ni][1], af[mi], bf[ni]);
    }
    __syncthreads();
  }
  // park the S tile in shared memory (As and Bs together hold 64 x 72 doubles): S(r, c) at Ss[r * 65 + c]
  double* Ss = As;
  static_assert(64 * 65 <= 2 * 64 * gSS, "S tile must fit in the staging buffers");
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int e = 0; e < 2; ++e) Ss[(wm * 32 + mi * 8 + g) * 65 + wn * 32 + ni * 8 + 2 * q + e] = acc[mi][ni][e];
  __syncthreads();
  const int r = tid & 63;
  const int64_t i = i0 + r;
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
  if (i < n) {
    const double xi = locs[2 * i], yi = locs[2 * i + 1], ai = alpha[i];
    for (int s2 = 0; s2 < 32; ++s2) {
      const int cc = (tid >> 6) + 2 * s2;
      const int64_t j = j0 + cc;
      if (j > i || j >= n) continue;
      const double w = (i == j) ? 1.0 : 2.0;
      const double cij = w * (ai * alpha[j] - Ss[r * 65 + cc]);
      double d0, d1, d2;
      matern_derivs(G, sqrt(model_dist2(G.m, xi, yi, locs[2 * j], locs[2 * j + 1])), d0, d1, d2);
      acc0 = fma(cij, d0, acc0);
      acc1 = fma(cij, d1, acc1);
      acc2 = fma(cij, d2, acc2);
    }
  }
  red[0][tid] = acc0;
  red[1][tid] = acc1;
  red[2][tid] = acc2;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (tid < w) {
      red[0][tid] += red[0][tid + w];
      red[1][tid] += red[1][tid + w];
      red[2][tid] += red[2][tid + w];
    }
    __syncthreads();
  }
  if (tid < 3) partial[(int64_t)blockIdx.x * 3 + tid] = red[tid][0];
}

// out[k] = 1/2 sum_b partial[b][k]  (one block per component, fixed order)
__global__ void __launch_bounds__(256) grad_finish_kernel(const double* __restrict__ partial, int64_t nblocks,
                                                          double* __restrict__ out) {
  __shared__ double sh[256];
  const int k = blockIdx.x, tid = threadIdx.x;
  double s = 0.0;
  for (int64_t b = tid; b < nblocks; b += 256) s += partial[b * 3 + k];
  sh[tid] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) sh[tid] += sh[tid + w];
    __syncthreads();
  }
  if (tid == 0) out[k] = 0.5 * sh[0];
}

// digamma for the host-side constant psi(nu): shift to x >= 12 with psi(x) = psi(x+1) - 1/x,
// then psi(x) = ln x - 1/(2x) - sum_k B_2k / (2k x^2k)  (Bernoulli numbers B_2..B_10).
static double host_digamma(double x) {
  double shift = 0.0;
  for (; x < 12.0; x += 1.0) shift += 1.0 / x;
  const double r = 1.0 / (x * x);
  const double tail = r * (1.0 / 12 - r * (1.0 / 120 - r * (1.0 / 252 - r * (1.0 / 240 - r * (1.0 / 132)))));
  return log(x) - 0.5 / x - tail - shift;
}

// sinv holds ssign * Sigma^-1 (lower triangle, ld npad).
static cudaError_t launch_gradient(exa_ctx* c, const double* locs, int64_t n, int64_t npad, const double theta[3],
                                   const double* alpha, const double* sinv, double ssign, double* partial,
                                   double* out) {
  GradParams G;
  model_params(c, theta, &G.m);
  G.psi_nu = host_digamma(theta[2]);
  const long long t = (n + 63) / 64;
  const long long blocks = t * (t + 1) / 2;
  grad_reduce_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(locs, n, G, alpha, sinv, npad, ssign, partial);
  grad_finish_kernel<<<3, 256, 0, c->stream>>>(partial, blocks, out);
  return cudaGetLastError();
}

// X = L^-1 in place of the FP64 factor in c->mat (block columns right to left:
// T = X22 L_panel, X_panel = -T W_j, X_jj = W_j).  Stream-ordered; the factor is consumed.
static cudaError_t factor_inverse_fp64(exa_ctx* c, int64_t npad, int nb) {
  const int T = (int)(npad / nb);
  double* A = (double*)c->mat.p;
  double* W = (double*)c->w_all.p;
  double* Tbuf = (double*)c->panel.p;  // npad x nb
  cudaStream_t s = c->stream;
  cudaError_t e = cudaSuccess;
  for (int j = T - 1; j >= 0 && e == cudaSuccess; --j) {
    const int64_t j0 = (int64_t)j * nb, l0 = j0 + nb, m = npad - l0;
    if (m > 0) {
      ProfScope ps(c, PK_GRAD, (double)m * m * nb + 2.0 * m * nb * nb, 8.0 * ((double)m * m / 2 + 3.0 * m * nb), 2);
      dim3 grid(nb / 64, (unsigned)(m / 64));
      trmm_lower_panel_kernel<<<grid, 128, 0, s>>>(A, npad, l0, j0, nb, Tbuf, c->d_status);
      e = cudaGetLastError();
      if (e == cudaSuccess)
        e = launch_dgemm_nt_small(s, (int)m, nb, nb, -1.0, Tbuf, nb, 1, W + (int64_t)j * nb * nb, 1, nb, 0.0,
                                  A + l0 + j0 * npad, 1, npad, c->d_status);
    }
    if (e == cudaSuccess) {
      put_diag_inverse_kernel<<<32, 256, 0, s>>>(A, npad, j0, nb, W + (int64_t)j * nb * nb);
      e = cudaGetLastError();
    }
  }
  return e;
}

// Sigma^-1 from the FP64 factor in c->mat: X = L^-1 in place, then the lower tiles of
// S = X^T X into S (ld npad).  Stream-ordered; the factor is consumed.
static cudaError_t sigma_inverse_fp64(exa_ctx* c, int64_t npad, int nb, double* S) {
  cudaError_t e = factor_inverse_fp64(c, npad, nb);
  if (e == cudaSuccess) {
    const long long t64 = npad / 64;
    ProfScope ps(c, PK_GRAD, (double)npad * npad * npad / 3.0, 8.0 * (double)npad * npad);
    lauum_tiles_kernel<<<(unsigned)(t64 * (t64 + 1) / 2), 128, 0, c->stream>>>((const double*)c->mat.p, npad, npad,
                                                                               S, npad, c->d_status);
    e = cudaGetLastError();
  }
  return e;
}

// Lower triangle of the panel-wide diagonal block at (i0, i0) <- W (row-major), strict
// upper triangle of the block <- 0 (so that row-block splits of X read zeros there).
__global__ void __launch_bounds__(256) put_block_inverse_kernel(double* __restrict__ a, int64_t ld, int64_t i0,
                                                                const double* __restrict__ w) {
  const int c = blockIdx.x;
  for (int r = threadIdx.x; r < kMixPanel; r += blockDim.x)
    a[(i0 + r) + (i0 + c) * ld] = (r >= c) ? w[(int64_t)r * kMixPanel + c] : 0.0;
}

// -Sigma^-1 (lower triangle, into Sneg, ld npad) from the mixed-precision factor in c->mat,
// every product on the tensor cores with the exact digit-slice arithmetic (5 signed 7-bit
// digits per value, exact sums up to K = 512, FP64 between passes).  512-row blocks of
// X = L^-1 are formed top to bottom in place of the factor:
//   T_i = sum_{l < i} L_il X_l      one product per earlier block, -T_i accumulated in FP64
//   X_i,<i = W_i (-T_i),  X_ii = W_i  (W_i the inverse of the diagonal block, kept by the
//                                     factorisation)
//   S -= X_i^T X_i                   over the leading (i + 1) 512 square, lower triangle
// so that Sneg = -X^T X = -Sigma^-1 of the factor.  The digit planes of every row block of X
// are kept (about 5 n^2 bytes) and serve both its products.
static exa_status mixed_inverse_tc(exa_ctx* c, int64_t npad, double* Sneg) {
  constexpr int NB = kMixPanel;
  const int T = (int)(npad / NB);
  double* A = (double*)c->mat.p;
  const double* Wall = (const double*)c->mx_wall.p;
  cudaStream_t s = c->stream;
  std::vector<size_t> off(T + 1, 0);
  for (int i = 0; i < T; ++i) off[i + 1] = off[i] + split_bytes((int64_t)(i + 1) * NB, NB, false, true);
  exa_status st;
  if ((st = ensure(c, c->gr_xsplit, off[T] + 1024, "digit planes of L^-1")) != EXA_OK) return st;
  const size_t big = split_bytes(npad, NB, false, true), small = split_bytes(NB, NB, false, true);
  if ((st = ensure(c, c->gr_lsplit, 2 * big + small + 1024, "inverse operands")) != EXA_OK) return st;
  if ((st = ensure(c, c->gr_t, (size_t)NB * npad * sizeof(double), "inverse row-block product")) != EXA_OK)
    return st;
  auto align = [](void* p) { return (uint8_t*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023); };
  uint8_t* xb = align(c->gr_xsplit.p);
  uint8_t* lb = align(c->gr_lsplit.p);
  std::vector<SplitOperand> X(T);
  SplitOperand LS, TS, WS;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < T && e == cudaSuccess; ++i)
    e = split_layout(X[i], xb + off[i], (int64_t)(i + 1) * NB, NB, false, true);
  if (e == cudaSuccess) e = split_layout(LS, lb, npad, NB, false, true);
  if (e == cudaSuccess) e = split_layout(TS, lb + big, npad, NB, false, true);
  if (e == cudaSuccess) e = split_layout(WS, lb + 2 * big, NB, NB, false, true);
  if (e != cudaSuccess) return cuda_err(c, e, "tensor map encode");
  double* Tb = (double*)c->gr_t.p;
  e = cudaMemsetAsync(Sneg, 0, (size_t)npad * npad * sizeof(double), s);
  GemmArgs g;
  memset(&g, 0, sizeof(g));
  g.st = c->d_status;
  g.K = NB;
  g.panel = NB;
  for (int i = 0; i < T && e == cudaSuccess; ++i) {
    const int64_t i0 = (int64_t)i * NB;
    const double* Wi = Wall + (size_t)i * NB * NB;
    if (i > 0) {
      // -T_i into Tb (NB x i0, ld NB): block l of L's row block i against X_l
      e = cudaMemsetAsync(Tb, 0, (size_t)NB * i0 * sizeof(double), s);
      {
        ProfScope ps(c, PK_SPLIT, 0.0, 18.0 * (double)NB * i0, i);
        for (int l = 0; l < i && e == cudaSuccess; ++l)
          e = launch_split_rows(s, A + i0 + (int64_t)l * NB * npad, 1, npad, NB, NB, LS, l * NB);
      }
      for (int l = 0; l < i && e == cudaSuccess; ++l) {
        g.C = Tb;
        g.ldc = NB;
        g.c_row0 = g.c_col0 = 0;
        g.a_row0 = l * NB;
        g.b_row0 = 0;
        g.enum_mode = kEnumFull;
        g.nt = (l + 1) * NB / 32;
        g.ntiles = (long long)(NB / 128) * g.nt;
        g.store = 0;
        g.lower_mask = 0;
        ProfScope ps(c, PK_GEMM_OZ, 2.0 * NB * (double)(l + 1) * NB * NB, 16.0 * NB * (double)(l + 1) * NB);
        e = launch_gemm_oz(s, LS, X[l], g);
      }
      // X_i,<i = W_i (-T_i), over L's row block i
      {
        ProfScope ps(c, PK_SPLIT, 0.0, 18.0 * (double)NB * (i0 + NB), 2);
        if (e == cudaSuccess) e = launch_split_rows(s, Wi, NB, 1, NB, NB, WS, 0);
        if (e == cudaSuccess) e = launch_split_rows(s, Tb, NB, 1, (int)i0, NB, TS, 0);
      }
      if (e == cudaSuccess) {
        g.C = A + i0;
        g.ldc = npad;
        g.a_row0 = g.b_row0 = 0;
        g.nt = (int)(i0 / 32);
        g.ntiles = (long long)(NB / 128) * g.nt;
        g.store = 1;
        ProfScope ps(c, PK_GEMM_OZ, 2.0 * NB * (double)i0 * NB, 8.0 * NB * (double)i0);
        e = launch_gemm_oz(s, WS, TS, g);
      }
    }
    if (e != cudaSuccess) break;
    put_block_inverse_kernel<<<NB, 256, 0, s>>>(A, npad, i0, Wi);
    e = cudaGetLastError();
    // digit planes of X's row block i: operand row c = X(i0 .. i0 + NB - 1, c), c < i0 + NB
    if (e == cudaSuccess) {
      ProfScope ps(c, PK_SPLIT, 0.0, 18.0 * (double)NB * (i0 + NB));
      e = launch_split_rows(s, A + i0, npad, 1, (int)(i0 + NB), NB, X[i], 0);
    }
    // S -= X_i^T X_i over every panel pair of the leading lower triangle
    if (e == cudaSuccess) {
      g.C = Sneg;
      g.ldc = npad;
      g.c_row0 = g.c_col0 = 0;
      g.a_row0 = g.b_row0 = 0;
      g.enum_mode = kEnumBand;
      g.band = i;
      g.panel = NB;
      g.store = 0;
      g.lower_mask = 1;
      const long long pairs = (long long)(i + 1) * (i + 2) / 2;
      g.ntiles = pairs * (NB / 128) * (NB / 32);
      const double e2 = (double)(i0 + NB);
      ProfScope ps(c, PK_GEMM_OZ, e2 * e2 * NB, 8.0 * e2 * e2);
      e = launch_gemm_oz(s, X[i], X[i], g);
      g.band = 0;
    }
  }
  if (e != cudaSuccess) return cuda_err(c, e, "tensor-core inverse launch");
  return EXA_OK;
}

// Mixed-precision log-likelihood and gradient: l from the mixed evaluation (TF32x3 /
// exact-band factor, FP64 refinement), a = Sigma^-1 z refined in FP64 to rounding level,
// Sigma^-1 of the mixed factor on the tensor cores (mixed_inverse_tc), and the same
// fused regeneration and reduction of dSigma/dtheta as the FP64 gradient.
static exa_status loglik_grad_mixed(exa_ctx* c, const double* d_locs, const double* d_z, const double theta[3],
                                    int64_t n, double* loglik, double grad[3]) {
  exa_result res;
  memset(&res, 0, sizeof(res));
  c->keep_block_inverses = 1;
  c->ir_tight = 1;
  exa_status st = loglik_mixed(c, d_locs, d_z, theta, n, EXA_MIXED_TF32X3, &res);
  c->keep_block_inverses = 0;
  c->ir_tight = 0;
  if (st != EXA_OK) return st;
  *loglik = res.loglik;
  const int64_t npad = round_up(n, kMixPanel);
  const double* x = (const double*)c->mx_vec.p + npad;  // refined Sigma^-1 z (loglik_mixed's layout)
  double* Sneg = (double*)c->mx_sigma.p;                // the FP64 copy of Sigma is no longer needed
  double ssign = -1.0;
  if (c->grad_inverse_fp64) {
    // X = L^-1 and X^T X on FP64 DMMA (the 128-tile inverses of the mixed factorisation)
    if ((st = ensure(c, c->panel, (size_t)npad * 128 * sizeof(double), "panel")) != EXA_OK) return st;
    const cudaError_t ei = sigma_inverse_fp64(c, npad, 128, Sneg);
    if (ei != cudaSuccess) return cuda_err(c, ei, "inverse launch");
    ssign = 1.0;
  } else if ((st = mixed_inverse_tc(c, npad, Sneg)) != EXA_OK) {
    return st;
  }
  const long long t64n = (n + 63) / 64;
  const size_t nblocks = (size_t)(t64n * (t64n + 1) / 2);
  if ((st = ensure(c, c->gr_blocks, nblocks * 3 * sizeof(double), "gradient partials")) != EXA_OK) return st;
  cudaError_t e;
  {
    ProfScope ps(c, PK_GRAD, 0.0, 4.0 * (double)n * (double)(n + 1));
    e = launch_gradient(c, d_locs, n, npad, theta, x, Sneg, ssign, (double*)c->gr_blocks.p, c->d_scalars + 8);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_scalars + 8, c->d_scalars + 8, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "gradient launch");
  if ((st = read_status(c)) != EXA_OK) return st;
  grad[0] = c->h_scalars[8];
  grad[1] = c->h_scalars[9];
  grad[2] = c->h_scalars[10];
  return EXA_OK;
}

}  // namespace exa

using namespace exa;

extern "C" exa_status exa_ctx_set_gradient_inverse(exa_ctx* c, int fp64) {
  if (!c) return EXA_ERR_ARG;
  c->grad_inverse_fp64 = fp64 ? 1 : 0;
  return EXA_OK;
}

extern "C" exa_status exa_loglik_grad(exa_ctx* c, const double* d_locs, const double* d_z, const double theta[3],
                                      int64_t n, exa_prec prec, double* loglik, double grad[3]) {
  if (!c) return EXA_ERR_ARG;
  c->err[0] = 0;
  c->last_pivot = -1;
  if (!loglik || !grad) return set_err(c, EXA_ERR_ARG, "loglik / grad is NULL");
  *loglik = NAN;
  grad[0] = grad[1] = grad[2] = NAN;
  if (n < 1 || !d_locs || !d_z) return set_err(c, EXA_ERR_ARG, "bad n or NULL device pointer");
  if (prec != EXA_FP64 && prec != EXA_MIXED_TF32X3)
    return set_err(c, EXA_ERR_ARG, "the gradient is offered in EXA_FP64 and EXA_MIXED_TF32X3 (precision %d)",
                   (int)prec);
  exa_status st = check_theta(c, theta);
  if (st != EXA_OK) return st;
  if (prec == EXA_MIXED_TF32X3) {
    st = loglik_grad_mixed(c, d_locs, d_z, theta, n, loglik, grad);
    prof_fold(c);
    return st;
  }
  const int nb = c->tile_nb;
  const int64_t npad = round_up(n, nb);
  const int T = (int)(npad / nb);
  // Sigma^-1 in a second n x n buffer when it fits beside the factor; otherwise the
  // one-buffer form: X = L^-1 overwrites the factor and each tile of X^T X is formed and
  // reduced at once (lauum_grad_fused_kernel), so no second n x n buffer is needed.
  // A second buffer already held by the context (Sigma^-1 of an earlier gradient, or the
  // FP64 copy of Sigma kept by the mixed-precision path) is reused as it is.
  const size_t nn_bytes = (size_t)npad * npad * sizeof(double);
  bool one_buffer = false;
  double* S = nullptr;
  if (c->gr_part.bytes >= nn_bytes) {
    S = (double*)c->gr_part.p;
  } else if (c->mx_sigma.bytes >= nn_bytes) {
    S = (double*)c->mx_sigma.p;
  } else {
    // the factor's own buffer is requested first, so the test below sees what remains
    if ((st = ensure(c, c->mat, nn_bytes, "matrix")) != EXA_OK) return st;
    st = ensure(c, c->gr_part, nn_bytes, "inverse covariance");
    if (st == EXA_ERR_NOMEM) {
      one_buffer = true;
      c->err[0] = 0;
    } else if (st != EXA_OK) {
      return st;
    } else {
      S = (double*)c->gr_part.p;
    }
  }
  exa_result res;
  memset(&res, 0, sizeof(res));
  double* y = nullptr;
  if ((st = loglik_fp64(c, d_locs, d_z, theta, n, &res, &y)) != EXA_OK) return st;
  *loglik = res.loglik;
  double* A = (double*)c->mat.p;
  double* W = (double*)c->w_all.p;
  double* part = (double*)c->partial.p;
  cudaStream_t s = c->stream;
  cudaError_t e = cudaSuccess;
  // a = L^-T y (in place in y)
  for (int k = T - 1; k >= 0 && e == cudaSuccess; --k) {
    const double rows = (double)(npad - (int64_t)k * nb);
    ProfScope ps(c, PK_TRSV, 2.0 * rows * nb, 8.0 * rows * nb, 2);
    e = launch_trsv_bwd_step(s, A, npad, npad, nb, k, W, y, part + 2 * kRedPartials, c->d_status);
  }
  const long long t64n = one_buffer ? npad / 64 : (n + 63) / 64;
  const size_t nblocks = (size_t)(t64n * (t64n + 1) / 2);
  if ((st = ensure(c, c->gr_blocks, nblocks * 3 * sizeof(double), "gradient partials")) != EXA_OK) return st;
  if (!one_buffer) {
    if (e == cudaSuccess) e = sigma_inverse_fp64(c, npad, nb, S);
    // fused regeneration of dSigma/dtheta and reduction
    if (e == cudaSuccess) {
      ProfScope ps(c, PK_GRAD, 0.0, 4.0 * (double)n * (double)(n + 1));
      e = launch_gradient(c, d_locs, n, npad, theta, y, S, 1.0, (double*)c->gr_blocks.p, c->d_scalars + 8);
    }
  } else {
    if (e == cudaSuccess) e = factor_inverse_fp64(c, npad, nb);
    if (e == cudaSuccess) {
      GradParams G;
      model_params(c, theta, &G.m);
      G.psi_nu = host_digamma(theta[2]);
      ProfScope ps(c, PK_GRAD, (double)npad * npad * npad / 3.0, 4.0 * (double)npad * (double)(npad + 1), 2);
      lauum_grad_fused_kernel<<<(unsigned)nblocks, 128, 0, s>>>(A, npad, npad, n, d_locs, G, y,
                                                                  (double*)c->gr_blocks.p, c->d_status);
      grad_finish_kernel<<<3, 256, 0, s>>>((double*)c->gr_blocks.p, (int64_t)nblocks, c->d_scalars + 8);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_scalars + 8, c->d_scalars + 8, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_err(c, e, "gradient launch");
  if ((st = read_status(c)) != EXA_OK) return st;
  grad[0] = c->h_scalars[8];
  grad[1] = c->h_scalars[9];
  grad[2] = c->h_scalars[10];
  return EXA_OK;
}

// ---------------------------------------------------------------------------
// Fisher information (exact_fisher): I_kl = 1/2 tr(Sigma^-1 D_k Sigma^-1 D_l).
//   S = Sigma^-1 (lower tiles, as for the gradient), mirrored to a full matrix;
//   D_k written as a full symmetric matrix into the factor's buffer (zero in the
//   padding); M_k = S D_k on FP64 DMMA; tr(M_k M_l) = sum_ij M_k(i, j) M_l(j, i)
//   from 32 x 32 tile pairs (I, J) / (J, I), per-tile partials summed in a fixed order.
// ---------------------------------------------------------------------------
namespace exa {

__global__ void __launch_bounds__(256) mirror_lower_kernel(double* __restrict__ s, int64_t ld, int64_t npad) {
  const int64_t j = blockIdx.y;  // column
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < j; i += (int64_t)gridDim.x * blockDim.x)
    s[i + j * ld] = s[j + i * ld];  // upper (i < j) from lower (j, i)
}

__global__ void __launch_bounds__(256) deriv_matrix_kernel(const double* __restrict__ locs, int64_t n, int64_t npad,
                                                           const __grid_constant__ GradParams G, int k,
                                                           double* __restrict__ D) {
  const int64_t j = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (i < n && j < n) {
      double d[3];
      matern_derivs(G, sqrt(model_dist2(G.m, locs[2 * i], locs[2 * i + 1], locs[2 * j], locs[2 * j + 1])), d[0], d[1],
                    d[2]);
      v = d[k];
    }
    D[i + j * npad] = v;
  }
}

// partial[tile][p] for the 6 pairs p = (0,0),(0,1),(0,2),(1,1),(1,2),(2,2)
__global__ void __launch_bounds__(256) trace_pairs_kernel(const double* __restrict__ M, int64_t npad,
                                                          double* __restrict__ partial) {
  __shared__ double a[3][32][33], b[3][32][33];
  __shared__ double red[6][8];
  const int64_t I = (int64_t)blockIdx.y * 32, J = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t nn = npad * npad;
  for (int k = 0; k < 3; ++k)
    for (int r = ty; r < 32; r += 8) {
      a[k][r][tx] = M[k * nn + (I + tx) + (J + r) * npad];  // a[k][c][r] = M_k(I + r, J + c): stored by column c
      b[k][r][tx] = M[k * nn + (J + tx) + (I + r) * npad];  // b[k][c][r] = M_k(J + r, I + c)
    }
  __syncthreads();
  // tr contribution: sum_{r, c} M_k(I + r, J + c) M_l(J + c, I + r) = sum a[k][c][r] b[l][r][c]
  const int pk[6] = {0, 0, 0, 1, 1, 2}, pl[6] = {0, 1, 2, 1, 2, 2};
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int c = ty; c < 32; c += 8) {
#pragma unroll
    for (int p = 0; p < 6; ++p) s[p] = fma(a[pk[p]][c][tx], b[pl[p]][tx][c], s[p]);
  }
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    double v = s[p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (tx == 0) red[p][ty] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += red[threadIdx.x][w];
    partial[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * 6 + threadIdx.x] = v;
  }
}

__global__ void __launch_bounds__(256) trace_finish_kernel(const double* __restrict__ partial, int64_t ntiles,
                                                           double* __restrict__ out) {
  __shared__ double sh[256];
  const int p = blockIdx.x, tid = threadIdx.x;
  double v = 0.0;
  for (int64_t t = tid; t < ntiles; t += 256) v += partial[t * 6 + p];
  sh[tid] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) sh[tid] += sh[tid + w];
    __syncthreads();
  }
  if (tid == 0) out[p] = 0.5 * sh[0];
}

}  // namespace exa

extern "C" exa_status exa_fisher(exa_ctx* c, const double* d_locs, const double theta[3], int64_t n,
                                 double fisher[9]) {
  if (!c) return EXA_ERR_ARG;
  c->err[0] = 0;
  c->last_pivot = -1;
  if (n < 1 || !d_locs || !fisher) return set_err(c, EXA_ERR_ARG, "bad n or NULL pointer");
  for (int i = 0; i < 9; ++i) fisher[i] = NAN;
  exa_status st = check_theta(c, theta);
  if (st != EXA_OK) return st;
  const int nb = c->tile_nb;
  const int64_t npad = round_up(n, 128);  // 32- and 64-tile kernels below; multiple of nb
  const size_t nn = (size_t)npad * npad;
  if ((st = ensure(c, c->gr_part, nn * sizeof(double), "inverse covariance")) != EXA_OK) return st;
  if ((st = ensure(c, c->fs_m, 3 * nn * sizeof(double), "Fisher products")) != EXA_OK) return st;
  if ((st = ensure(c, c->mat, nn * sizeof(double), "matrix")) != EXA_OK) return st;
  const int64_t t32 = npad / 32;
  if ((st = ensure(c, c->gr_blocks, (size_t)t32 * t32 * 6 * sizeof(double), "Fisher partials")) != EXA_OK) return st;
  if ((st = reset_status(c)) != EXA_OK) return st;
  double* A = (double*)c->mat.p;
  double* S = (double*)c->gr_part.p;
  double* M = (double*)c->fs_m.p;
  cudaStream_t s = c->stream;
  MaternParams P;
  model_params(c, theta, &P);
  const MaternTable* tab = nullptr;
  if ((st = matern_table(c, P, &tab)) != EXA_OK) return st;
  cudaError_t e;
  {
    ProfScope ps(c, PK_GEN, 0.0, 4.0 * (double)npad * (double)(npad + 1));
    e = launch_matern_gen(s, d_locs, n, npad, P, A, npad, nullptr, tab);
  }
  if (e != cudaSuccess) return cuda_err(c, e, "generation launch");
  if ((st = factor_fp64(c, A, npad, npad, nb)) != EXA_OK) return st;
  if ((st = read_status(c)) != EXA_OK) return st;
  e = sigma_inverse_fp64(c, npad, nb, S);
  if (e == cudaSuccess) {
    mirror_lower_kernel<<<dim3((unsigned)((npad + 255) / 256 < 32 ? (npad + 255) / 256 : 32), (unsigned)npad), 256, 0,
                          s>>>(S, npad, npad);
    e = cudaGetLastError();
  }
  GradParams G;
  G.m = P;
  G.psi_nu = host_digamma(theta[2]);
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
    {
      ProfScope ps(c, PK_GRAD, 0.0, 8.0 * (double)nn);
      deriv_matrix_kernel<<<dim3((unsigned)((npad + 255) / 256 < 32 ? (npad + 255) / 256 : 32), (unsigned)npad), 256,
                            0, s>>>(d_locs, n, npad, G, k, A);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      ProfScope ps(c, PK_DGEMM_SMALL, 2.0 * (double)npad * npad * npad, 24.0 * (double)nn);
      e = launch_dgemm_nt_small(s, (int)npad, (int)npad, (int)npad, 1.0, S, 1, npad, A, 1, npad, 0.0, M + k * nn, 1,
                                npad, c->d_status);
    }
  }
  if (e == cudaSuccess) {
    ProfScope ps(c, PK_GRAD, 0.0, 48.0 * (double)nn, 2);
    trace_pairs_kernel<<<dim3((unsigned)t32, (unsigned)t32), 256, 0, s>>>(M, npad, (double*)c->gr_blocks.p);
    trace_finish_kernel<<<6, 256, 0, s>>>((double*)c->gr_blocks.p, t32 * t32, c->d_scalars + 16);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_scalars + 16, c->d_scalars + 16, 6 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_err(c, e, "Fisher launch");
  if ((st = read_status(c)) != EXA_OK) return st;
  const double* v = c->h_scalars + 16;
  const int pk[6] = {0, 0, 0, 1, 1, 2}, pl[6] = {0, 1, 2, 1, 2, 2};
  for (int p = 0; p < 6; ++p) fisher[pk[p] * 3 + pl[p]] = fisher[pl[p] * 3 + pk[p]] = v[p];
  return EXA_OK;
}
