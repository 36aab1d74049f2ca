// Spatial prediction (kriging) at new locations from the FP64 factor of the
// observed field: the conditional mean and variance that the paper's
// exact_predict returns in the sea-surface-temperature tutorial (Section IV).
//
//   a = Sigma^-1 z                    (the factor and the two triangular solves
//                                      of the log-likelihood path)
//   mean_i = c_i^T a,                 c_i = (Sigma(new_i, obs_j))_j, Eq. 3
//   var_i  = sigma^2 - |L^-1 c_i|^2
//
// The mean never stores the cross covariance: each entry is generated from the
// interpolation table where it is used.  The variance needs L^-1 C for a block
// of new points: C (n_pad x 512) is generated, then solved block row by block
// row with the stored inverses of the diagonal tiles (Y_k = W_k C_k, then
// C_rest -= L_rest,k Y_k on FP64 DMMA), accumulating |Y|^2 per column in a
// fixed order.
#include <math.h>
#include <string.h>

#include "bessel.cuh"
#include "ctx.cuh"
#include "util.cuh"

namespace exa {

constexpr int kPredTile = 64;   // new points per CTA of the mean kernel
constexpr int kPredCols = 512;  // new points per block of the variance solve

// mean_i = sum_j Sigma(new_i, obs_j) a_j.  Thread (p, q) = (tid / 4, tid % 4) sums the
// observations j = q (mod 4) for new point p; the four partials are added in order.
__global__ void __launch_bounds__(256) krige_mean_kernel(const double* __restrict__ obs, int64_t n,
                                                         const double* __restrict__ a,
                                                         const double* __restrict__ nl, int64_t m,
                                                         const __grid_constant__ MaternParams P,
                                                         const MaternTable* __restrict__ tab,
                                                         double* __restrict__ mean) {
  __shared__ double sx[256], sy[256], sa[256];
  __shared__ double part[kPredTile][4];
  const int tid = threadIdx.x, p = tid >> 2, q = tid & 3;
  const int64_t i = (int64_t)blockIdx.x * kPredTile + p;
  const double xi = i < m ? nl[2 * i] : 0.0, yi = i < m ? nl[2 * i + 1] : 0.0;
  double acc = 0.0;
  for (int64_t j0 = 0; j0 < n; j0 += 256) {
    const int64_t j = j0 + tid;
    sx[tid] = j < n ? obs[2 * j] : 0.0;
    sy[tid] = j < n ? obs[2 * j + 1] : 0.0;
    sa[tid] = j < n ? a[j] : 0.0;
    __syncthreads();
    const int cnt = (int)((n - j0) < 256 ? (n - j0) : 256);
    for (int t = q; t < cnt; t += 4) {
      acc = fma(matern_value_tab(P, tab, model_dist2(P, xi, yi, sx[t], sy[t])), sa[t], acc);
    }
    __syncthreads();
  }
  part[p][q] = acc;
  __syncthreads();
  if (q == 0 && i < m) mean[i] = ((part[p][0] + part[p][1]) + part[p][2]) + part[p][3];
}

// C(j, c) = Sigma(obs_j, new_{c0 + c}) for j < n; zero for padding rows and past the last point.
__global__ void __launch_bounds__(256) cross_cov_kernel(const double* __restrict__ obs, int64_t n, int64_t npad,
                                                        const double* __restrict__ nl, int64_t m, int64_t c0,
                                                        const __grid_constant__ MaternParams P,
                                                        const MaternTable* __restrict__ tab, double* __restrict__ C) {
  const int64_t c = blockIdx.y;
  const int64_t i = c0 + c;
  const bool live = i < m;
  const double xi = live ? nl[2 * i] : 0.0, yi = live ? nl[2 * i + 1] : 0.0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < npad; j += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (live && j < n) {
      v = matern_value_tab(P, tab, model_dist2(P, obs[2 * j], obs[2 * j + 1], xi, yi));
    }
    C[j + c * npad] = v;
  }
}

// acc[c] += sum_t Y(t, c)^2 over the nb rows of one block (Y column-major, ld = nb); fixed order.
__global__ void col_sumsq_kernel(const double* __restrict__ Y, int nb, int ncols, double* __restrict__ acc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  double s = 0.0;
  for (int t = 0; t < nb; ++t) {
    const double y = Y[t + (int64_t)c * nb];
    s = fma(y, y, s);
  }
  acc[c] += s;
}

__global__ void krige_var_kernel(const double* __restrict__ acc, double sigma2, int64_t c0, int64_t m,
                                 double* __restrict__ var) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c0 + c < m && c < kPredCols) var[c0 + c] = sigma2 - acc[c];
}

}  // namespace exa

using namespace exa;

extern "C" exa_status exa_predict(exa_ctx* c, const double* d_locs, const double* d_z, const double theta[3],
                                  int64_t n, const double* d_new_locs, int64_t m, double* d_mean, double* d_var) {
  if (!c) return EXA_ERR_ARG;
  c->err[0] = 0;
  c->last_pivot = -1;
  if (n < 1 || m < 0 || !d_locs || !d_z || (m > 0 && (!d_new_locs || !d_mean)))
    return set_err(c, EXA_ERR_ARG, "bad sizes or NULL device pointer");
  exa_status st = check_theta(c, theta);
  if (st != EXA_OK) return st;
  if (m == 0) return EXA_OK;
  // factor, y = L^-1 z (log-likelihood path, FP64)
  exa_result res;
  memset(&res, 0, sizeof(res));
  double* y = nullptr;
  if ((st = loglik_fp64(c, d_locs, d_z, theta, n, &res, &y)) != EXA_OK) return st;
  const int nb = c->tile_nb;
  const int64_t npad = round_up(n, nb);
  const int T = (int)(npad / nb);
  double* A = (double*)c->mat.p;
  const double* W = (const double*)c->w_all.p;
  double* part = (double*)c->partial.p;
  cudaStream_t s = c->stream;
  cudaError_t e = cudaSuccess;
  // a = L^-T y (in place)
  for (int k = T - 1; k >= 0 && e == cudaSuccess; --k) {
    const double rows = (double)(npad - (int64_t)k * nb);
    ProfScope ps(c, PK_TRSV, 2.0 * rows * nb, 8.0 * rows * nb, 2);
    e = launch_trsv_bwd_step(s, A, npad, npad, nb, k, W, y, part + 2 * kRedPartials, c->d_status);
  }
  if (e != cudaSuccess) return cuda_err(c, e, "prediction solve");
  MaternParams P;
  model_params(c, theta, &P);
  const MaternTable* tab = nullptr;
  if ((st = matern_table(c, P, &tab)) != EXA_OK) return st;
  {
    ProfScope ps(c, PK_GEN, 0.0, 16.0 * (double)n + 24.0 * (double)m);
    krige_mean_kernel<<<(unsigned)((m + kPredTile - 1) / kPredTile), 256, 0, s>>>(d_locs, n, y, d_new_locs, m, P,
                                                                                 tab, d_mean);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_err(c, e, "prediction mean");
  if (d_var) {
    // variance: blocks of kPredCols new points
    if ((st = ensure(c, c->pr_c, (size_t)npad * kPredCols * sizeof(double), "prediction cross covariance")) !=
        EXA_OK)
      return st;
    if ((st = ensure(c, c->pr_y, (size_t)(nb + 1) * kPredCols * sizeof(double), "prediction solve block")) !=
        EXA_OK)
      return st;
    double* C = (double*)c->pr_c.p;
    double* Y = (double*)c->pr_y.p;
    double* acc = Y + (size_t)nb * kPredCols;
    for (int64_t c0 = 0; c0 < m && e == cudaSuccess; c0 += kPredCols) {
      {
        ProfScope ps(c, PK_GEN, 0.0, 8.0 * (double)npad * kPredCols);
        cross_cov_kernel<<<dim3((unsigned)((npad + 255) / 256 < 64 ? (npad + 255) / 256 : 64), kPredCols), 256, 0,
                           s>>>(d_locs, n, npad, d_new_locs, m, c0, P, tab, C);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, kPredCols * sizeof(double), s);
      for (int k = 0; k < T && e == cudaSuccess; ++k) {
        const int64_t k0 = (int64_t)k * nb, rest = npad - k0 - nb;
        ProfScope ps(c, PK_DGEMM_SMALL, 2.0 * (double)(nb + rest) * nb * kPredCols,
                     8.0 * ((double)(nb + rest) * nb + 2.0 * (double)(nb + rest) * kPredCols), 2 + (rest > 0));
        // Y = W_k C_k   (W_k row-major nb x nb; C_k rows k0.. of C)
        e = launch_dgemm_nt_small(s, nb, kPredCols, nb, 1.0, W + (int64_t)k * nb * nb, nb, 1, C + k0, npad, 1, 0.0,
                                  Y, 1, nb, c->d_status);
        if (e == cudaSuccess) {
          col_sumsq_kernel<<<kPredCols / 128, 128, 0, s>>>(Y, nb, kPredCols, acc);
          e = cudaGetLastError();
        }
        // C_rest -= L_rest,k Y
        if (e == cudaSuccess && rest > 0)
          e = launch_dgemm_nt_small(s, (int)rest, kPredCols, nb, -1.0, A + k0 + nb + k0 * npad, 1, npad, Y, nb, 1,
                                    1.0, C + k0 + nb, 1, npad, c->d_status);
      }
      if (e == cudaSuccess) {
        krige_var_kernel<<<kPredCols / 128, 128, 0, s>>>(acc, theta[0], c0, m, d_var);
        e = cudaGetLastError();
      }
    }
    if (e != cudaSuccess) return cuda_err(c, e, "prediction variance");
  }
  return read_status(c);
}
