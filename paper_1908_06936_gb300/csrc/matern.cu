// Step a1: Matérn covariance generation (Section I, Eq. 3) with a device
// modified Bessel function K_nu of fractional order.
//
// Per theta the host precomputes every quantity that depends only on nu
// (Gamma values, Temme's Gamma_1/Gamma_2, reciprocal tables), so the per-entry
// work is one log, one exp (+ one sqrt for x > 2) and division-free loops.
#include <math.h>

#include "bessel.cuh"
#include "exa_internal.cuh"

namespace exa {

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// D(mu) = (Gamma(1+mu) - Gamma(1-mu)) / (2 mu) = int_0^inf e^-t sinh(mu ln t) / mu dt.
// With t = e^u the integrand exp(u - e^u) sinh(mu u)/mu is analytic in the strip
// |Im u| < pi/2 and decays like e^{(1-|mu|) u} (u -> -inf) and doubly
// exponentially (u -> +inf), so the trapezoid rule with h = 1/16 on [-110, 5]
// is exact to rounding.  D(0) = Gamma'(1).  Written this way Gamma_1(mu) has no
// cancellation as mu -> 0 (integer nu).
static double temme_D(double mu) {
  const double h = 1.0 / 16.0;
  double s = 0.0;
  for (int k = -110 * 16; k <= 5 * 16; ++k) {
    const double u = h * k;
    const double w = mu * u;
    double sh;  // sinh(mu u) / mu
    if (fabs(w) < 1e-4)
      sh = u * (1.0 + w * w / 6.0);
    else
      sh = sinh(w) / mu;
    s += exp(u - exp(u)) * sh;
  }
  return s * h;
}

void matern_params(const double theta[3], MaternParams* p) {
  const double nu = theta[2];
  p->sigma2 = theta[0];
  p->beta = theta[1];
  p->nu = nu;
  p->logc = (1.0 - nu) * 0.69314718055994530942 - lgamma(nu);
  const int N = (int)floor(nu + 0.5);
  const double mu = nu - N;
  p->N = N;
  p->mu = mu;
  p->pad_ = 0;
  const double pi = 3.14159265358979323846;
  const double sinc = (mu == 0.0) ? 1.0 : sin(pi * mu) / (pi * mu);
  p->mupi_sin = 1.0 / sinc;
  p->gp = tgamma(1.0 + mu);
  p->gm = tgamma(1.0 - mu);
  // Gamma_1 = D(mu) / (Gamma(1+mu) Gamma(1-mu)) and Gamma(1+mu) Gamma(1-mu) = 1 / sinc
  p->gam1 = temme_D(mu) * sinc;
  p->gam2 = 0.5 * (1.0 / p->gm + 1.0 / p->gp);
  p->t_k2[0] = p->t_km[0] = p->t_kp[0] = 0.0;
  for (int k = 1; k <= kTemmeTerms; ++k) {
    p->t_k2[k] = 1.0 / ((double)k * k - mu * mu);
    p->t_km[k] = 1.0 / (k - mu);
    p->t_kp[k] = 1.0 / (k + mu);
  }
  p->m_c[0] = 1.0;
  for (int k = 0; k <= kMillerMax + 1; ++k) {
    p->m_a[k] = (k + 0.5) * (k + 0.5) - mu * mu;
    if (k + 1 <= kMillerMax + 1) p->m_c[k + 1] = p->m_c[k] * p->m_a[k] / (k + 1);
  }
}

// ---------------------------------------------------------------------------
// Device side (K_nu itself lives in bessel.cuh)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void tri_decode(long long b, int& ti, int& tj) {
  // b = ti (ti + 1) / 2 + tj,  0 <= tj <= ti
  long long t = (long long)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while (t * (t + 1) / 2 > b) --t;
  while ((t + 1) * (t + 2) / 2 <= b) ++t;
  ti = (int)t;
  tj = (int)(b - t * (t + 1) / 2);
}

// One 64 x 64 tile of the lower triangle per block; 256 threads, each thread
// 16 entries of one column strip (consecutive threads = consecutive rows, so
// the column-major stores coalesce).
__global__ void __launch_bounds__(256) matern_gen_kernel(const double* __restrict__ locs, int64_t n, int64_t npad,
                                                         const __grid_constant__ MaternParams P, double* __restrict__ a,
                                                         int64_t ld, unsigned long long* __restrict__ offmax) {
  int ti, tj;
  tri_decode(blockIdx.x, ti, tj);
  const int64_t i = (int64_t)ti * 64 + (threadIdx.x & 63);
  double vmax = 0.0;  // largest off-diagonal |Sigma_ij| of this thread (for the precision map)
  if (i < npad) {
  double xi = 0.0, yi = 0.0;
  if (i < n) {
    xi = __ldg(locs + 2 * i);
    yi = __ldg(locs + 2 * i + 1);
  }
  for (int s = 0; s < 16; ++s) {
    const int64_t j = (int64_t)tj * 64 + (threadIdx.x >> 6) + 4 * s;
    if (j > i || j >= npad) continue;
    double v;
    if (i >= n || j >= n) {
      v = (i == j) ? 1.0 : 0.0;  // identity padding
    } else if (i == j) {
      v = P.sigma2;
    } else {
      const double dx = xi - __ldg(locs + 2 * j);
      const double dy = yi - __ldg(locs + 2 * j + 1);
      v = matern_value(P, sqrt(dx * dx + dy * dy));
      vmax = fmax(vmax, fabs(v));
    }
    a[i + j * ld] = v;
  }
  }
  if (offmax) {
    // non-negative doubles order like their bit patterns: one atomicMax per warp
    unsigned long long b = (unsigned long long)__double_as_longlong(vmax);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, b, o);
      b = ob > b ? ob : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&offmax[(ti >> 2) - (tj >> 2)], b);
  }
}

cudaError_t launch_matern_gen(cudaStream_t s, const double* locs, int64_t n, int64_t npad, const MaternParams& p,
                              double* a, int64_t ld, unsigned long long* offmax) {
  const long long t = (npad + 63) / 64;
  const long long blocks = t * (t + 1) / 2;
  if (blocks <= 0) return cudaSuccess;
  matern_gen_kernel<<<(unsigned)blocks, 256, 0, s>>>(locs, n, npad, p, a, ld, offmax);
  return cudaGetLastError();
}

}  // namespace exa
