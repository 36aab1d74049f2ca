// Step a1: Matérn covariance generation (Section I, Eq. 3) with a device
// modified Bessel function K_nu of fractional order.
//
// Per theta the host precomputes every quantity that depends only on nu
// (Gamma values, Temme's Gamma_1/Gamma_2, reciprocal tables), so the per-entry
// work is one log, one exp (+ one sqrt for x > 2) and division-free loops.
#include <math.h>

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
// Device side
// ---------------------------------------------------------------------------

// K_mu(x), K_{mu+1}(x) for 0 < x <= 2 by Temme's series:
//   K_mu = sum_k c_k f_k,  K_{mu+1} = (2/x) sum_k c_k h_k,  c_k = (x^2/4)^k / k!,
//   f_0 = (mu pi / sin mu pi) [cosh(s) Gamma_1 + sinh(s)/s ln(2/x) Gamma_2],  s = mu ln(2/x),
//   p_0 = (x/2)^-mu Gamma(1+mu) / 2,  q_0 = (x/2)^mu Gamma(1-mu) / 2,
//   f_k = (k f_{k-1} + p_{k-1} + q_{k-1}) / (k^2 - mu^2),  p_k = p_{k-1}/(k - mu),
//   q_k = q_{k-1}/(k + mu),  h_k = p_k - k f_k.
__device__ __forceinline__ void bessel_temme(const MaternParams& P, double x, double lnx, double& k0, double& k1) {
  const double mu = P.mu;
  const double l2x = 0.69314718055994530942 - lnx;  // ln(2/x)
  const double s = mu * l2x;
  const double es = exp(s);                          // (x/2)^-mu
  const double ies = 1.0 / es;
  const double ch = 0.5 * (es + ies);
  double shs;                                        // sinh(s) / s
  if (fabs(s) < 1e-3) {
    const double s2 = s * s;
    shs = 1.0 + s2 * (1.0 / 6.0 + s2 * (1.0 / 120.0 + s2 * (1.0 / 5040.0)));
  } else {
    shs = 0.5 * (es - ies) / s;
  }
  double f = P.mupi_sin * (ch * P.gam1 + shs * l2x * P.gam2);
  double p = 0.5 * es * P.gp;
  double q = 0.5 * ies * P.gm;
  const double x2 = 0.25 * x * x;
  double c = 1.0;
  double s0 = f, s1 = p;
  for (int k = 1; k <= kTemmeTerms; ++k) {
    const double dk = (double)k;
    f = fma(dk, f, p + q) * P.t_k2[k];
    p *= P.t_km[k];
    q *= P.t_kp[k];
    c *= x2 / dk;
    const double h = fma(-dk, f, p);
    const double tf = c * f, th = c * h;
    s0 += tf;
    s1 += th;
    if (fabs(tf) <= 1e-17 * fabs(s0) && fabs(th) <= 1e-17 * fabs(s1)) break;
  }
  k0 = s0;
  k1 = 2.0 * s1 / x;
}

// e^x K_mu(x), e^x K_{mu+1}(x) for x > 2: z_k = U(mu + 1/2 + k, 2mu + 1, 2x) obey
//   z_{k-1} = 2(k + x) z_k - ((k + 1/2)^2 - mu^2) z_{k+1}      (DLMF 13.3.7),
// whose decaying solution is reached by running it backward from depth D
// (Miller), and sum_k C_k z_k = (2x)^(-mu-1/2) fixes its scale, so
//   e^x K_mu = sqrt(pi/(2x)) z_0 / sum_k C_k z_k,
//   K_{mu+1} / K_mu = (mu + 1/2 + x + (mu^2 - 1/4) z_1/z_0) / x.
// D = ceil(12 + 160/x) keeps the truncation error below 1e-16 for |mu| <= 1/2.
__device__ __forceinline__ void bessel_miller(const MaternParams& P, double x, double& k0s, double& k1s) {
  const double mu = P.mu;
  int D = (int)(12.0 + 160.0 / x) + 1;
  if (D > kMillerMax) D = kMillerMax;
  double zp1 = 0.0, z = 1.0;
  double S = P.m_c[D];
  for (int k = D; k >= 1; --k) {
    const double zm1 = fma(2.0 * ((double)k + x), z, -P.m_a[k] * zp1);
    zp1 = z;
    z = zm1;
    S = fma(P.m_c[k - 1], z, S);
  }
  const double r01 = zp1 / z;  // z_1 / z_0
  k0s = sqrt(1.5707963267948966192 / x) * (z / S);
  k1s = k0s / x * (mu + 0.5 + x + (mu * mu - 0.25) * r01);
}

// K_nu(x) and K_{nu-1}(x) with a common scale: returns scaled = true when the
// values are e^x K (x > 2).  x must be finite and > 0.
__device__ __forceinline__ bool bessel_k_nu(const MaternParams& P, double x, double lnx, double& knu, double& knum1) {
  double a, b;  // K_mu, K_{mu+1}
  bool scaled;
  if (x <= 2.0) {
    bessel_temme(P, x, lnx, a, b);
    scaled = false;
  } else {
    bessel_miller(P, x, a, b);
    scaled = true;
  }
  if (P.N == 0) {
    knu = a;
    knum1 = b - 2.0 * P.mu / x * a;  // K_{mu-1} = K_{mu+1} - (2 mu / x) K_mu
  } else {
    const double ix = 1.0 / x;
    for (int j = 1; j < P.N; ++j) {  // (a, b) = (K_{mu+j-1}, K_{mu+j}) -> (K_{mu+j}, K_{mu+j+1})
      const double c = fma(2.0 * (P.mu + j) * ix, b, a);
      a = b;
      b = c;
    }
    knu = b;
    knum1 = a;
  }
  return scaled;
}

// Eq. 3 at distance r.
__device__ __forceinline__ double matern_value(const MaternParams& P, double r) {
  if (r == 0.0) return P.sigma2;
  const double x = r / P.beta;
  if (!(x > 0.0)) return x;      // NaN propagates
  if (x > 800.0) return 0.0;     // sigma^2 c x^nu K_nu(x) < 1e-340: underflows to 0
  const double lnx = log(x);
  double knu, knum1;
  const bool scaled = bessel_k_nu(P, x, lnx, knu, knum1);
  const double e = P.logc + P.nu * lnx - (scaled ? x : 0.0);
  return P.sigma2 * exp(e) * knu;
}

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
