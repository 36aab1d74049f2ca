// Device modified Bessel function of the second kind K_nu for fractional nu,
// shared by the covariance generation (Eq. 3) and the gradient kernels.
#pragma once

#include <math.h>

#include "exa_internal.cuh"

namespace exa {

// D(mu) = (Gamma(1+mu) - Gamma(1-mu)) / (2 mu) = int_0^inf e^-t sinh(mu ln t) / mu dt.
// With t = e^u the integrand exp(u - e^u) sinh(mu u)/mu is analytic in the strip
// |Im u| < pi/2 and decays like e^{(1-|mu|) u} (u -> -inf) and doubly
// exponentially (u -> +inf), so the trapezoid rule with h = 1/16 on [-110, 5]
// is exact to rounding.  D(0) = Gamma'(1).  Written this way Gamma_1(mu) has no
// cancellation as mu -> 0 (integer nu).
__host__ __device__ inline double temme_D(double mu) {
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

// Per-theta constants (host, or device for parameters that live in device memory).
__host__ __device__ inline void matern_params_hd(const double theta[3], MaternParams* p) {
  const double nu = theta[2];
  p->sigma2 = theta[0];
  p->beta = theta[1];
  p->ib2 = 1.0 / (theta[1] * theta[1]);
  p->nugget = 0.0;
  p->radius = 6371.0;
  p->metric = 0;
  p->pad2_ = 0;
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

// Squared distance between two locations: Euclidean, or the great-circle distance
// (haversine form) between (longitude, latitude) pairs in degrees on a sphere of
// radius P.radius (the paper's dmetric = great_circle).
__device__ __forceinline__ double model_dist2(const MaternParams& P, double x1, double y1, double x2, double y2) {
  if (P.metric == 1) {
    const double rad = 3.14159265358979323846 / 180.0;
    const double p1 = y1 * rad, p2 = y2 * rad;
    const double sp = sin(0.5 * (p2 - p1)), sl = sin(0.5 * (x2 - x1) * rad);
    const double a = fmin(fma(cos(p1) * cos(p2), sl * sl, sp * sp), 1.0);
    const double d = 2.0 * P.radius * asin(sqrt(a));
    return d * d;
  }
  const double dx = x1 - x2, dy = y1 - y2;
  return dx * dx + dy * dy;
}

// Sigma / sigma^2 at x = r / beta > 0 (Eq. 3 without the variance).
__device__ __forceinline__ double matern_ratio(const MaternParams& P, double x) {
  if (x > 800.0) return 0.0;
  const double lnx = log(x);
  double knu, knum1;
  const bool scaled = bessel_k_nu(P, x, lnx, knu, knum1);
  return exp(P.logc + P.nu * lnx - (scaled ? x : 0.0)) * knu;
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

// Segment of s for the table (s finite, 2^kTabE0 <= s < 2^(kTabE0 + kTabOct)):
// integer work on the bit pattern only.
__device__ __forceinline__ int table_segment(double s) {
  const long long b = __double_as_longlong(s);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  const int sub = (int)((b >> (52 - kTabSubBits)) & (kTabSub - 1));
  return (e - kTabE0) * kTabSub + sub;
}

// Table construction.  Segment sgi covers [lo, lo + w) of s with lo = 2^e (1 + sub / kTabSub),
// w = 2^e / kTabSub.  Node id = sgi (kTabDeg + 1) + k is f at the k-th Chebyshev point.
__device__ __forceinline__ void segment_geometry(int sgi, double& centre, double& half) {
  const int e = kTabE0 + sgi / kTabSub, sub = sgi % kTabSub;
  const double lo = ldexp(1.0 + (double)sub / kTabSub, e);
  const double w = ldexp(1.0 / kTabSub, e);
  centre = lo + 0.5 * w;
  half = 0.5 * w;
}

__device__ __forceinline__ double table_node_value(const MaternParams& P, int id) {
  const int sgi = id / (kTabDeg + 1), k = id % (kTabDeg + 1);
  double centre, half;
  segment_geometry(sgi, centre, half);
  const double tk = cos(3.14159265358979323846 * (k + 0.5) / (kTabDeg + 1));
  // Sigma itself (sigma^2 folded in: one FP64 multiplication fewer per generated entry) at
  // the k-th Chebyshev point of s
  return P.sigma2 * matern_ratio(P, sqrt(centre + half * tk));
}

// Chebyshev coefficients of segment sgi from its nodes, then their monomial form in t.
__device__ __forceinline__ void table_segment_coefs(const double* __restrict__ nodes, int sgi,
                                                    MaternTable* __restrict__ T) {
  constexpr int N = kTabDeg + 1;
  const double* q = nodes + sgi * N;
  double cheb[N];
  for (int j = 0; j < N; ++j) {
    double s = 0.0;
    for (int k = 0; k < N; ++k) s += q[k] * cos(3.14159265358979323846 * j * (k + 0.5) / N);
    cheb[j] = (j == 0 ? 1.0 : 2.0) * s / N;
  }
  // T_0 = 1, T_1 = t, T_{j+1} = 2 t T_j - T_{j-1}
  double a[N], tm1[N], t0[N], t1[N];
  for (int i = 0; i < N; ++i) a[i] = tm1[i] = t0[i] = 0.0;
  tm1[0] = 1.0;
  t0[1] = 1.0;
  a[0] = cheb[0];
  for (int i = 0; i < N; ++i) a[i] += cheb[1] * t0[i];
  for (int j = 2; j < N; ++j) {
    for (int i = 0; i < N; ++i) t1[i] = (i > 0 ? 2.0 * t0[i - 1] : 0.0) - tm1[i];
    for (int i = 0; i < N; ++i) a[i] += cheb[j] * t1[i];
    for (int i = 0; i < N; ++i) {
      tm1[i] = t0[i];
      t0[i] = t1[i];
    }
  }
  double centre, half;
  segment_geometry(sgi, centre, half);
  T->ih[sgi] = 1.0 / half;
  T->mc[sgi] = -centre / half;
  for (int i = 0; i < N; ++i) T->a[sgi][i] = a[i];
}

// The exact routine as an out-of-line call for the table's rare out-of-range entries, so that
// its registers and stack stay out of the generators' per-entry loops.
static __device__ __noinline__ double matern_value_exact(const MaternParams& P, double r) { return matern_value(P, r); }

// Sigma at squared distance r2 = r^2 from the table (exact routine outside its range).  The
// tests are integer work on the bit patterns: FP64 instructions are the scarce resource of the
// generation (~2 per clock per SM on this part), FP64 comparisons included.
__device__ __forceinline__ double matern_value_tab(const MaternParams& P, const MaternTable* __restrict__ T,
                                                   double r2) {
  if (__double_as_longlong(r2) == 0) return P.sigma2;  // r2 >= 0: only +0 has all bits clear
  const double s = r2 * P.ib2;
  static_assert(kTabE0 == -8 && kTabE0 + kTabOct == 12, "table range below");
  // 2^-8 <= s < 2^12 exactly when the sign is clear and the biased exponent is in [1015, 1035)
  // (negative, zero, subnormal, infinite and NaN values all fall outside)
  const unsigned int se = (unsigned int)((unsigned long long)__double_as_longlong(s) >> 52);
  if (se - (unsigned int)(1023 + kTabE0) >= (unsigned int)kTabOct) return matern_value_exact(P, sqrt(r2));
  const int sgi = table_segment(s);
  const double t = fma(s, __ldg(&T->ih[sgi]), __ldg(&T->mc[sgi]));
  const double* c = T->a[sgi];
  double f = __ldg(&c[kTabDeg]);
#pragma unroll
  for (int k = kTabDeg - 1; k >= 0; --k) f = fma(f, t, __ldg(&c[k]));
  return f;  // the table holds Sigma, sigma^2 included
}

}  // namespace exa
