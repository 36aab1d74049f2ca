/*
 * FP64 CPU oracle for the exact Matérn Gaussian log-likelihood.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg may load or call this code.  The
 * product path (the CUDA library and its Python binding) never does, and
 * shares no code with it.
 *
 * Everything here is the plain mathematical definition, written out in
 * double precision, in the order the paper states it, so that it can be
 * checked against the paper by eye:
 *
 *   Eq. 2  Gaussian likelihood with zero mean (Section I):
 *          l(theta) = -n/2 log(2 pi) - 1/2 log|Sigma| - 1/2 Z^T Sigma^-1 Z
 *   Eq. 3  Matérn covariance (Section I):
 *          Sigma_ij = sigma^2 / (2^(nu-1) Gamma(nu)) (r/beta)^nu K_nu(r/beta),
 *          r = ||s_i - s_j|| (Euclidean), Sigma_ii = sigma^2 (the r -> 0 limit)
 *   Section I: Sigma^-1 Z and |Sigma| come from the Cholesky factor
 *          Sigma = L L^T:  log|Sigma| = 2 sum log L_ii,  Z^T Sigma^-1 Z = |L^-1 Z|^2.
 *
 * K_nu is evaluated from its integral representation (DLMF 10.32.9)
 *          K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt
 * by the trapezoidal rule.  The integrand is entire and decays doubly
 * exponentially, so the rule converges geometrically in 1/h; the step used
 * below keeps the discretisation error under 1e-17 relative (see
 * oracle_besselk_scaled).  dK_nu/dnu is the same integral differentiated
 * under the integral sign.  The gradient of l (not in the paper, whose
 * optimiser is derivative free) uses the standard identity
 *          dl/dtheta_k = 1/2 a^T D_k a - 1/2 tr(Sigma^-1 D_k),
 *          a = Sigma^-1 Z,  D_k = dSigma/dtheta_k,
 * with Sigma^-1 formed explicitly from L^-1.
 *
 * Storage: row-major n x n doubles.  Locations are n x 2 interleaved
 * (x_0, y_0, x_1, y_1, ...).  OpenMP parallel loops only split independent
 * rows; every entry is computed in the same order as the serial loop.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static const double ORACLE_LN2 = 0.69314718055994530941723212145818;
static const double ORACLE_LN_2PI = 1.8378770664093454835606594728112;

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Trapezoid step for the K_nu integrals.  Near the real axis the integrand
 * stays analytic in the strip |Im t| < pi/2; for large x the relevant width
 * shrinks like 1/sqrt(x).  h = min(1/8, 1/(2 sqrt x)) keeps the error
 * estimate exp(-2 pi^2 / (h^2 x)) or exp(-pi^2 / h) below e^-78.          */
static double oracle_quad_step(double x) {
  double h = 0.125;
  if (x > 16.0) h = 0.5 / sqrt(x);
  return h;
}

/* e^x K_nu(x) = int_0^inf exp(-x (cosh t - 1)) cosh(nu t) dt  (DLMF 10.32.9
 * multiplied by e^x so that large x does not underflow).  x > 0.          */
double oracle_besselk_scaled(double nu, double x) {
  const double h = oracle_quad_step(x);
  /* f(0) / 2 */
  double sum = 0.5;
  for (long k = 1; k < 2000000; ++k) {
    const double t = h * (double)k;
    const double sh = sinh(0.5 * t);
    const double f = exp(-x * 2.0 * sh * sh) * cosh(nu * t);
    sum += f;
    /* stop once past the peak of the integrand and the terms are negligible */
    const double past_peak = x * sinh(t) - fabs(nu) * tanh(fabs(nu) * t);
    if (past_peak > 0.0 && f < 1e-20 * sum) break;
  }
  return h * sum;
}

double oracle_besselk(double nu, double x) {
  return exp(-x) * oracle_besselk_scaled(nu, x);
}

/* e^x dK_nu(x)/dnu = int_0^inf t sinh(nu t) exp(-x (cosh t - 1)) dt        */
double oracle_dbesselk_dnu_scaled(double nu, double x) {
  if (nu == 0.0) return 0.0; /* K_nu is even in nu */
  const double h = oracle_quad_step(x);
  const double anu = fabs(nu);
  double sum = 0.0; /* the t = 0 node contributes 0 */
  for (long k = 1; k < 2000000; ++k) {
    const double t = h * (double)k;
    const double sh = sinh(0.5 * t);
    const double f = t * sinh(nu * t) * exp(-x * 2.0 * sh * sh);
    sum += f;
    /* log-derivative of the integrand is 1/t + nu coth(nu t) - x sinh t */
    const double past_peak = x * sinh(t) - 1.0 / t - anu / tanh(anu * t);
    if (past_peak > 0.0 && fabs(f) <= 1e-20 * fabs(sum)) break;
  }
  return h * sum;
}

double oracle_dbesselk_dnu(double nu, double x) {
  return exp(-x) * oracle_dbesselk_dnu_scaled(nu, x);
}

/* Digamma psi(x), x > 0: recurrence psi(x) = psi(x+1) - 1/x up to x >= 10,
 * then the asymptotic expansion psi(x) ~ ln x - 1/(2x) - sum B_2k/(2k x^2k)
 * (DLMF 5.11.2) with Bernoulli numbers B_2 .. B_14.                        */
double oracle_digamma(double x) {
  double acc = 0.0;
  while (x < 10.0) {
    acc -= 1.0 / x;
    x += 1.0;
  }
  const double x2 = 1.0 / (x * x);
  /* B_2k / (2k):  1/12, -1/120, 1/252, -1/240, 1/132, -691/32760, 1/12 */
  double series = x2 * (1.0 / 12.0 +
                  x2 * (-1.0 / 120.0 +
                  x2 * (1.0 / 252.0 +
                  x2 * (-1.0 / 240.0 +
                  x2 * (1.0 / 132.0 +
                  x2 * (-691.0 / 32760.0 +
                  x2 * (1.0 / 12.0)))))));
  return acc + log(x) - 0.5 / x - series;
}

/* Eq. 3: Matérn covariance at distance r for theta = (sigma^2, beta, nu).
 * Written as sigma^2 * exp((1 - nu) ln 2 - ln Gamma(nu) + nu ln x - x)
 *                    * (e^x K_nu(x)),  x = r / beta.                       */
double oracle_matern(const double theta[3], double r) {
  const double sigma2 = theta[0], beta = theta[1], nu = theta[2];
  if (r == 0.0) return sigma2;
  const double x = r / beta;
  const double logc = (1.0 - nu) * ORACLE_LN2 - lgamma(nu);
  return sigma2 * exp(logc + nu * log(x) - x) * oracle_besselk_scaled(nu, x);
}

/* The same value written directly as Eq. 3 prints it (used by tests to
 * check the log-space form above).                                         */
double oracle_matern_direct(const double theta[3], double r) {
  const double sigma2 = theta[0], beta = theta[1], nu = theta[2];
  if (r == 0.0) return sigma2;
  const double x = r / beta;
  return sigma2 / (pow(2.0, nu - 1.0) * tgamma(nu)) * pow(x, nu) * oracle_besselk(nu, x);
}

/* Partial derivatives of Eq. 3 with respect to (sigma^2, beta, nu) at r.
 *   d/dsigma^2 = Sigma / sigma^2
 *   d/dbeta    = sigma^2 c x^nu K_{nu-1}(x) x / beta   (d[x^nu K_nu]/dx = -x^nu K_{nu-1}, DLMF 10.29.4)
 *   d/dnu      = Sigma (-ln 2 - psi(nu) + ln x) + sigma^2 c x^nu dK_nu/dnu
 * with c = 2^(1-nu) / Gamma(nu); all three vanish except d/dsigma^2 at r = 0. */
void oracle_matern_grad(const double theta[3], double r, double out[3]) {
  const double sigma2 = theta[0], beta = theta[1], nu = theta[2];
  if (r == 0.0) {
    out[0] = 1.0;
    out[1] = 0.0;
    out[2] = 0.0;
    return;
  }
  const double x = r / beta;
  const double logc = (1.0 - nu) * ORACLE_LN2 - lgamma(nu);
  const double pref = sigma2 * exp(logc + nu * log(x) - x); /* sigma^2 c x^nu e^-x */
  const double s = pref * oracle_besselk_scaled(nu, x);
  out[0] = s / sigma2;
  out[1] = pref * oracle_besselk_scaled(nu - 1.0, x) * x / beta;
  out[2] = s * (-ORACLE_LN2 - oracle_digamma(nu) + log(x)) + pref * oracle_dbesselk_dnu_scaled(nu, x);
}

/* Model options (the paper's dmetric of Section III, Example 1, and the nugget of Section V):
 *   metric 0: Euclidean distance between (x, y) pairs;
 *   metric 1: great-circle distance (haversine form, the reference the paper cites
 *             for dmetric = great_circle) between (longitude, latitude) pairs in
 *             degrees on a sphere of the given radius;
 *   nugget:   tau^2 added to every diagonal entry (Sigma + tau^2 I).           */
static double g_nugget = 0.0;
static int g_metric = 0;
static double g_radius = 6371.0;

void oracle_set_model(double nugget, int metric, double radius) {
  g_nugget = nugget;
  g_metric = metric;
  g_radius = radius;
}

static double oracle_dist_xy(double x1, double y1, double x2, double y2) {
  if (g_metric == 1) {
    const double rad = 3.14159265358979323846 / 180.0;
    const double p1 = y1 * rad, p2 = y2 * rad;
    const double sp = sin(0.5 * (p2 - p1)), sl = sin(0.5 * (x2 - x1) * rad);
    double a = sp * sp + cos(p1) * cos(p2) * sl * sl;
    if (a > 1.0) a = 1.0;
    return 2.0 * g_radius * asin(sqrt(a));
  }
  const double dx = x1 - x2, dy = y1 - y2;
  return sqrt(dx * dx + dy * dy);
}

static double oracle_dist(const double* locs, int64_t i, int64_t j) {
  return oracle_dist_xy(locs[2 * i], locs[2 * i + 1], locs[2 * j], locs[2 * j + 1]);
}

/* Full symmetric covariance matrix, row-major n x n.                       */
void oracle_covariance(int64_t n, const double* locs, const double theta[3], double* S) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j <= i; ++j) {
      const double v = oracle_matern(theta, oracle_dist(locs, i, j)) + (i == j ? g_nugget : 0.0);
      S[i * n + j] = v;
      S[j * n + i] = v;
    }
  }
}

/* Selected entries Sigma_{rows[k], cols[k]} (for sampled checks at sizes
 * where the full matrix is out of reach).                                  */
void oracle_covariance_entries(int64_t m, const int64_t* rows, const int64_t* cols, const double* locs,
                               const double theta[3], double* out) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t k = 0; k < m; ++k)
    out[k] = oracle_matern(theta, oracle_dist(locs, rows[k], cols[k])) + (rows[k] == cols[k] ? g_nugget : 0.0);
}

/* Unblocked Cholesky (Cholesky-Crout, lower), in place on a row-major n x n
 * matrix; only the lower triangle is read and written.  Returns 0, or j + 1
 * when the pivot of column j is not positive (Sigma not positive definite). */
int64_t oracle_cholesky(int64_t n, double* A) {
  for (int64_t j = 0; j < n; ++j) {
    double* Lj = A + j * n;
    double s = Lj[j];
    for (int64_t k = 0; k < j; ++k) s -= Lj[k] * Lj[k];
    if (!(s > 0.0)) return j + 1;
    const double ljj = sqrt(s);
    Lj[j] = ljj;
#pragma omp parallel for schedule(static)
    for (int64_t i = j + 1; i < n; ++i) {
      double* Li = A + i * n;
      double t = Li[j];
      for (int64_t k = 0; k < j; ++k) t -= Li[k] * Lj[k];
      Li[j] = t / ljj;
    }
  }
  return 0;
}

/* y = L^-1 b by forward substitution (L lower, row-major).                 */
void oracle_forward_solve(int64_t n, const double* L, const double* b, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double t = b[i];
    const double* Li = L + i * n;
    for (int64_t k = 0; k < i; ++k) t -= Li[k] * y[k];
    y[i] = t / Li[i];
  }
}

/* a = L^-T y by backward substitution.                                     */
void oracle_backward_solve(int64_t n, const double* L, const double* y, double* a) {
  for (int64_t i = n - 1; i >= 0; --i) {
    double t = y[i];
    for (int64_t k = i + 1; k < n; ++k) t -= L[k * n + i] * a[k];
    a[i] = t / L[i * n + i];
  }
}

/* Log-likelihood, Eq. 2 with mu = 0.  out = {l, log|Sigma|, Z^T Sigma^-1 Z}.
 * Returns 0, or the not-positive-definite pivot index + 1 (out = NaN).     */
int64_t oracle_loglik(int64_t n, const double* locs, const double* Z, const double theta[3], double out[3]) {
  double* A = (double*)malloc((size_t)n * (size_t)n * sizeof(double));
  double* y = (double*)malloc((size_t)n * sizeof(double));
  if (!A || !y) {
    free(A);
    free(y);
    return -1;
  }
  oracle_covariance(n, locs, theta, A);
  const int64_t info = oracle_cholesky(n, A);
  if (info != 0) {
    out[0] = out[1] = out[2] = NAN;
    free(A);
    free(y);
    return info;
  }
  double logdet = 0.0;
  for (int64_t i = 0; i < n; ++i) logdet += log(A[i * n + i]);
  logdet *= 2.0;
  oracle_forward_solve(n, A, Z, y);
  double quad = 0.0;
  for (int64_t i = 0; i < n; ++i) quad += y[i] * y[i];
  out[0] = -0.5 * (double)n * ORACLE_LN_2PI - 0.5 * logdet - 0.5 * quad;
  out[1] = logdet;
  out[2] = quad;
  free(A);
  free(y);
  return 0;
}

/* Log-likelihood and its gradient with respect to (sigma^2, beta, nu).
 *   a = Sigma^-1 Z = L^-T L^-1 Z
 *   X = L^-1 (solve L X = I), Sigma^-1 = X^T X
 *   g_k = 1/2 a^T D_k a - 1/2 sum_ij (Sigma^-1)_ij (D_k)_ij
 * out = {l, log|Sigma|, quad}.  Returns as oracle_loglik.                  */
int64_t oracle_loglik_grad(int64_t n, const double* locs, const double* Z, const double theta[3], double out[3],
                           double grad[3]) {
  const size_t nn = (size_t)n * (size_t)n;
  double* A = (double*)malloc(nn * sizeof(double));
  double* X = (double*)calloc(nn, sizeof(double));
  double* Si = (double*)calloc(nn, sizeof(double));
  double* D = (double*)malloc(3 * nn * sizeof(double));
  double* y = (double*)malloc((size_t)n * sizeof(double));
  double* a = (double*)malloc((size_t)n * sizeof(double));
  int64_t info = -1;
  if (!A || !X || !Si || !D || !y || !a) goto done;
  oracle_covariance(n, locs, theta, A);
  info = oracle_cholesky(n, A);
  if (info != 0) {
    out[0] = out[1] = out[2] = NAN;
    grad[0] = grad[1] = grad[2] = NAN;
    goto done;
  }
  {
    double logdet = 0.0;
    for (int64_t i = 0; i < n; ++i) logdet += log(A[i * n + i]);
    logdet *= 2.0;
    oracle_forward_solve(n, A, Z, y);
    double quad = 0.0;
    for (int64_t i = 0; i < n; ++i) quad += y[i] * y[i];
    out[0] = -0.5 * (double)n * ORACLE_LN_2PI - 0.5 * logdet - 0.5 * quad;
    out[1] = logdet;
    out[2] = quad;
    oracle_backward_solve(n, A, y, a);
  }
  /* X = L^-1, one column at a time (forward substitution on e_c). */
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t c = 0; c < n; ++c) {
    for (int64_t i = c; i < n; ++i) {
      double t = (i == c) ? 1.0 : 0.0;
      for (int64_t k = c; k < i; ++k) t -= A[i * n + k] * X[k * n + c];
      X[i * n + c] = t / A[i * n + i];
    }
  }
  /* Sigma^-1 = X^T X: (Sigma^-1)_ij = sum_{k >= max(i,j)} X_ki X_kj. */
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j <= i; ++j) {
      double t = 0.0;
      for (int64_t k = i; k < n; ++k) t += X[k * n + i] * X[k * n + j];
      Si[i * n + j] = t;
      Si[j * n + i] = t;
    }
  }
  /* D_k, full symmetric. */
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j <= i; ++j) {
      double g[3];
      oracle_matern_grad(theta, oracle_dist(locs, i, j), g);
      for (int c = 0; c < 3; ++c) {
        D[c * nn + i * n + j] = g[c];
        D[c * nn + j * n + i] = g[c];
      }
    }
  }
  for (int c = 0; c < 3; ++c) {
    const double* Dc = D + c * nn;
    double quadform = 0.0, trace = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      double row = 0.0;
      for (int64_t j = 0; j < n; ++j) row += Dc[i * n + j] * a[j];
      quadform += a[i] * row;
    }
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) trace += Si[i * n + j] * Dc[i * n + j];
    grad[c] = 0.5 * quadform - 0.5 * trace;
  }
done:
  free(A);
  free(X);
  free(Si);
  free(D);
  free(y);
  free(a);
  return info;
}

/* Exact synthetic realisation (Section III, Example 1): Z = L eps with
 * Sigma(theta) = L L^T.  Returns 0 or the not-positive-definite pivot + 1. */
int64_t oracle_simulate(int64_t n, const double* locs, const double theta[3], const double* eps, double* Z) {
  double* A = (double*)malloc((size_t)n * (size_t)n * sizeof(double));
  if (!A) return -1;
  oracle_covariance(n, locs, theta, A);
  const int64_t info = oracle_cholesky(n, A);
  if (info == 0) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      double t = 0.0;
      for (int64_t k = 0; k <= i; ++k) t += A[i * n + k] * eps[k];
      Z[i] = t;
    }
  }
  free(A);
  return info;
}

/* Spatial prediction (kriging, the conditional expectation the paper's
 * exact_predict computes for the sea-surface-temperature tutorial of Section IV)
 * at m new locations from n observed ones, zero mean:
 *   mean_i = c_i^T Sigma^-1 Z,   var_i = sigma^2 - c_i^T Sigma^-1 c_i,
 *   c_i = (Sigma(new_i, obs_j))_j  (Eq. 3 at the cross distances).
 * Through the Cholesky factor: a = L^-T L^-1 Z, mean_i = c_i^T a;
 * w_i = L^-1 c_i, var_i = sigma^2 - w_i^T w_i.
 * Returns 0, or the not-positive-definite pivot + 1 (outputs NaN).          */
int64_t oracle_predict(int64_t n, const double* locs, const double* Z, const double theta[3], int64_t m,
                       const double* new_locs, double* mean, double* var) {
  double* A = (double*)malloc((size_t)n * (size_t)n * sizeof(double));
  double* y = (double*)malloc((size_t)n * sizeof(double));
  double* a = (double*)malloc((size_t)n * sizeof(double));
  if (!A || !y || !a) {
    free(A);
    free(y);
    free(a);
    return -1;
  }
  oracle_covariance(n, locs, theta, A);
  const int64_t info = oracle_cholesky(n, A);
  if (info != 0) {
    for (int64_t i = 0; i < m; ++i) mean[i] = var[i] = NAN;
  } else {
    oracle_forward_solve(n, A, Z, y);
    oracle_backward_solve(n, A, y, a);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < m; ++i) {
      double* c = (double*)malloc((size_t)n * sizeof(double));
      double* w = (double*)malloc((size_t)n * sizeof(double));
      for (int64_t j = 0; j < n; ++j)
        c[j] = oracle_matern(theta, oracle_dist_xy(new_locs[2 * i], new_locs[2 * i + 1], locs[2 * j], locs[2 * j + 1]));
      double mu = 0.0;
      for (int64_t j = 0; j < n; ++j) mu += c[j] * a[j];
      oracle_forward_solve(n, A, c, w);
      double ww = 0.0;
      for (int64_t j = 0; j < n; ++j) ww += w[j] * w[j];
      mean[i] = mu;
      var[i] = theta[0] - ww;
      free(c);
      free(w);
    }
  }
  free(A);
  free(y);
  free(a);
  return info;
}

/* Fisher information of theta = (sigma^2, beta, nu) for the zero-mean Gaussian
 * model (the paper's exact_fisher, listed with the package's functions in its
 * Appendix):  I_kl = 1/2 tr(Sigma^-1 D_k Sigma^-1 D_l),  D_k = dSigma/dtheta_k.
 * Sigma^-1 = X^T X with X = L^-1; M_k = Sigma^-1 D_k; I_kl = 1/2 sum_ij (M_k)_ij (M_l)_ji.
 * out: 3 x 3 row-major.  Returns 0, or the not-positive-definite pivot + 1 (NaN). */
int64_t oracle_fisher(int64_t n, const double* locs, const double theta[3], double out[9]) {
  const size_t nn = (size_t)n * (size_t)n;
  double* A = (double*)malloc(nn * sizeof(double));
  double* X = (double*)calloc(nn, sizeof(double));
  double* Si = (double*)calloc(nn, sizeof(double));
  double* D = (double*)malloc(3 * nn * sizeof(double));
  double* M = (double*)malloc(3 * nn * sizeof(double));
  int64_t info = -1;
  for (int c = 0; c < 9; ++c) out[c] = NAN;
  if (!A || !X || !Si || !D || !M) goto done;
  oracle_covariance(n, locs, theta, A);
  info = oracle_cholesky(n, A);
  if (info != 0) goto done;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t c = 0; c < n; ++c) {
    for (int64_t i = c; i < n; ++i) {
      double t = (i == c) ? 1.0 : 0.0;
      for (int64_t k = c; k < i; ++k) t -= A[i * n + k] * X[k * n + c];
      X[i * n + c] = t / A[i * n + i];
    }
  }
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j <= i; ++j) {
      double t = 0.0;
      for (int64_t k = i; k < n; ++k) t += X[k * n + i] * X[k * n + j];
      Si[i * n + j] = t;
      Si[j * n + i] = t;
    }
  }
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j <= i; ++j) {
      double g[3];
      oracle_matern_grad(theta, oracle_dist(locs, i, j), g);
      for (int c = 0; c < 3; ++c) {
        D[c * nn + i * n + j] = g[c];
        D[c * nn + j * n + i] = g[c];
      }
    }
  }
  /* M_k = Sigma^-1 D_k */
  for (int c = 0; c < 3; ++c) {
    const double* Dc = D + c * nn;
    double* Mc = M + c * nn;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t j = 0; j < n; ++j) {
        double t = 0.0;
        for (int64_t k = 0; k < n; ++k) t += Si[i * n + k] * Dc[k * n + j];
        Mc[i * n + j] = t;
      }
    }
  }
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) {
      const double* Mk = M + k * nn;
      const double* Ml = M + l * nn;
      double t = 0.0;
      for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) t += Mk[i * n + j] * Ml[j * n + i];
      out[k * 3 + l] = 0.5 * t;
    }
done:
  free(A);
  free(X);
  free(Si);
  free(D);
  free(M);
  return info;
}
