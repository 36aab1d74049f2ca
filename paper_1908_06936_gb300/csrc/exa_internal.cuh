// Internal declarations shared by the CUDA translation units of libexa.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/exa.h"

namespace exa {

// One-time set-up per device (function attributes such as the dynamic shared-memory
// limit, and cached device properties, hold for the current device only): runs f()
// once per device id 0..63 with that device current, thread-safe; a failed f() is
// retried on the next call.  Ids beyond 63 run f() every time.
class PerDeviceOnce {
 public:
  template <class F>
  cudaError_t operator()(F&& f) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return f();
    const uint64_t bit = 1ull << dev;
    if (done_.load(std::memory_order_acquire) & bit) return cudaSuccess;
    std::lock_guard<std::mutex> lock(mu_);
    if (done_.load(std::memory_order_relaxed) & bit) return cudaSuccess;
    e = f();
    if (e == cudaSuccess) done_.fetch_or(bit, std::memory_order_release);
    return e;
  }

 private:
  std::atomic<uint64_t> done_{0};
  std::mutex mu_;
};

// A device property cached per device (ids 0..63; beyond that, queried every call).
template <class F>
int per_device_int(std::atomic<int> (&cache)[64], F&& query) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return query();
  if (dev < 0 || dev >= 64) return query();
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  v = query();
  if (v > 0) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

// ---------------------------------------------------------------------------
// Matérn generation parameters (one per theta), computed on the host.
// Eq. 3 is evaluated as  Sigma = sigma^2 * exp(logc + nu ln x) * K_nu(x),
// logc = (1 - nu) ln 2 - ln Gamma(nu),  x = r / beta.
// K_nu is reached from K_mu, K_{mu+1} (mu = nu - N, N = round(nu), |mu| <= 1/2)
// by the forward recurrence K_{a+1} = K_{a-1} + (2a/x) K_a (DLMF 10.29.1).
// K_mu, K_{mu+1} come from
//   x <= 2: Temme's power series (N. M. Temme, J. Comput. Phys. 19, 1975),
//   x >  2: the three-term recurrence of z_k = U(mu + 1/2 + k, 2 mu + 1, 2x)
//           (DLMF 13.3.7) run backward from depth D(x) (Miller's algorithm),
//           normalised by sum_k C_k z_k = (2x)^(-mu-1/2) (the identity behind
//           the Thompson-Barnett / Steed CF2 method), with
//           K_mu(x) = sqrt(pi) (2x)^mu e^-x z_0 (DLMF 13.18.9).
// Per-theta constant tables remove every division from the inner loops.
// ---------------------------------------------------------------------------
constexpr int kTemmeTerms = 40;   // series terms kept in the tables
constexpr int kMillerMax = 96;    // deepest backward recurrence (x just above 2)

struct MaternParams {
  double sigma2, beta, nu;
  double ib2;        // 1 / beta^2
  double nugget;     // tau^2 added to the diagonal (0: none)
  double radius;     // sphere radius of the great-circle metric
  int metric;        // 0: Euclidean (x, y); 1: great circle between (longitude, latitude) in degrees
  int pad2_;
  double logc;       // (1 - nu) ln 2 - lgamma(nu)
  double mu;         // nu - N, in [-1/2, 1/2]
  int N;             // round(nu)
  int pad_;
  // Temme series at order mu
  double mupi_sin;   // mu pi / sin(mu pi)  (1 at mu = 0)
  double gam1;       // Gamma_1(mu) = (1/Gamma(1-mu) - 1/Gamma(1+mu)) / (2 mu)
  double gam2;       // Gamma_2(mu) = (1/Gamma(1-mu) + 1/Gamma(1+mu)) / 2
  double gp;         // Gamma(1 + mu)
  double gm;         // Gamma(1 - mu)
  double t_k2[kTemmeTerms + 1];  // 1 / (k^2 - mu^2)
  double t_km[kTemmeTerms + 1];  // 1 / (k - mu)
  double t_kp[kTemmeTerms + 1];  // 1 / (k + mu)
  // backward recurrence at order mu
  double m_a[kMillerMax + 2];    // (k + 1/2)^2 - mu^2
  double m_c[kMillerMax + 2];    // C_k,  C_0 = 1,  C_{k+1} = C_k ((k + 1/2)^2 - mu^2) / (k + 1)
};

// Host: fill the parameter block for theta (defined in matern.cu).
void matern_params(const double theta[3], MaternParams* p);

// Per-theta interpolation table of f(s) = Sigma (sigma^2 included) as a function of s = (r / beta)^2,
// so that an entry costs no square root, division or exponential.  Segments follow the
// binary exponent of s: octave [2^e, 2^(e+1)), e in [kTabE0, kTabE0 + kTabOct), split into
// kTabSub equal pieces; on each, f is a degree-kTabDeg polynomial in t = (s - centre) /
// half-width (Chebyshev interpolation on pieces 1/64 of an octave wide: the truncation
// error is below 1e-15 relative for x < 32 and about 1e-14 relative in the last octave,
// 45 <= x < 64, where f < 1e-18).  Below 2^kTabE0 (x < 1/16) and from
// 2^(kTabE0 + kTabOct) on (x >= 64) the exact routine applies.
constexpr int kTabE0 = -8;
constexpr int kTabOct = 20;
constexpr int kTabSubBits = 6;
constexpr int kTabSub = 1 << kTabSubBits;
constexpr int kTabSeg = kTabOct * kTabSub;
constexpr int kTabDeg = 8;
struct MaternTable {
  double mc[kTabSeg];                  // -centre / half-width
  double ih[kTabSeg];                  // 1 / half-width
  double a[kTabSeg][kTabDeg + 1];      // monomial coefficients in t
};
// Build the table for one theta (two small kernels) into device memory.
cudaError_t launch_matern_table(cudaStream_t s, const MaternParams& p, MaternTable* tab, double* nodes);

// Device status block (lives in device memory, one per context).
struct DevStatus {
  int32_t info;        // 0 ok; 1 not SPD
  int32_t pad;
  long long pivot;     // smallest failing global row (atomicMin), or LLONG_MAX
  int32_t timeout;     // bounded wait expired
  int32_t timeout_where;
};

// ---------------------------------------------------------------------------
// Kernel launchers (all asynchronous on `s`).
// ---------------------------------------------------------------------------

// Lower triangle (diagonal included) of Sigma for rows/cols < n into column-major
// `a` (leading dim ld).  Rows/cols in [n, npad) are filled as the identity so
// that a padded matrix factors as diag(L, I).
// If offmax is non-null, offmax[d] receives (as the bits of a non-negative double)
// the largest off-diagonal |Sigma_ij| over `panel`-wide tile pairs (I, J) with I - J = d.
// With tab != nullptr the entries with x >= 2^kTabE0 come from the table.  With a2 != nullptr
// every entry is stored at the same place in a2 as well (two copies for one evaluation).
cudaError_t launch_matern_gen(cudaStream_t s, const double* locs, int64_t n, int64_t npad, const MaternParams& p,
                              double* a, int64_t ld, unsigned long long* offmax = nullptr,
                              const MaternTable* tab = nullptr, int panel = 256, double* a2 = nullptr);
// One diagonal tile of a batched factorisation: FP64 Cholesky of the 128 x 128 tile at (k0, k0) of a
// (column-major, ld), its log sum to *logdet and its inverse (row-major) to w; failures to *st.
struct DiagTileTask {
  double* a;
  int64_t ld, k0;
  double* logdet;
  double* w;
  DevStatus* st;
};
cudaError_t launch_potrf128_tasks(cudaStream_t s, const DiagTileTask* d_tasks, int ntasks);
// FP64 Cholesky and inverse of the 512 x 512 diagonal block at (k0, k0) as one cooperative launch
// of `grid` CTAs (>= 2): L in place, log sums of the four 128 sub-tiles into logdet_part[0..3], their
// inverses (row-major) into w_sub, the block inverse (row-major) into w2; scratch holds
// diag_block_scratch_doubles() doubles.
size_t diag_block_scratch_doubles();
cudaError_t launch_diag_block(cudaStream_t s, double* a, int64_t ld, int64_t k0, double* w_sub, double* logdet_part,
                              double* w2, double* scratch, DevStatus* st, int grid);

// FP64 tiled Cholesky steps (tile nb <= 128, multiple of 64; n multiple of nb).
// The triangular-solve steps accept nb <= 256.
cudaError_t launch_potrf_diag(cudaStream_t s, double* a, int64_t ld, int64_t k0, int nb, double* w_out,
                              double* logdet_part, DevStatus* st);
cudaError_t launch_trsm_panel(cudaStream_t s, double* a, int64_t ld, int64_t k0, int nb, int64_t m,
                              const double* w, double* p, const DevStatus* st);
cudaError_t launch_syrk_update(cudaStream_t s, double* a, int64_t ld, int64_t r0, int64_t m, int nb,
                               const double* p, const DevStatus* st);

// Blocked forward solve y = L^-1 z using the stored inverted diagonal tiles
// w_all (T tiles of nb x nb, row-major).  z is overwritten by y (length npad).
cudaError_t launch_trsv_fwd_step(cudaStream_t s, const double* a, int64_t ld, int64_t npad, int nb, int k,
                                 const double* w_all, double* y, double* tmp, const DevStatus* st);
// Backward solve a = L^-T y (in place in y).
cudaError_t launch_trsv_bwd_step(cudaStream_t s, const double* a, int64_t ld, int64_t npad, int nb, int k,
                                 const double* w_all, double* y, double* tmp, const DevStatus* st);

// Deterministic reductions: out[0] = sum(v[i]^2) ; out[0] = sum(v[i]) over n values.
cudaError_t launch_sumsq(cudaStream_t s, const double* v, int64_t n, double* partial, double* out);
cudaError_t launch_sum(cudaStream_t s, const double* v, int64_t n, double* partial, double* out);

// Small strided FP64 DMMA product C = alpha A B^T + beta C (M, N, K multiples of 32).
cudaError_t launch_dgemm_nt_small(cudaStream_t s, int M, int N, int K, double alpha, const double* a, int64_t ar,
                                  int64_t ac, const double* b, int64_t br, int64_t bc, double beta, double* c,
                                  int64_t cr, int64_t cc, const DevStatus* st);
// Persistent forward + backward solve with 128-wide tiles: x = (L L^T)^-1 rhs.  The
// strictly upper off-diagonal tiles of a must hold L^T (launch_transpose_lower_to_upper).
// rhs_work (npad, overwritten) and flags (2 npad/128 + 1 ints) are scratch.
cudaError_t launch_llt_solve_persistent(cudaStream_t s, const double* a, int64_t ld, int64_t npad, const double* w,
                                        double* rhs_work, double* x, int* flags, DevStatus* st);
// Writes L^T into the strictly upper off-diagonal 128-tiles of a (npad % 128 == 0).
cudaError_t launch_transpose_lower_to_upper(cudaStream_t s, double* a, int64_t ld, int64_t npad);
// Refinement helpers.
// y = Sigma x from the lower triangle of Sigma (column-major, ld) in one pass over 128 x 128
// tiles (npad % 128 == 0); partials holds symv_tiled_partials(npad) doubles.  Fixed summation order.
int64_t symv_tiled_partials(int64_t npad);
cudaError_t launch_symv_lower_tiled(cudaStream_t s, const double* a, int64_t ld, int64_t npad, const double* x,
                                    double* y, double* partials);
cudaError_t launch_residual(cudaStream_t s, const double* z, const double* y, double* r, int64_t n);
cudaError_t launch_axpy(cudaStream_t s, double a, const double* x, double* y, int64_t n);
cudaError_t launch_dot(cudaStream_t s, const double* a, const double* b, int64_t n, double* partial, double* out);

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace exa
