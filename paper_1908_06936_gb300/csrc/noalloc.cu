// Allocation-free FP64 log-likelihood for small problems.
//
// Some callers cannot call cudaMalloc: a host application whose memory pool
// owns all device memory and forbids other allocators, or a latency-critical
// path where the implicit device-wide synchronisation of cudaMalloc/cudaFree
// is not acceptable.  exa_loglik_noalloc serves them with the same kernels as
// exa_loglik (FP64 generation, DMMA tiled Cholesky, log-determinant, solve),
// all of whose workspace lives in one file-scope __device__ array sized for
// n <= kNoAllocMaxN.  Every GPU that loads the library holds that array
// (about 36 MiB) until the process exits.
//
// The array's host-side name is only a stand-in for the device object, so the
// host looks its device address up with cudaGetSymbolAddress once per device
// (on the first call on that device) and passes the pointer to the kernels.
#include <math.h>
#include <string.h>

#include <climits>
#include <mutex>

#include "ctx.cuh"
#include "util.cuh"

namespace exa {

constexpr int64_t kNoAllocMaxN = 2048;  // largest problem accepted
constexpr int kNoAllocNb = 128;         // FP64 tile
constexpr int64_t kNoAllocT = kNoAllocMaxN / kNoAllocNb;

struct NoAllocScratch {
  double a[kNoAllocMaxN * kNoAllocMaxN];            // padded covariance / factor
  double w[kNoAllocT * kNoAllocNb * kNoAllocNb];    // inverted diagonal tiles
  double panel[kNoAllocMaxN * kNoAllocNb];          // row-major panel copy
  double vec[3 * kNoAllocMaxN];                     // right-hand side, solution
  double partial[2 * kRedPartials + (kNoAllocMaxN / 1024 + 2) * kNoAllocNb];
  double logdet_part[kNoAllocT];
  double scal[4];
  DevStatus st;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

static std::mutex g_noalloc_mu;
static NoAllocScratch* g_noalloc_ptr[128] = {};

__global__ void noalloc_status_init(DevStatus* st) {
  st->info = 0;
  st->pad = 0;
  st->pivot = LLONG_MAX;
  st->timeout = 0;
  st->timeout_where = 0;
}

// Device address of the scratch array on the current device (looked up once).
static NoAllocScratch* noalloc_scratch() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return nullptr;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    NoAllocScratch* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_noalloc_ptr[dev] = p;
  }
  return g_noalloc_ptr[dev];
}

}  // namespace exa

using namespace exa;

extern "C" exa_status exa_loglik_noalloc(void* cuda_stream, const double* d_locs, const double* d_z,
                                         const double theta[3], int64_t n, double* loglik) {
  if (!loglik) return EXA_ERR_ARG;
  *loglik = NAN;
  if (!d_locs || !d_z || !theta || n < 1 || n > kNoAllocMaxN) return EXA_ERR_ARG;
  for (int i = 0; i < 3; ++i)
    if (!(theta[i] > 0.0) || !isfinite(theta[i])) return EXA_ERR_ARG;
  NoAllocScratch* S = noalloc_scratch();
  if (!S) return EXA_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int nb = kNoAllocNb;
  const int64_t npad = round_up(n, nb);
  const int T = (int)(npad / nb);
  double* A = S->a;
  DevStatus* st = &S->st;
  MaternParams P;
  matern_params(theta, &P);
  // the array keeps the previous call's contents: reset what must start from zero
  noalloc_status_init<<<1, 1, 0, s>>>(st);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_matern_gen(s, d_locs, n, npad, P, A, npad);
  for (int k = 0; k < T && e == cudaSuccess; ++k) {
    const int64_t k0 = (int64_t)k * nb, m = npad - k0 - nb;
    e = launch_potrf_diag(s, A, npad, k0, nb, S->w, S->logdet_part, st);
    if (e == cudaSuccess) e = launch_trsm_panel(s, A, npad, k0, nb, m, S->w, S->panel, st);
    if (e == cudaSuccess) e = launch_syrk_update(s, A, npad, k0 + nb, m, nb, S->panel, st);
  }
  double* zw = S->vec;
  double* y = S->vec + npad;
  if (e == cudaSuccess) e = launch_pad_vector(s, d_z, n, npad, zw);
  for (int k = 0; k < T && e == cudaSuccess; ++k) e = launch_trsv_fwd_step(s, A, npad, npad, nb, k, S->w, y, zw, st);
  if (e == cudaSuccess) e = launch_sumsq(s, y, npad, S->partial, S->scal + 0);
  if (e == cudaSuccess) e = launch_sum(s, S->logdet_part, T, S->partial + kRedPartials, S->scal + 1);
  double h[2] = {0.0, 0.0};
  DevStatus hs;
  memset(&hs, 0, sizeof(hs));
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, S->scal, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return EXA_ERR_CUDA;
  }
  if (hs.info) return EXA_ERR_NOT_SPD;
  const double logdet = 2.0 * h[1];
  *loglik = -0.5 * (double)n * 1.8378770664093454836 - 0.5 * logdet - 0.5 * h[0];
  if (!isfinite(h[0])) return EXA_ERR_ARG;  // Sigma passed every pivot: z holds a non-finite entry
  return EXA_OK;
}
