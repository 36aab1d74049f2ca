// C ABI entry points (include/exa.h): context, workspace and the stream-ordered
// drivers that chain the kernels of steps a1-a5.
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include <climits>
#include <string>

#include "ctx.cuh"
#include "exa_internal.cuh"
#include "util.cuh"

using namespace exa;

// ---------------------------------------------------------------------------
// context helpers
// ---------------------------------------------------------------------------
namespace exa {

exa_status set_err(exa_ctx* c, exa_status st, const char* fmt, ...) {
  if (!c) return st;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(c->err, sizeof(c->err), fmt, ap);
  va_end(ap);
  return st;
}

exa_status cuda_err(exa_ctx* c, cudaError_t e, const char* what) {
  return set_err(c, EXA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Grow-only device buffer with the context's memory bound enforced.
exa_status ensure(exa_ctx* c, DevBuf& b, size_t bytes, const char* name) {
  if (bytes <= b.bytes) return EXA_OK;
  const size_t held = c->held_bytes - b.bytes;
  if (c->ws_limit && held + bytes > c->ws_limit)
    return set_err(c, EXA_ERR_NOMEM, "workspace %s needs %zu bytes; context bound is %zu (held %zu)", name, bytes,
                   c->ws_limit, held);
  if (b.p) {
    cudaStreamSynchronize(c->stream);
    cudaFree(b.p);
    c->held_bytes -= b.bytes;
    b.p = nullptr;
    b.bytes = 0;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, EXA_ERR_NOMEM, "cudaMalloc(%zu) for %s: %s", bytes, name, cudaGetErrorString(e));
  }
  b.p = p;
  b.bytes = bytes;
  c->held_bytes += bytes;
  return EXA_OK;
}

static void free_buf(exa_ctx* c, DevBuf& b) {
  if (b.p) cudaFree(b.p);
  c->held_bytes -= b.bytes;
  b.p = nullptr;
  b.bytes = 0;
}

exa_status check_theta(exa_ctx* c, const double theta[3]) {
  if (!theta) return set_err(c, EXA_ERR_ARG, "theta is NULL");
  for (int i = 0; i < 3; ++i)
    if (!(theta[i] > 0.0) || !isfinite(theta[i]))
      return set_err(c, EXA_ERR_ARG, "theta[%d] = %g must be finite and > 0", i, theta[i]);
  return EXA_OK;
}

exa_status reset_status(exa_ctx* c) {
  DevStatus init;
  memset(&init, 0, sizeof(init));
  init.pivot = LLONG_MAX;
  *c->h_status = init;
  cudaError_t e = cudaMemcpyAsync(c->d_status, c->h_status, sizeof(DevStatus), cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "status reset");
  return EXA_OK;
}

// FP64 factorisation of the padded workspace matrix (npad multiple of nb).
exa_status factor_fp64(exa_ctx* c, double* a, int64_t ld, int64_t npad, int nb) {
  const int T = (int)(npad / nb);
  exa_status st;
  if ((st = ensure(c, c->w_all, (size_t)T * nb * nb * sizeof(double), "inverted diagonal tiles")) != EXA_OK) return st;
  if ((st = ensure(c, c->panel, (size_t)npad * nb * sizeof(double), "panel")) != EXA_OK) return st;
  if ((st = ensure(c, c->logdet_part, (size_t)T * sizeof(double), "log-det partials")) != EXA_OK) return st;
  double* W = (double*)c->w_all.p;
  double* P = (double*)c->panel.p;
  double* LD = (double*)c->logdet_part.p;
  for (int k = 0; k < T; ++k) {
    const int64_t k0 = (int64_t)k * nb;
    const int64_t m = npad - k0 - nb;
    const double dnb = nb, dm = (double)m;
    cudaError_t e;
    {
      ProfScope ps(c, PK_POTRF, dnb * dnb * dnb, 24.0 * dnb * dnb);
      e = launch_potrf_diag(c->stream, a, ld, k0, nb, W, LD, c->d_status);
    }
    if (e == cudaSuccess && m > 0) {
      ProfScope ps(c, PK_TRSM64, 2.0 * dm * dnb * dnb, 24.0 * dm * dnb);
      e = launch_trsm_panel(c->stream, a, ld, k0, nb, m, W, P, c->d_status);
    }
    if (e == cudaSuccess && m > 0) {
      ProfScope ps(c, PK_SYRK64, dm * (dm + 64.0) * dnb, 8.0 * dm * (dm + 64.0) + 8.0 * dm * dnb);
      e = launch_syrk_update(c->stream, a, ld, k0 + nb, m, nb, P, c->d_status);
    }
    if (e != cudaSuccess) return cuda_err(c, e, "cholesky launch");
  }
  return EXA_OK;
}

void model_params(const exa_ctx* c, const double theta[3], MaternParams* P) {
  matern_params(theta, P);
  P->nugget = c->nugget;
  P->metric = c->metric;
  P->radius = c->radius;
}

exa_status matern_table(exa_ctx* c, const MaternParams& P, const MaternTable** tab) {
  const size_t bytes = sizeof(MaternTable) + (size_t)kTabSeg * (kTabDeg + 1) * sizeof(double) + 256;
  exa_status st = ensure(c, c->table, bytes, "interpolation table");
  if (st != EXA_OK) return st;
  MaternTable* t = (MaternTable*)c->table.p;
  double* nodes = (double*)((char*)c->table.p + ((sizeof(MaternTable) + 255) / 256) * 256);
  cudaError_t e;
  {
    ProfScope ps(c, PK_GEN, 0.0, 0.0, 2);
    e = launch_matern_table(c->stream, P, t, nodes);
  }
  if (e != cudaSuccess) return cuda_err(c, e, "table build");
  *tab = t;
  return EXA_OK;
}

// Read the device status after a synchronise; map a failed pivot to NOT_SPD.
exa_status read_status(exa_ctx* c) {
  cudaError_t e = cudaMemcpyAsync(c->h_status, c->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "status read");
  if (c->h_status->timeout) {
    return set_err(c, EXA_ERR_TIMEOUT, "device wait gave up (site %d)", c->h_status->timeout_where);
  }
  if (c->h_status->info) {
    c->last_pivot = c->h_status->pivot;
    return set_err(c, EXA_ERR_NOT_SPD, "Cholesky pivot %lld is not positive: Sigma(theta) is not numerically SPD",
                   (long long)c->h_status->pivot);
  }
  return EXA_OK;
}

}  // namespace exa

// ---------------------------------------------------------------------------
// exported entry points
// ---------------------------------------------------------------------------
extern "C" {

exa_status exa_ctx_set_model(exa_ctx* c, double nugget, int metric, double radius) {
  if (!c) return EXA_ERR_ARG;
  if (!(nugget >= 0.0) || !isfinite(nugget) || (metric != 0 && metric != 1) || !(radius >= 0.0) || !isfinite(radius))
    return set_err(c, EXA_ERR_ARG, "bad model options (nugget %g, metric %d, radius %g)", nugget, metric, radius);
  c->nugget = nugget;
  c->metric = metric;
  c->radius = radius > 0.0 ? radius : 6371.0;
  return EXA_OK;
}

exa_status exa_ctx_create(exa_ctx** out, void* cuda_stream, size_t workspace_bytes, int tile_nb) {
  if (!out) return EXA_ERR_ARG;
  *out = nullptr;
  if (tile_nb != 0 && tile_nb != 64 && tile_nb != 128) return EXA_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return EXA_ERR_CUDA;
  }
  exa_ctx* c = new exa_ctx();
  c->device = dev;
  c->stream = (cudaStream_t)cuda_stream;
  c->ws_limit = workspace_bytes;
  c->tile_nb = tile_nb ? tile_nb : 128;
  c->last_pivot = -1;
  c->err[0] = 0;
  if (cudaMalloc(&c->d_status, sizeof(DevStatus)) != cudaSuccess ||
      cudaMalloc(&c->d_scalars, 64 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&c->h_status, sizeof(DevStatus)) != cudaSuccess ||
      cudaMallocHost(&c->h_scalars, 64 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    exa_ctx_destroy(c);
    return EXA_ERR_CUDA;
  }
  for (int i = 0; i < kNumEvents; ++i) cudaEventCreate(&c->ev[i]);
  *out = c;
  return EXA_OK;
}

void exa_ctx_destroy(exa_ctx* c) {
  if (!c) return;
  if (c->stream || true) cudaStreamSynchronize(c->stream);
  free_buf(c, c->mat);
  free_buf(c, c->w_all);
  free_buf(c, c->panel);
  free_buf(c, c->logdet_part);
  free_buf(c, c->vec);
  free_buf(c, c->partial);
  free_buf(c, c->table);
  release_extra(c);
  release_batched(c);
  prof_release(c);
  if (c->d_status) cudaFree(c->d_status);
  if (c->d_scalars) cudaFree(c->d_scalars);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->h_scalars) cudaFreeHost(c->h_scalars);
  for (int i = 0; i < kNumEvents; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  delete c;
}

exa_status exa_ctx_set_stream(exa_ctx* c, void* cuda_stream) {
  if (!c) return EXA_ERR_ARG;
  c->stream = (cudaStream_t)cuda_stream;
  return EXA_OK;
}

exa_status exa_ctx_set_mixed_band(exa_ctx* c, int band) {
  if (!c) return EXA_ERR_ARG;
  c->mixed_band = band;
  return EXA_OK;
}

exa_status exa_ctx_set_lookahead(exa_ctx* c, int sms) {
  if (!c || sms < 0 || sms > 128) return EXA_ERR_ARG;
  c->lookahead_sms = sms;
  return EXA_OK;
}

exa_status exa_ctx_set_panel_fusion(exa_ctx* c, int64_t min_rows) {
  if (!c) return EXA_ERR_ARG;
  c->fuse_min_rows = min_rows < 0 ? -1 : min_rows;
  return EXA_OK;
}

const char* exa_last_error(const exa_ctx* c) { return c ? c->err : "null context"; }

int64_t exa_last_pivot(const exa_ctx* c) { return c ? c->last_pivot : -1; }

size_t exa_workspace_bytes(const exa_ctx* c) { return c ? c->held_bytes : 0; }

exa_status exa_covariance(exa_ctx* c, const double* d_locs, int64_t n, const double theta[3], double* d_sigma,
                          int64_t ld) {
  if (!c) return EXA_ERR_ARG;
  c->err[0] = 0;
  if (n < 1 || !d_locs || !d_sigma || ld < n) return set_err(c, EXA_ERR_ARG, "bad n / pointers / ld");
  exa_status st = check_theta(c, theta);
  if (st != EXA_OK) return st;
  MaternParams P;
  model_params(c, theta, &P);
  const MaternTable* tab = nullptr;
  if ((st = matern_table(c, P, &tab)) != EXA_OK) return st;
  cudaError_t e = launch_matern_gen(c->stream, d_locs, n, n, P, d_sigma, ld, nullptr, tab);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "covariance generation");
  return EXA_OK;
}

exa_status exa_potrf(exa_ctx* c, double* d_a, int64_t n, int64_t ld) {
  if (!c) return EXA_ERR_ARG;
  c->err[0] = 0;
  c->last_pivot = -1;
  if (n < 1 || !d_a || ld < n) return set_err(c, EXA_ERR_ARG, "bad n / pointer / ld");
  const int nb = c->tile_nb;
  const int64_t npad = round_up(n, nb);
  exa_status st = ensure(c, c->mat, (size_t)npad * npad * sizeof(double), "matrix");
  if (st != EXA_OK) return st;
  if ((st = reset_status(c)) != EXA_OK) return st;
  double* A = (double*)c->mat.p;
  cudaError_t e = launch_copy_lower_pad(c->stream, d_a, ld, n, npad, A, npad);
  if (e != cudaSuccess) return cuda_err(c, e, "pad copy");
  if ((st = factor_fp64(c, A, npad, npad, nb)) != EXA_OK) return st;
  st = read_status(c);
  if (st != EXA_OK) return st;
  e = launch_copy_lower_back(c->stream, A, npad, n, d_a, ld);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "copy back");
  return EXA_OK;
}

exa_status exa_loglik_ex(exa_ctx* c, const double* d_locs, const double* d_z, const double theta[3], int64_t n,
                         exa_prec prec, exa_result* out) {
  if (!c) return EXA_ERR_ARG;
  c->err[0] = 0;
  c->last_pivot = -1;
  if (!out) return set_err(c, EXA_ERR_ARG, "out is NULL");
  memset(out, 0, sizeof(*out));
  out->loglik = out->logdet = out->quad = NAN;
  if (n < 1 || !d_locs || !d_z) return set_err(c, EXA_ERR_ARG, "bad n or NULL device pointer");
  exa_status st = check_theta(c, theta);
  if (st != EXA_OK) return st;
  if (prec == EXA_FP64 || prec == EXA_MIXED_TF32X3 || prec == EXA_MIXED_BF16X3) {
    st = prec == EXA_FP64 ? loglik_fp64(c, d_locs, d_z, theta, n, out, nullptr)
                          : loglik_mixed(c, d_locs, d_z, theta, n, prec, out);
    prof_fold(c);  // the evaluation ended with a synchronise: recycle its timing events
    return st;
  }
  if (prec == EXA_MIXED_FP32)
    return set_err(c, EXA_ERR_ARG,
                   "EXA_MIXED_FP32 is offered by exa_loglik_batched only: on one field its FP32 FFMA tile "
                   "products run at a third of the TF32x3 tensor-core rate with fewer significant bits; use "
                   "EXA_MIXED_TF32X3");
  return set_err(c, EXA_ERR_ARG, "unknown precision %d", (int)prec);
}

exa_status exa_loglik(exa_ctx* c, const double* d_locs, const double* d_z, const double theta[3], int64_t n,
                      exa_prec prec, double* loglik) {
  if (!loglik) return c ? set_err(c, EXA_ERR_ARG, "loglik is NULL") : EXA_ERR_ARG;
  exa_result r;
  exa_status st = exa_loglik_ex(c, d_locs, d_z, theta, n, prec, &r);
  *loglik = r.loglik;
  return st;
}

}  // extern "C"

namespace exa {

// Steps a1-a5 in FP64.  If `keep` is non-null the factor stays in c->mat and the
// solve vector y = L^-1 z in the returned pointer (used by the gradient).
exa_status loglik_fp64(exa_ctx* c, const double* d_locs, const double* d_z, const double theta[3], int64_t n,
                       exa_result* out, double** keep_y) {
  const int nb = c->tile_nb;
  const int64_t npad = round_up(n, nb);
  const int T = (int)(npad / nb);
  exa_status st;
  if ((st = ensure(c, c->mat, (size_t)npad * npad * sizeof(double), "matrix")) != EXA_OK) return st;
  if ((st = ensure(c, c->vec, (size_t)3 * npad * sizeof(double), "vectors")) != EXA_OK) return st;
  if ((st = ensure(c, c->partial, (size_t)(kPartialDoubles(npad, nb)) * sizeof(double), "partials")) != EXA_OK)
    return st;
  if ((st = reset_status(c)) != EXA_OK) return st;
  double* A = (double*)c->mat.p;
  double* zw = (double*)c->vec.p;  // working right-hand side
  double* y = zw + npad;           // L^-1 z
  double* tmp = y + npad;
  double* part = (double*)c->partial.p;
  MaternParams P;
  model_params(c, theta, &P);
  cudaEventRecord(c->ev[0], c->stream);
  const MaternTable* tab = nullptr;
  if ((st = matern_table(c, P, &tab)) != EXA_OK) return st;
  cudaError_t e;
  {
    ProfScope ps(c, PK_GEN, 0.0, 4.0 * (double)npad * (double)(npad + 1));
    e = launch_matern_gen(c->stream, d_locs, n, npad, P, A, npad, nullptr, tab);
  }
  if (e != cudaSuccess) return cuda_err(c, e, "generation launch");
  cudaEventRecord(c->ev[1], c->stream);
  if ((st = factor_fp64(c, A, npad, npad, nb)) != EXA_OK) return st;
  cudaEventRecord(c->ev[2], c->stream);
  {
    ProfScope ps(c, PK_OTHER, 0.0, 16.0 * (double)npad);
    e = launch_pad_vector(c->stream, d_z, n, npad, zw);
  }
  for (int k = 0; k < T && e == cudaSuccess; ++k) {
    ProfScope ps(c, PK_TRSV, 2.0 * (double)(npad - (int64_t)k * nb) * nb, 8.0 * (double)(npad - (int64_t)k * nb) * nb);
    e = launch_trsv_fwd_step(c->stream, A, npad, npad, nb, k, (const double*)c->w_all.p, y, zw, c->d_status);
  }
  if (e == cudaSuccess) {
    ProfScope ps(c, PK_OTHER, 0.0, 8.0 * (double)npad, 4);
    e = launch_sumsq(c->stream, y, npad, part, c->d_scalars + 0);
    if (e == cudaSuccess)
      e = launch_sum(c->stream, (const double*)c->logdet_part.p, T, part + kRedPartials, c->d_scalars + 1);
  }
  if (e != cudaSuccess) return cuda_err(c, e, "solve launch");
  cudaEventRecord(c->ev[3], c->stream);
  e = cudaMemcpyAsync(c->h_scalars, c->d_scalars, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_err(c, e, "result copy");
  st = read_status(c);  // synchronises
  out->tile_nb = nb;
  cudaEventElapsedTime(&out->ms_gen, c->ev[0], c->ev[1]);
  cudaEventElapsedTime(&out->ms_chol, c->ev[1], c->ev[2]);
  cudaEventElapsedTime(&out->ms_solve, c->ev[2], c->ev[3]);
  cudaEventElapsedTime(&out->ms_total, c->ev[0], c->ev[3]);
  if (st != EXA_OK) return st;
  const double quad = c->h_scalars[0];
  const double logdet = 2.0 * c->h_scalars[1];
  out->quad = quad;
  out->logdet = logdet;
  out->loglik = -0.5 * (double)n * 1.8378770664093454836 - 0.5 * logdet - 0.5 * quad;
  // Sigma passed every pivot, so L^-1 is finite: a non-finite y^T y comes from z itself
  if (!isfinite(quad))
    return set_err(c, EXA_ERR_ARG, "z^T Sigma^-1 z = %g: z holds a non-finite entry (or its squares overflow)", quad);
  if (keep_y) *keep_y = y;
  return EXA_OK;
}

}  // namespace exa

extern "C" exa_status exa_simulate(exa_ctx* c, const double* d_locs, const double* d_eps, const double theta[3],
                                   int64_t n, exa_prec prec, double* d_z) {
  if (!c) return EXA_ERR_ARG;
  c->err[0] = 0;
  c->last_pivot = -1;
  if (n < 1 || !d_locs || !d_eps || !d_z) return set_err(c, EXA_ERR_ARG, "bad n or NULL device pointer");
  if (prec != EXA_FP64 && prec != EXA_MIXED_TF32X3) return set_err(c, EXA_ERR_ARG, "unsupported precision");
  exa_status st = check_theta(c, theta);
  if (st != EXA_OK) return st;
  const int nb = c->tile_nb;
  const int64_t npad = round_up(n, prec == EXA_FP64 ? nb : kMixPanel);
  if ((st = ensure(c, c->mat, (size_t)npad * npad * sizeof(double), "matrix")) != EXA_OK) return st;
  if ((st = reset_status(c)) != EXA_OK) return st;
  double* A = (double*)c->mat.p;
  cudaError_t e = cudaSuccess;
  if (prec == EXA_FP64) {
    MaternParams P;
    model_params(c, theta, &P);
    const MaternTable* tab = nullptr;
    if ((st = matern_table(c, P, &tab)) != EXA_OK) return st;
    e = launch_matern_gen(c->stream, d_locs, n, npad, P, A, npad, nullptr, tab);
    if (e != cudaSuccess) return cuda_err(c, e, "generation launch");
    if ((st = factor_fp64(c, A, npad, npad, nb)) != EXA_OK) return st;
  } else {
    if ((st = mixed_generate_factor(c, d_locs, n, theta, npad, prec, nullptr, nullptr)) != EXA_OK) return st;
  }
  e = launch_trmv_lower(c->stream, A, npad, n, d_eps, d_z, c->d_status);
  if (e != cudaSuccess) return cuda_err(c, e, "trmv launch");
  return read_status(c);
}
