// Mixed-precision driver (Section II-A, Fig. 1(d): diagonal tiles in double
// precision, off-diagonal tiles in reduced precision) and the component entry
// point for the tensor-core products.
#include <math.h>
#include <string.h>

#include "ctx.cuh"
#include "gemm_tc.cuh"
#include "util.cuh"

namespace exa {

exa_status ensure_split(exa_ctx* c, SplitOperand& op, DevBuf& buf, int64_t rows, int K, bool t3, bool oz) {
  const size_t t3_bytes = t3 ? (size_t)rows * K * 4 : 0;
  const size_t dig_bytes = oz ? (size_t)kOzSlices * rows * K * 2 : 0;
  const size_t ex_bytes = oz ? (size_t)round_up(rows, 64) * 4 : 0;
  const size_t total = 2 * t3_bytes + dig_bytes + ex_bytes + 1024;
  void* old = buf.p;
  exa_status st = ensure(c, buf, total, "split operands");
  if (st != EXA_OK) return st;
  const bool same = (old == buf.p) && op.rows == rows && op.K == K && ((op.hi != nullptr) == t3) &&
                    ((op.dig != nullptr) == oz);
  if (same) return EXA_OK;
  uint8_t* base = (uint8_t*)buf.p;
  op.rows = rows;
  op.K = K;
  op.hi = t3 ? (float*)base : nullptr;
  op.lo = t3 ? (float*)(base + t3_bytes) : nullptr;
  op.dig = oz ? (void*)(base + 2 * t3_bytes) : nullptr;
  op.ex = oz ? (int*)(base + 2 * t3_bytes + dig_bytes) : nullptr;
  cudaError_t e = make_split_maps(op);
  if (e != cudaSuccess) {
    op.rows = 0;
    return cuda_err(c, e, "tensor map encode");
  }
  return EXA_OK;
}

}  // namespace exa

using namespace exa;

extern "C" exa_status exa_gemm_update(exa_ctx* c, exa_gemm_kind kind, int64_t m, int64_t n, int64_t k,
                                      const double* d_a, const double* d_b, double* d_c, int64_t ldc, int store) {
  if (!c) return EXA_ERR_ARG;
  c->err[0] = 0;
  if (!d_a || !d_b || !d_c || m <= 0 || n <= 0 || k <= 0 || ldc < m)
    return set_err(c, EXA_ERR_ARG, "bad gemm arguments");
  const bool oz = (kind == EXA_GEMM_OZ);
  if (kind != EXA_GEMM_T3 && kind != EXA_GEMM_OZ) return set_err(c, EXA_ERR_ARG, "unknown gemm kind");
  if (m % 128 || k % 64 || k > kSplitMaxK || (oz ? (n % 32 || k > 256) : (n % 128)))
    return set_err(c, EXA_ERR_ARG, "gemm shape m=%lld n=%lld k=%lld not supported", (long long)m, (long long)n,
                   (long long)k);
  exa_status st;
  if ((st = ensure_split(c, c->sp_a, c->mx_split, m, (int)k, !oz, oz)) != EXA_OK) return st;
  if ((st = ensure_split(c, c->sp_b, c->mx_split_b, n, (int)k, !oz, oz)) != EXA_OK) return st;
  if ((st = reset_status(c)) != EXA_OK) return st;
  cudaError_t e = launch_split_rows(c->stream, d_a, k, 1, (int)m, (int)k, c->sp_a, 0);
  if (e == cudaSuccess) e = launch_split_rows(c->stream, d_b, k, 1, (int)n, (int)k, c->sp_b, 0);
  if (e != cudaSuccess) return cuda_err(c, e, "split launch");
  GemmArgs g;
  memset(&g, 0, sizeof(g));
  g.C = d_c;
  g.ldc = ldc;
  g.K = (int)k;
  g.enum_mode = kEnumFull;
  g.store = store ? 1 : 0;
  g.st = c->d_status;
  if (oz) {
    g.nt = (int)(n / 32);
    g.ntiles = (m / 128) * (n / 32);
    e = launch_gemm_oz(c->stream, c->sp_a, c->sp_b, g);
  } else {
    g.nt = (int)(n / 128);
    g.ntiles = (m / 128) * (n / 128);
    e = launch_gemm_t3(c->stream, c->sp_a, c->sp_b, g);
  }
  if (e != cudaSuccess) return cuda_err(c, e, "gemm launch");
  return read_status(c);
}
