// Batched evaluation of many independent replicate fields of uneven size (the
// replicate studies of Section III, Example 2, run as one device workload).
//
// Stream-ordered, graph-capturable sequence (no host synchronisation):
//   1. per-replicate Matérn constants from theta in device memory (so a captured
//      graph can be replayed with new parameters);
//   2. generation of every replicate's lower tiles in one launch;
//   3. ONE persistent launch that walks a work list of tile tasks
//        POTRF(r, k)    L_kk = chol(A_kk), W_k = L_kk^-1, log-det part
//        TRSM(r, i, k)  L_ik = A_ik W_k^T
//        UPDATE(r,i,j,k) A_ij -= L_ik L_jk^T
//      ordered by step k across replicates (a topological order of every
//      replicate's DAG).  CTAs claim tasks in list order; a task waits on
//      per-tile completion counters (bounded spin: on time-out the replicate
//      reports EXA_ERR_TIMEOUT and every CTA stops claiming work), runs on
//      FP64 DMMA, then bumps its tile's counter.  Since every dependency sits
//      earlier in the list and all CTAs are co-resident, the walk cannot
//      deadlock;
//   4. one CTA per replicate: blocked forward solve, log-det, quadratic form,
//      l = -n/2 log 2 pi - 1/2 log|Sigma| - 1/2 y^T y and the status.
#include <math.h>
#include <string.h>

#include <vector>

#include "bessel.cuh"
#include "ctx.cuh"

namespace exa {

enum : int { OP_POTRF = 0, OP_TRSM = 1, OP_UPDATE = 2, OP_STALL = 3 };

struct BTask {
  int r;
  short op, k;
  short i, j;
  short pad0, pad1;
};

struct BMeta {
  int64_t n, npad, T;
  int64_t mo;   // matrix offset (doubles)
  int64_t wo;   // inverse-tile offset (doubles)
  int64_t co;   // counter offset (ints), T (T+1) / 2 lower tiles
  int64_t lo;   // log-det part offset, T entries
  int64_t vo;   // vector offset (doubles), npad entries
  int64_t gt;   // first generation block of this replicate
  const double* locs;
  const double* z;
};

struct BCtl {
  int next;      // task counter
  int abort;     // set on any time-out
  int pad[2];
};

__device__ __forceinline__ int tri_index(int i, int j) { return i * (i + 1) / 2 + j; }

__global__ void batched_params_kernel(int nrep, const double* __restrict__ theta, MaternParams* __restrict__ P,
                                      int32_t* __restrict__ status) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrep) return;
  double th[3] = {theta[3 * r], theta[3 * r + 1], theta[3 * r + 2]};
  bool ok = true;
  for (int c = 0; c < 3; ++c) ok = ok && (th[c] > 0.0) && isfinite(th[c]);
  status[r] = ok ? EXA_OK : EXA_ERR_ARG;
  if (!ok) th[0] = th[1] = th[2] = 1.0;  // keep the arithmetic finite; the result is discarded
  matern_params_hd(th, &P[r]);
}

// Generation: block b -> replicate (binary search over first-block offsets) and lower tile.
template <int NB>
__global__ void __launch_bounds__(256) batched_gen_kernel(int nrep, const BMeta* __restrict__ M,
                                                          const MaternParams* __restrict__ P, double* __restrict__ mat) {
  int lo = 0, hi = nrep - 1;
  const int64_t b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (M[mid].gt <= b) lo = mid; else hi = mid - 1;
  }
  const int r = lo;
  const BMeta m = M[r];
  const MaternParams& Pr = P[r];
  int64_t t = b - m.gt;
  int ti = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((int64_t)ti * (ti + 1) / 2 > t) --ti;
  while ((int64_t)(ti + 1) * (ti + 2) / 2 <= t) ++ti;
  const int tj = (int)(t - (int64_t)ti * (ti + 1) / 2);
  double* a = mat + m.mo;
  constexpr int PER = NB * NB / 256;
  const int64_t i = (int64_t)ti * NB + (threadIdx.x % NB);
  double xi = 0.0, yi = 0.0;
  if (i < m.n) {
    xi = m.locs[2 * i];
    yi = m.locs[2 * i + 1];
  }
  for (int s = 0; s < PER; ++s) {
    const int64_t j = (int64_t)tj * NB + (threadIdx.x / NB) + (256 / NB) * s;
    if (j > i) continue;
    double v;
    if (i >= m.n || j >= m.n) {
      v = (i == j) ? 1.0 : 0.0;
    } else if (i == j) {
      v = Pr.sigma2;
    } else {
      const double dx = xi - m.locs[2 * j], dy = yi - m.locs[2 * j + 1];
      v = matern_value(Pr, sqrt(dx * dx + dy * dy));
    }
    a[i + j * m.npad] = v;
  }
}

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

// Wait until *p >= want (acquire).  Bounded; returns false on time-out or abort.
__device__ __forceinline__ bool wait_count(const int* p, int want, volatile int* abort, long long limit) {
  if (*(volatile const int*)p >= want) {
    __threadfence();
    return true;
  }
  const long long t0 = clock64();
  while (true) {
    if (*(volatile const int*)p >= want) {
      __threadfence();
      return true;
    }
    if (*abort) return false;
    if (clock64() - t0 > limit) return false;
    __nanosleep(200);
  }
}

template <int NB>
struct Tile {
  static constexpr int SS = NB + 4;  // padded smem row stride for the GEMM operands
};

// C (NB x NB) [-]= A B^T with A(r, t) from tile a (column-major, ld), B(c, t) from
// either a tile (column-major) or a row-major NB x NB matrix; result kept in acc.
// 4 warps in 2 x 2, each (NB/2) x (NB/2) = MI x MI m8n8 blocks.
template <int NB>
__device__ __forceinline__ void tile_gemm(const double* a, int64_t lda, const double* b, int64_t ldb, bool b_rowmajor,
                                          double* As, double* Bs, double (&acc)[NB / 16][NB / 16][2]) {
  constexpr int MI = NB / 16, SS = Tile<NB>::SS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3, wm = warp >> 1, wn = warp & 1;
  for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
    const int r = idx % NB, t = idx / NB;  // rows fastest: column-major tiles coalesce
    // L2-only loads: tiles are written by other SMs during this launch and L1 is not coherent
    As[r * SS + t] = __ldcg(a + r + (int64_t)t * lda);
    if (b_rowmajor) {
      const int c2 = idx / NB, t2 = idx % NB;
      Bs[c2 * SS + t2] = __ldcg(b + (int64_t)c2 * ldb + t2);
    } else {
      Bs[r * SS + t] = __ldcg(b + r + (int64_t)t * ldb);
    }
  }
  __syncthreads();
#pragma unroll
  for (int mi = 0; mi < MI; ++mi)
#pragma unroll
    for (int ni = 0; ni < MI; ++ni) acc[mi][ni][0] = acc[mi][ni][1] = 0.0;
#pragma unroll 4
  for (int kk = 0; kk < NB; kk += 4) {
    double af[MI], bf[MI];
#pragma unroll
    for (int mi = 0; mi < MI; ++mi) af[mi] = As[(wm * (NB / 2) + mi * 8 + g) * SS + kk + q];
#pragma unroll
    for (int ni = 0; ni < MI; ++ni) bf[ni] = Bs[(wn * (NB / 2) + ni * 8 + g) * SS + kk + q];
#pragma unroll
    for (int mi = 0; mi < MI; ++mi)
#pragma unroll
      for (int ni = 0; ni < MI; ++ni) dmma(acc[mi][ni][0], acc[mi][ni][1], af[mi], bf[ni]);
  }
  __syncthreads();
}

template <int NB>
__global__ void __launch_bounds__(128) batched_chol_kernel(const BTask* __restrict__ tasks, int ntasks,
                                                           const BMeta* __restrict__ M, double* __restrict__ mat,
                                                           double* __restrict__ wbuf, double* __restrict__ ldpart,
                                                           int* __restrict__ cnt, BCtl* ctl,
                                                           int32_t* __restrict__ rstatus, DevStatus* st,
                                                           long long spin_limit) {
  constexpr int MI = NB / 16, SS = Tile<NB>::SS;
  extern __shared__ double sm[];
  double* As = sm;
  double* Bs = sm + NB * SS;
  __shared__ int s_task;
  __shared__ int s_ok;
  volatile int* abort = &ctl->abort;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3, wm = warp >> 1, wn = warp & 1;
  while (true) {
    if (tid == 0) s_task = *abort ? ntasks : atomicAdd(&ctl->next, 1);
    __syncthreads();
    const int id = s_task;
    if (id >= ntasks) break;
    const BTask tk = tasks[id];
    const BMeta m = M[tk.r];
    int* c = cnt + m.co;
    double* a = mat + m.mo;
    const int64_t ld = m.npad;
    // ---- dependencies ----
    if (tid == 0) {
      bool ok = true;
      if (tk.op == OP_POTRF) {
        ok = wait_count(&c[tri_index(tk.k, tk.k)], tk.k, abort, spin_limit);
      } else if (tk.op == OP_TRSM) {
        ok = wait_count(&c[tri_index(tk.i, tk.k)], tk.k, abort, spin_limit) &&
             wait_count(&c[tri_index(tk.k, tk.k)], tk.k + 1, abort, spin_limit);
      } else if (tk.op == OP_UPDATE) {
        ok = wait_count(&c[tri_index(tk.i, tk.k)], tk.k + 1, abort, spin_limit) &&
             wait_count(&c[tri_index(tk.j, tk.k)], tk.k + 1, abort, spin_limit) &&
             wait_count(&c[tri_index(tk.i, tk.j)], tk.k, abort, spin_limit);
      } else {  // OP_STALL: a dependency nothing satisfies (failure-path test hook)
        ok = wait_count(&c[0], 1 << 30, abort, spin_limit);
      }
      if (!ok) {
        if (atomicExch(&ctl->abort, 1) == 0) {
          atomicExch(&st->timeout, 1);
          st->timeout_where = 31;
        }
        rstatus[tk.r] = EXA_ERR_TIMEOUT;
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) break;
    // ---- work ----
    if (tk.op == OP_POTRF) {
      double* S = As;  // NB x (NB + 1)
      double* tmp = As + NB * (NB + 1);
      const int sd = NB + 1;
      double* T = a + (int64_t)tk.k * NB + (int64_t)tk.k * NB * ld;
      for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
        const int i = idx % NB, j = idx / NB;
        S[i * sd + j] = (i >= j) ? __ldcg(T + i + (int64_t)j * ld) : 0.0;
      }
      __syncthreads();
      int bad = -1;
      for (int j = 0; j < NB; ++j) {
        const double d = S[j * sd + j];
        if (!(d > 0.0) || !isfinite(d)) {
          bad = j;
          break;
        }
        const double lj = sqrt(d), inv = 1.0 / lj;
        for (int i = j + 1 + tid; i < NB; i += blockDim.x) S[i * sd + j] *= inv;
        __syncthreads();
        if (tid == 0) S[j * sd + j] = lj;
        const int per = blockDim.x / NB > 0 ? blockDim.x / NB : 1;
        const int l = tid % NB, i0 = tid / NB;
        if (l > j && i0 < per) {
          const double slj = S[l * sd + j];
          for (int i = l + i0; i < NB; i += per) S[i * sd + l] = fma(-S[i * sd + j], slj, S[i * sd + l]);
        }
        __syncthreads();
      }
      if (bad >= 0) {
        // not SPD: record, and keep the task graph moving (its results are discarded)
        if (tid == 0) rstatus[tk.r] = EXA_ERR_NOT_SPD;
        for (int idx = tid; idx < NB * NB; idx += blockDim.x) S[(idx / NB) * sd + idx % NB] = (idx / NB == idx % NB);
        __syncthreads();
      }
      for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
        const int i = idx % NB, j = idx / NB;
        if (i >= j) T[i + (int64_t)j * ld] = S[i * sd + j];
      }
      if (tid == 0) {
        double sacc = 0.0;
        for (int i = 0; i < NB; ++i) sacc += log(S[i * sd + i]);
        ldpart[m.lo + tk.k] = sacc;
      }
      __syncthreads();
      for (int j = NB - 1; j >= 0; --j) {
        const double wjj = 1.0 / S[j * sd + j];
        for (int i = j + 1 + tid; i < NB; i += blockDim.x) {
          double t2 = 0.0;
          for (int l2 = j + 1; l2 <= i; ++l2) t2 = fma(S[i * sd + l2], S[l2 * sd + j], t2);
          tmp[i] = t2;
        }
        __syncthreads();
        for (int i = j + 1 + tid; i < NB; i += blockDim.x) S[i * sd + j] = -tmp[i] * wjj;
        if (tid == 0) S[j * sd + j] = wjj;
        __syncthreads();
      }
      double* W = wbuf + m.wo + (int64_t)tk.k * NB * NB;
      for (int idx = tid; idx < NB * NB; idx += blockDim.x) {
        const int rr = idx / NB, cc = idx % NB;
        W[idx] = (cc <= rr) ? S[rr * sd + cc] : 0.0;
      }
    } else if (tk.op == OP_TRSM || tk.op == OP_UPDATE) {
      double acc[MI][MI][2];
      double* out;
      if (tk.op == OP_TRSM) {
        const double* W = wbuf + m.wo + (int64_t)tk.k * NB * NB;
        out = a + (int64_t)tk.i * NB + (int64_t)tk.k * NB * ld;
        tile_gemm<NB>(out, ld, W, NB, true, As, Bs, acc);
      } else {
        const double* ai = a + (int64_t)tk.i * NB + (int64_t)tk.k * NB * ld;
        const double* aj = a + (int64_t)tk.j * NB + (int64_t)tk.k * NB * ld;
        out = a + (int64_t)tk.i * NB + (int64_t)tk.j * NB * ld;
        tile_gemm<NB>(ai, ld, aj, ld, false, As, Bs, acc);
      }
      const bool diag = (tk.op == OP_UPDATE && tk.i == tk.j);
#pragma unroll
      for (int mi = 0; mi < MI; ++mi)
#pragma unroll
        for (int ni = 0; ni < MI; ++ni)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int rr = wm * (NB / 2) + mi * 8 + g;
            const int cc = wn * (NB / 2) + ni * 8 + 2 * q + e;
            if (diag && cc > rr) continue;
            double* p = out + rr + (int64_t)cc * ld;
            *p = (tk.op == OP_TRSM) ? acc[mi][ni][e] : __ldcg(p) - acc[mi][ni][e];
          }
    }
    // ---- signal ----
    __syncthreads();
    if (tid == 0 && tk.op != OP_STALL) {
      __threadfence();
      const int tgt = (tk.op == OP_POTRF) ? tri_index(tk.k, tk.k)
                                          : (tk.op == OP_TRSM ? tri_index(tk.i, tk.k) : tri_index(tk.i, tk.j));
      atomicAdd(&c[tgt], 1);
    }
  }
}

// One CTA per replicate: y = L^-1 z (left-looking over NB blocks with the stored
// inverses), log|Sigma| = 2 sum log L_ii, l = -n/2 log 2pi - 1/2 log|Sigma| - 1/2 y^T y.
template <int NB>
__global__ void __launch_bounds__(256) batched_solve_kernel(int nrep, const BMeta* __restrict__ M,
                                                            const double* __restrict__ mat,
                                                            const double* __restrict__ wbuf,
                                                            const double* __restrict__ ldpart,
                                                            const int* __restrict__ cnt, double* __restrict__ yv,
                                                            double* __restrict__ loglik,
                                                            int32_t* __restrict__ rstatus) {
  __shared__ double part[256 / NB][NB];
  __shared__ double sv[NB];
  __shared__ double red[256];
  const int r = blockIdx.x;
  const BMeta m = M[r];
  const int tid = threadIdx.x;
  const int T = (int)m.T;
  // the factor is complete only if its last diagonal tile was factored
  const bool done = cnt[m.co + tri_index(T - 1, T - 1)] == T;
  if (!done && rstatus[r] == EXA_OK) rstatus[r] = EXA_ERR_TIMEOUT;
  if (rstatus[r] != EXA_OK) {
    if (tid == 0) loglik[r] = NAN;
    return;
  }
  const double* a = mat + m.mo;
  double* y = yv + m.vo;
  const int64_t ld = m.npad;
  const int row = tid % NB, slice = tid / NB;
  const int nslice = 256 / NB;
  double quad = 0.0;
  for (int k = 0; k < T; ++k) {
    // s = z_k - sum_{j < k} L_kj y_j   (slices of the column range, fixed order)
    double sacc = 0.0;
    const int64_t gi = (int64_t)k * NB + row;
    for (int64_t jc = slice; jc < (int64_t)k * NB; jc += nslice) sacc = fma(a[gi + jc * ld], y[jc], sacc);
    part[slice][row] = sacc;
    __syncthreads();
    if (tid < NB) {
      double sv0 = (gi < m.n) ? m.z[gi] : 0.0;
      for (int s2 = 0; s2 < nslice; ++s2) sv0 -= part[s2][tid];
      sv[tid] = sv0;
    }
    __syncthreads();
    if (tid < NB) {
      const double* W = wbuf + m.wo + (int64_t)k * NB * NB;
      double yk = 0.0;
      for (int t = 0; t <= tid; ++t) yk = fma(W[tid * NB + t], sv[t], yk);
      y[(int64_t)k * NB + tid] = yk;
      quad = fma(yk, yk, quad);
    }
    __syncthreads();
  }
  red[tid] = quad;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0) {
    double ldet = 0.0;
    for (int k = 0; k < T; ++k) ldet += ldpart[m.lo + k];
    ldet *= 2.0;
    loglik[r] = -0.5 * (double)m.n * 1.8378770664093454836 - 0.5 * ldet - 0.5 * red[0];
  }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
struct BatchPlan {
  std::vector<int64_t> ns;
  int nb = 0;
  int stall = 0;
  int64_t mat_doubles = 0, w_doubles = 0, cnt_ints = 0, ld_doubles = 0, vec_doubles = 0, gen_blocks = 0;
  int ntasks = 0;
  size_t meta_off = 0, params_off = 0, tasks_off = 0, ctl_off = 0, cnt_off = 0, meta_bytes = 0;
};

template <int NB>
static exa_status batched_run(exa_ctx* c, int nrep, const int64_t* h_n, const double* const* d_locs,
                              const double* const* d_z, const double* d_theta, double* d_loglik, int32_t* d_status) {
  cudaStream_t s = c->stream;
  BatchPlan& P = *c->bplan;
  const bool same = P.nb == NB && P.stall == c->batched_stall && (int)P.ns.size() == nrep &&
                    std::equal(P.ns.begin(), P.ns.end(), h_n);
  std::vector<BMeta> meta(nrep);
  int64_t mo = 0, wo = 0, co = 0, lo = 0, vo = 0, gt = 0;
  for (int r = 0; r < nrep; ++r) {
    BMeta& m = meta[r];
    m.n = h_n[r];
    m.npad = round_up(h_n[r], NB);
    m.T = m.npad / NB;
    m.mo = mo;
    m.wo = wo;
    m.co = co;
    m.lo = lo;
    m.vo = vo;
    m.gt = gt;
    m.locs = d_locs[r];
    m.z = d_z[r];
    mo += round_up(m.npad * m.npad, 32);
    wo += m.T * NB * NB;
    co += m.T * (m.T + 1) / 2;
    lo += m.T;
    vo += m.npad;
    gt += m.T * (m.T + 1) / 2;
  }
  std::vector<BTask> tasks;
  if (!same) {
    int Tmax = 0;
    for (int r = 0; r < nrep; ++r) Tmax = meta[r].T > Tmax ? (int)meta[r].T : Tmax;
    if (Tmax > 32000) return set_err(c, EXA_ERR_ARG, "replicate too large for the batched form");
    for (int k = 0; k < Tmax; ++k) {
      for (int r = 0; r < nrep; ++r) {
        const int T = (int)meta[r].T;
        if (k >= T) continue;
        tasks.push_back({r, (short)OP_POTRF, (short)k, (short)k, (short)k, 0, 0});
        for (int i = k + 1; i < T; ++i) tasks.push_back({r, (short)OP_TRSM, (short)k, (short)i, (short)k, 0, 0});
        for (int i = k + 1; i < T; ++i)
          for (int j = k + 1; j <= i; ++j) tasks.push_back({r, (short)OP_UPDATE, (short)k, (short)i, (short)j, 0, 0});
      }
      if (c->batched_stall && k == 0) tasks.push_back({0, (short)OP_STALL, 0, 0, 0, 0, 0});
    }
    P.ns.assign(h_n, h_n + nrep);
    P.nb = NB;
    P.stall = c->batched_stall;
    P.ntasks = (int)tasks.size();
  }
  P.mat_doubles = mo;
  P.w_doubles = wo;
  P.cnt_ints = co;
  P.ld_doubles = lo;
  P.vec_doubles = vo;
  P.gen_blocks = gt;
  // device layout of bt_meta: meta | params | ctl | counters | tasks
  const size_t meta_b = round_up((int64_t)nrep * sizeof(BMeta), 256);
  const size_t par_b = round_up((int64_t)nrep * sizeof(MaternParams), 256);
  const size_t ctl_b = 256;
  const size_t cnt_b = round_up(co * (int64_t)sizeof(int), 256);
  const size_t task_b = round_up((int64_t)P.ntasks * sizeof(BTask), 256);
  exa_status st;
  if ((st = ensure(c, c->bt_meta, meta_b + par_b + ctl_b + cnt_b + task_b, "batched metadata")) != EXA_OK) return st;
  if ((st = ensure(c, c->bt_mat, (size_t)mo * sizeof(double), "batched matrices")) != EXA_OK) return st;
  if ((st = ensure(c, c->bt_work, (size_t)(wo + lo) * sizeof(double), "batched inverses")) != EXA_OK) return st;
  if ((st = ensure(c, c->bt_vec, (size_t)vo * sizeof(double), "batched vectors")) != EXA_OK) return st;
  uint8_t* base = (uint8_t*)c->bt_meta.p;
  BMeta* dM = (BMeta*)base;
  MaternParams* dP = (MaternParams*)(base + meta_b);
  BCtl* dC = (BCtl*)(base + meta_b + par_b);
  int* dCnt = (int*)(base + meta_b + par_b + ctl_b);
  BTask* dT = (BTask*)(base + meta_b + par_b + ctl_b + cnt_b);
  // host staging (pinned, owned by the context so captured copies stay valid)
  const size_t stage_need = meta_b + (same ? 0 : task_b);
  if (c->bt_stage_bytes < stage_need) {
    if (c->bt_stage) cudaFreeHost(c->bt_stage);
    c->bt_stage = nullptr;
    c->bt_stage_bytes = 0;
    if (cudaMallocHost(&c->bt_stage, stage_need) != cudaSuccess) return set_err(c, EXA_ERR_NOMEM, "pinned staging");
    c->bt_stage_bytes = stage_need;
  }
  memcpy(c->bt_stage, meta.data(), nrep * sizeof(BMeta));
  cudaError_t e = cudaMemcpyAsync(dM, c->bt_stage, nrep * sizeof(BMeta), cudaMemcpyHostToDevice, s);
  if (!same && e == cudaSuccess) {
    memcpy((uint8_t*)c->bt_stage + meta_b, tasks.data(), tasks.size() * sizeof(BTask));
    e = cudaMemcpyAsync(dT, (uint8_t*)c->bt_stage + meta_b, tasks.size() * sizeof(BTask), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(dC, 0, ctl_b + cnt_b, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(DevStatus), s);
  if (e != cudaSuccess) return cuda_err(c, e, "batched setup");
  {
    ProfScope ps(c, PK_BATCH, 0.0, 0.0);
    batched_params_kernel<<<(nrep + 63) / 64, 64, 0, s>>>(nrep, d_theta, dP, d_status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    ProfScope ps(c, PK_GEN, 0.0, 8.0 * (double)gt * NB * NB / 2);
    batched_gen_kernel<NB><<<(unsigned)gt, 256, 0, s>>>(nrep, dM, dP, (double*)c->bt_mat.p);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_err(c, e, "batched generation");
  double flops = 0.0;
  for (int r = 0; r < nrep; ++r) flops += (double)meta[r].npad * meta[r].npad * meta[r].npad / 3.0;
  {
    const size_t smem = (size_t)2 * NB * Tile<NB>::SS * sizeof(double) > (size_t)(NB * (NB + 1) + NB) * sizeof(double)
                            ? (size_t)2 * NB * Tile<NB>::SS * sizeof(double)
                            : (size_t)(NB * (NB + 1) + NB) * sizeof(double);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(batched_chol_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      attr = true;
    }
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_chol_kernel<NB>, 128, smem);
    int want = c->batched_ctas_per_sm > 0 ? c->batched_ctas_per_sm : per_sm;
    if (want > per_sm) want = per_sm;  // every CTA must be resident: the walk relies on it
    if (want < 1) return set_err(c, EXA_ERR_CUDA, "batched kernel cannot be resident");
    const int grid = want * sms;
    ProfScope ps(c, PK_BATCH, 2.0 * flops, 0.0);
    batched_chol_kernel<NB><<<grid, 128, smem, s>>>(dT, P.ntasks, dM, (double*)c->bt_mat.p, (double*)c->bt_work.p,
                                                     (double*)c->bt_work.p + wo, dCnt, dC, d_status, c->d_status,
                                                     c->batched_spin);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    ProfScope ps(c, PK_TRSV, 0.0, 4.0 * (double)vo * vo / nrep);
    batched_solve_kernel<NB><<<nrep, 256, 0, s>>>(nrep, dM, (double*)c->bt_mat.p, (double*)c->bt_work.p,
                                                   (double*)c->bt_work.p + wo, dCnt, (double*)c->bt_vec.p, d_loglik,
                                                   d_status);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_err(c, e, "batched launch");
  return EXA_OK;
}

void release_batched(exa_ctx* c) {
  if (c->bt_stage) cudaFreeHost(c->bt_stage);
  c->bt_stage = nullptr;
  c->bt_stage_bytes = 0;
  delete c->bplan;
  c->bplan = nullptr;
}

}  // namespace exa

using namespace exa;

extern "C" exa_status exa_loglik_batched(exa_ctx* c, int32_t nrep, const int64_t* h_n, const double* const* d_locs,
                                         const double* const* d_z, const double* d_theta, exa_prec prec,
                                         double* d_loglik, int32_t* d_status) {
  if (!c) return EXA_ERR_ARG;
  c->err[0] = 0;
  if (nrep < 1 || !h_n || !d_locs || !d_z || !d_theta || !d_loglik || !d_status)
    return set_err(c, EXA_ERR_ARG, "bad batched arguments");
  for (int r = 0; r < nrep; ++r)
    if (h_n[r] < 1 || !d_locs[r] || !d_z[r]) return set_err(c, EXA_ERR_ARG, "replicate %d: bad size or pointer", r);
  if (prec != EXA_FP64) return set_err(c, EXA_ERR_ARG, "the batched form runs in EXA_FP64");
  if (!c->bplan) c->bplan = new BatchPlan();
  if (c->batched_nb == 32) return batched_run<32>(c, nrep, h_n, d_locs, d_z, d_theta, d_loglik, d_status);
  return batched_run<64>(c, nrep, h_n, d_locs, d_z, d_theta, d_loglik, d_status);
}

extern "C" exa_status exa_ctx_set_batched(exa_ctx* c, int tile_nb, int ctas_per_sm, long long spin_cycles,
                                          int inject_stall) {
  if (!c) return EXA_ERR_ARG;
  if (tile_nb != 0 && tile_nb != 32 && tile_nb != 64) return set_err(c, EXA_ERR_ARG, "tile must be 32 or 64");
  if (ctas_per_sm < 0 || spin_cycles < 0) return set_err(c, EXA_ERR_ARG, "bad batched option");
  c->batched_nb = tile_nb ? tile_nb : 64;
  c->batched_ctas_per_sm = ctas_per_sm;
  c->batched_spin = spin_cycles ? spin_cycles : 2000000000LL;
  c->batched_stall = inject_stall ? 1 : 0;
  return EXA_OK;
}
