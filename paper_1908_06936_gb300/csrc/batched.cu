// Batched evaluation of many independent replicate fields of uneven size (the
// replicate studies of Section III, Example 2, run as one device workload).
//
// Stream-ordered, graph-capturable sequence (no host synchronisation):
//   1. per-replicate Matérn constants and interpolation table of Eq. 3 from
//      theta in device memory (so a captured graph can be replayed with new
//      parameters);
//   2. generation of every replicate's lower tiles in one launch (mixed
//      precision also keeps an FP64 copy of Sigma for the refinement residual);
//   3. ONE persistent launch that walks a work list of tile tasks
//        POTRF(r, k)    L_kk = chol(A_kk), W_k = L_kk^-1, log-det part
//        TRSM(r, i, k)  L_ik = A_ik W_k^T
//        UPDATE(r,i,j,k) A_ij -= L_ik L_jk^T
//      ordered by step k across replicates (a topological order of every
//      replicate's DAG).  CTAs claim tasks in list order; a task waits on
//      per-tile completion counters (bounded spin: on time-out the replicate
//      reports EXA_ERR_TIMEOUT and every CTA stops claiming work), runs, then
//      bumps its tile's counter.  Since every dependency sits earlier in the
//      list and all CTAs are co-resident, the walk cannot deadlock.
//      FP64: every task on FP64 DMMA.  Mixed (the MP variant of Section II-A):
//      POTRF stays FP64; TRSM and UPDATE tiles farther than `band` tile
//      diagonals from the diagonal run as three TF32 tensor-core products
//      (hi*hi + hi*lo + lo*hi, FP32 accumulation over the tile's K) added to
//      the FP64 tile;
//   4. FP64: one CTA per replicate: blocked forward solve, log-det, quadratic
//      form, l = -n/2 log 2 pi - 1/2 log|Sigma| - 1/2 y^T y and the status.
//      Mixed: one CTA per replicate refines x = Sigma^-1 z in FP64
//      (x += L^-T L^-1 (z - Sigma x) with the FP64 copy of Sigma) and uses
//      q = z^T x.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "bessel.cuh"
#include "ctx.cuh"
#include "gemm_tc.cuh"

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
                                      int32_t* __restrict__ status, double nugget, int metric, double radius) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrep) return;
  double th[3] = {theta[3 * r], theta[3 * r + 1], theta[3 * r + 2]};
  bool ok = true;
  for (int c = 0; c < 3; ++c) ok = ok && (th[c] > 0.0) && isfinite(th[c]);
  status[r] = ok ? EXA_OK : EXA_ERR_ARG;
  if (!ok) th[0] = th[1] = th[2] = 1.0;  // keep the arithmetic finite; the result is discarded
  matern_params_hd(th, &P[r]);
  P[r].nugget = nugget;
  P[r].metric = metric;
  P[r].radius = radius;
}

// Per-replicate interpolation tables (blockIdx.y = replicate).
__global__ void batched_table_nodes_kernel(const MaternParams* __restrict__ P, double* __restrict__ nodes) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int NN = kTabSeg * (kTabDeg + 1);
  if (id >= NN) return;
  nodes[(int64_t)blockIdx.y * NN + id] = table_node_value(P[blockIdx.y], id);
}

__global__ void batched_table_coef_kernel(const double* __restrict__ nodes, MaternTable* __restrict__ T) {
  const int sgi = blockIdx.x * blockDim.x + threadIdx.x;
  if (sgi >= kTabSeg) return;
  table_segment_coefs(nodes + (int64_t)blockIdx.y * kTabSeg * (kTabDeg + 1), sgi, &T[blockIdx.y]);
}

// Generation: block b -> replicate (binary search over first-block offsets) and lower tile.
// mat2 (mixed precision) receives a second copy of every entry.
template <int NB>
__global__ void __launch_bounds__(256) batched_gen_kernel(int nrep, const BMeta* __restrict__ M,
                                                          const MaternParams* __restrict__ P,
                                                          const MaternTable* __restrict__ tabs,
                                                          double* __restrict__ mat, double* __restrict__ mat2) {
  int lo = 0, hi = nrep - 1;
  const int64_t b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (M[mid].gt <= b) lo = mid; else hi = mid - 1;
  }
  const int r = lo;
  const BMeta m = M[r];
  const MaternParams& Pr = P[r];
  const MaternTable* tab = tabs + r;
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
      v = Pr.sigma2 + Pr.nugget;
    } else {
      v = matern_value_tab(Pr, tab, model_dist2(Pr, xi, yi, m.locs[2 * j], m.locs[2 * j + 1]));
    }
    a[i + j * m.npad] = v;
    if (mat2) mat2[m.mo + i + j * m.npad] = v;
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

constexpr int kBThreads = 128;  // threads of the persistent factorisation CTA

// Modes of the persistent factorisation: every task in FP64; FP32 off-diagonal tiles
// with a band of FP64 tiles next to the diagonal; FP32 off-diagonal tiles everywhere.
enum : int { MODE_FP64 = 0, MODE_F32_BAND = 1, MODE_F32 = 2 };

template <int NB>
struct Tile {
  static constexpr int SS = NB + 4;   // padded smem row stride of the FP64 operands
  static constexpr int SA = NB + 4;   // padded smem stride of the FP32 operands (k-major)
  static constexpr int PER = NB * NB / kBThreads;       // tile elements per thread
  static constexpr int CH = PER < 16 ? PER : 16;        // loads in flight per operand
  static constexpr size_t smem(int mode) {
    const size_t f64 = (size_t)2 * NB * SS * sizeof(double);
    const size_t f32 = (size_t)2 * NB * SA * sizeof(float);
    const size_t po = (size_t)(NB * (NB + 1) + NB) * sizeof(double);
    const size_t m = f32 > po ? f32 : po;
    return mode == MODE_F32 ? m : (f64 > m ? f64 : m);
  }
};

template <int NB>
__device__ __forceinline__ void tile_gemm(const double* a, int64_t lda, const double* b, int64_t ldb, bool b_rowmajor,
                                          double* As, double* Bs, double (&acc)[NB / 16][NB / 16][2]) {
  constexpr int MI = NB / 16, SS = Tile<NB>::SS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, q = lane & 3, wm = warp >> 1, wn = warp & 1;
  // rows fastest: column-major tiles coalesce.  L2-only loads (tiles are written by
  // other SMs during this launch and L1 is not coherent), CH of each operand in flight.
  constexpr int PER = Tile<NB>::PER, CH = Tile<NB>::CH;
#pragma unroll
  for (int c0 = 0; c0 < PER; c0 += CH) {
    double va[CH], vb[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int idx = tid + (c0 + u) * kBThreads;
      const int r = idx % NB, t = idx / NB;
      va[u] = __ldcg(a + r + (int64_t)t * lda);
      // row-major B: element (row t, col r) at b[t ldb + r], also read along r
      vb[u] = b_rowmajor ? __ldcg(b + (int64_t)t * ldb + r) : __ldcg(b + r + (int64_t)t * ldb);
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int idx = tid + (c0 + u) * kBThreads;
      const int r = idx % NB, t = idx / NB;
      As[r * SS + t] = va[u];
      if (b_rowmajor) Bs[t * SS + r] = vb[u];
      else Bs[r * SS + t] = vb[u];
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

// ---- FP32 tile product (mixed precision) ----
// out (NB x NB, column-major, ld) = / -= A B^T with A(r, t) = a[r + t ld] and B(c, t) from
// either a column-major tile (b[c + t ld]) or a row-major NB x NB matrix (b[c NB + t]).
// Operands rounded to FP32, products accumulated in FP32 over the tile's K = NB (FFMA),
// the result added to the FP64 tile.  Thread (tr, tc) owns rows tr + (NB/4) i, i < 4, and
// the CT consecutive columns tc CT .. tc CT + CT - 1.
template <int NB>
__device__ __forceinline__ void tile_f32(const double* a, const double* b, bool b_rowmajor, double* out, int64_t ld,
                                         bool store, bool lower_only, float* sm) {
  constexpr int SA = Tile<NB>::SA, RG = NB / 4, CT = NB * NB / (kBThreads * 4);
  constexpr int PER = Tile<NB>::PER, CH = Tile<NB>::CH;
  float* As = sm;            // k-major: element (row, k) at As[k SA + row]
  float* Bs = sm + NB * SA;  // element (col, k) at Bs[k SA + col]
  const int tid = threadIdx.x, tr = tid % RG, tc = tid / RG;
#pragma unroll
  for (int c0 = 0; c0 < PER; c0 += CH) {
    double va[CH], vb[CH];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int idx = tid + (c0 + u) * kBThreads;
      const int r = idx % NB, t = idx / NB;
      va[u] = __ldcg(a + r + (int64_t)t * ld);
      // row-major B (NB x NB): element (row t, col r) at b[t NB + r]
      vb[u] = b_rowmajor ? __ldcg(b + (int64_t)t * NB + r) : __ldcg(b + r + (int64_t)t * ld);
    }
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      const int idx = tid + (c0 + u) * kBThreads;
      const int r = idx % NB, t = idx / NB;
      As[t * SA + r] = (float)va[u];
      if (b_rowmajor) Bs[r * SA + t] = (float)vb[u];  // B operand column t, k = r
      else Bs[t * SA + r] = (float)vb[u];
    }
  }
  __syncthreads();
  float acc[4][CT];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < CT; ++j) acc[i][j] = 0.0f;
#pragma unroll 8
  for (int k = 0; k < NB; ++k) {
    float av[4], bv[CT];
#pragma unroll
    for (int i = 0; i < 4; ++i) av[i] = As[k * SA + tr + RG * i];
    if constexpr (CT % 4 == 0) {
#pragma unroll
      for (int j = 0; j < CT; j += 4) {
        const float4 v = *reinterpret_cast<const float4*>(Bs + k * SA + tc * CT + j);
        bv[j] = v.x;
        bv[j + 1] = v.y;
        bv[j + 2] = v.z;
        bv[j + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < CT; ++j) bv[j] = Bs[k * SA + tc * CT + j];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < CT; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < CT; ++j) {
      const int rr = tr + RG * i, cc = tc * CT + j;
      if (lower_only && cc > rr) continue;
      double* p = out + rr + (int64_t)cc * ld;
      *p = store ? (double)acc[i][j] : __ldcg(p) - (double)acc[i][j];
    }
}

template <int NB, int MODE>
__global__ void __launch_bounds__(kBThreads) batched_chol_kernel(const BTask* __restrict__ tasks, int ntasks,
                                                           const BMeta* __restrict__ M, double* __restrict__ mat,
                                                           double* __restrict__ wbuf, double* __restrict__ ldpart,
                                                           int* __restrict__ cnt, BCtl* ctl,
                                                           int32_t* __restrict__ rstatus, DevStatus* st,
                                                           long long spin_limit, int band) {
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
#pragma unroll
      for (int c0 = 0; c0 < Tile<NB>::PER; c0 += Tile<NB>::CH) {
        double v[Tile<NB>::CH];
#pragma unroll
        for (int u = 0; u < Tile<NB>::CH; ++u) {
          const int idx = tid + (c0 + u) * kBThreads, i = idx % NB, j = idx / NB;
          v[u] = (i >= j) ? __ldcg(T + i + (int64_t)j * ld) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < Tile<NB>::CH; ++u) {
          const int idx = tid + (c0 + u) * kBThreads;
          S[(idx % NB) * sd + idx / NB] = v[u];
        }
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
    } else if (MODE != MODE_FP64 && (tk.op == OP_TRSM || tk.op == OP_UPDATE) &&
               (MODE == MODE_F32 || (tk.op == OP_TRSM ? tk.i - tk.k : tk.i - tk.j) >= band)) {
      if (tk.op == OP_TRSM) {
        const double* W = wbuf + m.wo + (int64_t)tk.k * NB * NB;
        double* out = a + (int64_t)tk.i * NB + (int64_t)tk.k * NB * ld;
        tile_f32<NB>(out, W, true, out, ld, true, false, (float*)sm);
      } else {
        const double* ai = a + (int64_t)tk.i * NB + (int64_t)tk.k * NB * ld;
        const double* aj = a + (int64_t)tk.j * NB + (int64_t)tk.k * NB * ld;
        double* out = a + (int64_t)tk.i * NB + (int64_t)tk.j * NB * ld;
        tile_f32<NB>(ai, aj, false, out, ld, false, tk.i == tk.j, (float*)sm);
      }
    } else if (MODE != MODE_F32 && (tk.op == OP_TRSM || tk.op == OP_UPDATE)) {
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
// Mixed precision: per-replicate FP64 refinement of x = Sigma^-1 z (one CTA of
// kIrThreads per replicate, largest replicates first).
// ---------------------------------------------------------------------------
constexpr int kIrThreads = 1024;
constexpr double kIrFail = 1e-8;  // relative residual above which a replicate reports EXA_ERR_IR_NOCONV
// The refinement ends once q is final to kIrQTol relative, by the variational estimate
// q = z^T x + x^T r + r^T d (d = (L L^T)^-1 r), off by r^T (Sigma^-1 - (L L^T)^-1) r, whose
// size is estimated as kIrQSafety times the last step's contraction times |r^T d| (the rule of
// the single-field mixed path).
constexpr double kIrQTol = 1e-8;
constexpr double kIrQSafety = 100.0;

// Block-wide sum, the same order on every call (warp shuffles, then warp 0).
__device__ __forceinline__ double ir_block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// y = L^-1 b, blocked by NB with the stored inverses W_k of the diagonal tiles:
// y_k = W_k (b_k - sum_{j < k} L_kj y_j).  Columns of the sum are split over
// kIrThreads / NB slices (fixed order), eight loads in flight per thread.
template <int NB>
__device__ void ir_forward(const double* __restrict__ L, const double* __restrict__ W, int64_t ld, int T,
                           const double* b, double* y, double (*part)[NB], double* sv) {
  constexpr int NS = kIrThreads / NB;
  const int tid = threadIdx.x, row = tid % NB, slice = tid / NB;
  for (int k = 0; k < T; ++k) {
    const int64_t kc = (int64_t)k * NB;
    const double* Lr = L + kc + row;
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t jc = slice;
    for (; jc + 7 * NS < kc; jc += 8 * NS) {
#pragma unroll
      for (int u = 0; u < 8; ++u) s[u] = fma(__ldcs(Lr + (jc + u * NS) * ld), y[jc + u * NS], s[u]);
    }
    for (; jc < kc; jc += NS) s[0] = fma(__ldcs(Lr + jc * ld), y[jc], s[0]);
    part[slice][row] = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
    __syncthreads();
    if (tid < NB) {
      double v = b[kc + tid];
      for (int q = 0; q < NS; ++q) v -= part[q][tid];
      sv[tid] = v;
    }
    __syncthreads();
    if (tid < NB) {
      const double* Wk = W + kc * NB;
      double yk = 0.0;
      for (int t = 0; t <= tid; ++t) yk = fma(Wk[tid * NB + t], sv[t], yk);
      y[kc + tid] = yk;
    }
    __syncthreads();
  }
}

// y := L^-T y in place: d_k = W_k^T (y_k - sum_{i > k} L_ik^T d_i).  Column c of
// the sum is contiguous below the tile: one warp per column, lanes over rows.
template <int NB>
__device__ void ir_backward(const double* __restrict__ L, const double* __restrict__ W, int64_t ld, int T,
                            int64_t npad, double* y, double* sv) {
  constexpr int NW = kIrThreads / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = T - 1; k >= 0; --k) {
    const int64_t kc = (int64_t)k * NB, r0 = kc + NB;
    for (int c = warp; c < NB; c += NW) {
      const double* col = L + (kc + c) * ld;
      double s[4] = {0, 0, 0, 0};
      int64_t i = r0 + lane;
      for (; i + 96 < npad; i += 128) {
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u] = fma(__ldcs(col + i + 32 * u), y[i + 32 * u], s[u]);
      }
      for (; i < npad; i += 32) s[0] = fma(__ldcs(col + i), y[i], s[0]);
      double v = (s[0] + s[1]) + (s[2] + s[3]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) sv[c] = y[kc + c] - v;
    }
    __syncthreads();
    if (tid < NB) {
      const double* Wk = W + kc * NB;
      double d = 0.0;
      for (int u = tid; u < NB; ++u) d = fma(Wk[u * NB + tid], sv[u], d);
      y[kc + tid] = d;
    }
    __syncthreads();
  }
}

// r = z - Sigma x from the lower triangle of Sigma (FP64 copy), returns ||r||^2.
// Row part sum_{j <= i} S_ij x_j: thread per row (coalesced along the column);
// column part sum_{j > i} S_ji x_j: warp per column.  Fixed order.
__device__ double ir_residual(const double* __restrict__ S, int64_t ld, int64_t n, int64_t npad,
                              const double* __restrict__ z, const double* x, double* rv, double* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = kIrThreads / 32;
  // column part first, into rv
  for (int64_t c = warp; c < npad; c += NW) {
    const double* col = S + c * ld;
    double s[4] = {0, 0, 0, 0};
    int64_t i = c + 1 + lane;
    for (; i + 96 < npad; i += 128) {
#pragma unroll
      for (int u = 0; u < 4; ++u) s[u] = fma(__ldcs(col + i + 32 * u), x[i + 32 * u], s[u]);
    }
    for (; i < npad; i += 32) s[0] = fma(__ldcs(col + i), x[i], s[0]);
    double v = (s[0] + s[1]) + (s[2] + s[3]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) rv[c] = v;
  }
  __syncthreads();
  double rr = 0.0;
  for (int64_t i0 = 0; i0 < npad; i0 += kIrThreads) {
    const int64_t i = i0 + tid;
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (i < npad) {
      const double* rowp = S + i;
      int64_t j = 0;
      for (; j + 7 <= i; j += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) s[u] = fma(__ldcs(rowp + (j + u) * ld), x[j + u], s[u]);
      }
      for (; j <= i; ++j) s[0] = fma(__ldcs(rowp + j * ld), x[j], s[0]);
      const double sx = ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7])) + rv[i];
      const double ri = (i < n) ? z[i] - sx : 0.0;
      rv[i] = ri;
      rr = fma(ri, ri, rr);
    }
  }
  return ir_block_sum(rr, red);
}

template <int NB>
__global__ void __launch_bounds__(kIrThreads) batched_ir_kernel(
    const int* __restrict__ order, const BMeta* __restrict__ M, const double* __restrict__ mat,
    const double* __restrict__ sig, const double* __restrict__ wbuf, const double* __restrict__ ldpart,
    const int* __restrict__ cnt, double* __restrict__ vec, int64_t vtot, double* __restrict__ loglik,
    int32_t* __restrict__ rstatus, int max_iter) {
  __shared__ double part[kIrThreads / NB][NB];
  __shared__ double sv[NB];
  __shared__ double red[33];
  const int r = order[blockIdx.x];
  const BMeta m = M[r];
  const int tid = threadIdx.x;
  const int T = (int)m.T;
  const bool done = cnt[m.co + tri_index(T - 1, T - 1)] == T;
  __syncthreads();
  if (tid == 0 && !done && rstatus[r] == EXA_OK) rstatus[r] = EXA_ERR_TIMEOUT;
  __syncthreads();
  if (rstatus[r] != EXA_OK) {
    if (tid == 0) loglik[r] = NAN;
    return;
  }
  const double* L = mat + m.mo;
  const double* S = sig + m.mo;
  const double* W = wbuf + m.wo;
  const int64_t ld = m.npad, npad = m.npad, n = m.n;
  double* x = vec + m.vo;
  double* rv = vec + vtot + m.vo;
  double* y = vec + 2 * vtot + m.vo;
  double zz = 0.0;
  for (int64_t i = tid; i < npad; i += kIrThreads) {
    const double zi = (i < n) ? m.z[i] : 0.0;
    x[i] = 0.0;
    rv[i] = zi;
    zz = fma(zi, zi, zz);
  }
  const double zn2 = ir_block_sum(zz, red);
  double prev = 1e300, rel = 1e300;
  double rel_cur = 1.0, rel_prev = 1.0;  // ||r|| / ||z|| of this step and the one before (r_0 = z)
  double q = 0.0;
  bool q_done = false;
  for (int it = 0; it < max_iter; ++it) {
    ir_forward<NB>(L, W, ld, T, rv, y, part, sv);
    ir_backward<NB>(L, W, ld, T, npad, y, sv);  // y = d = (L L^T)^-1 r
    if (it > 0) {  // at it = 0, x = 0 and r = z: the estimate is the plain first solve's
      double xr = 0.0, rd = 0.0, zx0 = 0.0;
      for (int64_t i = tid; i < npad; i += kIrThreads) {
        xr = fma(x[i], rv[i], xr);
        rd = fma(rv[i], y[i], rd);
        if (i < n) zx0 = fma(m.z[i], x[i], zx0);
      }
      const double a = ir_block_sum(xr, red);
      const double b = ir_block_sum(rd, red);
      const double c0 = ir_block_sum(zx0, red);
      const double q_hat = c0 + a + b;
      const double rho = rel_prev > 0.0 ? rel_cur / rel_prev : 1.0;
      if (kIrQSafety * rho * fabs(b) <= kIrQTol * fabs(q_hat)) {
        q = q_hat;
        q_done = true;
        rel = rel_cur;
        break;
      }
    }
    for (int64_t i = tid; i < npad; i += kIrThreads) x[i] += y[i];
    __syncthreads();
    const double rn2 = ir_residual(S, ld, n, npad, m.z, x, rv, red);
    rel = zn2 > 0.0 ? sqrt(rn2 / zn2) : 0.0;
    if (!(rel > 1e-15) || rel > 0.5 * prev) break;  // converged, or no longer contracting
    prev = rel;
    rel_prev = rel_cur;
    rel_cur = rel;
  }
  if (!q_done) {
    double zx = 0.0;
    for (int64_t i = tid; i < n; i += kIrThreads) zx = fma(m.z[i], x[i], zx);
    q = ir_block_sum(zx, red);
  }
  if (tid == 0) {
    double ldet = 0.0;
    for (int k = 0; k < T; ++k) ldet += ldpart[m.lo + k];
    ldet *= 2.0;
    if (q_done || rel <= kIrFail) {
      loglik[r] = -0.5 * (double)n * 1.8378770664093454836 - 0.5 * ldet - 0.5 * q;
    } else {
      loglik[r] = NAN;
      rstatus[r] = EXA_ERR_IR_NOCONV;
    }
  }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
struct TcStep {
  int diag_off, ndiag;       // DiagTileTask range
  int wsplit_off, psplit_off, nset, max_m;  // SplitTask ranges (inverse tiles, panels) and panel rows
  int trsm_off, ntrsm;       // TcTask ranges
  int upd_off, nupd;
};

struct BatchPlan {
  std::vector<int64_t> ns;
  int nb = 0;
  int stall = 0;
  bool mixed = false;
  int ntasks = 0;
  // tensor-core form (step-synchronous): per-step launch ranges, and the buffers the device task
  // lists point into (a change of any of them rebuilds the lists)
  bool tc = false;
  std::vector<TcStep> steps;
  const void* tc_mat = nullptr;
  const void* tc_work = nullptr;
  const void* tc_meta = nullptr;
  int64_t ps_rows = 0;
  SplitOperand ps, ws;
};

// Work-list order.  Every task gets its bottom level: the longest path, in
// estimated task durations, from the task to the end of its replicate's
// factorisation.  The list is sorted by decreasing bottom level (counting sort,
// stable).  A predecessor's bottom level exceeds each successor's by at least
// its own duration, so the order is topological (no CTA can wait on a task
// claimed after its own); and the long chains through the diagonal tiles come
// first, so CTAs rarely sit on a claimed task whose inputs are still being
// computed.  Relative durations: POTRF (FP64, unblocked, one CTA) dP, TRSM and
// UPDATE one unit each (in mixed precision those run on tensor cores).
static void build_task_list(const std::vector<BMeta>& meta, bool mixed, bool stall, std::vector<BTask>& tasks) {
  const int dP = mixed ? 16 : 2, dS = 1, dU = 1;
  std::vector<int> keys;
  std::vector<BTask> raw;
  int kmax = 0;
  const int nrep = (int)meta.size();
  for (int r = 0; r < nrep; ++r) {
    const int T = (int)meta[r].T;
    // bottom levels: U of step k+1 (cur, then swapped), S(i, k) over all (i, k), P(k)
    std::vector<int> bS((size_t)T * T, 0), bP(T, 0), un((size_t)T * T, 0), uc((size_t)T * T, 0);
    for (int k = T - 1; k >= 0; --k) {
      // UPDATE(i, j, k), k < j <= i: its successor is the next operation on tile (i, j)
      for (int i = k + 1; i < T; ++i)
        for (int j = k + 1; j <= i; ++j) {
          const int nxt = (j == k + 1) ? (i == j ? bP[j] : bS[(size_t)i * T + j]) : un[(size_t)i * T + j];
          const int key = dU + nxt;
          uc[(size_t)i * T + j] = key;
          raw.push_back({r, (short)OP_UPDATE, (short)k, (short)i, (short)j, 0, 0});
          keys.push_back(key);
        }
      // TRSM(i, k): feeds UPDATE(i, j, k) for k < j <= i and UPDATE(i2, i, k) for i2 > i
      for (int i = k + 1; i < T; ++i) {
        int m = 0;
        for (int j = k + 1; j <= i; ++j) m = std::max(m, uc[(size_t)i * T + j]);
        for (int i2 = i + 1; i2 < T; ++i2) m = std::max(m, uc[(size_t)i2 * T + i]);
        bS[(size_t)i * T + k] = dS + m;
        raw.push_back({r, (short)OP_TRSM, (short)k, (short)i, (short)k, 0, 0});
        keys.push_back(dS + m);
      }
      int m = 0;
      for (int i = k + 1; i < T; ++i) m = std::max(m, bS[(size_t)i * T + k]);
      bP[k] = dP + m;
      raw.push_back({r, (short)OP_POTRF, (short)k, (short)k, (short)k, 0, 0});
      keys.push_back(dP + m);
      std::swap(un, uc);
    }
  }
  for (int key : keys) kmax = std::max(kmax, key);
  std::vector<int64_t> start((size_t)kmax + 2, 0);
  for (int key : keys) ++start[(size_t)(kmax - key) + 1];
  for (size_t b = 1; b < start.size(); ++b) start[b] += start[b - 1];
  tasks.assign(raw.size(), BTask{});
  for (size_t t = 0; t < raw.size(); ++t) tasks[(size_t)start[(size_t)(kmax - keys[t])]++] = raw[t];
  if (stall) {
    // test hook: a task whose dependency nothing satisfies, early in the list
    const size_t at = tasks.size() < 8 ? tasks.size() : 8;
    tasks.insert(tasks.begin() + (int64_t)at, BTask{0, (short)OP_STALL, 0, 0, 0, 0, 0});
  }
}

struct CholArgs {
  const BTask* tasks;
  int ntasks;
  const BMeta* M;
  double* mat;
  double* wbuf;
  double* ldpart;
  int* cnt;
  BCtl* ctl;
  int32_t* rstatus;
  DevStatus* st;
  long long spin;
  int band;
  int ctas_per_sm;
};

// The persistent factorisation: as many CTAs per SM as fit (or the requested
// number, capped there: the walk relies on every CTA being resident).
template <int NB, int MODE>
static exa_status launch_chol(exa_ctx* c, cudaStream_t s, const CholArgs& a) {
  const size_t smem = Tile<NB>::smem(MODE);
  static PerDeviceOnce attr_once;
  const cudaError_t ea = attr_once([&] {
    return cudaFuncSetAttribute(batched_chol_kernel<NB, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (ea != cudaSuccess) return cuda_err(c, ea, "batched kernel attribute");
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_chol_kernel<NB, MODE>, kBThreads, smem);
  int want = a.ctas_per_sm > 0 ? a.ctas_per_sm : per_sm;
  if (want > per_sm) want = per_sm;
  if (want < 1) return set_err(c, EXA_ERR_CUDA, "batched kernel cannot be resident");
  batched_chol_kernel<NB, MODE><<<want * sms, kBThreads, smem, s>>>(a.tasks, a.ntasks, a.M, a.mat, a.wbuf, a.ldpart,
                                                                    a.cnt, a.ctl, a.rstatus, a.st, a.spin, a.band);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? EXA_OK : cuda_err(c, e, "batched factorisation launch");
}

template <int NB, int MODE>
static int max_ctas_per_sm() {
  const size_t smem = Tile<NB>::smem(MODE);
  cudaFuncSetAttribute(batched_chol_kernel<NB, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_chol_kernel<NB, MODE>, kBThreads, smem);
  return per_sm;
}

static int max_ctas_per_sm(int nb, int mode) {
  if (nb == 32)
    return mode == MODE_FP64 ? max_ctas_per_sm<32, MODE_FP64>()
                             : (mode == MODE_F32_BAND ? max_ctas_per_sm<32, MODE_F32_BAND>() : max_ctas_per_sm<32, MODE_F32>());
  return mode == MODE_FP64 ? max_ctas_per_sm<64, MODE_FP64>()
                           : (mode == MODE_F32_BAND ? max_ctas_per_sm<64, MODE_F32_BAND>() : max_ctas_per_sm<64, MODE_F32>());
}

template <int NB, bool MIXED>
static exa_status batched_run(exa_ctx* c, int nrep, const int64_t* h_n, const double* const* d_locs,
                              const double* const* d_z, const double* d_theta, double* d_loglik, int32_t* d_status) {
  cudaStream_t s = c->stream;
  BatchPlan& P = *c->bplan;
  const bool same = P.nb == NB && P.mixed == MIXED && P.stall == c->batched_stall && (int)P.ns.size() == nrep &&
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
  // replicates by decreasing size: the refinement CTAs of the largest start first
  std::vector<int> order(nrep);
  for (int r = 0; r < nrep; ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return h_n[x] > h_n[y]; });
  std::vector<BTask> tasks;
  if (!same) {
    int Tmax = 0;
    for (int r = 0; r < nrep; ++r) Tmax = meta[r].T > Tmax ? (int)meta[r].T : Tmax;
    if (Tmax > 32000) return set_err(c, EXA_ERR_ARG, "replicate too large for the batched form");
    build_task_list(meta, MIXED, c->batched_stall != 0, tasks);
    P.ns.assign(h_n, h_n + nrep);
    P.nb = NB;
    P.stall = c->batched_stall;
    P.mixed = MIXED;
    P.ntasks = (int)tasks.size();
  }
  // device layout of bt_meta: meta | order | params | tables | ctl | counters | tasks
  constexpr int64_t kNodes = kTabSeg * (kTabDeg + 1);
  const size_t meta_b = round_up((int64_t)nrep * sizeof(BMeta), 256);
  const size_t ord_b = round_up((int64_t)nrep * sizeof(int), 256);
  const size_t par_b = round_up((int64_t)nrep * sizeof(MaternParams), 256);
  const size_t tab_b = round_up((int64_t)nrep * sizeof(MaternTable), 256);
  const size_t ctl_b = 256;
  const size_t cnt_b = round_up(co * (int64_t)sizeof(int), 256);
  const size_t task_b = round_up((int64_t)P.ntasks * sizeof(BTask), 256);
  const size_t nodes_b = (size_t)nrep * kNodes * sizeof(double);
  exa_status st;
  if ((st = ensure(c, c->bt_meta, meta_b + ord_b + par_b + tab_b + ctl_b + cnt_b + task_b, "batched metadata")) !=
      EXA_OK)
    return st;
  if ((st = ensure(c, c->bt_mat, (size_t)mo * sizeof(double), "batched matrices")) != EXA_OK) return st;
  if (MIXED && (st = ensure(c, c->bt_mat2, (size_t)mo * sizeof(double), "batched FP64 copies")) != EXA_OK) return st;
  const size_t work_b = (size_t)(wo + lo) * sizeof(double);
  if ((st = ensure(c, c->bt_work, work_b > nodes_b ? work_b : nodes_b, "batched inverses")) != EXA_OK) return st;
  if ((st = ensure(c, c->bt_vec, (size_t)(MIXED ? 3 : 1) * vo * sizeof(double), "batched vectors")) != EXA_OK)
    return st;
  uint8_t* base = (uint8_t*)c->bt_meta.p;
  BMeta* dM = (BMeta*)base;
  int* dOrd = (int*)(base + meta_b);
  MaternParams* dP = (MaternParams*)(base + meta_b + ord_b);
  MaternTable* dTab = (MaternTable*)(base + meta_b + ord_b + par_b);
  BCtl* dC = (BCtl*)(base + meta_b + ord_b + par_b + tab_b);
  int* dCnt = (int*)(base + meta_b + ord_b + par_b + tab_b + ctl_b);
  BTask* dT = (BTask*)(base + meta_b + ord_b + par_b + tab_b + ctl_b + cnt_b);
  // the table nodes are scratch until the factorisation overwrites bt_work
  double* dNodes = (double*)c->bt_work.p;
  // host staging (pinned, owned by the context so captured copies stay valid)
  const size_t stage_need = meta_b + ord_b + (same ? 0 : task_b);
  if (c->bt_stage_bytes < stage_need) {
    if (c->bt_stage) cudaFreeHost(c->bt_stage);
    c->bt_stage = nullptr;
    c->bt_stage_bytes = 0;
    if (cudaMallocHost(&c->bt_stage, stage_need) != cudaSuccess) return set_err(c, EXA_ERR_NOMEM, "pinned staging");
    c->bt_stage_bytes = stage_need;
  }
  uint8_t* hs = (uint8_t*)c->bt_stage;
  memcpy(hs, meta.data(), nrep * sizeof(BMeta));
  memcpy(hs + meta_b, order.data(), nrep * sizeof(int));
  cudaError_t e = cudaMemcpyAsync(dM, hs, meta_b + ord_b, cudaMemcpyHostToDevice, s);
  if (!same && e == cudaSuccess) {
    memcpy(hs + meta_b + ord_b, tasks.data(), tasks.size() * sizeof(BTask));
    e = cudaMemcpyAsync(dT, hs + meta_b + ord_b, tasks.size() * sizeof(BTask), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(dC, 0, ctl_b + cnt_b, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(DevStatus), s);
  if (e != cudaSuccess) return cuda_err(c, e, "batched setup");
  {
    ProfScope ps(c, PK_OTHER, 0.0, 0.0, 3);
    batched_params_kernel<<<(nrep + 63) / 64, 64, 0, s>>>(nrep, d_theta, dP, d_status, c->nugget, c->metric,
                                                          c->radius);
    batched_table_nodes_kernel<<<dim3((unsigned)((kNodes + 127) / 128), (unsigned)nrep), 128, 0, s>>>(dP, dNodes);
    batched_table_coef_kernel<<<dim3((kTabSeg + 127) / 128, (unsigned)nrep), 128, 0, s>>>(dNodes, dTab);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    ProfScope ps(c, PK_GEN, 0.0, (MIXED ? 16.0 : 8.0) * (double)gt * NB * NB / 2);
    batched_gen_kernel<NB><<<(unsigned)gt, 256, 0, s>>>(nrep, dM, dP, dTab, (double*)c->bt_mat.p,
                                                        MIXED ? (double*)c->bt_mat2.p : nullptr);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_err(c, e, "batched generation");
  double flops = 0.0;
  for (int r = 0; r < nrep; ++r) flops += (double)meta[r].npad * meta[r].npad * meta[r].npad / 3.0;
  if (e == cudaSuccess) {
    const int mode = !MIXED ? MODE_FP64 : (c->batched_band > 0 ? MODE_F32_BAND : MODE_F32);
    ProfScope ps(c, PK_BATCH, 2.0 * flops, 0.0);
    const CholArgs ca{dT, P.ntasks, dM, (double*)c->bt_mat.p, (double*)c->bt_work.p, (double*)c->bt_work.p + wo,
                      dCnt, dC, d_status, c->d_status, c->batched_spin, c->batched_band, c->batched_ctas_per_sm};
    if (mode == MODE_FP64) st = launch_chol<NB, MODE_FP64>(c, s, ca);
    else if (mode == MODE_F32_BAND) st = launch_chol<NB, MODE_F32_BAND>(c, s, ca);
    else st = launch_chol<NB, MODE_F32>(c, s, ca);
    if (st != EXA_OK) return st;
  }
  if (e == cudaSuccess && !MIXED) {
    ProfScope ps(c, PK_TRSV, 0.0, 4.0 * (double)vo * vo / nrep);
    batched_solve_kernel<NB><<<nrep, 256, 0, s>>>(nrep, dM, (double*)c->bt_mat.p, (double*)c->bt_work.p,
                                                   (double*)c->bt_work.p + wo, dCnt, (double*)c->bt_vec.p, d_loglik,
                                                   d_status);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && MIXED) {
    double lower = 0.0;
    for (int r = 0; r < nrep; ++r) lower += 0.5 * (double)meta[r].npad * (double)(meta[r].npad + 1);
    ProfScope ps(c, PK_TRSV, 0.0, 16.0 * lower);  // bytes of one refinement step
    batched_ir_kernel<NB><<<nrep, kIrThreads, 0, s>>>(dOrd, dM, (double*)c->bt_mat.p, (double*)c->bt_mat2.p,
                                                       (double*)c->bt_work.p, (double*)c->bt_work.p + wo, dCnt,
                                                       (double*)c->bt_vec.p, vo, d_loglik, d_status,
                                                       c->batched_max_iter);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_err(c, e, "batched launch");
  return EXA_OK;
}

// ---------------------------------------------------------------------------
// Tensor-core batched form (EXA_MIXED_TF32X3): step-synchronous over 128-wide tile columns,
// every replicate advancing together.  Per step k, for the replicates that still have tile
// column k:
//   1. FP64 Cholesky and inverse W_k of each diagonal tile (one launch, a CTA per tile);
//   2. TF32 hi/lo splits of every W_k and of every panel below (two launches, all replicates'
//      rows stacked in one operand);
//   3. panel solve L_ik = A_ik W_k^T as ONE grouped tcgen05 launch of TF32x3 128 x 128 tiles;
//   4. split of the solved panels (one launch);
//   5. trailing update A_ij -= L_ik L_jk^T as ONE grouped tcgen05 launch over every replicate's
//      trailing lower tiles.
// Then the FP64 refinement of x = Sigma^-1 z per replicate (as the FP32 form).  Everything is
// stream-ordered with no host synchronisation (graph-capturable); the task lists depend only on
// the replicate sizes and are uploaded when they change.
// ---------------------------------------------------------------------------
constexpr int kTcNB = 128;

__global__ void batched_tc_finish_kernel(int nrep, const BMeta* __restrict__ M, const DevStatus* __restrict__ rst,
                                         const DevStatus* __restrict__ st, int* __restrict__ cnt,
                                         int32_t* __restrict__ rstatus) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrep) return;
  const BMeta m = M[r];
  if (rstatus[r] == EXA_OK) {
    if (st->timeout) rstatus[r] = EXA_ERR_TIMEOUT;
    else if (rst[r].info) rstatus[r] = EXA_ERR_NOT_SPD;
  }
  cnt[m.co + tri_index((int)m.T - 1, (int)m.T - 1)] = (int)m.T;  // factorisation done (refinement's check)
}

static exa_status batched_run_tc(exa_ctx* c, int nrep, const int64_t* h_n, const double* const* d_locs,
                                 const double* const* d_z, const double* d_theta, double* d_loglik,
                                 int32_t* d_status) {
  constexpr int NB = kTcNB;
  cudaStream_t s = c->stream;
  BatchPlan& P = *c->bplan;
  const bool same_shape = P.tc && P.nb == NB && (int)P.ns.size() == nrep && std::equal(P.ns.begin(), P.ns.end(), h_n);
  std::vector<BMeta> meta(nrep);
  int64_t mo = 0, wo = 0, co = 0, lo = 0, vo = 0, gt = 0;
  int Tmax = 0;
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
    Tmax = m.T > Tmax ? (int)m.T : Tmax;
  }
  if (Tmax > 32000) return set_err(c, EXA_ERR_ARG, "replicate too large for the batched form");
  std::vector<int> order(nrep);
  for (int r = 0; r < nrep; ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return h_n[x] > h_n[y]; });
  // panel rows of step 0 (the most): every replicate's rows below its first tile
  int64_t ps_rows = 0;
  for (int r = 0; r < nrep; ++r) ps_rows += meta[r].npad - NB;
  ps_rows = round_up(ps_rows > 0 ? ps_rows : NB, NB);
  // device layout of bt_meta: meta | order | params | tables | ctl | counters | replicate statuses
  const size_t meta_b = round_up((int64_t)nrep * sizeof(BMeta), 256);
  const size_t ord_b = round_up((int64_t)nrep * sizeof(int), 256);
  const size_t par_b = round_up((int64_t)nrep * sizeof(MaternParams), 256);
  const size_t tab_b = round_up((int64_t)nrep * sizeof(MaternTable), 256);
  const size_t ctl_b = 256;
  const size_t cnt_b = round_up(co * (int64_t)sizeof(int), 256);
  const size_t rst_b = round_up((int64_t)nrep * sizeof(DevStatus), 256);
  constexpr int64_t kNodes = kTabSeg * (kTabDeg + 1);
  const size_t nodes_b = (size_t)nrep * kNodes * sizeof(double);
  exa_status st;
  if ((st = ensure(c, c->bt_meta, meta_b + ord_b + par_b + tab_b + ctl_b + cnt_b + rst_b, "batched metadata")) !=
      EXA_OK)
    return st;
  if ((st = ensure(c, c->bt_mat, (size_t)mo * sizeof(double), "batched matrices")) != EXA_OK) return st;
  if ((st = ensure(c, c->bt_mat2, (size_t)mo * sizeof(double), "batched FP64 copies")) != EXA_OK) return st;
  const size_t work_b = (size_t)(wo + lo) * sizeof(double);
  if ((st = ensure(c, c->bt_work, work_b > nodes_b ? work_b : nodes_b, "batched inverses")) != EXA_OK) return st;
  if ((st = ensure(c, c->bt_vec, (size_t)3 * vo * sizeof(double), "batched vectors")) != EXA_OK) return st;
  const bool ps_new = c->bt_ps.bytes < split_bytes(ps_rows, NB, true, false) + 1024 ||
                      c->bt_ws.bytes < split_bytes((int64_t)nrep * NB, NB, true, false) + 1024;
  if ((st = ensure_split(c, P.ps, c->bt_ps, ps_rows, NB, true, false)) != EXA_OK) return st;
  if ((st = ensure_split(c, P.ws, c->bt_ws, (int64_t)nrep * NB, NB, true, false)) != EXA_OK) return st;
  uint8_t* base = (uint8_t*)c->bt_meta.p;
  BMeta* dM = (BMeta*)base;
  int* dOrd = (int*)(base + meta_b);
  MaternParams* dP = (MaternParams*)(base + meta_b + ord_b);
  MaternTable* dTab = (MaternTable*)(base + meta_b + ord_b + par_b);
  int* dCnt = (int*)(base + meta_b + ord_b + par_b + tab_b + ctl_b);
  DevStatus* dRst = (DevStatus*)(base + meta_b + ord_b + par_b + tab_b + ctl_b + cnt_b);
  double* mat = (double*)c->bt_mat.p;
  double* wbuf = (double*)c->bt_work.p;
  double* ldpart = wbuf + wo;
  // task lists (rebuilt when the sizes or the buffers they point into change)
  const bool rebuild = !same_shape || ps_new || P.tc_mat != c->bt_mat.p || P.tc_work != c->bt_work.p ||
                       P.tc_meta != c->bt_meta.p;
  std::vector<DiagTileTask> diag;
  std::vector<SplitTask> spl;
  std::vector<TcTask> tc;
  if (rebuild) {
    P.steps.clear();
    for (int k = 0; k < Tmax; ++k) {
      TcStep stp{};
      stp.diag_off = (int)diag.size();
      for (int r = 0; r < nrep; ++r) {
        const BMeta& m = meta[r];
        if (m.T <= k) continue;
        diag.push_back({mat + m.mo, m.npad, (int64_t)k * NB, ldpart + m.lo + k, wbuf + m.wo + (int64_t)k * NB * NB,
                        dRst + r});
      }
      stp.ndiag = (int)diag.size() - stp.diag_off;
      // replicates with a panel below tile k
      std::vector<int> set;
      for (int r = 0; r < nrep; ++r)
        if (meta[r].T > k + 1) set.push_back(r);
      stp.nset = (int)set.size();
      stp.wsplit_off = (int)spl.size();
      for (int q = 0; q < stp.nset; ++q) {
        const BMeta& m = meta[set[q]];
        spl.push_back({wbuf + m.wo + (int64_t)k * NB * NB, NB, 1, NB, q * NB});
      }
      stp.psplit_off = (int)spl.size();
      std::vector<int> prow(stp.nset);
      int rows = 0;
      stp.max_m = 0;
      for (int q = 0; q < stp.nset; ++q) {
        const BMeta& m = meta[set[q]];
        const int mr = (int)(m.npad - (int64_t)(k + 1) * NB);
        prow[q] = rows;
        spl.push_back({mat + m.mo + (int64_t)(k + 1) * NB + (int64_t)k * NB * m.npad, 1, m.npad, mr, rows});
        rows += mr;
        stp.max_m = mr > stp.max_m ? mr : stp.max_m;
      }
      stp.trsm_off = (int)tc.size();
      for (int q = 0; q < stp.nset; ++q) {
        const BMeta& m = meta[set[q]];
        const int nbk = (int)(m.T - k - 1);
        for (int i = 0; i < nbk; ++i)
          tc.push_back({mat + m.mo + (int64_t)(k + 1 + i) * NB + (int64_t)k * NB * m.npad, m.npad, prow[q] + i * NB,
                        q * NB, 0, 0});
      }
      stp.ntrsm = (int)tc.size() - stp.trsm_off;
      stp.upd_off = (int)tc.size();
      for (int q = 0; q < stp.nset; ++q) {
        const BMeta& m = meta[set[q]];
        const int nbk = (int)(m.T - k - 1);
        for (int i = 0; i < nbk; ++i)
          for (int j = 0; j <= i; ++j)
            tc.push_back({mat + m.mo + (int64_t)(k + 1 + i) * NB + (int64_t)(k + 1 + j) * NB * m.npad, m.npad,
                          prow[q] + i * NB, prow[q] + j * NB, i == j ? 1 : 0, 0});
      }
      stp.nupd = (int)tc.size() - stp.upd_off;
      P.steps.push_back(stp);
    }
  }
  // device task area: diag | split | tc (offsets fixed by the counts)
  const size_t diag_b = round_up((int64_t)(rebuild ? diag.size() : (size_t)P.ntasks) * sizeof(DiagTileTask), 256);
  (void)diag_b;
  size_t nd = 0, nsp = 0, ntc = 0;
  if (rebuild) {
    nd = diag.size();
    nsp = spl.size();
    ntc = tc.size();
  } else {
    const TcStep& L = P.steps.back();
    nd = (size_t)L.diag_off + L.ndiag;
    nsp = (size_t)L.psplit_off + L.nset;
    ntc = (size_t)L.upd_off + L.nupd;
  }
  const size_t d_b = round_up((int64_t)nd * sizeof(DiagTileTask), 256);
  const size_t s_b = round_up((int64_t)nsp * sizeof(SplitTask), 256);
  const size_t t_b = round_up((int64_t)ntc * sizeof(TcTask), 256);
  if ((st = ensure(c, c->bt_tasks, d_b + s_b + t_b + 256, "batched task lists")) != EXA_OK) return st;
  DiagTileTask* dDiag = (DiagTileTask*)c->bt_tasks.p;
  SplitTask* dSpl = (SplitTask*)((uint8_t*)c->bt_tasks.p + d_b);
  TcTask* dTc = (TcTask*)((uint8_t*)c->bt_tasks.p + d_b + s_b);
  // host staging (pinned, owned by the context so captured copies stay valid)
  const size_t stage_need = meta_b + ord_b + (rebuild ? d_b + s_b + t_b : 0);
  if (c->bt_stage_bytes < stage_need) {
    if (c->bt_stage) cudaFreeHost(c->bt_stage);
    c->bt_stage = nullptr;
    c->bt_stage_bytes = 0;
    if (cudaMallocHost(&c->bt_stage, stage_need) != cudaSuccess) return set_err(c, EXA_ERR_NOMEM, "pinned staging");
    c->bt_stage_bytes = stage_need;
  }
  uint8_t* hs = (uint8_t*)c->bt_stage;
  memcpy(hs, meta.data(), nrep * sizeof(BMeta));
  memcpy(hs + meta_b, order.data(), nrep * sizeof(int));
  cudaError_t e = cudaMemcpyAsync(dM, hs, meta_b + ord_b, cudaMemcpyHostToDevice, s);
  if (rebuild && e == cudaSuccess) {
    uint8_t* ht = hs + meta_b + ord_b;
    memcpy(ht, diag.data(), diag.size() * sizeof(DiagTileTask));
    memcpy(ht + d_b, spl.data(), spl.size() * sizeof(SplitTask));
    memcpy(ht + d_b + s_b, tc.data(), tc.size() * sizeof(TcTask));
    e = cudaMemcpyAsync(c->bt_tasks.p, ht, d_b + s_b + t_b, cudaMemcpyHostToDevice, s);
    P.ns.assign(h_n, h_n + nrep);
    P.nb = NB;
    P.tc = true;
    P.mixed = true;
    P.stall = 0;
    P.ntasks = (int)nd;
    P.tc_mat = c->bt_mat.p;
    P.tc_work = c->bt_work.p;
    P.tc_meta = c->bt_meta.p;
    P.ps_rows = ps_rows;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(dCnt, 0, cnt_b + rst_b, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(DevStatus), s);
  if (e != cudaSuccess) return cuda_err(c, e, "batched setup");
  double* dNodes = wbuf;  // scratch until the factorisation overwrites it
  {
    ProfScope ps(c, PK_OTHER, 0.0, 0.0, 3);
    batched_params_kernel<<<(nrep + 63) / 64, 64, 0, s>>>(nrep, d_theta, dP, d_status, c->nugget, c->metric,
                                                          c->radius);
    batched_table_nodes_kernel<<<dim3((unsigned)((kNodes + 127) / 128), (unsigned)nrep), 128, 0, s>>>(dP, dNodes);
    batched_table_coef_kernel<<<dim3((kTabSeg + 127) / 128, (unsigned)nrep), 128, 0, s>>>(dNodes, dTab);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    ProfScope ps(c, PK_GEN, 0.0, 16.0 * (double)gt * NB * NB / 2);
    batched_gen_kernel<NB><<<(unsigned)gt, 256, 0, s>>>(nrep, dM, dP, dTab, mat, (double*)c->bt_mat2.p);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_err(c, e, "batched generation");
  GemmArgs g;
  memset(&g, 0, sizeof(g));
  g.K = NB;
  g.panel = NB;
  g.enum_mode = kEnumTasks;
  g.st = c->d_status;
  for (size_t k = 0; k < P.steps.size() && e == cudaSuccess; ++k) {
    const TcStep& stp = P.steps[k];
    {
      ProfScope ps(c, PK_POTRF, (double)stp.ndiag * NB * NB * NB * 2.0 / 3.0, 0.0, 1);
      e = launch_potrf128_tasks(s, dDiag + stp.diag_off, stp.ndiag);
    }
    if (e != cudaSuccess || stp.nset == 0) continue;
    {
      ProfScope ps(c, PK_SPLIT, 0.0, 16.0 * (double)(stp.ntrsm + stp.nset) * NB * NB, 2);
      e = launch_split_rows_tasks(s, dSpl + stp.wsplit_off, stp.nset, NB, NB, P.ws);
      if (e == cudaSuccess) e = launch_split_rows_tasks(s, dSpl + stp.psplit_off, stp.nset, stp.max_m, NB, P.ps);
    }
    if (e == cudaSuccess) {
      g.tasks = dTc + stp.trsm_off;
      g.ntiles = stp.ntrsm;
      g.store = 1;
      ProfScope ps(c, PK_GEMM_T3, 2.0 * (double)stp.ntrsm * NB * NB * NB, 16.0 * (double)stp.ntrsm * NB * NB);
      e = launch_gemm_t3(s, P.ps, P.ws, g);
    }
    if (e == cudaSuccess) {
      ProfScope ps(c, PK_SPLIT, 0.0, 16.0 * (double)stp.ntrsm * NB * NB);
      e = launch_split_rows_tasks(s, dSpl + stp.psplit_off, stp.nset, stp.max_m, NB, P.ps);
    }
    if (e == cudaSuccess && stp.nupd > 0) {
      g.tasks = dTc + stp.upd_off;
      g.ntiles = stp.nupd;
      g.store = 0;
      ProfScope ps(c, PK_GEMM_T3, 2.0 * (double)stp.nupd * NB * NB * NB, 16.0 * (double)stp.nupd * NB * NB);
      e = launch_gemm_t3(s, P.ps, P.ps, g);
    }
  }
  if (e != cudaSuccess) return cuda_err(c, e, "batched tensor-core factorisation");
  batched_tc_finish_kernel<<<(nrep + 127) / 128, 128, 0, s>>>(nrep, dM, dRst, c->d_status, dCnt, d_status);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    double lower = 0.0;
    for (int r = 0; r < nrep; ++r) lower += 0.5 * (double)meta[r].npad * (double)(meta[r].npad + 1);
    ProfScope ps(c, PK_TRSV, 0.0, 16.0 * lower);
    batched_ir_kernel<NB><<<nrep, kIrThreads, 0, s>>>(dOrd, dM, mat, (double*)c->bt_mat2.p, wbuf, ldpart, dCnt,
                                                       (double*)c->bt_vec.p, vo, d_loglik, d_status,
                                                       c->batched_max_iter);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_err(c, e, "batched refinement launch");
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
  if (prec != EXA_FP64 && prec != EXA_MIXED_FP32 && prec != EXA_MIXED_TF32X3)
    return set_err(c, EXA_ERR_ARG, "the batched form runs in EXA_FP64, EXA_MIXED_FP32 or EXA_MIXED_TF32X3");
  if (!c->bplan) c->bplan = new BatchPlan();
  if (prec == EXA_MIXED_TF32X3) return batched_run_tc(c, nrep, h_n, d_locs, d_z, d_theta, d_loglik, d_status);
  if (c->bplan->tc) {  // the persistent form rebuilds its own work list
    c->bplan->tc = false;
    c->bplan->ns.clear();
  }
  const bool mixed = prec == EXA_MIXED_FP32;
  if (c->batched_nb == 32)
    return mixed ? batched_run<32, true>(c, nrep, h_n, d_locs, d_z, d_theta, d_loglik, d_status)
                 : batched_run<32, false>(c, nrep, h_n, d_locs, d_z, d_theta, d_loglik, d_status);
  return mixed ? batched_run<64, true>(c, nrep, h_n, d_locs, d_z, d_theta, d_loglik, d_status)
               : batched_run<64, false>(c, nrep, h_n, d_locs, d_z, d_theta, d_loglik, d_status);
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

// Tile autotuner: times every candidate (tile 32 / 64, the largest and the next
// CTAs-per-SM count that fit) on the caller's batch and keeps the fastest.
extern "C" exa_status exa_batched_autotune(exa_ctx* c, int32_t nrep, const int64_t* h_n, const double* const* d_locs,
                                           const double* const* d_z, const double* d_theta, exa_prec prec,
                                           double* d_loglik, int32_t* d_status, int* tile_nb, int* ctas_per_sm,
                                           float* best_ms) {
  if (!c || !tile_nb || !ctas_per_sm || !best_ms) return c ? set_err(c, EXA_ERR_ARG, "null output") : EXA_ERR_ARG;
  const int mode = prec == EXA_FP64 ? MODE_FP64 : (c->batched_band > 0 ? MODE_F32_BAND : MODE_F32);
  const int keep_nb = c->batched_nb, keep_cps = c->batched_ctas_per_sm;
  float best = 3.4e38f;
  int bnb = keep_nb, bcps = keep_cps;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_err(c, cudaGetLastError(), "autotune events");
  }
  exa_status st = EXA_OK;
  // the tensor-core form has one configuration (128-wide tiles, grids sized by the task
  // lists): it is timed once and reported with ctas_per_sm = 0
  const bool tc = prec == EXA_MIXED_TF32X3;
  for (int nb : {64, 32}) {
    const int top = tc ? 1 : max_ctas_per_sm(nb, mode);
    for (int cps : {top, top - 1}) {
      if (tc && (nb != 64 || cps != 1)) continue;
      if (cps < 1 || st != EXA_OK) continue;
      c->batched_nb = nb;
      c->batched_ctas_per_sm = cps;
      // first call builds the plan and the buffers for this tile; the second is timed
      st = exa_loglik_batched(c, nrep, h_n, d_locs, d_z, d_theta, prec, d_loglik, d_status);
      if (st == EXA_OK) {
        cudaEventRecord(e0, c->stream);
        st = exa_loglik_batched(c, nrep, h_n, d_locs, d_z, d_theta, prec, d_loglik, d_status);
        cudaEventRecord(e1, c->stream);
      }
      if (st == EXA_OK) {
        const cudaError_t e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          st = cuda_err(c, e != cudaSuccess ? e : cudaGetLastError(), "autotune timing");
        } else if (ms < best) {
          best = ms;
          bnb = tc ? keep_nb : nb;
          bcps = tc ? keep_cps : cps;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != EXA_OK) {
    c->batched_nb = keep_nb;
    c->batched_ctas_per_sm = keep_cps;
    return st;
  }
  c->batched_nb = bnb;
  c->batched_ctas_per_sm = bcps;
  *tile_nb = tc ? 128 : bnb;
  *ctas_per_sm = tc ? 0 : bcps;
  *best_ms = best;
  return EXA_OK;
}

extern "C" exa_status exa_ctx_set_batched_mixed(exa_ctx* c, int band, int max_iter) {
  if (!c) return EXA_ERR_ARG;
  if (band < 0 || max_iter < 0) return set_err(c, EXA_ERR_ARG, "bad batched mixed option");
  c->batched_band = band;
  c->batched_max_iter = max_iter ? max_iter : 10;
  return EXA_OK;
}
