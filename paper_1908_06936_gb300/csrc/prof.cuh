// Per-kernel-class launch counters (always on) and optional CUDA-event timing
// with the algorithmic flop / byte counts of each launch.
#pragma once

#include <vector>

#include "exa_internal.cuh"

struct exa_ctx;

namespace exa {

enum ProfKind : int {
  PK_GEN = 0,       // Matérn generation (a1)
  PK_POTRF,         // FP64 diagonal tile factorisation + inversion
  PK_TRSM64,        // FP64 DMMA panel solve
  PK_SYRK64,        // FP64 DMMA trailing update
  PK_DGEMM_SMALL,   // FP64 DMMA block-inverse products
  PK_SPLIT,         // split of FP64 rows into TF32 halves / BF16 digits
  PK_GEMM_T3,       // tcgen05 TF32x3 products, one CTA per 128 x 128 tile
  PK_GEMM_T3_PAIR,  // tcgen05 TF32x3 products on CTA pairs (256 x 256 tiles): the trailing update
  PK_GEMM_OZ,       // tcgen05 exact digit-slice products
  PK_TRSV,          // triangular solves
  PK_SYMV,          // refinement residual
  PK_GRAD,          // gradient kernels
  PK_BATCH,         // batched persistent factorisation
  PK_OTHER,         // reductions, copies, padding
  PK_COUNT
};

const char* prof_name(int kind);

struct ProfRec {
  int kind;
  int ev0, ev1;
  double flops, bytes;
  int side;  // issued on the look-ahead stream
};

struct TimelineRec {
  int kind, side;
  float t0, t1;  // ms from the first timed scope of the batch
};

struct Prof {
  bool on = false;
  int64_t launches[PK_COUNT] = {};
  double flops[PK_COUNT] = {};
  double bytes[PK_COUNT] = {};
  double ms[PK_COUNT] = {};
  int64_t timed[PK_COUNT] = {};
  double timed_flops[PK_COUNT] = {};  // flops / bytes of the timed scopes only, so that
  double timed_bytes[PK_COUNT] = {};  // timed work / timed milliseconds is a rate
  std::vector<cudaEvent_t> pool;
  std::vector<ProfRec> recs;
  size_t used = 0;
  bool timeline_on = false;          // keep start / end of every timed scope
  std::vector<TimelineRec> timeline; // bounded (kTimelineMax records)
};

constexpr size_t kTimelineMax = 1u << 20;

// Scope around the launch(es) of one kernel class on the context's stream.
class ProfScope {
 public:
  ProfScope(exa_ctx* c, int kind, double flops, double bytes, int nkernels = 1, cudaStream_t stream = nullptr,
            bool on_stream = false);
  ~ProfScope();

 private:
  exa_ctx* c_;
  cudaStream_t s_;
  int kind_;
  int ev0_ = -1;
  double flops_, bytes_;
};

void prof_collect(exa_ctx* c);  // synchronises and folds pending event pairs into the totals
// After an evaluation that ended with a synchronise: fold its event pairs so the
// event pool is reused (no-op when profiling is off).
void prof_fold(exa_ctx* c);
void prof_release(exa_ctx* c);

}  // namespace exa
