// Launch accounting and event timing per kernel class (see prof.cuh).
#include <string.h>

#include "ctx.cuh"
#include "prof.cuh"

namespace exa {

static const char* kNames[PK_COUNT] = {"matern_gen", "potrf_diag_fp64", "trsm_panel_fp64", "syrk_update_fp64",
                                       "dgemm_small_fp64", "split_rows", "gemm_tf32x3_tc", "gemm_tf32x3_pair",
                                       "gemm_ozaki_tc",
                                       "trsv", "symv_residual", "gradient", "batched_chol", "other"};

const char* prof_name(int kind) { return (kind >= 0 && kind < PK_COUNT) ? kNames[kind] : "?"; }

static int take_event(Prof& p) {
  if (p.used == p.pool.size()) {
    if (p.pool.size() >= (1u << 17)) return -1;  // bounded: stop timing, keep counting
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    p.pool.push_back(e);
  }
  return (int)p.used++;
}

ProfScope::ProfScope(exa_ctx* c, int kind, double flops, double bytes, int nkernels, cudaStream_t stream,
                     bool on_stream)
    : c_(c), s_(on_stream ? stream : c->stream), kind_(kind), flops_(flops), bytes_(bytes) {
  Prof& p = c->prof;
  p.launches[kind] += nkernels;
  p.flops[kind] += flops;
  p.bytes[kind] += bytes;
  if (p.on) {
    ev0_ = take_event(p);
    if (ev0_ >= 0) cudaEventRecord(p.pool[ev0_], s_);
  }
}

ProfScope::~ProfScope() {
  Prof& p = c_->prof;
  if (!p.on || ev0_ < 0) return;
  const int ev1 = take_event(p);
  if (ev1 < 0) return;
  cudaEventRecord(p.pool[ev1], s_);
  p.recs.push_back({kind_, ev0_, ev1, flops_, bytes_, (c_->side && s_ == c_->side) ? 1 : 0});
}

void prof_collect(exa_ctx* c) {
  Prof& p = c->prof;
  if (p.recs.empty()) {
    p.used = 0;
    return;
  }
  cudaStreamSynchronize(c->stream);
  if (c->side) cudaStreamSynchronize(c->side);
  const cudaEvent_t base = p.pool[p.recs.front().ev0];
  for (const ProfRec& r : p.recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.pool[r.ev0], p.pool[r.ev1]) == cudaSuccess) {
      p.ms[r.kind] += ms;
      p.timed[r.kind] += 1;
      p.timed_flops[r.kind] += r.flops;
      p.timed_bytes[r.kind] += r.bytes;
      float a = 0.f, b = 0.f;
      if (p.timeline_on && p.timeline.size() < kTimelineMax &&
          cudaEventElapsedTime(&a, base, p.pool[r.ev0]) == cudaSuccess &&
          cudaEventElapsedTime(&b, base, p.pool[r.ev1]) == cudaSuccess)
        p.timeline.push_back({r.kind, r.side, a, b});
    }
  }
  cudaGetLastError();
  p.recs.clear();
  p.used = 0;
}

void prof_fold(exa_ctx* c) {
  if (c->prof.on && !c->prof.recs.empty()) prof_collect(c);
}

void prof_release(exa_ctx* c) {
  for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
  c->prof.pool.clear();
  c->prof.recs.clear();
  c->prof.used = 0;
}

}  // namespace exa

using namespace exa;

extern "C" exa_status exa_profile_enable(exa_ctx* c, int on) {
  if (!c) return EXA_ERR_ARG;
  prof_collect(c);
  c->prof.on = on != 0;
  return EXA_OK;
}

extern "C" exa_status exa_profile_timeline_enable(exa_ctx* c, int on) {
  if (!c) return EXA_ERR_ARG;
  prof_collect(c);
  c->prof.timeline_on = on != 0;
  c->prof.timeline.clear();
  return EXA_OK;
}

extern "C" int exa_profile_timeline(exa_ctx* c, exa_timeline_rec* out, int max, int reset) {
  if (!c || !out || max <= 0) return 0;
  prof_collect(c);
  Prof& p = c->prof;
  const int k = (int)(p.timeline.size() < (size_t)max ? p.timeline.size() : (size_t)max);
  for (int i = 0; i < k; ++i) {
    const TimelineRec& r = p.timeline[i];
    memset(&out[i], 0, sizeof(out[i]));
    strncpy(out[i].name, kNames[r.kind], sizeof(out[i].name) - 1);
    out[i].stream = r.side;
    out[i].start_ms = r.t0;
    out[i].end_ms = r.t1;
  }
  if (reset) p.timeline.clear();
  return k;
}

extern "C" int exa_profile_read(exa_ctx* c, exa_kernel_stat* out, int max, int reset) {
  if (!c || !out || max <= 0) return 0;
  prof_collect(c);
  Prof& p = c->prof;
  int k = 0;
  for (int i = 0; i < PK_COUNT && k < max; ++i) {
    if (p.launches[i] == 0) continue;
    memset(&out[k], 0, sizeof(out[k]));
    strncpy(out[k].name, kNames[i], sizeof(out[k].name) - 1);
    out[k].launches = p.launches[i];
    out[k].timed_launches = p.timed[i];
    out[k].ms = p.ms[i];
    out[k].flops = p.flops[i];
    out[k].bytes = p.bytes[i];
    out[k].timed_flops = p.timed_flops[i];
    out[k].timed_bytes = p.timed_bytes[i];
    ++k;
  }
  if (reset) {
    for (int i = 0; i < PK_COUNT; ++i) {
      p.launches[i] = p.timed[i] = 0;
      p.flops[i] = p.bytes[i] = p.ms[i] = p.timed_flops[i] = p.timed_bytes[i] = 0.0;
    }
  }
  return k;
}
