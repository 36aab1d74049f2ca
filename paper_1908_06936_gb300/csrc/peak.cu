// Issue-rate probes of the FP64 pipes (the denominators of the FP64 Cholesky's roofline):
// every resident warp runs eight independent accumulation chains of either DFMA (one FP64
// fused multiply-add per thread and instruction) or DMMA (mma.sync m8n8k4 .f64: 8 x 8 x 4
// multiply-adds per warp and instruction), so that neither latency nor operand traffic
// limits the rate.  Timed with CUDA events on the given stream.
#include <math.h>

#include "exa_internal.cuh"

namespace exa {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) probe_dfma_kernel(int iters, double seed, double* sink) {
  double acc[kProbeChains];
  const double a = 1.0 - 1e-12 * (double)(threadIdx.x + 1), b = seed * 1e-9;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) acc[c] = seed + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += acc[c];
  if (s < 0.0) sink[0] = s;  // every chain stays positive: never taken, but keeps the chains live
}

__global__ void __launch_bounds__(kProbeThreads) probe_dmma_kernel(int iters, double seed, double* sink) {
  double d[kProbeChains][2];
  const double a = 1e-3 * (double)(threadIdx.x & 31), b = seed;  // >= 0
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) d[c][0] = d[c][1] = 0.0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(d[c][0]), "+d"(d[c][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += d[c][0] + d[c][1];
  if (s < 0.0) sink[0] = s;  // a, b >= 0: never taken
}

}  // namespace exa

using namespace exa;

extern "C" exa_status exa_probe_fp64_rate(void* cuda_stream, int kind, double* tflops) {
  if (!tflops || (kind != 0 && kind != 1)) return EXA_ERR_ARG;
  *tflops = NAN;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return EXA_ERR_CUDA;
  }
  const void* fn = kind ? (const void*)probe_dmma_kernel : (const void*)probe_dfma_kernel;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kProbeThreads, 0) != cudaSuccess || per < 1) {
    cudaGetLastError();
    return EXA_ERR_CUDA;
  }
  const int blocks = sms * per;
  // flops per thread (DFMA) or per warp (DMMA) and iteration
  const double per_iter = kind ? (double)kProbeChains * 2.0 * 8 * 8 * 4 * (blocks * (kProbeThreads / 32))
                               : (double)kProbeChains * 2.0 * blocks * kProbeThreads;
  const int iters = kind ? 4096 : 16384;
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first launch warms up
    e = cudaEventRecord(e0, s);
    if (kind)
      probe_dmma_kernel<<<blocks, kProbeThreads, 0, s>>>(iters, 1.0 + 1e-3 * rep, sink);
    else
      probe_dfma_kernel<<<blocks, kProbeThreads, 0, s>>>(iters, 1.0 + 1e-3 * rep, sink);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return EXA_ERR_CUDA;
  }
  *tflops = per_iter * iters / (best * 1e-3) / 1e12;
  return EXA_OK;
}
