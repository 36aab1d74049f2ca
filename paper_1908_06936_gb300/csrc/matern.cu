// Step a1: Matérn covariance generation (Section I, Eq. 3) with a device
// modified Bessel function K_nu of fractional order.
//
// Per theta the host precomputes every quantity that depends only on nu
// (Gamma values, Temme's Gamma_1/Gamma_2, reciprocal tables) for the exact
// routine, and the device builds from it an interpolation table of
// Sigma in s = (r / beta)^2, so that most entries cost a squared
// distance, a segment lookup on the bit pattern and a degree-8 polynomial.
#include <math.h>

#include "bessel.cuh"
#include "exa_internal.cuh"

namespace exa {

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

void matern_params(const double theta[3], MaternParams* p) { matern_params_hd(theta, p); }

// ---------------------------------------------------------------------------
// Device side (K_nu itself lives in bessel.cuh)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void tri_decode(long long b, int& ti, int& tj) {
  // b = ti (ti + 1) / 2 + tj,  0 <= tj <= ti
  long long t = (long long)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
  while (t * (t + 1) / 2 > b) --t;
  while ((t + 1) * (t + 2) / 2 <= b) ++t;
  ti = (int)t;
  tj = (int)(b - t * (t + 1) / 2);
}

// One 64 x 64 tile of the lower triangle per block; 256 threads, each thread
// 16 entries of one column strip (consecutive threads = consecutive rows, so
// the column-major stores coalesce).
__global__ void __launch_bounds__(256) matern_gen_kernel(const double* __restrict__ locs, int64_t n, int64_t npad,
                                                         const __grid_constant__ MaternParams P, double* __restrict__ a,
                                                         int64_t ld, unsigned long long* __restrict__ offmax,
                                                         const MaternTable* __restrict__ tab, int oshift,
                                                         double* __restrict__ a2) {
  int ti, tj;
  tri_decode(blockIdx.x, ti, tj);
  const int64_t i = (int64_t)ti * 64 + (threadIdx.x & 63);
  // largest off-diagonal |Sigma_ij| of this thread (for the precision map), as a bit pattern:
  // non-negative doubles order like their bits, so an integer maximum replaces an FP64 one
  unsigned long long vmax = 0;
  if (i < npad) {
  double xi = 0.0, yi = 0.0;
  if (i < n) {
    xi = __ldg(locs + 2 * i);
    yi = __ldg(locs + 2 * i + 1);
  }
  for (int s = 0; s < 16; ++s) {
    const int64_t j = (int64_t)tj * 64 + (threadIdx.x >> 6) + 4 * s;
    if (j > i || j >= npad) continue;
    double v;
    if (i >= n || j >= n) {
      v = (i == j) ? 1.0 : 0.0;  // identity padding
    } else if (i == j) {
      v = P.sigma2 + P.nugget;
    } else {
      const double r2 = model_dist2(P, xi, yi, __ldg(locs + 2 * j), __ldg(locs + 2 * j + 1));
      v = tab ? matern_value_tab(P, tab, r2) : matern_value_exact(P, sqrt(r2));
      const unsigned long long vb = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
      vmax = vb > vmax && vb <= 0x7FF0000000000000ull ? vb : vmax;  // NaN skipped, as fmax does
    }
    a[i + j * ld] = v;
    if (a2) a2[i + j * ld] = v;
  }
  }
  if (offmax) {
    // non-negative doubles order like their bit patterns: one atomicMax per warp
    unsigned long long b = vmax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, b, o);
      b = ob > b ? ob : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&offmax[(ti >> oshift) - (tj >> oshift)], b);
  }
}

cudaError_t launch_matern_gen(cudaStream_t s, const double* locs, int64_t n, int64_t npad, const MaternParams& p,
                              double* a, int64_t ld, unsigned long long* offmax, const MaternTable* tab, int panel,
                              double* a2) {
  const int oshift = panel == 512 ? 3 : 2;  // 64-row generator tiles per panel tile: 2^oshift
  const long long t = (npad + 63) / 64;
  const long long blocks = t * (t + 1) / 2;
  if (blocks <= 0) return cudaSuccess;
  matern_gen_kernel<<<(unsigned)blocks, 256, 0, s>>>(locs, n, npad, p, a, ld, offmax, tab, oshift, a2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Table construction (the per-segment arithmetic lives in bessel.cuh, shared
// with the batched form's per-replicate tables).
// ---------------------------------------------------------------------------
__global__ void matern_table_nodes_kernel(const __grid_constant__ MaternParams P, double* __restrict__ nodes) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= kTabSeg * (kTabDeg + 1)) return;
  nodes[id] = table_node_value(P, id);
}

__global__ void matern_table_coef_kernel(const double* __restrict__ nodes, MaternTable* __restrict__ T) {
  const int sgi = blockIdx.x * blockDim.x + threadIdx.x;
  if (sgi >= kTabSeg) return;
  table_segment_coefs(nodes, sgi, T);
}

cudaError_t launch_matern_table(cudaStream_t s, const MaternParams& p, MaternTable* tab, double* nodes) {
  const int total = kTabSeg * (kTabDeg + 1);
  matern_table_nodes_kernel<<<(total + 127) / 128, 128, 0, s>>>(p, nodes);
  matern_table_coef_kernel<<<(kTabSeg + 127) / 128, 128, 0, s>>>(nodes, tab);
  return cudaGetLastError();
}

}  // namespace exa
