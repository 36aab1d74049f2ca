// Data-movement helpers around the factorisation: padding a caller matrix
// into the workspace, copying a factor back, padding vectors, and the
// lower-triangular matrix-vector product used to draw exact realisations.
#include "exa_internal.cuh"
#include "util.cuh"

namespace exa {

// dst (npad x npad, ld_dst) lower triangle <- src (n x n, ld_src) lower triangle,
// identity in rows/cols [n, npad).
__global__ void copy_lower_pad_kernel(const double* __restrict__ src, int64_t ld_src, int64_t n, int64_t npad,
                                      double* __restrict__ dst, int64_t ld_dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  for (int64_t jj = j; jj < npad; jj += gridDim.y) {
    if (i < jj || i >= npad) continue;
    double v;
    if (i < n && jj < n)
      v = src[i + jj * ld_src];
    else
      v = (i == jj) ? 1.0 : 0.0;
    dst[i + jj * ld_dst] = v;
  }
}

cudaError_t launch_copy_lower_pad(cudaStream_t s, const double* src, int64_t ld_src, int64_t n, int64_t npad,
                                  double* dst, int64_t ld_dst) {
  dim3 grid((unsigned)((npad + 255) / 256), (unsigned)(npad < 4096 ? npad : 4096));
  copy_lower_pad_kernel<<<grid, 256, 0, s>>>(src, ld_src, n, npad, dst, ld_dst);
  return cudaGetLastError();
}

__global__ void copy_lower_back_kernel(const double* __restrict__ src, int64_t ld_src, int64_t n,
                                       double* __restrict__ dst, int64_t ld_dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t jj = blockIdx.y; jj < n; jj += gridDim.y) {
    if (i < jj || i >= n) continue;
    dst[i + jj * ld_dst] = src[i + jj * ld_src];
  }
}

cudaError_t launch_copy_lower_back(cudaStream_t s, const double* src, int64_t ld_src, int64_t n, double* dst,
                                   int64_t ld_dst) {
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)(n < 4096 ? n : 4096));
  copy_lower_back_kernel<<<grid, 256, 0, s>>>(src, ld_src, n, dst, ld_dst);
  return cudaGetLastError();
}

__global__ void pad_vector_kernel(const double* __restrict__ src, int64_t n, int64_t npad, double* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npad) dst[i] = (i < n) ? src[i] : 0.0;
}

cudaError_t launch_pad_vector(cudaStream_t s, const double* src, int64_t n, int64_t npad, double* dst) {
  pad_vector_kernel<<<(unsigned)((npad + 255) / 256), 256, 0, s>>>(src, n, npad, dst);
  return cudaGetLastError();
}

// out_i = sum_{j <= i} L_ij v_j  (column-major L), one thread per row.
__global__ void trmv_lower_kernel(const double* __restrict__ a, int64_t ld, int64_t n, const double* __restrict__ v,
                                  double* __restrict__ out, const DevStatus* st) {
  if (*(volatile const int32_t*)&st->info != 0) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t j = 0; j <= i; ++j) s = fma(a[i + j * ld], v[j], s);
  out[i] = s;
}

cudaError_t launch_trmv_lower(cudaStream_t s, const double* a, int64_t ld, int64_t n, const double* v, double* out,
                              const DevStatus* st) {
  trmv_lower_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, ld, n, v, out, st);
  return cudaGetLastError();
}

}  // namespace exa
