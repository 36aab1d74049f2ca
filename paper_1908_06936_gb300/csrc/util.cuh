// Launchers of the data-movement helpers in util.cu.
#pragma once
#include "exa_internal.cuh"

namespace exa {
cudaError_t launch_copy_lower_pad(cudaStream_t s, const double* src, int64_t ld_src, int64_t n, int64_t npad,
                                  double* dst, int64_t ld_dst);
cudaError_t launch_copy_lower_back(cudaStream_t s, const double* src, int64_t ld_src, int64_t n, double* dst,
                                   int64_t ld_dst);
cudaError_t launch_pad_vector(cudaStream_t s, const double* src, int64_t n, int64_t npad, double* dst);
cudaError_t launch_trmv_lower(cudaStream_t s, const double* a, int64_t ld, int64_t n, const double* v, double* out,
                              const DevStatus* st);
}  // namespace exa
