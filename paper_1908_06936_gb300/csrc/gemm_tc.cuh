// Tensor-core (tcgen05) split-precision GEMM kernels and their operand formats.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "exa_internal.cuh"

namespace exa {

constexpr int kOzSlices = 5;  // 7-bit digits per value in the exact (band) products
constexpr int kSplitMaxK = 512;  // longest row the split kernel converts
constexpr int kSplitRows = 16;   // rows per CTA of the split kernel

// Tile enumeration of one launch (kEnumTasks: T3 only, tile t described by GemmArgs::tasks[t]).
enum : int { kEnumFull = 0, kEnumLowerOffBand = 1, kEnumBand = 2, kEnumTasks = 3 };

// One 128 x 128 output tile of a grouped T3 launch: C (column-major, ldc) -= / = A B^T with the
// tile's A rows from a_row and B rows from b_row of the launch's operands; lower != 0 writes only
// entries on or below the tile's diagonal.
struct TcTask {
  double* C;
  int64_t ldc;
  int a_row, b_row;
  int lower, pad;
};

// One piece of a batched split: rows [0, rows) of src (element (r, k) at src[r rs + k cs]) to
// operand rows [out_row0, out_row0 + rows).
struct SplitTask {
  const double* src;
  int64_t rs, cs;
  int rows, out_row0;
};
constexpr int kRasterSuper = 16;  // supertile edge (in 128-tiles) of the lower off-band enumeration
constexpr int kPairSuper = 16;    // supertile edge (in 256-tiles) of the CTA-pair lower off-band enumeration

struct OzMaps {
  CUtensorMap m[kOzSlices];
};

// Kernel arguments (passed by value as a __grid_constant__).
struct GemmArgs {
  double* C;                  // FP64 output, column-major
  int64_t ldc;
  int64_t c_row0, c_col0;     // output origin
  int a_row0, b_row0;         // operand row origins
  int K;                      // reduction length (T3: % 32, OZ: % 64 and <= 512, its exact-sum limit)
  int enum_mode;              // kEnum*
  int nt;                     // tiles along N (kEnumFull); tile rows (kEnumLowerOffBand)
  int band;                   // band width in panel tiles (kEnumLowerOffBand / kEnumBand)
  int panel;                  // panel width (256 or 512) that `band` is measured in
  long long ntiles;           // number of enumerated tiles
  int store;                  // 1: C = A B^T ; 0: C -= A B^T
  int lower_mask;             // skip entries above the diagonal
  const int* ea;              // OZ: per-row power-of-two exponents of A (set by the launcher)
  const int* eb;              // OZ: per-row exponents of B
  // T3 on CTA pairs: with far_thr set (> INT_MIN), a 256 x 256 tile whose operand blocks have
  // maximum exponents eA + eB <= far_thr takes the single hi * hi product (see the kernel)
  const int* ea_blk;          // per 256-row block maximum exponent of A
  const int* eb_blk;          // per 256-row block maximum exponent of B
  int far_thr;
  // T3 on CTA pairs only: a second operand pair (A2, B2) reduced into the same tile after
  // the first, K2 more columns (0: none), rows from a2_row0 / b2_row0, with its own
  // block exponents for the far-tile test.
  int K2;
  int a2_row0, b2_row0;
  const int* ea2_blk;
  const int* eb2_blk;
  const TcTask* tasks;        // kEnumTasks: device array of ntiles tile descriptions (T3 only)
  DevStatus* st;
};

// One split operand: `rows` x K values held as T3 (tf32 hi/lo, row-major) and/or
// OZ digits (kOzSlices planes of rows x K BF16, row-major) with row exponents.
struct SplitOperand {
  int64_t rows = 0;
  int K = 0;
  float* hi = nullptr;
  float* lo = nullptr;
  void* dig = nullptr;
  int* ex = nullptr;
  int* exb = nullptr;         // per 256-row block maximum of ex
  CUtensorMap t_hi, t_lo;     // boxes 32 x 128
  OzMaps oz_a;                // boxes 64 x 128 (A role)
  OzMaps oz_b;                // boxes 64 x 32  (B role)
  OzMaps oz_ah;               // boxes 64 x 64  (A role, half a tile: multicast by a CTA pair)
  OzMaps oz_b48;              // boxes 64 x 48  (B role, 48-wide band tiles)
};

cudaError_t make_split_maps(SplitOperand& op);
// exb[b] = max(ex[256 b .. 256 b + 255]) over the first `rows` rows
cudaError_t launch_row_exp_blockmax(cudaStream_t s, SplitOperand& op, int64_t rows);
// rows [0, rows) of src (element (r, k) at src[r*rs + k*cs]) -> operand rows [out_row0, ...)
cudaError_t launch_split_rows(cudaStream_t s, const double* src, int64_t rs, int64_t cs, int rows, int K,
                              SplitOperand& op, int out_row0);
// ntasks pieces in one launch (max_rows: the longest piece), each to its own operand rows.
cudaError_t launch_split_rows_tasks(cudaStream_t s, const SplitTask* d_tasks, int ntasks, int max_rows, int K,
                                    SplitOperand& op);
// max_ctas > 0 caps the persistent grid (to leave SMs to concurrent work).
cudaError_t launch_gemm_t3(cudaStream_t s, const SplitOperand& A, const SplitOperand& B, const GemmArgs& g,
                           int max_ctas = 0);
cudaError_t launch_gemm_oz(cudaStream_t s, const SplitOperand& A, const SplitOperand& B, const GemmArgs& g,
                           int max_ctas = 0);
// T3 on CTA pairs, 256 x 256 tiles (kEnumFull with g.nt = n / 256, or kEnumLowerOffBand with
// g.nt = tile rows of 256); no lower_mask.  Uses pairs of SMs (max_ctas rounded down to even).
// With g.K2 > 0 each tile also takes -= A2 B2^T (K2 columns) in the same accumulator.
cudaError_t launch_gemm_t3_pair(cudaStream_t s, const SplitOperand& A, const SplitOperand& B, const GemmArgs& g,
                                int max_ctas = 0, const SplitOperand* A2 = nullptr,
                                const SplitOperand* B2 = nullptr);
int tc_num_sms();

}  // namespace exa
