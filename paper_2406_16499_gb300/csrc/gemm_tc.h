// gemm_tc.h -- host interface of the tcgen05 GEMM (gemm_tc.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstddef>

namespace mpir {

enum { TCM_TF32 = 0, TCM_TF32X3 = 1, TCM_BF16 = 2 };
enum { TCE_STORE = 0, TCE_SUB = 1 };

// Tensor map of a column-major FP32 matrix (rows contiguous, ld elements,
// ld*4 a multiple of 16, base 16-byte aligned); box 32 rows x box_cols.
int tmap_colmajor(CUtensorMap *tm, const float *base, long rows, long cols, long ld, int box_cols);

// D (M x N) = A (M x K) B (N x K)^T with A and B K-major (the tensor maps'
// row dimension is K).  A tile (m, k) is read at coordinates
// (a_x0 + k, a_y0 + m), B tile (n, k) at (b_x0 + k, b_y0 + n).
// mode: TCM_TF32, TCM_TF32X3 (A2 = A_lo map; B2 = B_lo map unless
// bsplit = 1, which splits B in shared memory) or TCM_BF16 (FP32 tiles
// rounded to bfloat16 in shared memory, kind::f16 MMAs with FP32
// accumulation; A2, B2 and bsplit unused).  epi: TCE_STORE writes split
// z of K to out + z*split_stride (column-major, ldo); TCE_SUB does out -= D.
int gemm_tc(int mode, int bsplit, int epi, const CUtensorMap &A, const CUtensorMap &A2, const CUtensorMap &B,
            const CUtensorMap &B2, int a_x0, int a_y0, int b_x0, int b_y0, int M, int N, int K, float *out,
            int ldo, size_t split_stride, int nsplit, int *err, cudaStream_t s);

} // namespace mpir
