/*
 * lieclosure_kernels.h -- unit-level entry points of the GB300 Lie-closure
 * library, for testing and profiling the kernels of the hot path in
 * isolation.  Same conventions as lieclosure.h (status codes, visibility).
 */
#ifndef LIECLOSURE_KERNELS_H
#define LIECLOSURE_KERNELS_H

#include "lieclosure.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * lc_split_gemm_f32 -- D = A B^T through the split-BF16 tcgen05 GEMM that the
 * projection (beta = H V^T, the inner products of Section 3.2) and the
 * residual (h - proj_V h) of the screening step run on.
 *
 * A : M x K FP32, row-major, device pointer (row stride K).
 * B : N x K FP32, row-major, device pointer (row stride K).
 * D : M x N FP32, row-major, device pointer (row stride N), written.
 * Each operand is split on the device into BF16 hi + lo parts and the product
 * is Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T accumulated in FP32 (relative error
 * about 2^-16 per product).  Any M, N, K >= 1; the library pads to its tile
 * sizes in a workspace it allocates and frees within the call.
 * stream : cudaStream_t as void* (NULL = legacy default stream); the call
 * returns after the stream has finished.
 * Returns LC_OK, LC_ERR_ARG, LC_ERR_OOM, LC_ERR_CUDA or LC_ERR_TIMEOUT.
 */
LC_API int lc_split_gemm_f32(const float* A, const float* B, int M, int N, int K, float* D, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LIECLOSURE_KERNELS_H */
