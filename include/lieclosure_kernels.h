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

/*
 * lc_gemm_f64_tc -- C = A B^T to FP64 accuracy on the BF16 tensor cores: the
 * product the FP64 Gram-Schmidt of the accept step (c = R V^T, R -= c V,
 * Section 3.2) runs on in mixed mode.  Each row is scaled by a power of two
 * and cut into S balanced base-2^beta digit slices, exact in BF16
 * (beta = 7, S = 8 for K <= 4096; beta = 6, S = 9 above); every slice pair
 * with s + t <= S - 1 is one tcgen05.mma chain whose FP32 accumulation is
 * exact (K 2^{2 beta - 2} <= 2^24 per chain; longer K is split), and the
 * chains are summed in FP64.  The error is of the order of 2^-53 times the
 * row-scale bound K max|a_i.| max|b_j.|, like an FP64 dot product's.
 *
 * A : M x K FP64, row-major, device pointer (row stride K).
 * B : N x K FP64, row-major, device pointer (row stride K).
 * C : M x N FP64, row-major, device pointer (row stride N), written.
 * Any M, N, K >= 1.  Workspace (slices, partials) is allocated and freed
 * within the call on `stream` (cudaStream_t as void*, NULL = legacy default);
 * the call returns after the stream has finished.
 * Returns LC_OK, LC_ERR_ARG, LC_ERR_OOM, LC_ERR_CUDA or LC_ERR_TIMEOUT.
 */
LC_API int lc_gemm_f64_tc(const double* A, const double* B, int M, int N, int K, double* C, void* stream);

/*
 * lc_split_gemm_f32_noalloc -- lc_split_gemm_f32 without any device memory
 * allocation.  The paper has no counterpart; this exists for callers that
 * cannot let a library allocate: a process whose own pool already owns the
 * free device memory, code under a hard memory cap, or a path where
 * cudaMalloc/cudaFree (which may synchronise the device) is not allowed.
 *
 * Arguments and result are those of lc_split_gemm_f32.  The workspace is one
 * fixed 32 MiB array in device global memory, created on every GPU that loads
 * the library and kept until the process exits.  The padded problem must fit
 * in it: 4 (Mp Kp + Np Kp) + 4 Mp Np bytes plus a little alignment, with
 * Mp = M rounded up to 128, Np = N rounded up to 256 and Kp = K rounded up to
 * 32 (for example M = N = K = 1024 fits); larger problems return
 * LC_ERR_TOO_LARGE without touching the GPU.
 * Returns LC_OK, LC_ERR_ARG (null pointer or an extent < 1),
 * LC_ERR_TOO_LARGE, LC_ERR_CUDA or LC_ERR_TIMEOUT; never LC_ERR_OOM, since it
 * allocates nothing.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.
 * All calls share the one array and it keeps the last call's contents; the
 * call clears what must start at zero.  Calls that overlap on the GPU (for
 * example on two streams at once) race on the array and give wrong results.
 */
LC_API int lc_split_gemm_f32_noalloc(const float* A, const float* B, int M, int N, int K, float* D,
                                     void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LIECLOSURE_KERNELS_H */
