// Digit slicing of FP64 values for the FP64-accurate tensor-core GEMM
// (k_ozaki_gemm): error-free splitting in the manner of Ozaki, Ogita, Oishi
// and Rump (2012), built on exact FP32 accumulation of BF16 digits.
//
// A row x of an operand is written as x = 2^e sum_{s<S} d_s 2^(-beta (s+1))
// + (a remainder below 2^(e - beta S - 1)), with integer digits
// |d_s| <= 2^(beta-1), each exact in BF16.  The functions are host and
// device code so that the host-side tests exercise the same arithmetic the
// kernels run.  Everything here is integer arithmetic on the FP64 bits (the
// FP64 pipe is the slowest pipe of the part).
#pragma once

#include <cuda_bf16.h>
#include <cstring>

namespace lc {

__host__ __device__ __forceinline__ long long oz_bits(double x) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(x);
#else
  long long b;
  memcpy(&b, &x, sizeof(b));
  return b;
#endif
}

// x 2^shift rounded to the nearest integer (halves away from zero), from
// x's bits.  Zero and subnormal inputs give 0 (they lie far below any digit
// kept).  Callers keep |x 2^shift| <= 2^55.
__host__ __device__ __forceinline__ long long oz_fixed(double x, int shift) {
  const long long b = oz_bits(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0) return 0;
  const long long m = (b & ((1LL << 52) - 1)) | (1LL << 52);   // |x| = m 2^(ex - 1075)
  const int sh = ex - 1075 + shift;
  long long v;
  if (sh >= 0) v = m << sh;
  else if (sh < -53) v = 0;                     // below 1/2
  else v = (m + (1LL << (-sh - 1))) >> (-sh);   // round half up (in magnitude)
  return b < 0 ? -v : v;
}

// S balanced base-2^beta digits of Y = round(x 2^(beta S - e)), |Y| <=
// 2^(beta S - 1): from the least significant, d = Y mod 2^beta in
// [-2^(beta-1), 2^(beta-1)), Y = (Y - d) / 2^beta; the top digit is what
// is left, within 2^(beta-1) in magnitude (it may equal +-2^(beta-1)).
// Slice s (weight 2^(-beta (s+1))) at out[s * sstride].
__host__ __device__ __forceinline__ void oz_digits(double x, int e, int S, int beta, __nv_bfloat16* out,
                                                   long long sstride) {
  long long Y = oz_fixed(x, beta * S - e);
  const long long half = 1LL << (beta - 1), mask = (1LL << beta) - 1;
  for (int s = S - 1; s >= 1; --s) {
    const long long d = ((Y + half) & mask) - half;
    Y = (Y - d) >> beta;
    out[s * sstride] = __float2bfloat16_rn((float)d);
  }
  out[0] = __float2bfloat16_rn((float)Y);   // the rest, |Y| <= 2^(beta-1)
}

// The same for two neighbouring entries, stored as BF16 pairs (one 4-byte
// store per slice for both).
__host__ __device__ __forceinline__ void oz_digits2(double x0, double x1, int e, int S, int beta,
                                                    __nv_bfloat162* out, long long sstride2) {
  long long Y0 = oz_fixed(x0, beta * S - e), Y1 = oz_fixed(x1, beta * S - e);
  const long long half = 1LL << (beta - 1), mask = (1LL << beta) - 1;
  for (int s = S - 1; s >= 1; --s) {
    const long long d0 = ((Y0 + half) & mask) - half, d1 = ((Y1 + half) & mask) - half;
    Y0 = (Y0 - d0) >> beta;
    Y1 = (Y1 - d1) >> beta;
    out[s * sstride2] = __floats2bfloat162_rn((float)d0, (float)d1);
  }
  out[0] = __floats2bfloat162_rn((float)Y0, (float)Y1);
}

// exponent e with |x| 2^-e < 1/2 for the largest |x| of a row, from the bits
// of max |x| (non-negative doubles order as their bit patterns); 0 for a zero
// (or subnormal) row
__host__ __device__ __forceinline__ int oz_row_exp(long long maxbits) {
  const int ex = (int)((maxbits >> 52) & 0x7FF);
  return ex == 0 ? 0 : ex - 1023 + 2;
}

}  // namespace lc
