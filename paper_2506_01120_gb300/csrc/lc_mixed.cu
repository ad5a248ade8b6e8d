// Mixed-precision helpers of the screening path:
//  * split_rows    -- new FP64 basis rows -> BF16 hi/lo copies, row-major
//                     (operand of the projection beta = H V^T) and transposed
//                     (operand of the residual R = H - beta V);
//  * bracket_mixed -- brackets of a block of pairs in FP32, written as split
//                     BF16 candidate rows plus FP32 squared norms.
#include "lc_internal.cuh"

namespace lc {
namespace {

__device__ __forceinline__ void split_bf16(double x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __double2bfloat16(x);
  lo = __double2bfloat16(x - (double)__bfloat162float(hi));
}

__device__ __forceinline__ void split_bf16f(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// 32 x 32 tiles: coalesced reads of V rows, coalesced writes of both copies.
__global__ void k_split_rows(const double* __restrict__ V, int ldv, int r0, int r1, int P,
                             __nv_bfloat16* __restrict__ Vhi, __nv_bfloat16* __restrict__ Vlo, int ldvs,
                             __nv_bfloat16* __restrict__ VThi, __nv_bfloat16* __restrict__ VTlo, int ldvt) {
  __shared__ __nv_bfloat16 th[32][33], tl[32][33];
  const int p0 = blockIdx.x * 32, i0 = r0 + blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int yy = ty; yy < 32; yy += 8) {
    const int i = i0 + yy, p = p0 + tx;
    __nv_bfloat16 hi = __float2bfloat16_rn(0.f), lo = hi;
    if (i < r1 && p < P) {
      split_bf16(V[(long long)i * ldv + p], hi, lo);
      Vhi[(long long)i * ldvs + p] = hi;
      Vlo[(long long)i * ldvs + p] = lo;
    }
    th[yy][tx] = hi;
    tl[yy][tx] = lo;
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    const int p = p0 + yy, i = i0 + tx;
    if (i < r1 && p < P) {
      VThi[(long long)p * ldvt + i] = th[tx][yy];
      VTlo[(long long)p * ldvt + i] = tl[tx][yy];
    }
  }
}

// FP32 bracket: same tiling as the FP64 kernel (tile pair (I, J), I <= J).
constexpr int BT = 32;
constexpr int BQ = 16;

__device__ __forceinline__ float2 herm_elem_f(const double* __restrict__ S, int d, int r, int c, double s1, double s2) {
  if (r >= d || c >= d) return make_float2(0.f, 0.f);
  if (r == c) return make_float2((float)(S[(long long)r * d + r] * s1), 0.f);
  if (r < c) return make_float2((float)(S[(long long)r * d + c] * s2), (float)(S[(long long)c * d + r] * s2));
  return make_float2((float)(S[(long long)c * d + r] * s2), (float)(-S[(long long)r * d + c] * s2));
}

__device__ __forceinline__ void cmacf(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

__global__ void __launch_bounds__(256) k_bracket_mixed(const double* __restrict__ V, int d, int ldv, long long t0,
                                                       __nv_bfloat16* __restrict__ Hhi, __nv_bfloat16* __restrict__ Hlo,
                                                       int ldh, float* __restrict__ hn2) {
  __shared__ float2 sAI[BT][BQ + 1], sAJ[BT][BQ + 1], sBI[BQ][BT + 1], sBJ[BQ][BT + 1];
  __shared__ float red[8];
  const int pair = blockIdx.y;
  int l, m;
  pair_from_index(t0 + pair, &l, &m);
  const double* SA = V + (long long)l * ldv;
  const double* SB = V + (long long)m * ldv;
  const int nt = (d + BT - 1) / BT;
  int tp = blockIdx.x, I = 0;
  while (tp >= nt - I) { tp -= nt - I; ++I; }
  const int J = I + tp;
  const double s1 = sqrt((double)d), s2 = sqrt((double)d / 2.0);
  const int tid = threadIdx.x;
  const int jj = tid >> 3, kk0 = (tid & 7) * 4;
  float2 c1[4], c2[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) { c1[u] = make_float2(0.f, 0.f); c2[u] = make_float2(0.f, 0.f); }
  for (int q0 = 0; q0 < d; q0 += BQ) {
    for (int e = tid; e < BT * BQ; e += 256) {
      const int r = e / BQ, c = e % BQ;
      sAI[r][c] = herm_elem_f(SA, d, I * BT + r, q0 + c, s1, s2);
      sAJ[r][c] = herm_elem_f(SA, d, J * BT + r, q0 + c, s1, s2);
      const int rb = e / BT, cb = e % BT;
      sBI[rb][cb] = herm_elem_f(SB, d, q0 + rb, I * BT + cb, s1, s2);
      sBJ[rb][cb] = herm_elem_f(SB, d, q0 + rb, J * BT + cb, s1, s2);
    }
    __syncthreads();
#pragma unroll 4
    for (int q = 0; q < BQ; ++q) {
      const float2 a1 = sAI[jj][q];
      const float2 b2 = sBI[q][jj];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        cmacf(c1[u], a1, sBJ[q][kk0 + u]);
        cmacf(c2[u], sAJ[kk0 + u][q], b2);
      }
    }
    __syncthreads();
  }
  __nv_bfloat16* Oh = Hhi + (long long)pair * ldh;
  __nv_bfloat16* Ol = Hlo + (long long)pair * ldh;
  const float o1 = (float)(1.0 / sqrt((double)d)), o2 = (float)sqrt(2.0 / (double)d);
  float ss = 0.f;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = I * BT + jj, k = J * BT + kk0 + u;
    if (j >= d || k >= d) continue;
    __nv_bfloat16 hi, lo;
    if (j < k) {
      const float re = -(c1[u].y + c2[u].y) * o2;
      const float im = (c1[u].x - c2[u].x) * o2;
      split_bf16f(re, hi, lo);
      Oh[(long long)j * d + k] = hi;
      Ol[(long long)j * d + k] = lo;
      split_bf16f(im, hi, lo);
      Oh[(long long)k * d + j] = hi;
      Ol[(long long)k * d + j] = lo;
      ss = fmaf(re, re, fmaf(im, im, ss));
    } else if (j == k) {
      const float dg = -2.f * c1[u].y * o1;
      split_bf16f(dg, hi, lo);
      Oh[(long long)j * d + j] = hi;
      Ol[(long long)j * d + j] = lo;
      ss = fmaf(dg, dg, ss);
    }
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if ((tid & 31) == 0) red[tid >> 5] = ss;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < 8; ++w) t += red[w];
    atomicAdd(&hn2[pair], t);
  }
}

}  // namespace

cudaError_t split_rows(const double* V, int ldv, int r0, int r1, int P, __nv_bfloat16* Vhi, __nv_bfloat16* Vlo,
                       int ldvs, __nv_bfloat16* VThi, __nv_bfloat16* VTlo, int ldvt, cudaStream_t s) {
  if (r1 <= r0) return cudaSuccess;
  dim3 grid((P + 31) / 32, (r1 - r0 + 31) / 32);
  k_split_rows<<<grid, 256, 0, s>>>(V, ldv, r0, r1, P, Vhi, Vlo, ldvs, VThi, VTlo, ldvt);
  return cudaGetLastError();
}

cudaError_t bracket_mixed(const double* V, int d, int ldv, long long t0, int count, __nv_bfloat16* Hhi,
                          __nv_bfloat16* Hlo, int ldh, float* hn2, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(hn2, 0, sizeof(float) * count, s);
  if (e != cudaSuccess) return e;
  const int nt = (d + BT - 1) / BT;
  dim3 grid(nt * (nt + 1) / 2, count);
  k_bracket_mixed<<<grid, 256, 0, s>>>(V, d, ldv, t0, Hhi, Hlo, ldh, hn2);
  return cudaGetLastError();
}

}  // namespace lc

// ------------------------------------------------ embeddings and compaction
namespace lc {
namespace {

// E[i] = [[Hr, -Hi], [-Hi, -Hr]] (R x R, R = 2d, split BF16) for basis rows
// i in [r0, r1), with H the Hermitian part of V[i] = iH unpacked from the
// packed FP64 row.
// With perm != 0 the rows are stored in the order used by the large-d
// bracket kernel: stored row 128c + w holds E row 64c + w (w < 64) and stored
// row 128c + 64 + w holds E row d + 64c + w.
__global__ void k_build_embedding(const double* __restrict__ V, int ldv, int r0, int r1, int d, int perm,
                                  __nv_bfloat16* __restrict__ Ehi, __nv_bfloat16* __restrict__ Elo) {
  const int R = 2 * d;
  const long long per = (long long)R * R;
  const long long tot = per * (r1 - r0);
  const double s1 = sqrt((double)d), s2 = sqrt((double)d / 2.0);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = r0 + e / per;
    const int r = (int)((e / R) % R), b = (int)(e % R);
    const int a = perm ? (((r & 127) < 64) ? 64 * (r >> 7) + (r & 127) : d + 64 * (r >> 7) + (r & 127) - 64) : r;
    const int ja = a % d, jb = b % d;
    const double* S = V + i * ldv;
    double hr, hi;
    if (ja == jb)      { hr = S[(long long)ja * d + ja] * s1; hi = 0.0; }
    else if (ja < jb)  { hr = S[(long long)ja * d + jb] * s2; hi = S[(long long)jb * d + ja] * s2; }
    else               { hr = S[(long long)jb * d + ja] * s2; hi = -S[(long long)ja * d + jb] * s2; }
    const bool top = a < d, left = b < d;
    const double v = (top && left) ? hr : ((top != left) ? -hi : -hr);
    __nv_bfloat16 h, lo;
    split_bf16(v, h, lo);
    const long long o = (i * R + r) * R + b;
    Ehi[o] = h;
    Elo[o] = lo;
  }
}

// Q[i] = [Hr; Hi] (2d x d, split BF16) for basis rows i in [r0, r1)
__global__ void k_build_q(const double* __restrict__ V, int ldv, int r0, int r1, int d,
                          __nv_bfloat16* __restrict__ Qhi, __nv_bfloat16* __restrict__ Qlo) {
  const long long per = 2LL * d * d;
  const long long tot = per * (r1 - r0);
  const double s1 = sqrt((double)d), s2 = sqrt((double)d / 2.0);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = r0 + e / per;
    const int a = (int)((e / d) % (2 * d)), b = (int)(e % d);
    const int ja = a % d;
    const double* S = V + i * ldv;
    double hr, hi;
    if (ja == b)      { hr = S[(long long)ja * d + ja] * s1; hi = 0.0; }
    else if (ja < b)  { hr = S[(long long)ja * d + b] * s2; hi = S[(long long)b * d + ja] * s2; }
    else              { hr = S[(long long)b * d + ja] * s2; hi = -S[(long long)ja * d + b] * s2; }
    __nv_bfloat16 h, lo;
    split_bf16(a < d ? hr : hi, h, lo);
    const long long o = i * per + (long long)a * d + b;
    Qhi[o] = h;
    Qlo[o] = lo;
  }
}

// ordered list of candidates with hn2 > eta2 (one CTA of 1024 threads)
__global__ void __launch_bounds__(1024) k_compact_nonzero(const float* __restrict__ hn2, int count, float eta2,
                                                          int* __restrict__ nz_idx, int* __restrict__ nnz,
                                                          const double* __restrict__ bn2, long long t0) {
  __shared__ int wsum[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c0 = 0; c0 < count; c0 += 1024) {
    const int c = c0 + threadIdx.x;
    int f = 0;
    if (c < count) {
      float floor2 = eta2;
      if (bn2) {
        int l, m;
        pair_from_index(t0 + c, &l, &m);
        floor2 = (float)((double)eta2 * bn2[l] * bn2[m]);
      }
      f = hn2[c] > floor2 ? 1 : 0;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, f);
    const int pre = __popc(mask & ((1u << lane) - 1u));
    if (lane == 0) wsum[w] = __popc(mask);
    __syncthreads();
    if (w == 0) {
      int v = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
      }
      wsum[lane] = v;
    }
    __syncthreads();
    if (f) nz_idx[base + (w ? wsum[w - 1] : 0) + pre] = c;
    __syncthreads();
    if (threadIdx.x == 0) base += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *nnz = base;
}

__device__ __forceinline__ int nonzero_flag(const float* hn2, int c, float eta2, const double* bn2, long long t0) {
  float floor2 = eta2;
  if (bn2) {
    int l, m;
    pair_from_index(t0 + c, &l, &m);
    floor2 = (float)((double)eta2 * bn2[l] * bn2[m]);
  }
  return hn2[c] > floor2 ? 1 : 0;
}

// two-pass forms of k_compact_nonzero (see cta_excl_scan)
__global__ void __launch_bounds__(kCmpThreads) k_nonzero_pass1(const float* __restrict__ hn2, int count, float eta2,
                                                            const double* __restrict__ bn2, long long t0,
                                                            int* __restrict__ part) {
  __shared__ int sw[kCmpThreads / 32];
  const int chunk = (count + gridDim.x - 1) / gridDim.x;
  const int c0 = blockIdx.x * chunk, c1 = min(count, c0 + chunk);
  int n = 0;
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) n += nonzero_flag(hn2, c, eta2, bn2, t0);
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int i = 0; i < kCmpThreads / 32; ++i) t += sw[i];
    part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kCmpThreads) k_nonzero_pass2(const float* __restrict__ hn2, int count, float eta2,
                                                            const double* __restrict__ bn2, long long t0,
                                                            int* __restrict__ nz_idx, int* __restrict__ nnz,
                                                            const int* __restrict__ part) {
  __shared__ int wsum[kCmpThreads / 32];
  __shared__ int base;
  const int chunk = (count + gridDim.x - 1) / gridDim.x;
  const int c0 = blockIdx.x * chunk, c1 = min(count, c0 + chunk);
  if (threadIdx.x == 0) {
    int o = 0;
    for (int b = 0; b < (int)blockIdx.x; ++b) o += part[b];
    base = o;
    if (blockIdx.x == 0) {
      int t = 0;
      for (int b = 0; b < (int)gridDim.x; ++b) t += part[b];
      *nnz = t;
    }
  }
  __syncthreads();
  for (int tt = c0; tt < c1; tt += blockDim.x) {
    const int c = tt + threadIdx.x;
    const int f = c < c1 ? nonzero_flag(hn2, c, eta2, bn2, t0) : 0;
    int tot;
    const int at = base + cta_excl_scan(f, &tot, wsum);
    if (f) nz_idx[at] = c;
    if (threadIdx.x == 0) base += tot;
    __syncthreads();
  }
}

// row i of the compacted block <- row nz_idx[i] (16-byte vectors)
__global__ void k_gather_candidates(const __nv_bfloat16* __restrict__ Hhi, const __nv_bfloat16* __restrict__ Hlo,
                                    int ldh, const float* __restrict__ hn2, const int* __restrict__ nz_idx,
                                    const int* __restrict__ nnz, int ncols, __nv_bfloat16* __restrict__ Chi,
                                    __nv_bfloat16* __restrict__ Clo, float* __restrict__ hn2c) {
  const int i = blockIdx.x;
  if (i >= *nnz) return;
  const int src = nz_idx[i];
  const uint4* sh = reinterpret_cast<const uint4*>(Hhi + (long long)src * ldh);
  const uint4* sl = reinterpret_cast<const uint4*>(Hlo + (long long)src * ldh);
  uint4* dh = reinterpret_cast<uint4*>(Chi + (long long)i * ldh);
  uint4* dl = reinterpret_cast<uint4*>(Clo + (long long)i * ldh);
  for (int v = threadIdx.x; v < ncols / 8; v += blockDim.x) {
    dh[v] = sh[v];
    dl[v] = sl[v];
  }
  if (threadIdx.x == 0) hn2c[i] = hn2[src];
}

}  // namespace

cudaError_t build_embedding(const double* V, int ldv, int r0, int r1, int d, __nv_bfloat16* Ehi,
                            __nv_bfloat16* Elo, cudaStream_t s, int perm) {
  if (r1 <= r0) return cudaSuccess;
  const long long tot = 4LL * d * d * (r1 - r0);
  long long g = (tot + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_build_embedding<<<(int)g, 256, 0, s>>>(V, ldv, r0, r1, d, perm, Ehi, Elo);
  return cudaGetLastError();
}

cudaError_t build_q(const double* V, int ldv, int r0, int r1, int d, __nv_bfloat16* Qhi, __nv_bfloat16* Qlo,
                    cudaStream_t s) {
  if (r1 <= r0) return cudaSuccess;
  const long long tot = 2LL * d * d * (r1 - r0);
  long long g = (tot + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  k_build_q<<<(int)g, 256, 0, s>>>(V, ldv, r0, r1, d, Qhi, Qlo);
  return cudaGetLastError();
}

cudaError_t compact_nonzero(const float* hn2, int count, float eta2, int* nz_idx, int* nnz, cudaStream_t s,
                            const double* bn2, long long t0, int* part) {
  if (part) {
    k_nonzero_pass1<<<kCmpCtas, kCmpThreads, 0, s>>>(hn2, count, eta2, bn2, t0, part);
    k_nonzero_pass2<<<kCmpCtas, kCmpThreads, 0, s>>>(hn2, count, eta2, bn2, t0, nz_idx, nnz, part);
    return cudaGetLastError();
  }
  k_compact_nonzero<<<1, 1024, 0, s>>>(hn2, count, eta2, nz_idx, nnz, bn2, t0);
  return cudaGetLastError();
}

cudaError_t gather_candidates(const __nv_bfloat16* Hhi, const __nv_bfloat16* Hlo, int ldh, const float* hn2,
                              const int* nz_idx, const int* nnz, int count, int ncols, __nv_bfloat16* Chi,
                              __nv_bfloat16* Clo, float* hn2c, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_gather_candidates<<<count, 256, 0, s>>>(Hhi, Hlo, ldh, hn2, nz_idx, nnz, ncols, Chi, Clo, hn2c);
  return cudaGetLastError();
}

// beta[i][j] = hi + lo of the screening GEMM's coefficient <h_c, v_j> of the
// flagged row i (compacted position c = cidx[i]), j < n, in FP64
__global__ void k_gather_coef(const __nv_bfloat16* __restrict__ Dhi, const __nv_bfloat16* __restrict__ Dlo, int ldd,
                              const int* __restrict__ cidx, int f, int n, double* __restrict__ beta, int ldb) {
  for (int i = blockIdx.y; i < f; i += gridDim.y) {
    const long long c = cidx[i];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
      beta[(long long)i * ldb + j] =
          (double)__bfloat162float(Dhi[c * ldd + j]) + (double)__bfloat162float(Dlo[c * ldd + j]);
  }
}

cudaError_t gather_coef(const __nv_bfloat16* Dhi, const __nv_bfloat16* Dlo, int ldd, const int* cidx, int f, int n,
                        double* beta, int ldb, cudaStream_t s) {
  if (f <= 0 || n <= 0) return cudaSuccess;
  const dim3 grid((unsigned)std::min((n + 255) / 256, 64), (unsigned)std::min(f, 65535));
  k_gather_coef<<<grid, 256, 0, s>>>(Dhi, Dlo, ldd, cidx, f, n, beta, ldb);
  return cudaGetLastError();
}

}  // namespace lc

// ------------------------------------------------------ screen noise probe
// The split-BF16 screen cannot certify a residual below its own rounding
// noise.  The probe measures that noise on vectors whose true residual is 0:
// S1 single basis rows and S - S1 combinations of 16 basis rows with random
// coefficients (both in span(V)), pushed through the same split and GEMMs as
// the candidates.  Rows are picked and weighted by splitmix64 of (seed, row).
namespace lc {
namespace {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

constexpr int PROBE_TERMS = 16;

__global__ void __launch_bounds__(256) k_probe_rows(const double* __restrict__ V, int ldv, int N, int P, int S1,
                                                    unsigned long long seed, __nv_bfloat16* __restrict__ Chi,
                                                    __nv_bfloat16* __restrict__ Clo, int ldc,
                                                    float* __restrict__ hn2c, int* __restrict__ nnz, int S) {
  __shared__ int rows[PROBE_TERMS];
  __shared__ double coef[PROBE_TERMS];
  __shared__ double red[8];
  const int j = blockIdx.x;
  if (threadIdx.x < PROBE_TERMS) {
    // every probe draws its own rows, except that for long rows (P > 2^16)
    // the combinations share one pool (drawn with the key 0xFFFF), read from
    // L2 instead of from memory once per combination.  (A shared pool at
    // small P spans too few directions: its eps came out low enough that the
    // su(128) chain flagged 3.5 times as many candidates by noise.)
    const unsigned long long key = (j < S1 || P <= (1 << 16)) ? (unsigned long long)j : 0xFFFFull;
    const unsigned long long hr = splitmix64(seed ^ splitmix64((key << 8) | threadIdx.x));
    rows[threadIdx.x] = (int)(hr % (unsigned long long)N);
    // coefficient uniform in [-1, -1/4] U [1/4, 1] (no near-cancellation of the combination)
    const unsigned long long h = splitmix64(seed ^ splitmix64(((unsigned long long)j << 8) | threadIdx.x));
    const double u = (double)(h >> 11) * (1.0 / 9007199254740992.0);
    coef[threadIdx.x] = (u < 0.5 ? -1.0 : 1.0) * (0.25 + 1.5 * fabs(u - 0.5));
  }
  __syncthreads();
  // combinations of PROBE_TERMS pool rows; of 4 for rows longer than 2^16
  const int T = j < S1 ? 1 : (P > (1 << 16) ? 4 : PROBE_TERMS);
  double ss = 0.0;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    double x = 0.0;
    for (int t = 0; t < T; ++t) x = fma(T == 1 ? 1.0 : coef[t], V[(long long)rows[t] * ldv + p], x);
    __nv_bfloat16 hi, lo;
    split_bf16(x, hi, lo);
    Chi[(long long)j * ldc + p] = hi;
    Clo[(long long)j * ldc + p] = lo;
    ss = fma(x, x, ss);
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    hn2c[j] = (float)t;
    if (j == 0) *nnz = S;
  }
}

// eps^2 = max over probes of rn2 / hn2; tau^2 = clamp(kappa^2 eps^2, lo, hi)
__global__ void k_probe_eps(const float* __restrict__ hn2c, const float* __restrict__ rn2, int S, DevStats* stats,
                            float kappa2, float tau2_lo, float tau2_hi) {
  __shared__ float wm[32];
  float m = 0.f;
  for (int j = threadIdx.x; j < S; j += blockDim.x)
    if (hn2c[j] > 0.f) m = fmaxf(m, rn2[j] / hn2c[j]);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float e2 = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) e2 = fmaxf(e2, wm[w]);
    stats->eps2 = e2;
    stats->tau2 = fminf(fmaxf(kappa2 * e2, tau2_lo), tau2_hi);
    const double e = sqrt((double)e2);
    atomicMax(&stats->eps_bits, (unsigned long long)__double_as_longlong(e));
  }
}

}  // namespace

cudaError_t probe_rows(const double* V, int ldv, int N, int P, int S, int S1, unsigned long long seed,
                       __nv_bfloat16* Chi, __nv_bfloat16* Clo, int ldc, float* hn2c, int* nnz, cudaStream_t s) {
  if (S <= 0 || N <= 0) return cudaSuccess;
  k_probe_rows<<<S, 256, 0, s>>>(V, ldv, N, P, S1, seed, Chi, Clo, ldc, hn2c, nnz, S);
  return cudaGetLastError();
}

cudaError_t probe_eps(const float* hn2c, const float* rn2, int S, DevStats* stats, float kappa, float tau_lo,
                      float tau_hi, cudaStream_t s) {
  k_probe_eps<<<1, 256, 0, s>>>(hn2c, rn2, S, stats, kappa * kappa, tau_lo * tau_lo, tau_hi * tau_hi);
  return cudaGetLastError();
}

}  // namespace lc
