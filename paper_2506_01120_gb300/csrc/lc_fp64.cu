// FP64 kernels of the closure path: packing, FP64 brackets, FP64 projection
// GEMMs, ordered screening/compaction and the sequential accept step.
//
// Every kernel here is SIMT FP64; GB300 has no fast FP64 tensor path, so these
// kernels are bounded by the FP64 FMA rate (brackets, GEMMs) or by HBM
// (packing, gathers, the accept step's row updates).
#include "lc_internal.cuh"

#include <cmath>

namespace lc {

namespace {

__device__ inline unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum; every thread gets the result.  blockDim.x % 32 == 0.
__device__ inline double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();                // red[] may still be read by a previous call
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (w == 0) {
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// ------------------------------------------------------------------ packing
// slot (j, k) of generator q.  H = -i g, so Re H = Im g and Im H = -Re g.
__global__ void k_pack(const double2* __restrict__ g, int k, int d, int ldp, double* __restrict__ out,
                       double* maxdev, double* maxabs, int* nonfinite) {
  const long long P = (long long)d * d;
  const long long tot = P * k;
  const double s1 = 1.0 / sqrt((double)d), s2 = sqrt(2.0 / (double)d);
  double dev = 0.0, mx = 0.0;
  int bad = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long q = e / P;
    const int r = (int)(e % P);
    const int j = r / d, c = r % d;
    const double2* G = g + q * P;
    const double2 a = G[(long long)j * d + c];
    const double2 b = G[(long long)c * d + j];
    if (!isfinite(a.x) || !isfinite(a.y)) bad = 1;
    // anti-Hermitian: a + conj(b) = 0
    dev = fmax(dev, fmax(fabs(a.x + b.x), fabs(a.y - b.y)));
    mx = fmax(mx, fmax(fabs(a.x), fabs(a.y)));
    double v;
    if (j == c)      v = a.y * s1;            // H[j][j] = Im g[j][j]
    else if (j < c)  v = a.y * s2;            // Re H[j][c] = Im g[j][c]
    else             v = -b.x * s2;           // slot (j>c) holds Im H[c][j] = -Re g[c][j]
    out[q * ldp + r] = v;
  }
  // reduce within the warp, then one atomic per warp
  for (int o = 16; o > 0; o >>= 1) {
    dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax((unsigned long long*)maxdev, dbits(dev));
    atomicMax((unsigned long long*)maxabs, dbits(mx));
    if (bad) atomicOr(nonfinite, 1);
  }
}

// g = iH: Re g = -Im H, Im g = Re H
__global__ void k_unpack(const double* __restrict__ V, int n, int d, int ldp, double2* __restrict__ out) {
  const long long P = (long long)d * d;
  const long long tot = P * n;
  const double s1 = sqrt((double)d), s2 = sqrt((double)d / 2.0);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long q = e / P;
    const int r = (int)(e % P);
    const int j = r / d, c = r % d;
    const double* S = V + q * ldp;
    double hr, hi;
    if (j == c)     { hr = S[r] * s1; hi = 0.0; }
    else if (j < c) { hr = S[r] * s2; hi = S[(long long)c * d + j] * s2; }
    else            { hr = S[(long long)c * d + j] * s2; hi = -S[r] * s2; }
    out[e] = make_double2(-hi, hr);
  }
}

// ------------------------------------------------------------ FP64 bracket
// One CTA per (tile pair (I, J), I <= J) x candidate.  It forms the two
// tiles C_IJ and C_JI of C = A B with A = H_l, B = H_m (Hermitian parts of
// V[l], V[m], unpacked on the fly), then writes the packed slots of the
// bracket [V_l, V_m] = C^dagger - C, whose Hermitian part is i (C - C^dagger):
//   Re H_h[j][k] = -(Im C[j][k] + Im C[k][j]),  Im H_h[j][k] = Re C[j][k] - Re C[k][j].
constexpr int BT = 32;   // tile edge
constexpr int BQ = 16;   // k-chunk

__device__ inline double2 herm_elem(const double* __restrict__ S, int d, int r, int c, double s1, double s2) {
  if (r >= d || c >= d) return make_double2(0.0, 0.0);
  if (r == c) return make_double2(S[(long long)r * d + r] * s1, 0.0);
  if (r < c) return make_double2(S[(long long)r * d + c] * s2, S[(long long)c * d + r] * s2);
  return make_double2(S[(long long)c * d + r] * s2, -S[(long long)r * d + c] * s2);
}

__device__ inline void cmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

__global__ void __launch_bounds__(256) k_bracket_f64(const double* __restrict__ V, int d, int ldv, long long t0,
                                                     const int* __restrict__ idx,
                                                     double* __restrict__ out, int ldo) {
  __shared__ double2 sAI[BT][BQ + 1], sAJ[BT][BQ + 1], sBI[BQ][BT + 1], sBJ[BQ][BT + 1];
  const int pair = blockIdx.y;
  const long long t = t0 + (idx ? idx[pair] : pair);
  int l, m;
  pair_from_index(t, &l, &m);
  const double* SA = V + (long long)l * ldv;
  const double* SB = V + (long long)m * ldv;
  const int nt = (d + BT - 1) / BT;
  int tp = blockIdx.x, I = 0;
  while (tp >= nt - I) { tp -= nt - I; ++I; }
  const int J = I + tp;
  const double s1 = sqrt((double)d), s2 = sqrt((double)d / 2.0);
  const int tid = threadIdx.x;
  const int jj = tid >> 3;           // 0..31
  const int kk0 = (tid & 7) * 4;     // 0..28
  double2 c1[4], c2[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) { c1[u] = make_double2(0, 0); c2[u] = make_double2(0, 0); }
  for (int q0 = 0; q0 < d; q0 += BQ) {
    for (int e = tid; e < BT * BQ; e += 256) {
      const int r = e / BQ, c = e % BQ;       // A tiles: row r, col c
      sAI[r][c] = herm_elem(SA, d, I * BT + r, q0 + c, s1, s2);
      sAJ[r][c] = herm_elem(SA, d, J * BT + r, q0 + c, s1, s2);
      const int rb = e / BT, cb = e % BT;     // B tiles: row rb (k), col cb
      sBI[rb][cb] = herm_elem(SB, d, q0 + rb, I * BT + cb, s1, s2);
      sBJ[rb][cb] = herm_elem(SB, d, q0 + rb, J * BT + cb, s1, s2);
    }
    __syncthreads();
#pragma unroll 4
    for (int q = 0; q < BQ; ++q) {
      const double2 a1 = sAI[jj][q];
      const double2 b2 = sBI[q][jj];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        cmac(c1[u], a1, sBJ[q][kk0 + u]);       // C[I*BT+jj][J*BT+kk]
        cmac(c2[u], sAJ[kk0 + u][q], b2);       // C[J*BT+kk][I*BT+jj]
      }
    }
    __syncthreads();
  }
  double* O = out + (long long)pair * ldo;
  const double o1 = 1.0 / sqrt((double)d), o2 = sqrt(2.0 / (double)d);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = I * BT + jj, k = J * BT + kk0 + u;
    if (j >= d || k >= d) continue;
    if (j < k) {
      O[(long long)j * d + k] = -(c1[u].y + c2[u].y) * o2;
      O[(long long)k * d + j] = (c1[u].x - c2[u].x) * o2;
    } else if (j == k) {
      O[(long long)j * d + j] = -2.0 * c1[u].y * o1;
    }
  }
}

// ------------------------------------------------------------ FP64 GEMMs
constexpr int GM = 64, GN = 64, GK = 16;

// C[M x N] = A[M x K] * B[N x K]^T
__global__ void __launch_bounds__(256) k_gemm_nt_f64(int M, int N, int K, const double* __restrict__ A, int lda,
                                                     const double* __restrict__ B, int ldb,
                                                     double* __restrict__ C, int ldc) {
  __shared__ double sA[GK][GM + 2], sB[GK][GN + 2];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int e = threadIdx.x; e < GM * GK; e += 256) {
      const int r = e / GK, c = e % GK;
      const int gm = m0 + r, gn = n0 + r, gk = k0 + c;
      sA[c][r] = (gm < M && gk < K) ? A[(long long)gm * lda + gk] : 0.0;
      sB[c][r] = (gn < N && gk < K) ? B[(long long)gn * ldb + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GK; ++q) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { a[i] = sA[q][ty + 16 * i]; b[i] = sB[q][tx + 16 * i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < M && gn < N) C[(long long)gm * ldc + gn] = acc[i][j];
    }
}

// C[M x N] -= A[M x K] * B[K x N]
__global__ void __launch_bounds__(256) k_gemm_nn_sub_f64(int M, int N, int K, const double* __restrict__ A, int lda,
                                                         const double* __restrict__ B, int ldb,
                                                         double* __restrict__ C, int ldc) {
  __shared__ double sA[GK][GM + 2], sB[GK][GN + 2];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int e = threadIdx.x; e < GM * GK; e += 256) {
      const int r = e / GK, c = e % GK;
      const int gm = m0 + r, gk = k0 + c;
      sA[c][r] = (gm < M && gk < K) ? A[(long long)gm * lda + gk] : 0.0;
      const int rb = e / GN, cb = e % GN;       // B: row k0+rb, col n0+cb
      const int bk = k0 + rb, bn = n0 + cb;
      sB[rb][cb] = (bk < K && bn < N) ? B[(long long)bk * ldb + bn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GK; ++q) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { a[i] = sA[q][ty + 16 * i]; b[i] = sB[q][tx + 16 * i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm < M && gn < N) C[(long long)gm * ldc + gn] -= acc[i][j];
    }
}

__global__ void k_rownorm2_f64(int M, int N, const double* __restrict__ A, int lda, double* __restrict__ out) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= M) return;
  const double* a = A + (long long)row * lda;
  double s = 0.0;
  for (int c = threadIdx.x & 31; c < N; c += 32) s = fma(a[c], a[c], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) out[row] = s;
}

__global__ void k_gather_rows(const double* __restrict__ src, int lds, const int* __restrict__ idx,
                              int ncols, double* __restrict__ dst, int ldd) {
  const int i = blockIdx.y;
  const double* s = src + (long long)idx[i] * lds;
  double* o = dst + (long long)i * ldd;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncols; c += gridDim.x * blockDim.x) o[c] = s[c];
}

// Ordered compaction of the flagged candidates (one CTA of 1024 threads).
template <typename T>
__global__ void __launch_bounds__(1024) k_screen_compact(const T* __restrict__ hn2, const T* __restrict__ rn2,
                                                         int count, T eta2, T tau2, int* __restrict__ idx,
                                                         DevStats* stats, const int* __restrict__ count_dev,
                                                         const int* __restrict__ map) {
  if (count_dev) count = min(count, *count_dev);
  __shared__ int wsum[32];
  __shared__ int base, nz_total;
  __shared__ double wmax[32];
  if (threadIdx.x == 0) { base = 0; nz_total = 0; }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double rej_max = 0.0;
  int nz = 0;
  for (int c0 = 0; c0 < count; c0 += 1024) {
    const int c = c0 + threadIdx.x;
    int f = 0;
    if (c < count) {
      const T h = hn2[c], r = rn2[c];
      f = (h > eta2 && r > tau2 * h) ? 1 : 0;
      if (h > eta2) {
        ++nz;
        if (!f) rej_max = fmax(rej_max, sqrt((double)r / (double)h));
      }
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
      wsum[lane] = v;   // inclusive
    }
    __syncthreads();
    const int off = base + (w ? wsum[w - 1] : 0) + pre;
    if (f) idx[off] = map ? map[c] : c;
    __syncthreads();
    if (threadIdx.x == 0) base += wsum[31];
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) {
    rej_max = fmax(rej_max, __shfl_xor_sync(0xffffffffu, rej_max, o));
    nz += __shfl_xor_sync(0xffffffffu, nz, o);
  }
  if (lane == 0) {
    wmax[w] = rej_max;
    atomicAdd(&nz_total, nz);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < 32; ++i) m = fmax(m, wmax[i]);
    atomicMax(&stats->max_screen_rej_bits, dbits(m));
    stats->nflag = base;
    stats->nnonzero = nz_total;
  }
}

// One step of the sequential in-block accept (Algorithm 4's test and append
// for flagged candidate i, in pair order).  Rows R[0..f) hold the flagged
// candidates, already orthogonalised twice against the basis rows that
// existed when the block started; rn2/hn2 hold their squared residual and
// bracket norms.  Every CTA takes the same decision
//   accept  <=>  ||h|| > eta_abs  and  ||r_i|| > tol ||h||.
// On accept CTA 0 appends w = r_i / ||r_i|| to V, and CTA b >= 1 removes the
// w component from row i + b twice (so later candidates are tested against
// the union of the old basis and this block's accepts, as the sequential
// algorithm does) and refreshes its squared norm.
__global__ void __launch_bounds__(256) k_accept_step(int i, int f, double* __restrict__ R, int ldr,
                                                     double* __restrict__ rn2, const double* __restrict__ hn2,
                                                     double tol, double eta2, double* __restrict__ V, int ldv,
                                                     int ncap, int P, DevStats* stats, DevStatus* st) {
  __shared__ double red[33];
  __shared__ int slot;
  const double h2 = hn2[i], r2 = rn2[i];
  const bool nonzero = h2 > eta2;
  const bool accept = nonzero && (r2 > tol * tol * h2);
  if (!accept) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && nonzero)
      atomicMax(&stats->max_rej_bits, dbits(sqrt(r2 / h2)));
    return;
  }
  const double inv = 1.0 / sqrt(r2);
  const double* ri = R + (long long)i * ldr;
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) {
      int s = stats->ncur;
      if (s >= ncap) {
        if (atomicCAS(&st->code, 0, (int)LC_ERR_CAPACITY) == 0) { st->where = SITE_ACCEPT_CAPACITY; st->info = i; }
        s = -1;
      } else {
        stats->ncur = s + 1;
        stats->naccepted += 1;
        atomicMin(&stats->min_acc_bits, dbits(sqrt(r2 / h2)));
      }
      slot = s;
    }
    __syncthreads();
    if (slot >= 0) {
      double* v = V + (long long)slot * ldv;
      for (int p = threadIdx.x; p < P; p += blockDim.x) v[p] = ri[p] * inv;
    }
    return;
  }
  const int j = i + blockIdx.x;
  if (j >= f) return;
  double* rj = R + (long long)j * ldr;
  for (int pass = 0; pass < 2; ++pass) {
    double s = 0.0;
    for (int p = threadIdx.x; p < P; p += blockDim.x) s = fma(ri[p], rj[p], s);
    const double c = block_sum(s, red) * inv * inv;    // <w, r_j> w = (r_i . r_j / ||r_i||^2) r_i
    for (int p = threadIdx.x; p < P; p += blockDim.x) rj[p] = fma(-c, ri[p], rj[p]);
  }
  double s = 0.0;
  for (int p = threadIdx.x; p < P; p += blockDim.x) s = fma(rj[p], rj[p], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) rn2[j] = s;
}

__global__ void k_zero_stats(DevStats* stats, int ncur) {
  stats->ncur = ncur;
  stats->naccepted = 0;
  stats->nflag = 0;
}

inline int grid_for(long long n, int block, int cap = 152 * 16) {
  long long g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

cudaError_t pack_generators(const double2* g, int k, int d, int ldp, double* out, double* dev_maxdev,
                            double* dev_maxabs, int* dev_nonfinite, cudaStream_t s) {
  const long long tot = (long long)k * d * d;
  k_pack<<<grid_for(tot, 256), 256, 0, s>>>(g, k, d, ldp, out, dev_maxdev, dev_maxabs, dev_nonfinite);
  return cudaGetLastError();
}

cudaError_t unpack_basis(const double* V, int n, int d, int ldp, double2* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long tot = (long long)n * d * d;
  k_unpack<<<grid_for(tot, 256), 256, 0, s>>>(V, n, d, ldp, out);
  return cudaGetLastError();
}

cudaError_t bracket_fp64(const double* V, int d, int ldv, long long t0, const int* idx, int count,
                         double* out, int ldo, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int nt = (d + BT - 1) / BT;
  dim3 grid(nt * (nt + 1) / 2, count);
  k_bracket_f64<<<grid, 256, 0, s>>>(V, d, ldv, t0, idx, out, ldo);
  return cudaGetLastError();
}

cudaError_t gemm_nt_f64(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
                        int ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + GN - 1) / GN, (M + GM - 1) / GM);
  k_gemm_nt_f64<<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
  return cudaGetLastError();
}

cudaError_t gemm_nn_sub_f64(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
                            int ldc, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  dim3 grid((N + GN - 1) / GN, (M + GM - 1) / GM);
  k_gemm_nn_sub_f64<<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
  return cudaGetLastError();
}

cudaError_t rownorm2_f64(int M, int N, const double* A, int lda, double* out, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  k_rownorm2_f64<<<(M + 7) / 8, 256, 0, s>>>(M, N, A, lda, out);
  return cudaGetLastError();
}

cudaError_t gather_rows_f64(const double* src, int lds, const int* idx, int count, int ncols, double* dst,
                            int ldd, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  dim3 grid(grid_for(ncols, 256, 64), count);
  k_gather_rows<<<grid, 256, 0, s>>>(src, lds, idx, ncols, dst, ldd);
  return cudaGetLastError();
}

cudaError_t screen_compact_f64(const double* hn2, const double* rn2, int count, double eta2, double tau2, int* idx,
                               DevStats* stats, cudaStream_t s) {
  k_screen_compact<double><<<1, 1024, 0, s>>>(hn2, rn2, count, eta2, tau2, idx, stats, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t screen_compact_f32(const float* hn2, const float* rn2, int count, float eta2, float tau2, int* idx,
                               DevStats* stats, cudaStream_t s, const int* count_dev, const int* map) {
  k_screen_compact<float><<<1, 1024, 0, s>>>(hn2, rn2, count, eta2, tau2, idx, stats, count_dev, map);
  return cudaGetLastError();
}

cudaError_t accept_step(int i, int f, double* R, int ldr, double* rn2, const double* hn2, double tol, double eta2,
                        double* V, int ldv, int ncap, int P, DevStats* stats, DevStatus* st, int* /*accepted_rows*/,
                        cudaStream_t s) {
  k_accept_step<<<f - i, 256, 0, s>>>(i, f, R, ldr, rn2, hn2, tol, eta2, V, ldv, ncap, P, stats, st);
  return cudaGetLastError();
}

cudaError_t zero_stats(DevStats* stats, int ncur, cudaStream_t s) {
  k_zero_stats<<<1, 1, 0, s>>>(stats, ncur);
  return cudaGetLastError();
}

}  // namespace lc
