// FP64 kernels of the closure path: packing, FP64 brackets, FP64 projection
// GEMMs, ordered screening/compaction and the sequential accept step.
//
// Every kernel here is SIMT FP64; GB300 has no fast FP64 tensor path, so these
// kernels are bounded by the FP64 FMA rate (brackets, GEMMs) or by HBM
// (packing, gathers, the accept step's row updates).
#include "lc_internal.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>

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
// The complex products take three real products instead of four (Gauss):
// with t1 = sum ar br, t2 = sum ai bi, t3 = sum (ar + ai)(br + bi),
// Re C = t1 - t2 and Im C = t3 - t1 - t2.  The sums ar + ai, br + bi are
// formed once when a tile is staged, so the FP64 pipe (the bound of this
// kernel) runs 3 instead of 4 FMAs per complex multiply-add.  Error: of the
// order of u (|ar| + |ai|)(|br| + |bi|) per term, i.e. u |A| |B| normwise.
constexpr int BT = 32;   // tile edge
constexpr int BQ = 8;    // k-chunk

__device__ inline double2 herm_elem(const double* __restrict__ S, int d, int r, int c, double s1, double s2) {
  if (r >= d || c >= d) return make_double2(0.0, 0.0);
  if (r == c) return make_double2(S[(long long)r * d + r] * s1, 0.0);
  if (r < c) return make_double2(S[(long long)r * d + c] * s2, S[(long long)c * d + r] * s2);
  return make_double2(S[(long long)c * d + r] * s2, -S[(long long)r * d + c] * s2);
}

struct Gauss3 { double t1, t2, t3; };

__device__ inline void gmac(Gauss3& acc, double ar, double ai, double as, double br, double bi, double bs) {
  acc.t1 = fma(ar, br, acc.t1);
  acc.t2 = fma(ai, bi, acc.t2);
  acc.t3 = fma(as, bs, acc.t3);
}

__global__ void __launch_bounds__(256) k_bracket_f64(const double* __restrict__ V, int d, int ldv, long long t0,
                                                     const int* __restrict__ idx,
                                                     double* __restrict__ out, int ldo) {
  // planes: 0 real, 1 imaginary, 2 real + imaginary
  __shared__ double sAI[3][BT][BQ + 1], sAJ[3][BT][BQ + 1], sBI[3][BQ][BT + 1], sBJ[3][BQ][BT + 1];
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
  Gauss3 c1[4], c2[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) { c1[u] = Gauss3{0, 0, 0}; c2[u] = Gauss3{0, 0, 0}; }
  for (int q0 = 0; q0 < d; q0 += BQ) {
    {
      const int e = tid;                     // BT * BQ = 256 slots per tile
      const int r = e / BQ, c = e % BQ;      // A tiles: row r, col c
      double2 v = herm_elem(SA, d, I * BT + r, q0 + c, s1, s2);
      sAI[0][r][c] = v.x; sAI[1][r][c] = v.y; sAI[2][r][c] = v.x + v.y;
      v = herm_elem(SA, d, J * BT + r, q0 + c, s1, s2);
      sAJ[0][r][c] = v.x; sAJ[1][r][c] = v.y; sAJ[2][r][c] = v.x + v.y;
      const int rb = e / BT, cb = e % BT;    // B tiles: row rb (k), col cb
      v = herm_elem(SB, d, q0 + rb, I * BT + cb, s1, s2);
      sBI[0][rb][cb] = v.x; sBI[1][rb][cb] = v.y; sBI[2][rb][cb] = v.x + v.y;
      v = herm_elem(SB, d, q0 + rb, J * BT + cb, s1, s2);
      sBJ[0][rb][cb] = v.x; sBJ[1][rb][cb] = v.y; sBJ[2][rb][cb] = v.x + v.y;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < BQ; ++q) {
      const double a1r = sAI[0][jj][q], a1i = sAI[1][jj][q], a1s = sAI[2][jj][q];
      const double b2r = sBI[0][q][jj], b2i = sBI[1][q][jj], b2s = sBI[2][q][jj];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        // C[I*BT+jj][J*BT+kk]
        gmac(c1[u], a1r, a1i, a1s, sBJ[0][q][kk0 + u], sBJ[1][q][kk0 + u], sBJ[2][q][kk0 + u]);
        // C[J*BT+kk][I*BT+jj]
        gmac(c2[u], sAJ[0][kk0 + u][q], sAJ[1][kk0 + u][q], sAJ[2][kk0 + u][q], b2r, b2i, b2s);
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
    const double c1x = c1[u].t1 - c1[u].t2, c1y = c1[u].t3 - c1[u].t1 - c1[u].t2;
    const double c2x = c2[u].t1 - c2[u].t2, c2y = c2[u].t3 - c2[u].t1 - c2[u].t2;
    if (j < k) {
      O[(long long)j * d + k] = -(c1y + c2y) * o2;
      O[(long long)k * d + j] = (c1x - c2x) * o2;
    } else if (j == k) {
      O[(long long)j * d + j] = -2.0 * c1y * o1;
    }
  }
}

// ------------------------------------------------------------ FP64 GEMMs
// One templated tile kernel for C = A B^T (B stored N x K) and C = A B (B
// stored K x N), 64 x 64 tiles, 4 x 4 outputs per thread.  blockIdx.z splits
// K; with more than one split each CTA writes its partial tile to a workspace
// and k_reduce_f64 adds the partials in a fixed order (deterministic).
// mode: 0 store, 1 subtract from C, 2 partial to workspace.
constexpr int GK = 16;

// TM x TN output tile (TM * TN = 4096), 256 threads in a 16 x 16 layout, each
// thread TM/16 rows x TN/16 columns.  TM = 16 for the skinny products of the
// accept path (few flagged rows), TM = 64 otherwise.
template <bool BT, int TM>
__global__ void __launch_bounds__(256) k_gemm_f64(int M, int N, int K, int kchunk, const double* __restrict__ A,
                                                  int lda, const double* __restrict__ B, int ldb,
                                                  double* __restrict__ C, int ldc, int mode,
                                                  double* __restrict__ ws, const int* __restrict__ run_if) {
  constexpr int TN = 4096 / TM, RI = TM / 16, RJ = TN / 16;
  if (run_if && *run_if == 0) return;
  __shared__ double sA[GK][TM + 2], sB[GK][TN + 2];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  double acc[RI][RJ] = {};
  for (int k0 = kb; k0 < ke; k0 += GK) {
    for (int e = threadIdx.x; e < TM * GK; e += 256) {
      const int r = e / GK, c = e % GK;
      const int gm = m0 + r, gk = k0 + c;
      sA[c][r] = (gm < M && gk < ke) ? A[(long long)gm * lda + gk] : 0.0;
    }
    for (int e = threadIdx.x; e < TN * GK; e += 256) {
      if (BT) {
        const int r = e / GK, c = e % GK;
        const int gn = n0 + r, gk = k0 + c;
        sB[c][r] = (gn < N && gk < ke) ? B[(long long)gn * ldb + gk] : 0.0;
      } else {
        const int rb = e / TN, cb = e % TN;
        const int bk = k0 + rb, bn = n0 + cb;
        sB[rb][cb] = (bk < ke && bn < N) ? B[(long long)bk * ldb + bn] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GK; ++q) {
      double a[RI], b[RJ];
#pragma unroll
      for (int i = 0; i < RI; ++i) a[i] = sA[q][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < RJ; ++j) b[j] = sB[q][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < RJ; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RI; ++i)
#pragma unroll
    for (int j = 0; j < RJ; ++j) {
      const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm >= M || gn >= N) continue;
      if (mode == 0) C[(long long)gm * ldc + gn] = acc[i][j];
      else if (mode == 1) C[(long long)gm * ldc + gn] -= acc[i][j];
      else ws[((long long)blockIdx.z * M + gm) * N + gn] = acc[i][j];
    }
}

__global__ void k_reduce_f64(int M, int N, int S, const double* __restrict__ ws, double* __restrict__ C, int ldc,
                             int subtract, const int* __restrict__ run_if) {
  if (run_if && *run_if == 0) return;
  const long long tot = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int z = 0; z < S; ++z) t += ws[(long long)z * tot + e];
    const long long o = (e / N) * ldc + (e % N);
    if (subtract) C[o] -= t; else C[o] = t;
  }
}

__global__ void k_rownorm2_f64(int M, int N, const double* __restrict__ A, int lda, double* __restrict__ out,
                               const int* __restrict__ run_if) {
  if (run_if && *run_if == 0) return;
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
                                                         int count, T eta2, T tau2, T tau2_abs, int* __restrict__ idx,
                                                         DevStats* stats, const int* __restrict__ count_dev,
                                                         const int* __restrict__ map, int measured,
                                                         float* __restrict__ rho2_flag) {
  if (count_dev) count = min(count, *count_dev);
  // measured threshold: tau^2 and the probe's eps^2 live in the stats block
  if (measured) tau2 = (T)stats->tau2;
  const double eps2 = measured ? (double)stats->eps2 : -1.0;
  int gray = 0;
  __shared__ int wsum[32];
  __shared__ int base, nz_total, gray_total;
  __shared__ double wmax[32];
  if (threadIdx.x == 0) { base = 0; nz_total = 0; gray_total = 0; }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double rej_max = 0.0;
  int nz = 0;
  for (int c0 = 0; c0 < count; c0 += 1024) {
    const int c = c0 + threadIdx.x;
    int f = 0;
    if (c < count) {
      const T h = hn2[c], r = rn2[c];
      f = (h > eta2 && r > tau2 * h + tau2_abs) ? 1 : 0;
      if (h > eta2) {
        ++nz;
        if (!f) {
          rej_max = fmax(rej_max, sqrt((double)r / (double)h));
          if ((double)r > eps2 * (double)h && eps2 >= 0.0) ++gray;
        }
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
    if (f) {
      idx[off] = map ? map[c] : c;
      if (rho2_flag) rho2_flag[off] = (float)((double)rn2[c] / (double)hn2[c]);
    }
    __syncthreads();
    if (threadIdx.x == 0) base += wsum[31];
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) {
    rej_max = fmax(rej_max, __shfl_xor_sync(0xffffffffu, rej_max, o));
    nz += __shfl_xor_sync(0xffffffffu, nz, o);
    gray += __shfl_xor_sync(0xffffffffu, gray, o);
  }
  if (lane == 0) {
    wmax[w] = rej_max;
    atomicAdd(&nz_total, nz);
    if (gray) atomicAdd(&gray_total, gray);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < 32; ++i) m = fmax(m, wmax[i]);
    atomicMax(&stats->max_screen_rej_bits, dbits(m));
    stats->nflag = base;
    stats->nnonzero = nz_total;
    stats->ngray = gray_total;
  }
}

// Multi-CTA ordered compaction (two launches).  The candidates are cut into
// kCmpCtas contiguous chunks; pass 1 counts each chunk's flags (and its
// statistics) into part[], pass 2 writes each chunk's flagged positions at
// the offset given by the counts of the chunks before it, so the output order
// is candidate order, as the single-CTA kernel produces.
template <typename T>
__device__ __forceinline__ int screen_flag(const T* hn2, const T* rn2, int c, T eta2, T tau2, T tau2_abs) {
  const T h = hn2[c], r = rn2[c];
  return (h > eta2 && r > tau2 * h + tau2_abs) ? 1 : 0;
}

template <typename T>
__global__ void __launch_bounds__(kCmpThreads) k_screen_pass1(const T* __restrict__ hn2, const T* __restrict__ rn2,
                                                           int count, T eta2, T tau2, T tau2_abs, DevStats* stats,
                                                           const int* __restrict__ count_dev, int measured,
                                                           int* __restrict__ part) {
  __shared__ int sf[kCmpThreads / 32], sn[kCmpThreads / 32], sg[kCmpThreads / 32];
  __shared__ double sm[kCmpThreads / 32];
  if (count_dev) count = min(count, *count_dev);
  if (measured) tau2 = (T)stats->tau2;
  const double eps2 = measured ? (double)stats->eps2 : -1.0;
  const int chunk = (count + gridDim.x - 1) / gridDim.x;
  const int c0 = blockIdx.x * chunk, c1 = min(count, c0 + chunk);
  int nf = 0, nz = 0, gray = 0;
  double rej = 0.0;
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
    const T h = hn2[c], r = rn2[c];
    const int f = screen_flag(hn2, rn2, c, eta2, tau2, tau2_abs);
    nf += f;
    if (h > eta2) {
      ++nz;
      if (!f) {
        rej = fmax(rej, sqrt((double)r / (double)h));
        if (eps2 >= 0.0 && (double)r > eps2 * (double)h) ++gray;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    nf += __shfl_xor_sync(0xffffffffu, nf, o);
    nz += __shfl_xor_sync(0xffffffffu, nz, o);
    gray += __shfl_xor_sync(0xffffffffu, gray, o);
    rej = fmax(rej, __shfl_xor_sync(0xffffffffu, rej, o));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { sf[w] = nf; sn[w] = nz; sg[w] = gray; sm[w] = rej; }
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0, b = 0, g = 0;
    double m = 0.0;
    for (int i = 0; i < kCmpThreads / 32; ++i) { a += sf[i]; b += sn[i]; g += sg[i]; m = fmax(m, sm[i]); }
    part[blockIdx.x] = a;
    part[kCmpCtas + blockIdx.x] = b;
    part[2 * kCmpCtas + blockIdx.x] = g;
    if (m > 0.0) atomicMax(&stats->max_screen_rej_bits, dbits(m));
    if (blockIdx.x == 0) stats->min_rho2_flag_bits = 0x7f800000u;   // +inf, lowered by pass 2
  }
}

template <typename T>
__global__ void __launch_bounds__(kCmpThreads) k_screen_pass2(const T* __restrict__ hn2, const T* __restrict__ rn2,
                                                           int count, T eta2, T tau2, T tau2_abs,
                                                           int* __restrict__ idx, DevStats* stats,
                                                           const int* __restrict__ count_dev,
                                                           const int* __restrict__ map, int measured,
                                                           float* __restrict__ rho2_flag,
                                                           const int* __restrict__ part, int* __restrict__ cidx) {
  __shared__ int wsum[kCmpThreads / 32];
  __shared__ unsigned int wmin[kCmpThreads / 32];
  __shared__ int base;
  unsigned int rmin = 0x7f800000u;   // float bits of the smallest flagged rho^2 this thread saw
  if (count_dev) count = min(count, *count_dev);
  if (measured) tau2 = (T)stats->tau2;
  const int chunk = (count + gridDim.x - 1) / gridDim.x;
  const int c0 = blockIdx.x * chunk, c1 = min(count, c0 + chunk);
  if (threadIdx.x == 0) {
    int o = 0;
    for (int b = 0; b < (int)blockIdx.x; ++b) o += part[b];
    base = o;
    if (blockIdx.x == 0) {
      int a = 0, z = 0, g = 0;
      for (int b = 0; b < (int)gridDim.x; ++b) { a += part[b]; z += part[kCmpCtas + b]; g += part[2 * kCmpCtas + b]; }
      stats->nflag = a;
      stats->nnonzero = z;
      stats->ngray = g;
    }
  }
  __syncthreads();
  for (int t0 = c0; t0 < c1; t0 += blockDim.x) {
    const int c = t0 + threadIdx.x;
    const int f = c < c1 ? screen_flag(hn2, rn2, c, eta2, tau2, tau2_abs) : 0;
    int tot;
    const int at = base + cta_excl_scan(f, &tot, wsum);
    if (f) {
      idx[at] = map ? map[c] : c;
      if (cidx) cidx[at] = c;
      if (rho2_flag) {
        const float r = (float)((double)rn2[c] / (double)hn2[c]);
        rho2_flag[at] = r;
        rmin = min(rmin, __float_as_uint(r));   // non-negative floats order as their bits
      }
    }
    if (threadIdx.x == 0) base += tot;
    __syncthreads();
  }
  if (rho2_flag) {
    for (int o = 16; o > 0; o >>= 1) rmin = min(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = rmin;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned int m = wmin[0];
      for (int i = 1; i < kCmpThreads / 32; ++i) m = min(m, wmin[i]);
      if (m != 0x7f800000u) atomicMin(&stats->min_rho2_flag_bits, m);
    }
  }
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  The
// wait is bounded: after limit_ns the CTA records LC_ERR_TIMEOUT and returns
// false, and the caller leaves the kernel.
__device__ bool grid_barrier(unsigned int* count, unsigned int* gen, unsigned int nblocks, uint64_t limit_ns,
                             DevStatus* st, int* ok_smem) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int g0 = ld_acquire_u32(gen);
    __threadfence();
    const unsigned int arrived = atomicAdd(count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      uint64_t t0;
      asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
      // poll with plain acquire loads (an atomic per poll from every waiting
      // SM would queue at the counter's L2 slice ahead of the last arrival)
      for (unsigned int it = 0;; ++it) {
        if (ld_acquire_u32(gen) != g0) break;
        if ((it & 63u) == 63u) {
          uint64_t t;
          asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
          if (t - t0 > limit_ns) {
            if (atomicCAS(&st->code, 0, (int)LC_ERR_TIMEOUT) == 0) { st->where = SITE_ACCEPT_BARRIER; st->info = 0; }
            ok = 0;
            break;
          }
        }
      }
    }
    __threadfence();
    *ok_smem = ok;
  }
  __syncthreads();
  return *ok_smem != 0;
}

// The whole in-block test-and-append of Algorithm 4 in one cooperative launch.
// Rows R[0..f) are the flagged candidates in pair order, already
// orthogonalised against the basis rows that existed when the block started;
// rn2/hn2 hold squared residual and bracket norms.  For each i in order every
// CTA takes the same decision (accept <=> ||h|| > eta_abs and ||r_i|| > tol
// ||h||); on accept CTA 0 appends w = r_i / ||r_i|| to V and each CTA removes
// the w component (twice) from the later rows it owns (row j belongs to CTA
// j mod gridDim.x) and refreshes their norms; one grid barrier then publishes
// the updated rows.  A rejected candidate changes nothing, so no barrier.
__global__ void __launch_bounds__(256) k_accept_seq(int f, double* __restrict__ R, int ldr,
                                                    double* __restrict__ rn2, const double* __restrict__ hn2,
                                                    double tol_rel2, double tol_abs2, double eta2,
                                                    double* __restrict__ V, int ldv,
                                                    int ncap, int P, DevStats* stats, DevStatus* st,
                                                    unsigned int* bar, uint64_t limit_ns, int phantom,
                                                    const double* __restrict__ Hraw, double* __restrict__ Bk,
                                                    double* __restrict__ bn2, const float* __restrict__ rho2_screen) {
  __shared__ double red[33];
  __shared__ int slot, ok_smem;
  const unsigned int G = gridDim.x;
  for (int i = 0; i < f; ++i) {
    const double h2 = hn2[i];
    const double r2 = __ldcg(&rn2[i]);
    const bool nonzero = h2 > eta2;
    if (!(nonzero && r2 > tol_rel2 * h2 + tol_abs2)) {
      if (blockIdx.x == 0 && threadIdx.x == 0 && nonzero) atomicMax(&stats->max_rej_bits, dbits(sqrt(r2 / h2)));
      continue;
    }
    const double inv = 1.0 / sqrt(r2);
    const double* ri = R + (long long)i * ldr;
    if (blockIdx.x == 0) {
      if (threadIdx.x == 0) {
        int sl = stats->ncur;
        if (sl >= ncap) {
          if (atomicCAS(&st->code, 0, (int)LC_ERR_CAPACITY) == 0) { st->where = SITE_ACCEPT_CAPACITY; st->info = i; }
          sl = -1;
        } else {
          stats->ncur = sl + 1;
          stats->naccepted += 1;
          atomicMin(&stats->min_acc_bits, dbits(sqrt(r2 / h2)));
          if (rho2_screen) atomicMin(&stats->min_acc_screen_bits, dbits(sqrt((double)rho2_screen[i])));
        }
        slot = sl;
      }
      __syncthreads();
      if (slot >= 0) {
        double* v = V + (long long)slot * ldv;
        #pragma unroll 8
        for (int p = threadIdx.x; p < P; p += blockDim.x) v[p] = __ldcg(&ri[p]) * inv;
        if (Bk) {   // Algorithm 3: the bracket itself joins B
          const double* hr = Hraw + (long long)i * ldr;
          double* b = Bk + (long long)slot * ldv;
          #pragma unroll 8
          for (int p = threadIdx.x; p < P; p += blockDim.x) b[p] = hr[p];
          if (threadIdx.x == 0) bn2[slot] = h2;
        }
      }
    }
    for (int j = i + 1 + (int)((blockIdx.x + G - (unsigned)((i + 1) % G)) % G); j < f; j += G) {
      double* rj = R + (long long)j * ldr;
      for (int pass = 0; pass < 2; ++pass) {
        double sacc = 0.0;
        #pragma unroll 8
        for (int p = threadIdx.x; p < P; p += blockDim.x) sacc = fma(__ldcg(&ri[p]), rj[p], sacc);
        const double c = block_sum(sacc, red) * inv * inv;
        #pragma unroll 8
        for (int p = threadIdx.x; p < P; p += blockDim.x) rj[p] = fma(-c, __ldcg(&ri[p]), rj[p]);
      }
      double sacc = 0.0;
      #pragma unroll 8
      for (int p = threadIdx.x; p < P; p += blockDim.x) sacc = fma(rj[p], rj[p], sacc);
      sacc = block_sum(sacc, red);
      if (threadIdx.x == 0) rn2[j] = sacc;
    }
    // phantom (test hook): one more arrival is expected than there are CTAs
    if (!grid_barrier(bar, bar + 1, G + (unsigned)phantom, limit_ns, st, &ok_smem)) return;
  }
}

// The same in-block test and append, sliced along the P components instead
// of the rows: every CTA of the cooperative grid owns one contiguous slice
// [pb, pe) of every row, so each row streams through all SMs even when only a
// few candidates are flagged (one CTA per row would leave most SMs idle while
// it walks rows of 2^20 doubles).  A CTA touches only its own slice of R and
// V; what crosses CTAs is the per-CTA partial sums of the dot products and
// squared norms, published through `part` and a grid barrier and summed by
// every CTA in the same fixed order, so every CTA takes the same decisions.
// Per accept: phase A partial dots <r_j, w'> (w' = r_i before scaling),
// barrier; phase B the first projection r_j -= c_j r_i fused with the second
// pass's partial dots; barrier; phase C the second projection fused with the
// partial squared norms; barrier.  Per component this is the arithmetic of
// k_accept_seq; only the order of the partial sums differs.  Threads carry
// kWideGroup rows at a time so that one CTA reduction serves kWideGroup rows.
constexpr int kWideGroup = 8;   // 256 threads = 8 warps

__device__ inline void wide_group_store(double (&acc)[kWideGroup], int j0, int jn, double* red, int par,
                                        double* __restrict__ part, unsigned int G) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* rb = red + par * 64;    // two 8 x 8 buffers, alternated per group
#pragma unroll
  for (int q = 0; q < kWideGroup; ++q) {
    const double v = warp_sum(acc[q]);
    if (lane == 0) rb[w * kWideGroup + q] = v;
  }
  __syncthreads();
  if ((int)threadIdx.x < jn) {
    double t = 0.0;
    for (int ww = 0; ww < 8; ++ww) t += rb[ww * kWideGroup + threadIdx.x];
    __stcg(&part[(size_t)(j0 + threadIdx.x) * G + blockIdx.x], t);
  }
}

// out[j] = sum over CTAs of part[j][.], j in [j_lo, f), in CTA order per lane
// and a fixed butterfly across lanes (identical in every CTA)
__device__ inline void wide_sum_partials(const double* __restrict__ part, int j_lo, int f, unsigned int G,
                                         double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = j_lo + w; j < f; j += 8) {
    double t = 0.0;
    for (unsigned int g = lane; g < G; g += 32) t += __ldcg(&part[(size_t)j * G + g]);
    t = warp_sum(t);
    if (lane == 0) out[j] = t;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) k_accept_wide(int f, double* __restrict__ R, int ldr,
                                                     double* __restrict__ rn2, const double* __restrict__ hn2,
                                                     double tol_rel2, double tol_abs2, double eta2,
                                                     double* __restrict__ V, int ldv, int ncap, int P,
                                                     DevStats* stats, DevStatus* st, unsigned int* bar,
                                                     uint64_t limit_ns, int phantom,
                                                     const double* __restrict__ Hraw, double* __restrict__ Bk,
                                                     double* __restrict__ bn2, const float* __restrict__ rho2_screen,
                                                     double* __restrict__ part) {
  __shared__ double red[2 * 64];
  __shared__ double coef[kAcceptWideMaxRows];
  __shared__ double rn2s[kAcceptWideMaxRows];
  __shared__ int ok_smem;
  const unsigned int G = gridDim.x;
  const unsigned int Gb = G + (unsigned)phantom;   // phantom (test hook): an arrival that never comes
  const int chunk = (((P + (int)G - 1) / (int)G) + 31) & ~31;
  const int pb = min(P, (int)blockIdx.x * chunk), pe = min(P, pb + chunk);
  double* part0 = part;
  double* part1 = part + (size_t)kAcceptWideMaxRows * G;
  double* part2 = part + (size_t)2 * kAcceptWideMaxRows * G;
  const int slot0 = stats->ncur;   // CTA 0 writes it back only after every CTA passed a barrier
  for (int j = threadIdx.x; j < f; j += blockDim.x) rn2s[j] = rn2[j];
  __syncthreads();
  int nacc = 0, nbar = 0;
  for (int i = 0; i < f; ++i) {
    const double h2 = hn2[i];
    const double r2 = rn2s[i];
    const bool nonzero = h2 > eta2;
    if (!(nonzero && r2 > tol_rel2 * h2 + tol_abs2)) {
      if (blockIdx.x == 0 && threadIdx.x == 0 && nonzero) atomicMax(&stats->max_rej_bits, dbits(sqrt(r2 / h2)));
      continue;
    }
    const int slot = slot0 + nacc;
    if (slot >= ncap) {   // the same test in every CTA
      if (blockIdx.x == 0 && threadIdx.x == 0 && atomicCAS(&st->code, 0, (int)LC_ERR_CAPACITY) == 0) {
        st->where = SITE_ACCEPT_CAPACITY;
        st->info = i;
      }
      break;
    }
    ++nacc;
    const double inv = 1.0 / sqrt(r2);
    const double inv2 = inv * inv;
    const double* ri = R + (long long)i * ldr;
    double* v = V + (long long)slot * ldv;
    for (int p = pb + threadIdx.x; p < pe; p += blockDim.x) v[p] = ri[p] * inv;
    if (Bk) {   // Algorithm 3: the bracket itself joins B
      const double* hr = Hraw + (long long)i * ldr;
      double* b = Bk + (long long)slot * ldv;
      for (int p = pb + threadIdx.x; p < pe; p += blockDim.x) b[p] = hr[p];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      atomicMin(&stats->min_acc_bits, dbits(sqrt(r2 / h2)));
      if (rho2_screen) atomicMin(&stats->min_acc_screen_bits, dbits(sqrt((double)rho2_screen[i])));
      if (Bk) bn2[slot] = h2;
    }
    if (i + 1 >= f) break;
    int par = 0;
    // phase A: partial <r_i, r_j>
    for (int j0 = i + 1; j0 < f; j0 += kWideGroup, par ^= 1) {
      const int jn = min(kWideGroup, f - j0);
      double acc[kWideGroup];
#pragma unroll
      for (int q = 0; q < kWideGroup; ++q) acc[q] = 0.0;
      for (int p = pb + threadIdx.x; p < pe; p += blockDim.x) {
        const double x = ri[p];
#pragma unroll
        for (int q = 0; q < kWideGroup; ++q)
          if (q < jn) acc[q] = fma(x, R[(long long)(j0 + q) * ldr + p], acc[q]);
      }
      wide_group_store(acc, j0, jn, red, par, part0, G);
    }
    ++nbar;
    if (!grid_barrier(bar, bar + 1, Gb, limit_ns, st, &ok_smem)) return;
    wide_sum_partials(part0, i + 1, f, G, coef);
    // phase B: first projection, then partial <r_i, r_j> of the second pass
    for (int j0 = i + 1; j0 < f; j0 += kWideGroup, par ^= 1) {
      const int jn = min(kWideGroup, f - j0);
      double acc[kWideGroup], c[kWideGroup];
#pragma unroll
      for (int q = 0; q < kWideGroup; ++q) {
        acc[q] = 0.0;
        c[q] = q < jn ? coef[j0 + q] * inv2 : 0.0;
      }
      for (int p = pb + threadIdx.x; p < pe; p += blockDim.x) {
        const double x = ri[p];
#pragma unroll
        for (int q = 0; q < kWideGroup; ++q)
          if (q < jn) {
            double* rq = R + (long long)(j0 + q) * ldr + p;
            const double y = fma(-c[q], x, *rq);
            *rq = y;
            acc[q] = fma(x, y, acc[q]);
          }
      }
      wide_group_store(acc, j0, jn, red, par, part1, G);
    }
    ++nbar;
    if (!grid_barrier(bar, bar + 1, Gb, limit_ns, st, &ok_smem)) return;
    wide_sum_partials(part1, i + 1, f, G, coef);
    // phase C: second projection, then partial ||r_j||^2
    for (int j0 = i + 1; j0 < f; j0 += kWideGroup, par ^= 1) {
      const int jn = min(kWideGroup, f - j0);
      double acc[kWideGroup], c[kWideGroup];
#pragma unroll
      for (int q = 0; q < kWideGroup; ++q) {
        acc[q] = 0.0;
        c[q] = q < jn ? coef[j0 + q] * inv2 : 0.0;
      }
      for (int p = pb + threadIdx.x; p < pe; p += blockDim.x) {
        const double x = ri[p];
#pragma unroll
        for (int q = 0; q < kWideGroup; ++q)
          if (q < jn) {
            double* rq = R + (long long)(j0 + q) * ldr + p;
            const double y = fma(-c[q], x, *rq);
            *rq = y;
            acc[q] = fma(y, y, acc[q]);
          }
      }
      wide_group_store(acc, j0, jn, red, par, part2, G);
    }
    ++nbar;
    if (!grid_barrier(bar, bar + 1, Gb, limit_ns, st, &ok_smem)) return;
    wide_sum_partials(part2, i + 1, f, G, rn2s);
    if (blockIdx.x == 0)
      for (int j = i + 1 + (int)threadIdx.x; j < f; j += blockDim.x) rn2[j] = rn2s[j];
  }
  if (nacc > 0 && nbar == 0) {   // every CTA must have read ncur before it changes
    if (!grid_barrier(bar, bar + 1, Gb, limit_ns, st, &ok_smem)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    stats->ncur = slot0 + nacc;
    stats->naccepted += nacc;
  }
}

// The in-block test and append with each later row held in shared memory
// by the CTA that owns it (CTA j owns row j; f <= co-resident CTAs, P
// doubles of dynamic shared memory each).  Per accept only the pivot row
// r_i streams from L2; the owner of row j runs three sweeps over its row:
// <r_i, r_j>; r_j -= c1 r_i fused with the second pass's <r_i, r_j>;
// r_j -= c2 r_i fused with ||r_j||^2 and the write-back of r_j (a later
// pivot is read from global memory).  Per component and per partial sum
// this is k_accept_seq's arithmetic in k_accept_seq's order; one bounded
// grid barrier per accept.  The pivot's owner appends it to V.
// NPT: components per thread (P <= 256 NPT); the pivot row is loaded into
// registers once per accept (one round trip to L2 for all three sweeps), in
// the same per-thread order of p as a strided loop.
template <int NPT>
__global__ void __launch_bounds__(256, 1) k_accept_rowsmem(int f, double* __restrict__ R, int ldr,
                                                           double* __restrict__ rn2, const double* __restrict__ hn2,
                                                           double tol_rel2, double tol_abs2, double eta2,
                                                           double* __restrict__ V, int ldv, int ncap, int P,
                                                           DevStats* stats, DevStatus* st, unsigned int* bar,
                                                           uint64_t limit_ns, int phantom,
                                                           const double* __restrict__ Hraw, double* __restrict__ Bk,
                                                           double* __restrict__ bn2,
                                                           const float* __restrict__ rho2_screen) {
  extern __shared__ double row[];
  __shared__ double red[33];
  __shared__ int ok_smem;
  const unsigned int Gb = gridDim.x + (unsigned)phantom;   // phantom (test hook): an arrival that never comes
  const int j = blockIdx.x;
  double* rj = R + (long long)j * ldr;
  const int slot0 = stats->ncur;   // CTA 0 writes it back only after every CTA passed a barrier
  #pragma unroll 8
  for (int p = threadIdx.x; p < P; p += blockDim.x) row[p] = rj[p];
  __syncthreads();
  int nacc = 0, nbar = 0;
  for (int i = 0; i < f; ++i) {
    const double h2 = hn2[i];
    const double r2 = __ldcg(&rn2[i]);
    const bool nonzero = h2 > eta2;
    if (!(nonzero && r2 > tol_rel2 * h2 + tol_abs2)) {
      if (j == 0 && threadIdx.x == 0 && nonzero) atomicMax(&stats->max_rej_bits, dbits(sqrt(r2 / h2)));
      continue;
    }
    const int slot = slot0 + nacc;
    if (slot >= ncap) {   // the same test in every CTA
      if (j == 0 && threadIdx.x == 0 && atomicCAS(&st->code, 0, (int)LC_ERR_CAPACITY) == 0) {
        st->where = SITE_ACCEPT_CAPACITY;
        st->info = i;
      }
      break;
    }
    ++nacc;
    const double inv = 1.0 / sqrt(r2);
    if (j == i) {
      double* v = V + (long long)slot * ldv;
      #pragma unroll 8
      for (int p = threadIdx.x; p < P; p += blockDim.x) v[p] = row[p] * inv;
      if (Bk) {   // Algorithm 3: the bracket itself joins B
        const double* hr = Hraw + (long long)i * ldr;
        double* b = Bk + (long long)slot * ldv;
        #pragma unroll 8
        for (int p = threadIdx.x; p < P; p += blockDim.x) b[p] = hr[p];
      }
      if (threadIdx.x == 0) {
        atomicMin(&stats->min_acc_bits, dbits(sqrt(r2 / h2)));
        if (rho2_screen) atomicMin(&stats->min_acc_screen_bits, dbits(sqrt((double)rho2_screen[i])));
        if (Bk) bn2[slot] = h2;
      }
    } else if (j > i) {
      const double* ri = R + (long long)i * ldr;
      double x[NPT];
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        const int p = threadIdx.x + k * 256;
        x[k] = p < P ? __ldcg(&ri[p]) : 0.0;
      }
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        const int p = threadIdx.x + k * 256;
        if (p < P) s = fma(x[k], row[p], s);
      }
      const double c1 = block_sum(s, red) * inv * inv;   // as k_accept_seq associates it
      s = 0.0;
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        const int p = threadIdx.x + k * 256;
        if (p < P) {
          const double y = fma(-c1, x[k], row[p]);
          row[p] = y;
          s = fma(x[k], y, s);
        }
      }
      const double c2 = block_sum(s, red) * inv * inv;
      s = 0.0;
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        const int p = threadIdx.x + k * 256;
        if (p < P) {
          const double y = fma(-c2, x[k], row[p]);
          row[p] = y;
          __stcg(&rj[p], y);
          s = fma(y, y, s);
        }
      }
      s = block_sum(s, red);
      if (threadIdx.x == 0) __stcg(&rn2[j], s);
    }
    if (i + 1 < f) {
      ++nbar;
      if (!grid_barrier(bar, bar + 1, Gb, limit_ns, st, &ok_smem)) return;
    }
  }
  if (nacc > 0 && nbar == 0) {   // every CTA must have read ncur before it changes
    if (!grid_barrier(bar, bar + 1, Gb, limit_ns, st, &ok_smem)) return;
  }
  if (j == 0 && threadIdx.x == 0) {
    stats->ncur = slot0 + nacc;
    stats->naccepted += nacc;
  }
}

// Second Gram-Schmidt pass needed?  After one FP64 pass the loss of
// orthogonality of r is about eps ||h|| / ||r||; when ||r|| >= ||h|| / sqrt(2)
// for every row (or the row is certainly dependent, ||r|| <= tol ||h|| / 2)
// one pass is already accurate to rounding (Daniel, Gragg, Kaufman and
// Stewart's criterion).  Writes 1 to *need if any row needs the second pass.
__global__ void k_need_pass2(int f, const double* __restrict__ hn2, const double* __restrict__ rn2, double eta2,
                             double tol_rel2, double tol_abs2, int* need) {
  int any = 0;
  for (int i = threadIdx.x; i < f; i += blockDim.x) {
    const double h2 = hn2[i], r2 = rn2[i];
    if (h2 > eta2 && r2 < 0.5 * h2 && r2 > 0.25 * (tol_rel2 * h2 + tol_abs2)) any = 1;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) *need = any;
}

// ordered list of candidates with hn2 > eta2 (one CTA of 1024 threads); the
// FP64 screen uses it to skip zero brackets, as the mixed screen does
__global__ void __launch_bounds__(1024) k_compact_nonzero_f64(const double* __restrict__ hn2, int count, double eta2,
                                                              int* __restrict__ nz_idx, int* __restrict__ nnz,
                                                              double* __restrict__ hn2c) {
  __shared__ int wsum[32];
  __shared__ int base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c0 = 0; c0 < count; c0 += 1024) {
    const int c = c0 + threadIdx.x;
    const int f = (c < count && hn2[c] > eta2) ? 1 : 0;
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
    if (f) {
      const int at = base + (w ? wsum[w - 1] : 0) + pre;
      nz_idx[at] = c;
      hn2c[at] = hn2[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) base += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *nnz = base;
}

// orthonormality defect of a block of Gram rows: max |G[i][j] - delta|
__global__ void k_defect_max(const double* __restrict__ G, int rows, int cols, int ldg, int r0,
                             unsigned long long* out_bits) {
  double m = 0.0;
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / cols), j = (int)(e % cols);
    const double g = G[(long long)i * ldg + j] - (r0 + i == j ? 1.0 : 0.0);
    m = fmax(m, fabs(g));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out_bits, dbits(m));
}

// two-pass forms of k_compact_nonzero_f64 (see cta_excl_scan)
__global__ void __launch_bounds__(kCmpThreads) k_nonzero_f64_pass1(const double* __restrict__ hn2, int count,
                                                                double eta2, int* __restrict__ part) {
  __shared__ int sw[kCmpThreads / 32];
  const int chunk = (count + gridDim.x - 1) / gridDim.x;
  const int c0 = blockIdx.x * chunk, c1 = min(count, c0 + chunk);
  int n = 0;
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) n += hn2[c] > eta2 ? 1 : 0;
  for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int i = 0; i < kCmpThreads / 32; ++i) t += sw[i];
    part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kCmpThreads) k_nonzero_f64_pass2(const double* __restrict__ hn2, int count,
                                                                double eta2, int* __restrict__ nz_idx,
                                                                int* __restrict__ nnz, double* __restrict__ hn2c,
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
  for (int t0 = c0; t0 < c1; t0 += blockDim.x) {
    const int c = t0 + threadIdx.x;
    const int f = (c < c1 && hn2[c] > eta2) ? 1 : 0;
    int tot;
    const int at = base + cta_excl_scan(f, &tot, wsum);
    if (f) {
      nz_idx[at] = c;
      hn2c[at] = hn2[c];
    }
    if (threadIdx.x == 0) base += tot;
    __syncthreads();
  }
}

__global__ void k_zero_stats(DevStats* stats, int ncur) {
  stats->ncur = ncur;
  stats->naccepted = 0;
  stats->nflag = 0;
  stats->ngray = 0;
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

namespace {
// Number of K splits.  FP64 work per CTA is uniform, so the CTA count should
// fill whole waves of the 152 SMs: S is the smallest split count giving at
// least c * 152 CTAs for the smallest c >= 1 whose last wave is >= 85 % full,
// subject to K / S >= 128 and the workspace holding S * M * N doubles.
int choose_splits(int M, int N, int K, int TM, int TN, size_t ws_doubles) {
  const long long tiles = (long long)((M + TM - 1) / TM) * ((N + TN - 1) / TN);
  const int smax_k = std::max(1, K / 128);
  const int smax_ws = (int)std::max<long long>(1, (long long)(ws_doubles / ((size_t)M * N)));
  const int smax = std::min(smax_k, smax_ws);
  if (tiles >= 4 * 152) return 1;
  int best = 1;
  double best_eff = 0.0;
  for (int S = 1; S <= smax; ++S) {
    const long long ctas = tiles * S;
    const long long waves = (ctas + 151) / 152;
    const double eff = (double)ctas / (double)(waves * 152);
    if (eff > best_eff + 1e-9) { best_eff = eff; best = S; }
    if (ctas >= 152 && eff >= 0.85) return S;
  }
  return best;
}

template <bool BT, int TM>
cudaError_t gemm_f64_tm(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
                        int ldc, bool subtract, double* ws, size_t ws_doubles, const int* run_if, cudaStream_t s) {
  constexpr int TN = 4096 / TM;
  const int S = ws ? choose_splits(M, N, K, TM, TN, ws_doubles) : 1;
  const int kchunk = (K + S - 1) / S;
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, S);
  if (S == 1) {
    k_gemm_f64<BT, TM><<<grid, 256, 0, s>>>(M, N, K, kchunk, A, lda, B, ldb, C, ldc, subtract ? 1 : 0, nullptr,
                                            run_if);
    return cudaGetLastError();
  }
  k_gemm_f64<BT, TM><<<grid, 256, 0, s>>>(M, N, K, kchunk, A, lda, B, ldb, C, ldc, 2, ws, run_if);
  k_reduce_f64<<<grid_for((long long)M * N, 256), 256, 0, s>>>(M, N, S, ws, C, ldc, subtract ? 1 : 0, run_if);
  return cudaGetLastError();
}

template <bool BT>
cudaError_t gemm_f64(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C, int ldc,
                     bool subtract, double* ws, size_t ws_doubles, const int* run_if, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  if (M < 128) return gemm_f64_tm<BT, 16>(M, N, K, A, lda, B, ldb, C, ldc, subtract, ws, ws_doubles, run_if, s);
  return gemm_f64_tm<BT, 64>(M, N, K, A, lda, B, ldb, C, ldc, subtract, ws, ws_doubles, run_if, s);
}
}  // namespace

cudaError_t gemm_nt_f64(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
                        int ldc, cudaStream_t s, double* ws, size_t ws_doubles, const int* run_if) {
  return gemm_f64<true>(M, N, K, A, lda, B, ldb, C, ldc, false, ws, ws_doubles, run_if, s);
}

cudaError_t gemm_nn_sub_f64(int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
                            int ldc, cudaStream_t s, double* ws, size_t ws_doubles, const int* run_if) {
  return gemm_f64<false>(M, N, K, A, lda, B, ldb, C, ldc, true, ws, ws_doubles, run_if, s);
}

cudaError_t rownorm2_f64(int M, int N, const double* A, int lda, double* out, cudaStream_t s, const int* run_if) {
  if (M <= 0) return cudaSuccess;
  k_rownorm2_f64<<<(M + 7) / 8, 256, 0, s>>>(M, N, A, lda, out, run_if);
  return cudaGetLastError();
}

cudaError_t gather_rows_f64(const double* src, int lds, const int* idx, int count, int ncols, double* dst,
                            int ldd, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  dim3 grid(grid_for(ncols, 256, 64), count);
  k_gather_rows<<<grid, 256, 0, s>>>(src, lds, idx, ncols, dst, ldd);
  return cudaGetLastError();
}

cudaError_t screen_compact_f64(const double* hn2, const double* rn2, int count, double eta2, double tau2,
                               double tau2_abs, int* idx, DevStats* stats, cudaStream_t s, const int* count_dev,
                               const int* map, int* part) {
  if (part) {
    k_screen_pass1<double><<<kCmpCtas, kCmpThreads, 0, s>>>(hn2, rn2, count, eta2, tau2, tau2_abs, stats, count_dev,
                                                            0, part);
    k_screen_pass2<double><<<kCmpCtas, kCmpThreads, 0, s>>>(hn2, rn2, count, eta2, tau2, tau2_abs, idx, stats,
                                                            count_dev, map, 0, nullptr, part, nullptr);
    return cudaGetLastError();
  }
  k_screen_compact<double><<<1, 1024, 0, s>>>(hn2, rn2, count, eta2, tau2, tau2_abs, idx, stats, count_dev, map, 0,
                                              nullptr);
  return cudaGetLastError();
}

cudaError_t screen_compact_f32(const float* hn2, const float* rn2, int count, float eta2, float tau2, int* idx,
                               DevStats* stats, cudaStream_t s, const int* count_dev, const int* map, int measured,
                               float* rho2_flag, int* part, int* cidx) {
  if (part) {
    k_screen_pass1<float><<<kCmpCtas, kCmpThreads, 0, s>>>(hn2, rn2, count, eta2, tau2, 0.f, stats, count_dev,
                                                           measured, part);
    k_screen_pass2<float><<<kCmpCtas, kCmpThreads, 0, s>>>(hn2, rn2, count, eta2, tau2, 0.f, idx, stats, count_dev,
                                                           map, measured, rho2_flag, part, cidx);
    return cudaGetLastError();
  }
  if (cidx) return cudaErrorInvalidValue;   // the single-CTA form writes no compacted positions
  k_screen_compact<float><<<1, 1024, 0, s>>>(hn2, rn2, count, eta2, tau2, 0.f, idx, stats, count_dev, map,
                                             measured, rho2_flag);
  return cudaGetLastError();
}

// co-resident CTAs of a cooperative launch of `kern` (256 threads), per device
static int coresident_ctas(const void* kern, int which) {
  static std::mutex mu;
  static int per_dev[2][128] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return 0;
  std::lock_guard<std::mutex> g(mu);
  if (!per_dev[which][dev]) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, 0);
    const int sms = device_sm_count();
    per_dev[which][dev] = std::max(1, sms * std::max(1, per));
  }
  return per_dev[which][dev];
}

// the sliced kernel runs on at most two CTAs per SM: more CTAs only shorten
// the slices and lengthen the partial sums and barriers
static int accept_wide_ctas() {
  const int co = coresident_ctas((const void*)k_accept_wide, 1);
  return std::max(1, std::min(co, 2 * device_sm_count()));
}

size_t accept_wide_part_doubles() { return (size_t)3 * kAcceptWideMaxRows * (size_t)(2 * device_sm_count()); }

// One CTA per row streams a row at one SM's bandwidth and leaves SMs idle
// when f is small; slicing the rows costs three grid barriers and
// 3 ceil((f - i - 1) / 8) CTA reductions per accept, which pay off once the
// rows are long.
// rows held in shared memory: one CTA per flagged row, all co-resident
static const void* accept_rowsmem_kernel(int P) {
  if (P <= 256) return (const void*)k_accept_rowsmem<1>;
  if (P <= 1024) return (const void*)k_accept_rowsmem<4>;
  if (P <= 4096) return (const void*)k_accept_rowsmem<16>;
  if (P <= 16384) return (const void*)k_accept_rowsmem<64>;
  return nullptr;
}

static bool accept_rowsmem_fits(int f, int P) {
  const void* kern = accept_rowsmem_kernel(P);
  if (!kern || (size_t)P * sizeof(double) > kAcceptRowSmemMax) return false;
  const int bytes = P * (int)sizeof(double);
  if (smem_optin(kern, bytes) != cudaSuccess) return false;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, bytes) != cudaSuccess) return false;
  return f <= per * device_sm_count();
}

int accept_kernel_for(int f, int P, int requested) {
  if (f > kAcceptWideMaxRows) return 1;
  if (requested == 3) return accept_rowsmem_fits(f, P) ? 3 : 1;
  if (requested == 1 || requested == 2) return requested;
  if (P >= (1 << 18)) return 2;
  if (P >= (1 << 16) && f <= 32) return 2;
  if (accept_rowsmem_fits(f, P)) return 3;
  return 1;
}

cudaError_t accept_seq(int f, double* R, int ldr, double* rn2, const double* hn2, double tol_rel2, double tol_abs2,
                       double eta2, double* V, int ldv, int ncap, int P, DevStats* stats, DevStatus* st,
                       unsigned int* bar, long long spin_cap, cudaStream_t s, int phantom, const double* Hraw,
                       double* Bk, double* bn2, const float* rho2_screen, int kernel, double* wpart) {
  if (f <= 0) return cudaSuccess;
  uint64_t lim = spin_cap > 0 ? (uint64_t)spin_cap : 4000000000ull;
  if (kernel == 2) {
    if (f > kAcceptWideMaxRows || !wpart) return cudaErrorInvalidValue;
    const int G = accept_wide_ctas();
    void* args[] = {&f,    &R,   &ldr,  &rn2,  (void*)&hn2, &tol_rel2, &tol_abs2,          &eta2,
                    &V,    &ldv, &ncap, &P,    &stats,      &st,       &bar,               &lim,
                    &phantom, (void*)&Hraw, &Bk, &bn2, (void*)&rho2_screen, &wpart};
    return cudaLaunchCooperativeKernel((const void*)k_accept_wide, dim3(G), dim3(256), args, 0, s);
  }
  if (kernel == 3) {
    if (!accept_rowsmem_fits(f, P)) return cudaErrorInvalidValue;
    void* args[] = {&f,     &R,   &ldr, &rn2, (void*)&hn2, &tol_rel2,    &tol_abs2, &eta2, &V,   &ldv,
                    &ncap,  &P,   &stats, &st, &bar,       &lim,         &phantom,  (void*)&Hraw, &Bk, &bn2,
                    (void*)&rho2_screen};
    return cudaLaunchCooperativeKernel(accept_rowsmem_kernel(P), dim3(f), dim3(256), args,
                                       (size_t)P * sizeof(double), s);
  }
  const int nblocks = coresident_ctas((const void*)k_accept_seq, 0);
  if (nblocks <= 0) return cudaErrorInvalidDevice;
  const int G = std::max(1, std::min(std::min(nblocks, device_sm_count()), f));
  void* args[] = {&f,     &R,   &ldr, &rn2, (void*)&hn2, &tol_rel2,    &tol_abs2, &eta2, &V,   &ldv,
                  &ncap,  &P,   &stats, &st, &bar,       &lim,         &phantom,  (void*)&Hraw, &Bk, &bn2,
                  (void*)&rho2_screen};
  return cudaLaunchCooperativeKernel((const void*)k_accept_seq, dim3(G), dim3(256), args, 0, s);
}

cudaError_t need_pass2(int f, const double* hn2, const double* rn2, double eta2, double tol_rel2, double tol_abs2,
                       int* need, cudaStream_t s) {
  k_need_pass2<<<1, 256, 0, s>>>(f, hn2, rn2, eta2, tol_rel2, tol_abs2, need);
  return cudaGetLastError();
}

cudaError_t compact_nonzero_f64(const double* hn2, int count, double eta2, int* nz_idx, int* nnz, double* hn2c,
                                cudaStream_t s, int* part) {
  if (part) {
    k_nonzero_f64_pass1<<<kCmpCtas, kCmpThreads, 0, s>>>(hn2, count, eta2, part);
    k_nonzero_f64_pass2<<<kCmpCtas, kCmpThreads, 0, s>>>(hn2, count, eta2, nz_idx, nnz, hn2c, part);
    return cudaGetLastError();
  }
  k_compact_nonzero_f64<<<1, 1024, 0, s>>>(hn2, count, eta2, nz_idx, nnz, hn2c);
  return cudaGetLastError();
}

cudaError_t defect_max(const double* G, int rows, int cols, int ldg, int r0, unsigned long long* out_bits,
                       cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  k_defect_max<<<grid_for((long long)rows * cols, 256), 256, 0, s>>>(G, rows, cols, ldg, r0, out_bits);
  return cudaGetLastError();
}

cudaError_t zero_stats(DevStats* stats, int ncur, cudaStream_t s) {
  k_zero_stats<<<1, 1, 0, s>>>(stats, ncur);
  return cudaGetLastError();
}

}  // namespace lc
