// Internal declarations shared by the library's translation units.
//
// Packed representation (used by every kernel): an anti-Hermitian a = iH is
// stored as P = d*d reals S, row-major d x d:
//   S[j][j] = H[j][j] / sqrt(d)
//   S[j][k] = sqrt(2/d) * Re H[j][k]   (j < k)
//   S[k][j] = sqrt(2/d) * Im H[j][k]   (j < k)
// With this scaling the paper's inner product <a, b> = tr(a^dagger b)/d
// (Section 2.2) is the plain dot product of the packed rows, so an
// orthonormal basis V is a matrix with orthonormal rows and the projection of
// Section 3.2 is two ordinary GEMMs.  tr(a^dagger b) is real for anti-Hermitian
// a and b, so real coefficients suffice and real and complex linear
// independence coincide.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>
#include <map>
#include <mutex>
#include <set>
#include <utility>

#include "../../include/lieclosure.h"

namespace lc {

// Device-side error word: the first failing check wins.
struct DevStatus {
  int code;            // lc_status value, 0 = ok
  int where;           // kernel-specific site id
  long long info;      // e.g. the spin iteration count or an index
};

enum : int {
  SITE_NONE = 0,
  SITE_ACCEPT_CAPACITY = 1,
  SITE_GEMM_TMA_WAIT = 2,
  SITE_GEMM_MMA_WAIT = 3,
  SITE_GEMM_EPI_WAIT = 4,
  SITE_ACCEPT_BARRIER = 5,
};

// Accept-path statistics kept on the device (doubles stored by bit pattern so
// that integer atomicMin/atomicMax order them; all values are >= 0).
struct DevStats {
  unsigned long long min_acc_bits;
  unsigned long long max_rej_bits;
  unsigned long long max_screen_rej_bits;  // largest screened rel. residual among screen rejects
  unsigned long long eps_bits;             // largest probe residual of the run (screen noise floor)
  unsigned long long min_acc_screen_bits;  // smallest screened rel. residual among accepts
  int ncur;            // current |V| (rows of the FP64 basis)
  int naccepted;       // accepts in the current block
  int nflag;           // flagged candidates in the current block
  int nnonzero;        // candidates above the norm floor in the current block
  int ngray;           // screen rejects in (eps, tau] in the current block
  float tau2;          // measured screen threshold tau^2 (mixed mode)
  float eps2;          // latest probe's eps^2
  unsigned int min_rho2_flag_bits;  // float bits: smallest screened rho^2 among the block's flagged rows
};

// pair index t = l(l-1)/2 + m, 0 <= m < l  <->  (l, m)
__host__ __device__ inline void pair_from_index(long long t, int* l, int* m) {
  long long L = (long long)((1.0 + sqrt(1.0 + 8.0 * (double)t)) * 0.5);
  while (L * (L - 1) / 2 > t) --L;
  while ((L + 1) * L / 2 <= t) ++L;
  *l = (int)L;
  *m = (int)(t - L * (L - 1) / 2);
}

inline long long pairs_below(long long n) { return n * (n - 1) / 2; }

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }
inline long long round_up_ll(long long x, long long m) { return (x + m - 1) / m * m; }

// Dynamic shared memory above 48 KB is an opt-in attribute of a kernel in
// one device's context (the launch limit for that kernel), so it is raised
// per (kernel, device) with the device current, never lowered: a kernel
// launched with several sizes keeps the largest limit asked for.  Up to the
// default 48 KB nothing is set.
inline cudaError_t smem_optin(const void* kernel, int bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  const auto key = std::make_pair(kernel, dev);
  auto it = limit.find(key);
  if (it != limit.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) limit[key] = bytes;
  return e;
}

// Multiprocessor count of the current device (cached per device).
inline int device_sm_count() {
  static std::mutex mu;
  static int cache[128] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return 1;
  std::lock_guard<std::mutex> g(mu);
  if (!cache[dev]) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = sms > 0 ? sms : 1;
  }
  return cache[dev];
}

// Multi-CTA ordered compaction: kCmpCtas contiguous chunks, kCmpThreads
// threads per CTA; part[] holds per-chunk counts between the two passes.
constexpr int kCmpCtas = 64;
constexpr int kCmpThreads = 256;

// exclusive prefix of f over the CTA (kCmpThreads threads), *total = the CTA's sum
__device__ __forceinline__ int cta_excl_scan(int f, int* total, int* wsum) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned mask = __ballot_sync(0xffffffffu, f);
  const int pre = __popc(mask & ((1u << lane) - 1u));
  if (lane == 0) wsum[w] = __popc(mask);
  __syncthreads();
  if (w == 0) {
    int v = lane < kCmpThreads / 32 ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += n;
    }
    if (lane < kCmpThreads / 32) wsum[lane] = v;          // inclusive
  }
  __syncthreads();
  const int r = (w ? wsum[w - 1] : 0) + pre;
  *total = wsum[kCmpThreads / 32 - 1];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------ FP64 kernels
// (lc_fp64.cu)
cudaError_t pack_generators(const double2* g, int k, int d, int ldp, double* out,
                            double* dev_maxdev, double* dev_maxabs, int* dev_nonfinite,
                            cudaStream_t s);
cudaError_t unpack_basis(const double* V, int n, int d, int ldp, double2* out, cudaStream_t s);
// brackets of pairs t0 + i, i = 0 .. count-1 (or t0 + idx[i] when idx is
// given), packed into rows of out (row stride ldo)
cudaError_t bracket_fp64(const double* V, int d, int ldv, long long t0, const int* idx,
                         int count, double* out, int ldo, cudaStream_t s);
// C = A * B^T and C = C - A * B; row-major FP64.  ws (optional, ws_doubles
// long) enables split-K for small outputs; run_if (optional, device): skip the
// launch's work when *run_if == 0.
cudaError_t gemm_nt_f64(int M, int N, int K, const double* A, int lda, const double* B, int ldb,
                        double* C, int ldc, cudaStream_t s, double* ws = nullptr, size_t ws_doubles = 0,
                        const int* run_if = nullptr);
cudaError_t gemm_nn_sub_f64(int M, int N, int K, const double* A, int lda, const double* B,
                            int ldb, double* C, int ldc, cudaStream_t s, double* ws = nullptr,
                            size_t ws_doubles = 0, const int* run_if = nullptr);
cudaError_t rownorm2_f64(int M, int N, const double* A, int lda, double* out, cudaStream_t s,
                         const int* run_if = nullptr);
// the in-block sequential test-and-append of f flagged rows, one cooperative
// launch (bar: two zeroed unsigned ints).  Accept iff hn2 > eta2 and
// rn2 > tol_rel2 * hn2 + tol_abs2 (relative or absolute tolerance);
// rho2_screen (optional): the rows' screened relative residuals squared.
// kernel: 1 = one CTA per row (k_accept_seq), 2 = every row sliced across the
// grid (k_accept_wide; f <= kAcceptWideMaxRows, wpart holds
// accept_wide_part_doubles() doubles), 3 = one CTA per row with the row in
// shared memory (k_accept_rowsmem; P <= 16384 and P doubles <= kAcceptRowSmemMax bytes, f
// co-resident CTAs), 0 = by shape
constexpr int kAcceptWideMaxRows = 128;
constexpr size_t kAcceptRowSmemMax = 200 * 1024;
size_t accept_wide_part_doubles();
int accept_kernel_for(int f, int P, int requested);
cudaError_t accept_seq(int f, double* R, int ldr, double* rn2, const double* hn2, double tol_rel2, double tol_abs2,
                       double eta2, double* V, int ldv, int ncap, int P, DevStats* stats, DevStatus* st,
                       unsigned int* bar, long long spin_cap, cudaStream_t s, int phantom = 0,
                       const double* Hraw = nullptr, double* Bk = nullptr, double* bn2 = nullptr,
                       const float* rho2_screen = nullptr, int kernel = 1, double* wpart = nullptr);
// *need = 1 iff some row needs a second Gram-Schmidt pass
cudaError_t need_pass2(int f, const double* hn2, const double* rn2, double eta2, double tol_rel2, double tol_abs2,
                       int* need, cudaStream_t s);
cudaError_t gather_rows_f64(const double* src, int lds, const int* idx, int count, int ncols,
                            double* dst, int ldd, cudaStream_t s);
// flags candidates with hn2 > eta^2 and rn2 > tau^2 hn2 + tau2_abs; writes the
// flagged candidate positions in order to idx and their count to stats->nflag
// part (optional, >= 3 * 64 ints of device scratch): use the multi-CTA
// two-pass form instead of one CTA
cudaError_t screen_compact_f64(const double* hn2, const double* rn2, int count, double eta2,
                               double tau2, double tau2_abs, int* idx, DevStats* stats, cudaStream_t s,
                               const int* count_dev = nullptr, const int* map = nullptr, int* part = nullptr);
// ordered indices of the candidates with hn2 > eta2, their count (*nnz) and
// norms (part: optional scratch of kCmpCtas ints for the multi-CTA form)
cudaError_t compact_nonzero_f64(const double* hn2, int count, double eta2, int* nz_idx, int* nnz,
                                double* hn2c, cudaStream_t s, int* part = nullptr);
// count_dev (optional): live count on the device; map (optional): idx[i] = map[position];
// measured != 0: tau^2 is stats->tau2 (the probe's threshold) and screen rejects
// with rho^2 > stats->eps2 are counted in stats->ngray; rho2_flag (optional)
// receives the flagged candidates' rn2 / hn2 in flag order
cudaError_t screen_compact_f32(const float* hn2, const float* rn2, int count, float eta2,
                               float tau2, int* idx, DevStats* stats, cudaStream_t s,
                               const int* count_dev = nullptr, const int* map = nullptr, int measured = 0,
                               float* rho2_flag = nullptr, int* part = nullptr, int* cidx = nullptr);
cudaError_t zero_stats(DevStats* stats, int ncur, cudaStream_t s);

// ------------------------------------------------------ FP64-accurate tensor-core GEMM
// (lc_tcgen05.cu)  An operand as a stack of S BF16 digit slices: slice s of
// row i at slices[(s * rows + i) * ld + k]; row i's value is
// 2^{e_i} sum_s 2^{-beta (s+1)} d_s(i, k) with e_i = exps[i] (or fixed_e
// when exps is null).
struct OzOperand {
  const __nv_bfloat16* slices;
  int rows;        // rows per slice (the stack's row stride between slices)
  int ld;          // elements per row, multiple of 8
  const int* exps;
  int fixed_e;
  long long total_rows = 0;   // rows the stack holds from `slices` on (0: S * rows)
};
int oz_beta_for(int K);          // digit width for contractions up to K terms
int oz_slices_for(int beta);     // slices for >= 54 bits
long long oz_max_k(int beta);    // longest exact FP32 chain for that width
// rows [0, rows) of X into slice rows [row0, row0 + rows); per-row exponents
// to exps[row0 + r] (or fixed_e when exps is null); columns [cols, cols_pad)
// of the slices are written as zero digits
// (col_exp: column c sliced as x[c] 2^col_exp[c])
cudaError_t oz_slice_rows(const double* X, int rows, int cols, int ldx, int S, int beta, int fixed_e,
                          __nv_bfloat16* out, int rows_alloc, int lds, int* exps, int row0, const int* run_if,
                          cudaStream_t s, int cols_pad = 0, const int* col_exp = nullptr);
// rows [r0, r1) of V as columns j - jbase of the transposed slices
// outT[s][p][j - jbase], row j in units of 2^row_exp[j]
cudaError_t oz_slice_cols(const double* V, int r0, int r1, int P, int ldv, int S, int beta, const int* row_exp,
                          __nv_bfloat16* outT, int P_alloc, int ldt, cudaStream_t s, int jbase = 0);
// C (M x N, ldc) = A B^T (or C -= A B^T) to FP64 accuracy; ws holds the
// FP64 partials of a K split (M * N doubles per split)
// max_level: slice pairs (s, t) with s + t <= max_level run (default S - 1;
// S keeps one level more, which brings the pairs dropped below the slices'
// own rounding)
cudaError_t ozaki_gemm_nt(int M, int N, int K, const OzOperand& A, const OzOperand& B, int S, int beta, double* C,
                          int ldc, bool subtract, double* ws, size_t ws_doubles, const int* run_if,
                          long long spin_cap, DevStatus* st, cudaStream_t s, long long* launches,
                          int max_level = -1);

// ------------------------------------------------------ mixed-precision path
// (lc_mixed.cu)
// FP64 rows [r0, r1) of V -> split BF16 copies (row-major and transposed)
cudaError_t split_rows(const double* V, int ldv, int r0, int r1, int P,
                       __nv_bfloat16* Vhi, __nv_bfloat16* Vlo, int ldvs,
                       __nv_bfloat16* VThi, __nv_bfloat16* VTlo, int ldvt, cudaStream_t s);
// brackets of pairs t0..t0+count-1 in FP32, written as split BF16 rows plus
// FP32 squared norms
cudaError_t bracket_mixed(const double* V, int d, int ldv, long long t0, int count,
                          __nv_bfloat16* Hhi, __nv_bfloat16* Hlo, int ldh, float* hn2,
                          cudaStream_t s);

// screen noise probe: S rows in span(V) (S1 single basis rows, the rest
// random 16-row combinations) as split BF16 candidate rows with their squared
// norms; *nnz = S.  probe_eps: stats->eps2 = max rn2 / hn2 over the S rows,
// stats->tau2 = clamp(kappa^2 eps2, tau_lo^2, tau_hi^2), eps_bits = run max.
cudaError_t probe_rows(const double* V, int ldv, int N, int P, int S, int S1, unsigned long long seed,
                       __nv_bfloat16* Chi, __nv_bfloat16* Clo, int ldc, float* hn2c, int* nnz, cudaStream_t s);
cudaError_t probe_eps(const float* hn2c, const float* rn2, int S, DevStats* stats, float kappa, float tau_lo,
                      float tau_hi, cudaStream_t s);
// max |G - I| of the Gram rows [r0, r0 + rows) (rows x cols, row stride ldg)
// into *out_bits (a double's bit pattern, atomicMax)
cudaError_t defect_max(const double* G, int rows, int cols, int ldg, int r0, unsigned long long* out_bits,
                       cudaStream_t s);

// real 2d x 2d embeddings [[Hr, -Hi], [-Hi, -Hr]] of basis rows [r0, r1), split BF16
// (perm: rows in the large-d bracket order, see lc_tcgen05.cu)
cudaError_t build_embedding(const double* V, int ldv, int r0, int r1, int d, __nv_bfloat16* Ehi,
                            __nv_bfloat16* Elo, cudaStream_t s, int perm = 0);
// [Hr; Hi] (2d x d, split BF16) of basis rows [r0, r1): operands of bracket_q64
cudaError_t build_q(const double* V, int ldv, int r0, int r1, int d, __nv_bfloat16* Qhi, __nv_bfloat16* Qlo,
                    cudaStream_t s);
// tensor-core brackets for d = 64 from the [Hr; Hi] rows (nelems elements)
cudaError_t bracket_q64(const __nv_bfloat16* Qhi, const __nv_bfloat16* Qlo, long long nelems, long long t0, int count,
                        __nv_bfloat16* Hhi, __nv_bfloat16* Hlo, int ldh, float* hn2, long long spin_cap,
                        DevStatus* st, cudaStream_t s);
// ordered indices of the candidates with hn2 > eta2; their count to *nnz (device)
// (bn2, optional: squared norms of the bracket operands' rows; the floor is
// then eta2 * bn2[l] * bn2[m] for the pair t0 + position)
cudaError_t compact_nonzero(const float* hn2, int count, float eta2, int* nz_idx, int* nnz, cudaStream_t s,
                            const double* bn2 = nullptr, long long t0 = 0, int* part = nullptr);
// rows nz_idx[0 .. *nnz) of H (and their norms) -> consecutive rows of C
cudaError_t gather_candidates(const __nv_bfloat16* Hhi, const __nv_bfloat16* Hlo, int ldh, const float* hn2,
                              const int* nz_idx, const int* nnz, int count, int ncols, __nv_bfloat16* Chi,
                              __nv_bfloat16* Clo, float* hn2c, cudaStream_t s);
// beta (f x n, FP64, row stride ldb) = the screening coefficients D = H V^T
// (BF16 hi + lo, row stride ldd) of the compacted rows cidx[0..f)
cudaError_t gather_coef(const __nv_bfloat16* Dhi, const __nv_bfloat16* Dlo, int ldd, const int* cidx, int f, int n,
                        double* beta, int ldb, cudaStream_t s);
// tensor-core brackets (d = 64, 128) from the embeddings E (nelems elements)
bool bracket_tc_supported(int d);
cudaError_t bracket_tc(const __nv_bfloat16* Ehi, const __nv_bfloat16* Elo, long long nelems, int d, long long t0,
                       int count, __nv_bfloat16* Hhi, __nv_bfloat16* Hlo, int ldh, float* hn2, long long spin_cap,
                       DevStatus* st, cudaStream_t s);
// tensor-core brackets for d >= 256, d % 128 == 0, from the permuted embeddings
bool bracket_big_supported(int d);
cudaError_t bracket_big(const __nv_bfloat16* Ehi, const __nv_bfloat16* Elo, long long nelems, int d, long long t0,
                        int count, __nv_bfloat16* Hhi, __nv_bfloat16* Hlo, int ldh, float* hn2, long long spin_cap,
                        DevStatus* st, cudaStream_t s);

// Algorithm 2, the matrix-inversion method (lc_alg2.cu), FP64 throughout
int closure_alg2_device(const double2* d_gens, int k, int d, double tol, double2* d_out, long long* dim_out,
                        long long max_dim, const lc_options& o, lc_report* rep, cudaStream_t s);

// tcgen05 split-BF16 GEMMs (lc_tcgen05.cu).  All operands K-major BF16.
// D[M x N] = Ahi*Bhi^T + Ahi*Blo^T + Alo*Bhi^T with FP32 accumulation.
struct SplitGemmArgs {
  const __nv_bfloat16 *Ahi, *Alo;  // M x K, row stride lda (elements)
  const __nv_bfloat16 *Bhi, *Blo;  // N x K, row stride ldb
  int M, N, K, lda, ldb;           // M % 128, N % split_gemm_tile_n(), K % split_gemm_tile_k() == 0
  const int* Mdev;                 // optional device row count: CTAs at or past it exit
  // epilogue 0: store split BF16 of D to Dhi/Dlo (row stride ldd)
  __nv_bfloat16 *Dhi, *Dlo;
  int ldd;
  // epilogue 1: rn2[m] += sum_n (H[m][n] - D[m][n])^2 with H = Hhi + Hlo (stride ldh)
  const __nv_bfloat16 *Hhi, *Hlo;
  int ldh;
  float* rn2;
  float* Df32;                     // epilogue 2: plain FP32 store (tests)
  int epilogue;
  long long spin_cap;
  DevStatus* st;
  int cfg;                         // tile configuration, 0 .. split_gemm_num_cfgs() - 1
  // optional FP32 workspace for a split-K projection (epilogue 0 with fewer
  // output tiles than SMs); null = no split
  float* ws;
  size_t ws_floats;
  long long* launches;             // optional: incremented by the kernels launched
};
cudaError_t split_gemm_tcgen05(const SplitGemmArgs& a, cudaStream_t s);
// tile extents of split_gemm_tcgen05: with N a multiple of split_gemm_tile_n(),
// K of split_gemm_tile_k() and M of 128 every configuration applies;
// the (int cfg) forms give one configuration's output tile width and k-slice
int split_gemm_num_cfgs();
int split_gemm_tile_n();
int split_gemm_tile_k();
int split_gemm_tile_n(int cfg);
int split_gemm_tile_k(int cfg);
bool tcgen05_available();

}  // namespace lc
