// Algorithm 2 of arXiv 2506.01120 (Section 3.1): the matrix-inversion method.
//
// B holds unit-norm operators (packed FP64 rows, the same packing as the rest
// of the library, so <a, b> is a plain dot product and the Gram matrix A is
// real symmetric for anti-Hermitian inputs).  A candidate h, normalised, is
// independent iff r = h - B^T (A^-1 beta) != 0 with beta = B h (Theorem 1);
// the test reads "!= 0" as ||r|| > tol.  Brackets are formed from B.
//
// Block form.  A block of pairs is screened in FP64 with three GEMMs
// (beta = H B^T, X = beta A^-1, R = H - X B); candidates with ||r|| <= tol/2
// against the block-start B stay dependent as B grows (the residual against a
// larger span is smaller) and are rejected.  The others are re-tested in pair
// order against the current B and A^-1, and on accept B grows by h and A^-1 by
// the bordered-inverse identity
//   [[A, b], [b^T, 1]]^-1 = [[A^-1 + x x^T / s, -x / s], [-x^T / s, 1 / s]],
//   x = A^-1 b, s = 1 - b^T x,
// which is the inverse Algorithm 2 stores, updated in O(N^2) instead of being
// recomputed.  s is taken as ||r||^2 (equal to 1 - b^T x in exact arithmetic,
// and not subject to cancellation when r is small).
#include "lc_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

namespace lc {
namespace {

__device__ inline double warp_sum2(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// rows with hn2 > eta2 scaled to unit norm (unit[i] = 1), others zeroed (0)
__global__ void k_normalise_rows(double* __restrict__ H, int ldh, int rows, int P, const double* __restrict__ hn2,
                                 double eta2, double* __restrict__ unit) {
  const int i = blockIdx.x;
  if (i >= rows) return;
  const double h2 = hn2[i];
  const double sc = h2 > eta2 ? 1.0 / sqrt(h2) : 0.0;
  double* h = H + (long long)i * ldh;
  for (int p = threadIdx.x; p < P; p += blockDim.x) h[p] *= sc;
  if (threadIdx.x == 0) unit[i] = h2 > eta2 ? 1.0 : 0.0;
}

// beta_j = <B_j, h> for j < N (one warp per row of B)
__global__ void k_a2_beta(const double* __restrict__ B, int ldb, const int* __restrict__ ncur,
                          const double* __restrict__ h, int P, double* __restrict__ beta, double* __restrict__ rr2) {
  const int N = *ncur;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (blockIdx.x == 0 && threadIdx.x == 0) *rr2 = 0.0;
  if (j >= N) return;
  const double* b = B + (long long)j * ldb;
  double s = 0.0;
  for (int p = threadIdx.x & 31; p < P; p += 32) s = fma(b[p], h[p], s);
  s = warp_sum2(s);
  if ((threadIdx.x & 31) == 0) beta[j] = s;
}

// x = A^-1 beta (one warp per row of A^-1)
__global__ void k_a2_x(const double* __restrict__ Ainv, int lda, const int* __restrict__ ncur,
                       const double* __restrict__ beta, double* __restrict__ x) {
  const int N = *ncur;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= N) return;
  const double* a = Ainv + (long long)j * lda;
  double s = 0.0;
  for (int q = threadIdx.x & 31; q < N; q += 32) s = fma(a[q], beta[q], s);
  s = warp_sum2(s);
  if ((threadIdx.x & 31) == 0) x[j] = s;
}

// r = h - B^T x, ||r||^2 accumulated into *rr2
__global__ void k_a2_resid(const double* __restrict__ B, int ldb, const int* __restrict__ ncur,
                           const double* __restrict__ x, const double* __restrict__ h, int P,
                           double* __restrict__ rr2) {
  __shared__ double red[32];
  const int N = *ncur;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  double r = 0.0;
  if (p < P) {
    double acc = h[p];
    for (int j = 0; j < N; ++j) acc = fma(-x[j], B[(long long)j * ldb + p], acc);
    r = acc * acc;
  }
  r = warp_sum2(r);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    t = warp_sum2(t);
    if (threadIdx.x == 0) atomicAdd(rr2, t);
  }
}

// accept test; on accept append h to B and border A^-1 (every element of the
// (N+1) x (N+1) inverse); the count itself is advanced by k_a2_commit
__global__ void k_a2_append(double* __restrict__ B, int ldb, double* __restrict__ Ainv, int lda,
                            const int* __restrict__ ncur, int ncap, const double* __restrict__ x,
                            const double* __restrict__ h, int P, const double* __restrict__ rr2,
                            const double* __restrict__ unit, double tol, int* __restrict__ accepted, DevStatus* st) {
  const int N = *ncur;
  const double s = *rr2;
  const bool acc = *unit > 0.0 && s > tol * tol;
  if (blockIdx.x == 0 && threadIdx.x == 0) *accepted = (acc && N < ncap) ? 1 : 0;
  if (!acc) return;
  if (N >= ncap) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && atomicCAS(&st->code, 0, (int)LC_ERR_CAPACITY) == 0) {
      st->where = SITE_ACCEPT_CAPACITY;
      st->info = N;
    }
    return;
  }
  const double inv_s = 1.0 / s;
  const long long n1 = N + 1;
  const long long tot = n1 * n1 + P;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < n1 * n1) {
      const int a = (int)(e / n1), b = (int)(e % n1);
      double* A = Ainv + (long long)a * lda + b;
      if (a < N && b < N) *A += x[a] * x[b] * inv_s;
      else if (a < N) *A = -x[a] * inv_s;
      else if (b < N) *A = -x[b] * inv_s;
      else *A = inv_s;
    } else {
      const int p = (int)(e - n1 * n1);
      B[(long long)N * ldb + p] = h[p];
    }
  }
}

__global__ void k_a2_commit(int* __restrict__ ncur, const int* __restrict__ accepted) {
  if (*accepted) *ncur += 1;
}

__global__ void k_a2_rows_unit(const double* __restrict__ unit_all, const int* __restrict__ idx, int f,
                               double* __restrict__ unit) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < f) unit[i] = unit_all[idx[i]];
}

double now_s2() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

#define A2_TRY(x)                                                              \
  do {                                                                         \
    cudaError_t e_ = (x);                                                      \
    if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? LC_ERR_OOM : LC_ERR_CUDA; \
  } while (0)

class Closure2 {
 public:
  Closure2(int k, int d, double tol, long long ncap, const lc_options& o, cudaStream_t s)
      : k_(k), d_(d), tol_(tol), ncap_(ncap), opt_(o), s_(s) {
    P_ = d * d;
    ldp_ = round_up(P_, 128);
    eta_ = o.eta_abs > 0 ? o.eta_abs : 1e-12;
    int K = o.block_k > 0 ? o.block_k : 1024;
    const double per = 24.0 * ldp_ + 16.0 * ncap_;
    K = (int)std::min<double>(K, std::max(1.0, 4.0e9 / per));
    K_ = std::max(K, k);
  }
  ~Closure2() {
    if (base_) cudaFreeAsync(base_, s_);
    if (host_) cudaFreeHost(host_);
  }

  int run(const double2* d_gens, double2* d_out, long long* dim_out, lc_report* rep) {
    const double t0 = now_s2();
    int rc = setup(d_gens);
    if (rc == LC_OK) {
      // generator pass: the normalised generators, in order
      A2_TRY(cudaMemcpy2DAsync(R64_, sizeof(double) * ldp_, G64_, sizeof(double) * ldp_, sizeof(double) * P_, k_,
                               cudaMemcpyDeviceToDevice, s_));
      A2_TRY(rownorm2_f64(k_, P_, R64_, ldp_, hn2_, s_));
      k_normalise_rows<<<k_, 256, 0, s_>>>(R64_, ldp_, k_, P_, hn2_, eta_ * eta_, unitf_);
      A2_TRY(cudaGetLastError());
      rc = sequential(k_);
    }
    if (rc == LC_OK) rc = sweep();
    if ((rc == LC_OK || rc == LC_ERR_CAPACITY) && d_out && N_ > 0)
      if (unpack_basis(B64_, (int)N_, d_, ldp_, d_out, s_) != cudaSuccess) rc = LC_ERR_CUDA;
    if (cudaStreamSynchronize(s_) != cudaSuccess && rc == LC_OK) rc = LC_ERR_CUDA;
    if (dim_out) *dim_out = N_;
    if (rep) {
      memset(rep, 0, sizeof(*rep));
      rep->dim = N_;
      rep->brackets_checked = checked_;
      rep->generators_checked = k_;
      rep->n_flagged = flagged_;
      rep->n_blocks = blocks_;
      int l = 1, m = 0;
      if (t_ > 0) pair_from_index(t_, &l, &m);
      rep->cursor_l = l;
      rep->cursor_m = m;
      rep->t_total_s = now_s2() - t0;
      rep->precision = LC_PREC_FP64;
      rep->status = rc;
    }
    return rc;
  }

 private:
  int k_, d_, P_, ldp_, K_;
  double tol_, eta_;
  long long ncap_;
  lc_options opt_;
  cudaStream_t s_;
  char* base_ = nullptr;
  struct Host {
    DevStats stats;
    DevStatus st;
    double chk[2];
    int nonfinite;
  }* host_ = nullptr;
  double *G64_, *B64_, *Ainv_, *H64_, *R64_, *beta_, *X_, *hn2_, *rn2_, *unit_, *unitf_, *vb_, *vx_, *rr2_,
      *chk_;
  int *idx_, *ncur_, *accepted_, *nonfinite_;
  DevStats* stats_;
  DevStatus* st_;
  long long N_ = 0, t_ = 0, checked_ = 0, flagged_ = 0, blocks_ = 0;

  int setup(const double2* d_gens) {
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t at = off; off = (off + bytes + 255) & ~size_t(255); return at; };
    const size_t oG = take(8ull * k_ * ldp_), oB = take(8ull * ncap_ * ldp_), oA = take(8ull * ncap_ * ncap_);
    const size_t oH = take(8ull * K_ * ldp_), oR = take(8ull * K_ * ldp_), obe = take(8ull * K_ * ncap_);
    const size_t oX = take(8ull * K_ * ncap_), ohn = take(8ull * K_), orn = take(8ull * K_), oun = take(8ull * K_);
    const size_t ouf = take(8ull * K_), ovb = take(8ull * ncap_), ovx = take(8ull * ncap_), orr = take(8);
    const size_t och = take(16), oid = take(4ull * K_), onc = take(4), oac = take(4), onf = take(4);
    const size_t ost = take(sizeof(DevStats)), oss = take(sizeof(DevStatus));
    A2_TRY(cudaHostAlloc(reinterpret_cast<void**>(&host_), sizeof(Host), cudaHostAllocDefault));
    A2_TRY(cudaMallocAsync(reinterpret_cast<void**>(&base_), off, s_));
    auto at = [&](size_t o) { return base_ + o; };
    G64_ = (double*)at(oG); B64_ = (double*)at(oB); Ainv_ = (double*)at(oA); H64_ = (double*)at(oH);
    R64_ = (double*)at(oR); beta_ = (double*)at(obe); X_ = (double*)at(oX); hn2_ = (double*)at(ohn);
    rn2_ = (double*)at(orn); unit_ = (double*)at(oun); unitf_ = (double*)at(ouf); vb_ = (double*)at(ovb);
    vx_ = (double*)at(ovx); rr2_ = (double*)at(orr); chk_ = (double*)at(och); idx_ = (int*)at(oid);
    ncur_ = (int*)at(onc); accepted_ = (int*)at(oac); nonfinite_ = (int*)at(onf);
    stats_ = (DevStats*)at(ost); st_ = (DevStatus*)at(oss);
    A2_TRY(cudaMemsetAsync(base_, 0, off, s_));
    A2_TRY(pack_generators(d_gens, k_, d_, ldp_, G64_, chk_, chk_ + 1, nonfinite_, s_));
    A2_TRY(cudaMemcpyAsync(host_->chk, chk_, 16, cudaMemcpyDeviceToHost, s_));
    A2_TRY(cudaMemcpyAsync(&host_->nonfinite, nonfinite_, 4, cudaMemcpyDeviceToHost, s_));
    A2_TRY(cudaStreamSynchronize(s_));
    if (host_->nonfinite) return LC_ERR_NONFINITE;
    if (host_->chk[0] > 1e-12 * host_->chk[1]) return LC_ERR_NOT_ANTIHERMITIAN;
    return LC_OK;
  }

  int read_state() {
    int n = 0;
    A2_TRY(cudaMemcpyAsync(&host_->stats, stats_, sizeof(DevStats), cudaMemcpyDeviceToHost, s_));
    A2_TRY(cudaMemcpyAsync(&host_->st, st_, sizeof(DevStatus), cudaMemcpyDeviceToHost, s_));
    A2_TRY(cudaMemcpyAsync(&n, ncur_, 4, cudaMemcpyDeviceToHost, s_));
    A2_TRY(cudaStreamSynchronize(s_));
    N_ = n;
    return host_->st.code;
  }

  // test-and-append of the f unit rows of R64 (unit flags in unitf_), in order
  int sequential(int f) {
    flagged_ += f;
    const int wrows = (int)((ncap_ + 7) / 8);
    for (int i = 0; i < f; ++i) {
      const double* h = R64_ + (long long)i * ldp_;
      k_a2_beta<<<wrows, 256, 0, s_>>>(B64_, ldp_, ncur_, h, P_, vb_, rr2_);
      k_a2_x<<<wrows, 256, 0, s_>>>(Ainv_, (int)ncap_, ncur_, vb_, vx_);
      k_a2_resid<<<(P_ + 255) / 256, 256, 0, s_>>>(B64_, ldp_, ncur_, vx_, h, P_, rr2_);
      k_a2_append<<<152 * 4, 256, 0, s_>>>(B64_, ldp_, Ainv_, (int)ncap_, ncur_, (int)ncap_, vx_, h, P_, rr2_,
                                          unitf_ + i, tol_, accepted_, st_);
      k_a2_commit<<<1, 1, 0, s_>>>(ncur_, accepted_);
      A2_TRY(cudaGetLastError());
    }
    return read_state();
  }

  int block(long long t0, int kb) {
    const int N = (int)N_;
    A2_TRY(bracket_fp64(B64_, d_, ldp_, t0, nullptr, kb, H64_, ldp_, s_));
    A2_TRY(rownorm2_f64(kb, P_, H64_, ldp_, hn2_, s_));
    k_normalise_rows<<<kb, 256, 0, s_>>>(H64_, ldp_, kb, P_, hn2_, eta_ * eta_, unit_);
    A2_TRY(cudaGetLastError());
    A2_TRY(gemm_nt_f64(kb, N, P_, H64_, ldp_, B64_, ldp_, beta_, (int)ncap_, s_));        // beta = H B^T
    A2_TRY(gemm_nt_f64(kb, N, N, beta_, (int)ncap_, Ainv_, (int)ncap_, X_, (int)ncap_, s_));  // X = beta A^-1
    A2_TRY(cudaMemcpy2DAsync(R64_, sizeof(double) * ldp_, H64_, sizeof(double) * ldp_, sizeof(double) * P_, kb,
                             cudaMemcpyDeviceToDevice, s_));
    A2_TRY(gemm_nn_sub_f64(kb, P_, N, X_, (int)ncap_, B64_, ldp_, R64_, ldp_, s_));        // R = H - X B
    A2_TRY(rownorm2_f64(kb, P_, R64_, ldp_, rn2_, s_));
    const double tau = 0.5 * tol_;
    A2_TRY(screen_compact_f64(unit_, rn2_, kb, 0.5, tau * tau, 0.0, idx_, stats_, s_));
    A2_TRY(cudaMemcpyAsync(&host_->stats, stats_, sizeof(DevStats), cudaMemcpyDeviceToHost, s_));
    A2_TRY(cudaStreamSynchronize(s_));
    const int f = host_->stats.nflag;
    if (f == 0) return LC_OK;
    A2_TRY(gather_rows_f64(H64_, ldp_, idx_, f, P_, R64_, ldp_, s_));
    k_a2_rows_unit<<<(f + 255) / 256, 256, 0, s_>>>(unit_, idx_, f, unitf_);
    A2_TRY(cudaGetLastError());
    return sequential(f);
  }

  int sweep() {
    t_ = 0;
    long long dmax = -1;
    if (opt_.saturation_exit) {
      // brackets are traceless: the closure lies in su(d) plus the trace
      // directions of the generators (at most one)
      std::vector<double> diag((size_t)d_);
      bool trace = false;
      for (int q = 0; q < k_ && !trace; ++q) {
        if (cudaMemcpy2DAsync(diag.data(), sizeof(double), G64_ + (size_t)q * ldp_, sizeof(double) * (d_ + 1),
                              sizeof(double), (size_t)d_, cudaMemcpyDeviceToHost, s_) != cudaSuccess ||
            cudaStreamSynchronize(s_) != cudaSuccess)
          return LC_ERR_CUDA;
        double t = 0.0, a = 0.0;
        for (double v : diag) { t += v; a = std::max(a, std::fabs(v)); }
        if (std::fabs(t) > 1e-12 * std::max(1.0, a * d_)) trace = true;
      }
      dmax = (long long)d_ * d_ - 1 + (trace ? 1 : 0);
    }
    for (;;) {
      const long long T = pairs_below(N_);
      if (t_ >= T) break;
      if (dmax >= 0 && N_ >= dmax) break;
      long long kb = std::min<long long>(K_, T - t_);
      if (opt_.max_candidates > 0) kb = std::min<long long>(kb, opt_.max_candidates - checked_);
      if (kb <= 0) break;
      const int rc = block(t_, (int)kb);
      ++blocks_;
      t_ += kb;
      checked_ += kb;
      if (rc != LC_OK) return rc;
    }
    return LC_OK;
  }
};

}  // namespace

int closure_alg2_device(const double2* d_gens, int k, int d, double tol, double2* d_out, long long* dim_out,
                        long long max_dim, const lc_options& o, lc_report* rep, cudaStream_t s) {
  const long long ncap = std::min<long long>(max_dim, (long long)d * d);
  Closure2 c(k, d, tol, ncap, o, s);
  return c.run(d_gens, d_out, dim_out, rep);
}

}  // namespace lc
