// Host driver and C ABI of the Lie-closure library.
//
// This host code runs Algorithm 4 of arXiv 2506.01120 (Section 3.2) in candidate
// blocks.  The basis V lives on the device as packed FP64 rows (see
// lc_internal.cuh); a block is a contiguous run of the pair sweep
// (l, m), m < l, l ascending then m ascending, restricted to l < |V| at the
// start of the block.  Each block is screened in one pass (FP64, or split-BF16
// tensor-core GEMMs in mixed mode); screened-in candidates are recomputed in
// FP64, orthogonalised twice against V, and then tested and appended one by
// one in pair order against V plus this block's earlier accepts -- the same
// decisions the sequential algorithm takes, since a block's brackets involve
// only elements that existed before the block.
#include "lc_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

using namespace lc;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------------ memory pool
cudaError_t get_pool(cudaMemPool_t* out) {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
  if (!pools[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p;
    e = cudaMemPoolCreate(&p, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = ~0ull;   // keep freed blocks for the next call
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  *out = pools[dev];
  return cudaSuccess;
}

// One allocation carved into 256-byte aligned pieces.
struct Arena {
  char* base = nullptr;
  size_t off = 0, cap = 0;
  cudaStream_t s = nullptr;
  bool planning = true;
  template <typename T>
  T* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = planning ? nullptr : reinterpret_cast<T*>(base + off);
    off += n * sizeof(T) + 256;
    return p;
  }
  cudaError_t allocate(cudaStream_t st) {
    s = st;
    cap = off;
    cudaMemPool_t pool;
    cudaError_t e = get_pool(&pool);
    if (e != cudaSuccess) return e;
    e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&base), cap, pool, s);
    off = 0;
    planning = false;
    return e;
  }
  ~Arena() {
    if (base) cudaFreeAsync(base, s);
  }
};

#define LC_TRY(x)                                                  \
  do {                                                             \
    cudaError_t e_ = (x);                                          \
    if (e_ != cudaSuccess) {                                       \
      if (opt.verbose)                                             \
        fprintf(stderr, "lieclosure: %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? LC_ERR_OOM : LC_ERR_CUDA; \
    }                                                              \
  } while (0)

struct HostMirror {
  DevStats stats;
  DevStatus st;
  double maxdev, maxabs;
  int nonfinite;
  int nnz;
  unsigned long long scratch_bits;
};

// Autotuner cache: the screening-GEMM tile and saturated-phase block size
// chosen for (device, d, Algorithm 3 or 4).
struct TuneKey {
  int dev, d, alg3;
  bool operator<(const TuneKey& o) const {
    return dev != o.dev ? dev < o.dev : (d != o.d ? d < o.d : alg3 < o.alg3);
  }
};
struct TuneVal {
  int cfg, kb;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

class Closure {
 public:
  Closure(int k, int d, double tol, long long ncap, const lc_options& o, cudaStream_t s, bool alg3 = false)
      : k_(k), d_(d), tol_(tol), ncap_(ncap), opt(o), s_(s), alg3_(alg3) {
    P_ = d * d;
    mixed_ = (o.precision == LC_PREC_MIXED_BF16X3);
    // pad to the screening GEMM's N tile (it runs over both the basis and the
    // packed components as its N extent)
    ldp_ = round_up(P_, std::max(128, split_gemm_tile_n()));
    ncap_pad_ = (int)round_up_ll(ncap_, std::max(128, split_gemm_tile_n()));
    int K = o.block_k > 0 ? o.block_k : (mixed_ ? (o.autotune ? 32768 : 16384) : 2048);
    // bound the candidate buffers to about 8 GB
    const double per = mixed_ ? (8.0 * ldp_ + 4.0 * ldp_ + 4.0 * ncap_pad_ + 8.0 * ncap_)
                              : (24.0 * ldp_ + 8.0 * ncap_);
    const int kmem = (int)std::max(1.0, std::min(1.0e9, 8.0e9 / per));
    K = std::min(K, kmem);
    K = std::max(K, k_);         // the generator pass is one block
    K_ = std::max(1, K);
    Kpad_ = round_up(K_, 128);
    // growth blocks: 1024 candidates; 256 for large d (P >= 2^16), where each
    // flagged candidate costs an FP64 bracket of 8 d^3 flop and smaller blocks
    // flag fewer in-block duplicates
    Kgrow_ = std::min(K_, o.block_k_growth > 0 ? o.block_k_growth : (P_ >= (1 << 16) ? 256 : 1024));
    // saturated-phase block: the allocated K_, except that an autotuned call
    // without an explicit block_k starts from the fixed default
    Ksat_ = (o.autotune && o.block_k <= 0) ? std::min(K_, mixed_ ? 16384 : 2048) : K_;
    measured_tau_ = mixed_ && !(o.tau_screen > 0);
    tau_ = o.tau_screen > 0 ? o.tau_screen : kTauHi;
    kappa_ = o.screen_kappa > 0 ? o.screen_kappa : kKappa;
    // accept iff ||r||^2 > a ||h||^2 + b: relative (a, b) = (tol^2, 0), absolute (0, tol^2)
    tol_rel2_ = o.tol_mode == LC_TOL_ABSOLUTE ? 0.0 : tol * tol;
    tol_abs2_ = o.tol_mode == LC_TOL_ABSOLUTE ? tol * tol : 0.0;
    eta_ = o.eta_abs > 0 ? o.eta_abs : 1e-12;
    eta_screen_ = std::max(eta_, 1e-5);
    big_bracket_ = mixed_ && !bracket_tc_supported(d) && bracket_big_supported(d);
    tc_bracket_ = mixed_ && (bracket_tc_supported(d) || big_bracket_);
    q_bracket_ = mixed_ && d == 64;      // [Hr; Hi] operands instead of the 2d x 2d embedding
    // FP64-accurate tensor-core GEMMs for the accept step's projections in
    // mixed mode at d = 64 .. 128 (the V slices take 4 S P ncap bytes)
    if (mixed_ && o.accept_gemm == 0 && P_ >= 4096 && P_ <= 16384) {
      oz_beta_ = oz_beta_for((int)std::max<long long>(P_, ncap_));
      oz_S_ = oz_slices_for(oz_beta_);
      const double vbytes = 4.0 * oz_S_ * (double)ldp_ * (double)ncap_pad_;
      oz_on_ = vbytes <= 12.0e9;
    }
  }

  // Resume: d_gens holds n_resume orthonormal basis elements returned by an
  // earlier call; the generator pass is skipped and the sweep continues at the
  // pair index t_resume.
  long long n_resume_ = -1, t_resume_ = 0;
  void set_resume(long long n, long long t) {
    n_resume_ = n;
    t_resume_ = t;
  }

  int run(const double2* d_gens, double2* d_basis_out, long long* dim_out, lc_report* rep,
          double2* d_nested_out = nullptr) {
    const double t_start = now_s();
    t_last_accept_ = 0.0;
    int rc = setup(d_gens);
    if (rc == LC_OK) rc = (n_resume_ >= 0) ? resume_state() : generator_pass();
    if (rc == LC_OK) rc = sweep();
    if ((rc == LC_OK || rc == LC_ERR_CAPACITY) && opt.ortho_check) {
      const int rc2 = ortho_check();
      if (rc2 != LC_OK) rc = rc2;
    }
    if (rc == LC_OK || rc == LC_ERR_CAPACITY) {
      if (d_basis_out && N_ > 0) {
        cudaError_t e = unpack_basis(V64_, (int)N_, d_, ldp_, d_basis_out, s_);
        if (e != cudaSuccess) rc = LC_ERR_CUDA;
      }
      if (alg3_ && d_nested_out && N_ > 0) {
        cudaError_t e = unpack_basis(B64_, (int)N_, d_, ldp_, d_nested_out, s_);
        if (e != cudaSuccess) rc = LC_ERR_CUDA;
      }
    }
    cudaError_t e = cudaStreamSynchronize(s_);
    if (e != cudaSuccess && rc == LC_OK) rc = LC_ERR_CUDA;
    if (dim_out) *dim_out = N_;
    if (rep) {
      memset(rep, 0, sizeof(*rep));
      rep->dim = N_;
      rep->brackets_checked = checked_;
      rep->generators_checked = k_;
      rep->n_nonzero = nonzero_;
      rep->n_flagged = flagged_;
      rep->n_blocks = blocks_;
      int l = 1, m = 0;
      if (t_ > 0) pair_from_index(t_, &l, &m);
      rep->cursor_l = l;
      rep->cursor_m = m;
      rep->t_total_s = now_s() - t_start;
      rep->t_last_accept_s = t_last_accept_ > 0 ? t_last_accept_ - t_start : 0.0;
      double mn = 0.0, mx = 0.0;
      if (host_) {
        memcpy(&mn, &host_->stats.min_acc_bits, 8);
        memcpy(&mx, &host_->stats.max_rej_bits, 8);
      }
      rep->min_acc_rel_res = mn;
      rep->max_rej_rel_res = mx;
      double sr = 0.0, eps = 0.0, mas = 0.0;
      if (host_) {
        memcpy(&sr, &host_->stats.max_screen_rej_bits, 8);
        memcpy(&eps, &host_->stats.eps_bits, 8);
        memcpy(&mas, &host_->stats.min_acc_screen_bits, 8);
      }
      rep->tau_screen = mixed_ ? (measured_tau_ ? tau_max_used_ : tau_) : 0.5 * tol_;
      rep->max_screen_rej_rel_res = sr;
      rep->n_gray = gray_;
      rep->eps_screen = mixed_ ? eps : 0.0;
      rep->min_acc_screen_rel_res = mixed_ ? mas : 0.0;
      rep->ortho_defect = ortho_defect_;
      rep->ortho_rows = ortho_rows_;
      rep->block_k_used = Ksat_;
      rep->block_k_growth_used = Kgrow_;
      rep->gemm_tile_n = split_gemm_tile_n(gemm_cfg_);
      rep->gemm_tile_k = split_gemm_tile_k(gemm_cfg_);
      rep->autotuned = autotuned_ ? 1 : 0;
      rep->autotune_trials = trials_done_;
      rep->accept_wide_launches = wide_launches_;
      rep->screen_pass1_blocks = scr_pass1_blocks_;
      rep->accept_tc_gemms = oz_gemms_;
      rep->kernel_launches = launches_ + 1 + (N_ > 0 && d_basis_out ? 1 : 0);
      rep->gemm_launches = gemm_launches_;
      rep->gemm_flops = gemm_flops_;
      destroy_events();
      for (int i = 0; i < 6; ++i) rep->t_phase_s[i] = t_phase_[i];
      rep->precision = opt.precision;
      rep->status = rc;
    }
    return rc;
  }

  ~Closure() {
    destroy_events();
    if (host_) cudaFreeHost(host_);
  }

 private:
  int k_, d_, P_, ldp_, ncap_pad_, K_, Kpad_, Kgrow_, Ksat_;
  double tol_, tau_, eta_, eta_screen_;
  double tol_rel2_ = 0.0, tol_abs2_ = 0.0;
  // measured screen threshold (mixed mode, opt.tau_screen == 0)
  static constexpr double kTauHi = 1e-3;                // upper clamp (and the fixed default before any probe)
  static constexpr double kTauLo = 4.76837158203125e-7; // 2^-21, a few FP32 ulps
  static constexpr int kProbeRows = 128, kProbeSingles = 64;
  bool measured_tau_ = false;
  // tau_screen = kKappa * eps: candidates screened above it are rechecked in
  // FP64 (so a noise flag costs time, never a wrong decision), while a true
  // residual in (tol, tau] would be rejected by the screen.  The probe rows
  // carry no bracket rounding, so a bracket's screened noise runs above the
  // probe's eps: the largest screened residual among millions of dependent
  // brackets measured up to 2.2 eps (random d = 64 pair), and at 4 eps the
  // su(128) chain's noise flags tripled its run time.  10 eps keeps noise
  // flags rare.
  static constexpr double kKappa = 10.0;
  double kappa_ = kKappa, tau_max_used_ = 0.0;
  long long N_probe_ = 0, probes_ = 0, gray_ = 0;
  float* rho2f_ = nullptr;            // screened rho^2 of the flagged candidates, flag order
  int* cidx_ = nullptr;               // compacted (GEMM-row) positions of the flagged candidates
  // FP64-accurate tensor-core GEMMs of the accept step (digit slices): V's
  // rows and transposed rows, each row in units of its own exponent eV (the
  // coefficients of R -= c V carry 2^eV in their columns), flagged rows and
  // their coefficients in chunks of kOzRows with per-row exponents; slice
  // pairs up to level S (one past the slices' own resolution)
  static constexpr int kOzRows = 2048;
  static constexpr int kOzMinK = 64;   // contractions shorter than one k-box run on zero-padded slices
  static constexpr size_t kOzWs = size_t(8) << 20;   // split-K partials, doubles (64 MB)
  bool oz_on_ = false;
  int oz_beta_ = 0, oz_S_ = 0, oz_rows_ = 0;
  __nv_bfloat16 *Vs_ = nullptr, *VsT_ = nullptr, *Rs_ = nullptr, *Cs_ = nullptr;
  int *eR_ = nullptr, *eC_ = nullptr, *eV_ = nullptr;   // row exponents (eV_: V's rows)
  __nv_bfloat16* WsT_ = nullptr;      // transposed slices of one panel's accepted rows
  int oz_w0_ = -1, oz_nw_ = -1;
  double* oz_ws_ = nullptr;
  long long oz_gemms_ = 0;
  long long scr_pass1_blocks_ = 0;    // blocks whose first projection took the screening coefficients
  // orthonormality check
  double* G64_ = nullptr;
  unsigned long long* defect_bits_ = nullptr;
  double ortho_defect_ = -1.0;
  long long ortho_rows_ = 0;
  static constexpr int kOrthoSample = 4096, kOrthoChunk = 128;
  // screening GEMM tile and the autotuner
  int gemm_cfg_ = 0;
  bool autotuned_ = false;
  int trials_done_ = 0;
  long long ncap_;
  lc_options opt;
  cudaStream_t s_;
  bool mixed_;
  bool alg3_;            // Algorithm 3: brackets of B, B kept beside V
  double *B64_ = nullptr, *Hraw_ = nullptr, *bn2_ = nullptr;
  Arena ar_;
  // rows the brackets are formed from: V (Algorithm 4) or B (Algorithm 3)
  const double* src() const { return alg3_ ? B64_ : V64_; }
  HostMirror* host_ = nullptr;
  long long N_ = 0, t_ = 0, checked_ = 0, nonzero_ = 0, flagged_ = 0, blocks_ = 0;
  double t_last_accept_ = 0.0;
  // device buffers
  double *Gen64_ = nullptr, *V64_ = nullptr, *H64_ = nullptr, *S64_ = nullptr, *R64_ = nullptr, *beta64_ = nullptr;
  double *hn2_ = nullptr, *rn2_ = nullptr, *hnf_ = nullptr, *rnf_ = nullptr, *chk_ = nullptr, *hn2c64_ = nullptr;
  int *idx_ = nullptr, *nonfinite_ = nullptr, *need_ = nullptr;
  unsigned int* bar_ = nullptr;
  double* wpart_ = nullptr;         // per-CTA partial sums of the row-sliced accept
  long long wide_launches_ = 0;
  double* ws64_ = nullptr;
  static constexpr size_t kWs64 = size_t(2) << 20;   // split-K workspace, doubles
  static constexpr int kPanel = kAcceptWideMaxRows;   // rows per in-block accept panel
  static constexpr float kScrPass1MaxRho2 = 0.5f;     // a second pass is needed below this
  static constexpr float kScrPass1MinRho2 = 1e-6f;    // screening coefficients too coarse below this
  static constexpr size_t kWsK = size_t(8) << 20;    // split-K partials of the projection, floats (32 MB)
  float* wsk_ = nullptr;
  int* part_ = nullptr;             // per-chunk counts of the multi-CTA compactions
  DevStats* stats_ = nullptr;
  DevStatus* st_ = nullptr;
  __nv_bfloat16 *Vhi_ = nullptr, *Vlo_ = nullptr, *VThi_ = nullptr, *VTlo_ = nullptr;
  __nv_bfloat16 *Hhi_ = nullptr, *Hlo_ = nullptr, *Bhi_ = nullptr, *Blo_ = nullptr;
  __nv_bfloat16 *Chi_ = nullptr, *Clo_ = nullptr, *Ehi_ = nullptr, *Elo_ = nullptr;
  float *hn2f_ = nullptr, *rn2f_ = nullptr, *hn2c_ = nullptr;
  int *nz_idx_ = nullptr, *nnz_ = nullptr;
  bool tc_bracket_ = false, big_bracket_ = false, q_bracket_ = false;

  void carve() {
    if (opt.ortho_check) {
      G64_ = ar_.take<double>((size_t)kOrthoChunk * kOrthoSample);
      defect_bits_ = ar_.take<unsigned long long>(1);
    }
    Gen64_ = ar_.take<double>((size_t)k_ * ldp_);
    V64_ = ar_.take<double>((size_t)ncap_ * ldp_);
    R64_ = ar_.take<double>((size_t)K_ * ldp_);
    beta64_ = ar_.take<double>((size_t)K_ * ncap_);
    hnf_ = ar_.take<double>(K_);
    rnf_ = ar_.take<double>(K_);
    idx_ = ar_.take<int>(K_);
    stats_ = ar_.take<DevStats>(1);
    st_ = ar_.take<DevStatus>(1);
    chk_ = ar_.take<double>(2);
    nonfinite_ = ar_.take<int>(1);
    need_ = ar_.take<int>(1);
    bar_ = ar_.take<unsigned int>(2);
    wpart_ = ar_.take<double>(accept_wide_part_doubles());
    ws64_ = ar_.take<double>(kWs64);
    part_ = ar_.take<int>(3 * kCmpCtas);
    if (alg3_) {
      B64_ = ar_.take<double>((size_t)ncap_ * ldp_);
      Hraw_ = ar_.take<double>((size_t)K_ * ldp_);
      bn2_ = ar_.take<double>(ncap_);
    }
    if (!mixed_) {
      H64_ = ar_.take<double>((size_t)K_ * ldp_);
      S64_ = ar_.take<double>((size_t)K_ * ldp_);
      hn2_ = ar_.take<double>(K_);
      rn2_ = ar_.take<double>(K_);
      hn2c64_ = ar_.take<double>(K_);
      nz_idx_ = ar_.take<int>(K_);
      nnz_ = ar_.take<int>(1);
    } else {
      Vhi_ = ar_.take<__nv_bfloat16>((size_t)ncap_pad_ * ldp_);
      Vlo_ = ar_.take<__nv_bfloat16>((size_t)ncap_pad_ * ldp_);
      VThi_ = ar_.take<__nv_bfloat16>((size_t)ldp_ * ncap_pad_);
      VTlo_ = ar_.take<__nv_bfloat16>((size_t)ldp_ * ncap_pad_);
      Hhi_ = ar_.take<__nv_bfloat16>((size_t)Kpad_ * ldp_);
      Hlo_ = ar_.take<__nv_bfloat16>((size_t)Kpad_ * ldp_);
      Bhi_ = ar_.take<__nv_bfloat16>((size_t)Kpad_ * ncap_pad_);
      Blo_ = ar_.take<__nv_bfloat16>((size_t)Kpad_ * ncap_pad_);
      hn2f_ = ar_.take<float>(Kpad_);
      rn2f_ = ar_.take<float>(Kpad_);
      Chi_ = ar_.take<__nv_bfloat16>((size_t)Kpad_ * ldp_);
      Clo_ = ar_.take<__nv_bfloat16>((size_t)Kpad_ * ldp_);
      hn2c_ = ar_.take<float>(Kpad_);
      rho2f_ = ar_.take<float>(Kpad_);
      cidx_ = ar_.take<int>(Kpad_);
      if (oz_on_) {
        Vs_ = ar_.take<__nv_bfloat16>((size_t)oz_S_ * ncap_pad_ * ldp_);
        VsT_ = ar_.take<__nv_bfloat16>((size_t)oz_S_ * ldp_ * ncap_pad_);
        Rs_ = ar_.take<__nv_bfloat16>((size_t)oz_S_ * kOzRows * ldp_);
        Cs_ = ar_.take<__nv_bfloat16>((size_t)oz_S_ * kOzRows * ncap_pad_);
        WsT_ = ar_.take<__nv_bfloat16>((size_t)oz_S_ * ldp_ * kPanel);
        eR_ = ar_.take<int>(kOzRows);
        eV_ = ar_.take<int>(ncap_pad_);
        eC_ = ar_.take<int>(kOzRows);
        oz_ws_ = ar_.take<double>(kOzWs);
      }
      wsk_ = ar_.take<float>(kWsK);
      nz_idx_ = ar_.take<int>(Kpad_);
      nnz_ = ar_.take<int>(1);
      if (tc_bracket_) {
        const size_t R = 2 * (size_t)d_;
        const size_t per = q_bracket_ ? R * d_ : R * R;
        Ehi_ = ar_.take<__nv_bfloat16>((size_t)ncap_ * per);
        Elo_ = ar_.take<__nv_bfloat16>((size_t)ncap_ * per);
      }
    }
  }

  int sync_read() {
    cudaError_t e = cudaMemcpyAsync(&host_->stats, stats_, sizeof(DevStats), cudaMemcpyDeviceToHost, s_);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_->st, st_, sizeof(DevStatus), cudaMemcpyDeviceToHost, s_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s_);
    if (e != cudaSuccess) return LC_ERR_CUDA;
    collect_phases();
    if (host_->st.code != 0) {
      if (opt.verbose)
        fprintf(stderr, "lieclosure: device status %d at site %d (info %lld)\n", host_->st.code, host_->st.where,
                host_->st.info);
      return host_->st.code;
    }
    return LC_OK;
  }

  int setup(const double2* d_gens) {
    carve();
    LC_TRY(cudaHostAlloc(reinterpret_cast<void**>(&host_), sizeof(HostMirror), cudaHostAllocDefault));
    LC_TRY(ar_.allocate(s_));
    carve();
    if (mixed_) {
      if (!tcgen05_available()) return LC_ERR_CUDA;
      // zero padding rows/columns once; kernels only ever write live regions
      LC_TRY(cudaMemsetAsync(Vhi_, 0, sizeof(__nv_bfloat16) * (size_t)ncap_pad_ * ldp_, s_));
      LC_TRY(cudaMemsetAsync(Vlo_, 0, sizeof(__nv_bfloat16) * (size_t)ncap_pad_ * ldp_, s_));
      LC_TRY(cudaMemsetAsync(VThi_, 0, sizeof(__nv_bfloat16) * (size_t)ldp_ * ncap_pad_, s_));
      LC_TRY(cudaMemsetAsync(VTlo_, 0, sizeof(__nv_bfloat16) * (size_t)ldp_ * ncap_pad_, s_));
      LC_TRY(cudaMemsetAsync(Hhi_, 0, sizeof(__nv_bfloat16) * (size_t)Kpad_ * ldp_, s_));
      LC_TRY(cudaMemsetAsync(Hlo_, 0, sizeof(__nv_bfloat16) * (size_t)Kpad_ * ldp_, s_));
      LC_TRY(cudaMemsetAsync(Bhi_, 0, sizeof(__nv_bfloat16) * (size_t)Kpad_ * ncap_pad_, s_));
      LC_TRY(cudaMemsetAsync(Blo_, 0, sizeof(__nv_bfloat16) * (size_t)Kpad_ * ncap_pad_, s_));
      LC_TRY(cudaMemsetAsync(Chi_, 0, sizeof(__nv_bfloat16) * (size_t)Kpad_ * ldp_, s_));
      LC_TRY(cudaMemsetAsync(Clo_, 0, sizeof(__nv_bfloat16) * (size_t)Kpad_ * ldp_, s_));
      // columns of V's transposed slices past the rows sliced so far stay zero digits
      if (oz_on_) LC_TRY(cudaMemsetAsync(VsT_, 0, sizeof(__nv_bfloat16) * (size_t)oz_S_ * ldp_ * ncap_pad_, s_));
    }
    if (ldp_ > P_) {
      // padding columns of the FP64 rows stay zero
      LC_TRY(cudaMemset2DAsync(V64_ + P_, sizeof(double) * ldp_, 0, sizeof(double) * (ldp_ - P_), ncap_, s_));
      if (alg3_)
        LC_TRY(cudaMemset2DAsync(B64_ + P_, sizeof(double) * ldp_, 0, sizeof(double) * (ldp_ - P_), ncap_, s_));
    }
    LC_TRY(cudaMemsetAsync(st_, 0, sizeof(DevStatus), s_));
    LC_TRY(cudaMemsetAsync(bar_, 0, 2 * sizeof(unsigned int), s_));
    LC_TRY(cudaMemsetAsync(stats_, 0, sizeof(DevStats), s_));
    {
      // min_acc starts at +inf
      DevStats init;
      memset(&init, 0, sizeof(init));
      double inf = INFINITY;
      memcpy(&init.min_acc_bits, &inf, 8);
      memcpy(&init.min_acc_screen_bits, &inf, 8);
      init.tau2 = (float)(tau_ * tau_);
      init.eps2 = 0.f;
      host_->stats = init;
      LC_TRY(cudaMemcpyAsync(stats_, &host_->stats, sizeof(DevStats), cudaMemcpyHostToDevice, s_));
    }
    LC_TRY(cudaMemsetAsync(chk_, 0, 2 * sizeof(double), s_));
    LC_TRY(cudaMemsetAsync(nonfinite_, 0, sizeof(int), s_));
    LC_TRY(pack_generators(d_gens, k_, d_, ldp_, Gen64_, chk_, chk_ + 1, nonfinite_, s_));
    LC_TRY(cudaMemcpyAsync(&host_->maxdev, chk_, 2 * sizeof(double), cudaMemcpyDeviceToHost, s_));
    LC_TRY(cudaMemcpyAsync(&host_->nonfinite, nonfinite_, sizeof(int), cudaMemcpyDeviceToHost, s_));
    LC_TRY(cudaStreamSynchronize(s_));
    if (host_->nonfinite) return LC_ERR_NONFINITE;
    if (host_->maxdev > 1e-12 * host_->maxabs) return LC_ERR_NOT_ANTIHERMITIAN;
    if (opt.saturation_exit) {
      // largest possible dimension: d^2 - 1, plus the trace direction
      std::vector<double> diag((size_t)k_ * d_);
      LC_TRY(cudaMemcpy2DAsync(diag.data(), sizeof(double), Gen64_, sizeof(double) * (d_ + 1), sizeof(double),
                               (size_t)d_, cudaMemcpyDeviceToHost, s_));
      // the 2-D copy above walks one generator's diagonal; repeat per generator
      for (int q = 1; q < k_; ++q)
        LC_TRY(cudaMemcpy2DAsync(diag.data() + (size_t)q * d_, sizeof(double), Gen64_ + (size_t)q * ldp_,
                                 sizeof(double) * (d_ + 1), sizeof(double), (size_t)d_, cudaMemcpyDeviceToHost,
                                 s_));
      LC_TRY(cudaStreamSynchronize(s_));
      bool trace = false;
      for (int q = 0; q < k_; ++q) {
        double t = 0.0, a = 0.0;
        for (int j = 0; j < d_; ++j) {
          t += diag[(size_t)q * d_ + j];
          a = std::max(a, std::fabs(diag[(size_t)q * d_ + j]));
        }
        if (std::fabs(t) > 1e-12 * std::max(1.0, a * d_)) trace = true;
      }
      dmax_ = (long long)d_ * d_ - 1 + (trace ? 1 : 0);
    }
    return LC_OK;
  }

  long long dmax_ = -1;

  // ---------------------------------------------------- phase timing
  // With opt.profile each phase is bracketed by CUDA events on the call's
  // stream; elapsed times are collected after the next synchronisation.
  enum { PH_BRACKET = 0, PH_GEMM1 = 1, PH_GEMM2 = 2, PH_SCREEN = 3, PH_ACCEPT = 4, PH_OTHER = 5 };
  struct Pending { int phase; cudaEvent_t a, b; };
  std::vector<cudaEvent_t> ev_pool_;
  std::vector<Pending> pending_;
  double t_phase_[6] = {0, 0, 0, 0, 0, 0};
  long long launches_ = 0, gemm_launches_ = 0;
  double gemm_flops_ = 0.0;
  cudaEvent_t ev_open_ = nullptr;

  cudaEvent_t get_ev() {
    if (!ev_pool_.empty()) {
      cudaEvent_t e = ev_pool_.back();
      ev_pool_.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void ph_begin() {
    if (!opt.profile) return;
    ev_open_ = get_ev();
    cudaEventRecord(ev_open_, s_);
  }
  void ph_end(int phase) {
    if (!opt.profile) return;
    cudaEvent_t b = get_ev();
    cudaEventRecord(b, s_);
    pending_.push_back({phase, ev_open_, b});
  }
  void collect_phases() {
    for (auto& p : pending_) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) t_phase_[p.phase] += ms * 1e-3;
      ev_pool_.push_back(p.a);
      ev_pool_.push_back(p.b);
    }
    pending_.clear();
  }
  void destroy_events() {
    collect_phases();
    for (auto e : ev_pool_) cudaEventDestroy(e);
    ev_pool_.clear();
  }

  // V rows [oz_rows_, n0) into both slice layouts (rows are final once appended)
  cudaError_t oz_sync_v(int n0) {
    if (n0 <= oz_rows_) return cudaSuccess;
    cudaError_t e = oz_slice_rows(V64_ + (size_t)oz_rows_ * ldp_, n0 - oz_rows_, P_, ldp_, oz_S_, oz_beta_, 0, Vs_,
                                  ncap_pad_, ldp_, eV_, oz_rows_, nullptr, s_);
    if (e == cudaSuccess)
      e = oz_slice_cols(V64_, oz_rows_, n0, P_, ldp_, oz_S_, oz_beta_, eV_, VsT_, ldp_, ncap_pad_, s_);
    launches_ += 2;
    oz_rows_ = n0;
    return e;
  }
  // the tensor-core form where the FP64 product is long enough to pay for
  // the slicing and the launches (about 2^24 multiply-adds and up)
  bool oz_use(int f, int n0) const { return oz_on_ && n0 >= 1 && (double)f * n0 * P_ >= 16777216.0; }

  // W^T slices of V rows [w0, w0 + nw) (nw <= kPanel) for the panel projections
  cudaError_t oz_sync_w(int w0, int nw) {
    if (w0 == oz_w0_ && nw == oz_nw_) return cudaSuccess;
    oz_w0_ = w0;
    oz_nw_ = nw;
    launches_ += 1;
    if (nw < kOzMinK) {   // the columns a short contraction pads to must be zero digits
      const cudaError_t e = cudaMemsetAsync(WsT_, 0, sizeof(__nv_bfloat16) * (size_t)oz_S_ * ldp_ * kPanel, s_);
      if (e != cudaSuccess) return e;
    }
    return oz_slice_cols(V64_, w0, w0 + nw, P_, ldp_, oz_S_, oz_beta_, eV_, WsT_, ldp_, kPanel, s_, w0);
  }

  // beta64 rows [0, f) (row stride ncap) = rows [0, f) of R (from Rb) times
  // V rows [w0, w0 + nw)^T
  cudaError_t proj_coef(double* Rb, int f, int w0, int nw, const int* run_if = nullptr) {
    if (!oz_use(f, nw)) {
      launches_ += 1;
      return gemm_nt_f64(f, nw, P_, Rb, ldp_, V64_ + (size_t)w0 * ldp_, ldp_, beta64_, (int)ncap_, s_, ws64_,
                         kWs64, run_if);
    }
    cudaError_t e = oz_sync_v(w0 + nw);
    const long long vtot = (long long)oz_S_ * ncap_pad_ - w0;    // rows from the offset base to the stack's end
    for (int r0 = 0; r0 < f && e == cudaSuccess; r0 += kOzRows) {
      const int c = std::min(kOzRows, f - r0);
      e = oz_slice_rows(Rb + (size_t)r0 * ldp_, c, P_, ldp_, oz_S_, oz_beta_, 0, Rs_, kOzRows, ldp_, eR_, 0, run_if,
                        s_);
      launches_ += 1;
      if (e != cudaSuccess) break;
      const OzOperand A{Rs_, kOzRows, ldp_, eR_, 0}, B{Vs_ + (size_t)w0 * ldp_, ncap_pad_, ldp_, eV_ + w0, 0, vtot};
      e = ozaki_gemm_nt(c, nw, P_, A, B, oz_S_, oz_beta_, beta64_ + (size_t)r0 * ncap_, (int)ncap_, false, oz_ws_,
                        kOzWs, run_if, opt.spin_cap, st_, s_, &launches_, oz_S_);
      oz_gemms_ += 1;
    }
    return e;
  }
  // rows [0, f) of R (from Rb) -= beta64 rows [0, f) times V rows [w0, w0 + nw)
  cudaError_t proj_sub(double* Rb, int f, int w0, int nw, const int* run_if = nullptr) {
    if (!oz_use(f, nw) || (w0 > 0 && nw > kPanel)) {
      launches_ += 1;
      return gemm_nn_sub_f64(f, P_, nw, beta64_, (int)ncap_, V64_ + (size_t)w0 * ldp_, ldp_, Rb, ldp_, s_, ws64_,
                             kWs64, run_if);
    }
    cudaError_t e = w0 == 0 ? oz_sync_v(nw) : oz_sync_w(w0, nw);
    for (int r0 = 0; r0 < f && e == cudaSuccess; r0 += kOzRows) {
      const int c = std::min(kOzRows, f - r0);
      const int kg = std::max(nw, kOzMinK);   // zero digits beyond nw on both sides
      // coefficient column j carries V row (w0 + j)'s scale 2^eV, the
      // transposed slices hold V in units of it
      e = oz_slice_rows(beta64_ + (size_t)r0 * ncap_, c, nw, (int)ncap_, oz_S_, oz_beta_, 0, Cs_, kOzRows,
                        ncap_pad_, eC_, 0, run_if, s_, kg, eV_ + w0);
      launches_ += 1;
      if (e != cudaSuccess) break;
      const OzOperand A{Cs_, kOzRows, ncap_pad_, eC_, 0};
      const OzOperand B = w0 == 0 ? OzOperand{VsT_, ldp_, ncap_pad_, nullptr, 0}
                                  : OzOperand{WsT_, ldp_, kPanel, nullptr, 0};
      e = ozaki_gemm_nt(c, P_, kg, A, B, oz_S_, oz_beta_, Rb + (size_t)r0 * ldp_, ldp_, true, oz_ws_, kOzWs, run_if,
                        opt.spin_cap, st_, s_, &launches_, oz_S_);
      oz_gemms_ += 1;
    }
    return e;
  }

  // Test-and-append of the f candidate rows in R64 (FP64, pair order):
  // classical Gram-Schmidt against the basis as it was when the block
  // started (a second pass only when some row needs it), then the in-order
  // test and append against that basis plus this block's accepts.
  int accept_rows(int f, const float* rho2_screen = nullptr, bool scr_coef = false) {
    flagged_ += f;
    ph_begin();
    if (alg3_)   // the raw bracket (or generator) is what Algorithm 3 appends to B
      LC_TRY(cudaMemcpy2DAsync(Hraw_, sizeof(double) * ldp_, R64_, sizeof(double) * ldp_, sizeof(double) * P_, f,
                               cudaMemcpyDeviceToDevice, s_));
    LC_TRY(rownorm2_f64(f, P_, R64_, ldp_, hnf_, s_));
    const int n0 = (int)N_;
    if (n0 > 0 && scr_coef) {
      // pass 1: h - V c with c the screening GEMM's coefficients (error of
      // order 1e-5 ||h||, in span(V)); pass 2 in FP64 removes what is left
      LC_TRY(gather_coef(Bhi_, Blo_, ncap_pad_, cidx_, f, n0, beta64_, (int)ncap_, s_));
      LC_TRY(proj_sub(R64_, f, 0, n0));
      LC_TRY(proj_coef(R64_, f, 0, n0));
      LC_TRY(proj_sub(R64_, f, 0, n0));
      LC_TRY(rownorm2_f64(f, P_, R64_, ldp_, rnf_, s_));
      launches_ += 2;
      scr_pass1_blocks_ += 1;
    } else if (n0 > 0) {
      LC_TRY(proj_coef(R64_, f, 0, n0));
      LC_TRY(proj_sub(R64_, f, 0, n0));
      LC_TRY(rownorm2_f64(f, P_, R64_, ldp_, rnf_, s_));
      LC_TRY(need_pass2(f, hnf_, rnf_, eta_ * eta_, tol_rel2_, tol_abs2_, need_, s_));
      LC_TRY(proj_coef(R64_, f, 0, n0, need_));
      LC_TRY(proj_sub(R64_, f, 0, n0, need_));
      LC_TRY(rownorm2_f64(f, P_, R64_, ldp_, rnf_, s_, need_));
      launches_ += 4;
    } else {
      LC_TRY(rownorm2_f64(f, P_, R64_, ldp_, rnf_, s_));
    }
    LC_TRY(zero_stats(stats_, n0, s_));
    launches_ += 1;
    // In-block test and append in panels of kPanel rows: the sequential
    // kernel decides a panel's rows in order (each accept projected out of
    // the panel's later rows), then the panel's accepted elements W are
    // projected out of all later rows at once, twice, by FP64 GEMMs.  The
    // rows' order of decision and their projections are those of the
    // sequential test; only the grouping of the later rows' projections
    // changes (one GEMM per panel instead of one rank-1 update per accept).
    long long nb = n0;
    int rc = LC_OK;
    for (int s0 = 0; s0 < f; s0 += kPanel) {
      const int e0 = std::min(f, s0 + kPanel);
      const size_t off = (size_t)s0 * ldp_;
      const int kern = accept_kernel_for(e0 - s0, P_, opt.accept_kernel);
      LC_TRY(accept_seq(e0 - s0, R64_ + off, ldp_, rnf_ + s0, hnf_ + s0, tol_rel2_, tol_abs2_, eta_ * eta_, V64_,
                        ldp_, (int)ncap_, P_, stats_, st_, bar_, opt.spin_cap, s_,
                        (s0 == 0 && opt.fault_inject) ? 1 : 0, alg3_ ? Hraw_ + off : nullptr,
                        alg3_ ? B64_ : nullptr, alg3_ ? bn2_ : nullptr, rho2_screen ? rho2_screen + s0 : nullptr,
                        kern, wpart_));
      launches_ += 1;
      if (kern == 2) wide_launches_ += 1;
      if (e0 >= f) break;
      rc = sync_read();
      if (rc != LC_OK) break;
      const long long na = host_->stats.ncur;
      const int a = (int)(na - nb);
      if (a > 0) {
        const int rest = f - e0;
        double* Rr = R64_ + (size_t)e0 * ldp_;
        for (int pass = 0; pass < 2; ++pass) {
          LC_TRY(proj_coef(Rr, rest, (int)nb, a));
          LC_TRY(proj_sub(Rr, rest, (int)nb, a));
        }
        LC_TRY(rownorm2_f64(rest, P_, Rr, ldp_, rnf_ + e0, s_));
        launches_ += 1;
      }
      nb = na;
    }
    ph_end(PH_ACCEPT);
    if (rc == LC_OK) rc = sync_read();
    const long long n1 = host_->stats.ncur;
    if (n1 > N_) t_last_accept_ = now_s();
    if (mixed_ && n1 > n0) {
      ph_begin();
      LC_TRY(split_rows(V64_, ldp_, n0, (int)n1, P_, Vhi_, Vlo_, ldp_, VThi_, VTlo_, ncap_pad_, s_));
      launches_ += 1;
      if (tc_bracket_) {
        if (q_bracket_) LC_TRY(build_q(src(), ldp_, n0, (int)n1, d_, Ehi_, Elo_, s_));
        else LC_TRY(build_embedding(src(), ldp_, n0, (int)n1, d_, Ehi_, Elo_, s_, big_bracket_ ? 1 : 0));
        launches_ += 1;
      }
      ph_end(PH_OTHER);
    }
    N_ = n1;
    return rc;
  }

  int resume_state() {
    if (n_resume_ > ncap_) return LC_ERR_CAPACITY;
    // the packed elements are already the basis rows
    LC_TRY(cudaMemcpy2DAsync(V64_, sizeof(double) * ldp_, Gen64_, sizeof(double) * ldp_, sizeof(double) * P_,
                             (size_t)n_resume_, cudaMemcpyDeviceToDevice, s_));
    if (mixed_ && n_resume_ > 0) {
      LC_TRY(split_rows(V64_, ldp_, 0, (int)n_resume_, P_, Vhi_, Vlo_, ldp_, VThi_, VTlo_, ncap_pad_, s_));
      if (q_bracket_) LC_TRY(build_q(src(), ldp_, 0, (int)n_resume_, d_, Ehi_, Elo_, s_));
      else if (tc_bracket_)
        LC_TRY(build_embedding(src(), ldp_, 0, (int)n_resume_, d_, Ehi_, Elo_, s_, big_bracket_ ? 1 : 0));
      launches_ += 2;
    }
    N_ = n_resume_;
    return LC_OK;
  }

  int generator_pass() {
    LC_TRY(cudaMemcpy2DAsync(R64_, sizeof(double) * ldp_, Gen64_, sizeof(double) * ldp_, sizeof(double) * P_, k_,
                             cudaMemcpyDeviceToDevice, s_));
    return accept_rows(k_);
  }

  int after_screen(long long t0) {
    int rc = sync_read();
    if (rc != LC_OK) return rc;
    nonzero_ += host_->stats.nnonzero;
    if (mixed_) {
      gemm_flops_ += 2.0 * 6.0 * (double)host_->stats.nnonzero * (double)N_ * (double)P_;
      gray_ += host_->stats.ngray;
      // (the device clamps in single precision: report the clamped double value)
      if (measured_tau_)
        tau_max_used_ = std::max(tau_max_used_, std::min(kTauHi, std::max(kTauLo, std::sqrt((double)host_->stats.tau2))));
    }
    const int f = host_->stats.nflag;
    if (f > 0) {
      if (mixed_) {
        ph_begin();
        LC_TRY(bracket_fp64(src(), d_, ldp_, t0, idx_, f, R64_, ldp_, s_));
        ph_end(PH_ACCEPT);
      } else {
        LC_TRY(gather_rows_f64(H64_, ldp_, idx_, f, P_, R64_, ldp_, s_));
      }
      launches_ += 1;
      // First projection from the screening coefficients when some flagged
      // row needs a second pass anyway (screened rho^2 < 1/2) and none has a
      // residual small enough (rho^2 < 1e-6) for the coefficients' BF16-level
      // error to dominate it.
      bool scr = false;
      if (mixed_ && !opt.fp64_first_pass && N_ > 0) {
        float m;
        const unsigned int b = host_->stats.min_rho2_flag_bits;
        memcpy(&m, &b, sizeof(m));
        scr = m < kScrPass1MaxRho2 && m >= kScrPass1MinRho2;
      }
      return accept_rows(f, mixed_ ? rho2f_ : nullptr, scr);
    }
    return LC_OK;
  }

  int block_fp64(long long t0, int kb) {
    ph_begin();
    LC_TRY(bracket_fp64(src(), d_, ldp_, t0, nullptr, kb, H64_, ldp_, s_));
    ph_end(PH_BRACKET);
    // zero brackets (commuting pairs) are rejected without a projection; the
    // rest are packed into consecutive rows of S64
    ph_begin();
    LC_TRY(rownorm2_f64(kb, P_, H64_, ldp_, hn2_, s_));
    LC_TRY(compact_nonzero_f64(hn2_, kb, eta_ * eta_, nz_idx_, nnz_, hn2c64_, s_, part_));
    LC_TRY(cudaMemcpyAsync(&host_->nnz, nnz_, sizeof(int), cudaMemcpyDeviceToHost, s_));
    LC_TRY(cudaStreamSynchronize(s_));
    const int nnz = host_->nnz;
    if (nnz > 0) LC_TRY(gather_rows_f64(H64_, ldp_, nz_idx_, nnz, P_, S64_, ldp_, s_));
    ph_end(PH_SCREEN);
    launches_ += 5;
    if (nnz == 0) {
      nonzero_ += 0;
      return LC_OK;
    }
    ph_begin();
    LC_TRY(gemm_nt_f64(nnz, (int)N_, P_, S64_, ldp_, V64_, ldp_, beta64_, (int)ncap_, s_, ws64_, kWs64));
    ph_end(PH_GEMM1);
    ph_begin();
    LC_TRY(gemm_nn_sub_f64(nnz, P_, (int)N_, beta64_, (int)ncap_, V64_, ldp_, S64_, ldp_, s_, ws64_, kWs64));
    LC_TRY(rownorm2_f64(nnz, P_, S64_, ldp_, rn2_, s_));
    ph_end(PH_GEMM2);
    // one FP64 projection pass: ||r1|| at most half the accept threshold
    // implies the two-pass residual is below it as well, so such candidates
    // are dependent
    ph_begin();
    LC_TRY(screen_compact_f64(hn2c64_, rn2_, nnz, eta_ * eta_, 0.25 * tol_rel2_, 0.25 * tol_abs2_, idx_, stats_, s_,
                              nullptr, nz_idx_, part_));
    ph_end(PH_SCREEN);
    launches_ += 5;
    return after_screen(t0);
  }

  // Screen noise probe (measured tau_screen): rows in span(V) through the
  // same split and GEMMs as a block's candidates; their screened residual is
  // pure noise.  Re-run whenever |V| has grown by 1/8 since the last probe.
  int maybe_probe() {
    if (!measured_tau_ || N_ <= 0) return LC_OK;
    if (N_probe_ > 0 && 8 * N_ < 9 * N_probe_) return LC_OK;
    N_probe_ = N_;
    const int S = kProbeRows;
    ph_begin();
    LC_TRY(probe_rows(V64_, ldp_, (int)N_, P_, S, kProbeSingles, 0x2506011200000000ull + (unsigned long long)probes_,
                      Chi_, Clo_, ldp_, hn2c_, nnz_, s_));
    ph_end(PH_SCREEN);
    LC_TRY(screen_gemms(S));
    gemm_flops_ += 2.0 * 6.0 * (double)S * (double)N_ * (double)P_;
    ph_begin();
    LC_TRY(probe_eps(hn2c_, rn2f_, S, stats_, (float)kappa_, (float)kTauLo, (float)kTauHi, s_));
    ph_end(PH_SCREEN);
    ++probes_;
    launches_ += 2;     // probe rows and eps; the GEMMs count themselves
    return LC_OK;
  }

  // max |<v_i, v_j> - delta_ij| in FP64 over every q-th row of V (all rows
  // when |V| <= kOrthoSample), in chunks of kOrthoChunk Gram rows.
  int ortho_check() {
    ortho_defect_ = -1.0;
    ortho_rows_ = 0;
    if (N_ <= 0 || !G64_) return LC_OK;
    const long long q = (N_ + kOrthoSample - 1) / kOrthoSample;
    const int S = (int)((N_ + q - 1) / q);
    const int ld = (int)(q * ldp_);
    LC_TRY(cudaMemsetAsync(defect_bits_, 0, sizeof(unsigned long long), s_));
    for (int c0 = 0; c0 < S; c0 += kOrthoChunk) {
      const int rows = std::min(kOrthoChunk, S - c0);
      LC_TRY(gemm_nt_f64(rows, S, P_, V64_ + (size_t)c0 * ld, ld, V64_, ld, G64_, S, s_, ws64_, kWs64));
      LC_TRY(defect_max(G64_, rows, S, S, c0, defect_bits_, s_));
      launches_ += 3;
    }
    unsigned long long bits = 0;
    LC_TRY(cudaMemcpyAsync(&host_->scratch_bits, defect_bits_, sizeof(bits), cudaMemcpyDeviceToHost, s_));
    LC_TRY(cudaStreamSynchronize(s_));
    bits = host_->scratch_bits;
    memcpy(&ortho_defect_, &bits, 8);
    ortho_rows_ = S;
    return LC_OK;
  }

  // projection beta = C V^T (split BF16 out) and residual ||C - beta V||^2 of
  // the first *nnz_ rows of C (M rows allocated)
  cudaError_t screen_gemms(int M_rows) {
    const int M = round_up(M_rows, 128);
    const int Npad = round_up((int)N_, std::max(128, split_gemm_tile_n()));
    SplitGemmArgs g1;
    memset(&g1, 0, sizeof(g1));
    g1.Ahi = Chi_;
    g1.Alo = Clo_;
    g1.Bhi = Vhi_;
    g1.Blo = Vlo_;
    g1.M = M;
    g1.Mdev = nnz_;
    g1.N = Npad;
    g1.K = ldp_;
    g1.lda = ldp_;
    g1.ldb = ldp_;
    g1.Dhi = Bhi_;
    g1.Dlo = Blo_;
    g1.ldd = ncap_pad_;
    g1.epilogue = 0;
    g1.spin_cap = opt.spin_cap;
    g1.st = st_;
    g1.cfg = gemm_cfg_;
    g1.ws = wsk_;
    g1.ws_floats = kWsK;
    g1.launches = &launches_;
    ph_begin();
    cudaError_t e = split_gemm_tcgen05(g1, s_);
    if (e != cudaSuccess) return e;
    ph_end(PH_GEMM1);
    SplitGemmArgs g2;
    memset(&g2, 0, sizeof(g2));
    g2.Ahi = Bhi_;
    g2.Alo = Blo_;
    g2.Bhi = VThi_;
    g2.Blo = VTlo_;
    g2.M = M;
    g2.Mdev = nnz_;
    g2.N = ldp_;
    g2.K = Npad;
    g2.lda = ncap_pad_;
    g2.ldb = ncap_pad_;
    g2.Hhi = Chi_;
    g2.Hlo = Clo_;
    g2.ldh = ldp_;
    g2.rn2 = rn2f_;
    g2.epilogue = 1;
    g2.spin_cap = opt.spin_cap;
    g2.st = st_;
    g2.cfg = gemm_cfg_;
    g2.launches = &launches_;
    e = cudaMemsetAsync(rn2f_, 0, sizeof(float) * M, s_);
    if (e != cudaSuccess) return e;
    ph_begin();
    e = split_gemm_tcgen05(g2, s_);
    if (e != cudaSuccess) return e;
    ph_end(PH_GEMM2);
    gemm_launches_ += 2;
    return cudaSuccess;
  }

  int block_mixed(long long t0, int kb) {
    {
      const int rc = maybe_probe();
      if (rc != LC_OK) return rc;
    }
    ph_begin();
    if (q_bracket_) {
      LC_TRY(bracket_q64(Ehi_, Elo_, ncap_, t0, kb, Hhi_, Hlo_, ldp_, hn2f_, opt.spin_cap, st_, s_));
    } else if (big_bracket_) {
      LC_TRY(bracket_big(Ehi_, Elo_, ncap_, d_, t0, kb, Hhi_, Hlo_, ldp_, hn2f_, opt.spin_cap, st_, s_));
    } else if (tc_bracket_) {
      LC_TRY(bracket_tc(Ehi_, Elo_, ncap_, d_, t0, kb, Hhi_, Hlo_, ldp_, hn2f_, opt.spin_cap, st_, s_));
    } else {
      LC_TRY(bracket_mixed(src(), d_, ldp_, t0, kb, Hhi_, Hlo_, ldp_, hn2f_, s_));
    }
    ph_end(PH_BRACKET);
    // candidates with a (numerically) zero bracket are rejected outright; the
    // rest are packed into consecutive rows so the GEMMs skip the zeros
    const float es = (float)eta_screen_, ts = (float)tau_;
    ph_begin();
    // (B is not normalised: for Algorithm 3 the floor scales with ||B_l|| ||B_m||)
    LC_TRY(compact_nonzero(hn2f_, kb, es * es, nz_idx_, nnz_, s_, alg3_ ? bn2_ : nullptr, t0, part_));
    LC_TRY(gather_candidates(Hhi_, Hlo_, ldp_, hn2f_, nz_idx_, nnz_, kb, ldp_, Chi_, Clo_, hn2c_, s_));
    ph_end(PH_SCREEN);
    LC_TRY(screen_gemms(kb));
    ph_begin();
    LC_TRY(screen_compact_f32(hn2c_, rn2f_, kb, es * es, ts * ts, idx_, stats_, s_, nnz_, nz_idx_,
                              measured_tau_ ? 1 : 0, rho2f_, part_, cidx_));
    ph_end(PH_SCREEN);
    launches_ += 6;     // bracket, compaction (2), gather, screen (2); the GEMMs count themselves
    return after_screen(t0);
  }

  // Block sizes: Kgrow_ while the basis grows (bounds the in-block sequential
  // work and the duplicates screened in together), doubling up to Ksat_ once a
  // block appends nothing.  Any partition of the pair order gives the same
  // result.
  //
  // Autotuner (mixed mode, opt.autotune): the blocks that follow a block that
  // appended nothing are trials -- each screening-GEMM tile configuration with
  // each block size in kTrialK (up to the allocated K_) -- timed with CUDA
  // events from the bracket launch to the end of the block.  The fastest
  // (candidates per second) is kept for the rest of the call and cached per
  // (device, d, algorithm); a cached choice is used without trials.  A trial
  // that was cut short or appended something is repeated on the next
  // saturated block.
  static constexpr int kTrialK[4] = {4096, 8192, 16384, 32768};
  struct Trial { int cfg, kb; double rate; };
  std::vector<Trial> trials_;
  size_t trial_next_ = 0;
  bool tuning_ = false;

  void autotune_setup() {
    if (!opt.autotune || !mixed_) return;
    int dev = 0;
    cudaGetDevice(&dev);
    {
      std::lock_guard<std::mutex> g(g_tune_mu);
      auto it = g_tune.find(TuneKey{dev, d_, alg3_ ? 1 : 0});
      if (it != g_tune.end()) {
        gemm_cfg_ = it->second.cfg;
        Ksat_ = std::min(K_, it->second.kb);
        autotuned_ = true;
        return;
      }
    }
    for (int c = 0; c < split_gemm_num_cfgs(); ++c)
      for (int kb : kTrialK)
        if (kb <= K_) trials_.push_back({c, kb, 0.0});
    if (trials_.empty()) trials_.push_back({0, K_, 0.0});
    tuning_ = true;
  }

  void autotune_finish() {
    tuning_ = false;
    const Trial* best = &trials_[0];
    for (const Trial& t : trials_)
      if (t.rate > best->rate) best = &t;
    gemm_cfg_ = best->cfg;
    Ksat_ = best->kb;
    autotuned_ = true;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune[TuneKey{dev, d_, alg3_ ? 1 : 0}] = TuneVal{best->cfg, best->kb};
  }

  int sweep() {
    t_ = n_resume_ >= 0 ? t_resume_ : 0;
    autotune_setup();
    long long knext = Kgrow_;
    bool saturated = false;              // the previous block appended nothing
    cudaEvent_t ta = nullptr, tb = nullptr;
    if (tuning_) {
      cudaEventCreate(&ta);
      cudaEventCreate(&tb);
    }
    int rc = LC_OK;
    for (;;) {
      const long long T = pairs_below(N_);
      if (t_ >= T) break;
      if (dmax_ >= 0 && N_ >= dmax_) break;
      const bool trial = tuning_ && saturated && trial_next_ < trials_.size();
      long long want = trial ? trials_[trial_next_].kb : std::min<long long>(knext, Ksat_);
      if (trial) gemm_cfg_ = trials_[trial_next_].cfg;
      long long kb = std::min<long long>(want, T - t_);
      if (opt.max_candidates > 0) kb = std::min<long long>(kb, opt.max_candidates - checked_);
      if (kb <= 0) break;
      const long long n_before = N_;
      if (trial) cudaEventRecord(ta, s_);
      rc = mixed_ ? block_mixed(t_, (int)kb) : block_fp64(t_, (int)kb);
      if (trial && rc == LC_OK) {
        cudaEventRecord(tb, s_);
        float ms = 0.f;
        if (cudaEventSynchronize(tb) == cudaSuccess && cudaEventElapsedTime(&ms, ta, tb) == cudaSuccess &&
            kb == want && N_ == n_before && ms > 0.f) {
          trials_[trial_next_].rate = (double)kb / (1e-3 * ms);
          ++trial_next_;
          ++trials_done_;
          if (trial_next_ == trials_.size()) autotune_finish();
        }
      }
      saturated = (N_ == n_before);
      knext = saturated ? std::min<long long>(2 * kb, Ksat_) : Kgrow_;
      ++blocks_;
      t_ += kb;
      checked_ += kb;
      if (opt.verbose)
        fprintf(stderr, "lieclosure: block %lld t=%lld kb=%lld cfg=%d flagged=%d dim %lld -> %lld\n", blocks_, t_ - kb,
                kb, gemm_cfg_, host_ ? host_->stats.nflag : -1, n_before, N_);
      if (rc != LC_OK) break;
    }
    if (tuning_) {
      // trials left unfinished: keep the best measured so far for this call
      // (not cached), else the defaults
      const Trial* best = nullptr;
      for (const Trial& t : trials_)
        if (t.rate > 0 && (!best || t.rate > best->rate)) best = &t;
      gemm_cfg_ = best ? best->cfg : 0;
      tuning_ = false;
    }
    if (ta) cudaEventDestroy(ta);
    if (tb) cudaEventDestroy(tb);
    return rc;
  }
};

int check_args(const void* g, int k, int d, double tol, long long max_dim, const lc_options& o) {
  if (!g || k < 1 || d < 2 || !(tol > 0.0) || max_dim < 1) return LC_ERR_ARG;
  if (o.precision != LC_PREC_FP64 && o.precision != LC_PREC_MIXED_BF16X3) return LC_ERR_ARG;
  if (o.block_k < 0 || o.block_k_growth < 0 || o.tau_screen < 0 || o.eta_abs < 0 || o.max_candidates < 0 ||
      o.screen_kappa < 0 || !(o.screen_kappa == o.screen_kappa))
    return LC_ERR_ARG;
  if (o.tol_mode != LC_TOL_RELATIVE && o.tol_mode != LC_TOL_ABSOLUTE) return LC_ERR_ARG;
  if (o.accept_kernel < 0 || o.accept_kernel > 3) return LC_ERR_ARG;
  if (o.accept_gemm < 0 || o.accept_gemm > 1) return LC_ERR_ARG;
  if ((long long)d * d > (1ll << 31) / 2) return LC_ERR_ARG;
  return LC_OK;
}

int closure_device(const double2* d_gens, int k, int d, double tol, double2* d_basis, long long* dim_out,
                   long long max_dim, const lc_options& o, lc_report* rep, cudaStream_t s, bool alg3 = false,
                   double2* d_nested = nullptr, long long resume_t = -1) {
  const long long ncap = std::min<long long>(max_dim, (long long)d * d);
  Closure c(k, d, tol, ncap, o, s, alg3);
  if (resume_t >= 0) c.set_resume(k, resume_t);
  int rc = c.run(d_gens, d_basis, dim_out, rep, d_nested);
  if (rc == LC_OK && max_dim < (long long)d * d && dim_out && *dim_out > max_dim) rc = LC_ERR_CAPACITY;
  return rc;
}

// One closure from host buffers on stream s (generators copied in, basis
// copied out), used by lie_closure and by each batched worker.
int closure_host(const lc_c128* generators, int k, int d, double tol, lc_c128* basis_out, long long* dim_out,
                 long long max_dim, const lc_options& o, lc_report* rep, cudaStream_t s, bool alg3 = false,
                 lc_c128* nested_out = nullptr, long long resume_t = -1) {
  if (dim_out) *dim_out = 0;
  int rc = check_args(generators, k, d, tol, max_dim, o);
  if (rc != LC_OK) return rc;
  const size_t gbytes = sizeof(double2) * (size_t)k * d * d;
  const long long ncap = std::min<long long>(max_dim, (long long)d * d);
  const size_t bbytes = basis_out ? sizeof(double2) * (size_t)ncap * d * d : 0;
  const size_t nbytes = (alg3 && nested_out) ? sizeof(double2) * (size_t)ncap * d * d : 0;
  double2 *dg = nullptr, *db = nullptr, *dn = nullptr;
  cudaMemPool_t pool;
  if (get_pool(&pool) != cudaSuccess) rc = LC_ERR_CUDA;
  if (rc == LC_OK && cudaMallocFromPoolAsync(reinterpret_cast<void**>(&dg), gbytes, pool, s) != cudaSuccess)
    rc = LC_ERR_OOM;
  if (rc == LC_OK && bbytes &&
      cudaMallocFromPoolAsync(reinterpret_cast<void**>(&db), bbytes, pool, s) != cudaSuccess)
    rc = LC_ERR_OOM;
  if (rc == LC_OK && nbytes &&
      cudaMallocFromPoolAsync(reinterpret_cast<void**>(&dn), nbytes, pool, s) != cudaSuccess)
    rc = LC_ERR_OOM;
  if (rc == LC_OK && cudaMemcpyAsync(dg, generators, gbytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    rc = LC_ERR_CUDA;
  long long dim = 0;
  if (rc == LC_OK) rc = closure_device(dg, k, d, tol, db, &dim, max_dim, o, rep, s, alg3, dn, resume_t);
  if ((rc == LC_OK || rc == LC_ERR_CAPACITY) && dim > 0) {
    const size_t out = sizeof(double2) * (size_t)std::min(dim, ncap) * d * d;
    if (db && cudaMemcpyAsync(basis_out, db, out, cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = LC_ERR_CUDA;
    if (dn && cudaMemcpyAsync(nested_out, dn, out, cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = LC_ERR_CUDA;
  }
  if (dg) cudaFreeAsync(dg, s);
  if (db) cudaFreeAsync(db, s);
  if (dn) cudaFreeAsync(dn, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == LC_OK) rc = LC_ERR_CUDA;
  if (dim_out) *dim_out = dim;
  return rc;
}

// Independent sets: worker threads, one CUDA stream each, take sets in order
// of decreasing size (d, then k) from a shared cursor, so the long closures
// start first and the many small, latency-bound ones fill the gaps.
// With parent != nullptr (the device-pointer form) the worker streams first
// wait for the work queued on parent, and each set runs closure_device on its
// device buffers.
int batched_host(int nsets, const lc_c128* const* generators, const int* k, const int* d, double tol,
                 lc_c128* const* basis_out, const long long* max_dim, long long* dim_out, int* status_out,
                 const lc_options& o, lc_report* rep, bool device = false, cudaStream_t parent = nullptr) {
  std::vector<int> order(nsets);
  for (int i = 0; i < nsets; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (d[a] != d[b]) return d[a] > d[b];
    return k[a] > k[b];
  });
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LC_ERR_CUDA;
  const int nworkers = std::max(1, std::min(nsets, 16));
  std::atomic<int> next(0);
  std::vector<int> status(nsets, LC_OK);
  cudaEvent_t ready = nullptr;
  if (device) {
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) return LC_ERR_CUDA;
    if (cudaEventRecord(ready, parent) != cudaSuccess) {
      cudaEventDestroy(ready);
      return LC_ERR_CUDA;
    }
  }
  auto work = [&]() {
    cudaSetDevice(dev);
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        (device && cudaStreamWaitEvent(s, ready, 0) != cudaSuccess)) {
      for (int i = next.fetch_add(1); i < nsets; i = next.fetch_add(1)) status[order[i]] = LC_ERR_CUDA;
      return;
    }
    for (int i = next.fetch_add(1); i < nsets; i = next.fetch_add(1)) {
      const int q = order[i];
      long long dim = 0;
      lc_c128* out = basis_out ? basis_out[q] : nullptr;
      if (device) {
        status[q] = check_args(generators[q], k[q], d[q], tol, max_dim[q], o);
        if (status[q] == LC_OK)
          status[q] = closure_device(reinterpret_cast<const double2*>(generators[q]), k[q], d[q], tol,
                                     reinterpret_cast<double2*>(out), &dim, max_dim[q], o, rep ? rep + q : nullptr,
                                     s);
      } else {
        status[q] = closure_host(generators[q], k[q], d[q], tol, out, &dim, max_dim[q], o, rep ? rep + q : nullptr,
                                 s);
      }
      if (dim_out) dim_out[q] = dim;
    }
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> pool;
  for (int w = 0; w < nworkers; ++w) pool.emplace_back(work);
  for (auto& t : pool) t.join();
  if (ready) cudaEventDestroy(ready);
  int first = LC_OK;
  for (int q = 0; q < nsets; ++q) {
    if (status_out) status_out[q] = status[q];
    if (status[q] != LC_OK && first == LC_OK) first = status[q];
  }
  return first;
}

}  // namespace

extern "C" {

void lc_default_options(lc_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = LC_PREC_MIXED_BF16X3;
  o->eta_abs = 1e-12;
  o->tau_screen = 0.0;          // measured
  o->screen_kappa = 10.0;
  o->tol_mode = LC_TOL_RELATIVE;
  o->autotune = 0;
  o->ortho_check = 0;
  o->block_k = 0;
  o->saturation_exit = 0;
  o->spin_cap = 0;
  o->max_candidates = 0;
  o->verbose = 0;
  o->profile = 0;
  o->fault_inject = 0;
}

const char* lc_status_string(int s) {
  switch (s) {
    case LC_OK: return "ok";
    case LC_ERR_ARG: return "invalid argument";
    case LC_ERR_NOT_ANTIHERMITIAN: return "generator is not anti-Hermitian";
    case LC_ERR_NONFINITE: return "non-finite value in the generators";
    case LC_ERR_CAPACITY: return "basis capacity (max_dim, or term_capacity of the Pauli-sum path) exceeded";
    case LC_ERR_CUDA: return "CUDA error";
    case LC_ERR_OOM: return "out of device memory";
    case LC_ERR_TIMEOUT: return "device wait timed out";
    case LC_ERR_TOO_LARGE: return "problem exceeds the fixed-size buffer";
    default: return "unknown status";
  }
}

const char* lc_version(void) {
  return "lieclosure-gb300 0.5 (sm_103a; screening GEMM 128x256x32, split-K; d = 64 bracket M = 128 persistent; "
         "FP64-accurate tensor-core accept projections; shared-memory in-block accept)";
}

int lie_closure_dev(const lc_c128* generators, int k, int d, double tol, lc_c128* basis_out, long long* dim_out,
                    long long max_dim, const lc_options* opt, lc_report* rep, void* stream) {
  lc_options o;
  if (opt) o = *opt; else lc_default_options(&o);
  if (dim_out) *dim_out = 0;
  int rc = check_args(generators, k, d, tol, max_dim, o);
  if (rc != LC_OK) return rc;
  return closure_device(reinterpret_cast<const double2*>(generators), k, d, tol,
                        reinterpret_cast<double2*>(basis_out), dim_out, max_dim, o, rep,
                        static_cast<cudaStream_t>(stream));
}

int lie_closure(const lc_c128* generators, int k, int d, double tol, lc_c128* basis_out, long long* dim_out,
                long long max_dim, const lc_options* opt, lc_report* rep) {
  lc_options o;
  if (opt) o = *opt; else lc_default_options(&o);
  if (dim_out) *dim_out = 0;
  int rc = check_args(generators, k, d, tol, max_dim, o);
  if (rc != LC_OK) return rc;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return LC_ERR_CUDA;
  rc = closure_host(generators, k, d, tol, basis_out, dim_out, max_dim, o, rep, s);
  cudaStreamDestroy(s);
  return rc;
}

int lie_closure_alg3(const lc_c128* generators, int k, int d, double tol, lc_c128* nested_out, lc_c128* basis_out,
                     long long* dim_out, long long max_dim, const lc_options* opt, lc_report* rep) {
  lc_options o;
  if (opt) o = *opt; else lc_default_options(&o);
  if (dim_out) *dim_out = 0;
  int rc = check_args(generators, k, d, tol, max_dim, o);
  if (rc != LC_OK) return rc;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return LC_ERR_CUDA;
  rc = closure_host(generators, k, d, tol, basis_out, dim_out, max_dim, o, rep, s, true, nested_out);
  cudaStreamDestroy(s);
  return rc;
}

int lie_closure_alg3_dev(const lc_c128* generators, int k, int d, double tol, lc_c128* nested_out,
                         lc_c128* basis_out, long long* dim_out, long long max_dim, const lc_options* opt,
                         lc_report* rep, void* stream) {
  lc_options o;
  if (opt) o = *opt; else lc_default_options(&o);
  if (dim_out) *dim_out = 0;
  int rc = check_args(generators, k, d, tol, max_dim, o);
  if (rc != LC_OK) return rc;
  return closure_device(reinterpret_cast<const double2*>(generators), k, d, tol,
                        reinterpret_cast<double2*>(basis_out), dim_out, max_dim, o, rep,
                        static_cast<cudaStream_t>(stream), true, reinterpret_cast<double2*>(nested_out));
}

int lie_closure_alg2_dev(const lc_c128* generators, int k, int d, double tol, lc_c128* basis_out,
                         long long* dim_out, long long max_dim, const lc_options* opt, lc_report* rep,
                         void* stream) {
  lc_options o;
  if (opt) o = *opt; else lc_default_options(&o);
  if (dim_out) *dim_out = 0;
  int rc = check_args(generators, k, d, tol, max_dim, o);
  if (rc != LC_OK) return rc;
  return closure_alg2_device(reinterpret_cast<const double2*>(generators), k, d, tol,
                             reinterpret_cast<double2*>(basis_out), dim_out, max_dim, o, rep,
                             static_cast<cudaStream_t>(stream));
}

int lie_closure_alg2(const lc_c128* generators, int k, int d, double tol, lc_c128* basis_out, long long* dim_out,
                     long long max_dim, const lc_options* opt, lc_report* rep) {
  lc_options o;
  if (opt) o = *opt; else lc_default_options(&o);
  if (dim_out) *dim_out = 0;
  int rc = check_args(generators, k, d, tol, max_dim, o);
  if (rc != LC_OK) return rc;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return LC_ERR_CUDA;
  const size_t gbytes = sizeof(double2) * (size_t)k * d * d;
  const long long ncap = std::min<long long>(max_dim, (long long)d * d);
  const size_t bbytes = basis_out ? sizeof(double2) * (size_t)ncap * d * d : 0;
  double2 *dg = nullptr, *db = nullptr;
  long long dim = 0;
  if (cudaMallocAsync(reinterpret_cast<void**>(&dg), gbytes, s) != cudaSuccess) rc = LC_ERR_OOM;
  if (rc == LC_OK && bbytes && cudaMallocAsync(reinterpret_cast<void**>(&db), bbytes, s) != cudaSuccess)
    rc = LC_ERR_OOM;
  if (rc == LC_OK && cudaMemcpyAsync(dg, generators, gbytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    rc = LC_ERR_CUDA;
  if (rc == LC_OK) rc = closure_alg2_device(dg, k, d, tol, db, &dim, max_dim, o, rep, s);
  if ((rc == LC_OK || rc == LC_ERR_CAPACITY) && db && dim > 0 &&
      cudaMemcpyAsync(basis_out, db, sizeof(double2) * (size_t)std::min(dim, ncap) * d * d,
                      cudaMemcpyDeviceToHost, s) != cudaSuccess)
    rc = LC_ERR_CUDA;
  if (dg) cudaFreeAsync(dg, s);
  if (db) cudaFreeAsync(db, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == LC_OK) rc = LC_ERR_CUDA;
  cudaStreamDestroy(s);
  if (dim_out) *dim_out = dim;
  return rc;
}

namespace {
int resume_args(const lc_c128* basis_in, long long n_in, long long l, long long m, int d, double tol,
                long long max_dim, const lc_options& o, long long* t) {
  if (!basis_in || n_in < 1 || n_in > (1ll << 30)) return LC_ERR_ARG;
  if (l < 1 || m < 0 || m >= l) return LC_ERR_ARG;
  if (max_dim < n_in) return LC_ERR_CAPACITY;
  int rc = check_args(basis_in, (int)n_in, d, tol, max_dim, o);
  if (rc != LC_OK) return rc;
  *t = l * (l - 1) / 2 + m;
  return LC_OK;
}
}  // namespace

int lie_closure_resume(const lc_c128* basis_in, long long n_in, long long cursor_l, long long cursor_m, int d,
                       double tol, lc_c128* basis_out, long long* dim_out, long long max_dim, const lc_options* opt,
                       lc_report* rep) {
  lc_options o;
  if (opt) o = *opt; else lc_default_options(&o);
  if (dim_out) *dim_out = 0;
  long long t = 0;
  int rc = resume_args(basis_in, n_in, cursor_l, cursor_m, d, tol, max_dim, o, &t);
  if (rc != LC_OK) return rc;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return LC_ERR_CUDA;
  rc = closure_host(basis_in, (int)n_in, d, tol, basis_out, dim_out, max_dim, o, rep, s, false, nullptr, t);
  cudaStreamDestroy(s);
  return rc;
}

int lie_closure_resume_dev(const lc_c128* basis_in, long long n_in, long long cursor_l, long long cursor_m, int d,
                           double tol, lc_c128* basis_out, long long* dim_out, long long max_dim,
                           const lc_options* opt, lc_report* rep, void* stream) {
  lc_options o;
  if (opt) o = *opt; else lc_default_options(&o);
  if (dim_out) *dim_out = 0;
  long long t = 0;
  int rc = resume_args(basis_in, n_in, cursor_l, cursor_m, d, tol, max_dim, o, &t);
  if (rc != LC_OK) return rc;
  return closure_device(reinterpret_cast<const double2*>(basis_in), (int)n_in, d, tol,
                        reinterpret_cast<double2*>(basis_out), dim_out, max_dim, o, rep,
                        static_cast<cudaStream_t>(stream), false, nullptr, t);
}

int lie_closure_batched(int nsets, const lc_c128* const* generators, const int* k, const int* d, double tol,
                        lc_c128* const* basis_out, const long long* max_dim, long long* dim_out, int* status_out,
                        const lc_options* opt, lc_report* rep) {
  if (nsets < 0 || (nsets > 0 && (!generators || !k || !d || !max_dim))) return LC_ERR_ARG;
  if (nsets == 0) return LC_OK;
  lc_options o;
  if (opt) o = *opt; else lc_default_options(&o);
  return batched_host(nsets, generators, k, d, tol, basis_out, max_dim, dim_out, status_out, o, rep);
}

int lie_closure_batched_dev(int nsets, const lc_c128* const* generators, const int* k, const int* d, double tol,
                            lc_c128* const* basis_out, const long long* max_dim, long long* dim_out, int* status_out,
                            const lc_options* opt, lc_report* rep, void* stream) {
  if (nsets < 0 || (nsets > 0 && (!generators || !k || !d || !max_dim))) return LC_ERR_ARG;
  if (nsets == 0) return LC_OK;
  lc_options o;
  if (opt) o = *opt; else lc_default_options(&o);
  return batched_host(nsets, generators, k, d, tol, basis_out, max_dim, dim_out, status_out, o, rep, true,
                      static_cast<cudaStream_t>(stream));
}

}  // extern "C"
