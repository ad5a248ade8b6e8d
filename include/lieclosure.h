/*
 * lieclosure.h -- C ABI of the GB300 (sm_103a) Lie-closure library.
 *
 * The library computes the closure of a set of d x d anti-Hermitian matrices
 * with Algorithm 4 of Iiyama, "Fast numerical generation of Lie closure"
 * (arXiv 2506.01120, Section 3.2): a generator pass, then a sweep over brackets
 * [V[l], V[m]] of the growing orthonormal basis V, each tested for linear
 * independence by projecting it onto span(V) (the Corollary of Theorem 1) and
 * appended, normalised, when its orthogonal part is non-zero.
 *
 * Definitions used throughout (Section 2.2 of the paper):
 *   bracket        [a, b] = ab - ba
 *   inner product  <a, b> = tr(a^dagger b) / d
 *   norm           ||a|| = sqrt(<a, a>)
 * Every basis element written by the library has ||v|| = 1 in this norm, i.e.
 * Frobenius norm sqrt(d), and <v_i, v_j> = delta_ij.
 *
 * Independence test ("h_perp != 0" in Algorithm 4, which the paper leaves
 * without a tolerance): a candidate h is accepted iff ||h|| > eta_abs and
 * ||h - proj_V h|| > tol * ||h||, the residual taken from two classical
 * Gram-Schmidt passes in FP64.  Each bracket (l, m), m < l, is formed once, in
 * the order l = 1, 2, ..., m = 0 .. l-1, and the sweep ends when l reaches |V|.
 *
 * Memory and threading: the library allocates its own device workspace for
 * the duration of a call (through a stream-ordered pool it keeps per device)
 * and frees it before returning; nothing it allocates is handed to the caller.
 * Calls on different streams may run concurrently; one call per stream.
 * No call uses more than the current CUDA device.
 */
#ifndef LIECLOSURE_H
#define LIECLOSURE_H

#if defined(__GNUC__)
#define LC_API __attribute__((visibility("default")))
#else
#define LC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Interleaved complex128, the layout of numpy.complex128 and std::complex<double>. */
typedef struct { double re, im; } lc_c128;

typedef enum {
  LC_OK = 0,
  LC_ERR_ARG = -1,               /* null pointer, k < 1, d < 1, tol <= 0, bad option */
  LC_ERR_NOT_ANTIHERMITIAN = -2, /* some generator has |g + g^dagger| > 1e-12 max|g| */
  LC_ERR_NONFINITE = -3,         /* NaN or Inf in the generators */
  LC_ERR_CAPACITY = -4,          /* the basis would exceed max_dim; dim_out = max_dim */
  LC_ERR_CUDA = -5,              /* a CUDA runtime call failed */
  LC_ERR_OOM = -6,               /* device workspace could not be allocated */
  LC_ERR_TIMEOUT = -7,           /* a bounded device-side wait ran out */
  LC_ERR_TOO_LARGE = -8          /* problem exceeds a fixed-size buffer (see
                                    lc_split_gemm_f32_noalloc) */
} lc_status;

typedef enum {
  /* every product, projection and residual in FP64 (SIMT) */
  LC_PREC_FP64 = 0,
  /* brackets and projections screened with split-BF16 tensor-core products
     (three BF16 MMAs per product, FP32 accumulation); candidates whose
     screened relative residual exceeds tau_screen are recomputed and decided
     in FP64, so every accepted element is an FP64 result */
  LC_PREC_MIXED_BF16X3 = 1
} lc_precision;

typedef enum {
  /* accept iff ||h - proj_V h|| > tol * ||h|| (default) */
  LC_TOL_RELATIVE = 0,
  /* accept iff ||h - proj_V h|| > tol (elements of V have unit norm, so this
     is the literal "h_perp != 0" of Algorithm 4 with an absolute threshold) */
  LC_TOL_ABSOLUTE = 1
} lc_tol_mode;

typedef struct {
  int precision;              /* lc_precision; default LC_PREC_MIXED_BF16X3 */
  double eta_abs;             /* absolute floor on ||h||; default 1e-12 */
  double tau_screen;          /* mixed mode: relative residual below which a
                                 screened candidate is rejected without the FP64
                                 recheck.  0 (default) = measured: tau_screen =
                                 screen_kappa * eps_screen, where eps_screen is
                                 the largest screened relative residual of
                                 probe vectors that lie in span(V) (true
                                 residual 0), re-measured whenever |V| has grown
                                 by 1/8; clamped to [2^-21, 1e-3] */
  int block_k;                /* candidates per block once the basis stops
                                 growing; 0 = automatic (16384 mixed, 2048 FP64,
                                 capped by an 8 GB buffer budget) */
  int block_k_growth;         /* candidates per block while the basis grows;
                                 0 = automatic (1024; 256 when d >= 256) */
  int saturation_exit;        /* nonzero: stop once |V| reaches the largest
                                 possible dimension (d^2 - 1, plus one if a
                                 generator has a trace); not in the paper,
                                 default 0 */
  long long spin_cap;         /* iteration bound for device spin-waits; 0 = default */
  long long max_candidates;   /* stop after this many bracket candidates
                                 (0 = run to the end); the report then carries
                                 the cursor (l, m) */
  int verbose;                /* nonzero: per-block log lines on stderr */
  int profile;                /* nonzero: time each phase with CUDA events on
                                 the call's stream (lc_report.t_phase_s) */
  int fault_inject;           /* test hook, 0 in normal use: nonzero makes the
                                 first grid barrier of the in-block accept wait
                                 for an arrival that never comes, so its bounded
                                 wait runs out (spin_cap) and the call returns
                                 LC_ERR_TIMEOUT with the device still usable */
  int tol_mode;               /* lc_tol_mode; default LC_TOL_RELATIVE (dense
                                 paths; lie_closure_alg2 and lie_closure_pauli
                                 ignore it) */
  int autotune;               /* mixed mode, nonzero: the first blocks after the
                                 basis stops growing try screening-GEMM tile
                                 shapes and block sizes on the real candidates,
                                 time them with CUDA events and keep the fastest
                                 for the rest of the call; the choice is cached
                                 per (device, d, Algorithm 3 or 4) and reused by
                                 later calls without trials.  Any choice gives
                                 the same basis (blocking does not change the
                                 decisions).  Default 0: fixed defaults */
  int ortho_check;            /* nonzero: before returning, compute
                                 rep->ortho_defect = max |<v_i, v_j> - delta_ij|
                                 in FP64 on the device, over all rows when
                                 |V| <= 4096, else over every q-th row with
                                 q = ceil(|V| / 4096).  Default 0 (the report
                                 field is then -1) */
  double screen_kappa;        /* factor of the measured tau_screen; 0 =
                                 default (10).  A smaller factor narrows the
                                 band of true residuals the screen could reject
                                 and flags more noise for the FP64 recheck
                                 (time, not correctness) */
  int accept_kernel;          /* in-block test and append: 0 = by shape
                                 (default), 1 = one CTA per flagged row,
                                 2 = every row sliced across all SMs (panels of
                                 at most 128 rows), 3 = one CTA per flagged
                                 row holding it in shared memory (rows of at
                                 most 16,384 components; else 1).  All take
                                 the same decisions in the same order; 1 and 3
                                 compute identical values, 2 differs in the
                                 order of the FP64 partial sums */
  int fp64_first_pass;        /* mixed mode: nonzero = the first projection of
                                 flagged candidates is always an FP64 GEMM.
                                 Default 0: when some flagged row of a block
                                 needs the second pass anyway (screened
                                 rho^2 < 1/2) and every one has rho^2 >= 1e-6,
                                 the first projection takes the screening
                                 GEMM's coefficients and the FP64 pass follows
                                 (three FP64 GEMMs instead of four) */
  int accept_gemm;            /* mixed mode, projections of the flagged rows
                                 against V (c = R V^T, R -= c V): 0 (default) =
                                 FP64-accurate BF16 tensor-core GEMMs
                                 (lc_gemm_f64_tc's digit slicing) at d = 64 ..
                                 128 when the product is large; 1 = FP64 SIMT
                                 GEMMs always.  FP64 mode always uses FP64 SIMT */
} lc_options;

typedef struct {
  long long dim;              /* |V| on return */
  long long brackets_checked; /* bracket candidates tested */
  long long generators_checked;
  long long n_nonzero;        /* bracket candidates with ||h|| above the floor */
  long long n_flagged;        /* candidates sent to the FP64 accept step */
  long long n_blocks;
  long long cursor_l, cursor_m; /* next pair of the sweep on return */
  double t_total_s;           /* wall time of the call */
  double t_last_accept_s;     /* wall time at the last accepted element */
  double min_acc_rel_res;     /* smallest relative residual among accepts */
  double max_rej_rel_res;     /* largest FP64 relative residual among flagged rejects */
  double tau_screen;          /* screen threshold used (mixed mode) */
  double max_screen_rej_rel_res; /* largest screened relative residual among
                                 candidates the screen rejected (after the
                                 basis stops growing this is the noise floor
                                 of the screen) */
  long long kernel_launches;  /* kernels this call launched */
  long long gemm_launches;    /* screening GEMM launches (projection + residual) */
  double gemm_flops;          /* sum over those launches of 3 * 2 * rows * cols *
                                 depth with the unpadded extents (three split
                                 products per multiply-add) */
  double t_phase_s[6];        /* with opt.profile: device time per phase --
                                 0 brackets, 1 projection GEMM, 2 residual GEMM,
                                 3 screen, 4 FP64 accept, 5 other */
  int precision;
  int status;
  long long n_gray;           /* mixed: screen rejects whose screened relative
                                 residual lay in (eps_screen, tau_screen], the
                                 band where the screen cannot tell a small true
                                 residual from its own noise */
  double eps_screen;          /* mixed: measured noise floor of the screen (the
                                 largest value over the run's probes) */
  double min_acc_screen_rel_res; /* mixed: smallest screened relative residual
                                 among candidates that were then accepted
                                 (their margin above tau_screen) */
  double ortho_defect;        /* with opt.ortho_check: max |<v_i, v_j> -
                                 delta_ij| over the checked rows, else -1 */
  long long ortho_rows;       /* rows in that check */
  int block_k_used;           /* saturated-phase block size used */
  int block_k_growth_used;    /* growth-phase block size used */
  int gemm_tile_n;            /* screening GEMM tile (128 x gemm_tile_n output, */
  int gemm_tile_k;            /*   gemm_tile_k-wide k-slices) */
  int autotuned;              /* 1 if block_k_used and the tile came from the
                                 autotuner (trials in this call or its cache) */
  int autotune_trials;        /* trial blocks this call spent */
  long long accept_wide_launches; /* in-block accept panels run by the
                                 row-sliced kernel (accept_kernel) */
  long long screen_pass1_blocks; /* blocks whose first projection took the
                                 screening coefficients (fp64_first_pass) */
  long long accept_tc_gemms;  /* projections run as FP64-accurate tensor-core
                                 GEMMs (accept_gemm) */
} lc_report;

/* Fills *opt with the defaults listed above. */
LC_API void lc_default_options(lc_options* opt);

/* Static, human-readable name of a status code. */
LC_API const char* lc_status_string(int status);

/* Library version string. */
LC_API const char* lc_version(void);

/*
 * lie_closure -- Algorithm 4 on one generator set (Section 3.2), host buffers.
 *
 * generators : k x d x d complex128, row-major, host memory, caller-owned,
 *              read only.  Each must be anti-Hermitian (g^dagger = -g) within
 *              1e-12 * max|g|; they are taken in the given order.
 * k, d       : number of generators (>= 1) and matrix size (>= 2).
 * tol        : relative residual tolerance (> 0) of the independence test.
 * basis_out  : host buffer for max_dim x d x d complex128 (row-major), or NULL
 *              to return the dimension only.  On LC_OK and LC_ERR_CAPACITY the
 *              first *dim_out elements are the orthonormal basis V in the
 *              order Algorithm 4 appends them.
 * dim_out    : receives |V| (always written when non-NULL).
 * max_dim    : capacity of basis_out in elements (>= 1); the library also uses
 *              it to size its device basis.  d*d always suffices.
 * opt, rep   : options (NULL = defaults) and report (NULL = none).
 * Returns an lc_status.  On error the contents of basis_out are unspecified
 * beyond *dim_out elements.
 */
LC_API int lie_closure(const lc_c128* generators, int k, int d, double tol,
                lc_c128* basis_out, long long* dim_out, long long max_dim,
                const lc_options* opt, lc_report* rep);

/*
 * lie_closure_dev -- as lie_closure, with device buffers and a stream.
 *
 * generators and basis_out are device pointers of the current device
 * (basis_out may be NULL); stream is a cudaStream_t passed as void*
 * (NULL = the legacy default stream).  The call is synchronous with respect
 * to the host: it returns after the stream has finished its work.
 */
LC_API int lie_closure_dev(const lc_c128* generators, int k, int d, double tol,
                    lc_c128* basis_out, long long* dim_out, long long max_dim,
                    const lc_options* opt, lc_report* rep, void* stream);

/*
 * lie_closure_alg2 -- Algorithm 2 of the paper (Section 3.1): the
 * matrix-inversion method.  B holds unit-norm operators (the normalised
 * generators and normalised brackets [B[l], B[m]], same pair order as
 * lie_closure); a candidate h (normalised) is independent iff
 * ||h - B^T (A^-1 beta)|| > tol, beta_i = <B_i, h>, with A the Gram matrix of B
 * (Theorem 1).  A^-1 is kept and grown by the bordered-inverse identity on each
 * append.  FP64 throughout (opt->precision is ignored).  The paper notes that
 * A can become ill-conditioned; lie_closure (Algorithm 4) is the stable method.
 *
 * basis_out : host buffer for max_dim x d x d complex128 receiving B (unit
 *             norm, not orthogonal), or NULL.  Other arguments as lie_closure;
 *             max_dim also sizes the stored max_dim x max_dim inverse.
 */
LC_API int lie_closure_alg2(const lc_c128* generators, int k, int d, double tol,
                     lc_c128* basis_out, long long* dim_out, long long max_dim,
                     const lc_options* opt, lc_report* rep);

/* lie_closure_alg2_dev -- as lie_closure_alg2 with device buffers and a stream
 * (conventions of lie_closure_dev). */
LC_API int lie_closure_alg2_dev(const lc_c128* generators, int k, int d, double tol,
                         lc_c128* basis_out, long long* dim_out, long long max_dim,
                         const lc_options* opt, lc_report* rep, void* stream);

/*
 * lie_closure_alg3 -- Algorithm 3 of the paper (Section 3.2): the
 * orthonormalisation method that keeps, beside the orthonormal basis V, the
 * basis B made of the accepted generators and nested brackets themselves.
 * Brackets are formed from elements of B ([B[l], B[m]], same pair order as
 * lie_closure) and tested against V with the same rule; an accepted bracket h
 * is appended to B as it is and to V as h_perp / ||h_perp||.  span(B) = span(V)
 * is the same algebra lie_closure returns.
 *
 * nested_out : host buffer for max_dim x d x d complex128 receiving B (or NULL).
 * basis_out  : host buffer receiving V (or NULL).
 * Other arguments, statuses and the report are those of lie_closure.  B is
 * not normalised: its elements are the brackets as formed, so their norms can
 * grow with nesting depth.
 */
LC_API int lie_closure_alg3(const lc_c128* generators, int k, int d, double tol,
                     lc_c128* nested_out, lc_c128* basis_out, long long* dim_out,
                     long long max_dim, const lc_options* opt, lc_report* rep);

/* lie_closure_alg3_dev -- as lie_closure_alg3 with device buffers and a stream
 * (conventions of lie_closure_dev). */
LC_API int lie_closure_alg3_dev(const lc_c128* generators, int k, int d, double tol,
                         lc_c128* nested_out, lc_c128* basis_out, long long* dim_out,
                         long long max_dim, const lc_options* opt, lc_report* rep,
                         void* stream);

/*
 * lie_closure_resume -- continue Algorithm 4 from a saved state.  The state of
 * Algorithm 4 is its basis V and its pair cursor (l, m) (Section 3.2): a call
 * stopped by opt->max_candidates (or LC_ERR_CAPACITY) returns both, the basis
 * in basis_out and the cursor in rep->cursor_l / rep->cursor_m.  Passing them
 * back here runs the rest of the sweep; a run split this way gives the same
 * basis as one uninterrupted run.
 *
 * basis_in : n_in x d x d complex128 host array, the orthonormal basis a
 *            previous call returned (in its order); read only.
 * cursor_l, cursor_m : the next pair, 0 <= cursor_m < cursor_l.
 * max_dim  : capacity (>= n_in) of basis_out and of the device basis.
 * basis_out, dim_out, opt, rep, return value: as lie_closure; basis_out
 *            receives the whole basis (the n_in given elements first).
 */
LC_API int lie_closure_resume(const lc_c128* basis_in, long long n_in, long long cursor_l,
                       long long cursor_m, int d, double tol, lc_c128* basis_out,
                       long long* dim_out, long long max_dim, const lc_options* opt,
                       lc_report* rep);

/* lie_closure_resume_dev -- as lie_closure_resume with device buffers and a
 * stream (conventions of lie_closure_dev). */
LC_API int lie_closure_resume_dev(const lc_c128* basis_in, long long n_in, long long cursor_l,
                           long long cursor_m, int d, double tol, lc_c128* basis_out,
                           long long* dim_out, long long max_dim, const lc_options* opt,
                           lc_report* rep, void* stream);

/*
 * lie_closure_batched -- Algorithm 4 on nsets independent generator sets
 * (Section 3.2 applied per set), host buffers.
 *
 * generators[s] : k[s] x d[s] x d[s] complex128 host array of set s.
 * basis_out[s]  : host buffer of max_dim[s] x d[s] x d[s] complex128 or NULL;
 *                 basis_out itself may be NULL (dimensions only).
 * max_dim[s]    : capacity of set s (>= 1).
 * dim_out[s], status_out[s] : per-set dimension and lc_status.
 * rep           : NULL or an array of nsets reports.
 * Returns LC_OK if every set returned LC_OK, else the first failing status.
 */
LC_API int lie_closure_batched(int nsets, const lc_c128* const* generators, const int* k,
                        const int* d, double tol, lc_c128* const* basis_out,
                        const long long* max_dim, long long* dim_out, int* status_out,
                        const lc_options* opt, lc_report* rep);

/*
 * lie_closure_batched_dev -- as lie_closure_batched with device buffers and a
 * stream.  generators[s] and basis_out[s] are device pointers of the current
 * device (the arrays of pointers themselves, k, d, max_dim, dim_out,
 * status_out and rep are host memory); basis_out or basis_out[s] may be NULL.
 * The sets run concurrently on streams of the library's own, ordered after the
 * work already queued on `stream` (cudaStream_t as void*, NULL = legacy
 * default stream); the call returns when every set is done.
 */
LC_API int lie_closure_batched_dev(int nsets, const lc_c128* const* generators, const int* k,
                            const int* d, double tol, lc_c128* const* basis_out,
                            const long long* max_dim, long long* dim_out, int* status_out,
                            const lc_options* opt, lc_report* rep, void* stream);

/*
 * lie_closure_pauli -- Algorithm 4 (Section 3.2) on operators held as sparse
 * sums of Pauli strings, the representation Section 3 recommends for large
 * systems and Section 4.2 uses for Table 2.  No d x d matrix is formed.
 *
 * Representation.  An operator is a = i * sum_t c_t P_t with real c_t (so a is
 * anti-Hermitian) and P_t an n-qubit Pauli string.  A string is packed into
 * one 64-bit word as x | (z << 32): bit q of x / z is the X / Z part on qubit
 * q+1 (qubit 1 is the leftmost Kronecker factor), so (x, z) = (1, 0) is X,
 * (1, 1) is Y and (0, 1) is Z on that qubit.  Distinct strings are orthonormal
 * under <a, b> = tr(a^dagger b) / d (Section 2.2), so <a, b> = sum_t a_t b_t
 * over common strings and every step of the method is done on the coefficient
 * lists: a bracket of two strings is zero when they commute and
 * +-2i times the string x1^x2 | z1^z2 when they anticommute.
 *
 * strings, coefs : the generators' terms, concatenated; generator j owns
 *              entries [offsets[j], offsets[j+1]).  Host memory, read only.
 *              Repeated strings inside one generator are summed.
 * offsets    : k + 1 non-decreasing entries, offsets[0] = 0.
 * n_qubits   : 1 .. 31; every string must have no bit at or above n_qubits in
 *              x or z (else LC_ERR_ARG).
 * tol        : relative tolerance of the independence test (as lie_closure).
 * basis_strings, basis_coefs : host buffers of term_capacity entries receiving
 *              the orthonormal basis V in the order Algorithm 4 appends it,
 *              each element's terms sorted by string; element i owns entries
 *              [basis_offsets[i], basis_offsets[i+1]).  Terms whose magnitude
 *              is below 1e-13 of the element's norm are dropped.  May be NULL
 *              (dimension only).
 * basis_offsets : host buffer of max_dim + 1 entries (or NULL).
 * term_capacity : total terms the basis may hold (>= 1); sizes the device
 *              arrays too.  Exceeding it returns LC_ERR_CAPACITY.
 * max_dim    : capacity in elements (>= 1).
 * opt, rep   : as lie_closure; opt->precision is ignored (everything is FP64,
 *              exact for single-string sets), opt->block_k is the candidate
 *              block (0 = 2^22), opt->fault_inject = 2 starts the per-candidate
 *              hash tables at their smallest size (a test hook that exercises
 *              the regrow path).
 * Report: brackets_checked, n_flagged, cursor and the residual margins as in
 * lie_closure; gemm_launches counts screen launches here, and with
 * opt->profile t_phase_s[3] / t_phase_s[4] are the device times of the screen
 * and of the in-order accept.
 * Limits: a candidate's terms (and its residual's) must fit 4096 distinct
 * strings and its projection 2048 basis elements (the per-warp tables in
 * shared memory, filled at most half); dense operators belong to lie_closure.
 * Returns LC_OK, LC_ERR_ARG, LC_ERR_NONFINITE, LC_ERR_CAPACITY (basis,
 * term or per-candidate table capacity exceeded; *dim_out elements are valid),
 * LC_ERR_CUDA or LC_ERR_OOM.
 */
LC_API int lie_closure_pauli(const unsigned long long* strings, const double* coefs,
                      const long long* offsets, int k, int n_qubits, double tol,
                      unsigned long long* basis_strings, double* basis_coefs,
                      long long* basis_offsets, long long term_capacity,
                      long long* dim_out, long long max_dim, const lc_options* opt,
                      lc_report* rep);

/* lie_closure_pauli_dev -- as lie_closure_pauli with every array (offsets
 * included) in device memory of the current device and a stream (conventions
 * of lie_closure_dev). */
LC_API int lie_closure_pauli_dev(const unsigned long long* strings, const double* coefs,
                          const long long* offsets, int k, int n_qubits, double tol,
                          unsigned long long* basis_strings, double* basis_coefs,
                          long long* basis_offsets, long long term_capacity,
                          long long* dim_out, long long max_dim, const lc_options* opt,
                          lc_report* rep, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LIECLOSURE_H */
