// Algorithm 4 of arXiv 2506.01120 (Section 3.2) on sparse Pauli-sum operators.
//
// Section 3 notes that generators acting on few qubits are sparse sums of
// Pauli strings and that the orthonormalisation test, unlike the rank test,
// keeps that form; Section 4.2 (Table 2) runs the method so, on CPU cores.
// Here every step works on coefficient lists on the GPU:
//
//   operator   a = i sum_s a_s P_s with real a_s and Hermitian Pauli strings
//              P_s; strings are orthonormal under <a, b> = tr(a^dagger b)/d
//              (Section 2.2), so <a, b> = sum_s a_s b_s.
//   bracket    [i a_s P_s, i b_t P_t] is zero when P_s and P_t commute; when
//              they anticommute, P_s P_t = i^g P_{s^t} with g odd and the
//              bracket is -2 a_s b_t i^g P_{s^t}, i.e. coefficient
//              -2 a_s b_t (g == 1 ? 1 : -1) on i P_{s^t}.
//   projection beta_r = sum_s x_s v_r(s) through an index string -> basis
//              terms, then x -= sum_r beta_r v_r (the Corollary of Theorem 1).
//
// Layout in HBM.  The basis is a term arena (string, coefficient, owning
// element, next term with the same string) with element offsets, plus an
// open-addressing table string -> most recent term; an append writes its
// terms to the arena and pushes each on its string's chain.  A candidate's
// terms live in a per-warp open-addressing table in shared memory
// (string -> coefficient, FP64 shared-memory atomics) and its projection
// coefficients in a second one (element -> beta).
//
// Block semantics are those of the dense path: a block is a contiguous run of
// the pair order with l < |V| at block start.  The screen (one warp per
// candidate) computes one classical Gram-Schmidt pass against the block-start
// basis in FP64 and flags candidates with ||r|| > (tol/2) ||h||; a smaller
// residual against that basis means a smaller one against any larger basis,
// so those are rejected exactly as Algorithm 4 rejects them.  One warp then
// takes the flagged candidates in pair order and re-tests each against the
// current basis with two passes, appending accepts at once: the sequential
// test of Algorithm 4.  A candidate whose terms do not fit the screen's table
// is flagged too and handled by the accept warp, whose tables are larger and
// grow on demand.  No kernel here waits on another thread or block.
#include "lc_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

namespace lc {
namespace {

using u64 = unsigned long long;

constexpr u64 kEmpty = ~0ull;        // never a string: x has no bit 31 for n <= 31
constexpr unsigned kFull = 0xffffffffu;
constexpr int kScreenMaxSlots = 4096;  // screen tables: terms / betas per warp
constexpr int kAcceptMaxSlots = 8192;  // accept tables at their largest
constexpr double kPrune = 1e-13;       // terms below this fraction of ||r|| are dropped

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// splitmix64 finaliser (Steele, Lea and Flood, "Fast splittable pseudorandom
// number generators", 2014) as the slot hash
__device__ __forceinline__ uint32_t slot_hash(u64 k) {
  k ^= k >> 30;
  k *= 0xbf58476d1ce4e5b9ull;
  k ^= k >> 27;
  k *= 0x94d049bb133111ebull;
  k ^= k >> 31;
  return (uint32_t)k;
}

// P_a P_b = i^g P_{a^b}; returns g mod 4, odd iff the strings anticommute.
// Per qubit XY = iZ, YZ = iX, ZX = iY add one to g, the reversed products
// subtract one, equal letters or an identity add nothing.
__device__ __forceinline__ int pauli_phase(u64 a, u64 b) {
  const uint32_t x1 = (uint32_t)a, z1 = (uint32_t)(a >> 32), x2 = (uint32_t)b, z2 = (uint32_t)(b >> 32);
  const uint32_t plus = (x1 & ~z1 & x2 & z2) | (x1 & z1 & ~x2 & z2) | (~x1 & z1 & x2 & ~z2);
  const uint32_t minus = (x1 & z1 & x2 & ~z2) | (~x1 & z1 & x2 & z2) | (x1 & ~z1 & ~x2 & z2);
  return (__popc(plus) - __popc(minus)) & 3;
}

// Reads of basis arrays: read-only (through the non-coherent cache) in the
// screen, whose basis does not change during the launch; plain volatile loads
// in the accept kernel, which appends while it reads.
template <bool RO, typename T>
__device__ __forceinline__ T ld(const T* p) {
  if constexpr (RO) return __ldg(p);
  else return *const_cast<const volatile T*>(p);
}

struct Table {       // open addressing, linear probing, shared memory
  u64* key;
  double* val;
  int* used;         // occupied slots
  uint32_t mask;     // slots - 1 (slots a power of two, >= 32)
};

// val[key] += v; false once a new key would fill more than half the slots
// (the load bound keeps every probe sequence short)
__device__ __forceinline__ bool table_add(const Table& t, u64 key, double v) {
  uint32_t i = slot_hash(key) & t.mask;
  for (uint32_t p = 0; p <= t.mask; ++p) {
    u64 cur = *const_cast<volatile u64*>(&t.key[i]);
    if (cur == kEmpty) {
      cur = atomicCAS(&t.key[i], kEmpty, key);
      if (cur == kEmpty) {
        if (atomicAdd(t.used, 1) >= (int)((t.mask + 1) >> 1)) return false;
        cur = key;
      }
    }
    if (cur == key) {
      atomicAdd(&t.val[i], v);
      return true;
    }
    i = (i + 1) & t.mask;
  }
  return false;
}

__device__ __forceinline__ void table_clear(const Table& t, int lane) {
  for (uint32_t i = lane; i <= t.mask; i += 32) {
    t.key[i] = kEmpty;
    t.val[i] = 0.0;
  }
  if (lane == 0) *t.used = 0;
}

// butterfly sum: every lane ends with the same value (additions commute)
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// FP64 issue is scarce on this part (each warp-wide FP64 instruction holds
// the SM's FP64 pipe for many cycles), so the norms below spend FP64
// instructions only where some lane holds a non-zero value; zero tests are
// integer tests on the bit pattern.  Skipped terms are exact zeros, so the
// sums are bit-for-bit those of the plain loop.
__device__ __forceinline__ bool nonzero(double v) { return (__double_as_longlong(v) << 1) != 0; }

// sum of per-lane partials; with at most one non-zero partial the result is
// that partial, moved by a shuffle
__device__ __forceinline__ double warp_sum_sparse(double v) {
  const unsigned bal = __ballot_sync(kFull, nonzero(v));
  if (bal == 0) return 0.0;
  if ((bal & (bal - 1)) == 0) return __shfl_sync(kFull, v, __ffs(bal) - 1);
  return warp_sum(v);
}

__device__ __forceinline__ double table_norm2(const Table& t, int lane) {
  double s = 0.0;
  for (uint32_t i = lane; i <= t.mask; i += 32) {
    const double v = t.val[i];
    const bool nz = nonzero(v);
    if (__any_sync(kFull, nz) && nz) s = fma(v, v, s);
  }
  return warp_sum_sparse(s);
}

struct PBasis {
  u64* key;          // term string
  double* val;       // term coefficient
  int* row;          // element that owns the term
  int* next;         // previous term pushed with the same string, -1 ends
  long long* off;    // element i owns terms [off[i], off[i+1])
  u64* ikey;         // index: string per slot (kEmpty = free)
  int* ihead;        // index: most recent term with that string, -1 none
  uint32_t imask;    // index slots - 1
};

struct PSrc {        // generator terms, generator j owns [off[j], off[j+1])
  const u64* key;
  const double* val;
  const long long* off;
};

struct PState {
  int n;             // |V|
  int maxT;          // most terms in one element
  long long tused;   // arena terms in use
  int start;         // accept: first block position to take
  int stop;          // accept: position it stopped at (count when done)
  int why;           // accept: 0 done, 1 candidate table full, 2 capacity, 3 index full
  int naccepted;     // accepts so far
  unsigned long long min_acc_bits, max_rej_bits, max_screen_rej_bits;
  int nflag, nnonzero, noverflow;   // screen counters of the current block
  int npure;         // flagged candidates that are one string absent from the basis
  int nfirst;        // distinct strings among them (first occurrences in pair order)
  int nonunit;       // some one-term element has a coefficient other than +-1
};

// pair index t = l(l-1)/2 + m -> (l, m): a single-precision square root
// estimate (relative error below 2^-22, so off by one at most while l < 2^21)
// made exact by integer steps; FP64 throughput is low on this part.
__device__ __forceinline__ void pair_of(long long t, int* l, int* m) {
  long long L = (long long)((1.0f + sqrtf(1.0f + 8.0f * (float)t)) * 0.5f);
  while (L > 1 && L * (L - 1) / 2 > t) --L;
  while ((L + 1) * L / 2 <= t) ++L;
  *l = (int)L;
  *m = (int)(t - L * (L - 1) / 2);
}

template <bool RO>
__device__ __forceinline__ int index_head(const PBasis& B, u64 s) {
  uint32_t i = slot_hash(s) & B.imask;
  for (uint32_t p = 0; p <= B.imask; ++p) {
    const u64 cur = ld<RO>(&B.ikey[i]);
    if (cur == s) return ld<RO>(&B.ihead[i]);
    if (cur == kEmpty) return -1;
    i = (i + 1) & B.imask;
  }
  return -1;
}

// push term e (string s) on the index; false if the index is full
__device__ __forceinline__ bool index_push(const PBasis& B, u64 s, int e) {
  uint32_t i = slot_hash(s) & B.imask;
  for (uint32_t p = 0; p <= B.imask; ++p) {
    const u64 cur = atomicCAS(&B.ikey[i], kEmpty, s);
    if (cur == kEmpty || cur == s) {
      B.next[e] = atomicExch(&B.ihead[i], e);
      return true;
    }
    i = (i + 1) & B.imask;
  }
  return false;
}

// The candidate's terms into h: generator id (gen) or the bracket
// [V_l, V_m] of pair id.  Warp-uniform result: false if h overflowed.
template <bool RO>
__device__ bool form(const PBasis& B, const PSrc& G, bool gen, long long id, const Table& h, int lane) {
  bool ok = true;
  if (gen) {
    const long long a0 = G.off[id], a1 = G.off[id + 1];
    for (long long q = a0 + lane; q < a1; q += 32) ok &= table_add(h, G.key[q], G.val[q]);
  } else {
    int l, m;
    pair_of(id, &l, &m);
    const long long a0 = ld<RO>(&B.off[l]), b0 = ld<RO>(&B.off[m]);
    const long long ta = ld<RO>(&B.off[l + 1]) - a0, tb = ld<RO>(&B.off[m + 1]) - b0;
    const long long tot = ta * tb;
    for (long long q = lane; q < tot; q += 32) {
      const long long i = q / tb, j = q - i * tb;
      const u64 ka = ld<RO>(&B.key[a0 + i]), kb = ld<RO>(&B.key[b0 + j]);
      const int g = pauli_phase(ka, kb);
      if (g & 1) {
        const double c = ld<RO>(&B.val[a0 + i]) * ld<RO>(&B.val[b0 + j]);
        ok &= table_add(h, ka ^ kb, g == 1 ? -2.0 * c : 2.0 * c);
      }
    }
  }
  ok = __all_sync(kFull, ok);
  __syncwarp();
  return ok;
}

// One classical Gram-Schmidt pass of h against the first nrows elements:
// beta = <V_r, h> through the index, then h -= sum_r beta_r V_r.
template <bool RO>
__device__ bool project(const PBasis& B, int nrows, const Table& h, const Table& bt, int lane) {
  table_clear(bt, lane);
  __syncwarp();
  bool ok = true;
  for (uint32_t i = lane; i <= h.mask; i += 32) {
    const u64 s = h.key[i];
    const double x = h.val[i];
    if (s == kEmpty || !nonzero(x)) continue;
    int e = index_head<RO>(B, s);
    for (int guard = 0; e >= 0 && guard < nrows; ++guard) {   // one term per element and string
      const int r = ld<RO>(&B.row[e]);
      if (r < nrows) ok &= table_add(bt, (u64)r, x * ld<RO>(&B.val[e]));
      e = ld<RO>(&B.next[e]);
    }
  }
  ok = __all_sync(kFull, ok);
  __syncwarp();
  if (!ok) return false;
  for (uint32_t j = lane; j <= bt.mask; j += 32) {
    const u64 r = bt.key[j];
    if (r == kEmpty) continue;
    const double be = bt.val[j];
    const long long e1 = ld<RO>(&B.off[r + 1]);
    for (long long e = ld<RO>(&B.off[r]); e < e1; ++e) ok &= table_add(h, ld<RO>(&B.key[e]), -be * ld<RO>(&B.val[e]));
  }
  ok = __all_sync(kFull, ok);
  __syncwarp();
  return ok;
}

__device__ __forceinline__ Table warp_table(unsigned char* base, int slots, int* used) {
  return Table{reinterpret_cast<u64*>(base), reinterpret_cast<double*>(base + 8ull * slots), used,
               (uint32_t)(slots - 1)};
}

// ------------------------------------------------------------------ kernels
// Screen of pairs t0 .. t0 + count - 1 against the first nrows elements;
// flag[c] = 1 for candidates the accept step must decide.  chunks: one bit per
// 1024 positions with a flag.
__global__ void __launch_bounds__(256) k_pauli_screen(PBasis B, long long t0, int count, int nrows, int hslots,
                                                      int bslots, double tol, double eta,
                                                      unsigned char* __restrict__ flag,
                                                      unsigned* __restrict__ chunks, u64* __restrict__ pkey,
                                                      double* __restrict__ pval, PState* ps) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int used[2 * 8];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  unsigned char* base = smem + (size_t)w * 16 * (hslots + bslots);
  const Table h = warp_table(base, hslots, &used[2 * w]), bt = warp_table(base + 16ull * hslots, bslots, &used[2 * w + 1]);
  const PSrc none{nullptr, nullptr, nullptr};
  int nz = 0, nf = 0, nov = 0, npure = 0;
  double maxrej = 0.0;
  const double eta2 = eta * eta, tau2 = 0.25 * tol * tol;
  for (long long c = (long long)blockIdx.x * warps + w; c < count; c += (long long)gridDim.x * warps) {
    table_clear(h, lane);
    __syncwarp();
    unsigned char fl = 0;
    if (!form<true>(B, none, false, t0 + c, h, lane)) {
      fl = 1;
      ++nov;
    } else {
      const double h2 = table_norm2(h, lane);
      if (h2 > eta2) {
        ++nz;
        if (!project<true>(B, nrows, h, bt, lane)) {
          fl = 1;
          ++nov;
        } else {
          const double r2 = table_norm2(h, lane);
          if (r2 > tau2 * h2) {
            fl = 1;
            ++nf;
            // pure: no basis element shares a string with h (beta empty, so
            // the residual is h) and h has one non-zero term
            if (*const_cast<volatile int*>(bt.used) == 0) {
              int nnz = 0;
              for (uint32_t q0 = 0; q0 <= h.mask; q0 += 32) {
                const uint32_t q = q0 + lane;
                const bool on = h.key[q] != kEmpty && nonzero(h.val[q]);
                const unsigned bal = __ballot_sync(kFull, on);
                if (on && nnz + __popc(bal & ((1u << lane) - 1u)) == 0) {
                  pkey[c] = h.key[q];
                  pval[c] = h.val[q];
                }
                nnz += __popc(bal);
              }
              if (nnz == 1) {
                fl = 2;
                ++npure;
              }
            }
          } else if (lane == 0 && nonzero(r2)) {
            maxrej = fmax(maxrej, sqrt(r2 / h2));
          }
        }
      }
    }
    if (lane == 0) {
      flag[c] = fl;
      if (fl) atomicOr(&chunks[c >> 15], 1u << ((c >> 10) & 31));
    }
    __syncwarp();
  }
  if (lane == 0) {
    if (nz) atomicAdd(&ps->nnonzero, nz);
    if (nf) atomicAdd(&ps->nflag, nf);
    if (nov) atomicAdd(&ps->noverflow, nov);
    if (npure) atomicAdd(&ps->npure, npure);
    if (maxrej > 0.0) atomicMax(&ps->max_screen_rej_bits, (unsigned long long)__double_as_longlong(maxrej));
  }
}

// Screen for a basis whose every element is one string with coefficient
// exactly +-1 (so element i owns term i): one thread per candidate.  A
// bracket of two such elements is zero (commuting strings) or +-2 times the
// product string; it is dependent exactly when that string is in the basis
// (the residual c - (c v) v is then 0 with v = +-1) and otherwise pure.  The
// flags, counters and pure records equal those of k_pauli_screen for such a
// basis, with no FP64 arithmetic outside the pure records.
__global__ void __launch_bounds__(256) k_pauli_screen1(PBasis B, long long t0, int count,
                                                       unsigned char* __restrict__ flag,
                                                       unsigned* __restrict__ chunks, u64* __restrict__ pkey,
                                                       double* __restrict__ pval, PState* ps) {
  int nz = 0, nf = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < count;
       c += (long long)gridDim.x * blockDim.x) {
    int l, m;
    pair_of(t0 + c, &l, &m);
    const u64 ka = __ldg(&B.key[l]), kb = __ldg(&B.key[m]);
    const int g = pauli_phase(ka, kb);
    unsigned char fl = 0;
    if (g & 1) {
      ++nz;
      const u64 s = ka ^ kb;
      if (index_head<true>(B, s) < 0) {
        fl = 2;
        ++nf;
        const double cv = __ldg(&B.val[l]) * __ldg(&B.val[m]);
        pkey[c] = s;
        pval[c] = g == 1 ? -2.0 * cv : 2.0 * cv;
        atomicOr(&chunks[c >> 15], 1u << ((c >> 10) & 31));
      }
    }
    flag[c] = fl;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nz += __shfl_xor_sync(kFull, nz, o);
    nf += __shfl_xor_sync(kFull, nf, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (nz) atomicAdd(&ps->nnonzero, nz);
    if (nf) {
      atomicAdd(&ps->nflag, nf);
      atomicAdd(&ps->npure, nf);
    }
  }
}

// ------------------------------------------------ blocks of pure candidates
// When every flagged candidate of a block is pure (one string, absent from the
// block-start basis), the in-order test reduces to string equality: a pure
// candidate is dependent on the basis plus the earlier accepts exactly when an
// earlier candidate of the block carries the same string.  So the accepts are
// the first occurrence of each string, appended in pair order, each
// normalised like the sequential step (v / sqrt(v * v)).

// first occurrence of each pure string: dmin[slot of s] = min position
__global__ void k_pure_first(const unsigned char* __restrict__ flag, const u64* __restrict__ pkey, int count,
                             u64* __restrict__ dkey, int* __restrict__ dmin, uint32_t dmask) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < count;
       c += (long long)gridDim.x * blockDim.x) {
    if (flag[c] != 2) continue;
    const u64 s = pkey[c];
    uint32_t i = slot_hash(s) & dmask;
    for (uint32_t p = 0; p <= dmask; ++p) {
      const u64 cur = atomicCAS(&dkey[i], kEmpty, s);
      if (cur == kEmpty || cur == s) {
        atomicMin(&dmin[i], (int)c);
        break;
      }
      i = (i + 1) & dmask;
    }
  }
}

// per 1024-position chunk: how many first occurrences (one warp per chunk)
__global__ void k_pure_count(const unsigned char* __restrict__ flag, const u64* __restrict__ pkey, int count,
                             const u64* __restrict__ dkey, const int* __restrict__ dmin, uint32_t dmask,
                             unsigned char* __restrict__ first, int* __restrict__ ccount, int nchunks) {
  const int ch = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (ch >= nchunks) return;
  int n = 0;
  for (int b = ch << 10; b < min(count, (ch + 1) << 10); b += 32) {
    const int c = b + lane;
    bool f = false;
    if (c < count && flag[c] == 2) {
      const u64 s = pkey[c];
      uint32_t i = slot_hash(s) & dmask;
      for (uint32_t p = 0; p <= dmask; ++p) {
        const u64 cur = dkey[i];
        if (cur == s) {
          f = dmin[i] == c;
          break;
        }
        if (cur == kEmpty) break;
        i = (i + 1) & dmask;
      }
    }
    if (c < count) first[c] = f ? 1 : 0;
    n += __popc(__ballot_sync(kFull, f));
  }
  if (lane == 0) ccount[ch] = n;
}

// exclusive scan of the chunk counts (one block of 1024 threads, nchunks <= 1024 * 64)
__global__ void __launch_bounds__(1024) k_pure_scan(int* __restrict__ ccount, int nchunks, PState* ps) {
  __shared__ int part[1024];
  const int per = (nchunks + 1023) / 1024;
  const int a = threadIdx.x * per, b = min(nchunks, a + per);
  int sum = 0;
  for (int i = a; i < b; ++i) sum += ccount[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {   // Hillis-Steele inclusive scan
    const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - sum;
  for (int i = a; i < b; ++i) {
    const int v = ccount[i];
    ccount[i] = run;
    run += v;
  }
  if (threadIdx.x == 1023) ps->nfirst = part[1023];
}

__device__ __forceinline__ int pure_take(const PState* ps, int n0, long long t0terms, int ncap, long long tcap) {
  return (int)min((long long)ps->nfirst, min((long long)(ncap - n0), tcap - t0terms));
}

// append the first occurrences in pair order (one warp per chunk), as many as
// fit the free rows and terms
__global__ void k_pure_append(PBasis B, const unsigned char* __restrict__ first, const u64* __restrict__ pkey,
                              const double* __restrict__ pval, int count, const int* __restrict__ coff,
                              int nchunks, int n0, long long t0terms, int ncap, long long tcap,
                              PState* ps) {
  const int ch = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (ch >= nchunks) return;
  const int take = pure_take(ps, n0, t0terms, ncap, tcap);
  int rank = coff[ch];
  for (int b = ch << 10; b < min(count, (ch + 1) << 10); b += 32) {
    const int c = b + lane;
    const bool f = c < count && first[c];
    const unsigned bal = __ballot_sync(kFull, f);
    if (f) {
      const int i = rank + __popc(bal & ((1u << lane) - 1u));
      if (i < take) {
        const double v = pval[c];
        const double r2 = fma(v, v, 0.0);
        const long long pos = t0terms + i;
        const u64 s = pkey[c];
        const double u = v * (1.0 / sqrt(r2));
        B.key[pos] = s;
        B.val[pos] = u;
        B.row[pos] = n0 + i;
        if (u != 1.0 && u != -1.0) atomicOr(&ps->nonunit, 1);
        B.off[n0 + i + 1] = pos + 1;
        index_push(B, s, (int)pos);
      }
    }
    rank += __popc(bal);
  }
}

__global__ void k_pure_commit(PState* ps, int n0, long long t0terms, int ncap, long long tcap) {
  const int take = pure_take(ps, n0, t0terms, ncap, tcap);
  ps->n = n0 + take;
  ps->tused = t0terms + take;
  ps->naccepted += take;
  ps->why = take < ps->nfirst ? 2 : 0;
  if (take > 0) {
    ps->maxT = max(ps->maxT, 1);
    atomicMin(&ps->min_acc_bits, (unsigned long long)__double_as_longlong(1.0));
  }
}

// In-order test-and-append, one warp.  gen: candidates are generators
// 0 .. count-1, all taken; otherwise pairs t0 + position with flag set.
// Starts at ps->start and stops early (ps->stop, ps->why) when a candidate
// does not fit the tables or the basis is full; nothing of that candidate has
// been written then.
__global__ void __launch_bounds__(32, 1) k_pauli_accept(PBasis B, PSrc G, int gen, long long t0, int count,
                                                        const unsigned char* __restrict__ flag,
                                                        const unsigned* __restrict__ chunks, int hslots,
                                                        int bslots, double tol, double eta, int ncap,
                                                        long long tcap, PState* ps) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int used[2];
  const int lane = threadIdx.x;
  const Table h = warp_table(smem, hslots, &used[0]), bt = warp_table(smem + 16ull * hslots, bslots, &used[1]);
  int N = ps->n, maxT = ps->maxT, nacc = 0;
  long long T = ps->tused;
  const int start = ps->start;
  int stop = count, why = 0;
  const double eta2 = eta * eta, tol2 = tol * tol;
  const int nchunks = (count + 1023) >> 10;
  for (int ch = start >> 10; ch < nchunks && why == 0; ++ch) {
    if (!gen && !((chunks[ch >> 5] >> (ch & 31)) & 1u)) continue;
    const int cend = min(count, (ch + 1) << 10);
    for (int b = ch << 10; b < cend && why == 0; b += 32) {
      const int c = b + lane;
      const bool f = c >= start && c < cend && (gen || flag[c]);
      unsigned msk = __ballot_sync(kFull, f);
      while (msk && why == 0) {
        const int cand = b + __ffs(msk) - 1;
        msk &= msk - 1;
        table_clear(h, lane);
        __syncwarp();
        if (!form<false>(B, G, gen != 0, gen ? (long long)cand : t0 + cand, h, lane)) {
          why = 1;
          stop = cand;
          break;
        }
        const double h2 = table_norm2(h, lane);
        if (!(h2 > eta2)) continue;
        if (!project<false>(B, N, h, bt, lane) || !project<false>(B, N, h, bt, lane)) {
          why = 1;
          stop = cand;
          break;
        }
        const double r2 = table_norm2(h, lane);
        const double rel = sqrt(r2 / h2);
        if (!(r2 > tol2 * h2)) {
          if (lane == 0 && rel > 0.0) atomicMax(&ps->max_rej_bits, (unsigned long long)__double_as_longlong(rel));
          continue;
        }
        const double nr = sqrt(r2), inv = 1.0 / nr, thr = kPrune * nr;
        int cnt = 0;
        for (uint32_t q = lane; q <= h.mask; q += 32) cnt += (h.key[q] != kEmpty && fabs(h.val[q]) > thr) ? 1 : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
        if (N >= ncap || T + cnt > tcap) {
          why = 2;
          stop = cand;
          break;
        }
        bool pushed = true;
        long long wpos = T;
        for (uint32_t q0 = 0; q0 <= h.mask; q0 += 32) {
          const uint32_t q = q0 + lane;
          const u64 s = h.key[q];
          const double v = h.val[q];
          const bool keep = s != kEmpty && fabs(v) > thr;
          const unsigned bal = __ballot_sync(kFull, keep);
          if (keep) {
            const long long pos = wpos + __popc(bal & ((1u << lane) - 1u));
            const double u = v * inv;
            B.key[pos] = s;
            B.val[pos] = u;
            B.row[pos] = N;
            pushed &= index_push(B, s, (int)pos);
            if (cnt == 1 && u != 1.0 && u != -1.0) atomicOr(&ps->nonunit, 1);
          }
          wpos += __popc(bal);
        }
        if (lane == 0) B.off[N + 1] = T + cnt;
        pushed = __all_sync(kFull, pushed);
        __syncwarp();
        if (!pushed) {   // cannot happen with the index at most half full
          why = 3;
          stop = cand;
          break;
        }
        ++N;
        ++nacc;
        T += cnt;
        maxT = max(maxT, cnt);
        if (lane == 0) atomicMin(&ps->min_acc_bits, (unsigned long long)__double_as_longlong(rel));
      }
    }
  }
  if (lane == 0) {
    ps->n = N;
    ps->tused = T;
    ps->maxT = maxT;
    ps->stop = stop;
    ps->why = why;
    ps->naccepted += nacc;
  }
}

// Validation of generator terms: strings inside n qubits, finite coefficients,
// whether some generator has an identity term (a trace direction).
__global__ void k_pauli_check(const u64* __restrict__ key, const double* __restrict__ val, long long nt, int nq,
                              int* __restrict__ bad) {
  const u64 lim = nq >= 32 ? 0ull : ~((1ull << nq) - 1ull);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nt; i += (long long)gridDim.x * blockDim.x) {
    const u64 s = key[i];
    const double v = val[i];
    if (((s & 0xffffffffull) & lim) || ((s >> 32) & lim)) atomicOr(&bad[0], 1);
    if (!isfinite(v)) atomicOr(&bad[1], 1);
    if (s == 0ull && v != 0.0) atomicOr(&bad[2], 1);
  }
}

// Sort the terms of every element by string (bitonic network in shared
// memory, one block per element, n2 a power of two >= the longest element).
__global__ void k_pauli_sort(u64* __restrict__ key, double* __restrict__ val, const long long* __restrict__ off, int n2) {
  extern __shared__ __align__(16) unsigned char smem[];
  u64* sk = reinterpret_cast<u64*>(smem);
  double* sv = reinterpret_cast<double*>(smem + 8ull * n2);
  const long long a = off[blockIdx.x], len = off[blockIdx.x + 1] - a;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    sk[i] = i < len ? key[a + i] : kEmpty;
    sv[i] = i < len ? val[a + i] : 0.0;
  }
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const int p = i ^ j;
        if (p > i) {
          const bool up = (i & k) == 0;
          if ((sk[i] > sk[p]) == up) {
            const u64 tk = sk[i];
            sk[i] = sk[p];
            sk[p] = tk;
            const double tv = sv[i];
            sv[i] = sv[p];
            sv[p] = tv;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    key[a + i] = sk[i];
    val[a + i] = sv[i];
  }
}

int pow2_at_least(long long x, int lo, int hi) {
  int p = lo;
  while (p < x && p < hi) p <<= 1;
  return p;
}

#define LP_TRY(x)                                                                                \
  do {                                                                                           \
    cudaError_t e_ = (x);                                                                        \
    if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? LC_ERR_OOM : LC_ERR_CUDA;    \
  } while (0)

class ClosureP {
 public:
  ClosureP(int k, int nq, double tol, long long ncap, long long tcap, const lc_options& o, cudaStream_t s)
      : k_(k), nq_(nq), tol_(tol), ncap_(ncap), tcap_(tcap), opt_(o), s_(s) {
    eta_ = o.eta_abs > 0 ? o.eta_abs : 1e-12;
    K_ = o.block_k > 0 ? o.block_k : (1 << 22);
    K_ = (int)std::max<long long>(1, std::min<long long>(K_, pairs_below(ncap)));   // no larger than the sweep
  }
  ~ClosureP() {
    for (cudaEvent_t& e : ev_)
      if (e) cudaEventDestroy(e);
    if (base_) cudaFreeAsync(base_, s_);
    if (hs_) cudaFreeHost(hs_);
  }

  int run(const u64* d_key, const double* d_val, const long long* d_off, const long long* h_off, u64* o_key,
          double* o_val, long long* o_off, long long* dim_out, lc_report* rep) {
    const double t0 = now_s();
    t_start_ = t0;
    int rc = setup(d_key, d_val, d_off, h_off);
    if (rc == LC_OK) rc = generator_pass();
    if (rc == LC_OK) rc = sweep();
    if ((rc == LC_OK || rc == LC_ERR_CAPACITY) && N_ > 0) {
      const int n2 = pow2_at_least(maxT_, 1, kAcceptMaxSlots);
      const size_t sm = 16ull * n2;
      if (cudaFuncSetAttribute(k_pauli_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        rc = LC_ERR_CUDA;
      if (rc != LC_ERR_CUDA) {
        k_pauli_sort<<<(unsigned)N_, 256, sm, s_>>>(B_.key, B_.val, B_.off, n2);
        ++launches_;
        if (cudaGetLastError() != cudaSuccess) rc = LC_ERR_CUDA;
      }
      if (rc != LC_ERR_CUDA && o_key && o_val && o_off) {
        if (cudaMemcpyAsync(o_key, B_.key, sizeof(u64) * T_, cudaMemcpyDeviceToDevice, s_) != cudaSuccess ||
            cudaMemcpyAsync(o_val, B_.val, sizeof(double) * T_, cudaMemcpyDeviceToDevice, s_) != cudaSuccess ||
            cudaMemcpyAsync(o_off, B_.off, sizeof(long long) * (N_ + 1), cudaMemcpyDeviceToDevice, s_) !=
                cudaSuccess)
          rc = LC_ERR_CUDA;
      }
    } else if (rc == LC_OK && o_off) {
      if (cudaMemsetAsync(o_off, 0, sizeof(long long), s_) != cudaSuccess) rc = LC_ERR_CUDA;
    }
    if (cudaStreamSynchronize(s_) != cudaSuccess && rc == LC_OK) rc = LC_ERR_CUDA;
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
      rep->t_total_s = now_s() - t0;
      rep->t_last_accept_s = t_last_ - t0;
      if (hs_) {
        const unsigned long long mb = hs_->min_acc_bits;
        rep->min_acc_rel_res = mb == ~0ull ? 0.0 : bits_to_double(mb);
        rep->max_rej_rel_res = bits_to_double(hs_->max_rej_bits);
        rep->max_screen_rej_rel_res = bits_to_double(hs_->max_screen_rej_bits);
      }
      rep->tau_screen = 0.5 * tol_;
      rep->kernel_launches = launches_;
      rep->gemm_launches = screens_;       // here: screen launches
      rep->t_phase_s[3] = t_screen_;
      rep->t_phase_s[4] = t_accept_;
      rep->precision = LC_PREC_FP64;
      rep->status = rc;
    }
    return rc;
  }

 private:
  int k_, nq_, K_;
  double tol_, eta_;
  long long ncap_, tcap_;
  lc_options opt_;
  cudaStream_t s_;
  char* base_ = nullptr;
  PState* hs_ = nullptr;     // pinned host copy of the state
  PState* ps_ = nullptr;
  PBasis B_{};
  PSrc G_{};
  unsigned char* flag_ = nullptr;
  u64* pkey_ = nullptr;          // pure candidates: string and coefficient
  double* pval_ = nullptr;
  unsigned char* first_ = nullptr;
  int* ccount_ = nullptr;        // per-chunk counts, then offsets
  u64* dkey_ = nullptr;          // first-occurrence table
  int* dmin_ = nullptr;
  long long dslots_ = 64;
  long long pure_blocks_ = 0;
  unsigned* chunks_ = nullptr;
  int* bad_ = nullptr;
  int hsl_ = 64, bsl_ = 32, hacc_ = 256, bacc_ = 128, maxT_ = 0, maxTg_ = 0;
  bool trace_ = false;
  long long N_ = 0, T_ = 0, t_ = 0, checked_ = 0, flagged_ = 0, nonzero_ = 0, blocks_ = 0, launches_ = 0;
  double t_start_ = 0.0, t_last_ = 0.0, t_screen_ = 0.0, t_accept_ = 0.0;
  long long screens_ = 0, screens1_ = 0;
  cudaEvent_t ev_[4] = {nullptr, nullptr, nullptr, nullptr};   // with opt.profile: screen, accept

  bool profiling() {
    if (!opt_.profile) return false;
    if (!ev_[0])
      for (cudaEvent_t& e : ev_)
        if (cudaEventCreate(&e) != cudaSuccess) return false;
    return true;
  }
  static double elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    return cudaEventElapsedTime(&ms, a, b) == cudaSuccess ? 1e-3 * ms : 0.0;
  }
  int nsm_ = 152;

  static double bits_to_double(unsigned long long b) {
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
  }

  int setup(const u64* d_key, const double* d_val, const long long* d_off, const long long* h_off) {
    long long islots = 64;
    while (islots < 2 * tcap_) islots <<= 1;
    const size_t Kc = (size_t)K_;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t at = off; off = (off + bytes + 255) & ~size_t(255); return at; };
    const size_t oK = take(8ull * tcap_), oV = take(8ull * tcap_), oR = take(4ull * tcap_), oN = take(4ull * tcap_);
    const size_t oO = take(8ull * (ncap_ + 1)), oIK = take(8ull * islots), oIH = take(4ull * islots);
    const size_t oF = take(Kc), oC = take(4ull * ((Kc + 32767) / 32768 + 1)), oS = take(sizeof(PState)),
                 oB = take(16);
    dslots_ = 64;
    while (dslots_ < 2 * (long long)Kc) dslots_ <<= 1;
    const size_t oPK = take(8ull * Kc), oPV = take(8ull * Kc), oFi = take(Kc), oCC = take(4ull * ((Kc + 1023) / 1024)),
                 oDK = take(8ull * dslots_), oDM = take(4ull * dslots_);
    int dev = 0;
    LP_TRY(cudaGetDevice(&dev));
    LP_TRY(cudaDeviceGetAttribute(&nsm_, cudaDevAttrMultiProcessorCount, dev));
    LP_TRY(cudaHostAlloc(reinterpret_cast<void**>(&hs_), sizeof(PState), cudaHostAllocDefault));
    LP_TRY(cudaMallocAsync(reinterpret_cast<void**>(&base_), off, s_));
    auto at = [&](size_t o) { return base_ + o; };
    B_.key = (u64*)at(oK);
    B_.val = (double*)at(oV);
    B_.row = (int*)at(oR);
    B_.next = (int*)at(oN);
    B_.off = (long long*)at(oO);
    B_.ikey = (u64*)at(oIK);
    B_.ihead = (int*)at(oIH);
    B_.imask = (uint32_t)(islots - 1);
    flag_ = (unsigned char*)at(oF);
    chunks_ = (unsigned*)at(oC);
    pkey_ = (u64*)at(oPK);
    pval_ = (double*)at(oPV);
    first_ = (unsigned char*)at(oFi);
    ccount_ = (int*)at(oCC);
    dkey_ = (u64*)at(oDK);
    dmin_ = (int*)at(oDM);
    ps_ = (PState*)at(oS);
    bad_ = (int*)at(oB);
    LP_TRY(cudaMemsetAsync(B_.off, 0, sizeof(long long) * (ncap_ + 1), s_));
    LP_TRY(cudaMemsetAsync(B_.ikey, 0xff, 8ull * islots, s_));
    LP_TRY(cudaMemsetAsync(B_.ihead, 0xff, 4ull * islots, s_));
    LP_TRY(cudaMemsetAsync(bad_, 0, 16, s_));
    PState z;
    memset(&z, 0, sizeof z);
    z.min_acc_bits = ~0ull;
    *hs_ = z;
    LP_TRY(cudaMemcpyAsync(ps_, hs_, sizeof(PState), cudaMemcpyHostToDevice, s_));
    G_ = PSrc{d_key, d_val, d_off};
    const long long nt = h_off[k_];
    for (int j = 0; j < k_; ++j) maxTg_ = (int)std::max<long long>(maxTg_, h_off[j + 1] - h_off[j]);
    if (nt > 0) {
      const int grid = (int)std::min<long long>((nt + 255) / 256, 4ll * nsm_);
      k_pauli_check<<<grid, 256, 0, s_>>>(d_key, d_val, nt, nq_, bad_);
      ++launches_;
      LP_TRY(cudaGetLastError());
    }
    int bad[4] = {0, 0, 0, 0};
    LP_TRY(cudaMemcpyAsync(bad, bad_, 16, cudaMemcpyDeviceToHost, s_));
    LP_TRY(cudaStreamSynchronize(s_));
    if (bad[0]) return LC_ERR_ARG;
    if (bad[1]) return LC_ERR_NONFINITE;
    trace_ = bad[2] != 0;
    // candidate tables: the accept warp's start from the generators' size
    hacc_ = pow2_at_least(4ll * maxTg_ + 32, 256, kAcceptMaxSlots);
    bacc_ = pow2_at_least(hacc_ / 2, 128, kAcceptMaxSlots / 2);
    if (opt_.fault_inject == 2) {   // test hook: smallest tables, so the regrow path runs
      hacc_ = 32;
      bacc_ = 32;
    }
    return LC_OK;
  }

  int read_state() {
    LP_TRY(cudaMemcpyAsync(hs_, ps_, sizeof(PState), cudaMemcpyDeviceToHost, s_));
    LP_TRY(cudaStreamSynchronize(s_));
    return LC_OK;
  }

  // accept step over count positions of the current block, regrowing the
  // tables as needed
  int accept(bool gen, long long t0, int count) {
    int start = 0;
    for (;;) {
      hs_->start = start;
      // only start is meant to change: write it alone
      LP_TRY(cudaMemcpyAsync(&ps_->start, &hs_->start, sizeof(int), cudaMemcpyHostToDevice, s_));
      const size_t sm = 16ull * (hacc_ + bacc_);
      LP_TRY(cudaFuncSetAttribute(k_pauli_accept, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      const bool prof = profiling();
      if (prof) cudaEventRecord(ev_[2], s_);
      k_pauli_accept<<<1, 32, sm, s_>>>(B_, G_, gen ? 1 : 0, t0, count, flag_, chunks_, hacc_, bacc_, tol_, eta_,
                                        (int)ncap_, tcap_, ps_);
      if (prof) cudaEventRecord(ev_[3], s_);
      ++launches_;
      LP_TRY(cudaGetLastError());
      int rc = read_state();
      if (rc != LC_OK) return rc;
      if (prof) t_accept_ += elapsed(ev_[2], ev_[3]);
      const long long before = N_;
      N_ = hs_->n;
      T_ = hs_->tused;
      maxT_ = hs_->maxT;
      if (N_ > before) t_last_ = now_s();
      if (hs_->why == 0) return LC_OK;
      if (hs_->why == 1 && hacc_ < kAcceptMaxSlots) {
        hacc_ *= 2;
        bacc_ = std::min(bacc_ * 2, kAcceptMaxSlots / 2);
        start = hs_->stop;
        continue;
      }
      return LC_ERR_CAPACITY;
    }
  }

  // a block whose flagged candidates are all pure: first occurrences in
  // pair order, appended in parallel
  int pure_block(int count) {
    long long ds = 64;
    while (ds < 2ll * hs_->npure) ds <<= 1;
    const uint32_t dmask = (uint32_t)(ds - 1);
    const int nchunks = (count + 1023) / 1024;
    const bool prof = profiling();
    if (prof) cudaEventRecord(ev_[2], s_);
    LP_TRY(cudaMemsetAsync(dkey_, 0xff, 8ull * ds, s_));
    LP_TRY(cudaMemsetAsync(dmin_, 0x7f, 4ull * ds, s_));
    const int g1 = (int)std::min<long long>((count + 255) / 256, 8ll * nsm_);
    k_pure_first<<<g1, 256, 0, s_>>>(flag_, pkey_, count, dkey_, dmin_, dmask);
    const int g2 = (nchunks + 7) / 8;
    k_pure_count<<<g2, 256, 0, s_>>>(flag_, pkey_, count, dkey_, dmin_, dmask, first_, ccount_, nchunks);
    k_pure_scan<<<1, 1024, 0, s_>>>(ccount_, nchunks, ps_);
    k_pure_append<<<g2, 256, 0, s_>>>(B_, first_, pkey_, pval_, count, ccount_, nchunks, (int)N_, T_, (int)ncap_,
                                       tcap_, ps_);
    k_pure_commit<<<1, 1, 0, s_>>>(ps_, (int)N_, T_, (int)ncap_, tcap_);
    if (prof) cudaEventRecord(ev_[3], s_);
    launches_ += 5;
    ++pure_blocks_;
    LP_TRY(cudaGetLastError());
    const int rc = read_state();
    if (rc != LC_OK) return rc;
    if (prof) t_accept_ += elapsed(ev_[2], ev_[3]);
    const long long before = N_;
    N_ = hs_->n;
    T_ = hs_->tused;
    maxT_ = hs_->maxT;
    if (N_ > before) t_last_ = now_s();
    return hs_->why == 2 ? LC_ERR_CAPACITY : LC_OK;
  }

  int generator_pass() {
    const int rc = accept(true, 0, k_);
    if (opt_.verbose) fprintf(stderr, "lieclosure-pauli: generators %d -> dim %lld\n", k_, N_);
    return rc;
  }

  void size_screen() {
    const long long est = (long long)maxT_ * maxT_ + 4ll * maxT_ + 16;
    hsl_ = std::max(hsl_, pow2_at_least(2 * est, 64, kScreenMaxSlots));
    bsl_ = std::max(bsl_, pow2_at_least(hsl_ / 2, 32, kScreenMaxSlots / 2));
    if (opt_.fault_inject != 2) {
      hacc_ = std::max(hacc_, hsl_);
      bacc_ = std::max(bacc_, bsl_);
    }
  }

  int sweep() {
    long long dmax = -1;
    if (opt_.saturation_exit && nq_ <= 31) dmax = (1ll << (2 * nq_)) - 1 + (trace_ ? 1 : 0);
    size_screen();
    for (;;) {
      const long long Tp = pairs_below(N_);
      if (t_ >= Tp) break;
      if (dmax >= 0 && N_ >= dmax) break;
      long long kb = std::min<long long>(K_, Tp - t_);
      if (opt_.max_candidates > 0) kb = std::min<long long>(kb, opt_.max_candidates - checked_);
      if (kb <= 0) break;
      const int count = (int)kb;
      // per-block counters and chunk bits
      hs_->nflag = hs_->nnonzero = hs_->noverflow = hs_->npure = hs_->nfirst = 0;
      LP_TRY(cudaMemcpyAsync(&ps_->nflag, &hs_->nflag, 5 * sizeof(int), cudaMemcpyHostToDevice, s_));
      LP_TRY(cudaMemsetAsync(chunks_, 0, 4ull * ((count + 32767) / 32768 + 1), s_));
      // one-term elements with unit coefficients: the thread-per-candidate
      // screen gives the same flags (needs ||h|| = 2 above the floor and a
      // new string's relative residual 1 above tol / 2)
      const bool unit1 = maxT_ == 1 && hs_->nonunit == 0 && eta_ < 2.0 && tol_ < 2.0;
      const bool prof = profiling();
      if (unit1) {
        const int grid = (int)std::max<long long>(1, std::min<long long>((count + 255) / 256, 8ll * nsm_));
        if (prof) cudaEventRecord(ev_[0], s_);
        k_pauli_screen1<<<grid, 256, 0, s_>>>(B_, t_, count, flag_, chunks_, pkey_, pval_, ps_);
        ++screens1_;
      } else {
        const int warps = std::max(1, std::min(8, (96 * 1024) / (16 * (hsl_ + bsl_))));
        const size_t sm = 16ull * (hsl_ + bsl_) * warps;
        LP_TRY(cudaFuncSetAttribute(k_pauli_screen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        const long long want = (count + warps - 1) / warps;
        const int grid = (int)std::max<long long>(1, std::min<long long>(want, 8ll * nsm_));
        if (prof) cudaEventRecord(ev_[0], s_);
        k_pauli_screen<<<grid, 32 * warps, sm, s_>>>(B_, t_, count, (int)N_, hsl_, bsl_, tol_, eta_, flag_,
                                                     chunks_, pkey_, pval_, ps_);
      }
      if (prof) cudaEventRecord(ev_[1], s_);
      ++screens_;
      ++launches_;
      LP_TRY(cudaGetLastError());
      const long long n_before = N_;
      int rc = read_state();
      if (rc != LC_OK) return rc;
      if (prof) t_screen_ += elapsed(ev_[0], ev_[1]);
      if (hs_->nflag + hs_->noverflow == 0) {
        rc = LC_OK;                                  // nothing to decide
      } else if (hs_->noverflow == 0 && hs_->npure == hs_->nflag) {
        rc = pure_block(count);
      } else {
        rc = accept(false, t_, count);
      }
      nonzero_ += hs_->nnonzero;
      flagged_ += hs_->nflag + hs_->noverflow;
      ++blocks_;
      t_ += kb;
      checked_ += kb;
      if (opt_.verbose)
        fprintf(stderr, "lieclosure-pauli: block %lld t=%lld kb=%lld flagged=%d (pure %d) overflow=%d dim %lld -> %lld\n",
                blocks_, t_ - kb, kb, hs_->nflag, hs_->npure, hs_->noverflow, n_before, N_);
      if (rc != LC_OK) return rc;
      if (hs_->noverflow > count / 64) {   // screen tables too small for this basis
        hsl_ = std::min(hsl_ * 2, kScreenMaxSlots);
        bsl_ = std::min(bsl_ * 2, kScreenMaxSlots / 2);
      }
      size_screen();
    }
    return LC_OK;
  }
};

int check_pauli_args(const void* key, const void* val, const void* off, int k, int nq, double tol,
                     long long tcap, long long max_dim, const lc_options& o) {
  if (!key || !val || !off || k < 1 || nq < 1 || nq > 31 || !(tol > 0.0) || max_dim < 1 || tcap < 1)
    return LC_ERR_ARG;
  if (tcap >= (1ll << 31) || max_dim >= (1ll << 31)) return LC_ERR_ARG;
  if (o.block_k < 0 || o.eta_abs < 0 || o.max_candidates < 0) return LC_ERR_ARG;
  return LC_OK;
}

bool offsets_ok(const long long* h_off, int k) {
  if (h_off[0] != 0) return false;
  for (int j = 0; j < k; ++j)
    if (h_off[j + 1] < h_off[j]) return false;
  return true;
}

int closure_pauli_device(const u64* d_key, const double* d_val, const long long* d_off, const long long* h_off,
                         int k, int nq, double tol, u64* o_key, double* o_val, long long* o_off, long long tcap,
                         long long* dim_out, long long max_dim, const lc_options& o, lc_report* rep, cudaStream_t s) {
  const long long ncap = std::min<long long>(max_dim, nq <= 15 ? (1ll << (2 * nq)) : max_dim);
  ClosureP c(k, nq, tol, ncap, tcap, o, s);
  return c.run(d_key, d_val, d_off, h_off, o_key, o_val, o_off, dim_out, rep);
}

}  // namespace
}  // namespace lc

using namespace lc;

extern "C" {

int lie_closure_pauli_dev(const unsigned long long* strings, const double* coefs, const long long* offsets, int k,
                          int n_qubits, double tol, unsigned long long* basis_strings, double* basis_coefs,
                          long long* basis_offsets, long long term_capacity, long long* dim_out, long long max_dim,
                          const lc_options* opt, lc_report* rep, void* stream) {
  if (dim_out) *dim_out = 0;
  lc_options o;
  lc_default_options(&o);
  if (opt) o = *opt;
  int rc = check_pauli_args(strings, coefs, offsets, k, n_qubits, tol, term_capacity, max_dim, o);
  if (rc != LC_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<long long> h_off((size_t)k + 1);
  if (cudaMemcpyAsync(h_off.data(), offsets, sizeof(long long) * (k + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return LC_ERR_CUDA;
  if (!offsets_ok(h_off.data(), k)) return LC_ERR_ARG;
  return closure_pauli_device(strings, coefs, offsets, h_off.data(), k, n_qubits, tol, basis_strings, basis_coefs,
                              basis_offsets, term_capacity, dim_out, max_dim, o, rep, s);
}

int lie_closure_pauli(const unsigned long long* strings, const double* coefs, const long long* offsets, int k,
                      int n_qubits, double tol, unsigned long long* basis_strings, double* basis_coefs,
                      long long* basis_offsets, long long term_capacity, long long* dim_out, long long max_dim,
                      const lc_options* opt, lc_report* rep) {
  if (dim_out) *dim_out = 0;
  lc_options o;
  lc_default_options(&o);
  if (opt) o = *opt;
  int rc = check_pauli_args(strings, coefs, offsets, k, n_qubits, tol, term_capacity, max_dim, o);
  if (rc != LC_OK) return rc;
  if (!offsets_ok(offsets, k)) return LC_ERR_ARG;
  const long long nt = offsets[k];
  const bool out = basis_strings && basis_coefs && basis_offsets;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return LC_ERR_CUDA;
  u64 *dk = nullptr, *ok = nullptr;
  double *dv = nullptr, *ov = nullptr;
  long long *doff = nullptr, *ooff = nullptr;
  auto alloc = [&](void** p, size_t bytes) {
    if (rc == LC_OK && cudaMallocAsync(p, std::max<size_t>(bytes, 16), s) != cudaSuccess) rc = LC_ERR_OOM;
  };
  alloc(reinterpret_cast<void**>(&dk), sizeof(u64) * nt);
  alloc(reinterpret_cast<void**>(&dv), sizeof(double) * nt);
  alloc(reinterpret_cast<void**>(&doff), sizeof(long long) * (k + 1));
  if (out) {
    alloc(reinterpret_cast<void**>(&ok), sizeof(u64) * term_capacity);
    alloc(reinterpret_cast<void**>(&ov), sizeof(double) * term_capacity);
    alloc(reinterpret_cast<void**>(&ooff), sizeof(long long) * (max_dim + 1));
  }
  if (rc == LC_OK && nt > 0 &&
      (cudaMemcpyAsync(dk, strings, sizeof(u64) * nt, cudaMemcpyHostToDevice, s) != cudaSuccess ||
       cudaMemcpyAsync(dv, coefs, sizeof(double) * nt, cudaMemcpyHostToDevice, s) != cudaSuccess))
    rc = LC_ERR_CUDA;
  if (rc == LC_OK &&
      cudaMemcpyAsync(doff, offsets, sizeof(long long) * (k + 1), cudaMemcpyHostToDevice, s) != cudaSuccess)
    rc = LC_ERR_CUDA;
  long long dim = 0;
  if (rc == LC_OK)
    rc = closure_pauli_device(dk, dv, doff, offsets, k, n_qubits, tol, ok, ov, ooff, term_capacity, &dim, max_dim, o,
                              rep, s);
  if (out && (rc == LC_OK || rc == LC_ERR_CAPACITY)) {
    std::vector<long long> hoff((size_t)std::max<long long>(dim, 0) + 1, 0);
    if (dim > 0 && (cudaMemcpyAsync(hoff.data(), ooff, sizeof(long long) * (dim + 1), cudaMemcpyDeviceToHost, s) !=
                        cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess))
      rc = LC_ERR_CUDA;
    const long long nterm = hoff[(size_t)dim];
    memcpy(basis_offsets, hoff.data(), sizeof(long long) * (dim + 1));
    if (nterm > 0 && (cudaMemcpyAsync(basis_strings, ok, sizeof(u64) * nterm, cudaMemcpyDeviceToHost, s) !=
                          cudaSuccess ||
                      cudaMemcpyAsync(basis_coefs, ov, sizeof(double) * nterm, cudaMemcpyDeviceToHost, s) !=
                          cudaSuccess))
      rc = LC_ERR_CUDA;
  }
  for (void* p : {(void*)dk, (void*)dv, (void*)doff, (void*)ok, (void*)ov, (void*)ooff})
    if (p) cudaFreeAsync(p, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == LC_OK) rc = LC_ERR_CUDA;
  cudaStreamDestroy(s);
  if (dim_out) *dim_out = dim;
  return rc;
}

}  // extern "C"
