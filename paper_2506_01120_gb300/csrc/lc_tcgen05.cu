// Split-BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   D[M x N] = Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T      (FP32 accumulation in TMEM)
//
// where X = Xhi + Xlo is the two-term BF16 split of an FP32/FP64 operand
// (Markidis et al. 2018; Henry, Tang and Heinecke 2019).  The dropped
// Alo Blo^T term and the split remainders leave a relative error near 2^-16
// per product, which is what the screening step budgets for.
//
// Both operands are K-major BF16 in global memory.  Each CTA owns one
// 128 x BN output tile.  Warp 0 (one lane) streams the four operand tiles of
// each 64-wide k-slice into shared memory with TMA (128-byte swizzle); warp 1
// (one lane) issues the three tcgen05.mma per 16-wide k-step into a TMEM
// accumulator and frees each stage with tcgen05.commit; afterwards all four
// warps read their 32 TMEM lanes (rows) back with tcgen05.ld and run the
// epilogue.  Every mbarrier wait is bounded by a wall-clock limit; on expiry
// the kernel records LC_ERR_TIMEOUT, drains what it issued and returns.
#include "lc_internal.cuh"
#include "lc_digits.cuh"
#include "../../include/lieclosure_kernels.h"

#include <cuda.h>
#include <algorithm>
#include <cstring>
#include <mutex>

namespace lc {
namespace {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 64;                       // 64 BF16 = 128 bytes = one swizzle row
constexpr int STAGES = 3;
constexpr int TILE_A_BYTES = BM * BK * 2;    // 16 KB
constexpr int TILE_B_BYTES = BN * BK * 2;    // 16 KB
constexpr int STAGE_BYTES = 2 * TILE_A_BYTES + 2 * TILE_B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;   // + alignment slack
constexpr int TMEM_COLS = BN;                // FP32 accumulator columns
constexpr int NTHREADS = 128;
// Limit for the waits that only let already-issued copies and MMAs land before
// a CTA leaves (kept independent of the caller's progress-wait limit).
constexpr uint64_t kDrainNs = 2000000000ull;

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait: true on success, false once limit_ns has elapsed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0 && globaltimer_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand tile with 128-byte swizzle: rows of 128 bytes, 8-row groups
// 1024 bytes apart (stride byte offset), leading byte offset unused (1),
// descriptor version 1 (bits 46-47), swizzle mode 2 = 128B (bits 61-63).
__device__ __forceinline__ uint64_t make_sw128_desc(uint32_t saddr) {
  uint64_t desc = 0;
  desc |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  desc |= (uint64_t)1u << 16;                  // LBO (ignored for swizzled K-major)
  desc |= (uint64_t)(1024u >> 4) << 32;        // SBO
  desc |= (uint64_t)1u << 46;                  // version
  desc |= (uint64_t)2u << 61;                  // SWIZZLE_128B
  return desc;
}

// The same for rows of 64 bytes (32 BF16) with 64-byte swizzle: 8-row groups
// 512 bytes apart, layout type 4.
__device__ __forceinline__ uint64_t make_sw64_desc(uint32_t saddr) {
  uint64_t desc = 0;
  desc |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  desc |= (uint64_t)1u << 16;
  desc |= (uint64_t)(512u >> 4) << 32;
  desc |= (uint64_t)1u << 46;
  desc |= (uint64_t)4u << 61;                  // SWIZZLE_64B
  return desc;
}

template <int SWB>
__device__ __forceinline__ uint64_t make_sw_desc(uint32_t saddr) {
  static_assert(SWB == 64 || SWB == 128, "swizzle");
  return SWB == 128 ? make_sw128_desc(saddr) : make_sw64_desc(saddr);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and B
// BF16 (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22,
// M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t make_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld_32cols(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ void record_timeout(DevStatus* st, int where, long long info) {
  if (st && atomicCAS(&st->code, 0, (int)LC_ERR_TIMEOUT) == 0) {
    st->where = where;
    st->info = info;
  }
}

// Tile configuration of the screening GEMM: 128 x BN output tile, BK-wide
// k-slices (BK BF16 = one swizzle row of 2 BK bytes), ST pipeline stages.
template <int BN_, int BK_, int ST_>
struct GemmCfg {
  static constexpr int BN = BN_, BK = BK_, STAGES = ST_;
  static constexpr int SWB = 2 * BK_;                 // swizzle width in bytes
  static constexpr int TILE_A = BM * BK_ * 2, TILE_B = BN_ * BK_ * 2;
  static constexpr int STAGE = 2 * TILE_A + 2 * TILE_B;
  static constexpr int SMEM = ST_ * STAGE + 1024;
  static constexpr int TMEM_COLS = BN_;
};
// 128 x 256 tiles with 32-wide k-slices: 25 % fewer operand bytes per MMA
// flop than 128 x 128, and 4 x 48 KB stages in flight (the default).  The
// autotuner also tries 128 x 128 tiles with 64-wide slices in 3 stages and
// with 32-wide slices in 6 stages; all three fill 192 KB of shared memory.
using ScreenCfg = GemmCfg<256, 32, 4>;
using ScreenCfg1 = GemmCfg<128, 64, 3>;
using ScreenCfg2 = GemmCfg<128, 32, 6>;
constexpr int kNumScreenCfgs = 3;

struct GemmParams {
  int M, N, K;
  const int* Mdev;
  __nv_bfloat16 *Dhi, *Dlo;
  int ldd;
  const __nv_bfloat16 *Hhi, *Hlo;
  int ldh;
  float* rn2;
  float* Df32;
  int epilogue;
  uint64_t limit_ns;
  DevStatus* st;
  int ksplit, kchunk;     // K split into ksplit ranges of kchunk k-slices (epilogue 3)
  float* Wpart;           // epilogue 3: FP32 partial tile of split s at Wpart[s][row][col] (row stride N)
};

template <class G>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_split_gemm(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                 const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo,
                 const GemmParams p) {
  extern __shared__ uint8_t smem_raw[];
  constexpr int BN = G::BN, BK = G::BK, STAGES = G::STAGES;
  constexpr int TILE_A_BYTES = G::TILE_A, TILE_B_BYTES = G::TILE_B, STAGE_BYTES = G::STAGE;
  constexpr int TMEM_COLS = G::TMEM_COLS;
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // Grouped tile order: consecutive CTAs sweep all N tiles of a group of
  // GROUP_M row tiles, so one wave touches a few M tiles and a few N tiles
  // and both operands are reused from L2 instead of re-read from DRAM.
  constexpr int GROUP_M = 8;
  const int ntn = p.N / BN, ntm = p.M / BM;
  // split-K (epilogue 3): CTA blockIdx.x covers tile id of k-range split
  const int split = blockIdx.x / (ntn * ntm);
  const int id = blockIdx.x - split * (ntn * ntm);
  const int per_group = GROUP_M * ntn;
  const int g = id / per_group, first_m = g * GROUP_M;
  const int gm = min(GROUP_M, ntm - first_m);
  const int in_g = id - g * per_group;
  const int m0 = (first_m + in_g % gm) * BM, n0 = (in_g / gm) * BN;
  const int kt_begin = p.epilogue == 3 ? split * p.kchunk : 0;
  const int nk = p.epilogue == 3 ? min(p.kchunk, p.K / BK - kt_begin) : p.K / BK;
  if (p.Mdev && m0 >= *p.Mdev) return;      // whole CTA: rows past the live count
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- producer: TMA
    int issued = 0;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      if (!mbar_wait_bounded(&empty_bar[s], ph ^ 1u, p.limit_ns)) {
        record_timeout(p.st, SITE_GEMM_TMA_WAIT, kt);
        abort_flag = 1;
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      uint8_t* st = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full_bar[s], STAGE_BYTES);
      const int kx = (kt_begin + kt) * BK;
      tma_load_2d(st, &mAhi, &full_bar[s], kx, m0);
      tma_load_2d(st + TILE_A_BYTES, &mAlo, &full_bar[s], kx, m0);
      tma_load_2d(st + 2 * TILE_A_BYTES, &mBhi, &full_bar[s], kx, n0);
      tma_load_2d(st + 2 * TILE_A_BYTES + TILE_B_BYTES, &mBlo, &full_bar[s], kx, n0);
      issued = kt + 1;
    }
    // drain: wait (bounded) until every issued stage has landed, so no copy
    // is still writing shared memory when the CTA exits
    for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; ++kt) {
      const int s = kt % STAGES;
      mbar_wait_bounded(&full_bar[s], (uint32_t)(kt / STAGES) & 1u, kDrainNs);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = make_idesc_bf16(BM, BN);
    bool ok = true;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      if (!mbar_wait_bounded(&full_bar[s], ph, p.limit_ns)) {
        record_timeout(p.st, SITE_GEMM_MMA_WAIT, kt);
        abort_flag = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t a_hi = smem_u32(smem + s * STAGE_BYTES);
      const uint32_t a_lo = a_hi + TILE_A_BYTES;
      const uint32_t b_hi = a_hi + 2 * TILE_A_BYTES;
      const uint32_t b_lo = b_hi + TILE_B_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint32_t off = kk * 32;   // 16 BF16 along K inside the swizzled row
        const uint64_t dAh = make_sw_desc<G::SWB>(a_hi + off), dAl = make_sw_desc<G::SWB>(a_lo + off);
        const uint64_t dBh = make_sw_desc<G::SWB>(b_hi + off), dBl = make_sw_desc<G::SWB>(b_lo + off);
        mma_bf16(tmem, dAh, dBh, idesc, (kt | kk) ? 1u : 0u);
        mma_bf16(tmem, dAh, dBl, idesc, 1u);
        mma_bf16(tmem, dAl, dBh, idesc, 1u);
      }
      mma_commit(&empty_bar[s]);     // stage s is free once these MMAs retire
    }
    (void)ok;
    mma_commit(&done_bar);           // accumulator complete (or drained on abort)
  }
  __syncwarp();

  // ---------------- epilogue: all four warps
  const bool have = mbar_wait_bounded(&done_bar, 0u, p.limit_ns);
  if (!have) {
    record_timeout(p.st, SITE_GEMM_EPI_WAIT, blockIdx.x);
    atomicExch(&abort_flag, 1);
    mbar_wait_bounded(&done_bar, 0u, kDrainNs);      // issued MMAs retire before TMEM is freed
  }
  __syncthreads();                   // makes the run decision uniform across the CTA
  tc_fence_after();
  const bool run = !(*(volatile int*)&abort_flag);
  const int row = m0 + warp * 32 + lane;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  float acc2 = 0.0f;
  if (run) {
    for (int c = 0; c < BN; c += 32) {
      float v[32];
      tmem_ld_32cols(trow + (uint32_t)c, v);     // warp-collective
      if (row < p.M) {
        const int col = n0 + c;
        if (p.epilogue == 0) {
          __align__(16) __nv_bfloat16 hi[32], lo[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            hi[i] = __float2bfloat16_rn(v[i]);
            lo[i] = __float2bfloat16_rn(v[i] - __bfloat162float(hi[i]));
          }
          uint4* dh = reinterpret_cast<uint4*>(p.Dhi + (long long)row * p.ldd + col);
          uint4* dl = reinterpret_cast<uint4*>(p.Dlo + (long long)row * p.ldd + col);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            dh[i] = reinterpret_cast<const uint4*>(hi)[i];
            dl[i] = reinterpret_cast<const uint4*>(lo)[i];
          }
        } else if (p.epilogue == 1) {
          const uint4* hh = reinterpret_cast<const uint4*>(p.Hhi + (long long)row * p.ldh + col);
          const uint4* hl = reinterpret_cast<const uint4*>(p.Hlo + (long long)row * p.ldh + col);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint4 a = hh[i], b = hl[i];
            const __nv_bfloat16* ah = reinterpret_cast<const __nv_bfloat16*>(&a);
            const __nv_bfloat16* bl = reinterpret_cast<const __nv_bfloat16*>(&b);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const float r = (__bfloat162float(ah[e]) + __bfloat162float(bl[e])) - v[i * 8 + e];
              acc2 = fmaf(r, r, acc2);
            }
          }
        } else {
          float* base = p.epilogue == 3 ? p.Wpart + ((long long)split * p.M + row) * p.N + col
                                        : p.Df32 + (long long)row * p.ldd + col;
          float4* o = reinterpret_cast<float4*>(base);
#pragma unroll
          for (int i = 0; i < 8; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
      }
    }
    if (p.epilogue == 1 && row < p.M) atomicAdd(&p.rn2[row], acc2);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  });
  return fn;
}

// 2-D BF16 map: rows x cols (cols contiguous, row stride ld elements),
// box = box_rows x 64 with 128-byte swizzle.
bool make_map(CUtensorMap* m, const __nv_bfloat16* base, long long rows, long long cols, long long ld,
              int box_rows, int box_cols = BK) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle sw = box_cols == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  if (box_cols != 64 && box_cols != 32) return false;
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

bool tcgen05_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && get_encode() != nullptr;
}

namespace {
// Sum of the split-K partials in split order (deterministic), stored as the
// split BF16 pair of epilogue 0; rows of tiles the GEMM skipped (at or past
// the live count) are skipped here too.
__global__ void k_splitk_reduce_bf16(const float* __restrict__ W, int S, int M, int N, const int* __restrict__ Mdev,
                                     __nv_bfloat16* __restrict__ Dhi, __nv_bfloat16* __restrict__ Dlo, int ldd) {
  const int rows = Mdev ? min(M, (*Mdev + BM - 1) / BM * BM) : M;
  const long long tot = (long long)rows * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / N), c = (int)(e % N);
    float v = 0.f;
    for (int q = 0; q < S; ++q) v += W[((long long)q * M + r) * N + c];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    Dhi[(long long)r * ldd + c] = h;
    Dlo[(long long)r * ldd + c] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

template <class G>
cudaError_t split_gemm_cfg(const SplitGemmArgs& a, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0) return cudaSuccess;
  if (a.M % BM || a.N % G::BN || a.K % G::BK || a.K <= 0) return cudaErrorInvalidValue;
  if ((a.lda % 8) || (a.ldb % 8)) return cudaErrorInvalidValue;   // TMA: 16-byte row strides
  CUtensorMap mAhi, mAlo, mBhi, mBlo;
  if (!make_map(&mAhi, a.Ahi, a.M, a.K, a.lda, BM, G::BK) || !make_map(&mAlo, a.Alo, a.M, a.K, a.lda, BM, G::BK) ||
      !make_map(&mBhi, a.Bhi, a.N, a.K, a.ldb, G::BN, G::BK) || !make_map(&mBlo, a.Blo, a.N, a.K, a.ldb, G::BN, G::BK))
    return cudaErrorInvalidValue;
  const cudaError_t attr_err = smem_optin(reinterpret_cast<const void*>(k_split_gemm<G>), G::SMEM);
  if (attr_err != cudaSuccess) return attr_err;
  GemmParams p;
  p.M = a.M;
  p.N = a.N;
  p.K = a.K;
  p.Mdev = a.Mdev;
  p.Dhi = a.Dhi;
  p.Dlo = a.Dlo;
  p.ldd = a.ldd;
  p.Hhi = a.Hhi;
  p.Hlo = a.Hlo;
  p.ldh = a.ldh;
  p.rn2 = a.rn2;
  p.Df32 = a.Df32;
  p.epilogue = a.epilogue;
  p.limit_ns = a.spin_cap > 0 ? (uint64_t)a.spin_cap : 4000000000ull;
  p.st = a.st;
  p.ksplit = 1;
  p.kchunk = a.K / G::BK;
  p.Wpart = nullptr;
  const int ntiles = (a.N / G::BN) * (a.M / BM);
  // Split-K for the projection when its output has fewer tiles than there are
  // SMs (few basis rows, long rows: large d): every split keeps >= 4 k-slices
  // and all splits are non-empty; the partials are summed in order.
  const int nkt = a.K / G::BK, sms = device_sm_count();
  if (a.epilogue == 0 && a.ws && ntiles < sms && nkt >= 8) {
    int S = std::min((sms + ntiles - 1) / ntiles, nkt / 4);
    S = (int)std::min<long long>(S, (long long)(a.ws_floats / ((size_t)a.M * a.N)));
    if (S > 1) {
      const int kchunk = (nkt + S - 1) / S;
      S = (nkt + kchunk - 1) / kchunk;
      p.epilogue = 3;
      p.ksplit = S;
      p.kchunk = kchunk;
      p.Wpart = a.ws;
      k_split_gemm<G><<<ntiles * S, NTHREADS, G::SMEM, s>>>(mAhi, mAlo, mBhi, mBlo, p);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      const long long tot = (long long)a.M * a.N;
      const int grid = (int)std::min<long long>((tot + 255) / 256, (long long)sms * 8);
      k_splitk_reduce_bf16<<<grid, 256, 0, s>>>(a.ws, S, a.M, a.N, a.Mdev, a.Dhi, a.Dlo, a.ldd);
      if (a.launches) *a.launches += 2;
      return cudaGetLastError();
    }
  }
  k_split_gemm<G><<<ntiles, NTHREADS, G::SMEM, s>>>(mAhi, mAlo, mBhi, mBlo, p);
  if (a.launches) *a.launches += 1;
  return cudaGetLastError();
}
}  // namespace

cudaError_t split_gemm_tcgen05(const SplitGemmArgs& a, cudaStream_t s) {
  switch (a.cfg) {
    case 0: return split_gemm_cfg<ScreenCfg>(a, s);
    case 1: return split_gemm_cfg<ScreenCfg1>(a, s);
    case 2: return split_gemm_cfg<ScreenCfg2>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

int split_gemm_num_cfgs() { return kNumScreenCfgs; }
int split_gemm_tile_n() { return std::max(ScreenCfg::BN, std::max(ScreenCfg1::BN, ScreenCfg2::BN)); }
int split_gemm_tile_k() { return std::max(ScreenCfg::BK, std::max(ScreenCfg1::BK, ScreenCfg2::BK)); }
int split_gemm_tile_n(int cfg) { return cfg == 1 ? ScreenCfg1::BN : (cfg == 2 ? ScreenCfg2::BN : ScreenCfg::BN); }
int split_gemm_tile_k(int cfg) { return cfg == 1 ? ScreenCfg1::BK : (cfg == 2 ? ScreenCfg2::BK : ScreenCfg::BK); }

}  // namespace lc

// ------------------------------------------------ unit-level entry point
namespace lc {
namespace {

__global__ void k_split_pad_f32(const float* __restrict__ X, int rows, int cols, int rows_pad, int cols_pad,
                                __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const long long tot = (long long)rows_pad * cols_pad;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols_pad), c = (int)(e % cols_pad);
    const float x = (r < rows && c < cols) ? X[(long long)r * cols + c] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[e] = h;
    lo[e] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

__global__ void k_crop_f32(const float* __restrict__ Dp, int ldp, int M, int N, float* __restrict__ D) {
  const long long tot = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / N), c = (int)(e % N);
    D[e] = Dp[(long long)r * ldp + c];
  }
}

}  // namespace
}  // namespace lc

extern "C" LC_API int lc_split_gemm_f32(const float* A, const float* B, int M, int N, int K, float* D,
                                        void* stream) {
  using namespace lc;
  if (!A || !B || !D || M < 1 || N < 1 || K < 1) return LC_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!tcgen05_available()) return LC_ERR_CUDA;
  const int Mp = round_up(M, BM), Np = round_up(N, ScreenCfg::BN), Kp = round_up(K, ScreenCfg::BK);
  const size_t nA = (size_t)Mp * Kp, nB = (size_t)Np * Kp, nD = (size_t)Mp * Np;
  char* ws = nullptr;
  const size_t bytes = 4 * ((nA + nB) * 2 + 256) + nD * 4 + sizeof(DevStatus) + 1024;
  if (cudaMallocAsync(reinterpret_cast<void**>(&ws), bytes, s) != cudaSuccess) return LC_ERR_OOM;
  size_t off = 0;
  auto take = [&](size_t b) { char* p = ws + off; off = (off + b + 255) & ~size_t(255); return p; };
  __nv_bfloat16* Ahi = reinterpret_cast<__nv_bfloat16*>(take(nA * 2));
  __nv_bfloat16* Alo = reinterpret_cast<__nv_bfloat16*>(take(nA * 2));
  __nv_bfloat16* Bhi = reinterpret_cast<__nv_bfloat16*>(take(nB * 2));
  __nv_bfloat16* Blo = reinterpret_cast<__nv_bfloat16*>(take(nB * 2));
  float* Dp = reinterpret_cast<float*>(take(nD * 4));
  DevStatus* st = reinterpret_cast<DevStatus*>(take(sizeof(DevStatus)));
  int rc = LC_OK;
  DevStatus hst;
  memset(&hst, 0, sizeof(hst));
  if (cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess) rc = LC_ERR_CUDA;
  if (rc == LC_OK) {
    k_split_pad_f32<<<1024, 256, 0, s>>>(A, M, K, Mp, Kp, Ahi, Alo);
    k_split_pad_f32<<<1024, 256, 0, s>>>(B, N, K, Np, Kp, Bhi, Blo);
    SplitGemmArgs g;
    memset(&g, 0, sizeof(g));
    g.Ahi = Ahi; g.Alo = Alo; g.Bhi = Bhi; g.Blo = Blo;
    g.M = Mp; g.N = Np; g.K = Kp; g.lda = Kp; g.ldb = Kp;
    g.Df32 = Dp; g.ldd = Np; g.epilogue = 2; g.st = st;
    if (split_gemm_tcgen05(g, s) != cudaSuccess) rc = LC_ERR_CUDA;
  }
  if (rc == LC_OK) {
    k_crop_f32<<<1024, 256, 0, s>>>(Dp, Np, M, N, D);
    if (cudaGetLastError() != cudaSuccess) rc = LC_ERR_CUDA;
    cudaMemcpyAsync(&hst, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
  }
  cudaFreeAsync(ws, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == LC_OK) rc = LC_ERR_CUDA;
  if (rc == LC_OK && hst.code != 0) rc = hst.code;
  return rc;
}

// ------------------------------------------------------- tensor-core brackets
// One CTA per pair (l, m) of the block.  Each basis element v = iH is also
// stored as its real 2d x 2d embedding E = [[Hr, -Hi], [-Hi, -Hr]] (split BF16,
// row-major).  With A = H_l, B = H_m:
//   E_l[0:d] E_m^T = [Re AB | Im AB],   E_m[0:d] E_l^T = [Re BA | Im BA]
// (Hr symmetric, Hi antisymmetric), so one TMEM accumulator receives
// D = [Re(AB - BA) | Im(AB - BA)] from 2 x 3 split MMAs per 16-wide k-step, the
// second three with the negate-A bit of the instruction descriptor.  The
// bracket [V_l, V_m] = -(AB - BA) has Hermitian part i(AB - BA), whose packed
// row j is, from row j of D alone (AB - BA is anti-Hermitian, so Re is
// antisymmetric):
//   S[j][k] = -sqrt(2/d) Im D[j][k] (k > j),  -Im D[j][j]/sqrt(d) (k = j),
//             -sqrt(2/d) Re D[j][k] (k < j).
// The A operand is the first 128 rows of the same shared-memory tile (for
// d = 64 rows 64..127 of D are unused).
namespace lc {
namespace {

template <int D>
struct BrCfg {
  // MMA rows: the first D rows of E_l.  For D <= 64 the M = 64 shape is used
  // (for D = 32 its last 32 rows are not needed); its accumulator row i sits
  // in TMEM lane 32 (i / 16) + i % 16.
  static constexpr int MM = D <= 64 ? 64 : 128;
  static constexpr int R = 2 * D;              // rows of E = MMA N = K extent
  static constexpr int TILE = R * 64 * 2;       // one R x 64 BF16 tile
  static constexpr int STAGE = 4 * TILE;        // El hi/lo, Em hi/lo
  static constexpr int NK = R / 64;             // 64-wide k-chunks
  static constexpr int SMEM = STAGE + 1024;
  static constexpr int TMEM_COLS = R;
};

template <int D>
__global__ void __launch_bounds__(128, 1)
    k_bracket_tc(const __grid_constant__ CUtensorMap mEhi, const __grid_constant__ CUtensorMap mElo, long long t0,
                 __nv_bfloat16* __restrict__ Hhi, __nv_bfloat16* __restrict__ Hlo, int ldh, float* __restrict__ hn2,
                 uint64_t limit_ns, DevStatus* st) {
  using C = BrCfg<D>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar, empty_bar, done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ float red[4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = blockIdx.x;
  int l, m;
  pair_from_index(t0 + pair, &l, &m);
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  if (threadIdx.x == 0) {
    mbar_init(&full_bar, 1);
    mbar_init(&empty_bar, 1);
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int kc = 0; kc < C::NK; ++kc) {
      if (kc > 0 && !mbar_wait_bounded(&empty_bar, (uint32_t)(kc - 1) & 1u, limit_ns)) {
        record_timeout(st, SITE_GEMM_TMA_WAIT, kc);
        abort_flag = 1;
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      mbar_expect_tx(&full_bar, C::STAGE);
      const int x = kc * 64;
      tma_load_2d(smem, &mEhi, &full_bar, x, l * C::R);
      tma_load_2d(smem + C::TILE, &mElo, &full_bar, x, l * C::R);
      tma_load_2d(smem + 2 * C::TILE, &mEhi, &full_bar, x, m * C::R);
      tma_load_2d(smem + 3 * C::TILE, &mElo, &full_bar, x, m * C::R);
      issued = kc + 1;
    }
    if (issued > 0) mbar_wait_bounded(&full_bar, (uint32_t)(issued - 1) & 1u, kDrainNs);
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = make_idesc_bf16(C::MM, C::R);
    constexpr uint32_t idesc_neg = idesc | (1u << 13);      // negate A
    for (int kc = 0; kc < C::NK; ++kc) {
      if (!mbar_wait_bounded(&full_bar, (uint32_t)kc & 1u, limit_ns)) {
        record_timeout(st, SITE_GEMM_MMA_WAIT, kc);
        abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t lh = smem_u32(smem), ll = lh + C::TILE, mh = lh + 2 * C::TILE, ml = lh + 3 * C::TILE;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t off = kk * 32;
        const uint64_t dlh = make_sw128_desc(lh + off), dll = make_sw128_desc(ll + off);
        const uint64_t dmh = make_sw128_desc(mh + off), dml = make_sw128_desc(ml + off);
        mma_bf16(tmem, dlh, dmh, idesc, (kc | kk) ? 1u : 0u);
        mma_bf16(tmem, dlh, dml, idesc, 1u);
        mma_bf16(tmem, dll, dmh, idesc, 1u);
        mma_bf16(tmem, dmh, dlh, idesc_neg, 1u);
        mma_bf16(tmem, dmh, dll, idesc_neg, 1u);
        mma_bf16(tmem, dml, dlh, idesc_neg, 1u);
      }
      mma_commit(&empty_bar);
    }
    mma_commit(&done_bar);
  }
  __syncwarp();
  const bool have = mbar_wait_bounded(&done_bar, 0u, limit_ns);
  if (!have) {
    record_timeout(st, SITE_GEMM_EPI_WAIT, pair);
    atomicExch(&abort_flag, 1);
    mbar_wait_bounded(&done_bar, 0u, kDrainNs);
  }
  __syncthreads();
  tc_fence_after();
  const bool run = !(*(volatile int*)&abort_flag);
  // output row of this lane (M = 64: lanes 0-15 of each warp quarter)
  const int j = C::MM == 64 ? warp * 16 + (lane & 15) : warp * 32 + lane;
  const bool mine = (C::MM == 64 ? lane < 16 : true) && j < D;
  float ss = 0.f;
  if (run && (C::MM == 64 || warp * 32 < D)) {         // warp-uniform
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    const float s1 = rsqrtf((float)D), s2 = sqrtf(2.f / (float)D);
    __nv_bfloat16* oh = Hhi + (long long)pair * ldh + (long long)j * D;
    __nv_bfloat16* ol = Hlo + (long long)pair * ldh + (long long)j * D;
    for (int c = 0; c < D; c += 32) {
      float re[32], im[32];
      tmem_ld_32cols(trow + (uint32_t)c, re);
      tmem_ld_32cols(trow + (uint32_t)(D + c), im);
      if (!mine) continue;
      __align__(16) __nv_bfloat16 hi[32], lo[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int k = c + i;
        const float v = (k > j) ? -s2 * im[i] : ((k == j) ? -s1 * im[i] : -s2 * re[i]);
        ss = fmaf(v, v, ss);
        hi[i] = __float2bfloat16_rn(v);
        lo[i] = __float2bfloat16_rn(v - __bfloat162float(hi[i]));
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        reinterpret_cast<uint4*>(oh + c)[i] = reinterpret_cast<const uint4*>(hi)[i];
        reinterpret_cast<uint4*>(ol + c)[i] = reinterpret_cast<const uint4*>(lo)[i];
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if (lane == 0) red[warp] = ss;
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && run) hn2[pair] = red[0] + red[1] + red[2] + red[3];
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS) : "memory");
  }
}

template <int D>
cudaError_t launch_bracket_tc(const __nv_bfloat16* Ehi, const __nv_bfloat16* Elo, long long nrows_elems,
                              long long t0, int count, __nv_bfloat16* Hhi, __nv_bfloat16* Hlo, int ldh, float* hn2,
                              long long spin_cap, DevStatus* st, cudaStream_t s) {
  using C = BrCfg<D>;
  CUtensorMap mh, ml;
  if (!make_map(&mh, Ehi, nrows_elems * C::R, C::R, C::R, C::R) ||
      !make_map(&ml, Elo, nrows_elems * C::R, C::R, C::R, C::R))
    return cudaErrorInvalidValue;
  const cudaError_t attr_err = smem_optin(reinterpret_cast<const void*>(k_bracket_tc<D>), C::SMEM);
  if (attr_err != cudaSuccess) return attr_err;
  const uint64_t lim = spin_cap > 0 ? (uint64_t)spin_cap : 4000000000ull;
  k_bracket_tc<D><<<count, 128, C::SMEM, s>>>(mh, ml, t0, Hhi, Hlo, ldh, hn2, lim, st);
  return cudaGetLastError();
}

}  // namespace

bool bracket_tc_supported(int d) { return d == 32 || d == 64 || d == 128; }

cudaError_t bracket_tc(const __nv_bfloat16* Ehi, const __nv_bfloat16* Elo, long long nelems, int d, long long t0,
                       int count, __nv_bfloat16* Hhi, __nv_bfloat16* Hlo, int ldh, float* hn2, long long spin_cap,
                       DevStatus* st, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (d == 32) return launch_bracket_tc<32>(Ehi, Elo, nelems, t0, count, Hhi, Hlo, ldh, hn2, spin_cap, st, s);
  if (d == 64) return launch_bracket_tc<64>(Ehi, Elo, nelems, t0, count, Hhi, Hlo, ldh, hn2, spin_cap, st, s);
  if (d == 128) return launch_bracket_tc<128>(Ehi, Elo, nelems, t0, count, Hhi, Hlo, ldh, hn2, spin_cap, st, s);
  return cudaErrorInvalidValue;
}

}  // namespace lc

// ------------------------------------------- allocation-free GEMM entry point
// Some callers cannot let a library allocate device memory: a serving process
// that hands all free device memory to its own pool at start-up, code running
// under a hard memory cap, or a latency-critical path where cudaMalloc/cudaFree
// (which can synchronise the whole device) must not appear.  For them,
// lc_split_gemm_f32_noalloc runs the same split + tcgen05 GEMM + crop kernels
// as lc_split_gemm_f32, but its workspace is this fixed file-scope device
// array instead of a per-call allocation.  The array exists on every GPU that
// loads the library and stays there until the process exits.
namespace lc {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device with that
// device current.  (In host code the symbol itself is only a host-side
// stand-in; kernels must be given this address.)
cudaError_t noalloc_scratch_address(void** out) {
  static std::mutex mu;
  static void* addr[128] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = p;
  }
  *out = addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace lc

extern "C" LC_API int lc_split_gemm_f32_noalloc(const float* A, const float* B, int M, int N, int K, float* D,
                                                void* stream) {
  using namespace lc;
  if (!A || !B || !D || M < 1 || N < 1 || K < 1) return LC_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Every padded extent is at least one tile, and the output alone takes
  // 4 Mp Np bytes, so no extent above the array size in elements can fit;
  // rejecting those first keeps the sizing arithmetic below far from overflow.
  const long long lim = (long long)(kNoAllocScratchBytes / 4);
  if ((long long)M > lim || (long long)N > lim || (long long)K > lim) return LC_ERR_TOO_LARGE;
  const unsigned long long Mp = (unsigned long long)round_up_ll(M, BM),
                           Np = (unsigned long long)round_up_ll(N, ScreenCfg::BN),
                           Kp = (unsigned long long)round_up_ll(K, ScreenCfg::BK);
  // layout inside the scratch array, every region 256-byte aligned; each
  // region is checked against the remaining room before it is added
  unsigned long long off = 0;
  bool fits = true;
  auto place = [&](unsigned long long bytes) {
    const unsigned long long at = off;
    if (!fits || bytes > kNoAllocScratchBytes - off) {
      fits = false;
      return at;
    }
    off = (off + bytes + 255) & ~255ull;
    if (off > kNoAllocScratchBytes) fits = false;
    return at;
  };
  // the products below are at most lim^2 * 4 < 2^62: no wrap
  const unsigned long long oAhi = place(Mp * Kp * 2), oAlo = place(Mp * Kp * 2);
  const unsigned long long oBhi = place(Np * Kp * 2), oBlo = place(Np * Kp * 2);
  const unsigned long long oD = place(Mp * Np * 4), oSt = place(sizeof(DevStatus));
  if (!fits) return LC_ERR_TOO_LARGE;
  if (!tcgen05_available()) return LC_ERR_CUDA;
  void* base = nullptr;
  if (noalloc_scratch_address(&base) != cudaSuccess) return LC_ERR_CUDA;
  char* ws = static_cast<char*>(base);
  __nv_bfloat16* Ahi = reinterpret_cast<__nv_bfloat16*>(ws + oAhi);
  __nv_bfloat16* Alo = reinterpret_cast<__nv_bfloat16*>(ws + oAlo);
  __nv_bfloat16* Bhi = reinterpret_cast<__nv_bfloat16*>(ws + oBhi);
  __nv_bfloat16* Blo = reinterpret_cast<__nv_bfloat16*>(ws + oBlo);
  float* Dp = reinterpret_cast<float*>(ws + oD);
  DevStatus* st = reinterpret_cast<DevStatus*>(ws + oSt);
  int rc = LC_OK;
  // the status word keeps the previous call's value: clear it.  The split
  // buffers (padding included) and Dp are fully rewritten below.
  if (cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess) rc = LC_ERR_CUDA;
  if (rc == LC_OK) {
    k_split_pad_f32<<<1024, 256, 0, s>>>(A, M, K, (int)Mp, (int)Kp, Ahi, Alo);
    k_split_pad_f32<<<1024, 256, 0, s>>>(B, N, K, (int)Np, (int)Kp, Bhi, Blo);
    SplitGemmArgs g;
    memset(&g, 0, sizeof(g));
    g.Ahi = Ahi; g.Alo = Alo; g.Bhi = Bhi; g.Blo = Blo;
    g.M = (int)Mp; g.N = (int)Np; g.K = (int)Kp; g.lda = (int)Kp; g.ldb = (int)Kp;
    g.Df32 = Dp; g.ldd = (int)Np; g.epilogue = 2; g.st = st;
    if (split_gemm_tcgen05(g, s) != cudaSuccess) rc = LC_ERR_CUDA;
  }
  DevStatus hst;
  memset(&hst, 0, sizeof(hst));
  if (rc == LC_OK) {
    k_crop_f32<<<1024, 256, 0, s>>>(Dp, (int)Np, M, N, D);
    if (cudaGetLastError() != cudaSuccess) rc = LC_ERR_CUDA;
    else if (cudaMemcpyAsync(&hst, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = LC_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == LC_OK) rc = LC_ERR_CUDA;
  if (rc == LC_OK && hst.code != 0) rc = hst.code;
  return rc;
}

// ------------------------------------------- d = 64 brackets from [Hr; Hi]
// Each basis element is also stored as Q = [Hr; Hi] (2d x d rows, split
// BF16).  For a pair (l, m) with A = H_l and B = H_m the kernel forms one
// complex product D = B A on the tensor cores and takes the bracket from D and
// its conjugate transpose: A and B are Hermitian, so (B A)^dagger = A B and
// [V_l, V_m] = [iA, iB] = -(AB - BA) = D - D^dagger.  With the tcgen05 product
// MMA(X, Y) = X Y^T and Hr^T = Hr, Hi^T = -Hi:
//   Re D = MMA(Br, Ar) + MMA(Bi, Ai),   Im D = -MMA(Br, Ai) + MMA(Bi, Ar),
// four N = 64 products into one 128-column accumulator [Re D | Im D] (the
// minus sign by the instruction's negate-A bit).  Two pairs (l, m), (l, m + 1)
// share A: their B operands fill the 128 rows of X, the full M = 128 shape.
// Persistent CTAs: CTA c takes a contiguous share of the block's pairs in
// pair order, so consecutive units mostly keep l and A's tiles (Ar, Ai, split
// hi/lo, 32 KB) stay in shared memory; a new l reloads them.  Warp 0 streams A
// and B with TMA (B through a two-stage ring, so the next unit's operands load
// during this unit's MMAs); warp 1 issues a unit's 48 MMAs into one of two
// TMEM accumulators; warps 2-9 drain an accumulator: each thread holds half of
// one accumulator row (its Re and Im columns) in registers, writes it
// transposed into a swizzled shared tile T, and after a barrier reads column j
// of D from T as 16-byte rows to write half of packed row j of the bracket:
//   S[j][k] = s2 (Im D[j][k] + Im D[k][j])   (k > j)
//   S[j][j] = s1 2 Im D[j][j]
//   S[j][k] = s2 (Re D[j][k] - Re D[k][j])   (k < j)
// with s1 = 1/sqrt(d), s2 = sqrt(2/d).  Every wait is bounded; a wait that
// runs out (or sees another role's abort) records LC_ERR_TIMEOUT, the roles
// leave their loops together, issued copies and MMAs are drained, and TMEM is
// released.
namespace lc {
namespace {

constexpr int Q_D = 64;
constexpr int QP_BOX = 64 * 64 * 2;       // one 64-row x 64-column BF16 tile (8 KB): one TMA box
constexpr int QP_Y = 4 * QP_BOX;          // Ar hi, Ar lo, Ai hi, Ai lo
constexpr int QP_XT = 2 * QP_BOX;         // one 128-row X tile (two pairs' 64-row boxes)
constexpr int QP_X = 4 * QP_XT;           // one X stage: Br hi, Br lo, Bi hi, Bi lo
constexpr int QP_XSTAGES = 2;
// T holds both pairs' D transposed: row 64 p + c is column c of D_p (Re D_p[k][c]
// at column k, Im at 64 + k), 4-float groups XOR-swizzled by (row % 8) so that
// column-wise scalar writes and row-wise 16-byte reads are both conflict-free
constexpr int QP_T = 128 * 128 * 4;
constexpr int QP_SMEM = QP_Y + QP_XSTAGES * QP_X + QP_T + 1024;
constexpr int QP_TMEM = 256;              // two 128-column accumulators
constexpr int QP_EPI_WARPS = 8;
constexpr int QP_THREADS = 64 + 32 * QP_EPI_WARPS;

// Bounded wait that also gives up as soon as another role has aborted.
__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, uint64_t limit_ns,
                                              volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0 && (*abort_flag || globaltimer_ns() - t0 > limit_ns)) return false;
  }
}

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Units of one or two pairs sharing l, walked identically by every role.
struct UnitWalk {
  long long t, tend;
  int l, m;
  __device__ void start(long long t_begin, long long t_end) {
    t = t_begin;
    tend = t_end;
    pair_from_index(t, &l, &m);
  }
  __device__ bool more() const { return t < tend; }
  __device__ int size() const { return (t + 1 < tend && m + 1 < l) ? 2 : 1; }
  __device__ void next(int n) {
    t += n;
    m += n;
    if (m >= l) {
      ++l;
      m = 0;
    }
  }
};

__global__ void __launch_bounds__(QP_THREADS, 1)
    k_bracket_q64(const __grid_constant__ CUtensorMap mQhi, const __grid_constant__ CUtensorMap mQlo, long long t0,
                  int count, __nv_bfloat16* __restrict__ Hhi, __nv_bfloat16* __restrict__ Hlo, int ldh,
                  float* __restrict__ hn2, uint64_t limit_ns, DevStatus* st) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t x_full[QP_XSTAGES], x_empty[QP_XSTAGES], y_full, done_bar;
  __shared__ __align__(8) uint64_t t_full[2], t_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag, epi_abort;
  const long long p0 = (long long)count * blockIdx.x / gridDim.x;
  const long long p1 = (long long)count * (blockIdx.x + 1) / gridDim.x;
  if (p0 >= p1) return;                                   // whole CTA: no pairs
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* Y = smem;                                        // Ar hi, Ar lo, Ai hi, Ai lo
  uint8_t* X = smem + QP_Y;                                 // stage s at X + s * QP_X
  float* T = reinterpret_cast<float*>(smem + QP_Y + QP_XSTAGES * QP_X);
  if (threadIdx.x == 0) {
    for (int q = 0; q < QP_XSTAGES; ++q) {
      mbar_init(&x_full[q], 1);
      mbar_init(&x_empty[q], 1);
    }
    mbar_init(&y_full, 1);
    mbar_init(&done_bar, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&t_full[b], 1);
      mbar_init(&t_empty[b], 1);
    }
    abort_flag = 0;
    epi_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(QP_TMEM)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int* ab = &abort_flag;
  const long long tb = t0 + p0, te = t0 + p1;

  if (warp == 0) {
    // ---------------- producer (lane 0): A's tiles per new l, B's per unit
    if (lane == 0) {
      UnitWalk w;
      w.start(tb, te);
      int cur_l = -1, ny = 0, nx = 0;
      while (w.more()) {
        const int n = w.size();
        const int xs = nx % QP_XSTAGES;
        // stage xs is free once the MMAs of unit nx - QP_XSTAGES retired
        if (nx >= QP_XSTAGES &&
            !wait_or_abort(&x_empty[xs], (uint32_t)(nx / QP_XSTAGES - 1) & 1u, limit_ns, ab)) {
          record_timeout(st, SITE_GEMM_TMA_WAIT, nx);
          *ab = 1;
          break;
        }
        if (w.l != cur_l) {
          // A's tiles may be replaced once every MMA reading them (up to unit nx - 1) retired
          if (nx > 0 && !wait_or_abort(&x_empty[(nx - 1) % QP_XSTAGES], (uint32_t)((nx - 1) / QP_XSTAGES) & 1u,
                                       limit_ns, ab)) {
            record_timeout(st, SITE_GEMM_TMA_WAIT, -nx);
            *ab = 1;
            break;
          }
          const int ra = w.l * 2 * Q_D, ri = ra + Q_D;
          mbar_expect_tx(&y_full, QP_Y);
          tma_load_2d(Y + 0 * QP_BOX, &mQhi, &y_full, 0, ra);
          tma_load_2d(Y + 1 * QP_BOX, &mQlo, &y_full, 0, ra);
          tma_load_2d(Y + 2 * QP_BOX, &mQhi, &y_full, 0, ri);
          tma_load_2d(Y + 3 * QP_BOX, &mQlo, &y_full, 0, ri);
          ++ny;
          cur_l = w.l;
        }
        uint8_t* Xs = X + xs * QP_X;
        mbar_expect_tx(&x_full[xs], n * 4 * QP_BOX);
        for (int q = 0; q < n; ++q) {
          const int rr = (w.m + q) * 2 * Q_D, rI = rr + Q_D;
          tma_load_2d(Xs + 0 * QP_XT + q * QP_BOX, &mQhi, &x_full[xs], 0, rr);
          tma_load_2d(Xs + 1 * QP_XT + q * QP_BOX, &mQlo, &x_full[xs], 0, rr);
          tma_load_2d(Xs + 2 * QP_XT + q * QP_BOX, &mQhi, &x_full[xs], 0, rI);
          tma_load_2d(Xs + 3 * QP_XT + q * QP_BOX, &mQlo, &x_full[xs], 0, rI);
        }
        ++nx;
        w.next(n);
      }
      // drain: no copy may still be writing shared memory when the CTA leaves
      for (int k = (nx > QP_XSTAGES ? nx - QP_XSTAGES : 0); k < nx; ++k)
        mbar_wait_bounded(&x_full[k % QP_XSTAGES], (uint32_t)(k / QP_XSTAGES) & 1u, kDrainNs);
      if (ny > 0) mbar_wait_bounded(&y_full, (uint32_t)(ny - 1) & 1u, kDrainNs);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (lane 0)
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc_bf16(128, 64);
      constexpr uint32_t idesc_neg = idesc | (1u << 13);        // negate A
      UnitWalk w;
      w.start(tb, te);
      int cur_l = -1, ny = 0, u = 0;
      while (w.more()) {
        const int n = w.size();
        const int b = u & 1;
        const int xs = u % QP_XSTAGES;
        bool ok = wait_or_abort(&x_full[xs], (uint32_t)(u / QP_XSTAGES) & 1u, limit_ns, ab);
        if (ok && w.l != cur_l) {
          ok = wait_or_abort(&y_full, (uint32_t)ny & 1u, limit_ns, ab);
          ++ny;
          cur_l = w.l;
        }
        if (ok && u >= 2) ok = wait_or_abort(&t_empty[b], (uint32_t)((u >> 1) - 1) & 1u, limit_ns, ab);
        if (!ok) {
          record_timeout(st, SITE_GEMM_MMA_WAIT, u);
          *ab = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * 128);
        const uint32_t xb = smem_u32(X + xs * QP_X), yb = smem_u32(Y);
        // (X tile, Y tile, accumulator column offset, negate): the four N = 64 products
        const uint32_t XT[4] = {xb, xb, xb + 2 * QP_XT, xb + 2 * QP_XT};            // Br, Br, Bi, Bi (hi)
        const uint32_t YT[4] = {yb, yb + 2 * QP_BOX, yb + 2 * QP_BOX, yb};          // Ar, Ai, Ai, Ar (hi)
        const uint32_t CO[4] = {0, 64, 0, 64};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const uint32_t dsc = (t == 1) ? idesc_neg : idesc;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t off = kk * 32;
            const uint64_t xh = make_sw128_desc(XT[t] + off), xl = make_sw128_desc(XT[t] + QP_XT + off);
            const uint64_t yh = make_sw128_desc(YT[t] + off), yl = make_sw128_desc(YT[t] + QP_BOX + off);
            mma_bf16(d + CO[t], xh, yh, dsc, (t >= 2 || kk) ? 1u : 0u);   // t = 0, 1 start their columns
            mma_bf16(d + CO[t], xh, yl, dsc, 1u);
            mma_bf16(d + CO[t], xl, yh, dsc, 1u);
          }
        }
        mma_commit(&x_empty[xs]);    // X stage xs (and A's tiles) may be overwritten once these retire
        mma_commit(&t_full[b]);      // accumulator b complete
        ++u;
        w.next(n);
      }
      mma_commit(&done_bar);         // every issued MMA has retired when this arrives
    }
  } else {
    // ---------------- epilogue: warps 2-9.  Warp w reads TMEM lane quarter
    // q = w % 4 (rows r = 32 q + lane: pair r / 64, row j = r % 64) and column
    // half h = (w - 2) / 4: Re D[j][32h .. 32h+31] and Im D[j][same].
    const int q = warp & 3, h = (warp - 2) >> 2;
    const int r = q * 32 + lane;
    const int p = r >> 6, j = r & 63;
    const int nthr = 32 * QP_EPI_WARPS;
    const float s1 = rsqrtf((float)Q_D), s2 = sqrtf(2.f / (float)Q_D);
    UnitWalk w;
    w.start(tb, te);
    int u = 0;
    while (w.more()) {
      const int n = w.size();
      const int b = u & 1;
      if (!wait_or_abort(&t_full[b], (uint32_t)(u >> 1) & 1u, limit_ns, ab)) epi_abort = 1;
      named_bar_sync(1, nthr);
      if (*(volatile int*)&epi_abort) break;     // uniform: only written before this barrier
      tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 128 + 32 * h);
      float re[32], im[32];
      tmem_ld_32cols(taddr, re);
      tmem_ld_32cols(taddr + 64u, im);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int row = p * 64 + 32 * h + i;                 // column 32h + i of D_p
        const int sw = (row & 7) << 2;
        T[row * 128 + (j ^ sw)] = re[i];
        T[row * 128 + ((Q_D + j) ^ sw)] = im[i];
      }
      tc_fence_before();
      named_bar_sync(1, nthr);                   // T complete; accumulator b free
      if (threadIdx.x == 64) mbar_arrive(&t_empty[b]);
      if (p < n) {
        const long long pidx = w.t + p - t0;     // position of the pair in the block
        const int row = p * 64 + j;              // column j of D_p
        const int sw = (row & 7) << 2;
        const float* Tj = T + row * 128;
        __align__(16) __nv_bfloat162 hi[16], lo[16];
        float ss = 0.f;
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          const int k0 = 32 * h + 4 * g;
          const float4 rc = *reinterpret_cast<const float4*>(Tj + (k0 ^ sw));          // Re D[k0 ..][j]
          const float4 ic = *reinterpret_cast<const float4*>(Tj + ((Q_D + k0) ^ sw));  // Im D[k0 ..][j]
          const float rk[4] = {rc.x, rc.y, rc.z, rc.w}, ik[4] = {ic.x, ic.y, ic.z, ic.w};
          float v[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int i = 4 * g + e, k = k0 + e;
            v[e] = (k > j) ? s2 * (im[i] + ik[e]) : ((k == j) ? s1 * (im[i] + ik[e]) : s2 * (re[i] - rk[e]));
            ss = fmaf(v[e], v[e], ss);
          }
#pragma unroll
          for (int e = 0; e < 4; e += 2) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[e], v[e + 1]);
            const float2 hf = __bfloat1622float2(h2);
            hi[2 * g + e / 2] = h2;
            lo[2 * g + e / 2] = __floats2bfloat162_rn(v[e] - hf.x, v[e + 1] - hf.y);
          }
        }
        __nv_bfloat16* oh = Hhi + pidx * ldh + (long long)j * Q_D + 32 * h;
        __nv_bfloat16* ol = Hlo + pidx * ldh + (long long)j * Q_D + 32 * h;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          reinterpret_cast<uint4*>(oh)[i] = reinterpret_cast<const uint4*>(hi)[i];
          reinterpret_cast<uint4*>(ol)[i] = reinterpret_cast<const uint4*>(lo)[i];
        }
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) atomicAdd(&hn2[pidx], ss);
      }
      named_bar_sync(1, nthr);                   // T may be overwritten by the next unit
      ++u;
      w.next(n);
    }
    if (*(volatile int*)&epi_abort) {
      if (threadIdx.x == 64) record_timeout(st, SITE_GEMM_EPI_WAIT, u);
      *ab = 1;
    }
  }
  // ---------------- teardown: every issued MMA retired before TMEM is released
  __syncwarp();
  if (!mbar_wait_bounded(&done_bar, 0u, limit_ns)) {
    record_timeout(st, SITE_GEMM_EPI_WAIT, -1);
    mbar_wait_bounded(&done_bar, 0u, kDrainNs);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(QP_TMEM) : "memory");
  }
}

}  // namespace

cudaError_t bracket_q64(const __nv_bfloat16* Qhi, const __nv_bfloat16* Qlo, long long nelems, long long t0, int count,
                        __nv_bfloat16* Hhi, __nv_bfloat16* Hlo, int ldh, float* hn2, long long spin_cap,
                        DevStatus* st, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  CUtensorMap mh, ml;
  if (!make_map(&mh, Qhi, nelems * 2 * Q_D, Q_D, Q_D, Q_D) || !make_map(&ml, Qlo, nelems * 2 * Q_D, Q_D, Q_D, Q_D))
    return cudaErrorInvalidValue;
  const cudaError_t attr_err = smem_optin(reinterpret_cast<const void*>(k_bracket_q64), QP_SMEM);
  if (attr_err != cudaSuccess) return attr_err;
  cudaError_t e = cudaMemsetAsync(hn2, 0, sizeof(float) * count, s);
  if (e != cudaSuccess) return e;
  const uint64_t lim = spin_cap > 0 ? (uint64_t)spin_cap : 4000000000ull;
  // one CTA per SM, each with a contiguous share of at least one unit
  const int G = std::max(1, std::min(device_sm_count(), (count + 1) / 2));
  k_bracket_q64<<<G, QP_THREADS, QP_SMEM, s>>>(mh, ml, t0, count, Hhi, Hlo, ldh, hn2, lim, st);
  return cudaGetLastError();
}

}  // namespace lc

// --------------------------------------------------- large-d tensor brackets
// For d >= 256 (d % 128 == 0) a bracket is a d x 2d x 2d real GEMM per term.
// The embedding is stored with its rows permuted in groups of 64:
//   E'[128c + w] = E[64c + w] (w < 64),  E'[128c + 64 + w] = E[d + 64c + w],
// so the 128-row N tile c of E' produces [Re | Im] of output columns
// 64c .. 64c+63, and the A operand (the first d rows of E) is E' rows
// 128c .. 128c+63 for c = 0 .. d/64-1 (two 64-row boxes per 128-row M tile).
// One CTA per (pair, M tile, N tile): K runs over 2d columns twice, first
// E_l[top] E'_m^T, then -E_m[top] E'_l^T, into one TMEM accumulator; the
// epilogue writes the packed slots of rows m0..m0+127, columns 64c..64c+63, as
// the small-d kernel does, and adds the row sums of squares to hn2[pair].
namespace lc {
namespace {

__global__ void __launch_bounds__(NTHREADS, 1)
    k_bracket_big(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                  const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo, int d,
                  long long t0, __nv_bfloat16* __restrict__ Hhi, __nv_bfloat16* __restrict__ Hlo, int ldh,
                  float* __restrict__ hn2, uint64_t limit_ns, DevStatus* st) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ float red[4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int R = 2 * d;
  const int ntm = d / BM, ntn = R / BN, tpp = ntm * ntn;
  const int pair = blockIdx.x / tpp, tile = blockIdx.x % tpp;
  const int tm = tile / ntn, tn = tile % ntn;
  int l, m;
  pair_from_index(t0 + pair, &l, &m);
  const int nkseg = R / BK, nk = 2 * nkseg;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      if (!mbar_wait_bounded(&empty_bar[s], ph ^ 1u, limit_ns)) {
        record_timeout(st, SITE_GEMM_TMA_WAIT, kt);
        abort_flag = 1;
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      const bool second = kt >= nkseg;
      const int a_elem = second ? m : l, b_elem = second ? l : m;
      const int kx = (kt % nkseg) * BK;
      uint8_t* sp = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full_bar[s], STAGE_BYTES);
      const int arow = a_elem * R + 256 * tm;           // two 64-row boxes: +0 and +128
      tma_load_2d(sp, &mAhi, &full_bar[s], kx, arow);
      tma_load_2d(sp + TILE_A_BYTES / 2, &mAhi, &full_bar[s], kx, arow + 128);
      tma_load_2d(sp + TILE_A_BYTES, &mAlo, &full_bar[s], kx, arow);
      tma_load_2d(sp + TILE_A_BYTES + TILE_A_BYTES / 2, &mAlo, &full_bar[s], kx, arow + 128);
      const int brow = b_elem * R + BN * tn;
      tma_load_2d(sp + 2 * TILE_A_BYTES, &mBhi, &full_bar[s], kx, brow);
      tma_load_2d(sp + 2 * TILE_A_BYTES + TILE_B_BYTES, &mBlo, &full_bar[s], kx, brow);
      issued = kt + 1;
    }
    for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; ++kt)
      mbar_wait_bounded(&full_bar[kt % STAGES], (uint32_t)(kt / STAGES) & 1u, kDrainNs);
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = make_idesc_bf16(BM, BN);
    constexpr uint32_t idesc_neg = idesc | (1u << 13);
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      if (!mbar_wait_bounded(&full_bar[s], ph, limit_ns)) {
        record_timeout(st, SITE_GEMM_MMA_WAIT, kt);
        abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t id = kt >= nkseg ? idesc_neg : idesc;
      const uint32_t a_hi = smem_u32(smem + s * STAGE_BYTES);
      const uint32_t a_lo = a_hi + TILE_A_BYTES;
      const uint32_t b_hi = a_hi + 2 * TILE_A_BYTES;
      const uint32_t b_lo = b_hi + TILE_B_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint32_t off = kk * 32;
        const uint64_t dAh = make_sw128_desc(a_hi + off), dAl = make_sw128_desc(a_lo + off);
        const uint64_t dBh = make_sw128_desc(b_hi + off), dBl = make_sw128_desc(b_lo + off);
        mma_bf16(tmem, dAh, dBh, id, (kt | kk) ? 1u : 0u);
        mma_bf16(tmem, dAh, dBl, id, 1u);
        mma_bf16(tmem, dAl, dBh, id, 1u);
      }
      mma_commit(&empty_bar[s]);
    }
    mma_commit(&done_bar);
  }
  __syncwarp();
  const bool have = mbar_wait_bounded(&done_bar, 0u, limit_ns);
  if (!have) {
    record_timeout(st, SITE_GEMM_EPI_WAIT, blockIdx.x);
    atomicExch(&abort_flag, 1);
    mbar_wait_bounded(&done_bar, 0u, kDrainNs);
  }
  __syncthreads();
  tc_fence_after();
  const bool run = !(*(volatile int*)&abort_flag);
  const int j = tm * BM + warp * 32 + lane;           // output row
  const int kbase = 64 * tn;                          // output columns kbase .. kbase+63
  float ss = 0.f;
  if (run) {
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    const float s1 = rsqrtf((float)d), s2 = sqrtf(2.f / (float)d);
    __nv_bfloat16* oh = Hhi + (long long)pair * ldh + (long long)j * d + kbase;
    __nv_bfloat16* ol = Hlo + (long long)pair * ldh + (long long)j * d + kbase;
    for (int c = 0; c < 64; c += 32) {
      float re[32], im[32];
      tmem_ld_32cols(trow + (uint32_t)c, re);
      tmem_ld_32cols(trow + (uint32_t)(64 + c), im);
      __align__(16) __nv_bfloat16 hi[32], lo[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int k = kbase + c + i;
        const float v = (k > j) ? -s2 * im[i] : ((k == j) ? -s1 * im[i] : -s2 * re[i]);
        ss = fmaf(v, v, ss);
        hi[i] = __float2bfloat16_rn(v);
        lo[i] = __float2bfloat16_rn(v - __bfloat162float(hi[i]));
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        reinterpret_cast<uint4*>(oh + c)[i] = reinterpret_cast<const uint4*>(hi)[i];
        reinterpret_cast<uint4*>(ol + c)[i] = reinterpret_cast<const uint4*>(lo)[i];
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if (lane == 0) red[warp] = ss;
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && run) atomicAdd(&hn2[pair], red[0] + red[1] + red[2] + red[3]);
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace

bool bracket_big_supported(int d) { return d >= 256 && d % 128 == 0; }

cudaError_t bracket_big(const __nv_bfloat16* Ehi, const __nv_bfloat16* Elo, long long nelems, int d, long long t0,
                        int count, __nv_bfloat16* Hhi, __nv_bfloat16* Hlo, int ldh, float* hn2, long long spin_cap,
                        DevStatus* st, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (!bracket_big_supported(d)) return cudaErrorInvalidValue;
  const long long R = 2LL * d;
  CUtensorMap ah, al, bh, bl;
  if (!make_map(&ah, Ehi, nelems * R, R, R, 64) || !make_map(&al, Elo, nelems * R, R, R, 64) ||
      !make_map(&bh, Ehi, nelems * R, R, R, BN) || !make_map(&bl, Elo, nelems * R, R, R, BN))
    return cudaErrorInvalidValue;
  const cudaError_t attr_err = smem_optin(reinterpret_cast<const void*>(k_bracket_big), SMEM_BYTES);
  if (attr_err != cudaSuccess) return attr_err;
  cudaError_t e = cudaMemsetAsync(hn2, 0, sizeof(float) * count, s);
  if (e != cudaSuccess) return e;
  const long long tpp = (long long)(d / BM) * (2 * d / BN);
  const uint64_t lim = spin_cap > 0 ? (uint64_t)spin_cap : 4000000000ull;
  k_bracket_big<<<(unsigned)(tpp * count), NTHREADS, SMEM_BYTES, s>>>(ah, al, bh, bl, d, t0, Hhi, Hlo, ldh, hn2, lim,
                                                                     st);
  return cudaGetLastError();
}

}  // namespace lc

// ------------------------------------------------ FP64-accurate GEMM on BF16 tensor cores
namespace lc {
namespace {

// C (M x N, FP64) = A (M x K) B^T (B stored N x K), both operands given as
// stacks of S slices (error-free splitting in the manner of Ozaki, Ogita,
// Oishi and Rump): row i of an operand is x_i = 2^{e_i} sum_s 2^{-beta (s+1)}
// d_s(i, .) with integer digits |d_s| <= 2^{beta-1}, each exact in BF16.
// A slice product T_st = sum_k dA_s(i, k) dB_t(j, k) is a sum of integers of
// magnitude <= 2^{2 beta - 2}; with K 2^{2 beta - 2} <= 2^24 every partial
// sum is an integer an FP32 accumulator holds exactly, so each tcgen05.mma
// chain over K yields T_st without rounding.  The CTA runs one such chain
// per pair (s, t) with s + t <= S - 1 (pairs of higher level lie below
// 2^{-beta S} of the row scales and are dropped), double-buffered in TMEM,
// and the epilogue warps add 2^{-beta (s + t + 2)} T_st into FP64 registers
// while the next chain runs; the row exponents 2^{e_i + e_j} are applied
// once at the end.
constexpr int OZ_BN = 128;
constexpr int OZ_BK = 64;                     // one 128-byte swizzle row of BF16
constexpr int OZ_TILE = 128 * OZ_BK * 2;      // 16 KB: 128 rows of A or of B
constexpr int OZ_STAGE = 2 * OZ_TILE;
constexpr int OZ_STAGES = 6;
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE + 1024;
constexpr int OZ_TMEM = 2 * OZ_BN;            // two 128-column FP32 accumulators
constexpr int OZ_EPI_WARPS = 8;
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;

struct OzParams {
  int M, N, K;
  int a_rows, b_rows;        // rows per slice in each stack (slice s starts at row s * rows)
  const int* eA;             // per-row exponents of A (nullptr: fA for every row)
  const int* eB;
  int fA, fB;
  int S, beta;
  // chains: a chain accumulates the pairs (s, l - s), s = s0 .. s0 + cnt - 1,
  // of one level l in one TMEM buffer (as many as keep the FP32 sums exact)
  int nchains;
  signed char ch_level[64], ch_s0[64], ch_cnt[64];
  int kchunk;                // k-slices of OZ_BK per K split
  int mode;                  // 0 store, 1 subtract from C, 2 partial to ws[split][row][col]
  double* C;
  int ldc;
  double* ws;
  const int* run_if;         // device flag: 0 = skip
  uint64_t limit_ns;
  DevStatus* st;
};


__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_ozaki_gemm(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB, const OzParams p) {
  if (p.run_if && *p.run_if == 0) return;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[OZ_STAGES], empty_bar[OZ_STAGES], t_full[2], t_empty[2], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntn = (p.N + OZ_BN - 1) / OZ_BN, ntm = (p.M + 127) / 128;
  const int split = blockIdx.x / (ntn * ntm);
  const int id = blockIdx.x - split * (ntn * ntm);
  constexpr int GROUP_M = 8;   // tile order as in k_split_gemm (operand reuse from L2)
  const int per_group = GROUP_M * ntn;
  const int g = id / per_group, first_m = g * GROUP_M;
  const int gm = min(GROUP_M, ntm - first_m);
  const int in_g = id - g * per_group;
  const int m0 = (first_m + in_g % gm) * 128, n0 = (in_g / gm) * OZ_BN;
  const int kt0 = split * p.kchunk;
  const int nk = min(p.kchunk, (p.K + OZ_BK - 1) / OZ_BK - kt0);   // >= 1: the host makes every split non-empty
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  if (threadIdx.x == 0) {
    for (int q = 0; q < OZ_STAGES; ++q) {
      mbar_init(&full_bar[q], 1);
      mbar_init(&empty_bar[q], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&t_full[b], 1);
      mbar_init(&t_empty[b], OZ_EPI_WARPS);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(OZ_TMEM)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  volatile int* ab = &abort_flag;

  if (warp == 0) {
    // ---------------- producer (lane 0): slice A_s and B_t tiles, pair by pair
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int q = 0; q < p.nchains && ok; ++q)
      for (int u = 0; u < p.ch_cnt[q] && ok; ++u) {
        const int s = p.ch_s0[q] + u, t = p.ch_level[q] - s;
        const int ya = s * p.a_rows + m0, yb = t * p.b_rows + n0;
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const int sg = it % OZ_STAGES;
          if (it >= OZ_STAGES &&
              !wait_or_abort(&empty_bar[sg], (uint32_t)(it / OZ_STAGES - 1) & 1u, p.limit_ns, ab)) {
            record_timeout(p.st, SITE_GEMM_TMA_WAIT, it);
            *ab = 1;
            ok = false;
            break;
          }
          uint8_t* sp = smem + sg * OZ_STAGE;
          mbar_expect_tx(&full_bar[sg], OZ_STAGE);
          const int kx = (kt0 + kt) * OZ_BK;
          tma_load_2d(sp, &mA, &full_bar[sg], kx, ya);
          tma_load_2d(sp + OZ_TILE, &mB, &full_bar[sg], kx, yb);
        }
      }
      // drain: no copy may still be writing shared memory when the CTA leaves
      for (int k = (it > OZ_STAGES ? it - OZ_STAGES : 0); k < it; ++k)
        mbar_wait_bounded(&full_bar[k % OZ_STAGES], (uint32_t)(k / OZ_STAGES) & 1u, kDrainNs);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (lane 0): one exact FP32 chain over K per pair
    if (lane == 0) {
      constexpr uint32_t idesc = make_idesc_bf16(128, OZ_BN);
      int it = 0;
      for (int q = 0; q < p.nchains; ++q) {
        const int b = q & 1;
        bool ok = true;
        if (q >= 2) ok = wait_or_abort(&t_empty[b], (uint32_t)((q >> 1) - 1) & 1u, p.limit_ns, ab);
        if (!ok) {
          record_timeout(p.st, SITE_GEMM_MMA_WAIT, -q);
          *ab = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * OZ_BN);
        for (int u = 0; u < p.ch_cnt[q] && ok; ++u)
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const int sg = it % OZ_STAGES;
          if (!wait_or_abort(&full_bar[sg], (uint32_t)(it / OZ_STAGES) & 1u, p.limit_ns, ab)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a = smem_u32(smem + sg * OZ_STAGE), bb = a + OZ_TILE;
#pragma unroll
          for (int kk = 0; kk < OZ_BK / 16; ++kk)
            mma_bf16(d, make_sw128_desc(a + kk * 32), make_sw128_desc(bb + kk * 32), idesc,
                     (u | kt | kk) ? 1u : 0u);
          mma_commit(&empty_bar[sg]);
        }
        if (!ok) {
          record_timeout(p.st, SITE_GEMM_MMA_WAIT, it);
          *ab = 1;
          break;
        }
        mma_commit(&t_full[b]);
      }
      mma_commit(&done_bar);   // every issued MMA has retired when this arrives
    }
  } else {
    // ---------------- epilogue: warps 2-9.  Warp w reads TMEM lane quarter
    // w % 4 (tile rows 32 (w % 4) + lane) and column half (w - 2) / 4.
    const int qd = warp & 3, h = (warp - 2) >> 2;
    const int r = qd * 32 + lane;
    double acc[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) acc[i] = 0.0;
    bool ok = true;
    for (int q = 0; q < p.nchains; ++q) {
      const int b = q & 1;
      ok = __all_sync(0xffffffffu, wait_or_abort(&t_full[b], (uint32_t)(q >> 1) & 1u, p.limit_ns, ab) ? 1 : 0);
      if (!ok) break;
      tc_fence_after();
      const double w = __longlong_as_double((long long)(1023 - p.beta * (p.ch_level[q] + 2)) << 52);
      const uint32_t taddr = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(b * OZ_BN + 64 * h);
      float v[32];
      tmem_ld_32cols(taddr, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[i] = fma(w, (double)v[i], acc[i]);
      tmem_ld_32cols(taddr + 32u, v);
#pragma unroll
      for (int i = 0; i < 32; ++i) acc[32 + i] = fma(w, (double)v[i], acc[32 + i]);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&t_empty[b]);   // accumulator b may be overwritten
    }
    if (!ok) {
      if (lane == 0) record_timeout(p.st, SITE_GEMM_EPI_WAIT, blockIdx.x);
      *ab = 1;
    } else {
      const int row = m0 + r;
      if (row < p.M) {
        const int ea = p.eA ? p.eA[row] : p.fA;
        const int cb = n0 + 64 * h;
#pragma unroll
        for (int i = 0; i < 64; ++i) {
          const int col = cb + i;
          if (col < p.N) {
            const int eb = p.eB ? p.eB[col] : p.fB;
            const double val = scalbn(acc[i], ea + eb);
            if (p.mode == 0)
              p.C[(long long)row * p.ldc + col] = val;
            else if (p.mode == 1)
              p.C[(long long)row * p.ldc + col] -= val;
            else
              p.ws[((long long)split * p.M + row) * p.N + col] = val;
          }
        }
      }
    }
  }
  // ---------------- teardown: every issued MMA retired before TMEM is released
  __syncwarp();
  if (!mbar_wait_bounded(&done_bar, 0u, p.limit_ns)) {
    record_timeout(p.st, SITE_GEMM_EPI_WAIT, -1);
    mbar_wait_bounded(&done_bar, 0u, kDrainNs);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM) : "memory");
  }
}

// Split-K partials summed in split order (deterministic), stored or
// subtracted.
__global__ void k_oz_reduce(int M, int N, int S, const double* __restrict__ ws, double* __restrict__ C, int ldc,
                            int subtract, const int* __restrict__ run_if) {
  if (run_if && *run_if == 0) return;
  const long long tot = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int z = 0; z < S; ++z) t += ws[(long long)z * tot + e];
    const long long o = (e / N) * ldc + (e % N);
    if (subtract) C[o] -= t;
    else C[o] = t;
  }
}

// One CTA of kOzSliceThreads per row of X (FP64): per-row exponent (or the
// fixed one when exps is null), then the digits into slices[s][row0 + r][c],
// two columns per thread (lds even); columns [cols, cols_pad) get zero digits.
constexpr int kOzSliceThreads = 128;

__global__ void __launch_bounds__(kOzSliceThreads)
    k_oz_slice_rows(const double* __restrict__ X, int rows, int cols, int cols_pad, int ldx, int S, int beta,
                    int fixed_e, __nv_bfloat16* __restrict__ out, int rows_alloc, int lds, int* __restrict__ exps,
                    int row0, const int* __restrict__ col_exp, const int* __restrict__ run_if) {
  if (run_if && *run_if == 0) return;
  __shared__ long long wmax[kOzSliceThreads / 32];
  const int r = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double* x = X + (long long)r * ldx;
  // column c of the row is sliced as x[c] 2^col_exp[c] when col_exp is given
  auto val = [&](int c) { return c < cols ? (col_exp ? scalbn(x[c], col_exp[c]) : x[c]) : 0.0; };
  int e = fixed_e;
  if (exps) {
    long long m = 0;
    for (int c = threadIdx.x; c < cols; c += blockDim.x)
      m = max(m, __double_as_longlong(val(c)) & 0x7FFFFFFFFFFFFFFFLL);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) wmax[w] = m;
    __syncthreads();
    m = wmax[0];
    for (int i = 1; i < kOzSliceThreads / 32; ++i) m = max(m, wmax[i]);
    e = oz_row_exp(m);
    if (threadIdx.x == 0) exps[row0 + r] = e;
  }
  const long long sstride2 = (long long)rows_alloc * lds / 2;
  __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(out + (long long)(row0 + r) * lds);
  const int ncol = max(cols, cols_pad);
  for (int c = 2 * threadIdx.x; c < ncol; c += 2 * blockDim.x) oz_digits2(val(c), val(c + 1), e, S, beta, o + c / 2, sstride2);
}

// Rows [r0, r1) of V (FP64) as columns j - jbase of the transposed slices
// outT[s][p][j - jbase], row j in units of its own exponent row_exp[j] (the
// product's other operand carries 2^row_exp[j] in its column j), through a
// 32 x 32 shared-memory tile.
__global__ void k_oz_slice_cols(const double* __restrict__ V, int r0, int r1, int P, int ldv, int S, int beta,
                                const int* __restrict__ row_exp, __nv_bfloat16* __restrict__ outT, int P_alloc,
                                int ldt, int jbase) {
  __shared__ double tile[32][33];
  const int j0 = r0 + blockIdx.y * 32, p0 = blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int j = j0 + k, pp = p0 + threadIdx.x;
    tile[k][threadIdx.x] = (j < r1 && pp < P) ? V[(long long)j * ldv + pp] : 0.0;
  }
  __syncthreads();
  const long long sstride = (long long)P_alloc * ldt;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int pp = p0 + k, j = j0 + threadIdx.x;
    if (pp < P && j < r1)
      oz_digits(tile[threadIdx.x][k], row_exp[j], S, beta, outT + (long long)pp * ldt + (j - jbase), sstride);
  }
}

}  // namespace

// columns the row slicer writes (pairs): max(cols, cols_pad) rounded up to even
static int ncol_even_check(int cols_pad, int cols) { return (std::max(cols, cols_pad) + 1) & ~1; }

int oz_beta_for(int K) {
  // largest beta <= 7 with K 2^{2 beta - 2} <= 2^24
  int lg = 0;
  while ((1LL << lg) < (long long)K) ++lg;
  const int b = (26 - lg) / 2;
  return std::max(1, std::min(7, b));
}

int oz_slices_for(int beta) { return (54 + beta - 1) / beta; }

long long oz_max_k(int beta) { return 1LL << (26 - 2 * beta); }

cudaError_t oz_slice_rows(const double* X, int rows, int cols, int ldx, int S, int beta, int fixed_e,
                          __nv_bfloat16* out, int rows_alloc, int lds, int* exps, int row0, const int* run_if,
                          cudaStream_t s, int cols_pad, const int* col_exp) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  cols_pad = std::max(cols, cols_pad);
  if (row0 < 0 || row0 + rows > rows_alloc || cols_pad > lds || beta < 1 || beta > 7) return cudaErrorInvalidValue;
  if ((lds & 1) || (ncol_even_check(cols_pad, cols) > lds)) return cudaErrorInvalidValue;
  k_oz_slice_rows<<<rows, kOzSliceThreads, 0, s>>>(X, rows, cols, cols_pad, ldx, S, beta, fixed_e, out, rows_alloc,
                                                   lds, exps, row0, col_exp, run_if);
  return cudaGetLastError();
}

cudaError_t oz_slice_cols(const double* V, int r0, int r1, int P, int ldv, int S, int beta, const int* row_exp,
                          __nv_bfloat16* outT, int P_alloc, int ldt, cudaStream_t s, int jbase) {
  if (r1 <= r0 || P <= 0) return cudaSuccess;
  if (P > P_alloc || jbase < 0 || jbase > r0 || r1 - jbase > ldt || beta < 1 || beta > 7)
    return cudaErrorInvalidValue;
  dim3 grid((unsigned)((P + 31) / 32), (unsigned)((r1 - r0 + 31) / 32));
  k_oz_slice_cols<<<grid, dim3(32, 8), 0, s>>>(V, r0, r1, P, ldv, S, beta, row_exp, outT, P_alloc, ldt, jbase);
  return cudaGetLastError();
}

cudaError_t ozaki_gemm_nt(int M, int N, int K, const OzOperand& A, const OzOperand& B, int S, int beta, double* C,
                          int ldc, bool subtract, double* ws, size_t ws_doubles, const int* run_if,
                          long long spin_cap, DevStatus* st, cudaStream_t s, long long* launches, int max_level) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  if (beta < 1 || beta > 7 || S < 1 || (A.ld % 8) || (B.ld % 8) || K > A.ld || K > B.ld || M > A.rows ||
      N > B.rows)
    return cudaErrorInvalidValue;
  CUtensorMap mA, mB;
  const long long ta = A.total_rows > 0 ? A.total_rows : (long long)S * A.rows;
  const long long tb = B.total_rows > 0 ? B.total_rows : (long long)S * B.rows;
  if (!make_map(&mA, A.slices, ta, K, A.ld, 128, OZ_BK) || !make_map(&mB, B.slices, tb, K, B.ld, 128, OZ_BK))
    return cudaErrorInvalidValue;
  const cudaError_t attr_err = smem_optin(reinterpret_cast<const void*>(k_ozaki_gemm), OZ_SMEM);
  if (attr_err != cudaSuccess) return attr_err;
  OzParams p;
  p.M = M;
  p.N = N;
  p.K = K;
  p.a_rows = A.rows;
  p.b_rows = B.rows;
  p.eA = A.exps;
  p.eB = B.exps;
  p.fA = A.fixed_e;
  p.fB = B.fixed_e;
  p.S = S;
  p.beta = beta;
  p.C = C;
  p.ldc = ldc;
  p.ws = ws;
  p.run_if = run_if;
  p.limit_ns = spin_cap > 0 ? (uint64_t)spin_cap : 4000000000ull;
  p.st = st;
  const int nkt = (K + OZ_BK - 1) / OZ_BK;
  const int tiles = ((M + 127) / 128) * ((N + OZ_BN - 1) / OZ_BN);
  const int sms = device_sm_count();
  // splits: exactness bounds each split's K; below one wave of tiles, split
  // K further (every split keeps >= 8 k-slices) as far as the workspace holds
  const int kmax_kt = (int)std::max<long long>(1, oz_max_k(beta) / OZ_BK);
  int nsplit = (nkt + kmax_kt - 1) / kmax_kt;
  if (tiles * nsplit < sms) nsplit = std::max(nsplit, std::min((sms + tiles - 1) / tiles, nkt / 8));
  if (nsplit > 1) {
    const size_t need = (size_t)M * N;
    const int cap = ws ? (int)std::min<size_t>((size_t)1 << 20, ws_doubles / need) : 0;
    const int must = (nkt + kmax_kt - 1) / kmax_kt;
    if (must > cap && must > 1) return cudaErrorInvalidValue;   // exactness needs more than the workspace holds
    nsplit = std::max(must, std::min(nsplit, std::max(cap, 1)));
  }
  int kchunk = (nkt + nsplit - 1) / nsplit;
  kchunk = std::min(kchunk, kmax_kt);
  nsplit = (nkt + kchunk - 1) / kchunk;              // every split non-empty
  p.kchunk = kchunk;
  p.mode = nsplit > 1 ? 2 : (subtract ? 1 : 0);
  // chains: up to g pairs of a level share an accumulator while
  // g (kchunk OZ_BK) 2^(2 beta - 2) <= 2^24
  const int g = (int)std::max<long long>(1, oz_max_k(beta) / ((long long)kchunk * OZ_BK));
  const int L = max_level >= 0 ? std::min(max_level, 2 * S - 2) : S - 1;
  p.nchains = 0;
  for (int l = 0; l <= L; ++l) {
    const int s_lo = std::max(0, l - (S - 1)), s_hi = std::min(l, S - 1);
    for (int s0 = s_lo; s0 <= s_hi; s0 += g) {
      if (p.nchains >= 64) return cudaErrorInvalidValue;
      p.ch_level[p.nchains] = (signed char)l;
      p.ch_s0[p.nchains] = (signed char)s0;
      p.ch_cnt[p.nchains] = (signed char)std::min(g, s_hi + 1 - s0);
      ++p.nchains;
    }
  }
  k_ozaki_gemm<<<(unsigned)(tiles * nsplit), OZ_THREADS, OZ_SMEM, s>>>(mA, mB, p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (launches) *launches += 1;
  if (nsplit > 1) {
    const long long tot = (long long)M * N;
    const int grid = (int)std::min<long long>((tot + 255) / 256, (long long)sms * 8);
    k_oz_reduce<<<grid, 256, 0, s>>>(M, N, nsplit, ws, C, ldc, subtract ? 1 : 0, run_if);
    if (launches) *launches += 1;
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace lc

extern "C" LC_API int lc_gemm_f64_tc(const double* A, const double* B, int M, int N, int K, double* C,
                                     void* stream) {
  using namespace lc;
  if (!A || !B || !C || M < 1 || N < 1 || K < 1) return LC_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!tcgen05_available()) return LC_ERR_CUDA;
  // rows padded with zero digits to a multiple of the 64-wide k-box
  const int ld = round_up(K, 64);
  const int beta = oz_beta_for(std::min(ld, 1 << 14));
  const int S = oz_slices_for(beta);
  const long long kmax = oz_max_k(beta);
  const int must = (int)((ld + kmax - 1) / kmax);
  const size_t nA = (size_t)S * M * ld, nB = (size_t)S * N * ld;
  // split-K partials: the splits exactness needs, or the occupancy splits of
  // a grid below one wave (as ozaki_gemm_nt chooses them)
  const int tiles = ((M + 127) / 128) * ((N + 127) / 128), sms = device_sm_count(), nkt = ld / 64;
  const int occ = tiles < sms ? std::min((sms + tiles - 1) / tiles, nkt / 8) : 1;
  const int nsplit_max = std::max(must, occ);
  const size_t ws_doubles = nsplit_max > 1 ? (size_t)M * N * (size_t)nsplit_max : 0;
  const size_t bytes = (nA + nB) * 2 + (size_t)(M + N) * 4 + ws_doubles * 8 + sizeof(DevStatus) + 2048;
  char* w = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&w), bytes, s) != cudaSuccess) return LC_ERR_OOM;
  size_t off = 0;
  auto take = [&](size_t b) { char* p = w + off; off = (off + b + 255) & ~size_t(255); return p; };
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(take(nA * 2));
  __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(take(nB * 2));
  int* eA = reinterpret_cast<int*>(take((size_t)M * 4));
  int* eB = reinterpret_cast<int*>(take((size_t)N * 4));
  double* ws = reinterpret_cast<double*>(take(ws_doubles * 8));
  DevStatus* st = reinterpret_cast<DevStatus*>(take(sizeof(DevStatus)));
  int rc = LC_OK;
  DevStatus hst;
  memset(&hst, 0, sizeof(hst));
  if (cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess ||
      cudaMemsetAsync(As, 0, nA * 2, s) != cudaSuccess || cudaMemsetAsync(Bs, 0, nB * 2, s) != cudaSuccess)
    rc = LC_ERR_CUDA;
  if (rc == LC_OK && (oz_slice_rows(A, M, K, K, S, beta, 0, As, M, ld, eA, 0, nullptr, s) != cudaSuccess ||
                      oz_slice_rows(B, N, K, K, S, beta, 0, Bs, N, ld, eB, 0, nullptr, s) != cudaSuccess))
    rc = LC_ERR_CUDA;
  if (rc == LC_OK) {
    const OzOperand oa{As, M, ld, eA, 0}, ob{Bs, N, ld, eB, 0};
    if (ozaki_gemm_nt(M, N, ld, oa, ob, S, beta, C, N, false, ws, ws_doubles, nullptr, 0, st, s, nullptr, S) !=
        cudaSuccess)
      rc = LC_ERR_CUDA;
  }
  if (rc == LC_OK) cudaMemcpyAsync(&hst, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(w, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == LC_OK) rc = LC_ERR_CUDA;
  if (rc == LC_OK && hst.code != 0) rc = hst.code;
  return rc;
}
