// ttm_tc.cu -- mode-n TTM on the 5th-generation tensor cores (tcgen05) for
// tensors stored in BF16: Out = In x_n F^T (Sec. 2.1), transposition-free.
//
// GEMM view (per tile): D[M = 128 free positions, N] += A[128 x L] * B[L x N]
//   column case (mode not last, C > 1): the 128 positions are 128 consecutive
//     c of one r; the A tile In[r, l0:l0+64, c0:c0+128] arrives by TMA as two
//     64 x 64 boxes with the 128-byte swizzle and is used MN-major;
//   row case (last mode, C = 1): the positions are 128 consecutive r; the A
//     tile In[r0:r0+128, l0:l0+64] is K-major.
// B holds F split into a high and a low BF16 part, [F_hi | F_lo] side by side
// along N (N = 2*Np, Np = K rounded up to 16), so the product carries F to
// ~16 bits while T keeps its storage precision; the epilogue adds the halves.
// Optionally the tensor itself comes as two BF16 tensors hi + lo (a split of an
// FP32 tensor): then each k-step issues a second MMA A_lo * F_hi into the
// first half.  Accumulation is FP32 in tensor memory (TMEM).
//
// Warp roles (320 threads, one CTA per SM, persistent over tiles):
//   warp 0  TMA producer (one lane) through a kStages-deep shared-memory ring;
//   warp 1  TMEM allocation and the MMA issuer (one lane);
//   warps 2-9  epilogue, two groups of four taking alternate tiles:
//              tcgen05.ld of the accumulator rows their TMEM lane quarter
//              owns, FP32 sum of the two halves, global stores.
// Four accumulator buffers in TMEM let the epilogues of earlier tiles overlap
// the MMAs of later ones (with one 64-wide l chunk per tile, as for L = 64, the
// epilogue is the longest stage).  Every mbarrier wait is bounded by a
// %globaltimer deadline; on expiry the kernel records an error word, drains
// its own copies (bounded), frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <atomic>
#include <mutex>

#include "tc_common.cuh"

namespace tk {

__device__ int g_tk_status = 0;  // 0 = ok, else the code of the first timeout

namespace {

using namespace tc;

constexpr int kStagesPlain = 8;  // ring depth, one A tensor per stage
constexpr int kStagesSplit = 5;  // ring depth, hi and lo A tensors per stage
__host__ __device__ constexpr int stages_for(bool split) { return split ? kStagesSplit : kStagesPlain; }
constexpr int kBoxL = 64;                       // l per stage (128 B of BF16)
constexpr int kTileM = 128;                     // positions per tile
constexpr int kStageBytes = kTileM * kBoxL * 2;  // one A tensor, 16 KB
constexpr int kAccBufs = 4;      // TMEM accumulator buffers
constexpr int kEpiGroups = 2;    // epilogue warp groups (4 warps each), alternate tiles
constexpr int kThreads = 64 + kEpiGroups * 128;

// Bounded wait on this translation unit's error word (see tc_common.cuh).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  return mbar_wait_status(bar, parity, abort_flag, &g_tk_status);
}


// Instruction descriptor for kind::f16 with BF16 A and B, FP32 accumulate,
// M = 128, B K-major; A K-major (0) or MN-major (1).
__host__ __device__ constexpr uint32_t idesc_bf16(int n, int a_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn_major << 15) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
template <typename TOut>
__device__ __forceinline__ TOut to_out(float v) {
  return OutCvt<TOut>::run(v);
}

struct TcParams {
  int64_t R, C;   // view [R][L][C]
  int L, K;       // contraction length, outputs per position
  int Np;         // K rounded up to 16
  int nk;         // number of 64-wide l chunks
  int64_t tiles;  // number of 128-position tiles
  int64_t ctiles; // column case: tiles per r
  int pack2;      // column case with C == 64: one tile = two consecutive r
  int vec_rows;   // row case: output rows 16-byte aligned (vector stores)
  const float* F; // L x K row-major (FP32)
};

// SMEM layout (dynamic, 1024-aligned):
//   [A ring: kStages x (1 or 2) x 16 KB][B: nk chunks x (2*Np rows) x 128 B]
//   [barriers][tmem slot][abort flag]
template <bool kRows, bool kSplitA, typename TOut>
__global__ void __launch_bounds__(kThreads, 1)
    ttm_tc_kernel(const __grid_constant__ CUtensorMap map_hi,
                  const __grid_constant__ CUtensorMap map_lo, TOut* __restrict__ Y,
                  const TcParams P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int kA = kSplitA ? 2 : 1;
  constexpr uint32_t kStages = (uint32_t)stages_for(kSplitA);
  unsigned char* ring = smem;
  unsigned char* bsm = ring + (size_t)kStages * kA * kStageBytes;
  const int N2 = 2 * P.Np;  // rows of B ([F_hi | F_lo] along N)
  const size_t b_bytes = (size_t)P.nk * N2 * 128;
  uint64_t* bars = reinterpret_cast<uint64_t*>(bsm + ((b_bytes + 15) & ~size_t(15)));
  uint64_t* full = bars;                // kStages
  uint64_t* empty = bars + kStages;     // kStages
  uint64_t* tfull = bars + 2 * kStages;  // kAccBufs
  uint64_t* tempty = tfull + kAccBufs;   // kAccBufs
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + kAccBufs);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // TMEM: kAccBufs accumulator buffers of N2 columns each
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(kAccBufs * N2)) ncols <<= 1;

  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < kAccBufs; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B = [F_hi | F_lo]^T as BF16, K-major without swizzle: core matrices of 8
  // rows x 8 l (16 B per row); LBO = 128 B between l-groups, SBO = (64/8)*128
  // between 8-row groups, one 64-l chunk after another.
  for (int idx = threadIdx.x; idx < N2 * P.nk * kBoxL; idx += kThreads) {
    const int row = idx / (P.nk * kBoxL);
    const int l = idx - row * (P.nk * kBoxL);
    const int k = row < P.Np ? row : row - P.Np;
    float f = 0.f;
    if (k < P.K && l < P.L) f = P.F[(int64_t)l * P.K + k];
    const uint16_t hi = f2bf(f);
    const float rem = f - __uint_as_float((uint32_t)hi << 16);
    const uint16_t v = row < P.Np ? hi : f2bf(rem);
    const int chunk = l / kBoxL, lc = l - chunk * kBoxL;
    const size_t off = (size_t)chunk * N2 * 128 + (size_t)(row >> 3) * 1024 + (size_t)(lc >> 3) * 128 +
                       (size_t)(row & 7) * 16 + (size_t)(lc & 7) * 2;
    *reinterpret_cast<uint16_t*>(bsm + off) = v;
  }
  // generic-proxy writes of B must be visible to the tensor core (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
        for (int kc = 0; kc < P.nk; ++kc, ++it) {
          const uint32_t s = it % kStages, ph = (it / kStages) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], (uint32_t)(kA * kStageBytes));
          unsigned char* dst = ring + (size_t)s * kA * kStageBytes;
          if (kRows) {
            const int r0 = (int)(t * kTileM);
            tma_load_2d(dst, &map_hi, &full[s], kc * kBoxL, r0);
            if (kSplitA) tma_load_2d(dst + kStageBytes, &map_lo, &full[s], kc * kBoxL, r0);
          } else {
            if (P.pack2) {
              // one {64 c, 64 l, 2 r} box: r and r+1 land 8 KB apart, the same
              // layout as the two 64-position halves of a wide tile
              tma_load_3d(dst, &map_hi, &full[s], 0, kc * kBoxL, (int)(2 * t));
              if (kSplitA) tma_load_3d(dst + kStageBytes, &map_lo, &full[s], 0, kc * kBoxL, (int)(2 * t));
              continue;
            }
            const int64_t r = t / P.ctiles;
            const int c0 = (int)((t - r * P.ctiles) * kTileM);
            tma_load_3d(dst, &map_hi, &full[s], c0, kc * kBoxL, (int)r);
            tma_load_3d(dst + kStageBytes / 2, &map_hi, &full[s], c0 + 64, kc * kBoxL, (int)r);
            if (kSplitA) {
              tma_load_3d(dst + kStageBytes, &map_lo, &full[s], c0, kc * kBoxL, (int)r);
              tma_load_3d(dst + kStageBytes + kStageBytes / 2, &map_lo, &full[s], c0 + 64,
                          kc * kBoxL, (int)r);
            }
          }
        }
      }
      // drain: wait (bounded) until every copy issued has landed
      const uint32_t issued = it;
      for (uint32_t j = (issued > kStages ? issued - kStages : 0); j < issued; ++j) {
        const uint32_t s = j % kStages, ph = (j / kStages) & 1u;
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(&full[s], ph) && globaltimer() - t0 < kTimeoutNs) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc_full = idesc_bf16(N2, kRows ? 0 : 1);
      const uint32_t idesc_half = idesc_bf16(P.Np, kRows ? 0 : 1);
      const uint32_t b_base = smem_u32(bsm);
      uint32_t it = 0, tcount = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < P.tiles && ok; t += gridDim.x, ++tcount) {
        const uint32_t buf = tcount % kAccBufs, aph = (tcount / kAccBufs) & 1u;
        if (!mbar_wait(&tempty[buf], aph ^ 1u, abort_flag)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + buf * (uint32_t)N2;
        for (int kc = 0; kc < P.nk; ++kc, ++it) {
          const uint32_t s = it % kStages, ph = (it / kStages) & 1u;
          if (!mbar_wait(&full[s], ph, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_u32(ring + (size_t)s * kA * kStageBytes);
#pragma unroll
          for (int ks = 0; ks < kBoxL / 16; ++ks) {
            uint64_t ad_hi, ad_lo;
            if (kRows) {
              // K-major, 128 rows of 128 B: 8-row groups 1024 B apart,
              // k-step of 16 elements = 32 B inside the swizzled row
              ad_hi = smem_desc(a_base + ks * 32, 16, 1024, kSwizzle128);
              ad_lo = smem_desc(a_base + kStageBytes + ks * 32, 16, 1024, kSwizzle128);
            } else {
              // MN-major: 64-position halves 8 KB apart (LBO), 8-row l-groups
              // 1024 B apart (SBO), k-step of 16 l = 2048 B
              ad_hi = smem_desc(a_base + ks * 2048, 8192, 1024, kSwizzle128);
              ad_lo = smem_desc(a_base + kStageBytes + ks * 2048, 8192, 1024, kSwizzle128);
            }
            const uint32_t b_chunk = b_base + (uint32_t)(kc * N2 * 128);
            const uint64_t bd = smem_desc(b_chunk + ks * 256, 128, 1024, kSwizzleNone);
            const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
            mma_bf16(d_tmem, ad_hi, bd, idesc_full, acc);
            if (kSplitA) mma_bf16(d_tmem, ad_lo, bd, idesc_half, 1u);
          }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&tfull[buf]);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // group g (warps 2+4g .. 5+4g) takes every kEpiGroups-th tile
    const int q = warp & 3;            // TMEM lane quarter of this warp
    const int row = q * 32 + lane;     // accumulator row = tile position
    const uint32_t group = (uint32_t)(warp - 2) / 4u;
    uint32_t tcount = group;
    for (int64_t t = blockIdx.x + (int64_t)group * gridDim.x; t < P.tiles;
         t += (int64_t)kEpiGroups * gridDim.x, tcount += kEpiGroups) {
      const uint32_t buf = tcount % kAccBufs, aph = (tcount / kAccBufs) & 1u;
      if (!mbar_wait(&tfull[buf], aph, abort_flag)) break;
      tc_fence_after();
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + buf * (uint32_t)N2;
      float hi[16], lo[16];
      for (int k0 = 0; k0 < P.Np; k0 += 16) {
        tmem_ld16(tbase + k0, hi);
        tmem_ld16(tbase + P.Np + k0, lo);
        tmem_wait_ld();
        if (k0 + 16 >= P.Np) {
          // the whole accumulator is in registers: hand the buffer back
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[buf]);
        }
        if (kRows) {
          const int64_t r = t * kTileM + row;
          if (r < P.R && TK_DBG_IN(r * P.K + k0, r * P.K + min(P.K, k0 + 16) - 1, P.R * P.K)) {
            TOut* yp = Y + r * P.K + k0;
            if (P.vec_rows && k0 + 16 <= P.K) {
              // 16 consecutive outputs of this row: 16-byte vector stores
              TOut o[16];
#pragma unroll
              for (int j = 0; j < 16; ++j) o[j] = to_out<TOut>(hi[j] + lo[j]);
              const uint4* src = reinterpret_cast<const uint4*>(o);
              uint4* dst = reinterpret_cast<uint4*>(yp);
#pragma unroll
              for (int v = 0; v < (int)(16 * sizeof(TOut) / 16); ++v) dst[v] = src[v];
            } else {
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (k0 + j < P.K) yp[j] = to_out<TOut>(hi[j] + lo[j]);
            }
          }
        } else if (P.pack2) {
          const int64_t r = 2 * t + (row >> 6);
          const int64_t c = row & 63;
          if (r < P.R && TK_DBG_IN((r * P.K) * P.C + c, (r * P.K + P.K - 1) * P.C + c, P.R * P.K * P.C)) {
            TOut* yp = Y + (r * P.K) * P.C + c;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (k0 + j < P.K) yp[(int64_t)(k0 + j) * P.C] = to_out<TOut>(hi[j] + lo[j]);
          }
        } else {
          const int64_t r = t / P.ctiles;
          const int64_t c = (t - r * P.ctiles) * kTileM + row;
          if (c < P.C && TK_DBG_IN((r * P.K) * P.C + c, (r * P.K + P.K - 1) * P.C + c, P.R * P.K * P.C)) {
            TOut* yp = Y + (r * P.K) * P.C + c;
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (k0 + j < P.K) yp[(int64_t)(k0 + j) * P.C] = to_out<TOut>(hi[j] + lo[j]);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(ncols));
  }
}

// ---------------------------------------------------------------------------
// FP32 tensors on the tensor cores (column case).  TMA brings 64 l x 128 c
// FP32 tiles into a staging ring (no swizzle); a converter warpgroup splits
// each value into three BF16 parts x1 = RNE(x), x2 = RNE(x - x1),
// x3 = RNE(x - x1 - x2) (together 24 significant bits) and writes them in the
// 128-byte-swizzled MN-major layout the MMA reads (the layout TMA produces for
// BF16 boxes: 16-byte chunk j of row l stored at chunk j ^ (l & 7)).  F is
// split the same way, B = [F1 | F2 | F3] along N.  Per k-step the MMA warp
// issues A1 [F1|F2|F3] (N = 3 Np), A2 [F1|F2] (2 Np) and A3 F1 (Np) into one
// accumulator, whose three column groups the epilogue adds: the six products
// x_i f_j with i + j <= 4 leave out terms below 2^-24 |x f|, so the result is
// as accurate as an FP32 contraction, read once at 4 bytes per element, with
// the arithmetic off the CUDA cores.
//
// Warp roles (448 threads): warp 0 TMA producer, warp 1 TMEM + MMA issuer,
// warps 2-5 converter, warps 6-13 two epilogue groups.
// ---------------------------------------------------------------------------
constexpr int kF32St = 2;                            // staging stages (FP32)
constexpr int kF32Cv = 2;                            // converted stages (3 BF16 parts)
constexpr int kF32StageBytes = kTileM * kBoxL * 4;   // 32 KB
constexpr int kF32CvBytes = 3 * kStageBytes;         // 48 KB
constexpr int kF32Threads = 64 + 128 + kEpiGroups * 128;

__device__ __forceinline__ uint32_t bf_hi_bits(float x) { return f2bf(x); }
__device__ __forceinline__ float bf_val(uint32_t b) { return __uint_as_float(b << 16); }

template <typename TOut>
__global__ void __launch_bounds__(kF32Threads, 1)
    ttm_tc_f32_kernel(const __grid_constant__ CUtensorMap map_x, TOut* __restrict__ Y,
                      const TcParams P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* stage = smem;                                        // kF32St x 32 KB
  unsigned char* conv = stage + (size_t)kF32St * kF32StageBytes;      // kF32Cv x 48 KB
  unsigned char* bsm = conv + (size_t)kF32Cv * kF32CvBytes;
  const int N3 = 3 * P.Np;
  const size_t b_bytes = (size_t)P.nk * N3 * 128;
  uint64_t* bars = reinterpret_cast<uint64_t*>(bsm + ((b_bytes + 15) & ~size_t(15)));
  uint64_t* st_full = bars;                   // kF32St
  uint64_t* st_empty = st_full + kF32St;      // kF32St
  uint64_t* cv_full = st_empty + kF32St;      // kF32Cv
  uint64_t* cv_empty = cv_full + kF32Cv;      // kF32Cv
  uint64_t* tfull = cv_empty + kF32Cv;        // kAccBufs
  uint64_t* tempty = tfull + kAccBufs;        // kAccBufs
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + kAccBufs);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(kAccBufs * N3)) ncols <<= 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kF32St; ++s) {
      mbar_init(&st_full[s], 1);
      mbar_init(&st_empty[s], 4);
    }
    for (int s = 0; s < kF32Cv; ++s) {
      mbar_init(&cv_full[s], 4);
      mbar_init(&cv_empty[s], 1);
    }
    for (int b = 0; b < kAccBufs; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B = [F1 | F2 | F3]^T as BF16, K-major without swizzle (as in ttm_tc_kernel)
  for (int idx = threadIdx.x; idx < N3 * P.nk * kBoxL; idx += kF32Threads) {
    const int row = idx / (P.nk * kBoxL);
    const int l = idx - row * (P.nk * kBoxL);
    const int part = row / P.Np, k = row - part * P.Np;
    float f = 0.f;
    if (k < P.K && l < P.L) f = P.F[(int64_t)l * P.K + k];
    const uint32_t f1 = bf_hi_bits(f);
    const float r1 = f - bf_val(f1);
    const uint32_t f2 = bf_hi_bits(r1);
    const uint32_t f3 = bf_hi_bits(r1 - bf_val(f2));
    const uint16_t v = (uint16_t)(part == 0 ? f1 : (part == 1 ? f2 : f3));
    const int chunk = l / kBoxL, lc = l - chunk * kBoxL;
    const size_t off = (size_t)chunk * N3 * 128 + (size_t)(row >> 3) * 1024 + (size_t)(lc >> 3) * 128 +
                       (size_t)(row & 7) * 16 + (size_t)(lc & 7) * 2;
    *reinterpret_cast<uint16_t*>(bsm + off) = v;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
        const int64_t r = t / P.ctiles;
        const int c0 = (int)((t - r * P.ctiles) * kTileM);
        for (int kc = 0; kc < P.nk; ++kc, ++it) {
          const uint32_t s = it % kF32St, ph = (it / kF32St) & 1u;
          if (!mbar_wait(&st_empty[s], ph ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&st_full[s], (uint32_t)kF32StageBytes);
          tma_load_3d(stage + (size_t)s * kF32StageBytes, &map_x, &st_full[s], c0, kc * kBoxL, (int)r);
        }
      }
      const uint32_t issued = it;
      for (uint32_t j = (issued > (uint32_t)kF32St ? issued - kF32St : 0); j < issued; ++j) {
        const uint32_t s = j % kF32St, ph = (j / kF32St) & 1u;
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(&st_full[s], ph) && globaltimer() - t0 < kTimeoutNs) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc3 = idesc_bf16(N3, 1);
      const uint32_t idesc2 = idesc_bf16(2 * P.Np, 1);
      const uint32_t idesc1 = idesc_bf16(P.Np, 1);
      const uint32_t b_base = smem_u32(bsm);
      uint32_t it = 0, tcount = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < P.tiles && ok; t += gridDim.x, ++tcount) {
        const uint32_t buf = tcount % kAccBufs, aph = (tcount / kAccBufs) & 1u;
        if (!mbar_wait(&tempty[buf], aph ^ 1u, abort_flag)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + buf * (uint32_t)N3;
        for (int kc = 0; kc < P.nk; ++kc, ++it) {
          const uint32_t s = it % kF32Cv, ph = (it / kF32Cv) & 1u;
          if (!mbar_wait(&cv_full[s], ph, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_u32(conv + (size_t)s * kF32CvBytes);
#pragma unroll
          for (int ks = 0; ks < kBoxL / 16; ++ks) {
            const uint64_t a1 = smem_desc(a_base + ks * 2048, 8192, 1024, kSwizzle128);
            const uint64_t a2 = smem_desc(a_base + kStageBytes + ks * 2048, 8192, 1024, kSwizzle128);
            const uint64_t a3 = smem_desc(a_base + 2 * kStageBytes + ks * 2048, 8192, 1024, kSwizzle128);
            const uint32_t b_chunk = b_base + (uint32_t)(kc * N3 * 128);
            const uint64_t bd = smem_desc(b_chunk + ks * 256, 128, 1024, kSwizzleNone);
            const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
            mma_bf16(d_tmem, a1, bd, idesc3, acc);
            mma_bf16(d_tmem, a2, bd, idesc2, 1u);
            mma_bf16(d_tmem, a3, bd, idesc1, 1u);
          }
          mma_commit(&cv_empty[s]);
        }
        if (!ok) break;
        mma_commit(&tfull[buf]);
      }
    }
  } else if (warp < 6) {
    // ------------------------------------------------------------ converter
    const int ct = threadIdx.x - 64;  // 0 .. 127
    uint32_t it = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
      for (int kc = 0; kc < P.nk; ++kc, ++it) {
        const uint32_t ss = it % kF32St, sph = (it / kF32St) & 1u;
        const uint32_t cs = it % kF32Cv, cph = (it / kF32Cv) & 1u;
        if (!mbar_wait(&st_full[ss], sph, abort_flag) || !mbar_wait(&cv_empty[cs], cph ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        const float* src = reinterpret_cast<const float*>(stage + (size_t)ss * kF32StageBytes);
        unsigned char* d1 = conv + (size_t)cs * kF32CvBytes;
#pragma unroll 4
        for (int i = 0; i < (kTileM * kBoxL / 2) / 128; ++i) {
          const int p = ct + 128 * i;  // pair index: l = p / 64, c = 2 (p % 64)
          const int l = p >> 6, c = (p & 63) << 1;
          const float2 x = *reinterpret_cast<const float2*>(src + l * kTileM + c);
          const uint32_t a0 = bf_hi_bits(x.x), b0 = bf_hi_bits(x.y);
          const float ra = x.x - bf_val(a0), rb = x.y - bf_val(b0);
          const uint32_t a1 = bf_hi_bits(ra), b1 = bf_hi_bits(rb);
          const uint32_t a2 = bf_hi_bits(ra - bf_val(a1)), b2 = bf_hi_bits(rb - bf_val(b1));
          const int cc = c & 63;
          const uint32_t off = (uint32_t)(c >> 6) * 8192u + (uint32_t)l * 128u +
                               ((uint32_t)((cc >> 3) ^ (l & 7)) << 4) + (uint32_t)((cc & 7) << 1);
          *reinterpret_cast<uint32_t*>(d1 + off) = a0 | (b0 << 16);
          *reinterpret_cast<uint32_t*>(d1 + kStageBytes + off) = a1 | (b1 << 16);
          *reinterpret_cast<uint32_t*>(d1 + 2 * kStageBytes + off) = a2 | (b2 << 16);
        }
        // the tensor core reads the converted tile through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&cv_full[cs]);
          mbar_arrive(&st_empty[ss]);
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t group = (uint32_t)(warp - 6) / 4u;
    uint32_t tcount = group;
    for (int64_t t = blockIdx.x + (int64_t)group * gridDim.x; t < P.tiles;
         t += (int64_t)kEpiGroups * gridDim.x, tcount += kEpiGroups) {
      const uint32_t buf = tcount % kAccBufs, aph = (tcount / kAccBufs) & 1u;
      if (!mbar_wait(&tfull[buf], aph, abort_flag)) break;
      tc_fence_after();
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + buf * (uint32_t)N3;
      const int64_t r = t / P.ctiles;
      const int64_t c = (t - r * P.ctiles) * kTileM + row;
      float g1[16], g2[16], g3[16];
      for (int k0 = 0; k0 < P.Np; k0 += 16) {
        tmem_ld16(tbase + k0, g1);
        tmem_ld16(tbase + P.Np + k0, g2);
        tmem_ld16(tbase + 2 * P.Np + k0, g3);
        tmem_wait_ld();
        if (k0 + 16 >= P.Np) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[buf]);
        }
        if (c < P.C && TK_DBG_IN((r * P.K) * P.C + c, (r * P.K + P.K - 1) * P.C + c, P.R * P.K * P.C)) {
          TOut* yp = Y + (r * P.K) * P.C + c;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (k0 + j < P.K) yp[(int64_t)(k0 + j) * P.C] = to_out<TOut>((g3[j] + g2[j]) + g1[j]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(ncols));
  }
}

// ---------------------------------------------------------------------------
// FP8 E4M3 tensors (one FP32 scale per 64 consecutive elements) on the tensor
// cores (column case, C % 256 == 0).  TMA brings 128 c x 64 l tiles of codes
// (8 KB) into a staging ring (no swizzle) and, on the same barrier, the
// tile's scales: the scale array read as [R L][C / 64] rows, a 4 x 64 box
// from the 16-byte-aligned column at or below c0 / 64 (the tile's two scale
// columns sit at 0 or 2 within it).  A converter of eight warps decodes eight
// codes at a time, multiplies them by their block's scale (exact in FP32: a
// 4-bit significand times a 24-bit one) and writes the value rounded to BF16
// (relative 2^-9, a 32nd of the E4M3 step) in the 128-byte-swizzled MN-major
// layout; per k-step the MMA warp issues A [F_hi | F_lo], so F keeps ~16
// bits.  The converter issues no global loads (earlier versions read the
// scales with per-thread loads six stages ahead).  Warp roles: warp 0 TMA
// producer, warp 1 TMEM + MMA issuer, warps 2-9 converter, warps 10-17 two
// epilogue groups.
// ---------------------------------------------------------------------------
constexpr int kF8St = 8;                          // staging stages (codes): 64 KB in flight
constexpr int kF8Cv = 6;                          // converted stages (BF16; 3 measured 1.6 % slower)
constexpr int kF8Warps = 8;                       // converter warps
constexpr int kF8StageBytes = kTileM * kBoxL;     // 8 KB
constexpr int kF8ScaleBytes = 4 * kBoxL * 4;       // 4 scale columns x 64 rows (1 KB)
constexpr int kF8CvBytes = kStageBytes;           // 16 KB
constexpr int kF8Threads = 64 + kF8Warps * 32 + kEpiGroups * 128;

template <typename TOut>
__global__ void __launch_bounds__(kF8Threads, 1)
    ttm_tc_fp8_kernel(const __grid_constant__ CUtensorMap map_q, const __grid_constant__ CUtensorMap map_s,
                      TOut* __restrict__ Y, const TcParams P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* stage = smem;                                        // kF8St x 8 KB
  unsigned char* conv = stage + (size_t)kF8St * kF8StageBytes;        // kF8Cv x 16 KB
  unsigned char* ssm = conv + (size_t)kF8Cv * kF8CvBytes;             // kF8St x 1 KB scales
  unsigned char* bsm = ssm + (size_t)kF8St * kF8ScaleBytes;
  const int N2 = 2 * P.Np;
  const size_t b_bytes = (size_t)P.nk * N2 * 128;
  uint64_t* bars = reinterpret_cast<uint64_t*>(bsm + ((b_bytes + 15) & ~size_t(15)));
  uint64_t* st_full = bars;                   // kF8St
  uint64_t* st_empty = st_full + kF8St;       // kF8St
  uint64_t* cv_full = st_empty + kF8St;       // kF8Cv
  uint64_t* cv_empty = cv_full + kF8Cv;       // kF8Cv
  uint64_t* tfull = cv_empty + kF8Cv;         // kAccBufs
  uint64_t* tempty = tfull + kAccBufs;        // kAccBufs
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + kAccBufs);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(kAccBufs * N2)) ncols <<= 1;

  if (threadIdx.x == 0) {
    for (int st = 0; st < kF8St; ++st) {
      mbar_init(&st_full[st], 1);
      mbar_init(&st_empty[st], kF8Warps);
    }
    for (int st = 0; st < kF8Cv; ++st) {
      mbar_init(&cv_full[st], kF8Warps);
      mbar_init(&cv_empty[st], 1);
    }
    for (int b = 0; b < kAccBufs; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B = [F_hi | F_lo]^T as BF16, K-major without swizzle (as in ttm_tc_kernel)
  for (int idx = threadIdx.x; idx < N2 * P.nk * kBoxL; idx += kF8Threads) {
    const int row = idx / (P.nk * kBoxL);
    const int l = idx - row * (P.nk * kBoxL);
    const int k = row < P.Np ? row : row - P.Np;
    float f = 0.f;
    if (k < P.K && l < P.L) f = P.F[(int64_t)l * P.K + k];
    const uint16_t hi = f2bf(f);
    const float rem = f - __uint_as_float((uint32_t)hi << 16);
    const uint16_t v = row < P.Np ? hi : f2bf(rem);
    const int chunk = l / kBoxL, lc = l - chunk * kBoxL;
    const size_t off = (size_t)chunk * N2 * 128 + (size_t)(row >> 3) * 1024 + (size_t)(lc >> 3) * 128 +
                       (size_t)(row & 7) * 16 + (size_t)(lc & 7) * 2;
    *reinterpret_cast<uint16_t*>(bsm + off) = v;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
        const int64_t r = t / P.ctiles;
        const int c0 = (int)((t - r * P.ctiles) * kTileM);
        for (int kc = 0; kc < P.nk; ++kc, ++it) {
          const uint32_t st = it % kF8St, ph = (it / kF8St) & 1u;
          if (!mbar_wait(&st_empty[st], ph ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&st_full[st], (uint32_t)(kF8StageBytes + kF8ScaleBytes));
          tma_load_3d(stage + (size_t)st * kF8StageBytes, &map_q, &st_full[st], c0, kc * kBoxL, (int)r);
          tma_load_2d(ssm + (size_t)st * kF8ScaleBytes, &map_s, &st_full[st], (c0 >> 6) & ~3,
                      (int)(r * P.L + kc * kBoxL));
        }
      }
      const uint32_t issued = it;
      for (uint32_t j = (issued > (uint32_t)kF8St ? issued - kF8St : 0); j < issued; ++j) {
        const uint32_t st = j % kF8St, ph = (j / kF8St) & 1u;
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(&st_full[st], ph) && globaltimer() - t0 < kTimeoutNs) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc_full = idesc_bf16(N2, 1);
      const uint32_t b_base = smem_u32(bsm);
      uint32_t it = 0, tcount = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < P.tiles && ok; t += gridDim.x, ++tcount) {
        const uint32_t buf = tcount % kAccBufs, aph = (tcount / kAccBufs) & 1u;
        if (!mbar_wait(&tempty[buf], aph ^ 1u, abort_flag)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + buf * (uint32_t)N2;
        for (int kc = 0; kc < P.nk; ++kc, ++it) {
          const uint32_t cs = it % kF8Cv, ph = (it / kF8Cv) & 1u;
          if (!mbar_wait(&cv_full[cs], ph, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_u32(conv + (size_t)cs * kF8CvBytes);
#pragma unroll
          for (int ks = 0; ks < kBoxL / 16; ++ks) {
            const uint64_t ad = smem_desc(a_base + ks * 2048, 8192, 1024, kSwizzle128);
            const uint32_t b_chunk = b_base + (uint32_t)(kc * N2 * 128);
            const uint64_t bd = smem_desc(b_chunk + ks * 256, 128, 1024, kSwizzleNone);
            mma_bf16(d_tmem, ad, bd, idesc_full, (kc > 0 || ks > 0) ? 1u : 0u);
          }
          mma_commit(&cv_empty[cs]);
        }
        if (!ok) break;
        mma_commit(&tfull[buf]);
      }
    }
  } else if (warp < 2 + kF8Warps) {
    // ------------------------------------------------------------ converter
    // Thread ct converts groups g = ct + 256 i (i < 4) of a stage: row
    // l = g >> 4, columns c = 8 (g & 15) .. + 7; the scale of (l, c) is the
    // stage's scale row l, column ((c0 / 64) & 3) + (c >> 6).
    const int ct = threadIdx.x - 64;  // 0 .. 255
    uint32_t it = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
      const int64_t r = t / P.ctiles;
      const int sx = (int)((((t - r * P.ctiles) * kTileM) >> 6) & 3);
      for (int kc = 0; kc < P.nk; ++kc, ++it) {
        const uint32_t ss = it % kF8St, sph = (it / kF8St) & 1u;
        const uint32_t cs = it % kF8Cv, cph = (it / kF8Cv) & 1u;
        if (!mbar_wait(&st_full[ss], sph, abort_flag) || !mbar_wait(&cv_empty[cs], cph ^ 1u, abort_flag)) {
          ok = false;
          break;
        }
        const unsigned char* src = stage + (size_t)ss * kF8StageBytes;
        const float* scl = reinterpret_cast<const float*>(ssm + (size_t)ss * kF8ScaleBytes);
        unsigned char* dst = conv + (size_t)cs * kF8CvBytes;
#pragma unroll
        for (int i = 0; i < (kTileM * kBoxL / 8) / (kF8Warps * 32); ++i) {
          const int g = ct + kF8Warps * 32 * i;   // eight consecutive c of one l
          const int l = g >> 4, c = (g & 15) << 3;
          // with C % 64 == 0 the 64-column half of row l is one scale block;
          // codes past the tensor were zero-filled by TMA
          const float sc = scl[l * 4 + sx + (c >> 6)];
          const uint2 w = *reinterpret_cast<const uint2*>(src + l * kTileM + c);
          const uint32_t words[2] = {w.x, w.y};
          uint32_t hw[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const __nv_fp8x2_storage_t pr = (__nv_fp8x2_storage_t)((words[j >> 1] >> (16 * (j & 1))) & 0xFFFFu);
            const float2 v = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(pr, __NV_E4M3)));
            // paired round-to-nearest-even conversion (the values are finite)
            const __nv_bfloat162 hb = __floats2bfloat162_rn(v.x * sc, v.y * sc);
            hw[j] = *reinterpret_cast<const uint32_t*>(&hb);
          }
          const uint32_t off = (uint32_t)(c >> 6) * 8192u + (uint32_t)l * 128u +
                               ((uint32_t)(((c & 63) >> 3) ^ (l & 7)) << 4);
          *reinterpret_cast<uint4*>(dst + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&cv_full[cs]);
          mbar_arrive(&st_empty[ss]);
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t group = (uint32_t)(warp - 2 - kF8Warps) / 4u;
    uint32_t tcount = group;
    for (int64_t t = blockIdx.x + (int64_t)group * gridDim.x; t < P.tiles;
         t += (int64_t)kEpiGroups * gridDim.x, tcount += kEpiGroups) {
      const uint32_t buf = tcount % kAccBufs, aph = (tcount / kAccBufs) & 1u;
      if (!mbar_wait(&tfull[buf], aph, abort_flag)) break;
      tc_fence_after();
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + buf * (uint32_t)N2;
      const int64_t r = t / P.ctiles;
      const int64_t c = (t - r * P.ctiles) * kTileM + row;
      float hi[16], lo[16];
      for (int k0 = 0; k0 < P.Np; k0 += 16) {
        tmem_ld16(tbase + k0, hi);
        tmem_ld16(tbase + P.Np + k0, lo);
        tmem_wait_ld();
        if (k0 + 16 >= P.Np) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[buf]);
        }
        if (c < P.C && TK_DBG_IN((r * P.K) * P.C + c, (r * P.K + P.K - 1) * P.C + c, P.R * P.K * P.C)) {
          TOut* yp = Y + (r * P.K) * P.C + c;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (k0 + j < P.K) yp[(int64_t)(k0 + j) * P.C] = to_out<TOut>(hi[j] + lo[j]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(ncols));
  }
}

// ---------------------------------------------------------------------------
// BF16 root pair (column case, L2-blocked).  A sweep's two root children read
// the same tensor T along modes a and b = a + 2.  With mode m = a + 1 as the
// block index the work list runs block after block (value of i_m); within a
// block first the tiles of mode a's TTM (T viewed as [R_a][L_a][L_m * S],
// tiles of 128 of one block's S positions), then those of mode b's TTM (T
// viewed as [R_hi][L_m][L_b][C_b], rows of block i_m), so the block of T
// (|T| / L_m elements, 33 MB at 64^5 in BF16) is read from HBM once and
// found in L2 by the second TTM (measured: 2.18 GB read from DRAM for the
// 2.15 GB tensor).  The pair is opt-in: at 1.50 ms it is slower than the two
// separate TTMs (2 x 0.56 ms) although it reads T once.  Per tile the pipeline is ttm_tc_kernel's
// column case: two 64-position boxes per 64-l stage by TMA (128-byte
// swizzle, MN-major A), [F_hi | F_lo] of the tile's job as B, four TMEM
// accumulators, two epilogue groups of four warps on alternate tiles.
// ---------------------------------------------------------------------------
struct PairJob {
  int L, K, Np, nk;
  int block_c;       // 1: positions g * S + c (mode a); 0: rows (rh * G + g) (mode b)
  int64_t R;         // rows (mode a) or R_hi (mode b)
  int64_t S;         // positions per row: S (mode a) or C_b (mode b)
  int64_t ct;        // 128-position tiles per row
  int64_t per_block; // tiles per block
  uint32_t b_off;    // byte offset of this job's B in shared memory
  const float* F;
  void* Y;
};
struct PairParams {
  PairJob job[2];
  int64_t G, per_block, units;
};
struct PairTile {
  int j;
  int64_t r, c0, g;
};
// Work list block after block (value of i_m): each block's tiles of mode a
// (streaming the block from HBM) and then its tiles of mode b (finding the
// block in L2).  (Interleaving block s's mode-a tiles with block s - 1's
// mode-b tiles, to keep HBM streaming during the second TTM, measured slower:
// 1.92 against 1.50 ms on 64^5.)
__device__ __forceinline__ PairTile pair_decode(const PairParams& P, int64_t w) {
  PairTile t;
  t.g = w / P.per_block;
  int64_t i = w - t.g * P.per_block;
  t.j = i >= P.job[0].per_block ? 1 : 0;
  if (t.j) i -= P.job[0].per_block;
  const PairJob& J = P.job[t.j];
  const int64_t row = i / J.ct;
  t.c0 = (i - row * J.ct) * kTileM;
  t.r = J.block_c ? row : row * P.G + t.g;
  return t;
}

// SMEM (dynamic, 1024-aligned): [A ring: kStagesPlain x 16 KB][B job 0][B job 1]
//   [barriers][tmem slot][abort flag]
template <typename TOut>
__global__ void __launch_bounds__(kThreads, 1)
    ttm_tc_pair_kernel(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
                       const PairParams P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr uint32_t kStages = (uint32_t)kStagesPlain;
  unsigned char* ring = smem;
  unsigned char* bsm = ring + (size_t)kStages * kStageBytes;
  const size_t b_end = (size_t)P.job[1].b_off + (size_t)P.job[1].nk * 2 * P.job[1].Np * 128;
  uint64_t* bars = reinterpret_cast<uint64_t*>(bsm + ((b_end + 15) & ~size_t(15)));
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* tfull = bars + 2 * kStages;
  uint64_t* tempty = tfull + kAccBufs;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + kAccBufs);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N2max = 2 * max(P.job[0].Np, P.job[1].Np);  // accumulator buffer stride
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(kAccBufs * N2max)) ncols <<= 1;

  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < kAccBufs; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B of each job = [F_hi | F_lo]^T as BF16, K-major without swizzle (as in
  // ttm_tc_kernel)
  for (int j = 0; j < 2; ++j) {
    const PairJob& J = P.job[j];
    const int N2 = 2 * J.Np;
    for (int idx = threadIdx.x; idx < N2 * J.nk * kBoxL; idx += kThreads) {
      const int row = idx / (J.nk * kBoxL);
      const int l = idx - row * (J.nk * kBoxL);
      const int k = row < J.Np ? row : row - J.Np;
      float f = 0.f;
      if (k < J.K && l < J.L) f = J.F[(int64_t)l * J.K + k];
      const uint16_t hi = f2bf(f);
      const float rem = f - __uint_as_float((uint32_t)hi << 16);
      const uint16_t v = row < J.Np ? hi : f2bf(rem);
      const int chunk = l / kBoxL, lc = l - chunk * kBoxL;
      const size_t off = (size_t)J.b_off + (size_t)chunk * N2 * 128 + (size_t)(row >> 3) * 1024 +
                         (size_t)(lc >> 3) * 128 + (size_t)(row & 7) * 16 + (size_t)(lc & 7) * 2;
      *reinterpret_cast<uint16_t*>(bsm + off) = v;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      tma_prefetch_map(&map0);
      tma_prefetch_map(&map1);
      uint32_t it = 0;
      bool ok = true;
      for (int64_t w = blockIdx.x; w < P.units && ok; w += gridDim.x) {
        const PairTile t = pair_decode(P, w);
        const PairJob& J = P.job[t.j];
        const CUtensorMap* map = t.j ? &map1 : &map0;
        const int cx = (int)(J.block_c ? t.g * J.S + t.c0 : t.c0);
        for (int kc = 0; kc < J.nk; ++kc, ++it) {
          const uint32_t s = it % kStages, ph = (it / kStages) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], (uint32_t)kStageBytes);
          unsigned char* dst = ring + (size_t)s * kStageBytes;
          tma_load_3d(dst, map, &full[s], cx, kc * kBoxL, (int)t.r);
          tma_load_3d(dst + kStageBytes / 2, map, &full[s], cx + 64, kc * kBoxL, (int)t.r);
        }
      }
      const uint32_t issued = it;
      for (uint32_t j = (issued > kStages ? issued - kStages : 0); j < issued; ++j) {
        const uint32_t s = j % kStages, ph = (j / kStages) & 1u;
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(&full[s], ph) && globaltimer() - t0 < kTimeoutNs) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t b_base = smem_u32(bsm);
      uint32_t it = 0, tcount = 0;
      bool ok = true;
      for (int64_t w = blockIdx.x; w < P.units && ok; w += gridDim.x, ++tcount) {
        const PairTile t = pair_decode(P, w);
        const PairJob& J = P.job[t.j];
        const int N2 = 2 * J.Np;
        const uint32_t idesc_full = idesc_bf16(N2, 1);
        const uint32_t buf = tcount % kAccBufs, aph = (tcount / kAccBufs) & 1u;
        if (!mbar_wait(&tempty[buf], aph ^ 1u, abort_flag)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + buf * (uint32_t)N2max;
        for (int kc = 0; kc < J.nk; ++kc, ++it) {
          const uint32_t s = it % kStages, ph = (it / kStages) & 1u;
          if (!mbar_wait(&full[s], ph, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_u32(ring + (size_t)s * kStageBytes);
#pragma unroll
          for (int ks = 0; ks < kBoxL / 16; ++ks) {
            const uint64_t ad = smem_desc(a_base + ks * 2048, 8192, 1024, kSwizzle128);
            const uint32_t b_chunk = b_base + J.b_off + (uint32_t)(kc * N2 * 128);
            const uint64_t bd = smem_desc(b_chunk + ks * 256, 128, 1024, kSwizzleNone);
            mma_bf16(d_tmem, ad, bd, idesc_full, (kc > 0 || ks > 0) ? 1u : 0u);
          }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&tfull[buf]);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const uint32_t group = (uint32_t)(warp - 2) / 4u;
    uint32_t tcount = group;
    for (int64_t w = blockIdx.x + (int64_t)group * gridDim.x; w < P.units;
         w += (int64_t)kEpiGroups * gridDim.x, tcount += kEpiGroups) {
      const PairTile t = pair_decode(P, w);
      const PairJob& J = P.job[t.j];
      const uint32_t buf = tcount % kAccBufs, aph = (tcount / kAccBufs) & 1u;
      if (!mbar_wait(&tfull[buf], aph, abort_flag)) break;
      tc_fence_after();
      const uint32_t tbase = tmem_base + ((uint32_t)(q * 32) << 16) + buf * (uint32_t)N2max;
      const int64_t c = t.c0 + row;
      int64_t ystride;
      TOut* yp;
      if (J.block_c) {
        ystride = P.G * J.S;
        yp = static_cast<TOut*>(J.Y) + (t.r * J.K) * ystride + t.g * J.S + c;
      } else {
        ystride = J.S;
        yp = static_cast<TOut*>(J.Y) + (t.r * J.K) * ystride + c;
      }
      float hi[16], lo[16];
      for (int k0 = 0; k0 < J.Np; k0 += 16) {
        tmem_ld16(tbase + k0, hi);
        tmem_ld16(tbase + J.Np + k0, lo);
        tmem_wait_ld();
        if (k0 + 16 >= J.Np) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[buf]);
        }
        // Y of either job holds R * G * K * S values (mode a: [R][K][G * S];
        // mode b: [R * G][K][S])
        const int64_t yo = yp - static_cast<TOut*>(J.Y);
        if (c < J.S && TK_DBG_IN(yo, yo + (int64_t)(J.K - 1) * ystride, J.R * P.G * J.K * J.S)) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (k0 + j < J.K) yp[(int64_t)(k0 + j) * ystride] = to_out<TOut>(hi[j] + lo[j]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(ncols));
  }
}

// One thread waits, through the kernels' bounded wait, on an mbarrier that no
// thread or copy ever completes: the wait gives up after its time limit and
// records TUCKER_ERR_TIMEOUT in the device error word, and the kernel returns
// normally (the failure path of the pipelines, exercised without a fault).
__global__ void wait_selftest_kernel(int* returned) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const bool ok = mbar_wait(&bar, 0u, &abort_flag);
    *returned = ok ? 1 : 2;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                              const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                              const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}

}  // namespace

int make_map(CUtensorMap* m, const void* base, int rank, const cuuint64_t* dims,
             const cuuint64_t* strides_bytes, const cuuint32_t* box, CUtensorMapDataType dtype,
             CUtensorMapSwizzle swz) {
  EncodeFn enc = encoder();
  if (!enc) return fail(TUCKER_ERR_CUDA, "ttm_tc: cuTensorMapEncodeTiled unavailable");
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(m, dtype, (cuuint32_t)rank, const_cast<void*>(base), dims, strides_bytes,
                         box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TUCKER_ERR_CUDA, "ttm_tc: cuTensorMapEncodeTiled failed");
  return TUCKER_OK;
}

int* device_status_ptr() {
  static int* ptr = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tk_status) == cudaSuccess) ptr = static_cast<int*>(p);
  });
  return ptr;
}

namespace {


size_t smem_bytes(int Np, int nk, bool split_a) {
  const size_t stages = (size_t)stages_for(split_a);
  const size_t ring = stages * (split_a ? 2 : 1) * kStageBytes;
  const size_t b = (size_t)nk * 2 * Np * 128;
  return 1024 + ring + ((b + 15) & ~size_t(15)) + (2 * stages + 2 * kAccBufs) * 8 + 16;
}

template <bool kRows, bool kSplitA, typename TOut>
int launch_variant(const CUtensorMap& mh, const CUtensorMap& ml, void* Y, const TcParams& P,
                   size_t smem, cudaStream_t s) {
  auto kern = ttm_tc_kernel<kRows, kSplitA, TOut>;
  TK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t grid = std::min<int64_t>(P.tiles, sm_count());
  kern<<<(unsigned)grid, kThreads, smem, s>>>(mh, ml, static_cast<TOut*>(Y), P);
  TK_LAUNCH_CHECK("ttm_tc");
  return TUCKER_OK;
}

}  // namespace

// Whether the tensor-core TTM handles this shape: BF16 tensor, 16-byte
// aligned rows for TMA (C % 8 == 0 in the column case, L % 8 == 0 in the row
// case), K <= 64 and L <= 1024 (B stays resident in shared memory).
bool ttm_tc_supported(int64_t R, int64_t L, int64_t C, int64_t K, const void* X, const void* X_lo) {
  if (K < 1 || K > 64 || L < 1 || L > 1024) return false;
  if ((uintptr_t)X % 16 != 0 || (X_lo && (uintptr_t)X_lo % 16 != 0)) return false;
  if (R > INT32_MAX || C > INT32_MAX) return false;
  if (C == 1) return L % 8 == 0 && R >= 1;
  return C % 8 == 0 && C >= 64;
}

bool ttm_tc_split_fits(int64_t R, int64_t L, int64_t C, int64_t K) {
  if (!ttm_tc_supported(R, L, C, K, nullptr, nullptr)) return false;
  const int Np = (int)((K + 15) / 16 * 16), nk = (int)((L + kBoxL - 1) / kBoxL);
  return smem_bytes(Np, nk, true) <= 227 * 1024;
}

// Share of a tensor-core tile's work that is the TTM's own: l runs in stages
// of 64 (the last one zero-filled past L) and the column case tiles each
// r-slab's C positions by 128 (by 64, two slabs per tile, at C = 64).
double ttm_tc_efficiency(int64_t L, int64_t C) {
  const double el = (double)L / (double)(kBoxL * ((L + kBoxL - 1) / kBoxL));
  if (C <= 64) return el;
  return el * (double)C / (double)(kTileM * ((C + kTileM - 1) / kTileM));
}

// Y (K outputs, FP32 or BF16) = X x_n F^T with X (and optionally X_lo) BF16.
int launch_ttm_tc(const void* X, const void* X_lo, int64_t R, int64_t L, int64_t C,
                  const float* F, int64_t K, void* Y, bool y_bf16, cudaStream_t s) {
  if (!ttm_tc_supported(R, L, C, K, X, X_lo))
    return fail(TUCKER_ERR_UNSUPPORTED, "ttm_tc: shape or alignment not supported");
  TcParams P{};
  P.R = R;
  P.C = C;
  P.L = (int)L;
  P.K = (int)K;
  P.Np = (int)((K + 15) / 16 * 16);
  P.nk = (int)((L + kBoxL - 1) / kBoxL);
  P.F = F;
  const bool rows = (C == 1);
  const size_t ysz = y_bf16 ? 2 : 4;
  P.vec_rows = rows && ((uintptr_t)Y % 16 == 0) && ((size_t)K * ysz % 16 == 0);
  P.pack2 = (!rows && C == 64) ? 1 : 0;
  CUtensorMap mh, ml;
  if (rows) {
    P.tiles = (R + kTileM - 1) / kTileM;
    P.ctiles = 1;
    const cuuint64_t dims[2] = {(cuuint64_t)L, (cuuint64_t)R};
    const cuuint64_t str[1] = {(cuuint64_t)L * 2};
    const cuuint32_t box[2] = {kBoxL, kTileM};
    int rc = make_map(&mh, X, 2, dims, str, box);
    if (rc) return rc;
    rc = make_map(&ml, X_lo ? X_lo : X, 2, dims, str, box);
    if (rc) return rc;
  } else {
    P.ctiles = (C + kTileM - 1) / kTileM;
    P.tiles = P.pack2 ? (R + 1) / 2 : R * P.ctiles;
    const cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)L, (cuuint64_t)R};
    const cuuint64_t str[2] = {(cuuint64_t)C * 2, (cuuint64_t)C * L * 2};
    const cuuint32_t box[3] = {64, kBoxL, P.pack2 ? 2u : 1u};
    int rc = make_map(&mh, X, 3, dims, str, box);
    if (rc) return rc;
    rc = make_map(&ml, X_lo ? X_lo : X, 3, dims, str, box);
    if (rc) return rc;
  }
  const bool split = X_lo != nullptr;
  const size_t smem = smem_bytes(P.Np, P.nk, split);
  if (smem > 227 * 1024) return fail(TUCKER_ERR_UNSUPPORTED, "ttm_tc: shared memory");
  if (rows) {
    if (split)
      return y_bf16 ? launch_variant<true, true, bf16_t>(mh, ml, Y, P, smem, s)
                    : launch_variant<true, true, float>(mh, ml, Y, P, smem, s);
    return y_bf16 ? launch_variant<true, false, bf16_t>(mh, ml, Y, P, smem, s)
                  : launch_variant<true, false, float>(mh, ml, Y, P, smem, s);
  }
  if (split)
    return y_bf16 ? launch_variant<false, true, bf16_t>(mh, ml, Y, P, smem, s)
                  : launch_variant<false, true, float>(mh, ml, Y, P, smem, s);
  return y_bf16 ? launch_variant<false, false, bf16_t>(mh, ml, Y, P, smem, s)
                : launch_variant<false, false, float>(mh, ml, Y, P, smem, s);
}

// The BF16 root pair (ttm_tc_pair_kernel): modes a and b = a + 2 of a BF16
// tensor blocked by mode a + 1; S = prod dims[a+2..] and C_b = prod
// dims[b+1..] multiples of 8 (16-byte TMA coordinates) and >= 64, K <= 64,
// L <= 1024, both B operands within shared memory, 32-bit coordinates.
bool ttm_tc_pair_supported(const int64_t* dims, int N, int a, int b, int64_t Ka, int64_t Kb, const void* X) {
  if (a < 0 || b != a + 2 || b >= N) return false;
  if (Ka < 1 || Ka > 64 || Kb < 1 || Kb > 64 || dims[a] > 1024 || dims[b] > 1024) return false;
  const int m = a + 1;
  const int64_t S = prod(dims, m + 1, N), Cb = prod(dims, b + 1, N);
  if (S < 64 || S % 8 != 0 || Cb < 64 || Cb % 8 != 0) return false;
  if ((uintptr_t)X % 16 != 0 || S * dims[m] > INT32_MAX || prod(dims, 0, a) > INT32_MAX ||
      prod(dims, 0, b) > INT32_MAX)
    return false;
  const int64_t Npa = (Ka + 15) / 16 * 16, Npb = (Kb + 15) / 16 * 16;
  const size_t bb = (size_t)((dims[a] + kBoxL - 1) / kBoxL) * 2 * Npa * 128 +
                    (size_t)((dims[b] + kBoxL - 1) / kBoxL) * 2 * Npb * 128;
  const size_t smem = 1024 + (size_t)kStagesPlain * kStageBytes + ((bb + 15) & ~size_t(15)) +
                      (2 * kStagesPlain + 2 * kAccBufs) * 8 + 16;
  return smem <= 227 * 1024 && 4 * 2 * std::max(Npa, Npb) <= 512;
}

int launch_ttm_tc_pair(const void* X, const int64_t* dims, int N, int a, int b, const float* Fa, int64_t Ka,
                       const float* Fb, int64_t Kb, void* Ya, void* Yb, bool y_bf16, cudaStream_t s) {
  if (!ttm_tc_pair_supported(dims, N, a, b, Ka, Kb, X))
    return fail(TUCKER_ERR_UNSUPPORTED, "ttm_tc_pair: shape or alignment not supported");
  const int m = a + 1;
  PairParams P{};
  P.G = dims[m];
  PairJob& A = P.job[0];
  A.L = (int)dims[a];
  A.K = (int)Ka;
  A.Np = (int)((Ka + 15) / 16 * 16);
  A.nk = (int)((dims[a] + kBoxL - 1) / kBoxL);
  A.block_c = 1;
  A.R = prod(dims, 0, a);
  A.S = prod(dims, m + 1, N);
  A.ct = (A.S + kTileM - 1) / kTileM;
  A.per_block = A.R * A.ct;
  A.b_off = 0;
  A.F = Fa;
  A.Y = Ya;
  PairJob& B = P.job[1];
  B.L = (int)dims[b];
  B.K = (int)Kb;
  B.Np = (int)((Kb + 15) / 16 * 16);
  B.nk = (int)((dims[b] + kBoxL - 1) / kBoxL);
  B.block_c = 0;
  B.R = prod(dims, 0, m);
  B.S = prod(dims, b + 1, N);
  B.ct = (B.S + kTileM - 1) / kTileM;
  B.per_block = B.R * B.ct;
  B.b_off = (uint32_t)((size_t)A.nk * 2 * A.Np * 128);
  B.F = Fb;
  B.Y = Yb;
  P.per_block = A.per_block + B.per_block;
  P.units = P.G * P.per_block;
  CUtensorMap ma, mb;
  {
    const int64_t Ca = P.G * A.S;
    const cuuint64_t d3[3] = {(cuuint64_t)Ca, (cuuint64_t)A.L, (cuuint64_t)A.R};
    const cuuint64_t st[2] = {(cuuint64_t)Ca * 2, (cuuint64_t)(Ca * A.L) * 2};
    const cuuint32_t box[3] = {64, kBoxL, 1};
    const int rc = make_map(&ma, X, 3, d3, st, box);
    if (rc) return rc;
  }
  {
    const cuuint64_t d3[3] = {(cuuint64_t)B.S, (cuuint64_t)B.L, (cuuint64_t)prod(dims, 0, b)};
    const cuuint64_t st[2] = {(cuuint64_t)B.S * 2, (cuuint64_t)(B.S * B.L) * 2};
    const cuuint32_t box[3] = {64, kBoxL, 1};
    const int rc = make_map(&mb, X, 3, d3, st, box);
    if (rc) return rc;
  }
  const size_t bb = (size_t)B.b_off + (size_t)B.nk * 2 * B.Np * 128;
  const size_t smem = 1024 + (size_t)kStagesPlain * kStageBytes + ((bb + 15) & ~size_t(15)) +
                      (2 * kStagesPlain + 2 * kAccBufs) * 8 + 16;
  const int64_t grid = std::min<int64_t>(P.units, sm_count());
  if (y_bf16) {
    auto kern = ttm_tc_pair_kernel<bf16_t>;
    TK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)grid, kThreads, smem, s>>>(ma, mb, P);
  } else {
    auto kern = ttm_tc_pair_kernel<float>;
    TK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)grid, kThreads, smem, s>>>(ma, mb, P);
  }
  TK_LAUNCH_CHECK("ttm_tc_pair");
  return TUCKER_OK;
}

size_t smem_bytes_f32(int Np, int nk) {
  return 1024 + (size_t)kF32St * kF32StageBytes + (size_t)kF32Cv * kF32CvBytes +
         (((size_t)nk * 3 * Np * 128 + 15) & ~size_t(15)) + (2 * kF32St + 2 * kF32Cv + 2 * kAccBufs) * 8 +
         16;
}

// FP32 column-case TTM on the tensor cores: C % 4 == 0 (16-byte TMA strides),
// C >= 64, K <= 32 (four accumulator buffers of 3 Np columns in TMEM), and B
// plus the rings within shared memory.
bool ttm_tc_f32_supported(int64_t R, int64_t L, int64_t C, int64_t K, const void* X) {
  if (K < 1 || K > 32 || L < 1 || L > 1024 || C < 64 || C % 4 != 0) return false;
  if ((uintptr_t)X % 16 != 0 || R > INT32_MAX || C > INT32_MAX) return false;
  const int Np = (int)((K + 15) / 16 * 16), nk = (int)((L + kBoxL - 1) / kBoxL);
  return smem_bytes_f32(Np, nk) <= 227 * 1024;
}

int launch_ttm_tc_f32(const float* X, int64_t R, int64_t L, int64_t C, const float* F, int64_t K,
                      float* Y, cudaStream_t s) {
  if (!ttm_tc_f32_supported(R, L, C, K, X))
    return fail(TUCKER_ERR_UNSUPPORTED, "ttm_tc_f32: shape or alignment not supported");
  TcParams P{};
  P.R = R;
  P.C = C;
  P.L = (int)L;
  P.K = (int)K;
  P.Np = (int)((K + 15) / 16 * 16);
  P.nk = (int)((L + kBoxL - 1) / kBoxL);
  P.F = F;
  P.ctiles = (C + kTileM - 1) / kTileM;
  P.tiles = R * P.ctiles;
  CUtensorMap mx;
  const cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)L, (cuuint64_t)R};
  const cuuint64_t str[2] = {(cuuint64_t)C * 4, (cuuint64_t)C * L * 4};
  const cuuint32_t box[3] = {(cuuint32_t)kTileM, (cuuint32_t)kBoxL, 1u};
  int rc = make_map(&mx, X, 3, dims, str, box, CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    CU_TENSOR_MAP_SWIZZLE_NONE);
  if (rc) return rc;
  const size_t smem = smem_bytes_f32(P.Np, P.nk);
  auto kern = ttm_tc_f32_kernel<float>;
  TK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t grid = std::min<int64_t>(P.tiles, sm_count());
  kern<<<(unsigned)grid, kF32Threads, smem, s>>>(mx, Y, P);
  TK_LAUNCH_CHECK("ttm_tc_f32");
  return TUCKER_OK;
}

size_t smem_bytes_fp8(int Np, int nk) {
  return 1024 + (size_t)kF8St * kF8StageBytes + (size_t)kF8Cv * kF8CvBytes + (size_t)kF8St * kF8ScaleBytes +
         (((size_t)nk * 2 * Np * 128 + 15) & ~size_t(15)) + (2 * kF8St + 2 * kF8Cv + 2 * kAccBufs) * 8 + 16;
}

// FP8 column-case TTM on the tensor cores: C % 256 == 0 (each 64-column half
// of a tile row is one scale block, and a scale row of C / 64 floats has a
// 16-byte TMA stride), K <= 32, codes 16-byte aligned, R * L within 32-bit
// TMA coordinates, B and the rings within shared memory.
bool ttm_tc_fp8_supported(int64_t R, int64_t L, int64_t C, int64_t K, const void* X) {
  if (K < 1 || K > 32 || L < 1 || L > 1024 || C < 256 || C % 256 != 0) return false;
  if ((uintptr_t)X % 16 != 0 || R > INT32_MAX || C > INT32_MAX || R * L + kBoxL > INT32_MAX) return false;
  const int Np = (int)((K + 15) / 16 * 16), nk = (int)((L + kBoxL - 1) / kBoxL);
  return smem_bytes_fp8(Np, nk) <= 227 * 1024;
}

int launch_ttm_tc_fp8(const void* Xq, const float* scales, int64_t R, int64_t L, int64_t C,
                      const float* F, int64_t K, void* Y, bool y_bf16, cudaStream_t s) {
  if (!ttm_tc_fp8_supported(R, L, C, K, Xq))
    return fail(TUCKER_ERR_UNSUPPORTED, "ttm_tc_fp8: shape or alignment not supported");
  TcParams P{};
  P.R = R;
  P.C = C;
  P.L = (int)L;
  P.K = (int)K;
  P.Np = (int)((K + 15) / 16 * 16);
  P.nk = (int)((L + kBoxL - 1) / kBoxL);
  P.F = F;
  P.ctiles = (C + kTileM - 1) / kTileM;
  P.tiles = R * P.ctiles;
  CUtensorMap mq;
  const cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)L, (cuuint64_t)R};
  const cuuint64_t str[2] = {(cuuint64_t)C, (cuuint64_t)C * L};
  const cuuint32_t box[3] = {(cuuint32_t)kTileM, (cuuint32_t)kBoxL, 1u};
  int rc = make_map(&mq, Xq, 3, dims, str, box, CU_TENSOR_MAP_DATA_TYPE_UINT8, CU_TENSOR_MAP_SWIZZLE_NONE);
  if (rc) return rc;
  // the scales as [R L] rows of C / 64 floats; a box of 4 columns x 64 rows
  CUtensorMap ms;
  const cuuint64_t sdims[2] = {(cuuint64_t)(C / 64), (cuuint64_t)(R * L)};
  const cuuint64_t sstr[1] = {(cuuint64_t)(C / 64) * 4};
  const cuuint32_t sbox[2] = {4u, (cuuint32_t)kBoxL};
  rc = make_map(&ms, scales, 2, sdims, sstr, sbox, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, CU_TENSOR_MAP_SWIZZLE_NONE);
  if (rc) return rc;
  const size_t smem = smem_bytes_fp8(P.Np, P.nk);
  const int64_t grid = std::min<int64_t>(P.tiles, sm_count());
  if (y_bf16) {
    auto kern = ttm_tc_fp8_kernel<bf16_t>;
    TK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)grid, kF8Threads, smem, s>>>(mq, ms, static_cast<bf16_t*>(Y), P);
  } else {
    auto kern = ttm_tc_fp8_kernel<float>;
    TK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)grid, kF8Threads, smem, s>>>(mq, ms, static_cast<float*>(Y), P);
  }
  TK_LAUNCH_CHECK("ttm_tc_fp8");
  return TUCKER_OK;
}

}  // namespace tk

namespace tk {
namespace {
std::atomic<int> g_policy{0};
}
int kernel_policy() { return g_policy.load(std::memory_order_relaxed); }
}  // namespace tk

extern "C" int tucker_set_kernel_policy(int policy) {
  if (policy < 0 || policy > 2047)
    return tk::fail(TUCKER_ERR_INVALID_ARG, "tucker_set_kernel_policy: policy must be in [0, 2047]");
  tk::g_policy.store(policy, std::memory_order_relaxed);
  return TUCKER_OK;
}

extern "C" int tucker_selftest_wait_timeout(int* outcome, void* stream) {
  if (!outcome) return tk::fail(TUCKER_ERR_INVALID_ARG, "tucker_selftest_wait_timeout: NULL");
  int* d = nullptr;
  TK_CUDA_TRY(cudaMalloc(&d, sizeof(int)));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    tk::wait_selftest_kernel<<<1, 32, 0, s>>>(d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(outcome, d, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess)
    return tk::fail(TUCKER_ERR_CUDA, std::string("tucker_selftest_wait_timeout: ") + cudaGetErrorString(e));
  tk::count_launches(1);
  return TUCKER_OK;
}

extern "C" int tucker_device_status(int* status, int reset) {
  if (!status) return tk::fail(TUCKER_ERR_INVALID_ARG, "tucker_device_status: NULL");
  TK_CUDA_TRY(cudaMemcpyFromSymbol(status, tk::g_tk_status, sizeof(int)));
  if (reset) {
    const int zero = 0;
    TK_CUDA_TRY(cudaMemcpyToSymbol(tk::g_tk_status, &zero, sizeof(int)));
  }
  return TUCKER_OK;
}
