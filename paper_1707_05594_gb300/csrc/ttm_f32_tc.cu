// ttm_f32_tc.cu -- FP32 mode-n TTM on the 5th-generation tensor cores:
// Out = In x_n F^T (Sec. 2.1) for FP32 tensors, column case (mode not
// last), transposition-free, in two forms:
//   - ttm_x3_kernel (opt-in, kernel policy bit 32): exact integer slices in
//     BF16 (further below), no rounding inside the tensor core;
//   - ttm_tf32_kernel (opt-in, kernel policy bit 64): tcgen05.mma kind::tf32
//     with split operands, described here.
// Both are slower than the CUDA-core column TTM on the 200^4 root (measured
// 2.52 and 2.02 ms against 1.48 ms): ncu shows them latency- and issue-bound
// (DRAM 34 % / 43 % of peak, issue 56 % / 37 %), the exact-slice converter
// costing ~13 instructions per element, so the CUDA cores stay the default.
//
// Precision: TF32 keeps 11 significant bits, so each operand is split into a
// TF32 high part and a low remainder, x = x_hi + x_lo and f = f_hi + f_lo
// (x_hi by Veltkamp's splitting with the factor 2^13 + 1, which leaves 11
// significant bits; x_lo = x - x_hi exactly), and three products are
// accumulated: x_hi f_hi + x_hi f_lo + x_lo f_hi.  The dropped term x_lo f_lo
// and the 19 bits the tensor core reads of the remainders move a product by
// a few 2^-23 |x f|, so the contraction is as accurate as FP32 arithmetic.
//
// GEMM view per tile: D[128 positions, N] = A[128 x l] B[l x N], where the
// 128 positions are consecutive c of one row r of the [R][L][C] view.
//   - TMA brings In[r, l0:l0+64, c0:c0+128] as a 32 KB FP32 tile (rows of 128
//     positions) into a shared-memory ring;
//   - eight converter warps split it: thread p of a warp takes position p of
//     its TMEM lane quarter and 32 of the 64 l, and writes x_hi and x_lo into
//     tensor memory (tcgen05.st), so that A is read by the MMA from TMEM and
//     shared-memory bandwidth is left to TMA and B;
//   - one thread issues, per k-step of 8 l, A_hi x [F_hi | F_lo] (N = 2 Kp)
//     and A_lo x F_hi (N = Kp, the first Kp rows of the same B);
//   - four epilogue warps read the accumulator (tcgen05.ld), add the halves
//     and store Y with coalesced 128-byte rows.
// With `chunk_acc` each 64-l chunk accumulates into a fresh TMEM buffer and
// the epilogue adds the chunk sums in FP32 registers (rounded to nearest), so
// at most eight k-steps share the tensor core's accumulator.
//
// Two jobs (L2-blocked root pair).  A sweep's two root children read the same
// tensor T along two modes a < b.  With the mode m = a + 1 < b as the block
// index, job A (mode a) sees T as [R_a][L_a][L_m * S] (tiles of 128 of the S
// positions of one block) and job B (mode b) as
// [R_hi][L_m][R_lo][L_b][C_b]; the work list runs block after block (value
// of i_m), each block's job-A tiles then its job-B tiles, so that the block
// of T (|T| / L_m elements, tens of MB) is read from HBM once and found in
// the 126 MB L2 by the second job.
//
// Warp roles (448 threads, one CTA per SM, persistent): warp 0 TMA producer,
// warp 1 TMEM allocation + MMA issuer, warps 2-9 converters, warps 10-13
// epilogue.  Every wait is bounded (%globaltimer); on timeout the kernel
// records TUCKER_ERR_TIMEOUT in the library's device error word, drains its
// own copies, frees TMEM and returns.
#include <algorithm>

#include "tc_common.cuh"

namespace tk {
namespace {

using namespace tc;

constexpr int kT32BoxL = 64;                              // l per stage
constexpr int kT32TileM = 128;                            // positions per tile
constexpr int kT32StageBytes = kT32TileM * kT32BoxL * 4;  // 32 KB FP32 tile
constexpr int kT32AStages = 2;     // TMEM A stages: [x_hi 64 cols | x_lo 64 cols]
constexpr int kT32AStageCols = 128;
constexpr int kT32AccBufs = 4;     // TMEM accumulators of 64 columns
constexpr int kT32AccCols = 64;    // 2 * Kp <= 64
constexpr uint32_t kT32TmemCols = 512;
constexpr int kT32CvWarps = 8;
constexpr int kT32EpiWarps = 4;
constexpr int kT32Threads = 64 + 32 * (kT32CvWarps + kT32EpiWarps);
constexpr int kT32MaxStages = 6;

enum : int { kJobPlain = 0, kJobBlockC = 1, kJobBlockR = 2 };

struct Tf32Job {
  int type;          // kJobPlain: [R][L][C];  kJobBlockC: [R][L][G*S];  kJobBlockR: [Rh][G][Rl][L][C]
  int L, K, Kp, nk;  // contraction length, outputs, K rounded to 16, 64-l chunks
  int64_t R;         // rows (plain, block-C) or Rh (block-R)
  int64_t Rl;        // block-R: rows after the block mode
  int64_t S;         // positions per row: C (plain, block-R) or S (block-C)
  int64_t ct;        // 128-position tiles per row
  int64_t per_block; // tiles per block
  float* Y;
  uint32_t b_off;    // byte offset of this job's B in shared memory
};

struct Tf32Params {
  Tf32Job job[2];
  int njobs;
  int stages;          // TMA ring depth
  int chunk_acc;       // fresh accumulator per 64-l chunk, chunks summed in registers
  int64_t G;           // blocks
  int64_t per_block;   // tiles of both jobs per block
  int64_t units;       // G * per_block
  const float* F[2];
  int* status;         // the library's device error word
};

// Values of a job's Y: R * K * S (plain), R * K * G * S (block-C: rows of
// G * S positions) or R * G * Rl * K * S (block-R: the block mode between
// the row indices).
__device__ __forceinline__ int64_t y_total(const Tf32Job& J, int64_t G) {
  const int64_t base = J.R * (int64_t)J.K * J.S;
  return J.type == kJobPlain ? base : J.type == kJobBlockC ? base * G : base * G * J.Rl;
}

// idesc for kind::tf32: D FP32, A and B TF32, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kT32TileM >> 4) << 24);
}

// D (TMEM) += A (TMEM) * B (shared memory descriptor)
__device__ __forceinline__ void mma_tf32_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// 32 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
      "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
      "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
      "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
      "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
      "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Veltkamp's splitting of an FP32 value with the factor 2^13 + 1: hi keeps
// 24 - 13 = 11 significant bits (a TF32 value), x - hi is exact.  The
// roundings must not be contracted into fused multiply-adds.
__device__ __forceinline__ float tf32_hi(float x) {
  const float c = __fmul_rn(x, 8193.0f);
  return __fsub_rn(c, __fsub_rn(c, x));
}

// Where unit w of the work list lies: its job, and the TMA coordinates and
// output placement of its tile.
struct Tile {
  int j;           // job
  int64_t r;       // row of the [R][L][C] view (the global row for block-R)
  int64_t c0;      // first position within the row's S (block-C) or C
  int64_t g;       // block
};

// The work list runs block after block (value of the block mode), each
// block's job-0 tiles and then its job-1 tiles (an interleaved order measured
// slower, as for the BF16 pair).
__device__ __forceinline__ Tile decode(const Tf32Params& P, int64_t w) {
  Tile t;
  t.g = w / P.per_block;
  int64_t i = w - t.g * P.per_block;
  t.j = 0;
  if (P.njobs > 1 && i >= P.job[0].per_block) {
    i -= P.job[0].per_block;
    t.j = 1;
  }
  const Tf32Job& J = P.job[t.j];
  const int64_t row = i / J.ct;
  t.c0 = (i - row * J.ct) * kT32TileM;
  if (J.type == kJobBlockR) {
    const int64_t rh = row / J.Rl, rl = row - rh * J.Rl;
    t.r = (rh * P.G + t.g) * J.Rl + rl;
  } else {
    t.r = row;
  }
  return t;
}

// SMEM (dynamic, 1024-aligned): [ring: stages x 32 KB][B of job 0][B of job 1]
//   [barriers][tmem slot][abort flag]
// B of a job: F split [F_hi | F_lo]^T (N1 = 2 Kp rows), K-major without
// swizzle, one 64-l chunk after another: core matrices of 8 rows x 4 l
// (16 B rows), LBO = 128 B between l-groups, SBO = 16 * 128 = 2048 B between
// 8-row groups, N1 * 256 B per chunk.
__global__ void __launch_bounds__(kT32Threads, 1)
    ttm_tf32_kernel(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
                    const Tf32Params P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t nst = (uint32_t)P.stages;
  unsigned char* ring = smem;
  unsigned char* bsm = ring + (size_t)nst * kT32StageBytes;
  size_t b_end = 0;
  for (int j = 0; j < P.njobs; ++j)
    b_end = std::max(b_end, (size_t)P.job[j].b_off + (size_t)P.job[j].nk * 2 * P.job[j].Kp * 256);
  uint64_t* bars = reinterpret_cast<uint64_t*>(bsm + ((b_end + 15) & ~size_t(15)));
  uint64_t* st_full = bars;                       // nst
  uint64_t* st_empty = st_full + nst;             // nst
  uint64_t* a_full = st_empty + nst;              // kT32AStages
  uint64_t* a_empty = a_full + kT32AStages;       // kT32AStages
  uint64_t* acc_full = a_empty + kT32AStages;     // kT32AccBufs
  uint64_t* acc_empty = acc_full + kT32AccBufs;   // kT32AccBufs
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + kT32AccBufs);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < nst; ++s) {
      mbar_init(&st_full[s], 1);
      mbar_init(&st_empty[s], kT32CvWarps);
    }
    for (int s = 0; s < kT32AStages; ++s) {
      mbar_init(&a_full[s], kT32CvWarps);
      mbar_init(&a_empty[s], 1);
    }
    for (int b = 0; b < kT32AccBufs; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kT32EpiWarps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B operands
  for (int j = 0; j < P.njobs; ++j) {
    const Tf32Job& J = P.job[j];
    const int N1 = 2 * J.Kp, lpad = J.nk * kT32BoxL;
    const float* F = P.F[j];
    for (int idx = threadIdx.x; idx < N1 * lpad; idx += kT32Threads) {
      const int row = idx / lpad, l = idx - row * lpad;
      const int k = row < J.Kp ? row : row - J.Kp;
      float f = 0.f;
      if (k < J.K && l < J.L) f = F[(int64_t)l * J.K + k];
      const float hi = tf32_hi(f);
      const float v = row < J.Kp ? hi : __fsub_rn(f, hi);
      const int chunk = l / kT32BoxL, lc = l - chunk * kT32BoxL;
      const size_t off = (size_t)J.b_off + (size_t)chunk * N1 * 256 + (size_t)(row >> 3) * 2048 +
                         (size_t)(lc >> 2) * 128 + (size_t)(row & 7) * 16 + (size_t)(lc & 3) * 4;
      *reinterpret_cast<float*>(bsm + off) = v;
    }
  }
  // generic-proxy writes of B must be visible to the tensor core (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kT32TmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint32_t acc_col0 = kT32AStages * kT32AStageCols;  // accumulators after the A stages

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t w = blockIdx.x; w < P.units && ok; w += gridDim.x) {
        const Tile t = decode(P, w);
        const Tf32Job& J = P.job[t.j];
        const CUtensorMap* map = t.j == 0 ? &map0 : &map1;
        for (int kc = 0; kc < J.nk; ++kc, ++it) {
          const uint32_t s = it % nst, ph = (it / nst) & 1u;
          if (!mbar_wait_sleep(&st_empty[s], ph ^ 1u, abort_flag, P.status)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&st_full[s], (uint32_t)kT32StageBytes);
          unsigned char* dst = ring + (size_t)s * kT32StageBytes;
          // block-C tiles address the row's positions g * S + c0 (a tile's
          // positions past S belong to the next block and are not stored)
          const int64_t cx = J.type == kJobBlockC ? t.g * J.S + t.c0 : t.c0;
          tma_load_3d(dst, map, &st_full[s], (int)cx, kc * kT32BoxL, (int)t.r);
        }
      }
      // drain: wait (bounded) until every copy issued has landed
      const uint32_t issued = it;
      for (uint32_t j = (issued > nst ? issued - nst : 0); j < issued; ++j) {
        const uint32_t s = j % nst, ph = (j / nst) & 1u;
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(&st_full[s], ph) && globaltimer() - t0 < kTimeoutNs) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t b_base = smem_u32(bsm);
      uint32_t it = 0, cnt = 0;
      bool ok = true;
      for (int64_t w = blockIdx.x; w < P.units && ok; w += gridDim.x) {
        const Tile t = decode(P, w);
        const Tf32Job& J = P.job[t.j];
        const int N1 = 2 * J.Kp;
        const uint32_t id1 = idesc_tf32(N1), id2 = idesc_tf32(J.Kp);
        uint32_t d_tmem = 0, buf = 0;
        for (int kc = 0; kc < J.nk; ++kc, ++it) {
          if (P.chunk_acc || kc == 0) {
            buf = cnt % kT32AccBufs;
            if (!mbar_wait_sleep(&acc_empty[buf], ((cnt / kT32AccBufs) & 1u) ^ 1u, abort_flag, P.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            d_tmem = tmem_base + acc_col0 + buf * (uint32_t)kT32AccCols;
          }
          const uint32_t as = it % kT32AStages, aph = (it / kT32AStages) & 1u;
          if (!mbar_wait_sleep(&a_full[as], aph, abort_flag, P.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int lval = min(kT32BoxL, J.L - kc * kT32BoxL);
          const int nks = (lval + 7) >> 3;
          const uint32_t a_hi = tmem_base + as * (uint32_t)kT32AStageCols;
          const uint32_t b_chunk = b_base + J.b_off + (uint32_t)(kc * N1 * 256);
          for (int ks = 0; ks < nks; ++ks) {
            const uint64_t bd = smem_desc(b_chunk + ks * 256, 128, 2048, kSwizzleNone);
            const uint32_t acc = (ks > 0 || (kc > 0 && !P.chunk_acc)) ? 1u : 0u;
            mma_tf32_ts(d_tmem, a_hi + ks * 8, bd, id1, acc);
            mma_tf32_ts(d_tmem, a_hi + kT32BoxL + ks * 8, bd, id2, 1u);
          }
          mma_commit(&a_empty[as]);
          if (P.chunk_acc || kc == J.nk - 1) {
            mma_commit(&acc_full[buf]);
            ++cnt;
          }
        }
      }
    }
  } else if (warp < 2 + kT32CvWarps) {
    // ------------------------------------------------------------ converters
    const int q = warp & 3;                      // TMEM lane quarter
    const int half = (warp - 2) / 4;             // which 32 l of a stage
    const int p = q * 32 + lane;                 // tile position = TMEM lane
    uint32_t it = 0;
    bool ok = true;
    for (int64_t w = blockIdx.x; w < P.units && ok; w += gridDim.x) {
      const Tile t = decode(P, w);
      const Tf32Job& J = P.job[t.j];
      for (int kc = 0; kc < J.nk; ++kc, ++it) {
        const uint32_t s = it % nst, ph = (it / nst) & 1u;
        const uint32_t as = it % kT32AStages, aph = (it / kT32AStages) & 1u;
        if (!mbar_wait_sleep(&st_full[s], ph, abort_flag, P.status) ||
            !mbar_wait_sleep(&a_empty[as], aph ^ 1u, abort_flag, P.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int lval = min(kT32BoxL, J.L - kc * kT32BoxL) - half * 32;
        if (lval > 0) {
          // rows past L and positions past the row were zero-filled by TMA
          const float* src = reinterpret_cast<const float*>(ring + (size_t)s * kT32StageBytes) +
                             (size_t)(half * 32) * kT32TileM + p;
          float hi[32], lo[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float x = src[i * kT32TileM];
            hi[i] = tf32_hi(x);
            lo[i] = __fsub_rn(x, hi[i]);
          }
          const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + as * (uint32_t)kT32AStageCols +
                              (uint32_t)(half * 32);
          tmem_st32(ta, hi);
          tmem_st32(ta + kT32BoxL, lo);
          tmem_wait_st();
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&a_full[as]);
          mbar_arrive(&st_empty[s]);
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    const int p = q * 32 + lane;
    uint32_t cnt = 0;
    bool ok = true;
    for (int64_t w = blockIdx.x; w < P.units && ok; w += gridDim.x) {
      const Tile t = decode(P, w);
      const Tf32Job& J = P.job[t.j];
      const int N1 = 2 * J.Kp;
      float acc[kT32AccCols];
#pragma unroll
      for (int i = 0; i < kT32AccCols; ++i) acc[i] = 0.f;
      const int nbuf = P.chunk_acc ? J.nk : 1;
      for (int b = 0; b < nbuf; ++b, ++cnt) {
        const uint32_t buf = cnt % kT32AccBufs;
        if (!mbar_wait_sleep(&acc_full[buf], (cnt / kT32AccBufs) & 1u, abort_flag, P.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tb = tmem_base + ((uint32_t)(q * 32) << 16) + acc_col0 + buf * (uint32_t)kT32AccCols;
#pragma unroll
        for (int k0 = 0; k0 < kT32AccCols; k0 += 16) {
          if (k0 < N1) {
            float v[16];
            tmem_ld16(tb + k0, v);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[k0 + i] += v[i];
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[buf]);
      }
      if (!ok) break;
      const int64_t c = t.c0 + p;
      if (c < J.S) {
        float* yp;
        int64_t ystride;
        if (J.type == kJobBlockC) {
          ystride = P.G * J.S;
          yp = J.Y + (t.r * J.K) * ystride + t.g * J.S + c;
        } else {
          ystride = J.S;
          yp = J.Y + (t.r * J.K) * ystride + c;
        }
        if (!TK_DBG_IN(yp - J.Y, (yp - J.Y) + (int64_t)(J.K - 1) * ystride, y_total(J, P.G))) continue;
        // columns [0, Kp): x_hi f_hi + x_lo f_hi; [Kp, 2 Kp): x_hi f_lo
        if (J.Kp == 16) {
#pragma unroll
          for (int k = 0; k < 16; ++k)
            if (k < J.K) yp[(int64_t)k * ystride] = acc[k] + acc[16 + k];
        } else {
#pragma unroll
          for (int k = 0; k < 32; ++k)
            if (k < J.K) yp[(int64_t)k * ystride] = acc[k] + acc[32 + k];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kT32TmemCols));
  }
}

// ---------------------------------------------------------------------------
// Exact slices.  The tensor core's FP32
// accumulation rounds toward zero (measured: over an L = 200 contraction the
// mean signed error of the TF32 kernel above is 0.8 of its mean absolute
// error), which biases every output toward zero and, through ||G||^2, the
// fit identity.  Here the tensor core never rounds: within a 64-l chunk each
// position p's values are scaled by a power of two s_p (the first power of
// two above their largest magnitude) and cut into three integer slices,
//   x * 2^6 / s_p = x0 + 2^-8 x1 + 2^-16 x2 (+ at most 2^-17),
// x0 in [-64, 64], x1, x2 in [-128, 128] (exact in BF16), and F's column k
// the same way with a power of two t_k per chunk.  The products of slices are
// exact and every sum of them over a chunk stays below 2^24, so the four
// groups g0 = sum x0 f0, g1 = sum (x0 f1 + x1 f0), g2 = sum (x0 f2 + x1 f1 +
// x2 f0), g3 = sum (x1 f2 + x2 f1) come out of the MMAs exactly; only the
// slicing (to nearest) and the epilogue's FP32 combination
//   y += (s_p t_k 2^-12) (g0 + ((2^-8 g1 + 2^-16 g2) + 2^-24 g3))
// round, so the result is as accurate as an FP32 contraction and unbiased.
//
// Per k-step of 16 l (kind::f16, BF16 slices, A from TMEM):
//   x0 [f0|f1|f2] -> columns [0, 3Kp),  x1 [f0|f1|f2] -> [Kp, 4Kp),
//   x2 [f0|f1] -> [2Kp, 4Kp);
// column group j of the accumulator is g_j.  The first MMA of a chunk starts
// the accumulator (columns [0, 3Kp)); the epilogue zeroes [3Kp, 4Kp) of a
// buffer when it hands it back, before the next chunk's second MMA adds to it.
//
// Roles as in the TF32 kernel; the two converter warps of a TMEM lane quarter
// exchange their halves' maxima through shared memory (an mbarrier per
// quarter, bounded wait) and the chunk's position scales reach the epilogue
// through an 8-deep shared-memory ring with its own full / empty barriers.
// ---------------------------------------------------------------------------
constexpr int kXAStageCols = 96;  // three slices x 32 packed BF16 pairs (64 l)
constexpr int kXAStages = 2;
constexpr int kXSxRing = 8;
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: x + M - M rounds x to an integer (|x| < 2^22)

// power-of-two scaling of a chunk whose largest magnitude is m: with E the
// biased exponent of m (clamped) and s = 2^(E - 126) > m, the factors 2^6 / s
// and 2^14 / s, and s * 2^-6 for the epilogue
struct XScale {
  float inv, inv256, s6;
};
__device__ __forceinline__ XScale x_scale(float m) {
  int E = (int)((__float_as_uint(m) >> 23) & 0xFFu);
  E = min(max(E, 13), 254);
  XScale r;
  r.inv = __uint_as_float((uint32_t)(259 - E) << 23);
  r.inv256 = __uint_as_float((uint32_t)(267 - E) << 23);
  r.s6 = __uint_as_float((uint32_t)(E - 5) << 23);
  return r;
}
// three integer slices of v * inv (each step exact but the roundings to the
// nearest integer, ties to even)
__device__ __forceinline__ void slice3(float v, const XScale& sc, float& a0, float& a1, float& a2) {
  a0 = __fsub_rn(__fmaf_rn(v, sc.inv, kMagic), kMagic);
  const float r1 = __fmaf_rn(a0, -256.0f, __fmul_rn(v, sc.inv256));
  a1 = __fsub_rn(__fadd_rn(r1, kMagic), kMagic);
  const float r2 = __fmaf_rn(a1, -256.0f, __fmul_rn(r1, 256.0f));
  a2 = __fsub_rn(__fadd_rn(r2, kMagic), kMagic);
}
// BF16 bits of two integer-valued floats (exact), the lower l in the low half
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}
__device__ __forceinline__ uint16_t bf16_bits_exact(float v) { return (uint16_t)(__float_as_uint(v) >> 16); }

// D (TMEM) += A (TMEM, BF16) * B (shared memory descriptor, BF16)
__device__ __forceinline__ void mma_bf16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
// idesc for kind::f16: D FP32, A and B BF16, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16_kk(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kT32TileM >> 4) << 24);
}
// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
      "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

// zeroes the g3 columns of both accumulator layouts in a buffer of width w
// starting at TMEM address tb (this thread's lane)
__device__ __forceinline__ void zero_g3(uint32_t tb, int w) {
  uint32_t z[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) z[i] = 0u;
  tmem_st16(tb + 48, z);
  if (w == 128) {
    tmem_st16(tb + 96, z);
    tmem_st16(tb + 112, z);
  }
}

// SMEM (dynamic, 1024-aligned): [ring: stages x 32 KB][B job 0][B job 1]
//   [t job 0][t job 1][position scale ring 8 x 128][max exchange 2 x 2 x 128]
//   [barriers][tmem slot][abort flag]
// B of a job: [f0 | f1 | f2]^T (3 Kp rows) BF16, K-major without swizzle:
// core matrices of 8 rows x 8 l (16 B rows), LBO = 128 B, SBO = 1024 B,
// 3 Kp * 128 B per 64-l chunk.  t of a job: nk x Kp floats t_k * 2^-6.
struct XParams {
  Tf32Params P;        // jobs (b_off = byte offset of B), ring, work list
  uint32_t t_off[2];   // byte offsets of the F scale tables
  uint32_t sx_off;     // position scale ring
  uint32_t xm_off;     // max exchange
  uint32_t bar_off;    // barriers
  int acc_w;           // accumulator buffer width in columns (4 Kp of the larger job)
  int acc_bufs;        // accumulator buffers
};

__global__ void __launch_bounds__(kT32Threads, 1)
    ttm_x3_kernel(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
                  const XParams X) {
  const Tf32Params& P = X.P;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t nst = (uint32_t)P.stages;
  const uint32_t nacc = (uint32_t)X.acc_bufs;
  unsigned char* ring = smem;
  unsigned char* bsm = ring + (size_t)nst * kT32StageBytes;
  float* sxr = reinterpret_cast<float*>(bsm + X.sx_off);
  float* xm = reinterpret_cast<float*>(bsm + X.xm_off);
  uint64_t* bars = reinterpret_cast<uint64_t*>(bsm + X.bar_off);
  uint64_t* st_full = bars;                      // nst
  uint64_t* st_empty = st_full + nst;            // nst
  uint64_t* a_full = st_empty + nst;             // kXAStages
  uint64_t* a_empty = a_full + kXAStages;        // kXAStages
  uint64_t* acc_full = a_empty + kXAStages;      // nacc
  uint64_t* acc_empty = acc_full + nacc;         // nacc
  uint64_t* sx_full = acc_empty + nacc;          // kXSxRing
  uint64_t* sx_empty = sx_full + kXSxRing;       // kXSxRing
  uint64_t* xchg = sx_empty + kXSxRing;          // 4 (one per lane quarter)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(xchg + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < nst; ++s) {
      mbar_init(&st_full[s], 1);
      mbar_init(&st_empty[s], kT32CvWarps);
    }
    for (int s = 0; s < kXAStages; ++s) {
      mbar_init(&a_full[s], kT32CvWarps);
      mbar_init(&a_empty[s], 1);
    }
    for (uint32_t b = 0; b < nacc; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kT32EpiWarps);
    }
    for (int j = 0; j < kXSxRing; ++j) {
      mbar_init(&sx_full[j], 4);  // the four half-0 converter warps
      mbar_init(&sx_empty[j], kT32EpiWarps);
    }
    for (int q = 0; q < 4; ++q) mbar_init(&xchg[q], 2);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B operands (F cut into three BF16 slices per 64-l chunk and column k)
  // and the F scale tables: one thread per (job, chunk, k)
  for (int j = 0; j < P.njobs; ++j) {
    const Tf32Job& J = P.job[j];
    const int N3 = 3 * J.Kp;
    const float* F = P.F[j];
    float* tt = reinterpret_cast<float*>(bsm + X.t_off[j]);
    for (int idx = threadIdx.x; idx < J.nk * J.Kp; idx += kT32Threads) {
      const int kc = idx / J.Kp, k = idx - kc * J.Kp;
      const int l0 = kc * kT32BoxL;
      float m = 0.f;
      if (k < J.K)
        for (int l = l0; l < min(l0 + kT32BoxL, J.L); ++l) m = fmaxf(m, fabsf(F[(int64_t)l * J.K + k]));
      const XScale sc = x_scale(m);
      tt[idx] = k < J.K ? sc.s6 : 0.f;
      for (int lc = 0; lc < kT32BoxL; ++lc) {
        const int l = l0 + lc;
        const float f = (k < J.K && l < J.L) ? F[(int64_t)l * J.K + k] : 0.f;
        float fs[3];
        slice3(f, sc, fs[0], fs[1], fs[2]);
#pragma unroll
        for (int g = 0; g < 3; ++g) {
          const int row = g * J.Kp + k;
          const size_t off = (size_t)J.b_off + (size_t)kc * N3 * 128 + (size_t)(row >> 3) * 1024 +
                             (size_t)(lc >> 3) * 128 + (size_t)(row & 7) * 16 + (size_t)(lc & 7) * 2;
          *reinterpret_cast<uint16_t*>(bsm + off) = bf16_bits_exact(fs[g]);
        }
      }
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kT32TmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint32_t acc_col0 = kXAStages * kXAStageCols;
  // The last column group g3 = [3 Kp, 4 Kp) of an accumulator buffer is only
  // added to, so it must hold zeros when a chunk starts: the epilogue warps
  // zero it in every buffer once here and again each time they release a
  // buffer.  Kp is 16 or 32 and the two jobs of a pair may differ, so both
  // layouts' g3 are zeroed ([48, 64) and, for 128-column buffers, [96, 128));
  // zeros that land inside another layout's [0, 3 Kp) are overwritten by
  // that chunk's first MMA.
  if (warp >= 2 + kT32CvWarps) {
    const uint32_t lb = tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + acc_col0;
    for (uint32_t b = 0; b < nacc; ++b) zero_g3(lb + b * (uint32_t)X.acc_w, X.acc_w);
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t w = blockIdx.x; w < P.units && ok; w += gridDim.x) {
        const Tile t = decode(P, w);
        const Tf32Job& J = P.job[t.j];
        const CUtensorMap* map = t.j == 0 ? &map0 : &map1;
        for (int kc = 0; kc < J.nk; ++kc, ++it) {
          const uint32_t s = it % nst, ph = (it / nst) & 1u;
          if (!mbar_wait_sleep(&st_empty[s], ph ^ 1u, abort_flag, P.status)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&st_full[s], (uint32_t)kT32StageBytes);
          const int64_t cx = J.type == kJobBlockC ? t.g * J.S + t.c0 : t.c0;
          tma_load_3d(ring + (size_t)s * kT32StageBytes, map, &st_full[s], (int)cx, kc * kT32BoxL, (int)t.r);
        }
      }
      const uint32_t issued = it;
      for (uint32_t j = (issued > nst ? issued - nst : 0); j < issued; ++j) {
        const uint32_t s = j % nst, ph = (j / nst) & 1u;
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(&st_full[s], ph) && globaltimer() - t0 < kTimeoutNs) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t b_base = smem_u32(bsm);
      uint32_t it = 0;
      bool ok = true;
      for (int64_t w = blockIdx.x; w < P.units && ok; w += gridDim.x) {
        const Tile t = decode(P, w);
        const Tf32Job& J = P.job[t.j];
        const uint32_t id3 = idesc_bf16_kk(3 * J.Kp), id2 = idesc_bf16_kk(2 * J.Kp);
        for (int kc = 0; kc < J.nk; ++kc, ++it) {
          const uint32_t buf = it % nacc;
          if (!mbar_wait_sleep(&acc_empty[buf], ((it / nacc) & 1u) ^ 1u, abort_flag, P.status)) {
            ok = false;
            break;
          }
          const uint32_t as = it % kXAStages, aph = (it / kXAStages) & 1u;
          if (!mbar_wait_sleep(&a_full[as], aph, abort_flag, P.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem_base + acc_col0 + buf * (uint32_t)X.acc_w;
          const uint32_t a0 = tmem_base + as * (uint32_t)kXAStageCols;
          const uint32_t b_chunk = b_base + J.b_off + (uint32_t)(kc * 3 * J.Kp * 128);
          const int lval = min(kT32BoxL, J.L - kc * kT32BoxL);
          const int nks = (lval + 15) >> 4;
          for (int ks = 0; ks < nks; ++ks) {
            const uint64_t bd = smem_desc(b_chunk + ks * 256, 128, 1024, kSwizzleNone);
            mma_bf16_ts(d, a0 + ks * 8, bd, id3, ks > 0 ? 1u : 0u);
            mma_bf16_ts(d + J.Kp, a0 + 32 + ks * 8, bd, id3, 1u);
            mma_bf16_ts(d + 2 * J.Kp, a0 + 64 + ks * 8, bd, id2, 1u);
          }
          mma_commit(&a_empty[as]);
          mma_commit(&acc_full[buf]);
        }
      }
    }
  } else if (warp < 2 + kT32CvWarps) {
    // ------------------------------------------------------------ converters
    const int q = warp & 3;
    const int half = (warp - 2) / 4;
    const int p = q * 32 + lane;
    uint32_t it = 0;
    bool ok = true;
    for (int64_t w = blockIdx.x; w < P.units && ok; w += gridDim.x) {
      const Tile t = decode(P, w);
      const Tf32Job& J = P.job[t.j];
      for (int kc = 0; kc < J.nk; ++kc, ++it) {
        const uint32_t s = it % nst, ph = (it / nst) & 1u;
        const uint32_t as = it % kXAStages, aph = (it / kXAStages) & 1u;
        if (!mbar_wait_sleep(&st_full[s], ph, abort_flag, P.status) ||
            !mbar_wait_sleep(&a_empty[as], aph ^ 1u, abort_flag, P.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int lval = min(kT32BoxL, J.L - kc * kT32BoxL) - half * 32;
        // rows past L and positions past the row were zero-filled by TMA
        const float* src = reinterpret_cast<const float*>(ring + (size_t)s * kT32StageBytes) +
                           (size_t)(half * 32) * kT32TileM + p;
        float v[32];
        float m = 0.f;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          v[i] = src[i * kT32TileM];
          m = fmaxf(m, fabsf(v[i]));
        }
        // the position's largest magnitude over the chunk's 64 l: exchange
        // with the other half's warp of this lane quarter
        float* xb = xm + (size_t)(it & 1u) * 256;
        xb[half * 128 + p] = m;
        __syncwarp();
        if (lane == 0) mbar_arrive(&xchg[q]);
        if (!mbar_wait_sleep(&xchg[q], it & 1u, abort_flag, P.status)) {
          ok = false;
          break;
        }
        m = fmaxf(m, xb[(1 - half) * 128 + p]);
        const XScale sc = x_scale(m);
        if (lval > 0) {
          uint32_t w0[16], w1[16], w2[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            float a0, a1, a2, b0, b1, b2;
            slice3(v[2 * i], sc, a0, a1, a2);
            slice3(v[2 * i + 1], sc, b0, b1, b2);
            w0[i] = pack_bf16x2(a0, b0);
            w1[i] = pack_bf16x2(a1, b1);
            w2[i] = pack_bf16x2(a2, b2);
          }
          const uint32_t ta = tmem_base + ((uint32_t)(q * 32) << 16) + as * (uint32_t)kXAStageCols +
                              (uint32_t)(half * 16);
          tmem_st16(ta, w0);
          tmem_st16(ta + 32, w1);
          tmem_st16(ta + 64, w2);
          tmem_wait_st();
        }
        if (half == 0) {
          // the chunk's position scale for the epilogue
          const uint32_t j = it % kXSxRing;
          if (!mbar_wait_sleep(&sx_empty[j], ((it / kXSxRing) & 1u) ^ 1u, abort_flag, P.status)) {
            ok = false;
            break;
          }
          sxr[j * kT32TileM + p] = sc.s6;
          __syncwarp();
          if (lane == 0) mbar_arrive(&sx_full[j]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&a_full[as]);
          mbar_arrive(&st_empty[s]);
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    const int p = q * 32 + lane;
    const uint32_t lane_base = tmem_base + ((uint32_t)(q * 32) << 16);
    uint32_t it = 0;
    bool ok = true;
    for (int64_t w = blockIdx.x; w < P.units && ok; w += gridDim.x) {
      const Tile t = decode(P, w);
      const Tf32Job& J = P.job[t.j];
      const float* tt = reinterpret_cast<const float*>(bsm + X.t_off[t.j]);
      float y[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) y[i] = 0.f;
      for (int kc = 0; kc < J.nk; ++kc, ++it) {
        const uint32_t buf = it % nacc, j = it % kXSxRing;
        if (!mbar_wait_sleep(&acc_full[buf], (it / nacc) & 1u, abort_flag, P.status) ||
            !mbar_wait_sleep(&sx_full[j], (it / kXSxRing) & 1u, abort_flag, P.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const float sxp = sxr[j * kT32TileM + p];
        __syncwarp();
        if (lane == 0) mbar_arrive(&sx_empty[j]);
        const uint32_t tb = lane_base + acc_col0 + buf * (uint32_t)X.acc_w;
        const float* tk = tt + kc * J.Kp;
#pragma unroll
        for (int k0 = 0; k0 < 32; k0 += 16) {
          if (k0 < J.Kp) {
            float g0[16], g1[16], g2[16], g3[16];
            tmem_ld16(tb + k0, g0);
            tmem_ld16(tb + J.Kp + k0, g1);
            tmem_ld16(tb + 2 * J.Kp + k0, g2);
            tmem_ld16(tb + 3 * J.Kp + k0, g3);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float lo = __fmaf_rn(g3[i], 0x1p-24f, __fmaf_rn(g1[i], 0x1p-8f, __fmul_rn(g2[i], 0x1p-16f)));
              const float vv = __fadd_rn(g0[i], lo);
              y[k0 + i] = __fmaf_rn(__fmul_rn(sxp, tk[k0 + i]), vv, y[k0 + i]);
            }
          }
        }
        // zero the last column group for the next chunk in this buffer
        zero_g3(tb, X.acc_w);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[buf]);
      }
      if (!ok) break;
      const int64_t c = t.c0 + p;
      if (c < J.S) {
        float* yp;
        int64_t ystride;
        if (J.type == kJobBlockC) {
          ystride = P.G * J.S;
          yp = J.Y + (t.r * J.K) * ystride + t.g * J.S + c;
        } else {
          ystride = J.S;
          yp = J.Y + (t.r * J.K) * ystride + c;
        }
        if (TK_DBG_IN(yp - J.Y, (yp - J.Y) + (int64_t)(J.K - 1) * ystride, y_total(J, P.G)))
#pragma unroll
          for (int k = 0; k < 32; ++k)
            if (k < J.K) yp[(int64_t)k * ystride] = y[k];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(kT32TmemCols));
  }
}

// ---------------------------------------------------------------------------
// host side (both kernels): jobs, shared-memory layout, launch
// ---------------------------------------------------------------------------
int64_t kp_of(int64_t K) { return (K + 15) / 16 * 16; }
int64_t nk_of(int64_t L) { return (L + kT32BoxL - 1) / kT32BoxL; }

// B bytes of one job: TF32 [F_hi | F_lo] (2 Kp rows of 64 l x 4 B per chunk)
// or BF16 slices [f0 | f1 | f2] (3 Kp rows of 64 l x 2 B per chunk)
size_t b_bytes(bool exact, int64_t L, int64_t K) {
  return exact ? (size_t)(nk_of(L) * 3 * kp_of(K) * 128) : (size_t)(nk_of(L) * 2 * kp_of(K) * 256);
}
size_t t_bytes(int64_t L, int64_t K) { return (size_t)(nk_of(L) * kp_of(K) * 4); }

// Shared-memory layout after the ring, in bytes from its end, and the total.
struct Layout {
  uint32_t b_off[2] = {0, 0}, t_off[2] = {0, 0}, sx_off = 0, xm_off = 0, bar_off = 0;
  size_t after_ring = 0;
};
Layout layout(bool exact, int njobs, const int64_t* L, const int64_t* K, int stages, int acc_bufs) {
  Layout y;
  size_t off = 0;
  for (int j = 0; j < njobs; ++j) {
    y.b_off[j] = (uint32_t)off;
    off += b_bytes(exact, L[j], K[j]);
  }
  if (exact) {
    for (int j = 0; j < njobs; ++j) {
      y.t_off[j] = (uint32_t)off;
      off += (t_bytes(L[j], K[j]) + 15) & ~size_t(15);
    }
    y.sx_off = (uint32_t)off;
    off += (size_t)kXSxRing * kT32TileM * 4;
    y.xm_off = (uint32_t)off;
    off += 2 * 2 * kT32TileM * 4;
  }
  off = (off + 15) & ~size_t(15);
  y.bar_off = (uint32_t)off;
  const size_t nbar = exact ? 2 * (size_t)stages + 2 * kXAStages + 2 * (size_t)acc_bufs + 2 * kXSxRing + 4
                            : 2 * (size_t)stages + 2 * kT32AStages + 2 * kT32AccBufs;
  off += nbar * 8 + 16;
  y.after_ring = off;
  return y;
}
size_t smem_total(int stages, const Layout& y) { return 1024 + (size_t)stages * kT32StageBytes + y.after_ring; }

// accumulator layout of the exact kernel: width 4 Kp (of the larger job) and
// as many buffers as fit next to the A stages in 512 TMEM columns (<= 4)
int acc_width(int njobs, const int64_t* K) {
  int64_t kp = 16;
  for (int j = 0; j < njobs; ++j) kp = std::max(kp, kp_of(K[j]));
  return (int)(4 * kp);
}
int acc_bufs_for(int w) { return std::min(4, (int)((kT32TmemCols - kXAStages * kXAStageCols) / (uint32_t)w)); }

// deepest ring that fits (0 if not even two stages fit)
int stages_for(bool exact, int njobs, const int64_t* L, const int64_t* K) {
  const int ab = exact ? acc_bufs_for(acc_width(njobs, K)) : kT32AccBufs;
  for (int st = kT32MaxStages; st >= 2; --st)
    if (smem_total(st, layout(exact, njobs, L, K, st, ab)) <= 227 * 1024) return st;
  return 0;
}

bool job_shape_ok(int64_t L, int64_t K) { return K >= 1 && K <= 32 && L >= 1 && L <= 1024; }

void fill_job(Tf32Job& J, int type, int64_t L, int64_t K, float* Y) {
  J.type = type;
  J.L = (int)L;
  J.K = (int)K;
  J.Kp = (int)kp_of(K);
  J.nk = (int)nk_of(L);
  J.Y = Y;
}

int launch(bool exact, const CUtensorMap& m0, const CUtensorMap& m1, Tf32Params& P, cudaStream_t s) {
  const int64_t L[2] = {P.job[0].L, P.job[1].L}, K[2] = {P.job[0].K, P.job[1].K};
  P.stages = stages_for(exact, P.njobs, L, K);
  if (P.stages == 0) return fail(TUCKER_ERR_UNSUPPORTED, "ttm_f32_tc: factors do not fit in shared memory");
  P.status = device_status_ptr();
  if (!P.status) return fail(TUCKER_ERR_CUDA, "ttm_f32_tc: device error word unavailable");
  P.chunk_acc = (kernel_policy() & 128) ? 0 : 1;
  const int64_t grid = std::min<int64_t>(P.units, sm_count());
  if (!exact) {
    const Layout y = layout(false, P.njobs, L, K, P.stages, kT32AccBufs);
    for (int j = 0; j < P.njobs; ++j) P.job[j].b_off = y.b_off[j];
    const size_t smem = smem_total(P.stages, y);
    TK_CUDA_TRY(cudaFuncSetAttribute(ttm_tf32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ttm_tf32_kernel<<<(unsigned)grid, kT32Threads, smem, s>>>(m0, m1, P);
    TK_LAUNCH_CHECK("ttm_tf32");
    return TUCKER_OK;
  }
  XParams X{};
  X.acc_w = acc_width(P.njobs, K);
  X.acc_bufs = acc_bufs_for(X.acc_w);
  const Layout y = layout(true, P.njobs, L, K, P.stages, X.acc_bufs);
  for (int j = 0; j < P.njobs; ++j) {
    P.job[j].b_off = y.b_off[j];
    X.t_off[j] = y.t_off[j];
  }
  X.sx_off = y.sx_off;
  X.xm_off = y.xm_off;
  X.bar_off = y.bar_off;
  X.P = P;
  const size_t smem = smem_total(P.stages, y);
  TK_CUDA_TRY(cudaFuncSetAttribute(ttm_x3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ttm_x3_kernel<<<(unsigned)grid, kT32Threads, smem, s>>>(m0, m1, X);
  TK_LAUNCH_CHECK("ttm_x3");
  return TUCKER_OK;
}

bool single_supported(bool exact, int64_t R, int64_t L, int64_t C, int64_t K, const void* X) {
  if (!job_shape_ok(L, K) || C < 64 || C % 4 != 0) return false;
  if ((uintptr_t)X % 16 != 0 || R > INT32_MAX || C > INT32_MAX) return false;
  const int64_t Ls[2] = {L, L}, Ks[2] = {K, K};
  return stages_for(exact, 1, Ls, Ks) >= 2;
}

int launch_single(bool exact, const float* X, int64_t R, int64_t L, int64_t C, const float* F, int64_t K,
                  float* Y, cudaStream_t s) {
  if (!single_supported(exact, R, L, C, K, X))
    return fail(TUCKER_ERR_UNSUPPORTED, "ttm_f32_tc: shape or alignment not supported");
  Tf32Params P{};
  P.njobs = 1;
  Tf32Job& J = P.job[0];
  fill_job(J, kJobPlain, L, K, Y);
  J.R = R;
  J.Rl = 1;
  J.S = C;
  J.ct = (C + kT32TileM - 1) / kT32TileM;
  J.per_block = R * J.ct;
  P.job[1] = J;
  P.G = 1;
  P.per_block = J.per_block;
  P.units = P.per_block;
  P.F[0] = P.F[1] = F;
  CUtensorMap m;
  const cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)L, (cuuint64_t)R};
  const cuuint64_t str[2] = {(cuuint64_t)C * 4, (cuuint64_t)C * L * 4};
  const cuuint32_t box[3] = {(cuuint32_t)kT32TileM, (cuuint32_t)kT32BoxL, 1u};
  const int rc = make_map(&m, X, 3, dims, str, box, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, CU_TENSOR_MAP_SWIZZLE_NONE);
  if (rc) return rc;
  return launch(exact, m, m, P, s);
}

bool pair_supported(bool exact, const int64_t* dims, int N, int a, int b, int64_t Ka, int64_t Kb, const void* X) {
  if (a < 0 || b != a + 2 || b >= N) return false;  // one mode between a and b
  if (!job_shape_ok(dims[a], Ka) || !job_shape_ok(dims[b], Kb)) return false;
  const int m = a + 1;
  const int64_t S = prod(dims, m + 1, N), Cb = prod(dims, b + 1, N);
  const int64_t Ra = prod(dims, 0, a), Rh = prod(dims, 0, m);
  if (S < 64 || S % 4 != 0 || Cb < 64 || Cb % 4 != 0) return false;
  if ((uintptr_t)X % 16 != 0 || S * dims[m] > INT32_MAX || Cb > INT32_MAX || Ra > INT32_MAX ||
      Rh * dims[m] > INT32_MAX)
    return false;
  const int64_t Ls[2] = {dims[a], dims[b]}, Ks[2] = {Ka, Kb};
  return stages_for(exact, 2, Ls, Ks) >= 2;
}

int launch_pair(bool exact, const float* X, const int64_t* dims, int N, int a, int b, const float* Fa,
                int64_t Ka, const float* Fb, int64_t Kb, float* Ya, float* Yb, cudaStream_t s) {
  if (!pair_supported(exact, dims, N, a, b, Ka, Kb, X))
    return fail(TUCKER_ERR_UNSUPPORTED, "ttm_f32_tc pair: shape or alignment not supported");
  const int m = a + 1;
  const int64_t G = dims[m];
  Tf32Params P{};
  P.njobs = 2;
  P.G = G;
  // job 0: mode a as [Ra][La][G * S], tiles within one block's S positions
  Tf32Job& A = P.job[0];
  fill_job(A, kJobBlockC, dims[a], Ka, Ya);
  A.R = prod(dims, 0, a);
  A.Rl = 1;
  A.S = prod(dims, m + 1, N);
  A.ct = (A.S + kT32TileM - 1) / kT32TileM;
  A.per_block = A.R * A.ct;
  // job 1: mode b as [Rh][G][Rl][Lb][Cb]
  Tf32Job& B = P.job[1];
  fill_job(B, kJobBlockR, dims[b], Kb, Yb);
  B.R = prod(dims, 0, m);
  B.Rl = prod(dims, m + 1, b);
  B.S = prod(dims, b + 1, N);
  B.ct = (B.S + kT32TileM - 1) / kT32TileM;
  B.per_block = B.R * B.Rl * B.ct;
  P.per_block = A.per_block + B.per_block;
  P.units = G * P.per_block;
  P.F[0] = Fa;
  P.F[1] = Fb;
  CUtensorMap ma, mb;
  {
    const int64_t Ca = G * A.S;
    const cuuint64_t d3[3] = {(cuuint64_t)Ca, (cuuint64_t)A.L, (cuuint64_t)A.R};
    const cuuint64_t st[2] = {(cuuint64_t)Ca * 4, (cuuint64_t)(Ca * A.L) * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kT32TileM, (cuuint32_t)kT32BoxL, 1u};
    const int rc = make_map(&ma, X, 3, d3, st, box, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (rc) return rc;
  }
  {
    const int64_t Rb = prod(dims, 0, b);
    const cuuint64_t d3[3] = {(cuuint64_t)B.S, (cuuint64_t)B.L, (cuuint64_t)Rb};
    const cuuint64_t st[2] = {(cuuint64_t)B.S * 4, (cuuint64_t)(B.S * B.L) * 4};
    const cuuint32_t box[3] = {(cuuint32_t)kT32TileM, (cuuint32_t)kT32BoxL, 1u};
    const int rc = make_map(&mb, X, 3, d3, st, box, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (rc) return rc;
  }
  return launch(exact, ma, mb, P, s);
}

}  // namespace

// Whether a tensor-core FP32 TTM takes this column shape: C % 4 == 0 (16-byte
// TMA row strides), C >= 64, K <= 32, L <= 1024, B (and the scale tables)
// within shared memory next to two ring stages, 32-bit grid coordinates,
// 16-byte aligned tensor.
bool ttm_tf32_supported(int64_t R, int64_t L, int64_t C, int64_t K, const void* X) {
  return single_supported(false, R, L, C, K, X);
}
int launch_ttm_tf32(const float* X, int64_t R, int64_t L, int64_t C, const float* F, int64_t K, float* Y,
                    cudaStream_t s) {
  return launch_single(false, X, R, L, C, F, K, Y, s);
}
bool ttm_x3_supported(int64_t R, int64_t L, int64_t C, int64_t K, const void* X) {
  return single_supported(true, R, L, C, K, X);
}
int launch_ttm_x3(const float* X, int64_t R, int64_t L, int64_t C, const float* F, int64_t K, float* Y,
                  cudaStream_t s) {
  return launch_single(true, X, R, L, C, F, K, Y, s);
}

// The L2-blocked pair: modes a and a + 2 <= b of an FP32 tensor with lengths
// dims[0..N-1], blocked by mode m = a + 1.  Needs S = prod dims[m+1..N-1] and
// C_b = prod dims[b+1..N-1] multiples of 4 and >= 64, both factors within the
// single-job limits, and both B operands within shared memory.
bool ttm_tf32_pair_supported(const int64_t* dims, int N, int a, int b, int64_t Ka, int64_t Kb,
                             const void* X) {
  return pair_supported(false, dims, N, a, b, Ka, Kb, X);
}
int launch_ttm_tf32_pair(const float* X, const int64_t* dims, int N, int a, int b, const float* Fa, int64_t Ka,
                         const float* Fb, int64_t Kb, float* Ya, float* Yb, cudaStream_t s) {
  return launch_pair(false, X, dims, N, a, b, Fa, Ka, Fb, Kb, Ya, Yb, s);
}
bool ttm_x3_pair_supported(const int64_t* dims, int N, int a, int b, int64_t Ka, int64_t Kb, const void* X) {
  return pair_supported(true, dims, N, a, b, Ka, Kb, X);
}
int launch_ttm_x3_pair(const float* X, const int64_t* dims, int N, int a, int b, const float* Fa, int64_t Ka,
                       const float* Fb, int64_t Kb, float* Ya, float* Yb, cudaStream_t s) {
  return launch_pair(true, X, dims, N, a, b, Fa, Ka, Fb, Kb, Ya, Yb, s);
}

}  // namespace tk
