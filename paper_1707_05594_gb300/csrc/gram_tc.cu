// gram_tc.cu -- Gram matrix of a mode-n unfolding on the 5th-generation tensor
// cores, W += Z_(n) Z_(n)^T (Sec. 5: the leading left singular vectors of
// Z_(n) come from its Gram and a symmetric EVD), for FP32 Z viewed as
// [R][L][C] with C > 1.  Column m = (r, c) of the unfolding is the fibre
// Z[r, :, c]; W[i, j] = sum_m Z[r, i, c] Z[r, j, c].
//
// GEMM view: the L rows are cut into blocks of 128; a job is a block pair
// (I, J), I <= J, computing D[128 rows of I, N] = A B^T over the columns,
// with A the rows of block I and B those of block J (N = the rows of J
// rounded up to 16).  Both operands are K-major: a stage is 32 columns, i.e.
// one 128-byte row per tensor row, which TMA lands with the 128-byte swizzle
// in exactly the layout the MMA reads (8-row groups 1024 B apart, a k-step of
// 8 columns = 32 B inside the swizzled row).
//
// Precision: TF32 keeps 11 significant bits, so every value is split in place
// into x_hi = x rounded to 11 bits and x_lo = x - x_hi rounded to 11 bits
// (|x_lo| <= 2^-11 |x|; x_hi + x_lo holds x to 2^-22 |x|), both exact TF32
// values, and each k-step issues three MMAs, A_hi B_hi + A_hi B_lo +
// A_lo B_hi (the dropped A_lo B_lo is below 2^-22 |x y|).  The tensor core's
// FP32 accumulation rounds toward zero, so an accumulator takes one stage
// only (12 MMAs); the work warps then add it to FP32 running sums in
// registers (rounded to nearest), fold those into a second FP32 level in
// TMEM every 16 stages, and add both levels to W with FP64 atomics at the
// end.
//
// Units: the R * ceil(C / 32) column chunks of every job are cut into the
// same number of contiguous ranges per job (about as many CTAs in all as the
// GPU has SMs, at least 32 chunks each: fewer CTAs, and fewer atomics, for
// small Grams), so that the jobs that share a block read the same columns at
// about the same time and the second read of a block is served by L2.  One
// CTA per SM (~200 KB of shared memory, 512 TMEM columns).
//
// Warp roles (576 threads): warp 0 TMA producer (one lane); warp 1 TMEM
// allocation and MMA issuer (one lane); warps 2-17 split each landed stage in
// shared memory (generic stores, then a proxy fence) and drain the
// accumulator of the stage two behind (tcgen05.ld; the warp's TMEM lane
// quarter, 32 of the N columns each).  Three TMEM accumulators of 128
// columns let the MMAs run two stages ahead of the drains; the last 128
// TMEM columns hold the second-level sums.  Every wait
// is bounded by %globaltimer; on expiry the kernel records TUCKER_ERR_TIMEOUT
// in the library's device error word, waits (bounded) for its own copies,
// frees TMEM and returns.
#include <algorithm>

#include "tc_common.cuh"

namespace tk {
namespace {

using namespace tc;

constexpr int kGB = 128;                    // rows per block: the MMA's M, N at most
constexpr int kGC = 32;                     // columns per stage (128 B of FP32)
constexpr int kGWork = 16;                  // split + drain warps
constexpr int kGThreads = 64 + 32 * kGWork;
constexpr int kGAcc = 3;                    // TMEM accumulators of kGB columns
constexpr int kGLag = 2;                    // stage s is drained after stage s + 2 is split
constexpr int kGFold = 16;                  // stage sums per level-1 run
constexpr int kGMaxStages = 16;
constexpr int kGMaxJobs = 10;               // block pairs for L <= 512
constexpr int kGMinChunks = 8;              // chunks per unit at least (leaf Grams of the 200^4 sweep, 250 chunks: 56 -> 30 us against 32)
constexpr uint32_t kGSum2 = kGAcc * kGB;     // TMEM column of the second-level sums
constexpr uint32_t kGTmemCols = 512;
constexpr size_t kGSmemBudget = 200 * 1024;  // ring
constexpr uint32_t kGBarBytes = 1024;         // barriers, TMEM slot, abort flag

struct GramParams {
  int64_t L;
  int64_t Q;          // column chunks per job: R * nc
  int64_t nc;         // chunks per r: ceil(C / 32)
  int rows;           // rows per TMA box: 128, or L rounded up to 16 for one block
  int two;            // two blocks per stage (some job has I != J)
  int stages;
  int njobs;
  int units;          // units per job
  int bi[kGMaxJobs], bj[kGMaxJobs], n[kGMaxJobs];
  double* W;
  int* status;
};

// idesc for kind::tf32: D FP32, A and B TF32, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_gram(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kGB >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32_ss(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// x rounded to 11 significant bits (ties away from zero): add half a unit of
// the 11th bit to the magnitude and clear the 13 bits below it.
__device__ __forceinline__ float round_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// The bounded wait of tc_common.cuh, inline: the work warps hold 64 running
// sums, which a call would have to save around it.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                         int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 255u) == 255u) {
      if (*abort_flag) return false;
      if (globaltimer() - t0 > kTimeoutNs) {
        *abort_flag = 1;
        atomicCAS(status, 0, TUCKER_ERR_TIMEOUT);
        return false;
      }
    }
  }
}

__global__ void __launch_bounds__(kGThreads, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap map, const GramParams P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t buf = (uint32_t)P.rows * 128u;          // one block's 32 columns
  const uint32_t lo_off = (P.two ? 2u : 1u) * buf;       // x_lo buffers after the x_hi ones
  const uint32_t stage_bytes = 2u * lo_off;
  const uint32_t S = (uint32_t)P.stages;
  // barriers in the first 1 KB, then the ring; with fewer than 128 rows per
  // block the MMA's A operand (always 128 rows) reads past a buffer into the
  // next one, or into the tail pad after the ring: those rows of D are
  // never used
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  unsigned char* ring = smem + kGBarBytes;
  uint64_t* conv = full + S;     // split done (kGWork arrivals)
  uint64_t* empty = conv + S;    // MMAs done reading the stage
  uint64_t* afull = empty + S;   // accumulator complete
  uint64_t* aempty = afull + kGAcc;  // accumulator drained (kGWork arrivals)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(aempty + kGAcc);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  // this CTA's unit: job j, chunk range [q0, q1)
  const int j = (int)blockIdx.x / P.units;
  const int64_t sidx = (int64_t)blockIdx.x - (int64_t)j * P.units;
  const int64_t q0 = P.Q * sidx / P.units, q1 = P.Q * (sidx + 1) / P.units;
  const uint32_t nq = (uint32_t)(q1 - q0);
  const int I = P.bi[j], J = P.bj[j], N = P.n[j];
  const bool diag = I == J;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], kGWork);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < kGAcc; ++b) {
      mbar_init(&afull[b], 1);
      mbar_init(&aempty[b], kGWork);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kGTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      tma_prefetch_map(&map);
      uint32_t it = 0;
      const uint32_t tx = (diag ? 1u : 2u) * buf;
      for (; it < nq; ++it) {
        const uint32_t s = it % S, ph = (it / S) & 1u;
        if (!mbar_wait_status(&empty[s], ph ^ 1u, abort_flag, P.status)) break;
        const int64_t q = q0 + it;
        const int64_t r = q / P.nc;
        const int c0 = (int)((q - r * P.nc) * kGC);
        unsigned char* dst = ring + (size_t)s * stage_bytes;
        mbar_expect_tx(&full[s], tx);
        tma_load_3d(dst, &map, &full[s], c0, I * kGB, (int)r);
        if (!diag) tma_load_3d(dst + buf, &map, &full[s], c0, J * kGB, (int)r);
      }
      // wait (bounded) until every copy issued has landed
      for (uint32_t k = (it > S ? it - S : 0); k < it; ++k) {
        const uint32_t s = k % S, ph = (k / S) & 1u;
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(&full[s], ph) && globaltimer() - t0 < kTimeoutNs) {
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_gram(N);
      for (uint32_t it = 0; it < nq; ++it) {
        const uint32_t s = it % S, ph = (it / S) & 1u;
        const uint32_t b = it % kGAcc, aph = (it / kGAcc) & 1u;
        if (!mbar_wait_status(&aempty[b], aph ^ 1u, abort_flag, P.status)) break;
        if (!mbar_wait_status(&conv[s], ph, abort_flag, P.status)) break;
        tc_fence_after();
        const uint32_t base = smem_u32(ring + (size_t)s * stage_bytes);
        const uint32_t a_hi = base, b_hi = diag ? base : base + buf;
        const uint32_t a_lo = base + lo_off, b_lo = diag ? a_lo : a_lo + buf;
        const uint32_t d = tmem_base + b * (uint32_t)kGB;
#pragma unroll
        for (int ks = 0; ks < kGC / 8; ++ks) {
          // K-major, 128-byte swizzle: 8-row groups 1024 B apart, the k-step
          // of 8 TF32 values = 32 B inside the swizzled row
          const uint64_t ah = smem_desc(a_hi + ks * 32, 16, 1024, kSwizzle128);
          const uint64_t bh = smem_desc(b_hi + ks * 32, 16, 1024, kSwizzle128);
          const uint64_t al = smem_desc(a_lo + ks * 32, 16, 1024, kSwizzle128);
          const uint64_t bl = smem_desc(b_lo + ks * 32, 16, 1024, kSwizzle128);
          mma_tf32_ss(d, ah, bh, idesc, ks > 0 ? 1u : 0u);
          mma_tf32_ss(d, ah, bl, idesc, 1u);
          mma_tf32_ss(d, al, bh, idesc, 1u);
        }
        mma_commit(&empty[s]);
        mma_commit(&afull[b]);
      }
    }
  } else {
    // ------------------------------------------------------------ split + drain
    const int tw = threadIdx.x - 64;          // 0 .. 32 * kGWork - 1
    const int q4 = warp & 3;                  // TMEM lane quarter of this warp
    const int part = (warp - 2) >> 2;         // which 32 of the N columns
    const int nf4 = (diag ? 1 : 2) * P.rows * (kGC / 4);
    float s1[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) s1[i] = 0.f;
    int fold = 0;
    bool have_s2 = false;
    bool ok = true;
    const uint32_t tcol = tmem_base + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(part * 32);
    const uint32_t t2 = tcol + kGSum2;  // this thread's second-level sums
    const bool c0ok = part * 32 < N, c1ok = part * 32 + 16 < N;  // warp-uniform

    // s1 += the second-level sums (when there are any)
    auto add_s2 = [&]() {
      if (!have_s2) return;
      float v[16];
      if (c0ok) {
        tmem_ld16(t2, v);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 16; ++i) s1[i] += v[i];
      }
      if (c1ok) {
        tmem_ld16(t2 + 16, v);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 16; ++i) s1[16 + i] += v[i];
      }
    };

    auto drain = [&](uint32_t c) -> bool {
      const uint32_t b = c % kGAcc, aph = (c / kGAcc) & 1u;
      if (!wait_bar(&afull[b], aph, abort_flag, P.status)) return false;
      tc_fence_after();
      const uint32_t ta = tcol + b * (uint32_t)kGB;
      {
        float v[32];
        // this warp's two 16-column groups that hold columns < N
        if (c0ok) tmem_ld16(ta, v);
        if (c1ok) tmem_ld16(ta + 16, v + 16);
        if (c0ok) {
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 16; ++i) s1[i] += v[i];
        }
        if (c1ok) {
#pragma unroll
          for (int i = 0; i < 16; ++i) s1[16 + i] += v[16 + i];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&aempty[b]);
      if (++fold == kGFold) {
        // second level: s2 = s2 + s1 in TMEM, s1 = 0
        fold = 0;
        add_s2();
        if (c0ok) tmem_st16(t2, s1);
        if (c1ok) tmem_st16(t2 + 16, s1 + 16);
        tmem_wait_st();
        have_s2 = true;
#pragma unroll
        for (int i = 0; i < 32; ++i) s1[i] = 0.f;
      }
      return true;
    };

    for (uint32_t it = 0; it < nq && ok; ++it) {
      const uint32_t s = it % S, ph = (it / S) & 1u;
      if (!wait_bar(&full[s], ph, abort_flag, P.status)) {
        ok = false;
        break;
      }
      unsigned char* st = ring + (size_t)s * stage_bytes;
      for (int i = tw; i < nf4; i += 32 * kGWork) {
        float4* hp = reinterpret_cast<float4*>(st) + i;
        float4* lp = reinterpret_cast<float4*>(st + lo_off) + i;
        const float4 x = *hp;
        float4 h, l;
        h.x = round_tf32(x.x);
        h.y = round_tf32(x.y);
        h.z = round_tf32(x.z);
        h.w = round_tf32(x.w);
        l.x = round_tf32(x.x - h.x);
        l.y = round_tf32(x.y - h.y);
        l.z = round_tf32(x.z - h.z);
        l.w = round_tf32(x.w - h.w);
        *hp = h;
        *lp = l;
      }
      // generic-proxy stores must be visible to the tensor core
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv[s]);
      if (it >= (uint32_t)kGLag && !drain(it - kGLag)) ok = false;
    }
    if (ok)
      for (uint32_t c = (nq > (uint32_t)kGLag ? nq - kGLag : 0); c < nq; ++c)
        if (!drain(c)) {
          ok = false;
          break;
        }
    if (ok) {
      add_s2();
      const int64_t row = (int64_t)I * kGB + q4 * 32 + lane;
      const int64_t col0 = (int64_t)J * kGB + part * 32;
      if (row < P.L) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int64_t col = col0 + i;
          if (part * 32 + i < N && col < P.L) {
            const double v = (double)s1[i];
            atomicAdd(&P.W[row * P.L + col], v);
            if (!diag) atomicAdd(&P.W[col * P.L + row], v);
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
                 "r"(kGTmemCols));
  }
}

}  // namespace

bool gram_tc_supported(int64_t R, int64_t L, int64_t C, const void* Z) {
  if (R < 1 || L < 1 || C < 16 || C % 4 != 0) return false;
  if (L > (int64_t)kGB * 4) return false;  // block pairs for up to 4 blocks
  if ((uintptr_t)Z % 16 != 0 || R > INT32_MAX || C > INT32_MAX) return false;
  const int64_t nc = (C + kGC - 1) / kGC;
  return R <= INT32_MAX / nc;  // chunk counts stay within 32 bits
}

int launch_gram_tc(const float* Z, int64_t R, int64_t L, int64_t C, double* W, cudaStream_t s) {
  if (!gram_tc_supported(R, L, C, Z))
    return fail(TUCKER_ERR_UNSUPPORTED, "gram_tc: shape or alignment not supported");
  GramParams P{};
  P.L = L;
  P.nc = (C + kGC - 1) / kGC;
  P.Q = R * P.nc;
  const int nb = (int)((L + kGB - 1) / kGB);
  P.rows = nb == 1 ? (int)((L + 15) / 16 * 16) : kGB;
  P.two = nb > 1 ? 1 : 0;
  P.njobs = 0;
  for (int I = 0; I < nb; ++I)
    for (int J = I; J < nb; ++J) {
      const int k = P.njobs++;
      const int64_t rowsJ = std::min<int64_t>(kGB, L - (int64_t)J * kGB);
      P.bi[k] = I;
      P.bj[k] = J;
      P.n[k] = (int)((rowsJ + 15) / 16 * 16);
    }
  // the same number of units per job, about one CTA per SM in all, at least
  // kGMinChunks chunks per unit
  const int64_t per_job = std::max<int64_t>(1, sm_count() / P.njobs);
  P.units = (int)std::max<int64_t>(1, std::min<int64_t>(per_job, P.Q / kGMinChunks));
  const size_t stage = (size_t)2 * (P.two ? 2 : 1) * (size_t)P.rows * 128;
  P.stages = (int)std::min<size_t>(kGMaxStages, kGSmemBudget / stage);
  if (P.stages < 2) return fail(TUCKER_ERR_UNSUPPORTED, "gram_tc: stage does not fit");
  P.W = W;
  P.status = device_status_ptr();
  if (!P.status) return fail(TUCKER_ERR_CUDA, "gram_tc: device error word unavailable");
  CUtensorMap m;
  const cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)L, (cuuint64_t)R};
  const cuuint64_t str[2] = {(cuuint64_t)C * 4, (cuuint64_t)C * L * 4};
  const cuuint32_t box[3] = {(cuuint32_t)kGC, (cuuint32_t)P.rows, 1u};
  const int rc = make_map(&m, Z, 3, dims, str, box, CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                          CU_TENSOR_MAP_SWIZZLE_128B);
  if (rc) return rc;
  // alignment slack + barriers + ring + tail pad for the A operand's rows
  // past the last buffer, at least 120 KB so that one CTA holds an SM (each
  // takes all 512 TMEM columns)
  static_assert((3 * kGMaxStages + 2 * kGAcc) * 8 + 16 <= kGBarBytes, "barrier area");
  size_t smem = 1024 + kGBarBytes + (size_t)P.stages * stage + (size_t)(kGB - P.rows) * 128;
  smem = std::max<size_t>(smem, 120 * 1024);
  TK_CUDA_TRY(cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  gram_tc_kernel<<<(unsigned)(P.njobs * P.units), kGThreads, smem, s>>>(m, P);
  TK_LAUNCH_CHECK("gram_tc");
  return TUCKER_OK;
}

}  // namespace tk
