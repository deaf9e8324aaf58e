// ttm_simt.cu -- mode-n tensor-times-matrix, Out = In x_n F^T (Sec. 2.1), on
// the CUDA cores, without unfolding the tensor (the blocked, transposition-free
// TTM of Sec. 5).
//
// The input is viewed as [R][L][C]: R = product of the lengths before mode n,
// L = L_n, C = product of the lengths after it; the output is [R][K][C] with
//   Out[r, k, c] = sum_l F[l, k] * In[r, l, c].
// Two kernels:
//   ttm_cols  C > 1: each thread owns VEC consecutive (r, c) positions and
//             all KB outputs of its k-block; it streams In[r, :, c..c+VEC)
//             (coalesced along c) and reads F from shared memory (broadcast).
//   ttm_rows  C == 1 (last mode): the fibres are contiguous rows; a block
//             stages 128 rows x 32 columns in shared memory with coalesced
//             loads and each thread reduces its own row.
// Accumulation is FP32 for FP32/BF16 inputs and FP64 for FP64 inputs.
#include <type_traits>

#include "common.cuh"

namespace tk {
namespace {

constexpr int kColsThreads = 256;
constexpr int kColsLChunk = 64;

template <typename TIn, typename TOut, int KB, int VEC>
__global__ void __launch_bounds__(kColsThreads)
    ttm_cols_kernel(const TIn* __restrict__ X, const typename AccOf<TIn>::type* __restrict__ F,
                    TOut* __restrict__ Y, int64_t R, int L, int64_t C, int K) {
  using A = typename AccOf<TIn>::type;
  __shared__ __align__(16) A Fs[kColsLChunk][KB];
  const int kb0 = blockIdx.y * KB;
  const int64_t total = R * C;
  const int64_t m0 = ((int64_t)blockIdx.x * kColsThreads + threadIdx.x) * VEC;
  bool active = m0 < total;
  int64_t r = 0, c = 0;
  if (active) {
    r = m0 / C;
    c = m0 - r * C;
    // this thread reads X[r, 0 .. L-1, c .. c+VEC-1], writes Y[r, kb0 .., c ..]
    active = TK_DBG_IN(r * L * C + c, (r * L + L - 1) * C + c + VEC - 1, R * L * C) &&
             TK_DBG_IN((r * K + kb0) * C + c, (r * K + min(K, kb0 + KB) - 1) * C + c + VEC - 1, R * K * C);
  }
  const TIn* xp = X + (r * L) * C + c;
  A acc[KB][VEC];
#pragma unroll
  for (int k = 0; k < KB; ++k)
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[k][v] = A(0);

  for (int l0 = 0; l0 < L; l0 += kColsLChunk) {
    const int lc = min(kColsLChunk, L - l0);
    __syncthreads();
    for (int i = threadIdx.x; i < kColsLChunk * KB; i += kColsThreads) {
      const int l = i / KB, k = i - (i / KB) * KB;
      const int64_t e = (int64_t)(l0 + l) * K + kb0 + k;
      Fs[l][k] = (l < lc && kb0 + k < K && TK_DBG_IN(e, e, (int64_t)L * K)) ? F[e] : A(0);
    }
    __syncthreads();
    if (active) {
      const TIn* p = xp + (int64_t)l0 * C;
      int l = 0;
      for (; l + 4 <= lc; l += 4) {
        A x0[VEC], x1[VEC], x2[VEC], x3[VEC];
        VecLoad<TIn, VEC>::run(p, x0);
        VecLoad<TIn, VEC>::run(p + C, x1);
        VecLoad<TIn, VEC>::run(p + 2 * C, x2);
        VecLoad<TIn, VEC>::run(p + 3 * C, x3);
        p += 4 * C;
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          const A f0 = Fs[l][k], f1 = Fs[l + 1][k], f2 = Fs[l + 2][k], f3 = Fs[l + 3][k];
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            acc[k][v] = fma(f0, x0[v], acc[k][v]);
            acc[k][v] = fma(f1, x1[v], acc[k][v]);
            acc[k][v] = fma(f2, x2[v], acc[k][v]);
            acc[k][v] = fma(f3, x3[v], acc[k][v]);
          }
        }
      }
      for (; l < lc; ++l) {
        A x0[VEC];
        VecLoad<TIn, VEC>::run(p, x0);
        p += C;
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          const A f0 = Fs[l][k];
#pragma unroll
          for (int v = 0; v < VEC; ++v) acc[k][v] = fma(f0, x0[v], acc[k][v]);
        }
      }
    }
  }
  if (!active) return;
  TOut* yp = Y + (r * K + kb0) * C + c;
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    if (kb0 + k < K) {
      TOut o[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) o[v] = OutCvt<TOut>::run(acc[k][v]);
      VecStore<TOut, VEC>::run(yp + (int64_t)k * C, o);
    }
  }
}

// ---------------------------------------------------------------------------
// ttm_cols_pipe: the same mapping as ttm_cols, but each thread streams its
// VEC-wide column slice through a private ring of kDepth shared-memory slots
// filled by cp.async, so kDepth loads per thread are in flight without
// holding registers.  Used when VEC*sizeof(TIn) is 8 or 16 bytes and aligned.
// Each thread reads back only the slots it filled itself, so no block-level
// barrier guards the ring; cp.async.wait_group orders its own copies.
// ---------------------------------------------------------------------------
constexpr int kDepth = 8;

__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <typename TIn, int VEC>
struct Slot {
  static constexpr int kBytes = VEC * (int)sizeof(TIn);
  static __device__ __forceinline__ void copy(void* smem, const TIn* g) {
    if constexpr (kBytes == 16) cp_async_16(smem, g);
    else cp_async_8(smem, g);
  }
};

// Slots in flight per thread of ttm_cols_pipe (the ring lives in dynamic
// shared memory so that the depth is free of the 48 KB static limit; on the
// 200^4 root, 12, 16 and 24 slots measured 7 %, 1 % and 14 % slower than 8).
template <int SB>
__host__ __device__ constexpr int pipe_depth() { return 8; }
// Rows l of F staged per chunk of ttm_cols_pipe (every chunk ends with a
// block barrier and a reload of F; 128 rows measured 1.7 % faster than 64 on
// the 200^4 root, 256 no better)
template <typename A>
__host__ __device__ constexpr int pipe_lchunk() { return sizeof(A) == 4 ? 128 : kColsLChunk; }

template <typename TIn, typename TOut, int KB, int VEC>
__global__ void __launch_bounds__(kColsThreads, (KB * VEC * sizeof(typename AccOf<TIn>::type) <= 384) ? 2 : 1)
    ttm_cols_pipe_kernel(const TIn* __restrict__ X, const typename AccOf<TIn>::type* __restrict__ F,
                         TOut* __restrict__ Y, int64_t R, int L, int64_t C, int K) {
  using A = typename AccOf<TIn>::type;
  constexpr int SB = Slot<TIn, VEC>::kBytes;
  static_assert(SB == 8 || SB == 16, "slot size");
  constexpr int kDepth = pipe_depth<SB>();
  constexpr int kLChunk = pipe_lchunk<A>();
  __shared__ __align__(16) A Fs[kLChunk][KB];
  // the ring, [kDepth][kColsThreads][SB] bytes of dynamic shared memory
  extern __shared__ __align__(16) unsigned char ring_mem[];
  unsigned char(*ring)[kColsThreads][SB] = reinterpret_cast<unsigned char(*)[kColsThreads][SB]>(ring_mem);
  const int tid = threadIdx.x;
  const int kb0 = blockIdx.y * KB;
  const int64_t total = R * C;
  const int64_t m0 = ((int64_t)blockIdx.x * kColsThreads + tid) * VEC;
  bool active = m0 < total;
  int64_t r = 0, c = 0;
  if (active) {
    r = m0 / C;
    c = m0 - r * C;
    // this thread reads X[r, 0 .. L-1, c .. c+VEC-1], writes Y[r, kb0 .., c ..]
    active = TK_DBG_IN(r * L * C + c, (r * L + L - 1) * C + c + VEC - 1, R * L * C) &&
             TK_DBG_IN((r * K + kb0) * C + c, (r * K + min(K, kb0 + KB) - 1) * C + c + VEC - 1, R * K * C);
  }
  const TIn* xp = X + (r * L) * C + c;
#pragma unroll
  for (int s = 0; s < kDepth; ++s) {
    if (active && s < L) Slot<TIn, VEC>::copy(&ring[s][tid][0], xp + (int64_t)s * C);
    cp_async_commit();
  }
  // FP32 accumulators in pairs of consecutive k: one packed FP32x2 FMA
  // (two IEEE FMAs, each rounded as fmaf) per pair and position, which halves
  // the issued multiply-add instructions; FP64 accumulators one by one
  constexpr bool kPacked = std::is_same<A, float>::value;
  static_assert(KB % 2 == 0, "k pairs");
  A acc[kPacked ? 1 : KB][VEC];
  float2 accp[kPacked ? KB / 2 : 1][VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    if constexpr (kPacked) {
#pragma unroll
      for (int kp = 0; kp < KB / 2; ++kp) accp[kp][v] = make_float2(0.f, 0.f);
    } else {
#pragma unroll
      for (int k = 0; k < KB; ++k) acc[k][v] = A(0);
    }
  }

  for (int l0 = 0; l0 < L; l0 += kLChunk) {
    const int lc = min(kLChunk, L - l0);
    __syncthreads();
    for (int i = tid; i < kLChunk * KB; i += kColsThreads) {
      const int l = i / KB, k = i - (i / KB) * KB;
      const int64_t e = (int64_t)(l0 + l) * K + kb0 + k;
      Fs[l][k] = (l < lc && kb0 + k < K && TK_DBG_IN(e, e, (int64_t)L * K)) ? F[e] : A(0);
    }
    __syncthreads();
    for (int ll = 0; ll < lc; ++ll) {
      const int l = l0 + ll;
      cp_async_wait<kDepth - 1>();
      A x[VEC];
      const unsigned char* slot = &ring[l % kDepth][tid][0];
      if constexpr (sizeof(TIn) == 2 && VEC == 8) {
        const uint4 q = *reinterpret_cast<const uint4*>(slot);
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          x[2 * j] = __uint_as_float(w[j] << 16);
          x[2 * j + 1] = __uint_as_float(w[j] & 0xFFFF0000u);
        }
      } else if constexpr (sizeof(TIn) == 2) {
        const uint2 q = *reinterpret_cast<const uint2*>(slot);
        x[0] = __uint_as_float(q.x << 16);
        x[1] = __uint_as_float(q.x & 0xFFFF0000u);
        x[2] = __uint_as_float(q.y << 16);
        x[3] = __uint_as_float(q.y & 0xFFFF0000u);
      } else {
        const TIn* q = reinterpret_cast<const TIn*>(slot);
#pragma unroll
        for (int v = 0; v < VEC; ++v) x[v] = q[v];
      }
      if (active && l + kDepth < L)
        Slot<TIn, VEC>::copy(&ring[l % kDepth][tid][0], xp + (int64_t)(l + kDepth) * C);
      cp_async_commit();
      if constexpr (kPacked) {
        const float2* f2 = reinterpret_cast<const float2*>(&Fs[ll][0]);
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const float2 xx = make_float2(x[v], x[v]);
#pragma unroll
          for (int kp = 0; kp < KB / 2; ++kp) accp[kp][v] = __ffma2_rn(f2[kp], xx, accp[kp][v]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          const A f = Fs[ll][k];
#pragma unroll
          for (int v = 0; v < VEC; ++v) acc[k][v] = fma(f, x[v], acc[k][v]);
        }
      }
    }
  }
  cp_async_wait<0>();
  if (!active) return;
  TOut* yp = Y + (r * K + kb0) * C + c;
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    if (kb0 + k < K) {
      TOut o[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        if constexpr (kPacked) o[v] = OutCvt<TOut>::run((k & 1) ? accp[k / 2][v].y : accp[k / 2][v].x);
        else o[v] = OutCvt<TOut>::run(acc[k][v]);
      }
      VecStore<TOut, VEC>::run(yp + (int64_t)k * C, o);
    }
  }
}

// ---------------------------------------------------------------------------
// ttm_rows_pipe: last mode (C == 1) with each thread owning one fibre (row r)
// and streaming it VEC elements at a time through its private cp.async ring;
// F is broadcast from shared memory.  Requires L % VEC == 0 and aligned rows.
// Consecutive threads read rows L apart; the two halves of each 32-byte sector
// are used by consecutive steps of the same thread (cp.async.ca keeps them in
// L1 for 8-byte slots; 16-byte slots fetch whole sectors).
// ---------------------------------------------------------------------------
template <typename TIn, typename TOut, int KB, int VEC>
__global__ void __launch_bounds__(kColsThreads, (KB * sizeof(typename AccOf<TIn>::type) <= 96) ? 2 : 1)
    ttm_rows_pipe_kernel(const TIn* __restrict__ X, const typename AccOf<TIn>::type* __restrict__ F,
                         TOut* __restrict__ Y, int64_t R, int L, int K) {
  using A = typename AccOf<TIn>::type;
  constexpr int SB = Slot<TIn, VEC>::kBytes;
  __shared__ __align__(16) A Fs[kColsLChunk][KB];
  __shared__ __align__(16) unsigned char ring[kDepth][kColsThreads][SB];
  const int tid = threadIdx.x;
  const int kb0 = blockIdx.y * KB;
  const int64_t r = (int64_t)blockIdx.x * kColsThreads + tid;
  // this thread reads row r of X (L elements) and writes Y[r, kb0 ..]
  const bool active = r < R && TK_DBG_IN(r * L, r * L + L - 1, R * L) &&
                      TK_DBG_IN(r * K + kb0, r * K + min(K, kb0 + KB) - 1, R * K);
  const TIn* xp = X + (active ? r : 0) * L;
  const int nsteps = L / VEC;
#pragma unroll
  for (int s = 0; s < kDepth; ++s) {
    if (active && s < nsteps) Slot<TIn, VEC>::copy(&ring[s][tid][0], xp + s * VEC);
    cp_async_commit();
  }
  A acc[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) acc[k] = A(0);
  for (int l0 = 0; l0 < L; l0 += kColsLChunk) {
    const int lc = min(kColsLChunk, L - l0);
    __syncthreads();
    for (int i = tid; i < kColsLChunk * KB; i += kColsThreads) {
      const int l = i / KB, k = i - (i / KB) * KB;
      const int64_t e = (int64_t)(l0 + l) * K + kb0 + k;
      Fs[l][k] = (l < lc && kb0 + k < K && TK_DBG_IN(e, e, (int64_t)L * K)) ? F[e] : A(0);
    }
    __syncthreads();
    for (int ll = 0; ll < lc; ll += VEC) {
      const int step = (l0 + ll) / VEC;
      cp_async_wait<kDepth - 1>();
      A x[VEC];
      const unsigned char* slot = &ring[step % kDepth][tid][0];
      if constexpr (sizeof(TIn) == 2) {
        const uint2 q = *reinterpret_cast<const uint2*>(slot);
        x[0] = __uint_as_float(q.x << 16);
        x[1] = __uint_as_float(q.x & 0xFFFF0000u);
        x[2] = __uint_as_float(q.y << 16);
        x[3] = __uint_as_float(q.y & 0xFFFF0000u);
      } else {
        const TIn* q = reinterpret_cast<const TIn*>(slot);
#pragma unroll
        for (int v = 0; v < VEC; ++v) x[v] = q[v];
      }
      if (active && step + kDepth < nsteps)
        Slot<TIn, VEC>::copy(&ring[step % kDepth][tid][0], xp + (step + kDepth) * VEC);
      cp_async_commit();
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
#pragma unroll
        for (int k = 0; k < KB; ++k) acc[k] = fma(Fs[ll + v][k], x[v], acc[k]);
      }
    }
  }
  cp_async_wait<0>();
  if (!active) return;
  TOut* yp = Y + r * K + kb0;
#pragma unroll
  for (int k = 0; k < KB; ++k)
    if (kb0 + k < K) yp[k] = OutCvt<TOut>::run(acc[k]);
}

// ---------------------------------------------------------------------------
// ttm_rows_multi: the last mode (C == 1) for FP32 accumulators when the rows
// are many: each thread owns RV consecutive rows (RV x K accumulators, in k
// pairs for the packed FP32x2 multiply-add), so that every F value read from
// shared memory serves RV rows (one row per thread reads F once per
// multiply-add pair); each row streams through the thread's own cp.async
// slots, kRowsDepth steps of VEC elements in flight per row.  Same sums as
// ttm_rows_pipe (l in increasing order, one FMA per term).
// ---------------------------------------------------------------------------
constexpr int kRowsDepth = 4;
// rows per thread: four up to KB = 20, two above (register budget of two
// 256-thread blocks per SM)
__host__ __device__ constexpr int rows_multi(int KB) { return KB <= 20 ? 4 : 2; }

template <typename TIn, typename TOut, int KB, int VEC, int RV>
__global__ void __launch_bounds__(kColsThreads, 2)
    ttm_rows_multi_kernel(const TIn* __restrict__ X, const float* __restrict__ F, TOut* __restrict__ Y,
                          int64_t R, int L, int K) {
  static_assert(sizeof(TIn) == 4 && VEC == 4 && KB % 2 == 0, "FP32 rows, 16-byte slots");
  constexpr int SB = VEC * 4;
  constexpr int kLChunk = 128;
  __shared__ __align__(16) float Fs[kLChunk][KB];
  // [kRowsDepth][RV][kColsThreads][SB] bytes of dynamic shared memory
  extern __shared__ __align__(16) unsigned char ring_mem[];
  const int tid = threadIdx.x;
  const int kb0 = blockIdx.y * KB;
  auto slot = [&](int st, int j) -> unsigned char* {
    return ring_mem + (((size_t)st * RV + j) * kColsThreads + tid) * SB;
  };
  const int64_t rb = ((int64_t)blockIdx.x * kColsThreads + tid) * RV;
  // rows rb .. rb + RV - 1 (consecutive, L elements each) and Y[r, kb0 ..]
  unsigned act = 0;
#pragma unroll
  for (int j = 0; j < RV; ++j) {
    const int64_t r = rb + j;
    if (r < R && TK_DBG_IN(r * L, r * L + L - 1, R * L) &&
        TK_DBG_IN(r * K + kb0, r * K + min(K, kb0 + KB) - 1, R * K))
      act |= 1u << j;
  }
  const TIn* xb = X + (act ? rb : 0) * L;
  const int nsteps = L / VEC;
#pragma unroll
  for (int st = 0; st < kRowsDepth; ++st) {
#pragma unroll
    for (int j = 0; j < RV; ++j)
      if (((act >> j) & 1) && st < nsteps) cp_async_16(slot(st, j), xb + j * L + st * VEC);
    cp_async_commit();
  }
  float2 acc[RV][KB / 2];
#pragma unroll
  for (int j = 0; j < RV; ++j)
#pragma unroll
    for (int kp = 0; kp < KB / 2; ++kp) acc[j][kp] = make_float2(0.f, 0.f);
  for (int l0 = 0; l0 < L; l0 += kLChunk) {
    const int lc = min(kLChunk, L - l0);
    __syncthreads();
    for (int i = tid; i < kLChunk * KB; i += kColsThreads) {
      const int l = i / KB, k = i - (i / KB) * KB;
      const int64_t e = (int64_t)(l0 + l) * K + kb0 + k;
      Fs[l][k] = (l < lc && kb0 + k < K && TK_DBG_IN(e, e, (int64_t)L * K)) ? F[e] : 0.f;
    }
    __syncthreads();
    for (int ll = 0; ll < lc; ll += VEC) {
      const int step = (l0 + ll) / VEC;
      cp_async_wait<kRowsDepth - 1>();
      float x[RV][VEC];
#pragma unroll
      for (int j = 0; j < RV; ++j) {
        const float4 q = *reinterpret_cast<const float4*>(slot(step % kRowsDepth, j));
        x[j][0] = q.x;
        x[j][1] = q.y;
        x[j][2] = q.z;
        x[j][3] = q.w;
      }
#pragma unroll
      for (int j = 0; j < RV; ++j)
        if (((act >> j) & 1) && step + kRowsDepth < nsteps)
          cp_async_16(slot(step % kRowsDepth, j), xb + j * L + (step + kRowsDepth) * VEC);
      cp_async_commit();
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        const float2* f2 = reinterpret_cast<const float2*>(&Fs[ll + v][0]);
#pragma unroll
        for (int kp = 0; kp < KB / 2; ++kp) {
          const float2 f = f2[kp];
#pragma unroll
          for (int j = 0; j < RV; ++j) acc[j][kp] = __ffma2_rn(f, make_float2(x[j][v], x[j][v]), acc[j][kp]);
        }
      }
    }
  }
  cp_async_wait<0>();
#pragma unroll
  for (int j = 0; j < RV; ++j) {
    if (!((act >> j) & 1)) continue;
    TOut* yp = Y + (rb + j) * K + kb0;
#pragma unroll
    for (int k = 0; k < KB; ++k)
      if (kb0 + k < K) yp[k] = OutCvt<TOut>::run((k & 1) ? acc[j][k / 2].y : acc[j][k / 2].x);
  }
}

// ---------------------------------------------------------------------------
// ttm_rows_tile: the last mode (C == 1) for FP32 rows with L % 8 == 0.  A
// block owns RB = 256 RV consecutive rows and streams them through S stages of
// 8 columns: each stage copies the tile's RB x 8 floats with 16-byte cp.async
// in row order (a warp's copy covers 16 whole 32-byte sectors, where a
// thread-per-row stream touches 32 sectors for 16 bytes each), into rows
// padded to 12 floats so that a quarter-warp's 16-byte reads of 8 consecutive
// rows hit distinct banks; the stage's 8 rows of F arrive in the same
// cp.async group (zero-filled past K).  Thread t owns rows t + 256 j of the
// tile, k in pairs by packed FP32x2 FMAs.  Same sums as ttm_rows_pipe.
// ---------------------------------------------------------------------------
constexpr int kTileLC = 8;    // columns l per stage
constexpr int kTileLD = 12;   // padded row stride of a stage (floats)
__host__ __device__ constexpr int rows_tile_rv(int KB) { return KB <= 20 ? 2 : 1; }
constexpr int kTileStages = 4;
constexpr bool kRowsTileOn = true;

__device__ __forceinline__ void cp_async_4_zfill(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}

template <typename TOut, int KB, int RV>
__global__ void __launch_bounds__(kColsThreads, 2)
    ttm_rows_tile_kernel(const float* __restrict__ X, const float* __restrict__ F, TOut* __restrict__ Y,
                         int64_t R, int L, int K) {
  static_assert(KB % 2 == 0, "k pairs");
  constexpr int RB = kColsThreads * RV;
  constexpr int S = kTileStages;
  // [S][RB][kTileLD] floats of row tiles, then [S][kTileLC][KB] floats of F
  extern __shared__ __align__(16) float tile_mem[];
  float* Xs = tile_mem;
  float* Fs = tile_mem + (size_t)S * RB * kTileLD;
  const int tid = threadIdx.x;
  const int kb0 = blockIdx.y * KB;
  const int64_t rb = (int64_t)blockIdx.x * RB;
  const int nch = L / kTileLC;
  // the block's rows rb .. rb + RB - 1 of X (L elements each), Y[r, kb0 ..]
  const int64_t rlast = min(R, rb + RB) - 1;
  const bool ok = TK_DBG_IN(rb * L, (rlast + 1) * L - 1, R * L) &&
                  TK_DBG_IN(rb * K + kb0, rlast * K + min(K, kb0 + KB) - 1, R * K);
  auto issue = [&](int c) {
    if (c < nch && ok) {
      float* xs = Xs + (size_t)(c % S) * RB * kTileLD;
      const int l0 = c * kTileLC;
#pragma unroll
      for (int q = 0; q < 2 * RV; ++q) {
        const int p = q * kColsThreads + tid;
        const int row = p >> 1, half = p & 1;
        if (rb + row < R) cp_async_16(xs + row * kTileLD + half * 4, X + (rb + row) * L + l0 + half * 4);
      }
      float* fs = Fs + (size_t)(c % S) * kTileLC * KB;
      for (int i = tid; i < kTileLC * KB; i += kColsThreads) {
        const int l = i / KB, k = i - (i / KB) * KB;
        const bool in = kb0 + k < K && TK_DBG_IN((int64_t)(l0 + l) * K + kb0 + k, (int64_t)(l0 + l) * K + kb0 + k, (int64_t)L * K);
        cp_async_4_zfill(fs + i, F + (in ? (int64_t)(l0 + l) * K + kb0 + k : 0), in ? 4 : 0);
      }
    }
    cp_async_commit();
  };
#pragma unroll
  for (int c = 0; c < S - 1; ++c) issue(c);
  float2 acc[RV][KB / 2];
#pragma unroll
  for (int j = 0; j < RV; ++j)
#pragma unroll
    for (int kp = 0; kp < KB / 2; ++kp) acc[j][kp] = make_float2(0.f, 0.f);
  for (int c = 0; c < nch; ++c) {
    cp_async_wait<S - 2>();
    __syncthreads();  // chunk c is in for every thread; chunk c - 1's slot is free
    issue(c + S - 1);
    const float* xs = Xs + (size_t)(c % S) * RB * kTileLD;
    const float* fs = Fs + (size_t)(c % S) * kTileLC * KB;
    // the stage's 8 columns in two halves of 4 (one 16-byte read per row)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float x[RV][4];
#pragma unroll
      for (int j = 0; j < RV; ++j) {
        const float4 a = *reinterpret_cast<const float4*>(xs + (j * kColsThreads + tid) * kTileLD + 4 * h);
        x[j][0] = a.x;
        x[j][1] = a.y;
        x[j][2] = a.z;
        x[j][3] = a.w;
      }
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const float2* f2 = reinterpret_cast<const float2*>(fs + (4 * h + l) * KB);
#pragma unroll
        for (int kp = 0; kp < KB / 2; ++kp) {
          const float2 f = f2[kp];
#pragma unroll
          for (int j = 0; j < RV; ++j) acc[j][kp] = __ffma2_rn(f, make_float2(x[j][l], x[j][l]), acc[j][kp]);
        }
      }
    }
  }
  cp_async_wait<0>();
  if (!ok) return;
#pragma unroll
  for (int j = 0; j < RV; ++j) {
    const int64_t r = rb + j * kColsThreads + tid;
    if (r >= R) continue;
    TOut* yp = Y + r * K + kb0;
#pragma unroll
    for (int k = 0; k < KB; ++k)
      if (kb0 + k < K) yp[k] = OutCvt<TOut>::run((k & 1) ? acc[j][k / 2].y : acc[j][k / 2].x);
  }
}

constexpr int kRowsThreads = 128;
constexpr int kRowsLChunk = 32;

template <typename TIn, typename TOut, int KB>
__global__ void __launch_bounds__(kRowsThreads)
    ttm_rows_kernel(const TIn* __restrict__ X, const typename AccOf<TIn>::type* __restrict__ F,
                    TOut* __restrict__ Y, int64_t R, int L, int K) {
  using A = typename AccOf<TIn>::type;
  __shared__ A Xs[kRowsThreads][kRowsLChunk + 1];
  __shared__ __align__(16) A Fs[kRowsLChunk][KB];
  const int kb0 = blockIdx.y * KB;
  const int64_t r0 = (int64_t)blockIdx.x * kRowsThreads;
  A acc[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) acc[k] = A(0);
  for (int l0 = 0; l0 < L; l0 += kRowsLChunk) {
    const int lc = min(kRowsLChunk, L - l0);
    __syncthreads();
    for (int i = threadIdx.x; i < kRowsThreads * kRowsLChunk; i += kRowsThreads) {
      const int rr = i / kRowsLChunk, ll = i - rr * kRowsLChunk;
      const int64_t r = r0 + rr;
      const int64_t e = r * L + l0 + ll;
      Xs[rr][ll] = (r < R && ll < lc && TK_DBG_IN(e, e, R * L)) ? load_one<TIn>(X + e) : A(0);
    }
    for (int i = threadIdx.x; i < kRowsLChunk * KB; i += kRowsThreads) {
      const int l = i / KB, k = i - (i / KB) * KB;
      const int64_t e = (int64_t)(l0 + l) * K + kb0 + k;
      Fs[l][k] = (l < lc && kb0 + k < K && TK_DBG_IN(e, e, (int64_t)L * K)) ? F[e] : A(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int l = 0; l < kRowsLChunk; ++l) {
      const A x = Xs[threadIdx.x][l];
#pragma unroll
      for (int k = 0; k < KB; ++k) acc[k] = fma(Fs[l][k], x, acc[k]);
    }
  }
  const int64_t r = r0 + threadIdx.x;
  if (r >= R || !TK_DBG_IN(r * K + kb0, r * K + min(K, kb0 + KB) - 1, R * K)) return;
  TOut* yp = Y + r * K + kb0;
#pragma unroll
  for (int k = 0; k < KB; ++k)
    if (kb0 + k < K) yp[k] = OutCvt<TOut>::run(acc[k]);
}

int pick_kb(int64_t K) {
  if (K <= 8) return 8;
  if (K <= 16) return 16;
  if (K <= 20) return 20;
  if (K <= 24) return 24;
  return 32;
}

// Element loaders of the staged short-row kernel (common.cuh).
struct LoadF32 {
  const float* p;
  __device__ __forceinline__ float operator()(int64_t e) const { return __ldg(p + e); }
};
struct LoadBF16 {
  const unsigned short* p;
  __device__ __forceinline__ float operator()(int64_t e) const { return bf16_to_float(__ldg(p + e)); }
};

template <typename TIn, typename TOut, int KB, int VEC>
int launch_cols_pipe(dim3 grid, const TIn* X, const typename AccOf<TIn>::type* F, TOut* Y, int64_t R,
                     int64_t L, int64_t C, int64_t K, cudaStream_t s) {
  constexpr int SB = Slot<TIn, VEC>::kBytes;
  constexpr size_t ring = (size_t)pipe_depth<SB>() * kColsThreads * SB;
  auto kern = ttm_cols_pipe_kernel<TIn, TOut, KB, VEC>;
  // (the static F chunk counts against the default 48 KB too)
  TK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring));
  kern<<<grid, kColsThreads, ring, s>>>(X, F, Y, R, (int)L, C, (int)K);
  return TUCKER_OK;
}

template <typename TIn, typename TOut, int KB>
int launch_kb(const TIn* X, int64_t R, int64_t L, int64_t C, const typename AccOf<TIn>::type* F,
              int64_t K, TOut* Y, cudaStream_t s) {
  const unsigned gy = (unsigned)((K + KB - 1) / KB);
  constexpr int V = sizeof(TIn) == 8 ? 2 : 4;
  // (16-byte slots for BF16 columns measured slower than 8-byte ones)
  constexpr int Vc = V;
  if constexpr (sizeof(TIn) != 8) {
    // short fibres of the last mode: whole rows staged through shared memory
    if (C == 1) {
      int rc = TUCKER_OK;
      bool done;
      if constexpr (sizeof(TIn) == 4)
        done = try_launch_rows_staged(LoadF32{reinterpret_cast<const float*>(X)}, R, L,
                                      reinterpret_cast<const float*>(F), K, Y, s, &rc);
      else
        done = try_launch_rows_staged(LoadBF16{reinterpret_cast<const unsigned short*>(X)}, R, L,
                                      reinterpret_cast<const float*>(F), K, Y, s, &rc);
      if (done) return rc;
    }
  }
  if constexpr (sizeof(TIn) == 4) {
    // FP32 rows of a multiple of 8 elements: row tiles staged by stages of 8
    // columns (enough blocks for one per SM), where measured faster than the
    // multi-row kernel: rows of up to 64 elements (64^5 and 16 x 64^4 mode-4
    // roots 2.36 -> 2.01 and 0.60 -> 0.52 ms) and inputs up to 2^28 elements
    // (20 x 200^3 mode 3: 0.291 -> 0.276 ms); above that, rows of 200 ran 4-5 %
    // slower than with four rows per thread
    if (C == 1 && kRowsTileOn && L % kTileLC == 0 && (uintptr_t)X % 16 == 0 &&
        (L <= 64 || R * L <= ((int64_t)1 << 28)) &&
        R >= (int64_t)rows_tile_rv(KB) * kColsThreads * sm_count()) {
      constexpr int RV = rows_tile_rv(KB);
      const int64_t rbk = (int64_t)RV * kColsThreads;
      const int64_t gx = (R + rbk - 1) / rbk;
      constexpr size_t smem = ((size_t)kTileStages * rbk * kTileLD + (size_t)kTileStages * kTileLC * KB) * 4;
      auto kern = ttm_rows_tile_kernel<TOut, KB, RV>;
      TK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      kern<<<dim3((unsigned)gx, gy), kColsThreads, smem, s>>>(reinterpret_cast<const float*>(X),
                                                             reinterpret_cast<const float*>(F), Y, R,
                                                             (int)L, (int)K);
      TK_LAUNCH_CHECK("ttm_rows_tile");
      return TUCKER_OK;
    }
    // many long FP32 rows: RV rows per thread (enough blocks for two per SM;
    // measured on C == 1 roots: 200^4 mode 3 2.97 -> 2.45 ms, 20 x 200^3
    // 0.313 -> 0.291 ms; rows of 64 or fewer elements no faster)
    if (C == 1 && L >= 128 && L % V == 0 && (uintptr_t)X % (V * sizeof(TIn)) == 0 &&
        R >= (int64_t)rows_multi(KB) * kColsThreads * 2 * sm_count()) {
      constexpr int RV = rows_multi(KB);
      const int64_t gx = (R + (int64_t)RV * kColsThreads - 1) / ((int64_t)RV * kColsThreads);
      constexpr size_t ring = (size_t)kRowsDepth * RV * kColsThreads * 16;
      auto kern = ttm_rows_multi_kernel<TIn, TOut, KB, 4, RV>;
      TK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring));
      kern<<<dim3((unsigned)gx, gy), kColsThreads, ring, s>>>(X, reinterpret_cast<const float*>(F), Y, R,
                                                              (int)L, (int)K);
      TK_LAUNCH_CHECK("ttm_rows_multi");
      return TUCKER_OK;
    }
  }
  if (C == 1 && L % V == 0 && (uintptr_t)X % (V * sizeof(TIn)) == 0) {
    const int64_t gx = (R + kColsThreads - 1) / kColsThreads;
    ttm_rows_pipe_kernel<TIn, TOut, KB, V><<<dim3((unsigned)gx, gy), kColsThreads, 0, s>>>(
        X, F, Y, R, (int)L, (int)K);
    TK_LAUNCH_CHECK("ttm_rows_pipe");
    return TUCKER_OK;
  }
  if (C == 1) {
    const int64_t gx = (R + kRowsThreads - 1) / kRowsThreads;
    ttm_rows_kernel<TIn, TOut, KB><<<dim3((unsigned)gx, gy), kRowsThreads, 0, s>>>(X, F, Y, R,
                                                                                   (int)L, (int)K);
    TK_LAUNCH_CHECK("ttm_rows");
    return TUCKER_OK;
  }
  const int64_t total = R * C;
  if (Vc != V && C % Vc == 0 && (uintptr_t)X % (Vc * sizeof(TIn)) == 0) {
    const int64_t gx = (total / Vc + kColsThreads - 1) / kColsThreads;
    const int rc = launch_cols_pipe<TIn, TOut, KB, Vc>(dim3((unsigned)gx, gy), X, F, Y, R, L, C, K, s);
    if (rc) return rc;
    TK_LAUNCH_CHECK("ttm_cols");
    return TUCKER_OK;
  }
  const bool vec_ok = (C % V == 0) && ((uintptr_t)X % (V * sizeof(TIn)) == 0) &&
                      ((uintptr_t)Y % (V * sizeof(TOut)) == 0);
  if (vec_ok) {
    const int64_t gx = (total / V + kColsThreads - 1) / kColsThreads;
    const int rc = launch_cols_pipe<TIn, TOut, KB, V>(dim3((unsigned)gx, gy), X, F, Y, R, L, C, K, s);
    if (rc) return rc;
  } else {
    const int64_t gx = (total + kColsThreads - 1) / kColsThreads;
    ttm_cols_kernel<TIn, TOut, KB, 1><<<dim3((unsigned)gx, gy), kColsThreads, 0, s>>>(
        X, F, Y, R, (int)L, C, (int)K);
  }
  TK_LAUNCH_CHECK("ttm_cols");
  return TUCKER_OK;
}

template <typename TIn, typename TOut>
int launch_typed(const void* X, int64_t R, int64_t L, int64_t C, const void* F, int64_t K,
                 void* Y, cudaStream_t s) {
  using A = typename AccOf<TIn>::type;
  const TIn* x = static_cast<const TIn*>(X);
  const A* f = static_cast<const A*>(F);
  TOut* y = static_cast<TOut*>(Y);
  switch (pick_kb(K)) {
    case 8: return launch_kb<TIn, TOut, 8>(x, R, L, C, f, K, y, s);
    case 16: return launch_kb<TIn, TOut, 16>(x, R, L, C, f, K, y, s);
    case 20: return launch_kb<TIn, TOut, 20>(x, R, L, C, f, K, y, s);
    case 24: return launch_kb<TIn, TOut, 24>(x, R, L, C, f, K, y, s);
    default: return launch_kb<TIn, TOut, 32>(x, R, L, C, f, K, y, s);
  }
}

}  // namespace

int launch_ttm(int x_dtype, const void* X, int64_t R, int64_t L, int64_t C, const void* F,
               int64_t K, void* Y, int y_dtype, cudaStream_t s) {
  if (R * C == 0 || K == 0) return TUCKER_OK;
  if (R * C / kColsThreads >= (int64_t)INT32_MAX || L > INT32_MAX || K > INT32_MAX)
    return fail(TUCKER_ERR_UNSUPPORTED, "ttm: tensor too large for the grid");
  switch (x_dtype) {
    case TUCKER_F32:
      if (y_dtype != TUCKER_F32) return fail(TUCKER_ERR_UNSUPPORTED, "ttm: FP32 input needs FP32 output");
      if ((kernel_policy() & 5) == 4 && ttm_tc_f32_supported(R, L, C, K, X))
        return launch_ttm_tc_f32(static_cast<const float*>(X), R, L, C, static_cast<const float*>(F), K,
                                 static_cast<float*>(Y), s);
      // column case on the tensor cores when a policy bit asks for it:
      // exact integer slices (bit 32) or the TF32 split kernel (bit 64)
      if ((kernel_policy() & 1) == 0 && C > 1) {
        if ((kernel_policy() & 64) && ttm_tf32_supported(R, L, C, K, X))
          return launch_ttm_tf32(static_cast<const float*>(X), R, L, C, static_cast<const float*>(F), K,
                                 static_cast<float*>(Y), s);
        if ((kernel_policy() & (32 | 64)) == 32 && ttm_x3_supported(R, L, C, K, X))
          return launch_ttm_x3(static_cast<const float*>(X), R, L, C, static_cast<const float*>(F), K,
                               static_cast<float*>(Y), s);
      }
      if ((kernel_policy() & 8) == 0 && ttm_slab_preferred(TUCKER_F32, R, L, C, K))
        return launch_ttm_slab(TUCKER_F32, X, R, L, C, static_cast<const float*>(F), K, Y, y_dtype, s);
      return launch_typed<float, float>(X, R, L, C, F, K, Y, s);
    case TUCKER_F64:
      if (y_dtype != TUCKER_F64) return fail(TUCKER_ERR_UNSUPPORTED, "ttm: FP64 input needs FP64 output");
      return launch_typed<double, double>(X, R, L, C, F, K, Y, s);
    case TUCKER_BF16: {
      const bool ybf = y_dtype == TUCKER_BF16;
      if (!ybf && y_dtype != TUCKER_F32)
        return fail(TUCKER_ERR_UNSUPPORTED, "ttm: BF16 input needs FP32 or BF16 output");
      // tensor cores, except for short last-mode fibres (a 128-row tile of
      // rows of at most 32 elements is too little work per pipeline stage)
      // and for column shapes whose tiles are mostly padding (measured: at
      // L = 40, C = 192, 47 % useful, the CUDA cores are 1.3x faster; at
      // L = 48, C = 7680, 75 %, the tensor cores 1.2x)
      const bool tc_any = (kernel_policy() & 16) != 0;
      if ((kernel_policy() & 1) == 0 && (tc_any || !(C == 1 && L <= kStagedMaxL)) &&
          (C == 1 || tc_any || ttm_tc_efficiency(L, C) >= 0.6) && ttm_tc_supported(R, L, C, K, X, nullptr))
        return launch_ttm_tc(X, nullptr, R, L, C, static_cast<const float*>(F), K, Y, ybf, s);
      // short rows (no tensor-core tile): runs of whole slabs through shared memory
      if ((kernel_policy() & 8) == 0 && ttm_slab_preferred(TUCKER_BF16, R, L, C, K))
        return launch_ttm_slab(TUCKER_BF16, X, R, L, C, static_cast<const float*>(F), K, Y, y_dtype, s);
      return ybf ? launch_typed<bf16_t, bf16_t>(X, R, L, C, F, K, Y, s)
                 : launch_typed<bf16_t, float>(X, R, L, C, F, K, Y, s);
    }
    case TUCKER_FP8_E4M3:
      return launch_ttm_fp8(X, R, L, C, static_cast<const float*>(F), K, Y, y_dtype, s);
    case TUCKER_BF16_SPLIT: {
      // hi and lo halves of one buffer; the tensor cores multiply both
      if (y_dtype != TUCKER_F32)
        return fail(TUCKER_ERR_UNSUPPORTED, "ttm: split BF16 input needs FP32 output");
      const void* X_lo = static_cast<const char*>(X) + bf16_split_lo_offset(R * L * C);
      if ((kernel_policy() & 1) != 0 || !ttm_tc_supported(R, L, C, K, X, X_lo))
        return fail(TUCKER_ERR_UNSUPPORTED, "ttm: split BF16 tensors are read by the tensor cores only");
      return launch_ttm_tc(X, X_lo, R, L, C, static_cast<const float*>(F), K, Y, false, s);
    }
    default: return fail(TUCKER_ERR_INVALID_ARG, "ttm: unknown dtype");
  }
}

}  // namespace tk
