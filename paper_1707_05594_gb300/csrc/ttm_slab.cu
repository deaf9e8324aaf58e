// ttm_slab.cu -- mode-n TTM (Sec. 2.1) for tensors whose rows after mode n
// are short: Y[r, k, c] = sum_l F[l, k] X[r, l, c] with C < 64.  The slab
// X[r, :, :] (L * C elements) is then small and contiguous, and a run of
// slabs is one contiguous stretch of memory.  A block copies its run (its
// tile) into shared memory with 16-byte cp.async in the tensor's own type
// (FP32 or BF16: no conversion on the copy, all copies in flight at once),
// then computes from shared memory:
//   ttm_rows_slab_kernel  C == 1, BF16: 256 or 512 rows per tile, one or two
//                         rows per thread read as 16-byte vectors when their
//                         byte length allows, F transposed in shared memory
//                         (four l of one k per 16-byte read); the tile's
//                         outputs (one contiguous run) go out through shared
//                         memory with consecutive lanes on consecutive
//                         elements;
//   ttm_rows_slab_f32_kernel  the same for FP32 rows, F as [L][KB] (fewer
//                         registers: twice the blocks per SM at FP32 sizes);
//   ttm_slab_kernel       1 < C < 64: S slabs per tile, PPT positions (r, c)
//                         per thread, 256 apart, so that neighbouring lanes
//                         read neighbouring elements.  (Four consecutive
//                         positions per thread, read together, measured
//                         slower for BF16 at C = 24.)
// (A persistent form with two staging buffers per block was measured slower:
// fewer blocks fit per SM and the prefetch distance of one tile is shorter
// than the load latency.)
// F enters shared memory as [L][KB] FP32 (zero beyond K); accumulation is FP32
// FMA in increasing l, as in the other CUDA-core TTMs.
#include <algorithm>

#include "slab_common.cuh"

namespace tk {
using namespace slab;
namespace {

template <int KB>
__device__ __forceinline__ void load_f(float* Fs, const float* __restrict__ F, int L, int K) {
  for (int i = threadIdx.x; i < L * KB; i += kSlabThreads) {
    const int l = i / KB, k = i - (i / KB) * KB;
    Fs[i] = k < K ? F[(int64_t)l * K + k] : 0.f;
  }
}


// C == 1: a tile of 256 * RPT rows of L elements per block, RPT rows per
// thread (256 apart).  F is kept transposed, Ft[k][l] with l padded to Lp (a
// multiple of 8, zeros beyond L), so that one 16-byte read gives four l of one
// k; the row is read 16 bytes at a time when its byte length allows.  Shared
// memory: Ft, then the staged rows (later the tile's outputs, FP32).
template <typename TIn, typename TOut, int KB, int RPT>
__global__ void __launch_bounds__(kSlabThreads)
    ttm_rows_slab_kernel(const TIn* __restrict__ X, const float* __restrict__ F, TOut* __restrict__ Y,
                         int64_t R, int L, int K) {
  extern __shared__ __align__(16) unsigned char slab_smem[];
  const int Lp = (L + 7) & ~7;
  float* Ft = reinterpret_cast<float*>(slab_smem);
  TIn* Xs = reinterpret_cast<TIn*>(slab_smem + align16((size_t)KB * Lp * 4));
  float* Os = reinterpret_cast<float*>(Xs);
  const int tid = threadIdx.x;
  constexpr int kTile = kSlabThreads * RPT;
  const int64_t r0 = (int64_t)blockIdx.x * kTile;
  // the tile's rows of X and of Y (the same range for every thread, so that
  // a failed check skips the block's accesses but keeps its barriers)
  const int nrows = TK_DBG_IN(r0 * L, (r0 + min((int64_t)kTile, R - r0)) * L - 1, R * L) &&
                            TK_DBG_IN(r0 * K, (r0 + min((int64_t)kTile, R - r0)) * K - 1, R * K)
                        ? (int)min((int64_t)kTile, R - r0)
                        : 0;
  for (int i = tid; i < KB * Lp; i += kSlabThreads) {
    const int k = i / Lp, l = i - (i / Lp) * Lp;
    Ft[i] = (k < K && l < L) ? F[(int64_t)l * K + k] : 0.f;
  }
  stage_issue(Xs, X + r0 * L, nrows * L);
  cp_wait_all();
  __syncthreads();
  constexpr int per = 16 / (int)sizeof(TIn);
  float acc[RPT][KB];
#pragma unroll
  for (int j = 0; j < RPT; ++j)
#pragma unroll
    for (int k = 0; k < KB; ++k) acc[j][k] = 0.f;
  bool act[RPT];
#pragma unroll
  for (int j = 0; j < RPT; ++j) act[j] = tid + kSlabThreads * j < nrows;
  if (act[0]) {
    if ((L * (int)sizeof(TIn)) % 16 == 0) {
      // rows start on 16-byte boundaries: `per` elements of each row per read
      for (int l0 = 0; l0 < L; l0 += per) {
        float x[RPT][per];
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
          const int row = act[j] ? tid + kSlabThreads * j : tid;
          const uint4 v = *reinterpret_cast<const uint4*>(Xs + (int64_t)row * L + l0);
          if constexpr (sizeof(TIn) == 4) {
            x[j][0] = __uint_as_float(v.x);
            x[j][1] = __uint_as_float(v.y);
            x[j][2] = __uint_as_float(v.z);
            x[j][3] = __uint_as_float(v.w);
          } else {
            const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              x[j][2 * q] = __uint_as_float(w[q] << 16);
              x[j][2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < KB; ++k) {
#pragma unroll
          for (int q = 0; q < per; q += 4) {
            const float4 f = *reinterpret_cast<const float4*>(Ft + k * Lp + l0 + q);
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
              acc[j][k] = fmaf(f.x, x[j][q], acc[j][k]);
              acc[j][k] = fmaf(f.y, x[j][q + 1], acc[j][k]);
              acc[j][k] = fmaf(f.z, x[j][q + 2], acc[j][k]);
              acc[j][k] = fmaf(f.w, x[j][q + 3], acc[j][k]);
            }
          }
        }
      }
    } else {
      for (int l = 0; l < L; ++l) {
        float x[RPT];
#pragma unroll
        for (int j = 0; j < RPT; ++j)
          x[j] = act[j] ? Elem<TIn>::cvt(Xs[(int64_t)(tid + kSlabThreads * j) * L + l]) : 0.f;
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          const float f = Ft[k * Lp + l];
#pragma unroll
          for (int j = 0; j < RPT; ++j) acc[j][k] = fmaf(f, x[j], acc[j][k]);
        }
      }
    }
  }
  __syncthreads();  // every read of the staged rows is done: Os reuses them
#pragma unroll
  for (int j = 0; j < RPT; ++j) {
    if (!act[j]) continue;
    const int row = tid + kSlabThreads * j;
#pragma unroll
    for (int k = 0; k < KB; ++k)
      if (k < K) Os[row * K + k] = acc[j][k];
  }
  __syncthreads();
  TOut* y = Y + r0 * K;
  for (int e = tid; e < nrows * K; e += kSlabThreads) store_out<TOut>(y + e, Os[e]);
}

// C == 1, FP32 rows (measured: the register-light form keeps twice the
// blocks per SM of the transposed-F form at FP32 row sizes): a tile of 256
// rows per block, one row per thread, F as [L][KB]; shared memory: F, then
// the staged rows (later the tile's outputs).
template <typename TOut, int KB>
__global__ void __launch_bounds__(kSlabThreads)
    ttm_rows_slab_f32_kernel(const float* __restrict__ X, const float* __restrict__ F,
                             TOut* __restrict__ Y, int64_t R, int L, int K) {
  extern __shared__ __align__(16) unsigned char slab_smem[];
  float* Fs = reinterpret_cast<float*>(slab_smem);
  float* Xs = reinterpret_cast<float*>(slab_smem + align16((size_t)L * KB * 4));
  float* Os = Xs;
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * kSlabThreads;
  // the tile's rows of X and of Y (block-uniform check, as above)
  const int nrows = TK_DBG_IN(r0 * L, (r0 + min((int64_t)kSlabThreads, R - r0)) * L - 1, R * L) &&
                            TK_DBG_IN(r0 * K, (r0 + min((int64_t)kSlabThreads, R - r0)) * K - 1, R * K)
                        ? (int)min((int64_t)kSlabThreads, R - r0)
                        : 0;
  load_f<KB>(Fs, F, L, K);
  stage_issue(Xs, X + r0 * L, nrows * L);
  cp_wait_all();
  __syncthreads();
  float acc[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) acc[k] = 0.f;
  const float* xr = Xs + (int64_t)tid * L;
  if (tid >= nrows) {
    // no row: only the barriers below
  } else if (L % 4 == 0) {
    for (int l0 = 0; l0 < L; l0 += 4) {
      const float4 v = *reinterpret_cast<const float4*>(xr + l0);
      const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int k = 0; k < KB; ++k) acc[k] = fmaf(Fs[(l0 + u) * KB + k], x[u], acc[k]);
    }
  } else {
    for (int l = 0; l < L; ++l) {
      const float x = xr[l];
#pragma unroll
      for (int k = 0; k < KB; ++k) acc[k] = fmaf(Fs[l * KB + k], x, acc[k]);
    }
  }
  __syncthreads();  // every read of the staged rows is done: Os reuses them
  if (tid < nrows) {
#pragma unroll
    for (int k = 0; k < KB; ++k)
      if (k < K) Os[tid * K + k] = acc[k];
  }
  __syncthreads();
  TOut* y = Y + r0 * K;
  for (int e = tid; e < nrows * K; e += kSlabThreads) store_out<TOut>(y + e, Os[e]);
}

// 1 < C < 64: a tile of S slabs per block; positions p = tid + 256 j (j < PPT)
// of the tile's S * C positions, each reading its column X[r, :, c] from
// shared memory.  Shared memory: F [L][KB], then the staged slabs.
template <typename TIn, typename TOut, int KB, int PPT>
__global__ void __launch_bounds__(kSlabThreads)
    ttm_slab_kernel(const TIn* __restrict__ X, const float* __restrict__ F, TOut* __restrict__ Y,
                    int64_t R, int L, int C, int K, int S) {
  extern __shared__ __align__(16) unsigned char slab_smem[];
  float* Fs = reinterpret_cast<float*>(slab_smem);
  TIn* Xs = reinterpret_cast<TIn*>(slab_smem + align16((size_t)L * KB * 4));
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * S;
  const int LC = L * C;
  // the tile's slabs of X and of Y (block-uniform check)
  const int ns = TK_DBG_IN(r0 * LC, (r0 + min((int64_t)S, R - r0)) * LC - 1, R * LC) &&
                         TK_DBG_IN(r0 * K * C, (r0 + min((int64_t)S, R - r0)) * K * C - 1, R * K * C)
                     ? (int)min((int64_t)S, R - r0)
                     : 0;
  load_f<KB>(Fs, F, L, K);
  stage_issue(Xs, X + r0 * LC, ns * LC);
  cp_wait_all();
  __syncthreads();
  const int P = ns * C;
  const SmallDiv dc(C);
  int off[PPT], yo[PPT];
  bool act[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    const int p = tid + kSlabThreads * j;
    act[j] = p < P;
    const int sl = act[j] ? dc.div(p) : 0, c = act[j] ? p - sl * C : 0;
    off[j] = sl * LC + c;
    yo[j] = sl * K * C + c;
  }
  if (!act[0]) return;
  float acc[PPT][KB];
#pragma unroll
  for (int j = 0; j < PPT; ++j)
#pragma unroll
    for (int k = 0; k < KB; ++k) acc[j][k] = 0.f;
  for (int l = 0; l < L; ++l) {
    float x[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) x[j] = act[j] ? Elem<TIn>::cvt(Xs[off[j] + l * C]) : 0.f;
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      const float f = Fs[l * KB + k];
#pragma unroll
      for (int j = 0; j < PPT; ++j) acc[j][k] = fmaf(f, x[j], acc[j][k]);
    }
  }
  TOut* y = Y + r0 * K * C;
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    if (!act[j]) continue;
#pragma unroll
    for (int k = 0; k < KB; ++k)
      if (k < K) store_out<TOut>(y + yo[j] + k * C, acc[j][k]);
  }
}


template <typename TIn, typename TOut, int KB, int RPT>
cudaError_t launch_rows_rpt(const TIn* X, const float* F, TOut* Y, int64_t R, int L, int K, cudaStream_t s) {
  auto kern = ttm_rows_slab_kernel<TIn, TOut, KB, RPT>;
  const size_t tile = (size_t)kSlabThreads * RPT;
  const size_t smem = align16((size_t)KB * ((L + 7) & ~7) * 4) +
                      std::max(tile * L * sizeof(TIn), tile * KB * sizeof(float));
  const cudaError_t e = allow_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)((R + (int64_t)tile - 1) / (int64_t)tile), kSlabThreads, smem, s>>>(X, F, Y, R, L, K);
  return cudaGetLastError();
}

// FP32 rows: the row-major-F kernel; BF16 rows: the transposed-F kernel,
// two rows per thread while a tile's rows and outputs fit in 32 KB each
template <typename TIn, typename TOut, int KB>
cudaError_t launch_rows(const TIn* X, const float* F, TOut* Y, int64_t R, int L, int K, cudaStream_t s) {
  if constexpr (sizeof(TIn) == 4) {
    auto kern = ttm_rows_slab_f32_kernel<TOut, KB>;
    const size_t smem = align16((size_t)L * KB * 4) + std::max((size_t)kSlabThreads * L * sizeof(float),
                                                               (size_t)kSlabThreads * KB * sizeof(float));
    const cudaError_t e = allow_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)((R + kSlabThreads - 1) / kSlabThreads), kSlabThreads, smem, s>>>(X, F, Y, R, L, K);
    return cudaGetLastError();
  } else {
    if (KB <= 16 && 2 * kSlabThreads * L * (int)sizeof(TIn) <= kSlabSmemX)
      return launch_rows_rpt<TIn, TOut, KB, (KB <= 16 ? 2 : 1)>(X, F, Y, R, L, K, s);
    return launch_rows_rpt<TIn, TOut, KB, 1>(X, F, Y, R, L, K, s);
  }
}

template <typename TIn, typename TOut, int KB, int PPT>
cudaError_t launch_slab_ppt(const TIn* X, const float* F, TOut* Y, int64_t R, int L, int C, int K, int S,
                            cudaStream_t s) {
  auto kern = ttm_slab_kernel<TIn, TOut, KB, PPT>;
  const size_t smem = align16((size_t)L * KB * 4) + (size_t)S * L * C * sizeof(TIn);
  const cudaError_t e = allow_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)((R + S - 1) / S), kSlabThreads, smem, s>>>(X, F, Y, R, L, C, K, S);
  return cudaGetLastError();
}

// S slabs per tile: as many as fit in the staging buffer and in PPTMAX
// positions per thread; the positions per thread then follow from S * C.
template <typename TIn, typename TOut, int KB, int PPTMAX>
cudaError_t launch_slab(const TIn* X, const float* F, TOut* Y, int64_t R, int L, int C, int K,
                        cudaStream_t s) {
  const int bySlab = kSlabSmemX / (L * C * (int)sizeof(TIn));
  const int S = std::max(1, std::min(kSlabThreads * PPTMAX / C, bySlab));
  const int P = S * C;
  if (P <= kSlabThreads) return launch_slab_ppt<TIn, TOut, KB, 1>(X, F, Y, R, L, C, K, S, s);
  if (PPTMAX >= 2 && P <= 2 * kSlabThreads)
    return launch_slab_ppt<TIn, TOut, KB, (PPTMAX >= 2 ? 2 : 1)>(X, F, Y, R, L, C, K, S, s);
  return launch_slab_ppt<TIn, TOut, KB, PPTMAX>(X, F, Y, R, L, C, K, S, s);
}

template <typename TIn, typename TOut>
cudaError_t dispatch(const TIn* X, const float* F, TOut* Y, int64_t R, int L, int C, int K, cudaStream_t s) {
  if (C == 1) {
    if (K <= 2) return launch_rows<TIn, TOut, 2>(X, F, Y, R, L, K, s);
    if (K <= 4) return launch_rows<TIn, TOut, 4>(X, F, Y, R, L, K, s);
    if (K <= 6) return launch_rows<TIn, TOut, 6>(X, F, Y, R, L, K, s);
    if (K <= 8) return launch_rows<TIn, TOut, 8>(X, F, Y, R, L, K, s);
    if (K <= 12) return launch_rows<TIn, TOut, 12>(X, F, Y, R, L, K, s);
    if (K <= 16) return launch_rows<TIn, TOut, 16>(X, F, Y, R, L, K, s);
    if (K <= 24) return launch_rows<TIn, TOut, 24>(X, F, Y, R, L, K, s);
    return launch_rows<TIn, TOut, 32>(X, F, Y, R, L, K, s);
  }
  if (K <= 4) return launch_slab<TIn, TOut, 4, 4>(X, F, Y, R, L, C, K, s);
  if (K <= 8) return launch_slab<TIn, TOut, 8, 2>(X, F, Y, R, L, C, K, s);
  if (K <= 16) return launch_slab<TIn, TOut, 16, 2>(X, F, Y, R, L, C, K, s);
  return launch_slab<TIn, TOut, 32, 1>(X, F, Y, R, L, C, K, s);
}

}  // namespace

bool ttm_slab_supported(int x_dtype, int64_t R, int64_t L, int64_t C, int64_t K) {
  if (x_dtype != TUCKER_F32 && x_dtype != TUCKER_BF16) return false;
  if (R < 1 || L < 1 || K < 1 || K > 32 || C < 1 || C >= 64) return false;
  const int64_t es = x_dtype == TUCKER_F32 ? 4 : 2;
  // F as [L][KB] FP32 (KB <= 32) within 16 KB of shared memory
  if (L * 32 * 4 > 16 * 1024) return false;
  if (C == 1) return (int64_t)kSlabThreads * L * es <= kSlabSmemX;
  return L * C * es <= kSlabSmemX / 4 && R <= (int64_t)INT32_MAX;
}

bool ttm_slab_preferred(int x_dtype, int64_t R, int64_t L, int64_t C, int64_t K) {
  // measured: C == 1 rows gain for both types; FP32 slabs with 1 < C are
  // slower than the FP32 column kernel's 16-byte stream
  if (!ttm_slab_supported(x_dtype, R, L, C, K)) return false;
  return C == 1 || x_dtype == TUCKER_BF16;
}

int launch_ttm_slab(int x_dtype, const void* X, int64_t R, int64_t L, int64_t C, const float* F,
                    int64_t K, void* Y, int y_dtype, cudaStream_t s) {
  if (!ttm_slab_supported(x_dtype, R, L, C, K))
    return fail(TUCKER_ERR_UNSUPPORTED, "ttm_slab: shape not supported");
  cudaError_t e;
  if (x_dtype == TUCKER_F32) {
    if (y_dtype != TUCKER_F32) return fail(TUCKER_ERR_UNSUPPORTED, "ttm_slab: FP32 input needs FP32 output");
    e = dispatch<float, float>(static_cast<const float*>(X), F, static_cast<float*>(Y), R, (int)L, (int)C,
                               (int)K, s);
  } else if (y_dtype == TUCKER_BF16) {
    e = dispatch<bf16_t, bf16_t>(static_cast<const bf16_t*>(X), F, static_cast<bf16_t*>(Y), R, (int)L,
                                 (int)C, (int)K, s);
  } else {
    e = dispatch<bf16_t, float>(static_cast<const bf16_t*>(X), F, static_cast<float*>(Y), R, (int)L,
                                (int)C, (int)K, s);
  }
  count_launches(1);
  if (e != cudaSuccess) return fail(TUCKER_ERR_CUDA, std::string("launch ttm_slab: ") + cudaGetErrorString(e));
  return TUCKER_OK;
}

}  // namespace tk
