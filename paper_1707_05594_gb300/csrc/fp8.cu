// fp8.cu -- FP8 E4M3 storage with one FP32 scale per 64 consecutive elements,
// the FP8 variant of the precision form: conversion from FP32, the TTM that
// reads it (the nodes of the tree whose input is T), and ||T||^2.
//
// Layout of an FP8 tensor of n elements (tucker_fp8_bytes(n) bytes): n E4M3
// codes, then, from the next 256-byte boundary, ceil(n / 64) FP32 scales; the
// stored value of element i is scale[i / 64] * E4M3(code[i]).
//
// Quantisation of one slab of 64: amax = max |x|, s = amax / 448 (s = 1 for an
// all-zero slab), code = E4M3 of x / s rounded to nearest even and saturated.
// The divisions are IEEE single precision, so the codes are reproducible
// bit for bit.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace tk {

size_t fp8_scale_offset(int64_t n) { return align_up((size_t)n); }
size_t fp8_bytes(int64_t n) { return fp8_scale_offset(n) + sizeof(float) * (size_t)((n + 63) / 64); }

namespace {

constexpr int kF8Threads = 256;

__device__ __forceinline__ float e4m3_to_float(uint32_t byte) {
  const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)byte, __NV_E4M3);
  return __half2float(__half(h));
}

__device__ __forceinline__ uint32_t float_to_e4m3(float v) {
  return (uint32_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}

// One warp per slab of 64: lane j quantises elements 2j and 2j + 1.
__global__ void __launch_bounds__(kF8Threads)
    convert_fp8_kernel(const float* __restrict__ x, uint8_t* __restrict__ q,
                       float* __restrict__ sc, int64_t n) {
  const int lane = threadIdx.x & 31;
  const int64_t nslab = (n + 63) / 64;
  const int64_t wstride = ((int64_t)gridDim.x * kF8Threads) >> 5;
  for (int64_t j = ((int64_t)blockIdx.x * kF8Threads + threadIdx.x) >> 5; j < nslab; j += wstride) {
    const int64_t i0 = j * 64 + 2 * lane;
    const float a = i0 < n ? x[i0] : 0.f;
    const float b = i0 + 1 < n ? x[i0 + 1] : 0.f;
    float m = fmaxf(fabsf(a), fabsf(b));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const float s = m > 0.f ? m / 448.0f : 1.0f;
    if (lane == 0) sc[j] = s;
    if (i0 < n) q[i0] = (uint8_t)float_to_e4m3(a / s);
    if (i0 + 1 < n) q[i0 + 1] = (uint8_t)float_to_e4m3(b / s);
  }
}

// Y = X x_n F^T on an FP8 tensor viewed as [R][L][C] with C % 4 == 0: a
// thread owns 4 consecutive c of one r (one 4-byte word per l, inside one
// scale slab since 64 % 4 == 0), KB outputs k of grid row blockIdx.y.
template <typename TOut, int KB>
__global__ void __launch_bounds__(kF8Threads)
    ttm_fp8_cols_kernel(const uint8_t* __restrict__ q, const float* __restrict__ sc,
                        const float* __restrict__ F, TOut* __restrict__ Y, int64_t R, int L,
                        int64_t C, int K) {
  __shared__ __align__(16) float Fs[64][KB];
  const int kb0 = blockIdx.y * KB;
  const int64_t C4 = C / 4;
  const int64_t g = (int64_t)blockIdx.x * kF8Threads + threadIdx.x;
  bool active = g < R * C4;
  int64_t r = 0, c = 0;
  if (active) {
    r = g / C4;
    c = (g - r * C4) * 4;
    // codes X[r, 0 .. L-1, c .. c+3] (their scales follow), outputs Y[r, kb0 .., c .. c+3]
    active = TK_DBG_IN(r * L * C + c, (r * L + L - 1) * C + c + 3, R * L * C) &&
             TK_DBG_IN((r * K + kb0) * C + c, (r * K + min(K, kb0 + KB) - 1) * C + c + 3, R * K * C);
  }
  const int64_t e0 = r * L * C + c;
  float acc[4][KB];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k = 0; k < KB; ++k) acc[j][k] = 0.f;
  for (int l0 = 0; l0 < L; l0 += 64) {
    const int lc = min(64, L - l0);
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * KB; i += kF8Threads) {
      const int l = i / KB, k = i - (i / KB) * KB;
      Fs[l][k] = (l < lc && kb0 + k < K) ? F[(int64_t)(l0 + l) * K + kb0 + k] : 0.f;
    }
    __syncthreads();
    if (active) {
#pragma unroll 2
      for (int l = 0; l < lc; ++l) {
        const int64_t e = e0 + (int64_t)(l0 + l) * C;
        const uint32_t w = __ldg(reinterpret_cast<const unsigned int*>(q + e));
        const float s = __ldg(sc + (e >> 6));
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = e4m3_to_float((w >> (8 * j)) & 0xFFu) * s;
#pragma unroll
        for (int k = 0; k < KB; ++k) {
          const float f = Fs[l][k];
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[j][k] = fmaf(f, v[j], acc[j][k]);
        }
      }
    }
  }
  if (!active) return;
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    if (kb0 + k >= K) break;
    TOut* yp = Y + (r * K + kb0 + k) * C + c;
#pragma unroll
    for (int j = 0; j < 4; ++j) yp[j] = OutCvt<TOut>::run(acc[j][k]);
  }
}

// The same along the last mode (C == 1): a thread owns one r and reads its
// contiguous fibre four codes at a time (L % 4 == 0).
template <typename TOut, int KB>
__global__ void __launch_bounds__(kF8Threads)
    ttm_fp8_rows_kernel(const uint8_t* __restrict__ q, const float* __restrict__ sc,
                        const float* __restrict__ F, TOut* __restrict__ Y, int64_t R, int L, int K) {
  __shared__ __align__(16) float Fs[64][KB];
  const int kb0 = blockIdx.y * KB;
  const int64_t r = (int64_t)blockIdx.x * kF8Threads + threadIdx.x;
  // codes of row r, outputs Y[r, kb0 ..]
  const bool active = r < R && TK_DBG_IN(r * L, r * L + L - 1, R * L) &&
                      TK_DBG_IN(r * K + kb0, r * K + min(K, kb0 + KB) - 1, R * K);
  float acc[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) acc[k] = 0.f;
  for (int l0 = 0; l0 < L; l0 += 64) {
    const int lc = min(64, L - l0);
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * KB; i += kF8Threads) {
      const int l = i / KB, k = i - (i / KB) * KB;
      Fs[l][k] = (l < lc && kb0 + k < K) ? F[(int64_t)(l0 + l) * K + kb0 + k] : 0.f;
    }
    __syncthreads();
    if (active) {
      for (int l = 0; l < lc; l += 4) {
        const int64_t e = r * L + l0 + l;
        const uint32_t w = __ldg(reinterpret_cast<const unsigned int*>(q + e));
        const float s = __ldg(sc + (e >> 6));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float v = e4m3_to_float((w >> (8 * j)) & 0xFFu) * s;
#pragma unroll
          for (int k = 0; k < KB; ++k) acc[k] = fmaf(Fs[l + j][k], v, acc[k]);
        }
      }
    }
  }
  if (!active) return;
  TOut* yp = Y + r * K + kb0;
#pragma unroll
  for (int k = 0; k < KB; ++k)
    if (kb0 + k < K) yp[k] = OutCvt<TOut>::run(acc[k]);
}

// Any shape: a thread per (r, c), one code per l.
template <typename TOut, int KB>
__global__ void __launch_bounds__(kF8Threads)
    ttm_fp8_any_kernel(const uint8_t* __restrict__ q, const float* __restrict__ sc,
                       const float* __restrict__ F, TOut* __restrict__ Y, int64_t R, int L,
                       int64_t C, int K) {
  __shared__ __align__(16) float Fs[64][KB];
  const int kb0 = blockIdx.y * KB;
  const int64_t p = (int64_t)blockIdx.x * kF8Threads + threadIdx.x;
  bool active = p < R * C;
  int64_t r = 0, c = 0;
  if (active) {
    r = p / C;
    c = p - r * C;
    // codes X[r, 0 .. L-1, c], outputs Y[r, kb0 .., c]
    active = TK_DBG_IN(r * L * C + c, (r * L + L - 1) * C + c, R * L * C) &&
             TK_DBG_IN((r * K + kb0) * C + c, (r * K + min(K, kb0 + KB) - 1) * C + c, R * K * C);
  }
  float acc[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) acc[k] = 0.f;
  for (int l0 = 0; l0 < L; l0 += 64) {
    const int lc = min(64, L - l0);
    __syncthreads();
    for (int i = threadIdx.x; i < 64 * KB; i += kF8Threads) {
      const int l = i / KB, k = i - (i / KB) * KB;
      Fs[l][k] = (l < lc && kb0 + k < K) ? F[(int64_t)(l0 + l) * K + kb0 + k] : 0.f;
    }
    __syncthreads();
    if (active) {
      for (int l = 0; l < lc; ++l) {
        const int64_t e = (r * L + l0 + l) * C + c;
        const float v = e4m3_to_float(__ldg(q + e)) * __ldg(sc + (e >> 6));
#pragma unroll
        for (int k = 0; k < KB; ++k) acc[k] = fmaf(Fs[l][k], v, acc[k]);
      }
    }
  }
  if (!active) return;
#pragma unroll
  for (int k = 0; k < KB; ++k)
    if (kb0 + k < K) Y[(r * K + kb0 + k) * C + c] = OutCvt<TOut>::run(acc[k]);
}

// ||X||^2 of an FP8 tensor: squares of groups of four in FP32, added in FP64.
__global__ void __launch_bounds__(kF8Threads)
    norm2_fp8_kernel(const uint8_t* __restrict__ q, const float* __restrict__ sc, int64_t n,
                     double* __restrict__ out) {
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * kF8Threads * 4;
  for (int64_t i = ((int64_t)blockIdx.x * kF8Threads + threadIdx.x) * 4; i < n; i += stride) {
    float g = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (i + j < n) {
        const float v = e4m3_to_float(q[i + j]) * sc[(i + j) >> 6];
        g = fmaf(v, v, g);
      }
    }
    acc += (double)g;
  }
  __shared__ double part[kF8Threads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kF8Threads / 32; ++w) t += part[w];
    atomicAdd(out, t);
  }
}

template <typename TOut, int KB>
int launch_fp8_kb(const uint8_t* q, const float* sc, int64_t R, int64_t L, int64_t C,
                  const float* F, int64_t K, TOut* Y, cudaStream_t s) {
  const unsigned gy = (unsigned)((K + KB - 1) / KB);
  const bool aligned = ((uintptr_t)q % 4) == 0;
  if (C == 1 && L % 4 == 0 && aligned) {
    const int64_t gx = (R + kF8Threads - 1) / kF8Threads;
    ttm_fp8_rows_kernel<TOut, KB><<<dim3((unsigned)gx, gy), kF8Threads, 0, s>>>(q, sc, F, Y, R, (int)L,
                                                                               (int)K);
    TK_LAUNCH_CHECK("ttm_fp8_rows");
    return TUCKER_OK;
  }
  if (C % 4 == 0 && aligned) {
    const int64_t gx = (R * (C / 4) + kF8Threads - 1) / kF8Threads;
    ttm_fp8_cols_kernel<TOut, KB><<<dim3((unsigned)gx, gy), kF8Threads, 0, s>>>(q, sc, F, Y, R, (int)L,
                                                                               C, (int)K);
    TK_LAUNCH_CHECK("ttm_fp8_cols");
    return TUCKER_OK;
  }
  const int64_t gx = (R * C + kF8Threads - 1) / kF8Threads;
  ttm_fp8_any_kernel<TOut, KB><<<dim3((unsigned)gx, gy), kF8Threads, 0, s>>>(q, sc, F, Y, R, (int)L, C,
                                                                            (int)K);
  TK_LAUNCH_CHECK("ttm_fp8_any");
  return TUCKER_OK;
}

template <typename TOut>
int launch_fp8_typed(const uint8_t* q, const float* sc, int64_t R, int64_t L, int64_t C,
                     const float* F, int64_t K, TOut* Y, cudaStream_t s) {
  if (K <= 8) return launch_fp8_kb<TOut, 8>(q, sc, R, L, C, F, K, Y, s);
  return launch_fp8_kb<TOut, 16>(q, sc, R, L, C, F, K, Y, s);
}

}  // namespace

int launch_ttm_fp8(const void* X, int64_t R, int64_t L, int64_t C, const float* F, int64_t K,
                   void* Y, int y_dtype, cudaStream_t s) {
  if (R * C == 0 || K == 0) return TUCKER_OK;
  const int64_t n = R * L * C;
  const uint8_t* q = static_cast<const uint8_t*>(X);
  const float* sc = reinterpret_cast<const float*>(q + fp8_scale_offset(n));
  // tensor cores (codes decoded to a BF16 hi + lo pair in shared memory) where
  // the column shape allows, unless the policy keeps TTMs on the CUDA cores
  if ((kernel_policy() & 1) == 0 && (y_dtype == TUCKER_F32 || y_dtype == TUCKER_BF16) &&
      ttm_tc_fp8_supported(R, L, C, K, q))
    return launch_ttm_tc_fp8(q, sc, R, L, C, F, K, Y, y_dtype == TUCKER_BF16, s);
  if ((R * C + kF8Threads - 1) / kF8Threads >= (int64_t)INT32_MAX || L > INT32_MAX)
    return fail(TUCKER_ERR_UNSUPPORTED, "ttm: tensor too large for the grid");
  if (y_dtype == TUCKER_BF16)
    return launch_fp8_typed<bf16_t>(q, sc, R, L, C, F, K, static_cast<bf16_t*>(Y), s);
  if (y_dtype == TUCKER_F32)
    return launch_fp8_typed<float>(q, sc, R, L, C, F, K, static_cast<float*>(Y), s);
  return fail(TUCKER_ERR_UNSUPPORTED, "ttm: FP8 input needs FP32 or BF16 output");
}

int launch_norm2_fp8(const void* X, int64_t n, double* out, cudaStream_t s) {
  const uint8_t* q = static_cast<const uint8_t*>(X);
  const float* sc = reinterpret_cast<const float*>(q + fp8_scale_offset(n));
  const int64_t blocks = std::min<int64_t>((n / 4 + kF8Threads - 1) / kF8Threads + 1, 8 * sm_count());
  norm2_fp8_kernel<<<(unsigned)blocks, kF8Threads, 0, s>>>(q, sc, n, out);
  TK_LAUNCH_CHECK("norm2_fp8");
  return TUCKER_OK;
}

}  // namespace tk

using namespace tk;

extern "C" {

size_t tucker_fp8_bytes(int64_t n) { return n > 0 ? fp8_bytes(n) : 0; }

int tucker_convert_fp8(const float* x, void* out, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !out)))
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_convert_fp8: invalid argument");
  if (n == 0) return TUCKER_OK;
  if ((uintptr_t)out % kAlign != 0)
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_convert_fp8: out must be 256-byte aligned");
  uint8_t* q = static_cast<uint8_t*>(out);
  float* sc = reinterpret_cast<float*>(q + fp8_scale_offset(n));
  const int64_t nslab = (n + 63) / 64;
  const int64_t blocks = std::min<int64_t>((nslab * 32 + kF8Threads - 1) / kF8Threads, 16 * sm_count());
  convert_fp8_kernel<<<(unsigned)blocks, kF8Threads, 0, static_cast<cudaStream_t>(stream)>>>(x, q, sc, n);
  TK_LAUNCH_CHECK("convert_fp8");
  return TUCKER_OK;
}

}  // extern "C"
