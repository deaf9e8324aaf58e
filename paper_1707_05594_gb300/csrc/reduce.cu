// reduce.cu -- squared Frobenius norms in FP64 and the fit of Sec. 2.2.
//
// ||T||^2 - ||G||^2 cancels (the residual is 1e-4..1e-6 of ||T||^2 in the
// target workloads), so both norms are accumulated in double: each thread
// squares FP32/BF16 values in groups of four in FP32 and adds each group to an
// FP64 register; blocks reduce in FP64 and add their sum with one atomic.
#include "common.cuh"

namespace tk {
namespace {

constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double part[kRedThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) part[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = lane < kRedThreads / 32 ? part[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;  // valid in thread 0
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads)
    norm2_kernel(const T* __restrict__ x, int64_t n, double* __restrict__ out) {
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * kRedThreads * 4;
  for (int64_t i = ((int64_t)blockIdx.x * kRedThreads + threadIdx.x) * 4; i < n; i += stride) {
    typename AccOf<T>::type v[4];
    if (i + 4 <= n) {
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = load_one<T>(x + i + j);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = (i + j < n) ? load_one<T>(x + i + j) : 0;
    }
    acc += (double)(v[0] * v[0] + v[1] * v[1]) + (double)(v[2] * v[2] + v[3] * v[3]);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(out, s);
}

// ||hi + lo||^2 of a split BF16 tensor: each value rebuilt in FP32 (exact:
// hi + lo has at most 16 significant bits) and squared in FP64.
__global__ void __launch_bounds__(kRedThreads)
    norm2_split_kernel(const uint16_t* __restrict__ hi, const uint16_t* __restrict__ lo, int64_t n,
                       double* __restrict__ out) {
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * kRedThreads;
  for (int64_t i = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; i < n; i += stride) {
    const double v = (double)(bf16_to_float(hi[i]) + bf16_to_float(lo[i]));
    acc += v * v;
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(out, s);
}

// fit = 1 - sqrt(max(0, ||T||^2 - ||G||^2)) / ||T||, with out[1] = ||G||^2
// already reduced by norm2_kernel.
__global__ void fit_finish_kernel(const double* __restrict__ normT2, double* __restrict__ out) {
  if (threadIdx.x == 0) {
    const double t2 = *normT2;
    double r2 = t2 - out[1];
    if (r2 < 0.0) r2 = 0.0;
    out[0] = 1.0 - sqrt(r2) / sqrt(t2);
  }
}

}  // namespace

int launch_norm2(int dtype, const void* X, int64_t n, double* out, cudaStream_t s) {
  TK_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double), s));
  if (n == 0) return TUCKER_OK;
  const int64_t want = (n + kRedThreads * 4 - 1) / (kRedThreads * 4);
  const unsigned grid = (unsigned)std::min<int64_t>(want, 8LL * sm_count());
  switch (dtype) {
    case TUCKER_F32:
      norm2_kernel<float><<<grid, kRedThreads, 0, s>>>(static_cast<const float*>(X), n, out);
      break;
    case TUCKER_F64:
      norm2_kernel<double><<<grid, kRedThreads, 0, s>>>(static_cast<const double*>(X), n, out);
      break;
    case TUCKER_BF16:
      norm2_kernel<bf16_t><<<grid, kRedThreads, 0, s>>>(static_cast<const bf16_t*>(X), n, out);
      break;
    case TUCKER_FP8_E4M3:
      return launch_norm2_fp8(X, n, out, s);
    case TUCKER_BF16_SPLIT: {
      const uint16_t* h = static_cast<const uint16_t*>(X);
      const uint16_t* l = reinterpret_cast<const uint16_t*>(static_cast<const char*>(X) + bf16_split_lo_offset(n));
      norm2_split_kernel<<<grid, kRedThreads, 0, s>>>(h, l, n, out);
      break;
    }
    default:
      return fail(TUCKER_ERR_INVALID_ARG, "norm2: unknown dtype");
  }
  TK_LAUNCH_CHECK("norm2");
  return TUCKER_OK;
}

int launch_fit(int g_dtype, const void* G, int64_t n, const double* normT2, double* out,
               cudaStream_t s) {
  const int rc = launch_norm2(g_dtype == TUCKER_F64 ? TUCKER_F64 : TUCKER_F32, G, n, out + 1, s);
  if (rc != TUCKER_OK) return rc;
  fit_finish_kernel<<<1, 32, 0, s>>>(normT2, out);
  TK_LAUNCH_CHECK("fit_finish");
  return TUCKER_OK;
}

}  // namespace tk
