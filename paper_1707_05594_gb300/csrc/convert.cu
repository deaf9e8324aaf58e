// convert.cu -- storage conversion for the precision form: FP32 -> BF16 with
// round-to-nearest-even, optionally with the low part lo = bf16(x - hi), so
// that hi + lo carries ~16 significand bits of x.  HBM-bound: one read of 4
// bytes and one (or two) writes of 2 bytes per element, 16-byte accesses.
#include "common.cuh"

namespace tk {
namespace {

constexpr int kCvtThreads = 256;

__global__ void __launch_bounds__(kCvtThreads)
    convert_bf16_kernel(const float* __restrict__ x, uint16_t* __restrict__ hi,
                        uint16_t* __restrict__ lo, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * kCvtThreads * 8;
  for (int64_t i = ((int64_t)blockIdx.x * kCvtThreads + threadIdx.x) * 8; i < n; i += stride) {
    if (i + 8 <= n) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(x + i));
      const float4 b = __ldg(reinterpret_cast<const float4*>(x + i + 4));
      const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
      uint16_t h[8], l[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        h[j] = f2bf(v[j]);
        l[j] = f2bf(v[j] - bf16_to_float(h[j]));
      }
      uint4 hq, lq;
      hq.x = h[0] | ((uint32_t)h[1] << 16);
      hq.y = h[2] | ((uint32_t)h[3] << 16);
      hq.z = h[4] | ((uint32_t)h[5] << 16);
      hq.w = h[6] | ((uint32_t)h[7] << 16);
      *reinterpret_cast<uint4*>(hi + i) = hq;
      if (lo) {
        lq.x = l[0] | ((uint32_t)l[1] << 16);
        lq.y = l[2] | ((uint32_t)l[3] << 16);
        lq.z = l[4] | ((uint32_t)l[5] << 16);
        lq.w = l[6] | ((uint32_t)l[7] << 16);
        *reinterpret_cast<uint4*>(lo + i) = lq;
      }
    } else {
      for (int64_t j = i; j < n; ++j) {
        const uint16_t h = f2bf(x[j]);
        hi[j] = h;
        if (lo) lo[j] = f2bf(x[j] - bf16_to_float(h));
      }
    }
  }
}

}  // namespace
}  // namespace tk

using namespace tk;

extern "C" int tucker_convert_bf16(const float* x, uint16_t* hi, uint16_t* lo, int64_t n,
                                   void* stream) {
  if (!x || !hi || n < 0) return fail(TUCKER_ERR_INVALID_ARG, "tucker_convert_bf16: invalid argument");
  if ((uintptr_t)x % 16 || (uintptr_t)hi % 16 || (lo && (uintptr_t)lo % 16))
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_convert_bf16: buffers must be 16-byte aligned");
  if (n == 0) return TUCKER_OK;
  const int64_t want = (n + kCvtThreads * 8 - 1) / (kCvtThreads * 8);
  const unsigned grid = (unsigned)std::min<int64_t>(want, 16LL * sm_count());
  convert_bf16_kernel<<<grid, kCvtThreads, 0, static_cast<cudaStream_t>(stream)>>>(x, hi, lo, n);
  TK_LAUNCH_CHECK("convert_bf16");
  return TUCKER_OK;
}

extern "C" size_t tucker_bf16_split_lo_offset(int64_t n) { return n > 0 ? bf16_split_lo_offset(n) : 0; }

extern "C" size_t tucker_bf16_split_bytes(int64_t n) {
  return n > 0 ? bf16_split_lo_offset(n) + (size_t)n * 2 : 0;
}
