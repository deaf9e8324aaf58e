// slab_common.cuh -- what the shared-memory-staged CUDA-core TTMs have in
// common (the short-row kernels in ttm_slab.cu and the fused root in
// ttm_fused_root.cu): block size, staging budget, 16-byte cp.async staging in
// the tensor's own type, element conversion and the shared-memory opt-in.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace tk {
namespace slab {

constexpr int kSlabThreads = 256;
constexpr int kSlabSmemX = 32 * 1024;  // bytes of staged input per block

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

template <typename T> struct Elem;
template <> struct Elem<float> {
  __device__ __forceinline__ static float cvt(float v) { return v; }
};
template <> struct Elem<bf16_t> {
  __device__ __forceinline__ static float cvt(bf16_t v) { return bf16_to_float(v.bits); }
};

template <typename T>
__device__ __forceinline__ void store_out(T* p, float v) {
  *p = OutCvt<T>::run(v);
}

// Starts copying n elements from src (global) to dst (shared, 16-byte
// aligned): 16-byte cp.async for the whole chunks when src is 16-byte aligned;
// element copies (complete on return) for the rest, or for everything when it
// is not.
template <typename TIn>
__device__ __forceinline__ void stage_issue(TIn* dst, const TIn* __restrict__ src, int n) {
  constexpr int per = 16 / (int)sizeof(TIn);
  int done = 0;
  if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    const int nch = n / per;
    for (int i = threadIdx.x; i < nch; i += kSlabThreads) cp_async16(dst + i * per, src + i * per);
    done = nch * per;
  }
  for (int e = done + (int)threadIdx.x; e < n; e += kSlabThreads) dst[e] = src[e];
}

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// more than 48 KB of dynamic shared memory needs the opt-in attribute
template <typename Kern>
cudaError_t allow_smem(Kern kern, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace slab
}  // namespace tk
