// common.cuh -- small device/host helpers shared by the CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <string>

#include "debug_check.cuh"
#include "internal.h"

#define TK_CUDA_TRY(expr)                                                                \
  do {                                                                                   \
    cudaError_t _e = (expr);                                                             \
    if (_e != cudaSuccess)                                                               \
      return ::tk::fail(TUCKER_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// Launch check: a failed launch returns TUCKER_ERR_CUDA with the kernel name;
// a successful one is counted (tucker_launch_count).
#define TK_LAUNCH_CHECK(name)                                                            \
  do {                                                                                   \
    ::tk::count_launches(1);                                                             \
    cudaError_t _e = cudaGetLastError();                                                 \
    if (_e != cudaSuccess)                                                               \
      return ::tk::fail(TUCKER_ERR_CUDA, std::string("launch ") + (name) + ": " +          \
                                             cudaGetErrorString(_e));                    \
  } while (0)

namespace tk {

// Accumulator / factor type per storage type: double for FP64 tensors, float
// otherwise (BF16 and FP32 tensors accumulate in FP32).
template <typename T>
struct AccOf {
  using type = float;
};
template <>
struct AccOf<double> {
  using type = double;
};

// bfloat16 storage as raw 16-bit patterns (no dependence on cuda_bf16 types in
// the ABI); widening is exact: the bf16 bits are the high half of a float.
struct bf16_t {
  uint16_t bits;
};

__device__ __forceinline__ float bf16_to_float(uint16_t b) {
  return __uint_as_float(((uint32_t)b) << 16);
}

// FP32 -> BF16 with round-to-nearest-even (NaN stays NaN).
__host__ __device__ __forceinline__ uint16_t f2bf(float f) {
  uint32_t u;
#ifdef __CUDA_ARCH__
  u = __float_as_uint(f);
#else
  std::memcpy(&u, &f, 4);
#endif
  if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)((u >> 16) | ((u & 0xFFFFu) ? 0x40u : 0u));
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// Accumulator -> output element conversion.
template <typename T>
struct OutCvt {
  template <typename A>
  static __device__ __forceinline__ T run(A v) {
    return (T)v;
  }
};
template <>
struct OutCvt<bf16_t> {
  template <typename A>
  static __device__ __forceinline__ bf16_t run(A v) {
    return bf16_t{f2bf((float)v)};
  }
};

template <typename T>
__device__ __forceinline__ typename AccOf<T>::type load_one(const T* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ float load_one<bf16_t>(const bf16_t* p) {
  return bf16_to_float(__ldg(reinterpret_cast<const unsigned short*>(p)));
}

// Load VEC consecutive elements (the pointer is VEC*sizeof(T) aligned).
template <typename T, int VEC>
struct VecLoad {
  static __device__ __forceinline__ void run(const T* p, typename AccOf<T>::type* out) {
#pragma unroll
    for (int v = 0; v < VEC; ++v) out[v] = load_one<T>(p + v);
  }
};
template <>
struct VecLoad<float, 4> {
  static __device__ __forceinline__ void run(const float* p, float* out) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    out[0] = q.x; out[1] = q.y; out[2] = q.z; out[3] = q.w;
  }
};
template <>
struct VecLoad<double, 2> {
  static __device__ __forceinline__ void run(const double* p, double* out) {
    const double2 q = __ldg(reinterpret_cast<const double2*>(p));
    out[0] = q.x; out[1] = q.y;
  }
};
template <>
struct VecLoad<bf16_t, 4> {
  static __device__ __forceinline__ void run(const bf16_t* p, float* out) {
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
    out[0] = __uint_as_float(q.x << 16);
    out[1] = __uint_as_float(q.x & 0xFFFF0000u);
    out[2] = __uint_as_float(q.y << 16);
    out[3] = __uint_as_float(q.y & 0xFFFF0000u);
  }
};

template <typename T, int VEC>
struct VecStore {
  template <typename A>
  static __device__ __forceinline__ void run(T* p, const A* v) {
#pragma unroll
    for (int i = 0; i < VEC; ++i) p[i] = (T)v[i];
  }
};
template <>
struct VecStore<float, 4> {
  static __device__ __forceinline__ void run(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct VecStore<double, 2> {
  static __device__ __forceinline__ void run(double* p, const double* v) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};

// Division by a small run-time divisor d (1 <= d < 2^16) for numerators below
// 2^16: q = floor(x * ceil(2^32 / d) / 2^32) is exact there (the error of the
// scaled reciprocal stays below 2^-16 <= 1/d).
struct SmallDiv {
  unsigned m;
  int d;
  __host__ __device__ __forceinline__ explicit SmallDiv(int d_) : m(0), d(d_) {
    if (d_ > 1) m = (unsigned)((0x100000000ull + (unsigned)d_ - 1) / (unsigned)d_);
  }
  __device__ __forceinline__ int div(int x) const { return d == 1 ? x : (int)__umulhi((unsigned)x, m); }
};

// ---------------------------------------------------------------------------
// TTM along the last mode (C == 1) for short fibres (L <= 32): a block takes
// 256 consecutive rows, whose elements are one contiguous run, reads them
// with coalesced loads into shared memory (converted to FP32 by the Load
// functor; row stride L | 1 keeps each thread's row reads conflict-free),
// each thread contracts its row with F from shared memory, and the 256 x K
// outputs leave through shared memory as one contiguous run.  Load(e) returns
// element e of the tensor as a float.
// ---------------------------------------------------------------------------
constexpr int kStagedRows = 256;
constexpr int kStagedMaxL = 32;  // measured: faster than the per-thread fibre stream up to here

template <typename Load, typename TOut, int KB>
__global__ void __launch_bounds__(kStagedRows)
    ttm_rows_staged_kernel(Load ld, const float* __restrict__ F, TOut* __restrict__ Y, int64_t R,
                           int L, int K) {
  extern __shared__ __align__(16) float rs_smem[];
  const int Ls = L | 1;
  float* Xs = rs_smem;                                      // [256][Ls], later [256][kn]
  float* Fs = rs_smem + kStagedRows * (Ls > KB ? Ls : KB);  // [L][KB]
  const int tid = threadIdx.x;
  const int kb0 = blockIdx.y * KB;
  const int64_t r0 = (int64_t)blockIdx.x * kStagedRows;
  const int nrows = (int)min((int64_t)kStagedRows, R - r0);
  for (int i = tid; i < L * KB; i += kStagedRows) {
    const int l = i / KB, k = i - (i / KB) * KB;
    Fs[i] = (kb0 + k < K) ? F[(int64_t)l * K + kb0 + k] : 0.f;
  }
  const int nel = nrows * L;
  const SmallDiv dl(L);
  const int64_t e0 = r0 * L;
  // eight independent loads in flight per thread, then their stores
  constexpr int kU = 8;
  for (int base = 0; base < nel; base += kStagedRows * kU) {
    float v[kU];
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const int e = base + tid + kStagedRows * j;
      v[j] = e < nel ? ld(e0 + e) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const int e = base + tid + kStagedRows * j;
      if (e < nel) {
        const int row = dl.div(e), col = e - row * L;
        Xs[row * Ls + col] = v[j];
      }
    }
  }
  __syncthreads();
  float acc[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) acc[k] = 0.f;
  if (tid < nrows) {
    const float* xr = Xs + tid * Ls;
    for (int l = 0; l < L; ++l) {
      const float x = xr[l];
#pragma unroll
      for (int k = 0; k < KB; ++k) acc[k] = fmaf(Fs[l * KB + k], x, acc[k]);
    }
  }
  __syncthreads();
  // outputs of this k block: row t, columns kb0 .. kb0 + kn - 1
  const int kn = min(KB, K - kb0);
  if (tid < nrows) {
#pragma unroll
    for (int k = 0; k < KB; ++k)
      if (k < kn) Xs[tid * kn + k] = acc[k];
  }
  __syncthreads();
  if (kn == K) {
    TOut* yb = Y + r0 * K;
    for (int e = tid; e < nrows * K; e += kStagedRows) yb[e] = OutCvt<TOut>::run(Xs[e]);
  } else {
    const SmallDiv dk(kn);
    for (int e = tid; e < nrows * kn; e += kStagedRows) {
      const int row = dk.div(e), k = e - row * kn;
      Y[(r0 + row) * K + kb0 + k] = OutCvt<TOut>::run(Xs[e]);
    }
  }
}

// Launches ttm_rows_staged_kernel when it applies (C == 1, L <= 32); returns
// false (nothing launched) otherwise.
template <typename Load, typename TOut>
bool try_launch_rows_staged(Load ld, int64_t R, int64_t L, const float* F, int64_t K, TOut* Y,
                            cudaStream_t s, int* rc) {
  if (L > kStagedMaxL || L < 1 || K < 1) return false;
  const int KB = K <= 8 ? 8 : (K <= 16 ? 16 : 32);
  const size_t rowf = (size_t)((L | 1) > KB ? (L | 1) : KB);
  const size_t smem = ((size_t)kStagedRows * rowf + (size_t)L * KB) * sizeof(float);
  const dim3 grid((unsigned)((R + kStagedRows - 1) / kStagedRows), (unsigned)((K + KB - 1) / KB));
  // more than 48 KB of dynamic shared memory needs the opt-in attribute
  auto run = [&](auto kern) -> cudaError_t {
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<grid, kStagedRows, smem, s>>>(ld, F, Y, R, (int)L, (int)K);
    return cudaGetLastError();
  };
  cudaError_t e;
  switch (KB) {
    case 8: e = run(ttm_rows_staged_kernel<Load, TOut, 8>); break;
    case 16: e = run(ttm_rows_staged_kernel<Load, TOut, 16>); break;
    default: e = run(ttm_rows_staged_kernel<Load, TOut, 32>); break;
  }
  count_launches(1);
  *rc = (e == cudaSuccess) ? TUCKER_OK
                           : fail(TUCKER_ERR_CUDA, std::string("launch ttm_rows_staged: ") + cudaGetErrorString(e));
  return true;
}

inline int64_t prod(const int64_t* d, int a, int b) {
  int64_t p = 1;
  for (int i = a; i < b; ++i) p *= d[i];
  return p;
}

// Number of SMs of the current device (cached per device).
int sm_count();

// ---- launchers implemented in the .cu files --------------------------------
// Y = X x_n F^T on a tensor viewed as [R][L][C] (R = modes before n, C = modes
// after n).  x_dtype: TUCKER_F32 / F64 / BF16; F in the factor type (double
// for F64, else float); y_dtype: F64 for F64 input, F32 or BF16 otherwise.
int launch_ttm(int x_dtype, const void* X, int64_t R, int64_t L, int64_t C, const void* F,
               int64_t K, void* Y, int y_dtype, cudaStream_t s);
// Tensor-core TTM for BF16 tensors (ttm_tc.cu): X, optionally plus a low part
// X_lo, contracted with FP32 F; Y is FP32 or BF16.
bool ttm_tc_supported(int64_t R, int64_t L, int64_t C, int64_t K, const void* X,
                      const void* X_lo);
int launch_ttm_tc(const void* X, const void* X_lo, int64_t R, int64_t L, int64_t C,
                  const float* F, int64_t K, void* Y, bool y_bf16, cudaStream_t s);
// useful share of the tensor-core tiles for a shape (l stages of 64, 128-position tiles)
double ttm_tc_efficiency(int64_t L, int64_t C);
// the two root children (modes a, b = a + 2) of a BF16 tensor from one pass
// over it blocked by mode a + 1 (ttm_tc_pair_kernel)
bool ttm_tc_pair_supported(const int64_t* dims, int N, int a, int b, int64_t Ka, int64_t Kb, const void* X);
int launch_ttm_tc_pair(const void* X, const int64_t* dims, int N, int a, int b, const float* Fa, int64_t Ka,
                       const float* Fb, int64_t Kb, void* Ya, void* Yb, bool y_bf16, cudaStream_t s);
// Short-row TTMs (ttm_slab.cu): C == 1 with 256 * L elements in 32 KB, or
// 1 < C < 64 with a slab of L * C elements in 8 KB; FP32 or BF16 input, F
// FP32, K <= 32; Y FP32 (or BF16 for BF16 input).
bool ttm_slab_supported(int x_dtype, int64_t R, int64_t L, int64_t C, int64_t K);
// the shapes launch_ttm sends to the short-row kernels (measured faster there)
bool ttm_slab_preferred(int x_dtype, int64_t R, int64_t L, int64_t C, int64_t K);
int launch_ttm_slab(int x_dtype, const void* X, int64_t R, int64_t L, int64_t C, const float* F,
                    int64_t K, void* Y, int y_dtype, cudaStream_t s);
// Fused root (ttm_slab.cu): T x_a Fa^T and T x_b Fb^T (a < b) from one read
// of T (FP32 -> FP32, BF16 -> BF16 or FP32), Ya as [A][Ka][M Lb B], Yb as
// [A La M][Kb][B]; the shape must pass fused_root_fits.
int launch_ttm_fused_root(int dtype, const void* X, const int64_t* L, int N, int a, int b,
                          const float* Fa, int64_t Ka, const float* Fb, int64_t Kb, void* Ya, void* Yb,
                          int y_dtype, cudaStream_t s);
// FP8 E4M3 tensors with per-64 scales (fp8.cu): Y = X x_n F^T with Y FP32 or
// BF16, and ||X||^2; X is the whole tensor (R * L * C elements) in the layout
// of tucker_fp8_bytes.
size_t fp8_scale_offset(int64_t n);
// FP8 column-case TTM on the tensor cores (ttm_tc.cu): Xq the codes, scales
// one FP32 per 64 elements of the row-major tensor, Y FP32 or BF16.
bool ttm_tc_fp8_supported(int64_t R, int64_t L, int64_t C, int64_t K, const void* Xq);
int launch_ttm_tc_fp8(const void* Xq, const float* scales, int64_t R, int64_t L, int64_t C,
                      const float* F, int64_t K, void* Y, bool y_bf16, cudaStream_t s);
int launch_ttm_fp8(const void* X, int64_t R, int64_t L, int64_t C, const float* F, int64_t K,
                   void* Y, int y_dtype, cudaStream_t s);
int launch_norm2_fp8(const void* X, int64_t n, double* out, cudaStream_t s);
// Tensor-core TTM for FP32 tensors (column case, ttm_tc.cu): FP32 tiles split
// into BF16 hi + lo in shared memory, products within ~2^-16 of FP32.
// FP32 TTMs on the tensor cores in TF32 with split operands (ttm_tf32.cu):
// one TTM of the column case, or the two root children of a sweep (modes a
// and b = a + 2) from one pass over T blocked by mode a + 1 (L2 reuse).
bool ttm_tf32_supported(int64_t R, int64_t L, int64_t C, int64_t K, const void* X);
int launch_ttm_tf32(const float* X, int64_t R, int64_t L, int64_t C, const float* F, int64_t K, float* Y,
                    cudaStream_t s);
bool ttm_tf32_pair_supported(const int64_t* dims, int N, int a, int b, int64_t Ka, int64_t Kb,
                             const void* X);
int launch_ttm_tf32_pair(const float* X, const int64_t* dims, int N, int a, int b, const float* Fa, int64_t Ka,
                         const float* Fb, int64_t Kb, float* Ya, float* Yb, cudaStream_t s);
// the same with exact BF16 integer slices (ttm_x3_kernel, the default)
bool ttm_x3_supported(int64_t R, int64_t L, int64_t C, int64_t K, const void* X);
int launch_ttm_x3(const float* X, int64_t R, int64_t L, int64_t C, const float* F, int64_t K, float* Y,
                  cudaStream_t s);
bool ttm_x3_pair_supported(const int64_t* dims, int N, int a, int b, int64_t Ka, int64_t Kb, const void* X);
int launch_ttm_x3_pair(const float* X, const int64_t* dims, int N, int a, int b, const float* Fa, int64_t Ka,
                       const float* Fb, int64_t Kb, float* Ya, float* Yb, cudaStream_t s);

bool ttm_tc_f32_supported(int64_t R, int64_t L, int64_t C, int64_t K, const void* X);
int launch_ttm_tc_f32(const float* X, int64_t R, int64_t L, int64_t C, const float* F, int64_t K,
                      float* Y, cudaStream_t s);
// kernel-selection policy (tucker_set_kernel_policy): 0 = auto, 1 = CUDA cores only
int kernel_policy();
// device address of the library's device error word (tucker_device_status)
int* device_status_ptr();
// W += Z_(n) Z_(n)^T for Z viewed as [R][L][C] (W must be zeroed first).
int launch_gram(int z_dtype, const void* Z, int64_t R, int64_t L, int64_t C, double* W,
                cudaStream_t s);
// the same for FP32 Z on the tensor cores (gram_tc.cu)
bool gram_tc_supported(int64_t R, int64_t L, int64_t C, const void* Z);
int launch_gram_tc(const float* Z, int64_t R, int64_t L, int64_t C, double* W, cudaStream_t s);
// out[0] += sum x^2 (out must be zeroed first)
int launch_norm2(int dtype, const void* X, int64_t n, double* out, cudaStream_t s);
// fit from G (factor type) and normT2
int launch_fit(int g_dtype, const void* G, int64_t n, const double* normT2, double* out,
               cudaStream_t s);

// Per-matrix state of the eigensolver (pointers into its scratch).
struct EigDesc {
  const double* W;
  void* F;
  const void* F0;  // warm start: L x K row-major input factor (or NULL)
  float* V0;       // [K][L]
  float* theta;    // [K]
  float* HV;       // [L][L] parked reflectors
  double* Q;       // [K][L]
  double* Y;       // [K][L]
  double* Qp;      // [K][L] previous basis (warm start)
  double* stat;    // [0] delta1, [1] delta2; ((int*)stat)[4] = need_cold flag
  int L, K;
};
// Carves one matrix's scratch (eig_bytes_per_matrix(L, K) bytes at p).
void eig_desc_layout(EigDesc& d, char* p, int L, int K);
// The eigensolver over `count` matrices whose descriptors are in device
// memory (dev; their F / F0 fields are byte offsets from f_base / f0_base),
// with maxL / maxK bounding every L / K.  A non-NULL f0_base selects the warm
// start from the input factors, with the full path for the matrices whose
// warm check fails; `cold` (1 + count ints of device memory) lists them.
int launch_eig_batched(const EigDesc* dev, int count, int maxL, int maxK, int f_dtype,
                       char* f_base, const char* f0_base, int* cold, cudaStream_t s);

struct EigProblem {
  const double* W;         // L x L
  void* F;                 // L x K output
  int L, K;
  const void* F0 = nullptr;  // optional L x K starting subspace (factor type)
};
int launch_eig_topk(const EigProblem* probs, int batch, int f_dtype, void* ws, size_t ws_bytes,
                    cudaStream_t s);

}  // namespace tk
