// gram.cu -- Gram matrix of a mode-n unfolding, W = Z_(n) Z_(n)^T (Sec. 5: the
// SVD of Z_(n) is computed from its Gram and an EVD).
//
// Z is viewed as [R][L][C]; column m of the unfolding is the fibre (r, c) with
// m = r*C + c.  The L x L result is tiled in 64 x 64 blocks; only tiles on or
// below the diagonal are computed (W is symmetric) and mirrored on output.
// The column range is split over blockIdx.y (split-K); every block
// accumulates FP32 products over runs of kRun columns, folds each run into
// FP64 registers, and adds its FP64 partial to W with atomics.  FP64 tensors
// accumulate in FP64 throughout.
#include "common.cuh"

namespace tk {
namespace {

constexpr int kTile = 64;
constexpr int kMStep = 32;
constexpr int kRun = 256;  // columns accumulated in FP32 before folding into FP64
constexpr int kGramThreads = 256;

constexpr int kPad = 4;  // row padding that keeps 16-byte alignment for vector reads

// Loads the kTile x kMStep panel Z[row0 .. row0+63, m0 .. m0+31] into S[mm][a].
// For C > 1 every thread keeps one column m = m0 + (tid % 32) for the whole
// panel, so `base` (the address of Z[r, 0, c] for that column, or NULL past
// the end) is computed once per panel by the caller.
template <typename TIn>
__device__ __forceinline__ void load_panel(const TIn* __restrict__ Z, int64_t L, int64_t C,
                                           int64_t M, int row0, int64_t m0, const TIn* base,
                                           typename AccOf<TIn>::type (*S)[kTile + kPad]) {
  using A = typename AccOf<TIn>::type;
  if (C == 1) {
    // element (l, m) at m*L + l: consecutive threads take consecutive l
    for (int i = threadIdx.x; i < kTile * kMStep; i += kGramThreads) {
      const int a = i % kTile, mm = i / kTile;
      const int64_t l = row0 + a, m = m0 + mm;
      S[mm][a] = (l < L && m < M && TK_DBG_IN(m * L + l, m * L + l, M * L)) ? load_one<TIn>(Z + m * L + l)
                                                                          : A(0);
    }
  } else {
    // element (l, m) at r*L*C + l*C + c: consecutive threads take consecutive m
    const int mm = threadIdx.x % kMStep;
    for (int a = threadIdx.x / kMStep; a < kTile; a += kGramThreads / kMStep) {
      const int64_t l = row0 + a;
      S[mm][a] = (base && l < L) ? load_one<TIn>(base + l * C) : A(0);
    }
  }
}

template <typename TIn>
__global__ void __launch_bounds__(kGramThreads)
    gram_kernel(const TIn* __restrict__ Z, int64_t R, int64_t L, int64_t C, double* __restrict__ W,
                int ntiles, int64_t m_per_block) {
  using A = typename AccOf<TIn>::type;
  __shared__ __align__(16) A As[kMStep][kTile + kPad];
  __shared__ __align__(16) A Bs[kMStep][kTile + kPad];
  // lower-triangular tile index -> (ti, tj), ti >= tj
  int t = blockIdx.x, ti = 0;
  while (t > ti) {
    t -= ti + 1;
    ++ti;
  }
  const int tj = t;
  (void)ntiles;
  const int64_t M = R * C;
  const int64_t mbeg = (int64_t)blockIdx.y * m_per_block;
  const int64_t mend = min(M, mbeg + m_per_block);
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  A acc[4][4];
  double acc64[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[i][j] = A(0);
      acc64[i][j] = 0.0;
    }
  int run = 0;
  for (int64_t m0 = mbeg; m0 < mend; m0 += kMStep) {
    const TIn* base = nullptr;
    if (C > 1) {
      const int64_t m = m0 + threadIdx.x % kMStep;
      if (m < mend) {
        const int64_t r = m / C;
        // this column's fibre Z[r, 0 .. L-1, c]
        if (TK_DBG_IN(r * L * C + (m - r * C), r * L * C + (L - 1) * C + (m - r * C), R * L * C))
          base = Z + r * L * C + (m - r * C);
      }
    }
    __syncthreads();
    load_panel<TIn>(Z, L, C, mend, ti * kTile, m0, base, As);
    load_panel<TIn>(Z, L, C, mend, tj * kTile, m0, base, Bs);
    __syncthreads();
#pragma unroll 8
    for (int mm = 0; mm < kMStep; ++mm) {
      A a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[mm][ty * 4 + i];
        b[i] = Bs[mm][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    run += kMStep;
    if (run >= kRun) {
      run = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc64[i][j] += (double)acc[i][j];
          acc[i][j] = A(0);
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const double v = acc64[i][j] + (double)acc[i][j];
      const int64_t row = (int64_t)ti * kTile + ty * 4 + i;
      const int64_t col = (int64_t)tj * kTile + tx * 4 + j;
      if (row < L && col < L) {
        atomicAdd(&W[row * L + col], v);
        if (ti != tj) atomicAdd(&W[col * L + row], v);
      }
    }
  }
}

}  // namespace

int launch_gram(int z_dtype, const void* Z, int64_t R, int64_t L, int64_t C, double* W,
                cudaStream_t s) {
  const int64_t M = R * C;
  if (L == 0) return TUCKER_OK;
  const int nt = (int)((L + kTile - 1) / kTile);
  const int tiles = nt * (nt + 1) / 2;
  // split the columns so the grid covers the GPU about four times
  const int64_t target_blocks = 4LL * sm_count();
  int64_t splits = std::max<int64_t>(1, target_blocks / tiles);
  int64_t mpb = (M + splits - 1) / splits;
  mpb = std::max<int64_t>(kRun, (mpb + kMStep - 1) / kMStep * kMStep);
  splits = (M + mpb - 1) / mpb;
  if (splits > 65535) {
    splits = 65535;
    mpb = (M + splits - 1) / splits;
    mpb = (mpb + kMStep - 1) / kMStep * kMStep;
    splits = (M + mpb - 1) / mpb;
  }
  if (M == 0) return TUCKER_OK;
  dim3 grid((unsigned)tiles, (unsigned)splits);
  switch (z_dtype) {
    case TUCKER_F32:
      if (!(kernel_policy() & (1 | 512)) && gram_tc_supported(R, L, C, Z))
        return launch_gram_tc(static_cast<const float*>(Z), R, L, C, W, s);
      gram_kernel<float><<<grid, kGramThreads, 0, s>>>(static_cast<const float*>(Z), R, L, C, W,
                                                       tiles, mpb);
      break;
    case TUCKER_F64:
      gram_kernel<double><<<grid, kGramThreads, 0, s>>>(static_cast<const double*>(Z), R, L, C,
                                                        W, tiles, mpb);
      break;
    case TUCKER_BF16:
      gram_kernel<bf16_t><<<grid, kGramThreads, 0, s>>>(static_cast<const bf16_t*>(Z), R, L, C,
                                                        W, tiles, mpb);
      break;
    case TUCKER_FP8_E4M3:
    case TUCKER_BF16_SPLIT:
      return fail(TUCKER_ERR_UNSUPPORTED,
                  "gram: FP8 and split BF16 tensors are read by TTMs only (run STHOSVD on the FP32 tensor)");
    default:
      return fail(TUCKER_ERR_INVALID_ARG, "gram: unknown dtype");
  }
  TK_LAUNCH_CHECK("gram");
  return TUCKER_OK;
}

}  // namespace tk
