// ttm_fused_root.cu -- the fused root of the TTM-tree: both root children
// (T x_a Fa^T and T x_b Fb^T, Sec. 2.1; the TTM-tree of Sec. 3.1) computed
// from one read of T.  T is staged into shared memory block by block with
// the helpers of slab_common.cuh and both contractions are taken from there,
// FP32 FMA in increasing l as in the single TTMs.
#include <algorithm>
#include <string>

#include "slab_common.cuh"

namespace tk {
using namespace slab;
namespace {

// Fused root (both root children of the TTM-tree from one read of T).  T is
// viewed as [A][La][M][Lb][B] (modes a < b; A, M, B the products of the
// lengths before a, between a and b, after b); a block stages S consecutive
// blocks X[alpha, :, :, :, :] (La M Lb B elements each) and computes from
// shared memory
//   Ya[alpha, ka, q] = sum_la Fa[la, ka] X[alpha, la, q]     (q = (mu, lb, beta))
//   Yb[r, kb, beta]  = sum_lb Fb[lb, kb] X[r, lb, beta]      (r = (alpha, la, mu))
// i.e. T x_a Fa^T as [A][Ka][M Lb B] and T x_b Fb^T as [A La M][Kb][B], each
// position's sum in increasing l as in the single TTMs.  When B == 1 and a
// row of Lb elements is a whole number of 16-byte vectors, the second
// contraction reads its rows as vectors against Fb transposed.
template <typename TIn, typename TOut, int KBA, int KBB>
__global__ void __launch_bounds__(kSlabThreads)
    ttm_fused_root_kernel(const TIn* __restrict__ X, const float* __restrict__ Fa,
                          const float* __restrict__ Fb, TOut* __restrict__ Ya, TOut* __restrict__ Yb,
                          int64_t A, int La, int M, int Lb, int B, int Ka, int Kb, int S) {
  extern __shared__ __align__(16) unsigned char slab_smem[];
  const int Lbp = (Lb + 7) & ~7;
  float* FsA = reinterpret_cast<float*>(slab_smem);                          // [La][KBA]
  float* FsB = FsA + align16((size_t)La * KBA * 4) / 4;                      // [Lb][KBB] or [KBB][Lbp]
  TIn* Xs = reinterpret_cast<TIn*>(slab_smem + align16((size_t)La * KBA * 4) +
                                   align16((size_t)KBB * Lbp * 4));
  const int tid = threadIdx.x;
  const int QA = M * Lb * B;           // positions of the first child per block
  const int SAB = La * QA;             // elements per block X[alpha]
  const int64_t a0 = (int64_t)blockIdx.x * S;
  // the tile's blocks of X, Ya and Yb (block-uniform check: a failed one
  // skips the block's accesses and keeps its barrier)
  const int64_t a1 = a0 + min((int64_t)S, A - a0);
  const int64_t ya_per = (int64_t)Ka * M * Lb * B, yb_per = (int64_t)La * M * Kb * B;
  const int ns = TK_DBG_IN(a0 * La * M * Lb * B, a1 * La * M * Lb * B - 1, A * La * M * Lb * B) &&
                         TK_DBG_IN(a0 * ya_per, a1 * ya_per - 1, A * ya_per) &&
                         TK_DBG_IN(a0 * yb_per, a1 * yb_per - 1, A * yb_per)
                     ? (int)(a1 - a0)
                     : 0;
  (void)ya_per;
  (void)yb_per;
  constexpr int per = 16 / (int)sizeof(TIn);
  const bool vecB = B == 1 && (Lb * (int)sizeof(TIn)) % 16 == 0;
  for (int i = tid; i < La * KBA; i += kSlabThreads) {
    const int l = i / KBA, k = i - (i / KBA) * KBA;
    FsA[i] = k < Ka ? Fa[(int64_t)l * Ka + k] : 0.f;
  }
  if (vecB) {
    for (int i = tid; i < KBB * Lbp; i += kSlabThreads) {
      const int k = i / Lbp, l = i - (i / Lbp) * Lbp;
      FsB[i] = (k < Kb && l < Lb) ? Fb[(int64_t)l * Kb + k] : 0.f;
    }
  } else {
    for (int i = tid; i < Lb * KBB; i += kSlabThreads) {
      const int l = i / KBB, k = i - (i / KBB) * KBB;
      FsB[i] = k < Kb ? Fb[(int64_t)l * Kb + k] : 0.f;
    }
  }
  stage_issue(Xs, X + a0 * SAB, ns * SAB);
  cp_wait_all();
  __syncthreads();
  // first child: positions (s, q), contraction over la at stride QA (a tile
  // holds too few positions for several per thread: measured slower)
  {
    const SmallDiv dq(QA);
    TOut* ya = Ya + a0 * (int64_t)Ka * QA;
    for (int p = tid; p < ns * QA; p += kSlabThreads) {
      const int sl = dq.div(p), q = p - sl * QA;
      const TIn* xp = Xs + sl * SAB + q;
      float acc[KBA];
#pragma unroll
      for (int k = 0; k < KBA; ++k) acc[k] = 0.f;
      for (int l = 0; l < La; ++l) {
        const float x = Elem<TIn>::cvt(xp[l * QA]);
#pragma unroll
        for (int k = 0; k < KBA; ++k) acc[k] = fmaf(FsA[l * KBA + k], x, acc[k]);
      }
      TOut* y = ya + (int64_t)sl * Ka * QA + q;
#pragma unroll
      for (int k = 0; k < KBA; ++k)
        if (k < Ka) store_out<TOut>(y + k * QA, acc[k]);
    }
  }
  // second child: rows r = (s, la, mu) of Lb B elements, positions (r, beta)
  {
    const int nr = ns * La * M;
    TOut* yb = Yb + a0 * (int64_t)La * M * Kb * B;
    if (vecB) {
      for (int r = tid; r < nr; r += kSlabThreads) {
        const TIn* xr = Xs + r * Lb;
        float acc[KBB];
#pragma unroll
        for (int k = 0; k < KBB; ++k) acc[k] = 0.f;
        for (int l0 = 0; l0 < Lb; l0 += per) {
          const uint4 v = *reinterpret_cast<const uint4*>(xr + l0);
          float x[per];
          if constexpr (sizeof(TIn) == 4) {
            x[0] = __uint_as_float(v.x);
            x[1] = __uint_as_float(v.y);
            x[2] = __uint_as_float(v.z);
            x[3] = __uint_as_float(v.w);
          } else {
            const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              x[2 * q] = __uint_as_float(w[q] << 16);
              x[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
            }
          }
#pragma unroll
          for (int k = 0; k < KBB; ++k) {
#pragma unroll
            for (int q = 0; q < per; q += 4) {
              const float4 f = *reinterpret_cast<const float4*>(FsB + k * Lbp + l0 + q);
              acc[k] = fmaf(f.x, x[q], acc[k]);
              acc[k] = fmaf(f.y, x[q + 1], acc[k]);
              acc[k] = fmaf(f.z, x[q + 2], acc[k]);
              acc[k] = fmaf(f.w, x[q + 3], acc[k]);
            }
          }
        }
        TOut* y = yb + (int64_t)r * Kb;
#pragma unroll
        for (int k = 0; k < KBB; ++k)
          if (k < Kb) store_out<TOut>(y + k, acc[k]);
      }
    } else {
      const SmallDiv db(B);
      for (int p = tid; p < nr * B; p += kSlabThreads) {
        const int r = db.div(p), be = p - r * B;
        const TIn* xp = Xs + r * Lb * B + be;
        float acc[KBB];
#pragma unroll
        for (int k = 0; k < KBB; ++k) acc[k] = 0.f;
        for (int l = 0; l < Lb; ++l) {
          const float x = Elem<TIn>::cvt(xp[l * B]);
#pragma unroll
          for (int k = 0; k < KBB; ++k) acc[k] = fmaf(FsB[l * KBB + k], x, acc[k]);
        }
        TOut* y = yb + (int64_t)r * Kb * B + be;
#pragma unroll
        for (int k = 0; k < KBB; ++k)
          if (k < Kb) store_out<TOut>(y + k * B, acc[k]);
      }
    }
  }
}

}  // namespace

namespace {

inline int kb_class(int K) { return K <= 8 ? 8 : (K <= 16 ? 16 : 32); }

template <typename TIn, typename TOut, int KBA, int KBB>
cudaError_t launch_fused_kb(const TIn* X, int64_t A, int La, int M, int Lb, int B, const float* Fa, int Ka,
                            const float* Fb, int Kb, TOut* Ya, TOut* Yb, cudaStream_t s) {
  auto kern = ttm_fused_root_kernel<TIn, TOut, KBA, KBB>;
  const int SAB = La * M * Lb * B;
  const int S = std::max(1, kSlabSmemX / (SAB * (int)sizeof(TIn)));
  const size_t smem = align16((size_t)La * KBA * 4) + align16((size_t)KBB * ((Lb + 7) & ~7) * 4) +
                      (size_t)S * SAB * sizeof(TIn);
  const cudaError_t e = allow_smem(kern, smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)((A + S - 1) / S), kSlabThreads, smem, s>>>(X, Fa, Fb, Ya, Yb, A, La, M, Lb, B, Ka, Kb, S);
  return cudaGetLastError();
}

template <typename TIn, typename TOut, int KBA>
cudaError_t launch_fused_b(const TIn* X, int64_t A, int La, int M, int Lb, int B, const float* Fa, int Ka,
                           const float* Fb, int Kb, TOut* Ya, TOut* Yb, cudaStream_t s) {
  switch (kb_class(Kb)) {
    case 8: return launch_fused_kb<TIn, TOut, KBA, 8>(X, A, La, M, Lb, B, Fa, Ka, Fb, Kb, Ya, Yb, s);
    case 16: return launch_fused_kb<TIn, TOut, KBA, 16>(X, A, La, M, Lb, B, Fa, Ka, Fb, Kb, Ya, Yb, s);
    default: return launch_fused_kb<TIn, TOut, KBA, 32>(X, A, La, M, Lb, B, Fa, Ka, Fb, Kb, Ya, Yb, s);
  }
}

template <typename TIn, typename TOut>
cudaError_t launch_fused(const TIn* X, int64_t A, int La, int M, int Lb, int B, const float* Fa, int Ka,
                         const float* Fb, int Kb, TOut* Ya, TOut* Yb, cudaStream_t s) {
  switch (kb_class(Ka)) {
    case 8: return launch_fused_b<TIn, TOut, 8>(X, A, La, M, Lb, B, Fa, Ka, Fb, Kb, Ya, Yb, s);
    case 16: return launch_fused_b<TIn, TOut, 16>(X, A, La, M, Lb, B, Fa, Ka, Fb, Kb, Ya, Yb, s);
    default: return launch_fused_b<TIn, TOut, 32>(X, A, La, M, Lb, B, Fa, Ka, Fb, Kb, Ya, Yb, s);
  }
}

}  // namespace

bool fused_root_fits(int dtype, int N, const int64_t* L, const int64_t* K, int a, int b) {
  if (dtype != TUCKER_F32 && dtype != TUCKER_BF16) return false;
  if (a < 0 || b <= a || b >= N) return false;
  if (K[a] < 1 || K[a] > 32 || K[b] < 1 || K[b] > 32) return false;
  const int64_t es = dtype == TUCKER_F32 ? 4 : 2;
  int64_t sab = 1;
  for (int n = a; n < N; ++n) sab *= L[n];
  if (sab * es > kSlabSmemX / 4) return false;
  // the factors in shared memory (KB <= 32 each, the second one padded)
  const int64_t fa = L[a] * 32 * 4, fb = 32 * ((L[b] + 7) & ~7) * 4 + L[b] * 32 * 4;
  return fa + fb <= 48 * 1024;
}

int launch_ttm_fused_root(int dtype, const void* X, const int64_t* L, int N, int a, int b,
                          const float* Fa, int64_t Ka, const float* Fb, int64_t Kb, void* Ya, void* Yb,
                          int y_dtype, cudaStream_t s) {
  int64_t A = 1, M = 1, B = 1;
  for (int n = 0; n < a; ++n) A *= L[n];
  for (int n = a + 1; n < b; ++n) M *= L[n];
  for (int n = b + 1; n < N; ++n) B *= L[n];
  cudaError_t e;
  if (dtype == TUCKER_F32 && y_dtype == TUCKER_F32) {
    e = launch_fused<float, float>(static_cast<const float*>(X), A, (int)L[a], (int)M, (int)L[b], (int)B, Fa,
                                   (int)Ka, Fb, (int)Kb, static_cast<float*>(Ya), static_cast<float*>(Yb), s);
  } else if (dtype == TUCKER_BF16 && y_dtype == TUCKER_BF16) {
    e = launch_fused<bf16_t, bf16_t>(static_cast<const bf16_t*>(X), A, (int)L[a], (int)M, (int)L[b], (int)B,
                                     Fa, (int)Ka, Fb, (int)Kb, static_cast<bf16_t*>(Ya),
                                     static_cast<bf16_t*>(Yb), s);
  } else if (dtype == TUCKER_BF16 && y_dtype == TUCKER_F32) {
    e = launch_fused<bf16_t, float>(static_cast<const bf16_t*>(X), A, (int)L[a], (int)M, (int)L[b], (int)B,
                                    Fa, (int)Ka, Fb, (int)Kb, static_cast<float*>(Ya), static_cast<float*>(Yb),
                                    s);
  } else {
    return fail(TUCKER_ERR_UNSUPPORTED, "fused root TTM: FP32 -> FP32 or BF16 -> BF16 / FP32 only");
  }
  count_launches(1);
  if (e != cudaSuccess) return fail(TUCKER_ERR_CUDA, std::string("launch fused root TTM: ") + cudaGetErrorString(e));
  return TUCKER_OK;
}

// The tensor-core pairs are opt-in (kernel policy read when the plan is
// made): measured slower than two separate TTMs on the 64^5 (BF16) and 200^4
// (FP32 tensor-core kernels) workloads.
bool root_pair_fits(int dtype, int N, const int64_t* L, const int64_t* K, int a, int b) {
  if (fused_root_fits(dtype, N, L, K, a, b)) return true;
  if (dtype == TUCKER_BF16)
    return (kernel_policy() & 256) && ttm_tc_pair_supported(L, N, a, b, K[a], K[b], nullptr);
  if (dtype == TUCKER_F32 && (kernel_policy() & (32 | 64)))
    return ttm_x3_pair_supported(L, N, a, b, K[a], K[b], nullptr) ||
           ttm_tf32_pair_supported(L, N, a, b, K[a], K[b], nullptr);
  return false;
}

}  // namespace tk
