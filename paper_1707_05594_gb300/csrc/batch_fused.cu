// batch_fused.cu -- one sweep of the batched form (many small tensors of
// uneven lengths and ranks) as a single persistent launch: every CTA takes
// tensors from a device queue (an atomic counter, largest tensors first) and
// runs the whole HOOI sweep of each inside the CTA (Fig. 2 per tensor):
//   the tensor's TTM tree (Sec. 3.3), parents before children;
//   its leaf Grams (Sec. 5);
//   the core of the input factors from the smallest leaf input;
//   the fit of the input factors from the direct residual (Sec. 2.2);
//   per mode, the eigensolver warm-started from the input factor: two FP64
//   subspace-iteration steps, the a-posteriori check, Rayleigh-Ritz.
// A matrix whose check fails is listed for the full eigensolver path, which
// runs after this kernel over the listed matrices only (the fit and the core
// depend on the input factors alone, so nothing here waits for it); its
// stage 1 needs more shared memory than this kernel keeps per CTA.
// The per-tile and per-matrix arithmetic is the same code as the per-site
// kernels' (batch_bodies.cuh, eig_bodies.cuh), so factors, cores and fits
// equal theirs (the fit's per-tensor sum of squares is added in another
// order).  No CTA waits for another: the queue is a fetch-and-add, and the
// last CTA to finish checks that every tensor was taken (else it records
// TUCKER_ERR_INCOMPLETE in the device error word) and resets the counters
// for the next launch.
#include <algorithm>

#include "batch_bodies.cuh"
#include "batch_fused.h"
#include "eig_bodies.cuh"

namespace tk {
namespace {

// CTAs per SM the registers allow (64 each); every phase is latency-bound,
// so more tensors in flight per SM pay: measured 17.7, 14.8 and 14.0 ms per
// sweep of the 4096-tensor batch with 2, 3 and 4
constexpr int kFusedBlocksPerSM = 4;

template <typename TIn>
__device__ __forceinline__ void wmul_all(const EigDesc& P, int use_v0, double (*Ws)[kMulJ + 1],
                                         double (*Vs)[kMaxEigK + 1]) {
  for (int r0 = 0; r0 < P.L; r0 += 32) eig_wmul_block<TIn, 32>(P, use_v0, r0, Ws, Vs);
}

template <int KMAX>
__global__ void __launch_bounds__(kBThreads, kFusedBlocksPerSM) bfused_kernel(const BFusedArgs A) {
  __shared__ __align__(16) float Fs[32 * KMAX];
  // TTM staging (Ts), reused as the Gram tiles' panels, the reconstruction's
  // factor rows and the eigensolver's W and In panels (each phase ends with a
  // barrier)
  __shared__ __align__(16) float Ts[32][kBThreads + 1];
  __shared__ double red[kBThreads / 32];
  __shared__ int s_idx;
  static_assert(sizeof(Ts) >= 2 * 32 * 33 * sizeof(float), "Gram panels");
  static_assert(sizeof(Ts) >= (size_t)kExpMaxL * KMAX * sizeof(float), "reconstruction factor rows");
  static_assert(sizeof(Ts) >= (32 * (kMulJ + 1) + kMulJ * (kMaxEigK + 1)) * sizeof(double), "W panels");
  float(*As)[33] = reinterpret_cast<float(*)[33]>(&Ts[0][0]);
  float(*Bs)[33] = As + 32;
  float(*Fe)[KMAX] = reinterpret_cast<float(*)[KMAX]>(&Ts[0][0]);
  double(*Ws)[kMulJ + 1] = reinterpret_cast<double(*)[kMulJ + 1]>(&Ts[0][0]);
  double(*Vs)[kMaxEigK + 1] = reinterpret_cast<double(*)[kMaxEigK + 1]>(Ws + 32);

  const BNode* nodes = static_cast<const BNode*>(A.nodes);
  const BNode* cores = static_cast<const BNode*>(A.cores);
  const BGram* grams = static_cast<const BGram*>(A.grams);
  const BExp* steps = static_cast<const BExp*>(A.steps);
  int mine = 0;  // tensors this CTA took (thread 0)
  for (;;) {
    __syncthreads();  // s_idx and every shared buffer of the previous tensor are free
    if (threadIdx.x == 0) s_idx = atomicAdd(&A.queue[0], 1);
    __syncthreads();
    const int idx = s_idx;
    if (idx >= A.count) break;
    ++mine;
    const int i = A.order[idx];
    const BFusedTensor W = A.work[i];
    // ---- the tensor's TTM tree, parents before children (long rows by the
    // cp.async tiles: 12.61 -> 12.42 ms per sweep of the 4096-tensor batch
    // against register-loaded tiles; two positions per thread 13.19 ms)
    for (int k = 0; k < W.nnodes; ++k) {
      const BNode nd = nodes[W.node0 + k];
      const int64_t tiles = node_tiles(nd.R, nd.C, BCfg{});
      for (int64_t t = 0; t < tiles; ++t)
        bttm_dispatch<KMAX, 1, true>(nd, t, A.T, A.F, A.inter, nullptr, Fs, Ts);
      __syncthreads();  // a child reads its parent's output
    }
    // ---- leaf Grams
    for (int g = 0; g < W.ngram; ++g) bgram_tile(grams[W.gram0 + g], A.T, A.inter, A.gram, As, Bs);
    // ---- core of the input factors
    {
      __syncthreads();
      const BNode nd = cores[i];
      const int64_t tiles = node_tiles(nd.R, nd.C, BCfg{});
      for (int64_t t = 0; t < tiles; ++t)
        bttm_dispatch<KMAX, 1, false>(nd, t, A.T, A.F, A.inter, A.G, Fs, Ts);
      __syncthreads();  // the reconstruction reads the core
    }
    // ---- fit of the input factors: the residual of the reconstruction
    {
      double res = 0.0;
      for (int s = 0; s < A.N; ++s) {
        const BExp st = steps[(size_t)s * A.count + i];
        const int64_t tiles = (st.R * st.C + kBThreads - 1) / kBThreads;
        for (int64_t t = 0; t < tiles; ++t)
          res += bexpand_tile<KMAX, 1>(st, t, A.T, A.F, A.G, A.fit_inter, Fe, red);
        __syncthreads();  // the next step reads this one's output
      }
      if (threadIdx.x == 0) A.fit[i] = 1.0 - sqrt(res) / sqrt(A.normT2[i]);
    }
    // ---- the new factors: eigensolver warm-started from the input factors
    for (int n = 0; n < A.N; ++n) {
      const unsigned m = (unsigned)(n * A.count + i);
      EigDesc P = A.eigs[m];
      P.F = A.f_base + reinterpret_cast<size_t>(P.F);
      P.F0 = A.f0_base + reinterpret_cast<size_t>(P.F0);
      __syncthreads();
      eig_seed_body<float>(P);
      __syncthreads();
      wmul_all<float>(P, 1, Ws, Vs);
      __syncthreads();
      eig_orth_body(P, 1, A.tol, m, A.cold);
      __syncthreads();
      wmul_all<double>(P, 0, Ws, Vs);
      __syncthreads();
      eig_orth_body(P, 2, A.tol, m, A.cold);
      __syncthreads();
      if (need_cold(P)) continue;  // listed for the full path (uniform over the CTA)
      wmul_all<double>(P, 0, Ws, Vs);
      __syncthreads();
      eig_finalize_body<float>(P);
    }
  }
  if (threadIdx.x == 0) {
    atomicAdd(&A.queue[2], mine);
    __threadfence();
    if (atomicAdd(&A.queue[1], 1) == (int)gridDim.x - 1) {
      // the last CTA: every other CTA has taken its last (empty) queue slot
      if (atomicAdd(&A.queue[2], 0) != A.count) atomicCAS(A.status, 0, TUCKER_ERR_INCOMPLETE);
      A.queue[0] = 0;
      A.queue[1] = 0;
      A.queue[2] = 0;
      __threadfence();
    }
  }
}

size_t batch_fused_smem_impl(int maxL, int maxK) {
  // dynamic shared memory of the orthonormalisation and of Rayleigh-Ritz
  const size_t smo = ((size_t)maxK * (maxL + 1) + (size_t)maxK * maxK) * 8;
  const size_t sm3 = ((size_t)2 * maxK * maxK + (size_t)maxL * maxK) * 8 + (size_t)2 * maxK * maxK * 4;
  return std::max(smo, sm3);
}

template <int KB>
int launch_kb(const BFusedArgs& a, size_t smem, cudaStream_t s) {
  auto kern = bfused_kernel<KB>;
  TK_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // a persistent grid: as many CTAs as fit at once (shared memory may allow
  // fewer than the registers)
  int per_sm = 0;
  TK_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBThreads, smem));
  const int64_t grid = std::min<int64_t>(a.count, (int64_t)std::max(1, per_sm) * sm_count());
  kern<<<(unsigned)grid, kBThreads, smem, s>>>(a);
  return TUCKER_OK;
}

}  // namespace

size_t batch_fused_smem(int maxL, int maxK) { return batch_fused_smem_impl(maxL, maxK); }

int launch_batch_fused(const BFusedArgs& a, int maxL, int maxK, cudaStream_t s) {
  if (a.count <= 0) return TUCKER_OK;
  const size_t smem = batch_fused_smem(maxL, maxK);
  const int rc = a.KB == 8    ? launch_kb<8>(a, smem, s)
                 : a.KB == 16 ? launch_kb<16>(a, smem, s)
                              : launch_kb<32>(a, smem, s);
  if (rc) return rc;
  TK_LAUNCH_CHECK("batch_fused");
  return TUCKER_OK;
}

}  // namespace tk
