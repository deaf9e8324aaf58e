// eig.cu -- leading-K eigenvectors of symmetric L x L Gram matrices (the EVD
// step of Sec. 5, which the paper runs with LAPACK's dsyevx: Householder
// tridiagonalisation, bisection for the wanted eigenvalues, inverse iteration
// for their eigenvectors, back-transformation).
//
// GB300 has little FP64 throughput, so the O(L^3) part runs in FP32 and the
// answer is then refined in FP64:
//   stage 1 (one CTA per matrix, FP32, all in shared memory):
//     Householder tridiagonalisation T = Q^T W Q; multisection bisection on
//     Sturm counts for the K largest eigenvalues (one warp per eigenvalue, 32
//     points per step); inverse iteration with partial pivoting for each
//     eigenvector, re-orthogonalised inside clusters of close eigenvalues;
//     back-transformation by the stored reflectors  -> V0 (L x K), theta.
//   refinement (FP64): one or more subspace-iteration steps Y = W V,
//     Q = orth(Y diag(1/theta)) (classical Gram-Schmidt, twice), then
//     Rayleigh-Ritz: H = Q^T (W Q), Jacobi on the K x K matrix H, F = Q U.
//   The result's eigenvectors are sorted by decreasing eigenvalue and each
//   column's entry of largest magnitude (lowest row on ties) is made positive.
//
// One step multiplies the FP32 error of V0 by lambda_{K+1}/lambda_K; the FP64
// orthogonalisation and Rayleigh-Ritz keep F orthonormal to FP64 accuracy, so
// the orthonormal-factor identity used for the fit holds.
#include <algorithm>

#include "batch_fused.h"
#include "eig_bodies.cuh"
#include "eig_cluster.cuh"

namespace tk {
namespace {

template <typename TF>
__global__ void __launch_bounds__(256) eig_seed_kernel(const EigBatch B) {
  for (unsigned m = blockIdx.x; m < (unsigned)B.batch; m += gridDim.x) eig_seed_body<TF>(get_desc(B, m));
}

// The barrier at the top of each iteration keeps the previous matrix's shared
// data live until every thread is done with it.
__global__ void __launch_bounds__(kEigThreads) eig_stage1_kernel(const EigBatch B, int gate) {
  const int cnt = visit_count(B, gate);
  for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
    const EigDesc P = get_desc(B, visit_index(B, gate, i));
    __syncthreads();
    eig_stage1_body<kEigThreads>(P);
  }
}

template <typename TIn, int ROWS>
__global__ void __launch_bounds__(256) eig_wmul_kernel(const EigBatch B, int use_v0, int gate) {
  __shared__ double Ws[ROWS][kMulJ + 1];
  __shared__ double Vs[kMulJ][kMaxEigK + 1];
  const int r0 = blockIdx.x * ROWS;
  const int cnt = visit_count(B, gate);
  for (int i = blockIdx.y; i < cnt; i += gridDim.y)
    eig_wmul_block<TIn, ROWS>(get_desc(B, visit_index(B, gate, i)), use_v0, r0, Ws, Vs);
}

// Y = W In for every matrix of the batch: 32-row blocks when the batch alone
// fills the GPU, 8-row blocks (four times the blocks) otherwise.
template <typename TIn>
void launch_wmul(const EigBatch& EB, int nb, int maxL, int use_v0, int gate, cudaStream_t s) {
  const int rows = ((int64_t)nb * ((maxL + 31) / 32) >= 2 * (int64_t)sm_count()) ? 32 : 8;
  const int per_y = (maxL + rows - 1) / rows;
  const int cap = std::max(1, 8 * sm_count() / per_y);
  const dim3 g((unsigned)per_y, (unsigned)std::min(nb, cap));
  if (rows == 32)
    eig_wmul_kernel<TIn, 32><<<g, 256, 0, s>>>(EB, use_v0, gate);
  else
    eig_wmul_kernel<TIn, 8><<<g, 256, 0, s>>>(EB, use_v0, gate);
}

__global__ void __launch_bounds__(256) eig_orth_kernel(const EigBatch B, int mode, int gate,
                                                       double tol) {
  const int cnt = visit_count(B, gate);
  for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
    const unsigned m = visit_index(B, gate, i);
    const EigDesc P = get_desc(B, m);
    __syncthreads();
    eig_orth_body(P, mode, tol, m, B.cold);
  }
}

template <typename TOut>
__global__ void __launch_bounds__(256) eig_finalize_kernel(const EigBatch B, int gate) {
  const int cnt = visit_count(B, gate);
  for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
    const EigDesc P = get_desc(B, visit_index(B, gate, i));
    __syncthreads();
    eig_finalize_body<TOut>(P);
  }
}

// The warm path's orthonormalisation and Rayleigh-Ritz with a cluster of
// kEigCS CTAs per matrix (descriptors by value: a few large matrices).
__global__ void __launch_bounds__(256) eig_orth_cluster_kernel(const EigBatch B, int mode, double tol) {
  const unsigned m = blockIdx.x / kEigCS;
  eig_orth_cluster_body(get_desc(B, m), mode, tol, m, B.cold);
}

template <typename TOut>
__global__ void __launch_bounds__(256) eig_finalize_cluster_kernel(const EigBatch B) {
  eig_finalize_cluster_body<TOut>(get_desc(B, blockIdx.x / kEigCS));
}

int max_smem_optin() {
  static int v = 0;
  if (v == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (v <= 0) v = 48 * 1024;
  }
  return v;
}

}  // namespace

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

namespace {
int run_eig(const EigBatch& EB, int nb, int maxL, int maxK, int f_dtype, bool warm,
            cudaStream_t s, bool cold_only = false);
}  // namespace

int launch_eig_topk(const EigProblem* probs, int batch, int f_dtype, void* ws, size_t ws_bytes,
                    cudaStream_t s) {
  if (batch <= 0) return TUCKER_OK;
  int64_t Ls[kMaxBatch], Ks[kMaxBatch];
  for (int b0 = 0; b0 < batch; b0 += kMaxBatch) {
    const int nb = std::min(kMaxBatch, batch - b0);
    for (int b = 0; b < nb; ++b) {
      Ls[b] = probs[b0 + b].L;
      Ks[b] = probs[b0 + b].K;
      if (Ls[b] < 1 || Ls[b] > kMaxEigL || Ks[b] < 1 || Ks[b] > Ls[b] || Ks[b] > kMaxEigK)
        return fail(TUCKER_ERR_UNSUPPORTED,
                    "eig: need 1 <= K <= min(L, 64) and L <= 200 for every matrix");
    }
    const size_t need = eig_ws_bytes(nb, Ls, Ks);
    if (!ws || ws_bytes < need) return fail(TUCKER_ERR_WORKSPACE, "eig: workspace too small");
    EigBatch EB{};
    EB.batch = nb;
    EB.dev = nullptr;
    EB.cold = static_cast<int*>(ws);
    char* p = static_cast<char*>(ws) + kAlign;
    int maxL = 1, maxK = 1;
    bool warm = (kernel_policy() & 2) == 0;
    for (int b = 0; b < nb; ++b) {
      const EigProblem& pr = probs[b0 + b];
      EigDesc& d = EB.d[b];
      eig_desc_layout(d, p, pr.L, pr.K);
      p += eig_bytes_per_matrix((size_t)pr.L, (size_t)pr.K);
      d.W = pr.W;
      d.F = pr.F;
      d.F0 = pr.F0;
      maxL = std::max(maxL, pr.L);
      maxK = std::max(maxK, pr.K);
      if (!pr.F0) warm = false;
    }
    const int rc = run_eig(EB, nb, maxL, maxK, f_dtype, warm, s);
    if (rc) return rc;
  }
  return TUCKER_OK;
}

int launch_eig_batched(const EigDesc* dev, int count, int maxL, int maxK, int f_dtype,
                       char* f_base, const char* f0_base, int* cold, cudaStream_t s) {
  if (count <= 0) return TUCKER_OK;
  if (maxL > kMaxEigL || maxK > kMaxEigK || maxK > maxL)
    return fail(TUCKER_ERR_UNSUPPORTED, "eig: need K <= min(L, 64) and L <= 200");
  if (count > 65535) return fail(TUCKER_ERR_UNSUPPORTED, "eig: at most 65535 matrices per launch");
  EigBatch EB{};
  EB.batch = count;
  EB.dev = dev;
  EB.f_base = f_base;
  EB.f0_base = f0_base;
  EB.cold = cold;
  const bool warm = f0_base != nullptr && (kernel_policy() & 2) == 0;
  return run_eig(EB, count, maxL, maxK, f_dtype, warm, s);
}

int launch_eig_cold_path(const EigDesc* dev, int count, int maxL, int maxK, char* f_base,
                         const char* f0_base, int* cold, cudaStream_t s) {
  if (count <= 0) return TUCKER_OK;
  if (maxL > kMaxEigL || maxK > kMaxEigK || maxK > maxL)
    return fail(TUCKER_ERR_UNSUPPORTED, "eig: need K <= min(L, 64) and L <= 200");
  if (count > 65535) return fail(TUCKER_ERR_UNSUPPORTED, "eig: at most 65535 matrices per launch");
  EigBatch EB{};
  EB.batch = count;
  EB.dev = dev;
  EB.f_base = f_base;
  EB.f0_base = f0_base;
  EB.cold = cold;
  return run_eig(EB, count, maxL, maxK, TUCKER_F32, true, s, true);
}

namespace {

// Matrices of at least this many rows take the cluster form (an eighth of
// the rows per CTA); smaller ones stay in one CTA.
constexpr int kEigClusterMinL = 64;

// nb clusters of kEigCS CTAs (one cluster per matrix), 256 threads each.
template <typename... Args>
cudaError_t launch_cluster(void (*kern)(Args...), int nb, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nb * kEigCS));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kEigCS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// The launch sequence for nb matrices described by EB (by value or device).
int run_eig(const EigBatch& EB, int nb, int maxL, int maxK, int f_dtype, bool warm,
            cudaStream_t s, bool cold_only) {
  {
    const int smax = max_smem_optin();
    // grids of at most a few blocks per SM; kernels loop over their matrices
    const int gb = std::min(nb, 8 * sm_count());
    const size_t sm1 = stage1_smem(maxL, maxK);
    if (sm1 > (size_t)smax)
      return fail(TUCKER_ERR_UNSUPPORTED, "eig: matrix too large for shared memory");
    const size_t sm3 = ((size_t)2 * maxK * maxK + (size_t)maxL * maxK) * 8 + (size_t)2 * maxK * maxK * 4;
    if (sm3 > (size_t)smax) return fail(TUCKER_ERR_UNSUPPORTED, "eig: K too large");
    TK_CUDA_TRY(cudaFuncSetAttribute(eig_stage1_kernel,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
    if (f_dtype == TUCKER_F64)
      TK_CUDA_TRY(cudaFuncSetAttribute(eig_finalize_kernel<double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
    else
      TK_CUDA_TRY(cudaFuncSetAttribute(eig_finalize_kernel<float>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
    const size_t smo = ((size_t)maxK * (maxL + 1) + (size_t)maxK * maxK) * 8;
    if (smo > (size_t)smax) return fail(TUCKER_ERR_UNSUPPORTED, "eig: L * K too large");
    TK_CUDA_TRY(cudaFuncSetAttribute(eig_orth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smo));
    auto finalize = [&](int gate) -> int {
      if (f_dtype == TUCKER_F64)
        eig_finalize_kernel<double><<<gb, 256, sm3, s>>>(EB, gate);
      else
        eig_finalize_kernel<float><<<gb, 256, sm3, s>>>(EB, gate);
      TK_LAUNCH_CHECK("eig_finalize");
      return TUCKER_OK;
    };
    int gate = cold_only ? 1 : 0;
    if (warm && !cold_only) {
      // warm start from the input factors: two subspace-iteration steps with
      // an a-posteriori check, then Rayleigh-Ritz; the full path below runs
      // only where the check failed (need-cold flag)
      const double tol = (f_dtype == TUCKER_F64) ? 1e-18 : 1e-12;
      TK_CUDA_TRY(cudaMemsetAsync(EB.cold, 0, sizeof(int), s));
      if (f_dtype == TUCKER_F64)
        eig_seed_kernel<double><<<gb, 256, 0, s>>>(EB);
      else
        eig_seed_kernel<float><<<gb, 256, 0, s>>>(EB);
      TK_LAUNCH_CHECK("eig_seed");
      // a few large matrices (descriptors by value): a cluster of CTAs per
      // matrix for the orthonormalisations and Rayleigh-Ritz, whose FP64 row
      // sums one SM's FP64 pipe bounds
      const size_t smoc = orth_cluster_smem(maxL, maxK), smfc = finalize_cluster_smem(maxL, maxK);
      const bool clus = !EB.dev && maxL >= kEigClusterMinL && smoc <= (size_t)smax && smfc <= (size_t)smax &&
                        (kernel_policy() & 1024) == 0;
      auto orth = [&](int mode) -> int {
        if (!clus) {
          eig_orth_kernel<<<gb, 256, smo, s>>>(EB, mode, 0, tol);
          TK_LAUNCH_CHECK("eig_orth");
          return TUCKER_OK;
        }
        TK_CUDA_TRY(cudaFuncSetAttribute(eig_orth_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smoc));
        TK_CUDA_TRY(launch_cluster(eig_orth_cluster_kernel, nb, smoc, s, EB, mode, tol));
        TK_LAUNCH_CHECK("eig_orth_cluster");
        return TUCKER_OK;
      };
      launch_wmul<float>(EB, nb, maxL, 1, 0, s);
      TK_LAUNCH_CHECK("eig_wmul");
      int rc = orth(1);
      if (rc) return rc;
      launch_wmul<double>(EB, nb, maxL, 0, 0, s);
      TK_LAUNCH_CHECK("eig_wmul");
      rc = orth(2);
      if (rc) return rc;
      launch_wmul<double>(EB, nb, maxL, 0, 0, s);
      TK_LAUNCH_CHECK("eig_wmul");
      if (clus) {
        if (f_dtype == TUCKER_F64) {
          TK_CUDA_TRY(cudaFuncSetAttribute(eig_finalize_cluster_kernel<double>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smfc));
          TK_CUDA_TRY(launch_cluster(eig_finalize_cluster_kernel<double>, nb, smfc, s, EB));
        } else {
          TK_CUDA_TRY(cudaFuncSetAttribute(eig_finalize_cluster_kernel<float>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smfc));
          TK_CUDA_TRY(launch_cluster(eig_finalize_cluster_kernel<float>, nb, smfc, s, EB));
        }
        TK_LAUNCH_CHECK("eig_finalize_cluster");
      } else {
        rc = finalize(0);
        if (rc) return rc;
      }
      gate = 1;
    }
    eig_stage1_kernel<<<gb, kEigThreads, sm1, s>>>(EB, gate);
    TK_LAUNCH_CHECK("eig_stage1");
    // one subspace-iteration step: Y = W V0, Q = orth(Y / theta)
    launch_wmul<float>(EB, nb, maxL, 1, gate, s);
    TK_LAUNCH_CHECK("eig_wmul");
    eig_orth_kernel<<<gb, 256, smo, s>>>(EB, 0, gate, 0.0);
    TK_LAUNCH_CHECK("eig_orth");
    if (f_dtype == TUCKER_F64) {
      // a second step for FP64 factors
      launch_wmul<double>(EB, nb, maxL, 0, gate, s);
      TK_LAUNCH_CHECK("eig_wmul");
      eig_orth_kernel<<<gb, 256, smo, s>>>(EB, 0, gate, 0.0);
      TK_LAUNCH_CHECK("eig_orth");
    }
    // Rayleigh-Ritz on span(Q): Y = W Q, then the K x K problem
    launch_wmul<double>(EB, nb, maxL, 0, gate, s);
    TK_LAUNCH_CHECK("eig_wmul");
    int rc = finalize(gate);
    if (rc) return rc;
  }
  return TUCKER_OK;
}

}  // namespace

void eig_desc_layout(EigDesc& d, char* p, int L, int K) {
  const size_t l = (size_t)L, k = (size_t)K;
  d.L = L;
  d.K = K;
  d.F0 = nullptr;
  d.V0 = reinterpret_cast<float*>(p);
  p += align_up(l * k * 4);
  d.theta = reinterpret_cast<float*>(p);
  p += align_up(k * 4);
  d.HV = reinterpret_cast<float*>(p);
  p += align_up(l * l * 4);
  d.Q = reinterpret_cast<double*>(p);
  p += align_up(l * k * 8);
  d.Y = reinterpret_cast<double*>(p);
  p += align_up(l * k * 8);
  d.Qp = reinterpret_cast<double*>(p);
  p += align_up(l * k * 8);
  d.stat = reinterpret_cast<double*>(p);
}

}  // namespace tk
