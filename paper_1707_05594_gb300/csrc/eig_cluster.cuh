// eig_cluster.cuh -- the warm path's orthonormalisation and Rayleigh-Ritz for
// a handful of large matrices (the N matrices of one sweep of one tensor):
// a cluster of kEigCS CTAs per matrix, each owning an eighth of the rows.
// The same method as eig_orth_body / eig_finalize_body (eig_bodies.cuh), with
// the row sums that dominate the FP64 work -- Q^T Q of each Cholesky-QR
// pass, the Rayleigh quotients, V^T Q of the a-posteriori check, Q^T Y of
// Rayleigh-Ritz, F = Q U -- taken by the CTAs on their own rows (one SM's
// FP64 pipe bounds the single-CTA form) and summed across the cluster through
// distributed shared memory, always in rank order, so that every CTA holds
// the same K x K matrices and takes the same decisions (Cholesky pivots,
// Jacobi rotations, Newton-Schulz steps, signs).  Nearly dependent columns
// (a failed Cholesky pass) are gathered into rank 0, which runs the
// Gram-Schmidt fallback on all rows and hands the rows back.  Every CTA
// passes a final cluster barrier before it exits, so no CTA's shared memory
// is read after its block has finished.
#pragma once

#include <cooperative_groups.h>

#include "eig_bodies.cuh"

namespace tk {
namespace {

namespace cg = cooperative_groups;

constexpr int kEigCS = 8;  // CTAs per matrix (the portable maximum; 4 measured 8 % slower on 200^4)

__device__ __forceinline__ void own_rows(int n, int rank, int* r0, int* r1) {
  const int per = (n + kEigCS - 1) / kEigCS;
  *r0 = min(n, rank * per);
  *r1 = min(n, *r0 + per);
}

// Sums the K x K partials `part` (row-major, every entry, or the upper
// triangle a <= b when upper) of the cluster's CTAs in rank order into out.
__device__ __forceinline__ void cluster_sum_kk(cg::cluster_group& cl, double* part, double* out, int K,
                                               bool upper) {
  for (int idx = threadIdx.x; idx < K * K; idx += 256) {
    const int a = idx / K, b = idx - (idx / K) * K;
    if (upper && a > b) continue;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kEigCS; ++q) s += cl.map_shared_rank(part, q)[idx];
    out[idx] = s;
  }
}

// One Cholesky-QR pass over the cluster's rows [r0, r1) of Qs (full-height
// layout, stride ld): partial S of the own rows, cluster sum, Cholesky on the
// sum (the same in every CTA), Qs <- Qs R^-1 on the own rows.  Returns as
// chol_qr_pass (0: nearly dependent, 1: done, 2: already orthonormal).
__device__ __forceinline__ int chol_qr_pass_cluster(cg::cluster_group& cl, double* Qs, int ld, double* S,
                                                    double* Sp, int r0, int r1, int K) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ int bad, near;
  __shared__ double rdiag[kMaxEigK];
  for (int idx = tid; idx < K * K; idx += 256) {
    const int a = idx / K, b = idx - (idx / K) * K;
    if (a > b) continue;
    const double* qa = Qs + a * ld;
    const double* qb = Qs + b * ld;
    double s0 = 0.0, s1 = 0.0;
    int r = r0;
    for (; r + 1 < r1; r += 2) {
      s0 = fma(qa[r], qb[r], s0);
      s1 = fma(qa[r + 1], qb[r + 1], s1);
    }
    if (r < r1) s0 = fma(qa[r], qb[r], s0);
    Sp[idx] = s0 + s1;
  }
  cl.sync();
  cluster_sum_kk(cl, Sp, S, K, true);
  cl.sync();  // every CTA has read the partials (Sp is written again by the next pass)
  if (warp == 0) {
    double smax = 0.0, dev = 0.0;
    for (int j = 0; j < K; ++j) smax = fmax(smax, S[j * K + j]);
    for (int idx = lane; idx < K * K; idx += 32) {
      const int a = idx / K, b = idx - (idx / K) * K;
      if (a <= b) dev = fmax(dev, fabs(S[idx] - (a == b ? 1.0 : 0.0)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    int fail = 0;
    for (int j = 0; j < K && !fail; ++j) {
      double d = 0.0;
      for (int a = lane; a < j; a += 32) d = fma(S[a * K + j], S[a * K + j], d);
      d = S[j * K + j] - warp_sum(d);
      if (!(d > 1e-10 * smax)) {
        fail = 1;
        break;
      }
      const double rinv = rsqrt_nr(d), rjj = d * rinv;
      __syncwarp();
      for (int b = j + 1 + lane; b < K; b += 32) {
        double v = S[j * K + b];
        for (int a = 0; a < j; ++a) v -= S[a * K + j] * S[a * K + b];
        S[j * K + b] = v * rinv;
      }
      if (lane == 0) rdiag[j] = rinv;
      __syncwarp();
      if (lane == 0) S[j * K + j] = rjj;
      __syncwarp();
    }
    if (lane == 0) {
      bad = fail;
      near = dev * K <= 0.1;
    }
  }
  __syncthreads();
  if (bad) return 0;
  const int result = near ? 2 : 1;
  for (int r = r0 + tid; r < r1; r += 256) {
    for (int c = 0; c < K; ++c) {
      double v = Qs[c * ld + r];
      for (int a = 0; a < c; ++a) v -= S[a * K + c] * Qs[a * ld + r];
      Qs[c * ld + r] = v * rdiag[c];
    }
  }
  __syncthreads();
  return result;
}

// Gram-Schmidt fallback: rank 0 gathers every row, orthonormalises all
// columns, and every CTA takes its rows back.
__device__ __forceinline__ void cgs2_cluster(cg::cluster_group& cl, double* Qs, int ld, int n, int K,
                                             int rank, double* dots, double* red) {
  cl.sync();
  if (rank == 0) {
    for (int q = 1; q < kEigCS; ++q) {
      int q0, q1;
      own_rows(n, q, &q0, &q1);
      const double* rq = cl.map_shared_rank(Qs, q);
      for (int i = threadIdx.x; i < K * (q1 - q0); i += 256) {
        const int c = i / (q1 - q0), r = q0 + (i - (i / (q1 - q0)) * (q1 - q0));
        Qs[c * ld + r] = rq[c * ld + r];
      }
    }
    __syncthreads();
    cgs2(Qs, ld, n, K, dots, red);
  }
  cl.sync();
  if (rank != 0) {
    int r0, r1;
    own_rows(n, rank, &r0, &r1);
    const double* q0p = cl.map_shared_rank(Qs, 0);
    for (int i = threadIdx.x; i < K * (r1 - r0); i += 256) {
      const int c = i / (r1 - r0), r = r0 + (i - (i / (r1 - r0)) * (r1 - r0));
      Qs[c * ld + r] = q0p[c * ld + r];
    }
  }
  __syncthreads();
}

// The warm path's Q = orth(Y diag(1/theta)) with the a-posteriori check
// (modes 1 and 2 of eig_orth_body).  Dynamic shared memory:
// (K * (L | 1) + 3 K * K) doubles.
__device__ __forceinline__ void eig_orth_cluster_body(const EigDesc& P, int mode, double tol, unsigned m,
                                                      int* cold) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int n = P.L, K = P.K, ld = n | 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int r0, r1;
  own_rows(n, rank, &r0, &r1);
  __shared__ double dots[kMaxEigK];
  __shared__ double thp[kMaxEigK];
  __shared__ double th[kMaxEigK];
  __shared__ double thinv[kMaxEigK];
  __shared__ double red[8];
  extern __shared__ __align__(16) double csm[];
  double* Qs = csm;             // [K][ld], own rows used
  double* S = Qs + K * ld;      // [K][K]
  double* Sp = S + K * K;       // [K][K] partials (read by the cluster)
  double* Gp = Sp + K * K;      // [K][K] partials of the check
  if (mode == 1)
    for (int i = tid; i < K * (r1 - r0); i += 256) {
      const int t = i / (r1 - r0), r = r0 + (i - (i / (r1 - r0)) * (r1 - r0));
      P.Qp[(int64_t)t * n + r] = (double)P.V0[(int64_t)t * n + r];
    }
  __syncthreads();
  // Rayleigh quotients of the starting vectors: partial sums over the own rows
  for (int t = warp; t < K; t += 8) {
    const double* a = P.Qp + (int64_t)t * n;
    const double* y = P.Y + (int64_t)t * n;
    double s = 0.0;
    for (int r = r0 + lane; r < r1; r += 32) s = fma(a[r], y[r], s);
    s = warp_sum(s);
    if (lane == 0) thp[t] = s;
  }
  cl.sync();
  for (int t = tid; t < K; t += 256) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kEigCS; ++q) s += cl.map_shared_rank(thp, q)[t];
    th[t] = s;
  }
  __syncthreads();
  if (tid < K) {
    double tmx = 0.0;
    for (int t = 0; t < K; ++t) tmx = fmax(tmx, fabs(th[t]));
    const double v = th[tid];
    thinv[tid] = (fabs(v) > 1e-30 * tmx && v != 0.0) ? 1.0 / v : 0.0;
  }
  __syncthreads();
  for (int i = tid; i < K * (r1 - r0); i += 256) {
    const int t = i / (r1 - r0), r = r0 + (i - (i / (r1 - r0)) * (r1 - r0));
    const double w = thinv[t];
    Qs[t * ld + r] = (w != 0.0) ? P.Y[(int64_t)t * n + r] * w : P.Qp[(int64_t)t * n + r];
  }
  __syncthreads();
  const int first = chol_qr_pass_cluster(cl, Qs, ld, S, Sp, r0, r1, K);
  if (first == 0) {
    cgs2_cluster(cl, Qs, ld, n, K, rank, dots, red);
  } else if (first == 1) {
    if (chol_qr_pass_cluster(cl, Qs, ld, S, Sp, r0, r1, K) == 0) cgs2_cluster(cl, Qs, ld, n, K, rank, dots, red);
  }
  for (int i = tid; i < K * (r1 - r0); i += 256) {
    const int t = i / (r1 - r0), r = r0 + (i - (i / (r1 - r0)) * (r1 - r0));
    P.Q[(int64_t)t * n + r] = Qs[t * ld + r];
  }
  // the check: K - ||A^T Q||_F^2 with A the starting basis, A^T Q summed over
  // the cluster
  for (int idx = tid; idx < K * K; idx += 256) {
    const int a = idx / K, b = idx - (idx / K) * K;
    const double* pa = P.Qp + (int64_t)a * n;
    const double* qb = Qs + b * ld;
    double s0 = 0.0, s1 = 0.0;
    int r = r0;
    for (; r + 1 < r1; r += 2) {
      s0 = fma(pa[r], qb[r], s0);
      s1 = fma(pa[r + 1], qb[r + 1], s1);
    }
    if (r < r1) s0 = fma(pa[r], qb[r], s0);
    Gp[idx] = s0 + s1;
  }
  cl.sync();
  if (rank == 0) {
    double acc = 0.0;
    for (int idx = tid; idx < K * K; idx += 256) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < kEigCS; ++q) s += cl.map_shared_rank(Gp, q)[idx];
      acc = fma(s, s, acc);
    }
    const double gap = fmax(0.0, (double)K - block_sum256(acc, red));
    if (tid == 0) {
      if (mode == 1) {
        P.stat[0] = gap;
      } else {
        const double d1 = P.stat[0];
        P.stat[1] = gap;
        const bool ok = (gap == gap) && gap <= tol && (d1 <= tol || gap <= 0.25 * d1);
        need_cold(P) = ok ? 0 : 1;
        if (!ok && cold) cold[1 + atomicAdd(cold, 1)] = (int)m;
      }
    }
  }
  if (mode == 1) {
    __syncthreads();  // the check read the starting basis from Qp
    for (int i = tid; i < K * (r1 - r0); i += 256) {
      const int t = i / (r1 - r0), r = r0 + (i - (i / (r1 - r0)) * (r1 - r0));
      P.Qp[(int64_t)t * n + r] = Qs[t * ld + r];
    }
  }
  cl.sync();  // no CTA leaves while another may read its shared memory
}

// Rayleigh-Ritz of the warm path (eig_finalize_body) over a cluster: H's
// partials over the own rows summed in rank order; the K x K work repeated in
// every CTA (same inputs, same results); F's own rows; each column's sign
// from the cluster's largest-magnitude entry.  Dynamic shared memory: as
// eig_finalize_body plus K * K doubles.
template <typename TOut>
__device__ __forceinline__ void eig_finalize_cluster_body(const EigDesc& P) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int n = P.L, K = P.K;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int r0, r1;
  own_rows(n, rank, &r0, &r1);
  extern __shared__ __align__(16) double dsm[];
  double* H = dsm;          // K x K
  double* U = H + K * K;    // K x K
  double* Fs = U + K * K;   // n x K (own rows used)
  float* Hf = reinterpret_cast<float*>(Fs + n * K);  // K x K
  float* Uf = Hf + K * K;                            // K x K
  double* Hp = reinterpret_cast<double*>(Uf + K * K);  // K x K partials (2 K^2 floats above Fs: 8-byte aligned)
  __shared__ int order[kMaxEigK];
  __shared__ int flip[kMaxEigK];
  __shared__ double pbest[kMaxEigK];
  __shared__ int pidx[kMaxEigK];
  for (int idx = tid; idx < K * K; idx += 256) {
    const int a = idx / K, b = idx - (idx / K) * K;
    if (a > b) continue;
    const double* qa = P.Q + (int64_t)a * n;
    const double* yb = P.Y + (int64_t)b * n;
    double s0 = 0.0, s1 = 0.0;
    int r = r0;
    for (; r + 1 < r1; r += 2) {
      s0 = fma(qa[r], yb[r], s0);
      s1 = fma(qa[r + 1], yb[r + 1], s1);
    }
    if (r < r1) s0 = fma(qa[r], yb[r], s0);
    Hp[idx] = s0 + s1;
  }
  cl.sync();
  for (int idx = tid; idx < K * K; idx += 256) {
    const int a = idx / K, b = idx - (idx / K) * K;
    if (a > b) continue;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kEigCS; ++q) s += cl.map_shared_rank(Hp, q)[idx];
    Hf[a * K + b] = Hf[b * K + a] = (float)s;
  }
  for (int idx = tid; idx < K * K; idx += 256) Uf[idx] = (idx / K == idx % K) ? 1.f : 0.f;
  __syncthreads();
  if (warp == 0) {
    float hmax = 0.f;
    for (int i = 0; i < K; ++i) hmax = fmaxf(hmax, fabsf(Hf[i * K + i]));
    const float floor_abs = 2e-7f * hmax;
    jacobi_sweeps(Hf, Uf, K, lane, floor_abs);
    if (lane == 0) {
      for (int i = 0; i < K; ++i) order[i] = i;
      for (int i = 0; i < K; ++i) {
        int best = i;
        for (int j = i + 1; j < K; ++j)
          if (Hf[order[j] * K + order[j]] > Hf[order[best] * K + order[best]]) best = j;
        const int tmp = order[i];
        order[i] = order[best];
        order[best] = tmp;
      }
    }
  }
  __syncthreads();
  for (int idx = tid; idx < K * K; idx += 256) {
    const int a = idx / K, c = idx - (idx / K) * K;
    U[idx] = (double)Uf[a * K + order[c]];
  }
  __syncthreads();
  newton_schulz2(U, H, Fs, K);
  // F = Q U on the own rows
  for (int idx = tid; idx < (r1 - r0) * K; idx += 256) {
    const int r = r0 + idx / K, c = idx - (idx / K) * K;
    double s = 0.0;
    for (int a = 0; a < K; ++a) s += P.Q[(int64_t)a * n + r] * U[a * K + c];
    Fs[r * K + c] = s;
  }
  __syncthreads();
  // each column's entry of largest magnitude (lowest row on ties) over the
  // own rows, then over the cluster in rank order (rows increase with rank)
  for (int c = warp; c < K; c += 8) {
    double best = -1.0;
    int bi = n;
    for (int r = r0 + lane; r < r1; r += 32) {
      const double v = fabs(Fs[r * K + c]);
      if (v > best) {
        best = v;
        bi = r;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (lane == 0) {
      pbest[c] = best;
      pidx[c] = bi;
    }
  }
  cl.sync();
  for (int c = tid; c < K; c += 256) {
    double best = -1.0;
    int bi = n, owner = 0;
    for (int q = 0; q < kEigCS; ++q) {
      const double ob = cl.map_shared_rank(pbest, q)[c];
      const int oi = cl.map_shared_rank(pidx, q)[c];
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
        owner = q;
      }
    }
    // the sign of that entry, read from its owner's rows
    flip[c] = (bi < n && cl.map_shared_rank(Fs, owner)[bi * K + c] < 0.0) ? 1 : 0;
  }
  __syncthreads();
  TOut* F = static_cast<TOut*>(P.F);
  for (int idx = tid; idx < (r1 - r0) * K; idx += 256) {
    const int r = r0 + idx / K, c = idx - (idx / K) * K;
    const double v = flip[c] ? -Fs[r * K + c] : Fs[r * K + c];
    F[(int64_t)r * K + c] = (TOut)v;
  }
  cl.sync();  // no CTA leaves while another may read its shared memory
}

inline size_t orth_cluster_smem(int L, int K) {
  return ((size_t)K * (size_t)(L | 1) + 3 * (size_t)K * K) * 8;
}
inline size_t finalize_cluster_smem(int L, int K) {
  return ((size_t)2 * K * K + (size_t)L * K) * 8 + (size_t)2 * K * K * 4 + (size_t)K * K * 8;
}

}  // namespace
}  // namespace tk
