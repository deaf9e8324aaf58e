// eig_bodies.cuh -- device code of the eigensolver (eig.cu): descriptors,
// reductions, and the per-matrix bodies of its stages, which the batched
// eigensolver kernels and the fused batched sweep (batch_fused.cu) run:
//   eig_seed_body            starting subspace from the input factor
//   eig_stage1_body<NT>      FP32 Householder tridiagonalisation, bisection,
//                            inverse iteration, back-transformation (NT threads)
//   eig_wmul_block           32 (or 8) rows of Y = W In in FP64 (256 threads)
//   eig_orth_body            orthonormalisation (CholeskyQR2 / Gram-Schmidt)
//                            and the warm start's a-posteriori check
//   eig_finalize_body        Rayleigh-Ritz and the output factor
// The method and its precision split are described at the top of eig.cu.
#pragma once

#include <algorithm>

#include "common.cuh"

namespace tk {
namespace {

constexpr int kEigThreads = 512;
constexpr int kEigWarps = kEigThreads / 32;
// inverse iteration: per-lane arrays (LU of T - lambda I and the iterate),
// interleaved [i][lane] with a padded stride so lanes and rows are both
// conflict-free
constexpr int kInvArrays = 6;
constexpr int kInvLD = 33;
constexpr int kMaxEigL = 200;
constexpr int kMaxEigK = 64;
constexpr int kMaxBatch = TUCKER_MAX_MODES;

// Descriptors come either by value (up to kMaxBatch matrices) or, for large
// batches, from a device array (dev != NULL).
// In a device array F and F0 are byte offsets from f_base / f0_base (so the
// table does not change when the caller swaps factor buffers).
struct EigBatch {
  EigDesc d[kMaxBatch];
  int batch;
  const EigDesc* dev;
  char* f_base;
  const char* f0_base;
  int* cold;  // list of matrices sent to the full path: cold[0] = count, cold[1 ..]
};
__device__ __forceinline__ EigDesc get_desc(const EigBatch& B, unsigned i) {
  if (!B.dev) {
    // constant offsets into the parameter block (a run-time index would make
    // every thread copy the whole block to local memory first)
    switch (i) {
      case 0: return B.d[0];
      case 1: return B.d[1];
      case 2: return B.d[2];
      case 3: return B.d[3];
      case 4: return B.d[4];
      case 5: return B.d[5];
      case 6: return B.d[6];
      default: return B.d[7];
    }
  }
  EigDesc d = B.dev[i];
  d.F = B.f_base + reinterpret_cast<size_t>(d.F);
  d.F0 = B.f0_base ? static_cast<const void*>(B.f0_base + reinterpret_cast<size_t>(d.F0)) : nullptr;
  return d;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum over NT threads; every thread receives the result.  `red`
// holds >= NT / 32 floats.
template <int NT>
__device__ float block_sum(float v, float* red) {
  __syncthreads();  // red may still be read by a previous call
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < NT / 32; ++i) s += red[i];
  return s;
}

// Number of eigenvalues of the symmetric tridiagonal (d, e) below x.
__device__ int sturm_count(const float* d, const float* e2, int n, float x, float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int c = q < 0.f;
  for (int i = 1; i < n; ++i) {
    q = (d[i] - x) - e2[i - 1] / q;
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

__device__ __forceinline__ float start_value(int i, int t) {
  unsigned h = (unsigned)(i * 2654435761u) ^ (unsigned)((t + 1) * 40503u);
  h ^= h >> 13;
  h *= 0x5bd1e995u;
  h ^= h >> 15;
  return 1.0f + 0.5f * ((float)(h & 0xFFFFu) / 65536.0f - 0.5f);
}

// Warm start bookkeeping: stat[0] / stat[1] hold the subspace movement of the
// two warm subspace-iteration steps, the int at stat + 4 words says whether the
// full (cold) path must run, and such matrices are also appended to the list
// B.cold.  Kernels of the full path launched with gate = 1 visit only the
// listed matrices (an empty list costs each block one load); with gate = 0
// they visit all of them.  Blocks take their matrices in a grid-stride loop.
__device__ __forceinline__ int& need_cold(const EigDesc& P) {
  return reinterpret_cast<int*>(P.stat)[4];
}
__device__ __forceinline__ int visit_count(const EigBatch& B, int gate) {
  return gate ? *reinterpret_cast<volatile const int*>(B.cold) : B.batch;
}
__device__ __forceinline__ unsigned visit_index(const EigBatch& B, int gate, int i) {
  return gate ? (unsigned)B.cold[1 + i] : (unsigned)i;
}

// Starting subspace from the input factor: V0[c][r] = F0[r][c].
template <typename TF>
__device__ __forceinline__ void eig_seed_body(const EigDesc& P) {
  const TF* F0 = static_cast<const TF*>(P.F0);
  for (int idx = threadIdx.x; idx < P.L * P.K; idx += 256) {
    const int r = idx / P.K, c = idx - (idx / P.K) * P.K;
    P.V0[c * P.L + r] = (float)F0[idx];
  }
}

// ---------------------------------------------------------------------------
// Stage 1: FP32 tridiagonalisation, bisection, inverse iteration, back-transform.
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ void eig_stage1_body(const EigDesc& P) {
  const int n = P.L, K = P.K, LD = n | 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  extern __shared__ __align__(16) float sm[];
  // region 0 holds A during the tridiagonalisation and the back-transform,
  // and the per-lane inverse-iteration arrays in between (the reflectors are
  // parked in global scratch meanwhile)
  const int reg0 = max(n * LD, kInvArrays * n * kInvLD);
  float* A = sm;            // n x LD
  float* Zs = sm + reg0;    // K x n
  float* dv = Zs + K * n;   // n
  float* ev = dv + n;       // n
  float* e2 = ev + n;       // n
  float* tau = e2 + n;      // n
  float* vv = tau + n;      // n
  float* pp = vv + n;       // n
  float* lam = pp + n;      // K
  float* sj = lam + K;      // K
  float* red = sj + K;      // 48
  int* cstart = reinterpret_cast<int*>(red + 48);  // K + 1
  int* clus_of = cstart + K + 1;                   // K: start index of t's cluster

  for (int i = tid; i < n * n; i += NT) {
    const int r = i / n, c = i - (i / n) * n;
    A[r * LD + c] = (float)P.W[i];
  }
  __syncthreads();

  // ---- Householder tridiagonalisation (lower), reflectors kept in A ----
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    float part = 0.f;
    for (int i = 1 + tid; i < m; i += NT) {
      const float x = A[(k + 1 + i) * LD + k];
      part += x * x;
    }
    const float xn2 = block_sum<NT>(part, red);
    if (tid == 0) {
      const float alpha = A[(k + 1) * LD + k];
      dv[k] = A[k * LD + k];
      if (xn2 == 0.f) {
        tau[k] = 0.f;
        ev[k] = alpha;
        red[32] = 0.f;
      } else {
        const float beta = -copysignf(sqrtf(alpha * alpha + xn2), alpha);
        tau[k] = (beta - alpha) / beta;
        red[32] = 1.0f / (alpha - beta);
        ev[k] = beta;
      }
    }
    __syncthreads();
    const float tk = tau[k];
    if (tk == 0.f) continue;  // uniform over the block
    const float scale = red[32];
    for (int i = tid; i < m; i += NT) {
      float v = 1.f;
      if (i > 0) {
        v = A[(k + 1 + i) * LD + k] * scale;
        A[(k + 1 + i) * LD + k] = v;
      }
      vv[i] = v;
    }
    __syncthreads();
    // p = tau * A22 v with tpr threads per row; only the lower triangle of
    // A22 is kept, so entries above the diagonal are read from their mirror
    int tpr = 1;
    while (tpr < 32 && m * tpr * 2 <= NT) tpr *= 2;
    {
      const int row = tid / tpr, sub = tid - (tid / tpr) * tpr;
      float s = 0.f;
      if (row < m) {
        const float* arow = A + (k + 1 + row) * LD + (k + 1);
        const float* acol = A + (k + 1) * LD + (k + 1 + row);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int j = sub;
        for (; j + 3 * tpr <= row; j += 4 * tpr) {
          s0 += arow[j] * vv[j];
          s1 += arow[j + tpr] * vv[j + tpr];
          s2 += arow[j + 2 * tpr] * vv[j + 2 * tpr];
          s3 += arow[j + 3 * tpr] * vv[j + 3 * tpr];
        }
        for (; j <= row; j += tpr) s0 += arow[j] * vv[j];
        for (; j + 3 * tpr < m; j += 4 * tpr) {
          s0 += acol[j * LD] * vv[j];
          s1 += acol[(j + tpr) * LD] * vv[j + tpr];
          s2 += acol[(j + 2 * tpr) * LD] * vv[j + 2 * tpr];
          s3 += acol[(j + 3 * tpr) * LD] * vv[j + 3 * tpr];
        }
        for (; j < m; j += tpr) s0 += acol[j * LD] * vv[j];
        s = (s0 + s1) + (s2 + s3);
      }
      for (int o = tpr >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (row < m && sub == 0) pp[row] = tk * s;
    }
    __syncthreads();
    float part2 = 0.f;
    for (int i = tid; i < m; i += NT) part2 += pp[i] * vv[i];
    const float pv = block_sum<NT>(part2, red);
    const float Kc = 0.5f * tk * pv;
    for (int i = tid; i < m; i += NT) pp[i] -= Kc * vv[i];
    __syncthreads();
    // rank-2 update of the lower triangle: warp w takes rows w, w+16, ...
    for (int i = warp; i < m; i += (NT / 32)) {
      const float vi = vv[i], wi = pp[i];
      float* arow = A + (k + 1 + i) * LD + (k + 1);
#pragma unroll 4
      for (int j = lane; j <= i; j += 32) arow[j] -= vi * pp[j] + wi * vv[j];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      dv[n - 2] = A[(n - 2) * LD + (n - 2)];
      ev[n - 2] = A[(n - 1) * LD + (n - 2)];
    }
    dv[n - 1] = A[(n - 1) * LD + (n - 1)];
    // Gershgorin interval, scale of T, pivot floor
    float lo = 3.0e38f, hi = -3.0e38f;
    for (int i = 0; i < n; ++i) {
      const float r = (i > 0 ? fabsf(ev[i - 1]) : 0.f) + (i + 1 < n ? fabsf(ev[i]) : 0.f);
      lo = fminf(lo, dv[i] - r);
      hi = fmaxf(hi, dv[i] + r);
    }
    const float tnorm = fmaxf(fabsf(lo), fabsf(hi));
    const float pivmin = fmaxf(tnorm * 1e-30f, 1e-36f);
    red[33] = lo - 1e-6f * tnorm - pivmin;
    red[34] = hi + 1e-6f * tnorm + pivmin;
    red[35] = tnorm;
    red[36] = pivmin;
  }
  __syncthreads();
  for (int i = tid; i + 1 < n; i += NT) e2[i] = ev[i] * ev[i];
  __syncthreads();
  const float glo = red[33], ghi = red[34], tnorm = red[35], pivmin = red[36];

  // ---- multisection bisection: eigenvalue t (descending) = index n-1-t ----
  for (int t = warp; t < K; t += (NT / 32)) {
    const int j = n - 1 - t;
    float lo = glo, hi = ghi;
    for (int it = 0; it < 12; ++it) {
      const float x = lo + (hi - lo) * ((float)(lane + 1) / 33.0f);
      const int c = sturm_count(dv, e2, n, x, pivmin);
      const unsigned mask = __ballot_sync(0xffffffffu, c > j);
      const int first = mask ? (__ffs(mask) - 1) : 32;
      const float xl = __shfl_sync(0xffffffffu, x, first > 0 ? first - 1 : 0);
      const float xh = __shfl_sync(0xffffffffu, x, first < 32 ? first : 31);
      const float nlo = first > 0 ? xl : lo;
      const float nhi = first < 32 ? xh : hi;
      lo = nlo;
      hi = nhi;
      if (hi - lo <= 2.4e-7f * fmaxf(fabsf(lo), fabsf(hi)) + pivmin) break;
    }
    if (lane == 0) lam[t] = 0.5f * (lo + hi);
  }
  __syncthreads();

  // ---- clusters of close eigenvalues ----
  if (tid == 0) {
    int nc = 0, cs = 0;
    for (int t = 0; t < K; ++t) {
      if (t == 0 || lam[t - 1] - lam[t] > 1e-3f * tnorm) {
        cs = t;
        cstart[nc++] = t;
      }
      clus_of[t] = cs;
    }
    cstart[nc] = K;
  }
  // park the reflectors (rows >= column + 2 of A) in global scratch: region 0
  // holds the inverse-iteration arrays until the back-transformation
  for (int idx = tid; idx < n * n; idx += NT) {
    const int r = idx / n, c = idx - (idx / n) * n;
    if (r >= c + 2) P.HV[idx] = A[r * LD + c];
  }
  __syncthreads();

  // ---- inverse iteration: lane u of warp 0 iterates eigenvector t0 + u ----
  if (warp == 0) {
    float* dd = sm;
    float* du = dd + n * kInvLD;
    float* du2 = du + n * kInvLD;
    float* dl = du2 + n * kInvLD;
    float* pv = dl + n * kInvLD;
    float* x = pv + n * kInvLD;
    const float eps_piv = fmaxf(1.2e-7f * tnorm, 1e-30f);
    for (int t0 = 0; t0 < K; t0 += 32) {
      const int kr = min(32, K - t0);
      const bool act = lane < kr;
      const int t = t0 + lane;
      if (act) {
        const float lmb = lam[t];
        // LU with partial pivoting of T - lmb I (rows i, i+1 may swap)
        for (int i = 0; i < n; ++i) {
          const int o = i * kInvLD + lane;
          dd[o] = dv[i] - lmb;
          du[o] = (i + 1 < n) ? ev[i] : 0.f;
          dl[o] = (i + 1 < n) ? ev[i] : 0.f;
          du2[o] = 0.f;
          pv[o] = 0.f;
          x[o] = start_value(i, t);
        }
        float d_i = dd[lane];
        for (int i = 0; i + 1 < n; ++i) {
          const int o = i * kInvLD + lane, o1 = o + kInvLD;
          const float l_i = dl[o];
          if (fabsf(d_i) >= fabsf(l_i)) {
            if (d_i == 0.f) d_i = eps_piv;
            const float f = l_i / d_i;
            dd[o] = d_i;
            dl[o] = f;
            d_i = dd[o1] - f * du[o];
          } else {
            const float f = d_i / l_i;
            dd[o] = l_i;
            dl[o] = f;
            const float tmp = du[o];
            const float dnext = dd[o1];
            du[o] = dnext;
            d_i = tmp - f * dnext;
            if (i + 2 < n) {
              du2[o] = du[o1];
              du[o1] = -f * du[o1];
            }
            pv[o] = 1.f;
          }
        }
        dd[(n - 1) * kInvLD + lane] = d_i;
        for (int i = 0; i < n; ++i) {
          const int o = i * kInvLD + lane;
          if (fabsf(dd[o]) < eps_piv * 1e-3f)
            dd[o] = copysignf(eps_piv * 1e-3f, dd[o] == 0.f ? 1.f : dd[o]);
        }
      }
      __syncwarp();
      for (int iter = 0; iter < 3; ++iter) {
        if (act) {
          for (int i = 0; i + 1 < n; ++i) {
            const int o = i * kInvLD + lane, o1 = o + kInvLD;
            if (pv[o] == 0.f) {
              x[o1] -= dl[o] * x[o];
            } else {
              const float tmp = x[o];
              x[o] = x[o1];
              x[o1] = tmp - dl[o] * x[o];
            }
          }
          const int on = (n - 1) * kInvLD + lane;
          x[on] /= dd[on];
          if (n >= 2) {
            const int o = on - kInvLD;
            x[o] = (x[o] - du[o] * x[on]) / dd[o];
          }
          for (int i = n - 3; i >= 0; --i) {
            const int o = i * kInvLD + lane;
            x[o] = (x[o] - du[o] * x[o + kInvLD] - du2[o] * x[o + 2 * kInvLD]) / dd[o];
          }
        }
        __syncwarp();
        // normalise each iterate (scaled by its max first to stay in range)
        // and orthogonalise it against the earlier members of its cluster,
        // in eigenvalue order, with the whole warp
        for (int u = 0; u < kr; ++u) {
          float* xu = x + u;
          const int tu = t0 + u;
          for (int pass = 0; pass < 2; ++pass) {
            float mx = 0.f;
            for (int i = lane; i < n; i += 32) mx = fmaxf(mx, fabsf(xu[i * kInvLD]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (!(mx > 0.f) || !isfinite(mx)) {
              for (int i = lane; i < n; i += 32) xu[i * kInvLD] = start_value(i, tu + 7 * iter + 1);
              mx = 2.f;
            }
            const float inv = 1.f / mx;
            float ss = 0.f;
            for (int i = lane; i < n; i += 32) {
              const float y = xu[i * kInvLD] * inv;
              xu[i * kInvLD] = y;
              ss += y * y;
            }
            ss = warp_sum(ss);
            const float rn = rsqrtf(ss);
            for (int i = lane; i < n; i += 32) xu[i * kInvLD] *= rn;
            __syncwarp();
            if (pass == 1) break;
            for (int q = clus_of[tu]; q < tu; ++q) {
              const float* zq = (q >= t0) ? x + (q - t0) : Zs + q * n;
              const int sq = (q >= t0) ? kInvLD : 1;
              float dt = 0.f;
              for (int i = lane; i < n; i += 32) dt += zq[i * sq] * xu[i * kInvLD];
              dt = warp_sum(dt);
              for (int i = lane; i < n; i += 32) xu[i * kInvLD] -= dt * zq[i * sq];
              __syncwarp();
            }
          }
        }
        __syncwarp();
      }
      for (int u = 0; u < kr; ++u)
        for (int i = lane; i < n; i += 32) Zs[(t0 + u) * n + i] = x[i * kInvLD + u];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int idx = tid; idx < n * n; idx += NT) {
    const int r = idx / n, c = idx - (idx / n) * n;
    if (r >= c + 2) A[r * LD + c] = P.HV[idx];
  }
  __syncthreads();

  // ---- back-transformation V0 = H_0 ... H_{n-3} Z ----
  for (int k = n - 3; k >= 0; --k) {
    const float tk = tau[k];
    if (tk == 0.f) continue;
    const int m = n - k - 1;
    for (int j = warp; j < K; j += (NT / 32)) {
      const float* zj = Zs + j * n + (k + 1);
      float s = 0.f;
      for (int i = lane; i < m; i += 32) s += (i == 0 ? 1.f : A[(k + 1 + i) * LD + k]) * zj[i];
      s = warp_sum(s);
      if (lane == 0) sj[j] = tk * s;
    }
    __syncthreads();
    for (int idx = tid; idx < K * m; idx += NT) {
      const int j = idx / m, i = idx - (idx / m) * m;
      const float v = (i == 0) ? 1.f : A[(k + 1 + i) * LD + k];
      Zs[j * n + k + 1 + i] -= sj[j] * v;
    }
    __syncthreads();
  }
  for (int i = tid; i < K * n; i += NT) P.V0[i] = Zs[i];
  for (int t = tid; t < K; t += NT) P.theta[t] = lam[t];
}

// ---------------------------------------------------------------------------
// Out[c][r] = sum_j W[r][j] * In[c][j] in FP64 (In: [K][L], float or double).
// A block computes 32 rows r and every column c; W and In pass through shared
// memory in chunks of 32 j.  Thread t owns row r0 + t % 32 and the columns
// c = t / 32 + 8 q, so W is read with one row per lane and In is broadcast:
// the FP64 multiply-adds are the whole inner loop.
// ---------------------------------------------------------------------------
constexpr int kMulJ = 32;


template <typename TIn, int ROWS>
__device__ __forceinline__ void eig_wmul_block(const EigDesc& P, int use_v0, int r0,
                                               double (*Ws)[kMulJ + 1], double (*Vs)[kMaxEigK + 1]) {
  constexpr int kGroups = 256 / ROWS;                       // column groups
  constexpr int kCPer = (kMaxEigK + kGroups - 1) / kGroups;  // columns per thread
  const int tid = threadIdx.x, rl = tid % ROWS, cg = tid / ROWS;
  const int n = P.L, K = P.K;
  if (r0 >= n) return;
  const TIn* in = use_v0 ? reinterpret_cast<const TIn*>(P.V0) : reinterpret_cast<const TIn*>(P.Q);
  double acc[kCPer];
#pragma unroll
  for (int q = 0; q < kCPer; ++q) acc[q] = 0.0;
  for (int j0 = 0; j0 < n; j0 += kMulJ) {
    __syncthreads();
    for (int i = tid; i < ROWS * kMulJ; i += 256) {
      const int rr = i / kMulJ, jj = i % kMulJ;
      const int r = r0 + rr, j = j0 + jj;
      Ws[rr][jj] = (r < n && j < n) ? P.W[(int64_t)r * n + j] : 0.0;
    }
    for (int i = tid; i < K * kMulJ; i += 256) {
      const int c = i / kMulJ, jj = i % kMulJ;
      const int j = j0 + jj;
      Vs[jj][c] = j < n ? (double)in[(int64_t)c * n + j] : 0.0;
    }
    __syncthreads();
    // one branch around a whole run of multiply-adds per column: the
    // condition is the same for the lanes of a warp (all of them for
    // 32-row blocks), so absent columns issue no FP64 instructions
#pragma unroll
    for (int q = 0; q < kCPer; ++q) {
      const int c = cg + kGroups * q;
      if (c < K) {
        double a = acc[q];
#pragma unroll 8
        for (int jj = 0; jj < kMulJ; ++jj) a = fma(Ws[rl][jj], Vs[jj][c], a);
        acc[q] = a;
      }
    }
  }
  const int r = r0 + rl;
  if (r < n) {
#pragma unroll
    for (int q = 0; q < kCPer; ++q) {
      const int c = cg + kGroups * q;
      if (c < K) P.Y[(int64_t)c * n + r] = acc[q];
    }
  }
}

// 1 / sqrt(d) for d > 0: an FP32 estimate refined by two Newton steps
// r <- r (3 - d r^2) / 2 in FP64 (each step squares the relative error:
// ~2^-22 -> 2^-43 -> FP64 rounding), which on GB300 costs far less than the
// FP64 square root and divide; d outside FP32's normal range takes those.
__device__ __forceinline__ double rsqrt_nr(double d) {
  if (!(d >= 1e-37 && d <= 1e37)) return 1.0 / sqrt(d);
  double r = (double)rsqrtf((float)d);
  r = r * fma(-0.5 * d, r * r, 1.5);
  r = r * fma(-0.5 * d, r * r, 1.5);
  return r;
}

// Block sum in FP64 for 256 threads; every thread receives the result.
__device__ __forceinline__ double block_sum256(double v, double* red) {
  __syncthreads();
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < 8; ++w) t += red[w];
  return t;
}


// The dot products below give each thread whole (a, b) entries: on GB300 the
// FP64 pipe is narrow, and a warp-wide reduction spends five FP64 additions
// per entry, more than the products themselves for columns of a few dozen.
// Columns in shared memory have an odd stride ld so that the threads of a
// warp, which read column b = b0 .. b0 + 15 at one row, hit distinct banks.

// One Cholesky-QR pass on the K columns of length n held in shared memory
// (Qs[c * ld + r]): S = Qs^T Qs, S = R^T R, Qs <- Qs R^-1.  Returns 0 (and
// leaves Qs unchanged) when a pivot is not clearly positive, i.e. when the
// columns are too far from independent for this pass to be accurate; 2 when
// the columns were already close to orthonormal (K max|S - I| <= 0.1, so the
// condition number is below 1.3 and this one pass leaves them orthonormal to
// rounding), else 1.
__device__ __forceinline__ int chol_qr_pass(double* Qs, int ld, double* S, int n, int K) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ int bad, near;
  __shared__ double rdiag[kMaxEigK];  // 1 / R[j][j]
  // S (upper triangle), a thread per entry
  for (int idx = tid; idx < K * K; idx += 256) {
    const int a = idx / K, b = idx - (idx / K) * K;
    if (a > b) continue;
    const double* qa = Qs + a * ld;
    const double* qb = Qs + b * ld;
    double s0 = 0.0, s1 = 0.0;
    int r = 0;
    for (; r + 1 < n; r += 2) {
      s0 = fma(qa[r], qb[r], s0);
      s1 = fma(qa[r + 1], qb[r + 1], s1);
    }
    if (r < n) s0 = fma(qa[r], qb[r], s0);
    S[a * K + b] = s0 + s1;
  }
  __syncthreads();
  // Cholesky S = R^T R in place (upper triangle), by warp 0: row j of R is
  // finished before row j + 1 starts; lanes take the entries of a row
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
      // a pivot below 1e-10 of the largest diagonal entry means the columns
      // are close to dependent (cond > ~1e5): leave it to Gram-Schmidt
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
  // Qs <- Qs R^-1, row by row (forward substitution along c)
  for (int r = tid; r < n; r += 256) {
    for (int c = 0; c < K; ++c) {
      double v = Qs[c * ld + r];
      for (int a = 0; a < c; ++a) v -= S[a * K + c] * Qs[a * ld + r];
      Qs[c * ld + r] = v * rdiag[c];
    }
  }
  __syncthreads();
  return result;
}

// Classical Gram-Schmidt applied twice, column by column (the fallback of
// chol_qr_pass for nearly dependent columns).
__device__ __forceinline__ void cgs2(double* Q, int ld, int n, int K, double* dots, double* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = 0; j < K; ++j) {
    double* qj = Q + (int64_t)j * ld;
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = warp; i < j; i += 8) {
        const double* qi = Q + (int64_t)i * ld;
        double s = 0.0;
        for (int r = lane; r < n; r += 32) s += qi[r] * qj[r];
        s = warp_sum(s);
        if (lane == 0) dots[i] = s;
      }
      __syncthreads();
      for (int r = tid; r < n; r += 256) {
        double v = qj[r];
        for (int i = 0; i < j; ++i) v -= dots[i] * Q[(int64_t)i * ld + r];
        qj[r] = v;
      }
      __syncthreads();
    }
    double s = 0.0;
    for (int r = tid; r < n; r += 256) s += qj[r] * qj[r];
    const double tot = block_sum256(s, red);
    const double inv = tot > 0.0 ? 1.0 / sqrt(tot) : 0.0;
    for (int r = tid; r < n; r += 256) qj[r] *= inv;
    __syncthreads();
  }
}

// K - ||A^T Q||_F^2 for the K x n basis A ([K][n] in global memory) and the
// columns Q in shared memory (stride ld), a thread per entry of A^T Q.
__device__ __forceinline__ double subspace_gap(const double* A, const double* Qs, int ld, int n,
                                               int K, double* red) {
  double acc = 0.0;
  for (int idx = threadIdx.x; idx < K * K; idx += 256) {
    const int a = idx / K, b = idx - (idx / K) * K;
    const double* pa = A + (int64_t)a * n;
    const double* qb = Qs + b * ld;
    double s0 = 0.0, s1 = 0.0;
    int r = 0;
    for (; r + 1 < n; r += 2) {
      s0 = fma(pa[r], qb[r], s0);
      s1 = fma(pa[r + 1], qb[r + 1], s1);
    }
    if (r < n) s0 = fma(pa[r], qb[r], s0);
    const double v = s0 + s1;
    acc = fma(v, v, acc);
  }
  return fmax(0.0, (double)K - block_sum256(acc, red));
}

// ---------------------------------------------------------------------------
// Q = orth(Y diag(1/theta)) in FP64, in shared memory: two Cholesky-QR passes
// (CholeskyQR2; one where the scaled columns are already close to
// orthonormal), or Gram-Schmidt applied twice where the first Cholesky pass
// finds them nearly dependent.  Writes Q.
//   mode 0 (full path): theta from stage 1, a negligible theta falls back to V0;
//   mode 1 (warm step 1): theta_j = V0_j . Y_j (Rayleigh quotient of the
//     starting vector); records delta1 = K - ||V0^T Q||_F^2 and keeps Q in Qp;
//   mode 2 (warm step 2): theta_j = Qp_j . Y_j; records delta2 = K -
//     ||Qp^T Q||_F^2 and accepts the warm result when delta2 <= tol and the
//     iteration contracts (delta2 <= delta1 / 4, or delta1 <= tol too);
//     otherwise it raises the need-cold flag and lists the matrix for the
//     full path.
// Dynamic shared memory: (K * (L + 1) + K * K) doubles.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void eig_orth_body(const EigDesc& P, int mode, double tol, unsigned m,
                                              int* cold) {
  const int n = P.L, K = P.K, ld = n | 1;
  const int tid = threadIdx.x;
  __shared__ double dots[kMaxEigK];
  __shared__ double th[kMaxEigK];
  __shared__ double thinv[kMaxEigK];
  __shared__ double red[8];
  extern __shared__ __align__(16) double osm[];
  double* Qs = osm;             // [K][ld]
  double* S = osm + K * ld;     // [K][K]
  // warm step 1: the starting basis V0 converted to FP64 once, into Qp (Qp
  // receives Q at the end of this step)
  if (mode == 1)
    for (int i = tid; i < K * n; i += 256) P.Qp[i] = (double)P.V0[i];
  __syncthreads();
  if (mode == 0) {
    float tmax = 0.f;
    for (int t = 0; t < K; ++t) tmax = fmaxf(tmax, fabsf(P.theta[t]));
    for (int t = tid; t < K; t += 256) {
      const float v = P.theta[t];
      th[t] = (fabsf(v) > 1e-20f * tmax && v != 0.f) ? (double)v : 0.0;
    }
  } else {
    // a warp per column, its lanes along the rows: the K dot products of
    // length n as short chains (a thread per column would run n dependent
    // FP64 multiply-adds)
    const int lane = tid & 31, warp = tid >> 5;
    for (int t = warp; t < K; t += 8) {
      const double* a = P.Qp + (int64_t)t * n;
      const double* y = P.Y + (int64_t)t * n;
      double s = 0.0;
      for (int r = lane; r < n; r += 32) s = fma(a[r], y[r], s);
      s = warp_sum(s);
      if (lane == 0) th[t] = s;
    }
  }
  __syncthreads();
  // 1 / theta once per column (element-wise FP64 divisions are costly on the
  // FP64 pipe); a negligible theta keeps the starting vector instead
  if (tid < K) {
    double tmx = 0.0;
    for (int t = 0; t < K; ++t) tmx = fmax(tmx, fabs(th[t]));
    const double v = th[tid];
    thinv[tid] = (fabs(v) > 1e-30 * tmx && v != 0.0) ? 1.0 / v : 0.0;
  }
  __syncthreads();
  for (int i = tid; i < K * n; i += 256) {
    const int t = i / n, r = i - (i / n) * n;
    const double w = thinv[t];
    Qs[t * ld + r] = (w != 0.0) ? P.Y[i] * w : ((mode == 0) ? (double)P.V0[i] : P.Qp[i]);
  }
  __syncthreads();
  // CholeskyQR2: the second pass only where the first started from columns
  // not already close to orthonormal
  const int first = chol_qr_pass(Qs, ld, S, n, K);
  if (first == 0) {
    cgs2(Qs, ld, n, K, dots, red);
  } else if (first == 1) {
    if (chol_qr_pass(Qs, ld, S, n, K) == 0) cgs2(Qs, ld, n, K, dots, red);
  }
  for (int i = tid; i < K * n; i += 256) {
    const int t = i / n, r = i - (i / n) * n;
    P.Q[i] = Qs[t * ld + r];
  }
  if (mode == 1) {
    const double gap = subspace_gap(P.Qp, Qs, ld, n, K, red);
    __syncthreads();
    for (int i = tid; i < K * n; i += 256) {
      const int t = i / n, r = i - (i / n) * n;
      P.Qp[i] = Qs[t * ld + r];
    }
    if (tid == 0) P.stat[0] = gap;
  } else if (mode == 2) {
    const double d2 = subspace_gap(P.Qp, Qs, ld, n, K, red);
    if (tid == 0) {
      const double d1 = P.stat[0];
      P.stat[1] = d2;
      const bool ok = (d2 == d2) && d2 <= tol && (d1 <= tol || d2 <= 0.25 * d1);
      need_cold(P) = ok ? 0 : 1;
      if (!ok && cold) cold[1 + atomicAdd(cold, 1)] = (int)m;
    }
  }
}

// Cyclic Jacobi sweeps on the K x K FP32 matrix Hf (rotations accumulated
// in Uf), by one warp: at most 30 sweeps; pairs below the rotation
// threshold (floor_abs, or 1e-9 of the geometric mean of their diagonal
// entries) are zeroed without rotating.
__device__ __forceinline__ void jacobi_sweeps(float* Hf, float* Uf, int K, int lane, float floor_abs) {
  for (int sweep = 0; sweep < 30; ++sweep) {
    // a sweep in which no pair reaches the rotation threshold only zeroes
    // the off-diagonal entries: test every pair at once first and do that
    // directly (the common case once Q approximates the eigenvectors)
    bool big = false;
    for (int idx = lane; idx < K * K; idx += 32) {
      const int p = idx / K, q = idx - (idx / K) * K;
      if (p >= q) continue;
      const float apq = Hf[idx];
      const float app = Hf[p * K + p], aqq = Hf[q * K + q];
      big = big || (apq != 0.f && !(fabsf(apq) <= floor_abs ||
                                    fabsf(apq) <= 1e-9f * sqrtf(fabsf(app) * fabsf(aqq))));
    }
    if (!__any_sync(0xffffffffu, big)) {
      __syncwarp();
      for (int idx = lane; idx < K * K; idx += 32)
        if (idx / K != idx - (idx / K) * K) Hf[idx] = 0.f;
      __syncwarp();
      break;
    }
    int rotated = 0;
    for (int p = 0; p < K - 1; ++p) {
      for (int q = p + 1; q < K; ++q) {
        const float apq = Hf[p * K + q];
        const float app = Hf[p * K + p], aqq = Hf[q * K + q];
        if (apq == 0.f) continue;
        if (fabsf(apq) <= floor_abs || fabsf(apq) <= 1e-9f * sqrtf(fabsf(app) * fabsf(aqq))) {
          __syncwarp();
          if (lane == 0) Hf[p * K + q] = Hf[q * K + p] = 0.f;
          __syncwarp();
          continue;
        }
        rotated = 1;
        const float th = (aqq - app) / (2.f * apq);
        const float t = (th >= 0.f) ? 1.f / (th + sqrtf(1.f + th * th))
                                    : -1.f / (-th + sqrtf(1.f + th * th));
        const float c = rsqrtf(1.f + t * t), s = t * c;
        __syncwarp();
        for (int k = lane; k < K; k += 32) {
          const float hkp = Hf[k * K + p], hkq = Hf[k * K + q];
          Hf[k * K + p] = c * hkp - s * hkq;
          Hf[k * K + q] = s * hkp + c * hkq;
        }
        __syncwarp();
        for (int k = lane; k < K; k += 32) {
          const float hpk = Hf[p * K + k], hqk = Hf[q * K + k];
          Hf[p * K + k] = c * hpk - s * hqk;
          Hf[q * K + k] = s * hpk + c * hqk;
          const float ukp = Uf[k * K + p], ukq = Uf[k * K + q];
          Uf[k * K + p] = c * ukp - s * ukq;
          Uf[k * K + q] = s * ukp + c * ukq;
        }
        __syncwarp();
        if (lane == 0) Hf[p * K + q] = Hf[q * K + p] = 0.f;
        __syncwarp();
      }
    }
    if (!rotated) break;
  }}

// Two Newton-Schulz steps U <- U (3 I - U^T U) / 2 on the K x K FP64 matrix
// U (G and T are K x K scratch), all threads of the block.
__device__ __forceinline__ void newton_schulz2(double* U, double* G, double* T, int K) {
  const int tid = threadIdx.x;
  for (int it = 0; it < 2; ++it) {
    for (int idx = tid; idx < K * K; idx += 256) {
      const int b = idx / K, c = idx - (idx / K) * K;
      if (b > c) continue;
      double g = 0.0;
      for (int a = 0; a < K; ++a) g = fma(U[a * K + b], U[a * K + c], g);
      G[b * K + c] = G[c * K + b] = g;
    }
    __syncthreads();
    for (int idx = tid; idx < K * K; idx += 256) {
      const int a = idx / K, c = idx - (idx / K) * K;
      double v = 0.0;
      for (int b = 0; b < K; ++b) v = fma(U[a * K + b], G[b * K + c], v);
      T[idx] = 1.5 * U[idx] - 0.5 * v;
    }
    __syncthreads();
    for (int idx = tid; idx < K * K; idx += 256) U[idx] = T[idx];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Rayleigh-Ritz: H = Q^T Y (Y = W Q) in FP64; the K x K eigenproblem of H by
// cyclic Jacobi in FP32 (one warp; H is nearly diagonal here, since Q already
// approximates the eigenvectors), its eigenvector matrix re-orthonormalised
// in FP64 (two Newton-Schulz steps) so that F = Q U stays orthonormal to FP64
// accuracy; columns sorted by decreasing eigenvalue, signs fixed, F written as
// L x K row-major.
// ---------------------------------------------------------------------------
template <typename TOut>
__device__ __forceinline__ void eig_finalize_body(const EigDesc& P) {
  const int n = P.L, K = P.K;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  extern __shared__ __align__(16) double dsm[];
  double* H = dsm;          // K x K
  double* U = H + K * K;    // K x K
  double* Fs = U + K * K;   // n x K
  float* Hf = reinterpret_cast<float*>(Fs + n * K);  // K x K
  float* Uf = Hf + K * K;                            // K x K
  __shared__ int order[kMaxEigK];
  __shared__ int flip[kMaxEigK];
  // H = Q^T Y, a thread per entry of the upper triangle (no warp reductions
  // on the FP64 pipe), mirrored: Q^T W Q is symmetric, and H is rounded to
  // FP32 for the Jacobi step, far above the FP64 asymmetry of Q^T Y
  for (int idx = tid; idx < K * K; idx += 256) {
    const int a = idx / K, b = idx - (idx / K) * K;
    if (a > b) continue;
    const double* qa = P.Q + (int64_t)a * n;
    const double* yb = P.Y + (int64_t)b * n;
    double s0 = 0.0, s1 = 0.0;
    int r = 0;
    for (; r + 1 < n; r += 2) {
      s0 = fma(qa[r], yb[r], s0);
      s1 = fma(qa[r + 1], yb[r + 1], s1);
    }
    if (r < n) s0 = fma(qa[r], yb[r], s0);
    Hf[a * K + b] = Hf[b * K + a] = (float)(s0 + s1);
  }
  for (int idx = tid; idx < K * K; idx += 256) Uf[idx] = (idx / K == idx % K) ? 1.f : 0.f;
  __syncthreads();
  if (warp == 0) {
    // an off-diagonal entry at the FP32 rounding level of H (2e-7 max|h_ii|)
    // counts as zero: otherwise rounding noise would keep every pair rotating
    // and the sweep loop would always run to its cap; such entries only turn
    // vectors inside the K-dimensional Ritz space
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
  // U = Uf(:, order) in FP64; the FP32 rotations leave it orthonormal to a
  // few K 2^-24, and two Newton-Schulz steps U <- U (3 I - U^T U) / 2 (the
  // error squares each step) bring it to FP64 rounding without square roots
  // or divisions (G in H, the new U through Fs)
  for (int idx = tid; idx < K * K; idx += 256) {
    const int a = idx / K, c = idx - (idx / K) * K;
    U[idx] = (double)Uf[a * K + order[c]];
  }
  __syncthreads();
  newton_schulz2(U, H, Fs, K);
  // F = Q U
  for (int idx = tid; idx < n * K; idx += 256) {
    const int r = idx / K, c = idx - (idx / K) * K;
    double s = 0.0;
    for (int a = 0; a < K; ++a) s += P.Q[(int64_t)a * n + r] * U[a * K + c];
    Fs[idx] = s;
  }
  __syncthreads();
  for (int c = warp; c < K; c += 8) {
    double best = -1.0;
    int bi = n;
    for (int r = lane; r < n; r += 32) {
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
    if (lane == 0) flip[c] = (bi < n && Fs[bi * K + c] < 0.0) ? 1 : 0;
  }
  __syncthreads();
  TOut* F = static_cast<TOut*>(P.F);
  for (int idx = tid; idx < n * K; idx += 256) {
    const int c = idx - (idx / K) * K;
    const double v = flip[c] ? -Fs[idx] : Fs[idx];
    F[idx] = (TOut)v;
  }
}

inline size_t stage1_smem(int L, int K) {
  const size_t LD = (size_t)(L | 1);
  const size_t reg0 = std::max((size_t)L * LD, (size_t)kInvArrays * L * kInvLD);
  const size_t floats = reg0 + (size_t)K * L + 6 * (size_t)L + 2 * (size_t)K + 48;
  return floats * 4 + (size_t)(2 * K + 1) * 4 + 16;
}


}  // namespace
}  // namespace tk
