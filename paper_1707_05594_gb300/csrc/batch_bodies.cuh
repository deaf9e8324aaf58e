// batch_bodies.cuh -- device code of the batched form shared by its per-site
// kernels (batch.cu) and the fused batched sweep (batch_fused.cu): the work
// items (tree TTM nodes, Gram tiles, reconstruction steps) and the per-tile
// bodies that run them with 256 threads.
#pragma once

#include "common.cuh"

namespace tk {
namespace {


constexpr int kBThreads = 256;

// One TTM work unit (a tree node of one tensor, or one STHOSVD step, or the
// core step).  Offsets are in elements.
struct BNode {
  int64_t in_off;    // into T (in_src 0) or the intermediate region (1)
  int64_t out_off;   // into the intermediate region (out_dst 0) or G (1)
  int64_t f_off;     // into F (L x K factor, applied transposed)
  int64_t R, C;      // view [R][L][C] of the input
  int32_t L, K;
  int64_t tile0;     // first tile of this node
  int8_t in_src, out_dst;
  int8_t staged;     // rows staged through shared memory (set with the tile map)
  int8_t pad[5];
};

// One 32 x 32 tile of a leaf Gram W = Z_(n) Z_(n)^T (lower triangle, ti >= tj).
struct BGram {
  int64_t z_off;     // into T (z_src 0) or intermediates (1)
  int64_t w_off;     // into the Gram region (doubles)
  int64_t R, C;
  int32_t L, ti, tj, z_src;
};

// Launch configuration of one batched launch site (a tree level, the core
// step, an STHOSVD step or a fit step), picked by tucker_batch_autotune.
// None of the knobs changes the order in which any output's terms are summed.
//   ppt:     positions per thread of the direct (long-row) tiles: a tile is
//            256 * ppt consecutive (r, c) positions
//   stage_c: nodes with rows shorter than stage_c (C < stage_c) take whole
//            rows per tile, staged through shared memory (0: never)
//   order:   0 = nodes in plan order (tensor by tensor), 1 = nodes with the
//            most tiles first (longest-processing-time order)
//   async:   direct tiles copy each chunk of 32 input rows into shared memory
//            with cp.async before the multiply-adds (one position per thread)
struct BCfg {
  int ppt = 1, stage_c = 32, order = 0, async = 0;
};

// Tiles of a node under a configuration.  Staged tiles take 256 / C whole
// rows; direct tiles take 256 * ppt consecutive positions and read along c.
__host__ __device__ inline bool node_staged(int64_t C, const BCfg& cfg) { return C < cfg.stage_c; }
__host__ __device__ inline int64_t node_tiles(int64_t R, int64_t C, const BCfg& cfg) {
  if (node_staged(C, cfg)) {
    const int64_t rt = kBThreads / C;
    return (R + rt - 1) / rt;
  }
  const int64_t tp = (int64_t)kBThreads * cfg.ppt;
  return (R * C + tp - 1) / tp;
}

// Out[r, k, c] = sum_l F[l, k] In[r, l, c] for one tile of one node, F in
// chunks of 32 l through shared memory.  Each thread accumulates the K
// outputs of each of its positions (KB >= K registers per position), l in
// increasing order.  Staged tiles (short rows) copy the rows of the chunk
// into shared memory transposed, Ts[l][position], with coalesced loads, and
// write their outputs back the same way; they take one position per thread.
template <int KB>
__device__ __forceinline__ void bttm_staged(const BNode& nd, int64_t t, const float* __restrict__ src,
                                            float* __restrict__ dst, const float* __restrict__ f,
                                            float* Fs /* [32][KB] */, float (*Ts)[kBThreads + 1]) {
  const int tid = threadIdx.x;
  const int C = (int)nd.C;
  const int rt = kBThreads / C;
  const int64_t r0 = t * rt;
  // the tile's rows of the node's input and output views (block-uniform
  // check: a failed one skips the tile's accesses and keeps its barriers)
  const int64_t r1 = r0 + min((int64_t)rt, nd.R - r0);
  const int nrows = TK_DBG_IN(r0 * nd.L * C, r1 * nd.L * C - 1, nd.R * nd.L * C) &&
                            TK_DBG_IN(r0 * nd.K * C, r1 * nd.K * C - 1, nd.R * nd.K * C)
                        ? (int)(r1 - r0)
                        : 0;
  const bool active = tid < nrows * C;
  float acc[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) acc[k] = 0.f;
  for (int l0 = 0; l0 < nd.L; l0 += 32) {
    const int lc = min(32, nd.L - l0);
    __syncthreads();
    for (int i = tid; i < 32 * KB; i += kBThreads) {
      const int l = i / KB, k = i - (i / KB) * KB;
      Fs[i] = (l < lc && k < nd.K) ? f[(int64_t)(l0 + l) * nd.K + k] : 0.f;
    }
    // row rr of the chunk: lc * C contiguous elements
    const int seg = lc * C;
    const SmallDiv dseg(seg), dc(C);
    for (int i = tid; i < nrows * seg; i += kBThreads) {
      const int rr = dseg.div(i), o = i - rr * seg;
      const int l = dc.div(o), cc = o - l * C;
      Ts[l][rr * C + cc] = src[((r0 + rr) * nd.L + l0) * C + o];
    }
    __syncthreads();
    if (active) {
      for (int l = 0; l < lc; ++l) {
        const float x = Ts[l][tid];
#pragma unroll
        for (int k = 0; k < KB; ++k) acc[k] = fmaf(Fs[l * KB + k], x, acc[k]);
      }
    }
  }
  // outputs through shared memory: row rr owns K * C contiguous elements
  __syncthreads();
  if (active) {
#pragma unroll
    for (int k = 0; k < KB; ++k)
      if (k < nd.K) Ts[k][tid] = acc[k];
  }
  __syncthreads();
  const int seg = nd.K * C;
  const SmallDiv dseg(seg), dc(C);
  for (int i = tid; i < nrows * seg; i += kBThreads) {
    const int rr = dseg.div(i), o = i - rr * seg;
    const int k = dc.div(o), cc = o - k * C;
    dst[(r0 + rr) * seg + o] = Ts[k][rr * C + cc];
  }
}

constexpr int kDepth = 8;  // rows of a chunk loaded ahead by the direct TTM tiles

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Direct tile, one position per thread, each chunk of up to 32 input rows
// copied into Ts[l][thread] by cp.async (32 copies per thread in flight, no
// registers held while they travel), then multiplied from shared memory.
template <int KB>
__device__ __forceinline__ void bttm_async(const BNode& nd, int64_t t, const float* __restrict__ src,
                                           float* __restrict__ dst, const float* __restrict__ f,
                                           float* Fs /* [32][KB] */, float (*Ts)[kBThreads + 1]) {
  const int tid = threadIdx.x;
  const int64_t p = t * kBThreads + tid;
  bool act = p < nd.R * nd.C;
  const int64_t r = act ? p / nd.C : 0, c = act ? p - r * nd.C : 0;
  // input fibre In[r, :, c] and outputs Out[r, :, c] of the node's views
  act = act && TK_DBG_IN((r * nd.L) * nd.C + c, (r * nd.L + nd.L - 1) * nd.C + c, nd.R * nd.L * nd.C) &&
        TK_DBG_IN((r * nd.K) * nd.C + c, (r * nd.K + nd.K - 1) * nd.C + c, nd.R * nd.K * nd.C);
  const float* in = src + (r * nd.L) * nd.C + c;
  float acc[KB];
#pragma unroll
  for (int k = 0; k < KB; ++k) acc[k] = 0.f;
  for (int l0 = 0; l0 < nd.L; l0 += 32) {
    const int lc = min(32, nd.L - l0);
    __syncthreads();  // the previous chunk's reads of Ts and Fs are done
    if (act)
      for (int l = 0; l < lc; ++l) cp_async4(&Ts[l][tid], in + (int64_t)(l0 + l) * nd.C);
    for (int i = tid; i < 32 * KB; i += kBThreads) {
      const int l = i / KB, k = i - (i / KB) * KB;
      Fs[i] = (l < lc && k < nd.K) ? f[(int64_t)(l0 + l) * nd.K + k] : 0.f;
    }
    cp_async_commit_wait_all();
    __syncthreads();
    if (act) {
      for (int l = 0; l < lc; ++l) {
        const float x = Ts[l][tid];
#pragma unroll
        for (int k = 0; k < KB; ++k) acc[k] = fmaf(Fs[l * KB + k], x, acc[k]);
      }
    }
  }
  if (!act) return;
  float* out = dst + (r * nd.K) * nd.C + c;
#pragma unroll
  for (int k = 0; k < KB; ++k)
    if (k < nd.K) out[(int64_t)k * nd.C] = acc[k];
}

template <int KB, int PPT>
__device__ __forceinline__ void bttm_direct(const BNode& nd, int64_t t, const float* __restrict__ src,
                                            float* __restrict__ dst, const float* __restrict__ f,
                                            float* Fs /* [32][KB] */) {
  const int tid = threadIdx.x;
  const int64_t M = nd.R * nd.C;
  const float* in[PPT];
  int64_t ob[PPT];
  bool act[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    const int64_t p = (t * PPT + j) * kBThreads + tid;
    act[j] = p < M;
    const int64_t r = act[j] ? p / nd.C : 0, c = act[j] ? p - r * nd.C : 0;
    // input fibre In[r, :, c] and outputs Out[r, :, c] of the node's views
    act[j] = act[j] && TK_DBG_IN((r * nd.L) * nd.C + c, (r * nd.L + nd.L - 1) * nd.C + c, nd.R * nd.L * nd.C) &&
             TK_DBG_IN((r * nd.K) * nd.C + c, (r * nd.K + nd.K - 1) * nd.C + c, nd.R * nd.K * nd.C);
    in[j] = src + (r * nd.L) * nd.C + c;
    ob[j] = (r * nd.K) * nd.C + c;
  }
  float acc[PPT][KB];
#pragma unroll
  for (int j = 0; j < PPT; ++j)
#pragma unroll
    for (int k = 0; k < KB; ++k) acc[j][k] = 0.f;
  for (int l0 = 0; l0 < nd.L; l0 += 32) {
    const int lc = min(32, nd.L - l0);
    __syncthreads();
    for (int i = tid; i < 32 * KB; i += kBThreads) {
      const int l = i / KB, k = i - (i / KB) * KB;
      Fs[i] = (l < lc && k < nd.K) ? f[(int64_t)(l0 + l) * nd.K + k] : 0.f;
    }
    __syncthreads();
    if (act[0]) {
      // kDepth rows of the chunk are loaded before their multiply-adds, so
      // that each thread has kDepth * PPT loads in flight
      for (int lb = 0; lb < lc; lb += kDepth) {
        float x[kDepth][PPT];
#pragma unroll
        for (int u = 0; u < kDepth; ++u)
#pragma unroll
          for (int j = 0; j < PPT; ++j)
            x[u][j] = (lb + u < lc && act[j]) ? __ldg(in[j] + (int64_t)(l0 + lb + u) * nd.C) : 0.f;
#pragma unroll
        for (int u = 0; u < kDepth; ++u) {
          if (lb + u < lc) {
#pragma unroll
            for (int k = 0; k < KB; ++k) {
              const float fk = Fs[(lb + u) * KB + k];
#pragma unroll
              for (int j = 0; j < PPT; ++j) acc[j][k] = fmaf(fk, x[u][j], acc[j][k]);
            }
          }
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    if (!act[j]) continue;
    float* out = dst + ob[j];
#pragma unroll
    for (int k = 0; k < KB; ++k)
      if (k < nd.K) out[(int64_t)k * nd.C] = acc[j][k];
  }
}

template <int KB, int PPT, bool ASYNC>
__device__ __forceinline__ void bttm_tile(const BNode& nd, int64_t t, const float* __restrict__ T,
                                          const float* __restrict__ F, float* __restrict__ inter,
                                          float* __restrict__ G, float* Fs,
                                          float (*Ts)[kBThreads + 1]) {
  const float* src = (nd.in_src ? inter : T) + nd.in_off;
  float* dst = (nd.out_dst ? G : inter) + nd.out_off;
  const float* f = F + nd.f_off;
  if (nd.staged) bttm_staged<KB>(nd, t, src, dst, f, Fs, Ts);
  else if (ASYNC) bttm_async<KB>(nd, t, src, dst, f, Fs, Ts);
  else bttm_direct<KB, PPT>(nd, t, src, dst, f, Fs);
}

// One block per tile; the block runs the variant whose KB is the smallest of
// 4, 8, 12, 16, 24, 32 that holds its node's K (KMAX bounds the variants so
// that the kernel's register count follows the batch's largest rank).
// The variant whose KB is the smallest of 4, 8, 12, 16, 24, 32 that holds
// the node's K (KMAX bounds the variants so that the kernel's register count
// follows the batch's largest rank).
template <int KMAX, int PPT, bool ASYNC>
__device__ __forceinline__ void bttm_dispatch(const BNode& nd, int64_t t, const float* __restrict__ T,
                                              const float* __restrict__ F, float* __restrict__ inter,
                                              float* __restrict__ G, float* Fs, float (*Ts)[kBThreads + 1]) {
  if (nd.K <= 4) bttm_tile<4, PPT, ASYNC>(nd, t, T, F, inter, G, Fs, Ts);
  else if (nd.K <= 8 || KMAX <= 8) bttm_tile<(KMAX < 8 ? KMAX : 8), PPT, ASYNC>(nd, t, T, F, inter, G, Fs, Ts);
  else if (nd.K <= 12 || KMAX <= 12) bttm_tile<(KMAX < 12 ? KMAX : 12), PPT, ASYNC>(nd, t, T, F, inter, G, Fs, Ts);
  else if (nd.K <= 16 || KMAX <= 16) bttm_tile<(KMAX < 16 ? KMAX : 16), PPT, ASYNC>(nd, t, T, F, inter, G, Fs, Ts);
  else if (nd.K <= 24 || KMAX <= 24) bttm_tile<(KMAX < 24 ? KMAX : 24), PPT, ASYNC>(nd, t, T, F, inter, G, Fs, Ts);
  else bttm_tile<KMAX, PPT, ASYNC>(nd, t, T, F, inter, G, Fs, Ts);
}

// 32 x 32 Gram tile over all M = R*C columns: FP32 products summed in runs of
// 32 columns, runs added in FP64.  The tile (and its mirror) is written whole.
__device__ __forceinline__ void bgram_tile(const BGram& g, const float* __restrict__ T,
                                           const float* __restrict__ inter, double* __restrict__ gram,
                                           float (*As)[33], float (*Bs)[33]) {
  const float* Z = (g.z_src ? inter : T) + g.z_off;
  const int64_t M = g.R * g.C;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 2 x 2 entries each
  double acc64[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int64_t m0 = 0; m0 < M; m0 += 32) {
    __syncthreads();
    for (int i = threadIdx.x; i < 32 * 32; i += kBThreads) {
      const int mm = i % 32, a = i / 32;
      const int64_t m = m0 + mm;
      float va = 0.f, vb = 0.f;
      if (m < M) {
        const int64_t r = m / g.C, c = m - (m / g.C) * g.C;
        const int la = g.ti * 32 + a, lb = g.tj * 32 + a;
        const int64_t ea = (r * g.L + la) * g.C + c, eb = (r * g.L + lb) * g.C + c;
        if (la < g.L && TK_DBG_IN(ea, ea, M * g.L)) va = Z[ea];
        if (lb < g.L && TK_DBG_IN(eb, eb, M * g.L)) vb = Z[eb];
      }
      As[a][mm] = va;
      Bs[a][mm] = vb;
    }
    __syncthreads();
    float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 8
    for (int mm = 0; mm < 32; ++mm) {
      const float a0 = As[ty * 2][mm], a1 = As[ty * 2 + 1][mm];
      const float b0 = Bs[tx * 2][mm], b1 = Bs[tx * 2 + 1][mm];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) acc64[i][j] += (double)acc[i][j];
  }
  double* W = gram + g.w_off;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int a = g.ti * 32 + ty * 2 + i, b = g.tj * 32 + tx * 2 + j;
      if (a < g.L && b < g.L) {
        W[(int64_t)a * g.L + b] = acc64[i][j];
        if (g.ti != g.tj) W[(int64_t)b * g.L + a] = acc64[i][j];
      }
    }
  }
}
// One step of the reconstruction G x_0 F_0 ... x_{N-1} F_{N-1} of one tensor
// (the expansion of mode m): In is viewed as [R][K][C], Out as [R][L][C] with
// Out[r, l, c] = sum_k F[l, k] In[r, k, c].  The last step of a tensor is not
// written: it is compared with T and the squared differences are summed.
struct BExp {
  int64_t in_off;   // into G (in_src 0) or the intermediate region (1)
  int64_t out_off;  // into the intermediate region, or T offset for the last step
  int64_t f_off;
  int64_t R, C;
  int32_t K, L;     // contracted length (rank) and output length
  int64_t tile0;
  int32_t in_src, last, tensor, pad;
};

constexpr int kExpMaxL = 200;

// Each thread owns PPT (r, c) positions, 256 apart: it keeps the K inputs
// In[r, :, c] of each in registers and produces the L outputs one after
// another (F from shared memory, broadcast).  In the last step the FP32
// differences T - Out are squared and summed in FP32 per position, then
// reduced in FP64 per block and added to res2[tensor].
// Returns, in thread 0, the tile's sum of squared differences (last step;
// 0 otherwise).  Fs holds kExpMaxL x KB floats.
template <int KB, int PPT>
__device__ __forceinline__ double bexpand_tile(const BExp& st, int64_t t, const float* __restrict__ T,
                                               const float* __restrict__ F, const float* __restrict__ G,
                                               float* __restrict__ inter, float (*Fs)[KB], double* red) {
  __syncthreads();  // Fs and red may still be read for the previous tile
  const float* f = F + st.f_off;
  for (int i = threadIdx.x; i < st.L * KB; i += kBThreads) {
    const int l = i / KB, k = i - (i / KB) * KB;
    Fs[l][k] = k < st.K ? f[(int64_t)l * st.K + k] : 0.f;
  }
  __syncthreads();
  const int64_t M = st.R * st.C;
  float y[PPT][KB];
  int64_t ob[PPT];
  bool act[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    const int64_t p = (t * PPT + j) * kBThreads + threadIdx.x;
    act[j] = p < M;
    const int64_t r = act[j] ? p / st.C : 0, c = act[j] ? p - r * st.C : 0;
    // inputs In[r, :, c] ([R][K][C]) and outputs Out[r, :, c] ([R][L][C])
    act[j] = act[j] && TK_DBG_IN((r * st.K) * st.C + c, (r * st.K + st.K - 1) * st.C + c, M * st.K) &&
             TK_DBG_IN((r * st.L) * st.C + c, (r * st.L + st.L - 1) * st.C + c, M * st.L);
    const float* in = (st.in_src ? inter : G) + st.in_off + (r * st.K) * st.C + c;
#pragma unroll
    for (int k = 0; k < KB; ++k) y[j][k] = (act[j] && k < st.K) ? in[(int64_t)k * st.C] : 0.f;
    ob[j] = (r * st.L) * st.C + c;
  }
  float part[PPT];
#pragma unroll
  for (int j = 0; j < PPT; ++j) part[j] = 0.f;
  if (act[0]) {
    if (st.last) {
      // kDepth rows of T are loaded ahead of their comparisons
      const float* t = T + st.out_off;
      for (int lb = 0; lb < st.L; lb += kDepth) {
        float tv[kDepth][PPT];
#pragma unroll
        for (int u = 0; u < kDepth; ++u)
#pragma unroll
          for (int j = 0; j < PPT; ++j)
            tv[u][j] = (lb + u < st.L && act[j]) ? __ldg(t + ob[j] + (int64_t)(lb + u) * st.C) : 0.f;
#pragma unroll
        for (int u = 0; u < kDepth; ++u) {
          if (lb + u >= st.L) break;
#pragma unroll
          for (int j = 0; j < PPT; ++j) {
            float v = 0.f;
#pragma unroll
            for (int k = 0; k < KB; ++k) v = fmaf(Fs[lb + u][k], y[j][k], v);
            if (act[j]) {
              const float d = tv[u][j] - v;
              part[j] = fmaf(d, d, part[j]);
            }
          }
        }
      }
    } else {
      float* o = inter + st.out_off;
      for (int l = 0; l < st.L; ++l) {
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
          float v = 0.f;
#pragma unroll
          for (int k = 0; k < KB; ++k) v = fmaf(Fs[l][k], y[j][k], v);
          if (act[j]) o[ob[j] + (int64_t)l * st.C] = v;
        }
      }
    }
  }
  if (!st.last) return 0.0;
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < PPT; ++j) s += (double)part[j];
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kBThreads / 32; ++w) tot += red[w];
  return tot;
}
}  // namespace
}  // namespace tk
