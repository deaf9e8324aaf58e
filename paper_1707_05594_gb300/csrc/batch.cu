// batch.cu -- the batched form: many independent small dense tensors (of
// uneven lengths and ranks) decomposed together.  Each tensor gets its own
// optimal TTM-tree (Sec. 3.3); the trees are executed level by level, so one
// sweep of the whole batch is a fixed, short sequence of launches, each over
// every tensor at once:
//   for each tree depth: one batched TTM over all nodes of that depth;
//   one batched Gram over all leaves (Sec. 5);
//   one batched TTM for the cores of the input factors (smallest leaf input
//     x_n F_n^T, as in tucker_hooi_sweep_core);
//   the eigensolver over all N * count Gram matrices (warm-started from the
//     input factors, full path where the on-GPU check fails);
//   optionally the fit of every tensor.
// Tables of work items live in the workspace and hold element offsets, not
// pointers, so they are built once (tucker_batch_prepare) and a whole sweep can
// be captured in a CUDA graph (tucker_batch_graph_create) and replayed.
//
// Data layout (all packed back to back, row-major per tensor):
//   T: tensor i at t_off[i];  F: factor (i, n) at f_off[i*N + n] (L x K);
//   G: core i at g_off[i].
#include <algorithm>
#include <cstring>
#include <numeric>
#include <unordered_map>
#include <vector>

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
  int64_t tile0;     // first tile (256 positions) of this node
  int32_t in_src, out_dst;
};

// One 32 x 32 tile of a leaf Gram W = Z_(n) Z_(n)^T (lower triangle, ti >= tj).
struct BGram {
  int64_t z_off;     // into T (z_src 0) or intermediates (1)
  int64_t w_off;     // into the Gram region (doubles)
  int64_t R, C;
  int32_t L, ti, tj, z_src;
};

// Tiles of a node: nodes whose rows are at least 32 elements long (C >= 32)
// take 256 consecutive (r, c) positions per tile and read along c; shorter
// rows take 256 / C whole rows per tile, staged through shared memory.
constexpr int kStageC = 32;
inline int64_t node_tiles(int64_t R, int64_t C) {
  if (C < kStageC) {
    const int64_t rt = kBThreads / C;
    return (R + rt - 1) / rt;
  }
  return (R * C + kBThreads - 1) / kBThreads;
}

// Out[r, k, c] = sum_l F[l, k] In[r, l, c] for one tile of one node, F in
// chunks of 32 l through shared memory.  Each thread accumulates the K
// outputs of one position (KB >= K registers).  Staged tiles (C < 32) copy
// the rows of the chunk into shared memory transposed, Ts[l][position], with
// coalesced loads, and write their outputs back the same way.
template <int KB>
__device__ __forceinline__ void bttm_tile(const BNode& nd, int64_t t, const float* __restrict__ T,
                                          const float* __restrict__ F, float* __restrict__ inter,
                                          float* __restrict__ G, float* Fs /* [32][KB] */,
                                          float (*Ts)[kBThreads + 1]) {
  const int tid = threadIdx.x;
  const bool staged = nd.C < kStageC;
  const float* src = (nd.in_src ? inter : T) + nd.in_off;
  float* dst = (nd.out_dst ? G : inter) + nd.out_off;
  const float* f = F + nd.f_off;
  // staged: rows r0 .. r0 + nrows - 1, position tid = (r - r0) * C + c
  // direct: position p = t * 256 + tid
  int64_t r0 = 0, r = 0, c = 0;
  int nrows = 0, C = (int)(staged ? nd.C : 0);
  bool active;
  if (staged) {
    const int rt = kBThreads / C;
    r0 = t * rt;
    nrows = (int)min((int64_t)rt, nd.R - r0);
    active = tid < nrows * C;
  } else {
    const int64_t p = t * kBThreads + tid;
    active = p < nd.R * nd.C;
    if (active) {
      r = p / nd.C;
      c = p - r * nd.C;
    }
  }
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
    if (staged) {
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
    } else {
      __syncthreads();
      if (active) {
        const float* in = src + (r * nd.L + l0) * nd.C + c;
#pragma unroll 4
        for (int l = 0; l < lc; ++l) {
          const float x = __ldg(in + (int64_t)l * nd.C);
#pragma unroll
          for (int k = 0; k < KB; ++k) acc[k] = fmaf(Fs[l * KB + k], x, acc[k]);
        }
      }
    }
  }
  if (staged) {
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
    return;
  }
  if (!active) return;
  float* out = dst + (r * nd.K) * nd.C + c;
#pragma unroll
  for (int k = 0; k < KB; ++k)
    if (k < nd.K) out[(int64_t)k * nd.C] = acc[k];
}

// One block per tile; the block runs the variant whose KB is the smallest of
// 4, 8, 12, 16, 24, 32 that holds its node's K (KMAX bounds the variants so
// that the kernel's register count follows the batch's largest rank).
template <int KMAX>
__global__ void __launch_bounds__(kBThreads)
    bttm_kernel(const BNode* __restrict__ nodes, int nnodes, const float* __restrict__ T,
                const float* __restrict__ F, float* __restrict__ inter, float* __restrict__ G) {
  __shared__ __align__(16) float Fs[32 * KMAX];
  __shared__ float Ts[32][kBThreads + 1];
  __shared__ int node_idx;
  const int64_t tile = blockIdx.x;
  if (threadIdx.x == 0) {
    int lo = 0, hi = nnodes - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (nodes[mid].tile0 <= tile) lo = mid;
      else hi = mid - 1;
    }
    node_idx = lo;
  }
  __syncthreads();
  const BNode nd = nodes[node_idx];
  const int64_t t = tile - nd.tile0;
  if (nd.K <= 4) bttm_tile<4>(nd, t, T, F, inter, G, Fs, Ts);
  else if (nd.K <= 8 || KMAX <= 8) bttm_tile<(KMAX < 8 ? KMAX : 8)>(nd, t, T, F, inter, G, Fs, Ts);
  else if (nd.K <= 12 || KMAX <= 12) bttm_tile<(KMAX < 12 ? KMAX : 12)>(nd, t, T, F, inter, G, Fs, Ts);
  else if (nd.K <= 16 || KMAX <= 16) bttm_tile<(KMAX < 16 ? KMAX : 16)>(nd, t, T, F, inter, G, Fs, Ts);
  else if (nd.K <= 24 || KMAX <= 24) bttm_tile<(KMAX < 24 ? KMAX : 24)>(nd, t, T, F, inter, G, Fs, Ts);
  else bttm_tile<KMAX>(nd, t, T, F, inter, G, Fs, Ts);
}

// 32 x 32 Gram tile over all M = R*C columns: FP32 products summed in runs of
// 32 columns, runs added in FP64.  The tile (and its mirror) is written whole.
__global__ void __launch_bounds__(kBThreads)
    bgram_kernel(const BGram* __restrict__ tiles, const float* __restrict__ T,
                 const float* __restrict__ inter, double* __restrict__ gram) {
  const BGram g = tiles[blockIdx.x];
  __shared__ float As[32][33];
  __shared__ float Bs[32][33];
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
        if (la < g.L) va = Z[(r * g.L + la) * g.C + c];
        if (lb < g.L) vb = Z[(r * g.L + lb) * g.C + c];
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

// ||X_i||^2 per tensor (one block per tensor), FP64 accumulation.
__global__ void __launch_bounds__(kBThreads)
    bnorm_kernel(const int64_t* __restrict__ off, const int64_t* __restrict__ size,
                 const float* __restrict__ X, double* __restrict__ out) {
  const int64_t o = off[blockIdx.x], n = size[blockIdx.x];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kBThreads) {
    const double v = X[o + i];
    s += v * v;
  }
  __shared__ double red[kBThreads / 32];
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBThreads / 32; ++w) t += red[w];
    out[blockIdx.x] = t;
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

// Each thread owns one (r, c) position: it keeps the K inputs In[r, :, c] in
// registers and produces the L outputs one after another (F from shared
// memory, broadcast).  In the last step the FP32 differences T - Out are
// squared and summed in FP32 per thread, then reduced in FP64 per block and
// added to res2[tensor].
template <int KB>
__global__ void __launch_bounds__(kBThreads)
    bexpand_kernel(const BExp* __restrict__ steps, int nsteps, const float* __restrict__ T,
                   const float* __restrict__ F, const float* __restrict__ G,
                   float* __restrict__ inter, double* __restrict__ res2) {
  __shared__ __align__(16) float Fs[kExpMaxL][KB];
  __shared__ int step_idx;
  __shared__ double red[kBThreads / 32];
  const int64_t tile = blockIdx.x;
  if (threadIdx.x == 0) {
    int lo = 0, hi = nsteps - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (steps[mid].tile0 <= tile) lo = mid;
      else hi = mid - 1;
    }
    step_idx = lo;
  }
  __syncthreads();
  const BExp st = steps[step_idx];
  const float* f = F + st.f_off;
  for (int i = threadIdx.x; i < st.L * KB; i += kBThreads) {
    const int l = i / KB, k = i - (i / KB) * KB;
    Fs[l][k] = k < st.K ? f[(int64_t)l * st.K + k] : 0.f;
  }
  __syncthreads();
  const int64_t p = (tile - st.tile0) * kBThreads + threadIdx.x;
  float part = 0.f;
  if (p < st.R * st.C) {
    const int64_t r = p / st.C, c = p - (p / st.C) * st.C;
    const float* in = (st.in_src ? inter : G) + st.in_off + (r * st.K) * st.C + c;
    float y[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) y[k] = k < st.K ? in[(int64_t)k * st.C] : 0.f;
    const int64_t ob = (r * st.L) * st.C + c;
    if (st.last) {
      const float* t = T + st.out_off + ob;
      for (int l = 0; l < st.L; ++l) {
        float v = 0.f;
#pragma unroll
        for (int k = 0; k < KB; ++k) v = fmaf(Fs[l][k], y[k], v);
        const float d = __ldg(t + (int64_t)l * st.C) - v;
        part = fmaf(d, d, part);
      }
    } else {
      float* o = inter + st.out_off + ob;
      for (int l = 0; l < st.L; ++l) {
        float v = 0.f;
#pragma unroll
        for (int k = 0; k < KB; ++k) v = fmaf(Fs[l][k], y[k], v);
        o[(int64_t)l * st.C] = v;
      }
    }
  }
  if (!st.last) return;
  double s = (double)part;
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kBThreads / 32; ++w) t += red[w];
    atomicAdd(res2 + st.tensor, t);
  }
}

// fit_i = 1 - ||T_i - G_i x F||_F / ||T_i||_F (Sec. 2.2), from the residual.
__global__ void bfit_finish_kernel(int count, const double* __restrict__ res2,
                                   const double* __restrict__ normT2, double* __restrict__ fit) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) fit[i] = 1.0 - sqrt(res2[i]) / sqrt(normT2[i]);
}

int64_t prod64(const int64_t* d, int a, int b) {
  int64_t p = 1;
  for (int i = a; i < b; ++i) p *= d[i];
  return p;
}

}  // namespace
}  // namespace tk

using namespace tk;

struct tucker_batch_s {
  int count = 0, N = 0, maxL = 1, maxK = 1, KB = 8;
  std::vector<int64_t> dims, ranks;           // count * N
  std::vector<int64_t> t_off, t_size, f_off, g_off, g_size;
  int64_t t_total = 0, f_total = 0, g_total = 0;
  // host tables (offsets only)
  std::vector<std::vector<BNode>> levels;     // sweep tree levels
  std::vector<BNode> core_nodes;              // one per tensor
  std::vector<BGram> gram_tiles;              // sweep leaves
  std::vector<std::vector<BNode>> sth_ttm;    // STHOSVD step n
  std::vector<std::vector<BGram>> sth_gram;   // STHOSVD Gram of step n
  std::vector<EigDesc> eig;                   // [mode][tensor]
  std::vector<std::vector<BExp>> fit_steps;   // reconstruction step s of every tensor
  int64_t level_tiles_max = 0;
  // workspace layout (bytes)
  size_t off_inter = 0, bytes_inter = 0;      // floats
  size_t off_gram = 0, bytes_gram = 0;        // doubles
  size_t off_eig = 0, bytes_eig = 0;
  size_t off_res = 0;                         // count doubles: residuals
  size_t off_cold = 0;                        // 1 + count * N ints: full-path list
  size_t off_tables = 0, bytes_tables = 0;
  size_t ws_total = 0;
  // device table addresses (valid after prepare)
  void* prepared_ws = nullptr;
  std::vector<const BNode*> d_levels;
  std::vector<int64_t> level_tiles;
  const BNode* d_core = nullptr;
  int64_t core_tiles = 0;
  const BGram* d_gram = nullptr;
  std::vector<const BNode*> d_sth_ttm;
  std::vector<int64_t> sth_tiles;
  std::vector<const BGram*> d_sth_gram;
  const EigDesc* d_eig = nullptr;
  std::vector<const BExp*> d_fit;
  std::vector<int64_t> fit_tiles;
  const int64_t* d_t_off = nullptr;
  const int64_t* d_t_size = nullptr;

  std::unordered_map<void*, uint64_t> graph_launches;  // kernels recorded per graph
};

namespace {

void add_tiles(std::vector<BNode>& v, int64_t* total) {
  int64_t t = 0;
  for (BNode& nd : v) {
    nd.tile0 = t;
    t += node_tiles(nd.R, nd.C);
  }
  *total = t;
}

void add_tiles(std::vector<BExp>& v, int64_t* total) {
  int64_t t = 0;
  for (BExp& e : v) {
    e.tile0 = t;
    t += (e.R * e.C + kBThreads - 1) / kBThreads;
  }
  *total = t;
}

void gram_tiles_for(std::vector<BGram>& v, int64_t z_off, int z_src, int64_t w_off, int64_t R,
                    int64_t L, int64_t C) {
  const int nt = (int)((L + 31) / 32);
  for (int ti = 0; ti < nt; ++ti)
    for (int tj = 0; tj <= ti; ++tj) {
      BGram g{};
      g.z_off = z_off;
      g.w_off = w_off;
      g.R = R;
      g.C = C;
      g.L = (int)L;
      g.ti = ti;
      g.tj = tj;
      g.z_src = z_src;
      v.push_back(g);
    }
}

int launch_bttm(const tucker_batch_s& b, const BNode* d_nodes, int64_t nnodes, int64_t tiles,
                const float* T, const float* F, float* inter, float* G, cudaStream_t s) {
  if (nnodes == 0 || tiles == 0) return TUCKER_OK;
  if (tiles > INT32_MAX) return fail(TUCKER_ERR_UNSUPPORTED, "batch: too many tiles");
  switch (b.KB) {
    case 8: bttm_kernel<8><<<(unsigned)tiles, kBThreads, 0, s>>>(d_nodes, (int)nnodes, T, F, inter, G); break;
    case 16: bttm_kernel<16><<<(unsigned)tiles, kBThreads, 0, s>>>(d_nodes, (int)nnodes, T, F, inter, G); break;
    default: bttm_kernel<32><<<(unsigned)tiles, kBThreads, 0, s>>>(d_nodes, (int)nnodes, T, F, inter, G); break;
  }
  TK_LAUNCH_CHECK("batch_ttm");
  return TUCKER_OK;
}

int check_batch_ws(const tucker_batch_s* b, void* ws, size_t ws_bytes, const char* who) {
  if (!ws || ws_bytes < b->ws_total)
    return fail(TUCKER_ERR_WORKSPACE, std::string(who) + ": workspace smaller than ws_bytes");
  if (b->prepared_ws != ws)
    return fail(TUCKER_ERR_INVALID_ARG,
                std::string(who) + ": call tucker_batch_prepare with this workspace first");
  return TUCKER_OK;
}

}  // namespace

extern "C" {

int tucker_batch_plan(int count, int N, const int64_t* dims, const int64_t* ranks,
                      tucker_batch_t* out) {
  if (!out || count < 1 || N < 2 || N > kMaxModes || !dims || !ranks)
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_plan: invalid argument");
  *out = nullptr;
  if ((int64_t)count * N > 65535)
    return fail(TUCKER_ERR_UNSUPPORTED, "tucker_batch_plan: at most 65535 eigenproblems per sweep");
  tucker_batch_s* b = new tucker_batch_s();
  b->count = count;
  b->N = N;
  b->dims.assign(dims, dims + (size_t)count * N);
  b->ranks.assign(ranks, ranks + (size_t)count * N);
  b->t_off.resize(count);
  b->t_size.resize(count);
  b->f_off.resize((size_t)count * N);
  b->g_off.resize(count);
  b->g_size.resize(count);
  b->levels.assign((size_t)N, {});
  b->sth_ttm.assign((size_t)N, {});
  b->sth_gram.assign((size_t)N, {});
  b->eig.resize((size_t)count * N);
  b->fit_steps.assign((size_t)N, {});
  size_t inter = 0, gram = 0, eigb = 0, fit_inter = 0;
  for (int i = 0; i < count; ++i) {
    const int64_t* L = dims + (size_t)i * N;
    const int64_t* K = ranks + (size_t)i * N;
    tucker_plan_t p = nullptr;
    const int rc = tucker_plan(N, L, K, nullptr, &p);
    if (rc) {
      delete b;
      return fail(rc, "tucker_batch_plan: tensor " + std::to_string(i) + ": " + tucker_last_error());
    }
    const Plan& pl = p->p;
    b->t_off[(size_t)i] = b->t_total;
    b->t_size[(size_t)i] = prod64(L, 0, N);
    b->t_total += b->t_size[(size_t)i];
    for (int n = 0; n < N; ++n) {
      b->f_off[(size_t)i * N + n] = b->f_total;
      b->f_total += L[n] * K[n];
      b->maxL = std::max<int>(b->maxL, (int)L[n]);
      b->maxK = std::max<int>(b->maxK, (int)K[n]);
      if (L[n] > 200 || K[n] > 32) {
        tucker_plan_destroy(p);
        delete b;
        return fail(TUCKER_ERR_UNSUPPORTED, "tucker_batch_plan: needs L_n <= 200 and K_n <= 32");
      }
    }
    b->g_off[(size_t)i] = b->g_total;
    b->g_size[(size_t)i] = prod64(K, 0, N);
    b->g_total += b->g_size[(size_t)i];
    // tree nodes: every internal node gets its own intermediate buffer
    std::vector<int64_t> out_off(pl.nodes.size(), 0);
    std::vector<int> depth(pl.nodes.size(), 0);
    int best_leaf = -1;
    uint64_t best = ~0ull;
    for (size_t j = 1; j < pl.nodes.size(); ++j) {
      const PlanNode& nd = pl.nodes[j];
      const PlanNode& par = pl.nodes[(size_t)nd.parent];
      depth[j] = depth[(size_t)nd.parent] + 1;
      int64_t R, Ln, C;
      const int mode = nd.label >= 0 ? nd.label : -nd.label - 2;
      R = prod64(par.out_dims, 0, mode);
      Ln = par.out_dims[mode];
      C = prod64(par.out_dims, mode + 1, N);
      if (nd.label >= 0) {
        out_off[j] = (int64_t)inter;
        inter += nd.out_elems;
        BNode bn{};
        bn.in_off = nd.parent == 0 ? b->t_off[(size_t)i] : out_off[(size_t)nd.parent];
        bn.in_src = nd.parent == 0 ? 0 : 1;
        bn.out_off = out_off[j];
        bn.out_dst = 0;
        bn.f_off = b->f_off[(size_t)i * N + mode];
        bn.R = R;
        bn.C = C;
        bn.L = (int)Ln;
        bn.K = (int)K[mode];
        b->levels[(size_t)depth[j] - 1].push_back(bn);
      } else {
        // leaf of mode `mode`: Gram of its parent's output
        const int64_t w_off = (int64_t)gram;
        gram += (size_t)Ln * (size_t)Ln;
        const bool from_T = nd.parent == 0;
        gram_tiles_for(b->gram_tiles, from_T ? b->t_off[(size_t)i] : out_off[(size_t)nd.parent],
                       from_T ? 0 : 1, w_off, R, Ln, C);
        EigDesc& d = b->eig[(size_t)mode * count + i];
        d.W = reinterpret_cast<const double*>(w_off);  // element offset, fixed at prepare
        d.F = reinterpret_cast<void*>(b->f_off[(size_t)i * N + mode] * sizeof(float));
        d.F0 = reinterpret_cast<const void*>(b->f_off[(size_t)i * N + mode] * sizeof(float));
        d.L = (int)Ln;
        d.K = (int)K[mode];
        d.stat = reinterpret_cast<double*>(eigb);  // byte offset, fixed at prepare
        eigb += eig_bytes_per_matrix((size_t)Ln, (size_t)K[mode]);
        if (nd.in_elems < best) {
          best = nd.in_elems;
          best_leaf = (int)j;
        }
      }
    }
    {
      // core of the input factors from the smallest leaf input
      const PlanNode& leaf = pl.nodes[(size_t)best_leaf];
      const PlanNode& par = pl.nodes[(size_t)leaf.parent];
      const int mode = -leaf.label - 2;
      BNode bn{};
      bn.in_off = leaf.parent == 0 ? b->t_off[(size_t)i] : out_off[(size_t)leaf.parent];
      bn.in_src = leaf.parent == 0 ? 0 : 1;
      bn.out_off = b->g_off[(size_t)i];
      bn.out_dst = 1;
      bn.f_off = b->f_off[(size_t)i * N + mode];
      bn.R = prod64(par.out_dims, 0, mode);
      bn.L = (int)par.out_dims[mode];
      bn.C = prod64(par.out_dims, mode + 1, N);
      bn.K = (int)K[mode];
      b->core_nodes.push_back(bn);
    }
    // STHOSVD, natural mode order: Y_0 = T, Y_{n+1} = Y_n x_n F_n^T, G = Y_N
    {
      int64_t yd[kMaxModes];
      std::memcpy(yd, L, sizeof(int64_t) * (size_t)N);
      int64_t prev_off = b->t_off[(size_t)i];
      int prev_src = 0;
      for (int n = 0; n < N; ++n) {
        const int64_t R = prod64(yd, 0, n), Ln = yd[n], C = prod64(yd, n + 1, N);
        // the Gram of Y_n along mode n uses the same matrix slot as the sweep
        const EigDesc& d = b->eig[(size_t)n * count + i];
        gram_tiles_for(b->sth_gram[(size_t)n], prev_off, prev_src,
                       (int64_t)reinterpret_cast<size_t>(d.W), R, Ln, C);
        BNode bn{};
        bn.in_off = prev_off;
        bn.in_src = prev_src;
        bn.f_off = b->f_off[(size_t)i * N + n];
        bn.R = R;
        bn.L = (int)Ln;
        bn.C = C;
        bn.K = (int)K[n];
        if (n == N - 1) {
          bn.out_off = b->g_off[(size_t)i];
          bn.out_dst = 1;
        } else {
          bn.out_off = (int64_t)inter;
          bn.out_dst = 0;
          inter += (size_t)(R * K[n] * C);
        }
        b->sth_ttm[(size_t)n].push_back(bn);
        yd[n] = K[n];
        prev_off = bn.out_off;
        prev_src = 1;
      }
    }
    // reconstruction for the fit: expand the modes from the core; the last
    // step, fused with the comparison against T, is the only one over |T|
    // positions, so it takes the mode of smallest rank among modes 0..N-2
    // (a mode before the last keeps its reads of T along contiguous rows);
    // the others go by increasing L_n / K_n
    {
      int last = 0;
      for (int n = 1; n < N - 1; ++n)
        if (K[n] < K[last]) last = n;
      std::vector<int> order;
      for (int n = 0; n < N; ++n)
        if (n != last) order.push_back(n);
      std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return (double)L[a] / (double)K[a] < (double)L[c] / (double)K[c];
      });
      order.push_back(last);
      int64_t cur[kMaxModes];
      std::memcpy(cur, K, sizeof(int64_t) * (size_t)N);
      int64_t prev = b->g_off[(size_t)i];
      int src = 0;
      for (int s = 0; s < N; ++s) {
        const int m = order[(size_t)s];
        BExp e{};
        e.in_off = prev;
        e.in_src = src;
        e.f_off = b->f_off[(size_t)i * N + m];
        e.R = prod64(cur, 0, m);
        e.C = prod64(cur, m + 1, N);
        e.K = (int)K[m];
        e.L = (int)L[m];
        e.tensor = i;
        e.last = s == N - 1;
        cur[m] = L[m];
        if (e.last) {
          e.out_off = b->t_off[(size_t)i];
        } else {
          e.out_off = (int64_t)fit_inter;
          fit_inter += (size_t)(e.R * e.L * e.C);
        }
        b->fit_steps[(size_t)s].push_back(e);
        prev = e.out_off;
        src = 1;
      }
    }
    tucker_plan_destroy(p);
  }
  inter = std::max(inter, fit_inter);
  while (!b->levels.empty() && b->levels.back().empty()) b->levels.pop_back();
  b->KB = b->maxK <= 8 ? 8 : (b->maxK <= 16 ? 16 : 32);
  // workspace layout
  size_t off = 0;
  b->off_inter = off;
  b->bytes_inter = align_up(inter * sizeof(float));
  off += b->bytes_inter;
  b->off_gram = off;
  b->bytes_gram = align_up(gram * sizeof(double));
  off += b->bytes_gram;
  b->off_eig = off;
  b->bytes_eig = align_up(eigb);
  off += b->bytes_eig;
  b->off_res = off;
  off += align_up((size_t)count * sizeof(double));
  b->off_cold = off;
  off += align_up((size_t)(1 + (size_t)count * N) * sizeof(int));
  b->off_tables = off;
  size_t tb = 0;
  for (auto& v : b->fit_steps) tb += align_up(v.size() * sizeof(BExp));
  for (auto& v : b->levels) tb += align_up(v.size() * sizeof(BNode));
  tb += align_up(b->core_nodes.size() * sizeof(BNode));
  tb += align_up(b->gram_tiles.size() * sizeof(BGram));
  for (auto& v : b->sth_ttm) tb += align_up(v.size() * sizeof(BNode));
  for (auto& v : b->sth_gram) tb += align_up(v.size() * sizeof(BGram));
  tb += align_up(b->eig.size() * sizeof(EigDesc));
  tb += 2 * align_up((size_t)count * sizeof(int64_t));
  b->bytes_tables = tb;
  off += align_up(tb);
  b->ws_total = off;
  *out = b;
  return TUCKER_OK;
}

int tucker_batch_info(tucker_batch_t b, size_t* ws_bytes, int64_t* t_elems, int64_t* f_elems,
                      int64_t* g_elems) {
  if (!b) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_info: NULL batch");
  if (ws_bytes) *ws_bytes = b->ws_total;
  if (t_elems) *t_elems = b->t_total;
  if (f_elems) *f_elems = b->f_total;
  if (g_elems) *g_elems = b->g_total;
  return TUCKER_OK;
}

int tucker_batch_offsets(tucker_batch_t b, int64_t* t_off, int64_t* f_off, int64_t* g_off) {
  if (!b) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_offsets: NULL batch");
  if (t_off) std::memcpy(t_off, b->t_off.data(), sizeof(int64_t) * b->t_off.size());
  if (f_off) std::memcpy(f_off, b->f_off.data(), sizeof(int64_t) * b->f_off.size());
  if (g_off) std::memcpy(g_off, b->g_off.data(), sizeof(int64_t) * b->g_off.size());
  return TUCKER_OK;
}

void tucker_batch_destroy(tucker_batch_t b) { delete b; }

int tucker_batch_prepare(tucker_batch_t b, void* ws, size_t ws_bytes, void* stream) {
  if (!b || !ws) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_prepare: NULL argument");
  if (ws_bytes < b->ws_total)
    return fail(TUCKER_ERR_WORKSPACE, "tucker_batch_prepare: workspace smaller than ws_bytes");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  char* tp = base + b->off_tables;
  auto upload = [&](const void* src, size_t bytes) -> char* {
    char* dst = tp;
    if (bytes) {
      if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return nullptr;
    }
    tp += align_up(bytes);
    return dst;
  };
  b->d_levels.clear();
  b->level_tiles.clear();
  for (auto& v : b->levels) {
    int64_t tiles = 0;
    add_tiles(v, &tiles);
    b->level_tiles.push_back(tiles);
    b->d_levels.push_back(reinterpret_cast<const BNode*>(upload(v.data(), v.size() * sizeof(BNode))));
  }
  add_tiles(b->core_nodes, &b->core_tiles);
  b->d_core = reinterpret_cast<const BNode*>(upload(b->core_nodes.data(), b->core_nodes.size() * sizeof(BNode)));
  b->d_gram = reinterpret_cast<const BGram*>(upload(b->gram_tiles.data(), b->gram_tiles.size() * sizeof(BGram)));
  b->d_sth_ttm.clear();
  b->sth_tiles.clear();
  for (auto& v : b->sth_ttm) {
    int64_t tiles = 0;
    add_tiles(v, &tiles);
    b->sth_tiles.push_back(tiles);
    b->d_sth_ttm.push_back(reinterpret_cast<const BNode*>(upload(v.data(), v.size() * sizeof(BNode))));
  }
  b->d_fit.clear();
  b->fit_tiles.clear();
  for (auto& v : b->fit_steps) {
    int64_t tiles = 0;
    add_tiles(v, &tiles);
    b->fit_tiles.push_back(tiles);
    b->d_fit.push_back(reinterpret_cast<const BExp*>(upload(v.data(), v.size() * sizeof(BExp))));
  }
  b->d_sth_gram.clear();
  for (auto& v : b->sth_gram)
    b->d_sth_gram.push_back(reinterpret_cast<const BGram*>(upload(v.data(), v.size() * sizeof(BGram))));
  // eigen descriptors: absolute addresses in this workspace; F / F0 stay offsets
  std::vector<EigDesc> ed(b->eig.size());
  double* gram = reinterpret_cast<double*>(base + b->off_gram);
  for (size_t j = 0; j < ed.size(); ++j) {
    const EigDesc& src = b->eig[j];
    EigDesc d{};
    eig_desc_layout(d, base + b->off_eig + reinterpret_cast<size_t>(src.stat), src.L, src.K);
    d.W = gram + reinterpret_cast<size_t>(src.W);
    d.F = src.F;
    d.F0 = src.F0;
    ed[j] = d;
  }
  b->d_eig = reinterpret_cast<const EigDesc*>(upload(ed.data(), ed.size() * sizeof(EigDesc)));
  b->d_t_off = reinterpret_cast<const int64_t*>(upload(b->t_off.data(), b->t_off.size() * sizeof(int64_t)));
  b->d_t_size = reinterpret_cast<const int64_t*>(upload(b->t_size.data(), b->t_size.size() * sizeof(int64_t)));
  if (!b->d_core || !b->d_gram || !b->d_eig || !b->d_t_size)
    return fail(TUCKER_ERR_CUDA, "tucker_batch_prepare: table upload failed");
  TK_CUDA_TRY(cudaStreamSynchronize(s));  // the host tables above go out of scope
  b->prepared_ws = ws;
  return TUCKER_OK;
}

int tucker_batch_sweep(tucker_batch_t b, const float* T, const float* F_in, float* F_out,
                       float* G_in, void* ws, size_t ws_bytes, void* stream) {
  if (!b || !T || !F_in || !F_out) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_sweep: NULL argument");
  if (F_in == F_out) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_sweep: F_out aliases F_in");
  int rc = check_batch_ws(b, ws, ws_bytes, "tucker_batch_sweep");
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  float* inter = reinterpret_cast<float*>(base + b->off_inter);
  double* gram = reinterpret_cast<double*>(base + b->off_gram);
  for (size_t lv = 0; lv < b->levels.size(); ++lv) {
    rc = launch_bttm(*b, b->d_levels[lv], (int64_t)b->levels[lv].size(), b->level_tiles[lv], T,
                     F_in, inter, nullptr, s);
    if (rc) return rc;
  }
  if (!b->gram_tiles.empty()) {
    bgram_kernel<<<(unsigned)b->gram_tiles.size(), kBThreads, 0, s>>>(b->d_gram, T, inter, gram);
    TK_LAUNCH_CHECK("batch_gram");
  }
  if (G_in) {
    rc = launch_bttm(*b, b->d_core, (int64_t)b->core_nodes.size(), b->core_tiles, T, F_in, inter, G_in, s);
    if (rc) return rc;
  }
  return launch_eig_batched(b->d_eig, b->count * b->N, b->maxL, b->maxK, TUCKER_F32,
                            reinterpret_cast<char*>(F_out), reinterpret_cast<const char*>(F_in),
                            reinterpret_cast<int*>(base + b->off_cold), s);
}

int tucker_batch_sthosvd(tucker_batch_t b, const float* T, float* F, float* G, void* ws,
                         size_t ws_bytes, void* stream) {
  if (!b || !T || !F || !G) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_sthosvd: NULL argument");
  int rc = check_batch_ws(b, ws, ws_bytes, "tucker_batch_sthosvd");
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  float* inter = reinterpret_cast<float*>(base + b->off_inter);
  double* gram = reinterpret_cast<double*>(base + b->off_gram);
  for (int n = 0; n < b->N; ++n) {
    bgram_kernel<<<(unsigned)b->sth_gram[(size_t)n].size(), kBThreads, 0, s>>>(b->d_sth_gram[(size_t)n], T,
                                                                             inter, gram);
    TK_LAUNCH_CHECK("batch_gram");
    rc = launch_eig_batched(b->d_eig + (size_t)n * b->count, b->count, b->maxL, b->maxK, TUCKER_F32,
                            reinterpret_cast<char*>(F), nullptr,
                            reinterpret_cast<int*>(base + b->off_cold), s);
    if (rc) return rc;
    rc = launch_bttm(*b, b->d_sth_ttm[(size_t)n], (int64_t)b->sth_ttm[(size_t)n].size(),
                     b->sth_tiles[(size_t)n], T, F, inter, G, s);
    if (rc) return rc;
  }
  return TUCKER_OK;
}

int tucker_batch_norm2(tucker_batch_t b, const float* T, double* normT2, void* ws, size_t ws_bytes,
                       void* stream) {
  if (!b || !T || !normT2) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_norm2: NULL argument");
  int rc = check_batch_ws(b, ws, ws_bytes, "tucker_batch_norm2");
  if (rc) return rc;
  bnorm_kernel<<<(unsigned)b->count, kBThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      b->d_t_off, b->d_t_size, T, normT2);
  TK_LAUNCH_CHECK("batch_norm2");
  return TUCKER_OK;
}

int tucker_batch_fit(tucker_batch_t b, const float* T, const float* F, const float* G,
                     const double* normT2, double* fit, void* ws, size_t ws_bytes, void* stream) {
  if (!b || !T || !F || !G || !normT2 || !fit)
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_fit: NULL argument");
  int rc = check_batch_ws(b, ws, ws_bytes, "tucker_batch_fit");
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  float* inter = reinterpret_cast<float*>(base + b->off_inter);
  double* res2 = reinterpret_cast<double*>(base + b->off_res);
  TK_CUDA_TRY(cudaMemsetAsync(res2, 0, sizeof(double) * (size_t)b->count, s));
  for (size_t st = 0; st < b->fit_steps.size(); ++st) {
    const int64_t tiles = b->fit_tiles[st];
    const int n = (int)b->fit_steps[st].size();
    if (tiles > INT32_MAX) return fail(TUCKER_ERR_UNSUPPORTED, "batch: too many tiles");
    switch (b->KB) {
      case 8: bexpand_kernel<8><<<(unsigned)tiles, kBThreads, 0, s>>>(b->d_fit[st], n, T, F, G, inter, res2); break;
      case 16: bexpand_kernel<16><<<(unsigned)tiles, kBThreads, 0, s>>>(b->d_fit[st], n, T, F, G, inter, res2); break;
      default: bexpand_kernel<32><<<(unsigned)tiles, kBThreads, 0, s>>>(b->d_fit[st], n, T, F, G, inter, res2); break;
    }
    TK_LAUNCH_CHECK("batch_fit_expand");
  }
  bfit_finish_kernel<<<(b->count + 255) / 256, 256, 0, s>>>(b->count, res2, normT2, fit);
  TK_LAUNCH_CHECK("batch_fit_finish");
  return TUCKER_OK;
}

int tucker_batch_graph_create(tucker_batch_t b, const float* T, const float* F_in, float* F_out,
                              float* G_in, const double* normT2, double* fit, void* ws,
                              size_t ws_bytes, void** graph_exec) {
  if (!graph_exec) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_graph_create: NULL out");
  *graph_exec = nullptr;
  cudaStream_t cs;
  TK_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  const uint64_t launches0 = tucker_launch_count();
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return fail(TUCKER_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
  }
  int rc = tucker_batch_sweep(b, T, F_in, F_out, G_in, ws, ws_bytes, cs);
  if (rc == TUCKER_OK && G_in && normT2 && fit)
    rc = tucker_batch_fit(b, T, F_in, G_in, normT2, fit, ws, ws_bytes, cs);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (rc != TUCKER_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(TUCKER_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(TUCKER_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  // recording launched nothing: take the recorded kernels off the counter and
  // count them at every replay instead
  const uint64_t recorded = tucker_launch_count() - launches0;
  count_launches((uint64_t)0 - recorded);
  b->graph_launches[ex] = recorded;
  *graph_exec = ex;
  return TUCKER_OK;
}

int tucker_batch_graph_launch(tucker_batch_t b, void* graph_exec, void* stream) {
  if (!b || !graph_exec) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_graph_launch: NULL argument");
  TK_CUDA_TRY(cudaGraphLaunch(static_cast<cudaGraphExec_t>(graph_exec),
                              static_cast<cudaStream_t>(stream)));
  const auto it = b->graph_launches.find(graph_exec);
  if (it != b->graph_launches.end()) count_launches(it->second);
  return TUCKER_OK;
}

void tucker_batch_graph_destroy(void* graph_exec) {
  if (graph_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(graph_exec));
}

}  // extern "C"
