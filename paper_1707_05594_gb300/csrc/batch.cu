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
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "batch_bodies.cuh"
#include "batch_fused.h"

namespace tk {
namespace {

// One block per tile.
template <int KMAX, int PPT, bool ASYNC>
__global__ void __launch_bounds__(kBThreads)
    bttm_kernel(const BNode* __restrict__ nodes, const int* __restrict__ tile_node,
                const float* __restrict__ T, const float* __restrict__ F, float* __restrict__ inter,
                float* __restrict__ G) {
  __shared__ __align__(16) float Fs[32 * KMAX];
  __shared__ float Ts[32][kBThreads + 1];
  const int64_t tile = blockIdx.x;
  const BNode nd = nodes[tile_node[tile]];
  bttm_dispatch<KMAX, PPT, ASYNC>(nd, tile - nd.tile0, T, F, inter, G, Fs, Ts);
}

__global__ void __launch_bounds__(kBThreads)
    bgram_kernel(const BGram* __restrict__ tiles, const float* __restrict__ T,
                 const float* __restrict__ inter, double* __restrict__ gram) {
  __shared__ float As[32][33];
  __shared__ float Bs[32][33];
  bgram_tile(tiles[blockIdx.x], T, inter, gram, As, Bs);
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

template <int KB, int PPT>
__global__ void __launch_bounds__(kBThreads)
    bexpand_kernel(const BExp* __restrict__ steps, const int* __restrict__ tile_step,
                   const float* __restrict__ T,
                   const float* __restrict__ F, const float* __restrict__ G,
                   float* __restrict__ inter, double* __restrict__ res2) {
  __shared__ __align__(16) float Fs[kExpMaxL][KB];
  __shared__ double red[kBThreads / 32];
  const int64_t tile = blockIdx.x;
  const BExp st = steps[tile_step[tile]];
  const double s = bexpand_tile<KB, PPT>(st, tile - st.tile0, T, F, G, inter, Fs, red);
  if (st.last && threadIdx.x == 0) atomicAdd(res2 + st.tensor, s);
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

// Device side of one launch site: its work table, the tile -> item map (one
// int per tile, so that a block finds its item with one load), the tile
// count of the current configuration and the map's capacity (the most tiles
// any configuration gives).
template <class Item>
struct DevSite {
  Item* items = nullptr;
  int* map = nullptr;
  int64_t tiles = 0, cap = 0;
};

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
  // the fused sweep (batch_fused.cu): the same work, tensor by tensor
  std::vector<BNode> fz_nodes;                // tree nodes, tensor after tensor, parents first
  std::vector<BNode> fz_cores;                // core node of each tensor
  std::vector<BFusedTensor> fz_work;          // per tensor: its nodes and leaf Gram tiles
  std::vector<int> fz_order;                  // tensors by decreasing size (queue order)
  std::vector<BExp> fz_steps;                 // reconstruction steps [N][count]
  // workspace layout (bytes)
  size_t off_inter = 0, bytes_inter = 0;      // floats
  size_t off_gram = 0, bytes_gram = 0;        // doubles
  size_t off_eig = 0, bytes_eig = 0;
  size_t off_res = 0;                         // count doubles: residuals
  size_t off_cold = 0;                        // 1 + count * N ints: full-path list
  size_t off_fzfit = 0, bytes_fzfit = 0;      // floats: the fused sweep's reconstruction intermediates
  size_t off_queue = 0;                       // 4 ints: the fused sweep's work queue
  size_t off_tables = 0, bytes_tables = 0;
  size_t ws_total = 0;
  // device table addresses (valid after prepare)
  void* prepared_ws = nullptr;
  std::vector<DevSite<BNode>> d_levels;       // per tree level
  DevSite<BNode> d_core;
  const BGram* d_gram = nullptr;
  std::vector<DevSite<BNode>> d_sth;          // STHOSVD step n
  std::vector<const BGram*> d_sth_gram;
  const EigDesc* d_eig = nullptr;
  std::vector<DevSite<BExp>> d_fit;           // reconstruction step s
  const int64_t* d_t_off = nullptr;
  const int64_t* d_t_size = nullptr;
  const BNode* d_fz_nodes = nullptr;
  const BNode* d_fz_cores = nullptr;
  const BFusedTensor* d_fz_work = nullptr;
  const int* d_fz_order = nullptr;
  const BExp* d_fz_steps = nullptr;
  int fused = 0;                              // graphs record the fused sweep
  // launch configurations per site (defaults until tucker_batch_autotune)
  std::vector<BCfg> lvl_cfg;                  // per tree level
  BCfg core_cfg;
  std::vector<BCfg> fit_cfg;                  // per reconstruction step
  std::vector<float> tune_ms_default, tune_ms_best;  // per site, from the last autotune
  uint64_t epoch = 0;                         // bumped when the tile maps change

  struct GraphRec {
    uint64_t launches;                        // kernels recorded in the graph
    uint64_t epoch;                           // tile maps the graph was recorded with
  };
  std::unordered_map<void*, GraphRec> graph_launches;
};

namespace {

// The table of one launch site under a configuration: the nodes in the
// configuration's order, each with its first tile and its staging flag, and
// the tile -> node map.
std::vector<BNode> site_table(const std::vector<BNode>& v, const BCfg& cfg, int64_t* total,
                              std::vector<int>* map) {
  std::vector<BNode> out(v);
  if (cfg.order == 1)
    std::stable_sort(out.begin(), out.end(), [&](const BNode& a, const BNode& c) {
      return node_tiles(a.R, a.C, cfg) > node_tiles(c.R, c.C, cfg);
    });
  int64_t t = 0;
  map->clear();
  for (size_t i = 0; i < out.size(); ++i) {
    BNode& nd = out[i];
    nd.tile0 = t;
    nd.staged = node_staged(nd.C, cfg) ? 1 : 0;
    const int64_t n = node_tiles(nd.R, nd.C, cfg);
    map->insert(map->end(), (size_t)n, (int)i);
    t += n;
  }
  *total = t;
  return out;
}

inline int64_t exp_tiles(const BExp& e, const BCfg& cfg) {
  const int64_t tp = (int64_t)kBThreads * cfg.ppt;
  return (e.R * e.C + tp - 1) / tp;
}

std::vector<BExp> site_table(const std::vector<BExp>& v, const BCfg& cfg, int64_t* total,
                             std::vector<int>* map) {
  std::vector<BExp> out(v);
  if (cfg.order == 1)
    std::stable_sort(out.begin(), out.end(), [&](const BExp& a, const BExp& c) {
      return exp_tiles(a, cfg) > exp_tiles(c, cfg);
    });
  int64_t t = 0;
  map->clear();
  for (size_t i = 0; i < out.size(); ++i) {
    BExp& e = out[i];
    e.tile0 = t;
    const int64_t n = exp_tiles(e, cfg);
    map->insert(map->end(), (size_t)n, (int)i);
    t += n;
  }
  *total = t;
  return out;
}

// The most tiles a site can have under any configuration (one position per
// thread; rows staged up to the largest staging length, or not at all).
int64_t site_cap(const std::vector<BNode>& v) {
  int64_t c = 0;
  for (const BNode& nd : v)
    c += std::max(node_tiles(nd.R, nd.C, BCfg{1, 64, 0}), node_tiles(nd.R, nd.C, BCfg{1, 0, 0}));
  return c;
}
int64_t site_cap(const std::vector<BExp>& v) {
  int64_t c = 0;
  for (const BExp& e : v) c += exp_tiles(e, BCfg{1, 32, 0});
  return c;
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

// positions per thread allowed with the batch's largest rank class (4 only
// up to KB = 8: at KB = 16 its 64 accumulators per position set spill)
inline bool ppt_allowed(int KB, int ppt) { return ppt == 1 || ppt == 2 || (ppt == 4 && KB <= 8); }

template <int KMAX>
void bttm_launch(const BCfg& c, unsigned grid, cudaStream_t s, const BNode* d, const int* map,
                 const float* T, const float* F, float* inter, float* G) {
  if (c.async) bttm_kernel<KMAX, 1, true><<<grid, kBThreads, 0, s>>>(d, map, T, F, inter, G);
  else if (c.ppt == 4 && KMAX <= 8)
    bttm_kernel<KMAX, (KMAX <= 8 ? 4 : 2), false><<<grid, kBThreads, 0, s>>>(d, map, T, F, inter, G);
  else if (c.ppt == 2) bttm_kernel<KMAX, 2, false><<<grid, kBThreads, 0, s>>>(d, map, T, F, inter, G);
  else bttm_kernel<KMAX, 1, false><<<grid, kBThreads, 0, s>>>(d, map, T, F, inter, G);
}

int launch_bttm(const tucker_batch_s& b, const BCfg& cfg, const DevSite<BNode>& site, int64_t tiles,
                const float* T, const float* F, float* inter, float* G, cudaStream_t s) {
  if (tiles == 0) return TUCKER_OK;
  if (tiles > INT32_MAX || tiles > site.cap) return fail(TUCKER_ERR_UNSUPPORTED, "batch: tile map overflow");
  if (!ppt_allowed(b.KB, cfg.ppt) || (cfg.async && cfg.ppt != 1))
    return fail(TUCKER_ERR_INVALID_ARG, "batch: positions per thread");
  switch (b.KB) {
    case 8: bttm_launch<8>(cfg, (unsigned)tiles, s, site.items, site.map, T, F, inter, G); break;
    case 16: bttm_launch<16>(cfg, (unsigned)tiles, s, site.items, site.map, T, F, inter, G); break;
    default: bttm_launch<32>(cfg, (unsigned)tiles, s, site.items, site.map, T, F, inter, G); break;
  }
  TK_LAUNCH_CHECK("batch_ttm");
  return TUCKER_OK;
}

template <int KB>
void bexpand_launch(int ppt, unsigned grid, cudaStream_t s, const BExp* d, const int* map, const float* T,
                    const float* F, const float* G, float* inter, double* res2) {
  if (ppt == 4 && KB <= 8) bexpand_kernel<KB, (KB <= 8 ? 4 : 2)><<<grid, kBThreads, 0, s>>>(d, map, T, F, G, inter, res2);
  else if (ppt == 2) bexpand_kernel<KB, 2><<<grid, kBThreads, 0, s>>>(d, map, T, F, G, inter, res2);
  else bexpand_kernel<KB, 1><<<grid, kBThreads, 0, s>>>(d, map, T, F, G, inter, res2);
}

int launch_bexpand(const tucker_batch_s& b, const BCfg& cfg, const DevSite<BExp>& site, int64_t tiles,
                   const float* T, const float* F, const float* G, float* inter, double* res2,
                   cudaStream_t s) {
  if (tiles == 0) return TUCKER_OK;
  if (tiles > INT32_MAX || tiles > site.cap) return fail(TUCKER_ERR_UNSUPPORTED, "batch: tile map overflow");
  if (!ppt_allowed(b.KB, cfg.ppt)) return fail(TUCKER_ERR_INVALID_ARG, "batch: positions per thread");
  switch (b.KB) {
    case 8: bexpand_launch<8>(cfg.ppt, (unsigned)tiles, s, site.items, site.map, T, F, G, inter, res2); break;
    case 16: bexpand_launch<16>(cfg.ppt, (unsigned)tiles, s, site.items, site.map, T, F, G, inter, res2); break;
    default: bexpand_launch<32>(cfg.ppt, (unsigned)tiles, s, site.items, site.map, T, F, G, inter, res2); break;
  }
  TK_LAUNCH_CHECK("batch_fit_expand");
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
    BFusedTensor fw{};
    fw.node0 = (int32_t)b->fz_nodes.size();
    fw.gram0 = (int32_t)b->gram_tiles.size();
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
        BNode fz = bn;
        fz.staged = node_staged(bn.C, BCfg()) ? 1 : 0;
        b->fz_nodes.push_back(fz);
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
      BNode fz = bn;
      fz.staged = node_staged(bn.C, BCfg()) ? 1 : 0;
      b->fz_cores.push_back(fz);
      fw.nnodes = (int32_t)b->fz_nodes.size() - fw.node0;
      fw.ngram = (int32_t)b->gram_tiles.size() - fw.gram0;
      b->fz_work.push_back(fw);
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
  // the fused sweep: reconstruction steps [N][count] (their intermediates get
  // a region of their own: tensors are in different phases at once), queue
  // order by decreasing size
  for (size_t st = 0; st < b->fit_steps.size(); ++st)
    b->fz_steps.insert(b->fz_steps.end(), b->fit_steps[st].begin(), b->fit_steps[st].end());
  b->fz_order.resize((size_t)count);
  std::iota(b->fz_order.begin(), b->fz_order.end(), 0);
  std::stable_sort(b->fz_order.begin(), b->fz_order.end(),
                   [&](int a, int c) { return b->t_size[(size_t)a] > b->t_size[(size_t)c]; });
  b->bytes_fzfit = align_up(fit_inter * sizeof(float));
  inter = std::max(inter, fit_inter);
  while (!b->levels.empty() && b->levels.back().empty()) b->levels.pop_back();
  b->lvl_cfg.assign(b->levels.size(), BCfg());
  b->fit_cfg.assign(b->fit_steps.size(), BCfg());
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
  b->off_fzfit = off;
  off += b->bytes_fzfit;
  b->off_queue = off;
  off += align_up(4 * sizeof(int));
  b->off_tables = off;
  // work tables: each TTM / reconstruction site holds its items and a tile
  // map sized for the configuration with the most tiles
  size_t tb = 0;
  b->d_levels.assign(b->levels.size(), {});
  b->d_sth.assign(b->sth_ttm.size(), {});
  b->d_fit.assign(b->fit_steps.size(), {});
  auto site_bytes = [&](auto& site, const auto& items) {
    site.cap = site_cap(items);
    tb += align_up(items.size() * sizeof(items[0])) + align_up((size_t)site.cap * sizeof(int));
  };
  for (size_t st = 0; st < b->fit_steps.size(); ++st) site_bytes(b->d_fit[st], b->fit_steps[st]);
  for (size_t lv = 0; lv < b->levels.size(); ++lv) site_bytes(b->d_levels[lv], b->levels[lv]);
  site_bytes(b->d_core, b->core_nodes);
  tb += align_up(b->gram_tiles.size() * sizeof(BGram));
  for (size_t n = 0; n < b->sth_ttm.size(); ++n) site_bytes(b->d_sth[n], b->sth_ttm[n]);
  for (auto& v : b->sth_gram) tb += align_up(v.size() * sizeof(BGram));
  tb += align_up(b->eig.size() * sizeof(EigDesc));
  tb += 2 * align_up((size_t)count * sizeof(int64_t));
  tb += align_up(b->fz_nodes.size() * sizeof(BNode)) + align_up(b->fz_cores.size() * sizeof(BNode)) +
        align_up(b->fz_work.size() * sizeof(BFusedTensor)) + align_up(b->fz_order.size() * sizeof(int)) +
        align_up(b->fz_steps.size() * sizeof(BExp));
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
  // a site's items, then its tile map in a slot of `cap` ints
  bool ok = true;
  auto upload_site = [&](auto& site, const auto& items, const BCfg& cfg) {
    using Item = typename std::decay_t<decltype(items)>::value_type;
    std::vector<int> map;
    const std::vector<Item> t = site_table(items, cfg, &site.tiles, &map);
    site.items = reinterpret_cast<Item*>(upload(t.data(), t.size() * sizeof(Item)));
    site.map = reinterpret_cast<int*>(tp);
    if (!map.empty() && cudaMemcpyAsync(tp, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice,
                                        s) != cudaSuccess)
      ok = false;
    tp += align_up((size_t)site.cap * sizeof(int));
    if (!site.items || (int64_t)map.size() > site.cap || cudaStreamSynchronize(s) != cudaSuccess) ok = false;
  };
  for (size_t st = 0; st < b->fit_steps.size(); ++st) upload_site(b->d_fit[st], b->fit_steps[st], b->fit_cfg[st]);
  for (size_t lv = 0; lv < b->levels.size(); ++lv) upload_site(b->d_levels[lv], b->levels[lv], b->lvl_cfg[lv]);
  upload_site(b->d_core, b->core_nodes, b->core_cfg);
  b->d_gram = reinterpret_cast<const BGram*>(upload(b->gram_tiles.data(), b->gram_tiles.size() * sizeof(BGram)));
  for (size_t n = 0; n < b->sth_ttm.size(); ++n) upload_site(b->d_sth[n], b->sth_ttm[n], BCfg());
  if (!ok) return fail(TUCKER_ERR_CUDA, "tucker_batch_prepare: table upload failed");
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
  b->d_fz_nodes = reinterpret_cast<const BNode*>(upload(b->fz_nodes.data(), b->fz_nodes.size() * sizeof(BNode)));
  b->d_fz_cores = reinterpret_cast<const BNode*>(upload(b->fz_cores.data(), b->fz_cores.size() * sizeof(BNode)));
  b->d_fz_work = reinterpret_cast<const BFusedTensor*>(
      upload(b->fz_work.data(), b->fz_work.size() * sizeof(BFusedTensor)));
  b->d_fz_order = reinterpret_cast<const int*>(upload(b->fz_order.data(), b->fz_order.size() * sizeof(int)));
  b->d_fz_steps = reinterpret_cast<const BExp*>(upload(b->fz_steps.data(), b->fz_steps.size() * sizeof(BExp)));
  if (!b->d_core.items || !b->d_gram || !b->d_eig || !b->d_t_size || !b->d_fz_nodes || !b->d_fz_cores ||
      !b->d_fz_work || !b->d_fz_order || !b->d_fz_steps)
    return fail(TUCKER_ERR_CUDA, "tucker_batch_prepare: table upload failed");
  TK_CUDA_TRY(cudaMemsetAsync(base + b->off_queue, 0, 4 * sizeof(int), s));
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
    rc = launch_bttm(*b, b->lvl_cfg[lv], b->d_levels[lv], b->d_levels[lv].tiles, T, F_in, inter, nullptr, s);
    if (rc) return rc;
  }
  if (!b->gram_tiles.empty()) {
    bgram_kernel<<<(unsigned)b->gram_tiles.size(), kBThreads, 0, s>>>(b->d_gram, T, inter, gram);
    TK_LAUNCH_CHECK("batch_gram");
  }
  if (G_in) {
    rc = launch_bttm(*b, b->core_cfg, b->d_core, b->d_core.tiles, T, F_in, inter, G_in, s);
    if (rc) return rc;
  }
  return launch_eig_batched(b->d_eig, b->count * b->N, b->maxL, b->maxK, TUCKER_F32,
                            reinterpret_cast<char*>(F_out), reinterpret_cast<const char*>(F_in),
                            reinterpret_cast<int*>(base + b->off_cold), s);
}

int tucker_batch_sweep_fused(tucker_batch_t b, const float* T, const float* F_in, float* F_out,
                             float* G_in, const double* normT2, double* fit, void* ws, size_t ws_bytes,
                             void* stream) {
  if (!b || !T || !F_in || !F_out || !G_in || !normT2 || !fit)
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_sweep_fused: NULL argument");
  if (F_in == F_out) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_sweep_fused: F_out aliases F_in");
  int rc = check_batch_ws(b, ws, ws_bytes, "tucker_batch_sweep_fused");
  if (rc) return rc;
  if ((kernel_policy() & 2) != 0)
    return fail(TUCKER_ERR_UNSUPPORTED, "tucker_batch_sweep_fused: the fused sweep starts from the input factors "
                                        "(kernel policy bit 1 asks for the full eigensolver path)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  int* cold = reinterpret_cast<int*>(base + b->off_cold);
  TK_CUDA_TRY(cudaMemsetAsync(cold, 0, sizeof(int), s));
  BFusedArgs a{};
  a.work = b->d_fz_work;
  a.order = b->d_fz_order;
  a.count = b->count;
  a.N = b->N;
  a.KB = b->KB;
  a.nodes = b->d_fz_nodes;
  a.cores = b->d_fz_cores;
  a.grams = b->d_gram;
  a.steps = b->d_fz_steps;
  a.eigs = b->d_eig;
  a.f_base = reinterpret_cast<char*>(F_out);
  a.f0_base = reinterpret_cast<const char*>(F_in);
  a.T = T;
  a.F = F_in;
  a.inter = reinterpret_cast<float*>(base + b->off_inter);
  a.fit_inter = reinterpret_cast<float*>(base + b->off_fzfit);
  a.G = G_in;
  a.gram = reinterpret_cast<double*>(base + b->off_gram);
  a.normT2 = normT2;
  a.fit = fit;
  a.cold = cold;
  a.queue = reinterpret_cast<int*>(base + b->off_queue);
  a.status = device_status_ptr();
  if (!a.status) return fail(TUCKER_ERR_CUDA, "tucker_batch_sweep_fused: device error word unavailable");
  a.tol = 1e-12;
  rc = launch_batch_fused(a, b->maxL, b->maxK, s);
  if (rc) return rc;
  return launch_eig_cold_path(b->d_eig, b->count * b->N, b->maxL, b->maxK, a.f_base, a.f0_base, cold, s);
}

int tucker_batch_queue_offset(tucker_batch_t b, size_t* off) {
  if (!b || !off) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_queue_offset: NULL argument");
  *off = b->off_queue;
  return TUCKER_OK;
}

int tucker_batch_set_fused(tucker_batch_t b, int on) {
  if (!b || (on != 0 && on != 1)) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_set_fused: invalid argument");
  b->fused = on;
  return TUCKER_OK;
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
    rc = launch_bttm(*b, BCfg(), b->d_sth[(size_t)n], b->d_sth[(size_t)n].tiles, T, F, inter, G, s);
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
    rc = launch_bexpand(*b, b->fit_cfg[st], b->d_fit[st], b->d_fit[st].tiles, T, F, G, inter, res2, s);
    if (rc) return rc;
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
  int rc;
  if (b->fused && G_in && normT2 && fit) {
    rc = tucker_batch_sweep_fused(b, T, F_in, F_out, G_in, normT2, fit, ws, ws_bytes, cs);
  } else {
    rc = tucker_batch_sweep(b, T, F_in, F_out, G_in, ws, ws_bytes, cs);
    if (rc == TUCKER_OK && G_in && normT2 && fit)
      rc = tucker_batch_fit(b, T, F_in, G_in, normT2, fit, ws, ws_bytes, cs);
  }
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
  b->graph_launches[ex] = tucker_batch_s::GraphRec{recorded, b->epoch};
  *graph_exec = ex;
  return TUCKER_OK;
}

int tucker_batch_graph_launch(tucker_batch_t b, void* graph_exec, void* stream) {
  if (!b || !graph_exec) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_graph_launch: NULL argument");
  const auto it = b->graph_launches.find(graph_exec);
  if (it == b->graph_launches.end())
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_graph_launch: graph not created from this batch");
  if (it->second.epoch != b->epoch)
    return fail(TUCKER_ERR_INVALID_ARG,
                "tucker_batch_graph_launch: graph recorded before tucker_batch_autotune changed the tile "
                "maps; create it again");
  TK_CUDA_TRY(cudaGraphLaunch(static_cast<cudaGraphExec_t>(graph_exec),
                              static_cast<cudaStream_t>(stream)));
  count_launches(it->second.launches);
  return TUCKER_OK;
}

void tucker_batch_graph_destroy(void* graph_exec) {
  if (graph_exec) cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(graph_exec));
}

int tucker_batch_autotune(tucker_batch_t b, const float* T, const float* F, float* G, void* ws,
                          size_t ws_bytes, int reps, void* stream) {
  if (!b || !T || !F || !G) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_autotune: NULL argument");
  if (reps < 1 || reps > 1000) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_autotune: reps in 1..1000");
  int rc = check_batch_ws(b, ws, ws_bytes, "tucker_batch_autotune");
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  float* inter = reinterpret_cast<float*>(base + b->off_inter);
  double* res2 = reinterpret_cast<double*>(base + b->off_res);
  cudaEvent_t e0, e1;
  TK_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(TUCKER_ERR_CUDA, "tucker_batch_autotune: cudaEventCreate");
  }
  // candidates: the default first; another replaces the best only when at
  // least 2 % faster, so that timing noise does not pick a variant
  std::vector<BCfg> ttm_cands, exp_cands;
  const int ppts[3] = {1, 2, 4};
  const int stages[4] = {32, 0, 16, 64};  // staged rows need C <= 256
  for (int o = 0; o < 2; ++o) {
    for (int ppt : ppts) {
      if (!ppt_allowed(b->KB, ppt)) continue;
      for (int sc : stages) ttm_cands.push_back(BCfg{ppt, sc, o, 0});
      exp_cands.push_back(BCfg{ppt, 32, o, 0});
    }
    for (int sc : stages) ttm_cands.push_back(BCfg{1, sc, o, 1});
  }
  b->tune_ms_default.clear();
  b->tune_ms_best.clear();
  // time one site: upload each candidate's table to the site's slot, launch
  // once untimed, then `reps` times between events; keep the fastest
  auto tune_site = [&](const auto& items, auto& site, BCfg* cfg, const std::vector<BCfg>& cands,
                       auto&& launch) -> int {
    using Item = typename std::decay_t<decltype(items)>::value_type;
    // upload a candidate's table and tile map into the site's slots
    auto put = [&](const BCfg& c, int64_t* tiles) -> int {
      std::vector<int> map;
      const std::vector<Item> t = site_table(items, c, tiles, &map);
      if ((int64_t)map.size() > site.cap) return fail(TUCKER_ERR_UNSUPPORTED, "batch: tile map overflow");
      TK_CUDA_TRY(cudaMemcpyAsync(site.items, t.data(), t.size() * sizeof(Item), cudaMemcpyHostToDevice, s));
      if (!map.empty())
        TK_CUDA_TRY(cudaMemcpyAsync(site.map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      TK_CUDA_TRY(cudaStreamSynchronize(s));  // t and map go out of scope
      return TUCKER_OK;
    };
    float best_ms = 0.f, def_ms = 0.f;
    BCfg best = cands[0];
    for (size_t ci = 0; ci < cands.size(); ++ci) {
      int64_t tiles = 0;
      int r = put(cands[ci], &tiles);
      if (r) return r;
      r = launch(cands[ci], tiles);
      if (r) return r;
      TK_CUDA_TRY(cudaEventRecord(e0, s));
      for (int i = 0; i < reps && !r; ++i) r = launch(cands[ci], tiles);
      if (r) return r;
      TK_CUDA_TRY(cudaEventRecord(e1, s));
      TK_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      TK_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      ms /= (float)reps;
      if (ci == 0) {
        def_ms = best_ms = ms;
      } else if (ms < 0.98f * best_ms) {
        best_ms = ms;
        best = cands[ci];
      }
    }
    const int r = put(best, &site.tiles);
    if (r) return r;
    *cfg = best;
    b->tune_ms_default.push_back(def_ms);
    b->tune_ms_best.push_back(best_ms);
    return TUCKER_OK;
  };
  // tree levels in order (each reads the previous level's outputs), then the
  // core step (reads the tree's intermediates), then the reconstruction steps
  // of the fit (which reuse the intermediate region)
  for (size_t lv = 0; lv < b->levels.size() && !rc; ++lv) {
    const DevSite<BNode>& site = b->d_levels[lv];
    rc = tune_site(b->levels[lv], b->d_levels[lv], &b->lvl_cfg[lv], ttm_cands,
                   [&](const BCfg& c, int64_t tiles) {
                     return launch_bttm(*b, c, site, tiles, T, F, inter, nullptr, s);
                   });
  }
  if (!rc)
    rc = tune_site(b->core_nodes, b->d_core, &b->core_cfg, ttm_cands, [&](const BCfg& c, int64_t tiles) {
      return launch_bttm(*b, c, b->d_core, tiles, T, F, inter, G, s);
    });
  for (size_t st = 0; st < b->fit_steps.size() && !rc; ++st) {
    const DevSite<BExp>& site = b->d_fit[st];
    rc = tune_site(b->fit_steps[st], b->d_fit[st], &b->fit_cfg[st], exp_cands,
                   [&](const BCfg& c, int64_t tiles) {
                     return launch_bexpand(*b, c, site, tiles, T, F, G, inter, res2, s);
                   });
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ++b->epoch;  // graphs recorded before now hold the old tile counts
  return rc;
}

int tucker_batch_set_tuning(tucker_batch_t b, int n_sites, const int* cfg) {
  if (!b || !cfg) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_set_tuning: NULL argument");
  const int want = (int)b->levels.size() + 1 + (int)b->fit_steps.size();
  if (n_sites != want)
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_set_tuning: expected " + std::to_string(want) + " sites");
  std::vector<BCfg> lv(b->levels.size()), ft(b->fit_steps.size());
  BCfg core;
  for (int i = 0; i < n_sites; ++i) {
    const int* c = cfg + 6 * i;
    const int kind = i < (int)lv.size() ? 0 : (i == (int)lv.size() ? 1 : 2);
    const int index = kind == 0 ? i : (kind == 1 ? 0 : i - (int)lv.size() - 1);
    if (c[0] != kind || c[1] != index)
      return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_set_tuning: site " + std::to_string(i) +
                                              " out of order (as tucker_batch_tuning lists them)");
    if (!ppt_allowed(b->KB, c[2]) || c[3] < 0 || c[3] > 64 || (c[4] != 0 && c[4] != 1) ||
        (c[5] != 0 && c[5] != 1) || (c[5] == 1 && (kind == 2 || c[2] != 1)))
      return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_set_tuning: site " + std::to_string(i) +
                                              ": configuration out of range");
    const BCfg v{c[2], kind == 2 ? 32 : c[3], c[4], c[5]};
    if (kind == 0) lv[(size_t)index] = v;
    else if (kind == 1) core = v;
    else ft[(size_t)index] = v;
  }
  b->lvl_cfg = lv;
  b->core_cfg = core;
  b->fit_cfg = ft;
  b->tune_ms_default.clear();
  b->tune_ms_best.clear();
  b->prepared_ws = nullptr;  // the tables must be uploaded again
  ++b->epoch;
  return TUCKER_OK;
}

int tucker_batch_tuning(tucker_batch_t b, int cap, int* n_sites, int* cfg, float* ms) {
  if (!b || !n_sites) return fail(TUCKER_ERR_INVALID_ARG, "tucker_batch_tuning: NULL argument");
  std::vector<std::pair<int, int>> sites;  // (kind, index)
  std::vector<BCfg> cfgs;
  for (size_t lv = 0; lv < b->levels.size(); ++lv) {
    sites.push_back({0, (int)lv});
    cfgs.push_back(b->lvl_cfg[lv]);
  }
  sites.push_back({1, 0});
  cfgs.push_back(b->core_cfg);
  for (size_t st = 0; st < b->fit_steps.size(); ++st) {
    sites.push_back({2, (int)st});
    cfgs.push_back(b->fit_cfg[st]);
  }
  *n_sites = (int)sites.size();
  const bool timed = b->tune_ms_best.size() == sites.size();
  for (int i = 0; i < std::min(cap, (int)sites.size()); ++i) {
    if (cfg) {
      int* c = cfg + 6 * i;
      c[0] = sites[(size_t)i].first;
      c[1] = sites[(size_t)i].second;
      c[2] = cfgs[(size_t)i].ppt;
      c[3] = cfgs[(size_t)i].stage_c;
      c[4] = cfgs[(size_t)i].order;
      c[5] = cfgs[(size_t)i].async;
    }
    if (ms) {
      ms[2 * i] = timed ? b->tune_ms_default[(size_t)i] : -1.f;
      ms[2 * i + 1] = timed ? b->tune_ms_best[(size_t)i] : -1.f;
    }
  }
  return TUCKER_OK;
}

}  // extern "C"
