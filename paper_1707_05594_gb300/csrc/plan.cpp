// plan.cpp -- host-side planner: optimal TTM-tree by dynamic programming
// (Sec. 3.3), the prior-scheme trees of Sec. 3.2, the depth-first execution
// order with its stack memory plan (Sec. 3.1: the live intermediates are
// bounded by the tree depth), the new-core chain order, and the workspace
// layout.  No device work happens here.
#include <algorithm>
#include <cstring>
#include <functional>
#include <limits>
#include <new>
#include <string>

#include "internal.h"

namespace tk {

thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

uint64_t tensor_size(const Plan& p, unsigned P) {
  uint64_t s = 1;
  for (int n = 0; n < p.N; ++n) s *= (uint64_t)(((P >> n) & 1u) ? p.K[n] : p.L[n]);
  return s;
}

namespace {

constexpr uint64_t kInf = std::numeric_limits<uint64_t>::max();

int popcount(unsigned x) { return __builtin_popcount(x); }

// Cost of the TTM along mode m applied to T[P] (Sec. 3.1 "Computational Load",
// or the elements it moves).
uint64_t node_cost(const Plan& p, unsigned P, int m) {
  const uint64_t in = tensor_size(p, P);
  if (p.cost_model == TUCKER_COST_ELEMS) return in + tensor_size(p, P | (1u << m));
  return (uint64_t)p.K[m] * in;
}

// DP table entry for the subproblem (P, Q); R is the complement of P u Q.
struct Cell {
  uint64_t cost = kInf;
  int reuse = -1;     // mode reused at the root of the partial tree, or -1
  unsigned q1 = 0;    // first group of a split (valid when reuse == -1)
};

// Bottom-up DP over (P, Q).  Supersets of P are finished before P (they are
// numerically larger), and subsets of Q before Q.  The split of Q into Q1, Q2
// passes Q2's modes to Q1's subproblem as reusable and vice versa (the
// subproblems are (P, Q1, R u Q2) and (P, Q2, R u Q1)).  Ties: reuse before
// split, lower mode first, then the first split met.
std::vector<Cell> solve_dp(const Plan& p) {
  const int N = p.N;
  const unsigned full = (1u << N) - 1u;
  std::vector<Cell> tab((size_t)1 << (2 * N));
  auto at = [&](unsigned P, unsigned Q) -> Cell& { return tab[((size_t)P << N) | Q]; };
  for (int P = (int)full; P >= 0; --P) {
    const unsigned notP = full & ~(unsigned)P;
    // iterate non-empty Q subset of notP in increasing numeric order
    for (unsigned Q = 1; Q <= notP; ++Q) {
      if ((Q & ~notP) != 0) continue;
      Cell& c = at((unsigned)P, Q);
      const unsigned R = notP & ~Q;
      if (popcount(Q) == 1 && R == 0) {
        c.cost = 0;
        continue;
      }
      for (int m = 0; m < N; ++m) {
        if (!((R >> m) & 1u)) continue;
        const Cell& sub = at((unsigned)P | (1u << m), Q);
        if (sub.cost == kInf) continue;
        const uint64_t v = node_cost(p, (unsigned)P, m) + sub.cost;
        if (v < c.cost) {
          c.cost = v;
          c.reuse = m;
        }
      }
      if (popcount(Q) >= 2) {
        const unsigned low = Q & (~Q + 1u);
        const unsigned rest = Q & ~low;
        unsigned S = 0;
        for (;;) {
          const unsigned q1 = low | S, q2 = Q & ~q1;
          if (q2 != 0) {
            const Cell& a = at((unsigned)P, q1);
            const Cell& b = at((unsigned)P, q2);
            if (a.cost != kInf && b.cost != kInf && a.cost + b.cost < c.cost) {
              c.cost = a.cost + b.cost;
              c.reuse = -1;
              c.q1 = q1;
            }
          }
          if (S == rest) break;
          S = (S - rest) & rest;
        }
      }
    }
  }
  return tab;
}

struct Builder {
  Plan& p;
  explicit Builder(Plan& pp) : p(pp) {}

  int add_node(int label, int parent, unsigned P) {
    PlanNode nd;
    nd.label = label;
    nd.parent = parent;
    nd.P = P;
    for (int n = 0; n < p.N; ++n) nd.out_dims[n] = ((P >> n) & 1u) ? p.K[n] : p.L[n];
    if (label >= 0) {
      const unsigned Pin = P & ~(1u << label);
      nd.in_elems = tensor_size(p, Pin);
      nd.out_elems = tensor_size(p, P);
      nd.macs = (uint64_t)p.K[label] * nd.in_elems;
    } else if (label == -1) {
      nd.in_elems = nd.out_elems = tensor_size(p, 0);
    } else {
      nd.in_elems = tensor_size(p, P);
      nd.out_elems = 0;
    }
    p.nodes.push_back(nd);
    return (int)p.nodes.size() - 1;
  }

  // Emit the partial tree for (P, Q) hanging off node `u` (whose Out is T[P]).
  void emit_opt(const std::vector<Cell>& tab, int u, unsigned P, unsigned Q) {
    const int N = p.N;
    const unsigned full = (1u << N) - 1u;
    const Cell& c = tab[((size_t)P << N) | Q];
    const unsigned R = full & ~(P | Q);
    if (popcount(Q) == 1 && R == 0) {
      const int n = __builtin_ctz(Q);
      add_node(-(n + 2), u, P);
      return;
    }
    if (c.reuse >= 0) {
      const int v = add_node(c.reuse, u, P | (1u << c.reuse));
      emit_opt(tab, v, P | (1u << c.reuse), Q);
    } else {
      emit_opt(tab, u, P, c.q1);
      emit_opt(tab, u, P, Q & ~c.q1);
    }
  }

  // Chain of modes `order` (skipping n) from the root, ending in leaf n.
  void emit_chain(const std::vector<int>& order, int n) {
    int u = 0;
    unsigned P = 0;
    for (int m : order) {
      if (m == n) continue;
      P |= 1u << m;
      u = add_node(m, u, P);
    }
    add_node(-(n + 2), u, P);
  }

  // Balanced tree (Sec. 3.2) over `modes` below node u with Out = T[P].
  void emit_balanced(int u, unsigned P, const std::vector<int>& modes) {
    if (modes.size() == 1) {
      add_node(-(modes[0] + 2), u, P);
      return;
    }
    const size_t m = modes.size() / 2;
    std::vector<int> g1(modes.begin(), modes.begin() + (long)m);
    std::vector<int> g2(modes.begin() + (long)m, modes.end());
    for (int side = 0; side < 2; ++side) {
      const std::vector<int>& chain = side == 0 ? g1 : g2;
      const std::vector<int>& rest = side == 0 ? g2 : g1;
      int v = u;
      unsigned Pc = P;
      for (int md : chain) {
        Pc |= 1u << md;
        v = add_node(md, v, Pc);
      }
      emit_balanced(v, Pc, rest);
    }
  }
};

// Stack memory plan: a node's output stays live while its subtree runs, so
// the buffer of a node sits right after its parent's buffer.  With a fused
// root the second root child's output is written together with the first
// one's and stays live through the first one's subtree: it goes after the
// peak of the plain stack plan, and its own subtree after it.
void memory_plan(Plan& p) {
  size_t peak = 0;
  std::vector<size_t> end(p.nodes.size(), 0);
  for (int pass = 0; pass < (p.fused_u2 > 0 ? 2 : 1); ++pass) {
    const size_t plain_peak = peak;
    for (size_t i = 0; i < p.nodes.size(); ++i) {
      PlanNode& nd = p.nodes[i];
      if (nd.label < 0) continue;  // root (T is the input) and leaves own no buffer
      const int par = nd.parent;
      size_t base = (par <= 0) ? 0 : end[(size_t)par];
      if (pass == 1 && (int)i == p.fused_u2) base = plain_peak;
      nd.ws_off = base;
      end[i] = base + align_up((size_t)nd.out_elems * p.inter_bytes());
      peak = std::max(peak, end[i]);
    }
  }
  p.bytes_scratch = std::max(p.bytes_scratch, peak);
}

// Fused root: the first two root children in depth-first order, when both
// are TTM nodes whose pair of modes one kernel takes (root_pair_fits).
void choose_fused_root(Plan& p) {
  int u[2] = {-1, -1}, found = 0;
  for (size_t i = 1; i < p.nodes.size() && found < 2; ++i)
    if (p.nodes[i].parent == 0 && p.nodes[i].label >= 0) u[found++] = (int)i;
  if (found < 2) return;
  const int m1 = p.nodes[(size_t)u[0]].label, m2 = p.nodes[(size_t)u[1]].label;
  if (!root_pair_fits(p.dtype, p.N, p.L, p.K, std::min(m1, m2), std::max(m1, m2))) return;
  p.fused_u1 = u[0];
  p.fused_u2 = u[1];
}

// Mode order of the new-core chain minimising multiply-adds: DP over the set
// S of modes already applied.  Among equal-cost orders the higher modes go
// last, so the full tensor is read by a leading-mode TTM (long contiguous
// fibres) rather than by the last-mode one.
void core_chain(Plan& p) {
  const int N = p.N;
  const unsigned full = (1u << N) - 1u;
  std::vector<uint64_t> best((size_t)1 << N, kInf);
  std::vector<int> last((size_t)1 << N, -1);
  best[0] = 0;
  for (unsigned S = 1; S <= full; ++S) {
    for (int m = N - 1; m >= 0; --m) {
      if (!((S >> m) & 1u)) continue;
      const unsigned prev = S & ~(1u << m);
      if (best[prev] == kInf) continue;
      const uint64_t v = best[prev] + (uint64_t)p.K[m] * tensor_size(p, prev);
      if (v < best[S]) {
        best[S] = v;
        last[S] = m;
      }
    }
  }
  p.core_macs = best[full];
  p.core_order.assign((size_t)N, 0);
  unsigned S = full;
  for (int i = N - 1; i >= 0; --i) {
    p.core_order[(size_t)i] = last[S];
    S &= ~(1u << last[S]);
  }
  // two ping-pong buffers large enough for every step after the first
  size_t mx = 0;
  unsigned P = 0;
  for (int i = 0; i < N; ++i) {
    P |= 1u << p.core_order[(size_t)i];
    mx = std::max(mx, (size_t)tensor_size(p, P));
  }
  p.bytes_scratch = std::max(p.bytes_scratch, 2 * align_up(mx * p.inter_bytes()));
}

// Gauss-Seidel sweeps: for each n a chain over the other modes in the
// core-chain order, in two ping-pong buffers.
void gs_buffers(Plan& p) {
  size_t mx = 0;
  for (int n = 0; n < p.N; ++n) {
    unsigned P = 0;
    for (int i = 0; i < p.N; ++i) {
      const int m = p.core_order[(size_t)i];
      if (m == n) continue;
      P |= 1u << m;
      mx = std::max(mx, (size_t)tensor_size(p, P));
    }
  }
  p.bytes_scratch = std::max(p.bytes_scratch, 2 * align_up(mx * p.inter_bytes()));
}

// Cost of one STHOSVD step on mode m of T[P] (the modes of P already
// truncated): the Gram Y_(m) Y_(m)^T (L_m * |Y| multiply-adds, reading Y)
// and the TTM Y x_m F_m^T (K_m * |Y|, reading Y and writing T[P + m]).
uint64_t sthosvd_step_cost(const Plan& p, unsigned P, int m) {
  const uint64_t y = tensor_size(p, P);
  if (p.cost_model == TUCKER_COST_ELEMS) return 2 * y + tensor_size(p, P | (1u << m));
  return (uint64_t)(p.L[m] + p.K[m]) * y;
}

// STHOSVD mode order: natural, or (TUCKER_PLAN_STHOSVD_ORDER) the order of
// least cost by a DP over the set S of modes already truncated -- the cost of
// a step depends only on S and the mode taken, as a TTM-tree node's does on
// (P, n).  Among equal-cost orders the higher mode goes last, so the natural
// order is kept whenever it is optimal.  Y then lives in two ping-pong
// buffers sized for the largest tensor after a step (the last one is G).
void sthosvd_order(Plan& p, bool optimise) {
  const int N = p.N;
  const unsigned full = (1u << N) - 1u;
  p.sth_order.assign((size_t)N, 0);
  for (int n = 0; n < N; ++n) p.sth_order[(size_t)n] = n;
  if (optimise) {
    std::vector<uint64_t> best((size_t)1 << N, kInf);
    std::vector<int> last((size_t)1 << N, -1);
    best[0] = 0;
    for (unsigned S = 1; S <= full; ++S) {
      for (int m = N - 1; m >= 0; --m) {
        if (!((S >> m) & 1u)) continue;
        const unsigned prev = S & ~(1u << m);
        if (best[prev] == kInf) continue;
        const uint64_t v = best[prev] + sthosvd_step_cost(p, prev, m);
        if (v < best[S]) {
          best[S] = v;
          last[S] = m;
        }
      }
    }
    unsigned S = full;
    for (int i = N - 1; i >= 0; --i) {
      p.sth_order[(size_t)i] = last[S];
      S &= ~(1u << last[S]);
    }
  }
  p.sth_cost = 0;
  size_t mx = 0;
  unsigned P = 0;
  for (int i = 0; i < N; ++i) {
    const int m = p.sth_order[(size_t)i];
    p.sth_cost += sthosvd_step_cost(p, P, m);
    P |= 1u << m;
    mx = std::max(mx, (size_t)tensor_size(p, P));
  }
  p.bytes_scratch = std::max(p.bytes_scratch, 2 * align_up(mx * p.inter_bytes()));
}

}  // namespace

size_t eig_ws_bytes(int batch, const int64_t* L, const int64_t* K) {
  size_t total = kAlign;  // list of the matrices sent to the full path
  if (batch <= 0) return 0;
  for (int b = 0; b < batch; ++b) total += eig_bytes_per_matrix((size_t)L[b], (size_t)K[b]);
  return total;
}

// Buffer placement of a built tree: the fused root (when asked for and the
// kernel takes it), the stack memory plan, the core chain, the Gauss-Seidel
// chains and STHOSVD buffers, then the workspace layout.
void layout(Plan& p, bool fuse, bool sth_opt) {
  p.fused_u1 = p.fused_u2 = -1;
  p.bytes_scratch = 0;
  if (fuse) choose_fused_root(p);
  memory_plan(p);
  core_chain(p);
  gs_buffers(p);
  sthosvd_order(p, sth_opt);
  size_t off = 0;
  p.off_scratch = off;
  off += align_up(p.bytes_scratch);
  for (int n = 0; n < p.N; ++n) {
    p.off_gram[n] = off;
    off += align_up((size_t)p.L[n] * (size_t)p.L[n] * 8);
  }
  p.off_eig = off;
  p.bytes_eig = eig_ws_bytes(p.N, p.L, p.K);
  off += align_up(p.bytes_eig);
  p.off_misc = off;
  off += align_up(64 * 8);
  p.ws_total = off;
}

}  // namespace tk

using namespace tk;

extern "C" {

const char* tucker_last_error(void) { return g_last_error.c_str(); }

int tucker_version(void) { return 100; }

int tucker_plan(int N, const int64_t* L, const int64_t* K, const tucker_plan_opts_t* opts,
                tucker_plan_t* out) {
  if (!out) return fail(TUCKER_ERR_INVALID_ARG, "tucker_plan: out is NULL");
  *out = nullptr;
  if (N < 2 || N > kMaxModes)
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_plan: N must be in [2, 8]");
  if (!L || !K) return fail(TUCKER_ERR_INVALID_ARG, "tucker_plan: L or K is NULL");
  tucker_plan_opts_t o{TUCKER_F32, TUCKER_TREE_OPTIMAL, TUCKER_COST_MACS, 0, 0};
  if (opts) o = *opts;
  if (o.dtype != TUCKER_F32 && o.dtype != TUCKER_F64 && o.dtype != TUCKER_BF16 &&
      o.dtype != TUCKER_FP8_E4M3 && o.dtype != TUCKER_BF16_SPLIT)
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_plan: unknown dtype");
  if (o.tree < TUCKER_TREE_OPTIMAL || o.tree > TUCKER_TREE_BALANCED)
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_plan: unknown tree kind");
  if (o.cost_model != TUCKER_COST_MACS && o.cost_model != TUCKER_COST_ELEMS)
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_plan: unknown cost model");
  if (o.flags & ~(TUCKER_PLAN_NO_FUSED_ROOT | TUCKER_PLAN_STHOSVD_ORDER))
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_plan: unknown flags");
  long double total = 1;
  for (int n = 0; n < N; ++n) {
    if (L[n] < 1 || K[n] < 1 || K[n] > L[n])
      return fail(TUCKER_ERR_INVALID_ARG, "tucker_plan: need 1 <= K_n <= L_n for every mode");
    total *= (long double)L[n];
  }
  if (total >= (long double)(1ull << 40))
    return fail(TUCKER_ERR_UNSUPPORTED, "tucker_plan: tensor has 2^40 elements or more");
  for (int n = 0; n < N; ++n) {
    long double other = 1;
    for (int j = 0; j < N; ++j)
      if (j != n) other *= (long double)K[j];
    if ((long double)K[n] > other)
      return fail(TUCKER_ERR_INVALID_ARG,
                  "tucker_plan: K_n exceeds the product of the other core lengths "
                  "(Z_(n) would have rank below K_n)");
  }

  if (o.dtype == TUCKER_BF16_SPLIT) {
    // every TTM whose input is T reads the split tensor on the tensor cores
    for (int n = 0; n < N; ++n) {
      int64_t R = 1, C = 1;
      for (int j = 0; j < n; ++j) R *= L[j];
      for (int j = n + 1; j < N; ++j) C *= L[j];
      if (!ttm_tc_split_fits(R, L[n], C, K[n]))
        return fail(TUCKER_ERR_UNSUPPORTED,
                    "tucker_plan: TUCKER_BF16_SPLIT needs every mode's TTM of T on the tensor cores "
                    "(later lengths' product a multiple of 8 and >= 64, or a last mode whose length "
                    "is a multiple of 8; K_n <= 64)");
    }
  }

  tucker_plan_s* h = new (std::nothrow) tucker_plan_s();
  if (!h) return fail(TUCKER_ERR_INVALID_ARG, "tucker_plan: out of host memory");
  Plan& p = h->p;
  p.N = N;
  for (int n = 0; n < N; ++n) {
    p.L[n] = L[n];
    p.K[n] = K[n];
  }
  p.dtype = o.dtype;
  p.tree = o.tree;
  p.cost_model = o.cost_model;

  Builder b(p);
  b.add_node(-1, -1, 0u);
  const unsigned full = (1u << N) - 1u;
  std::vector<int> natural(N);
  for (int n = 0; n < N; ++n) natural[(size_t)n] = n;
  if (p.tree == TUCKER_TREE_OPTIMAL) {
    std::vector<Cell> tab = solve_dp(p);
    b.emit_opt(tab, 0, 0u, full);
  } else if (p.tree == TUCKER_TREE_BALANCED) {
    b.emit_balanced(0, 0u, natural);
  } else {
    std::vector<int> order = natural;
    if (p.tree == TUCKER_TREE_CHAIN_K)
      std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return p.K[a] < p.K[c]; });
    if (p.tree == TUCKER_TREE_CHAIN_H)
      std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        // h_a < h_c  <=>  K_a * L_c < K_c * L_a (exact)
        return (__int128)p.K[a] * p.L[c] < (__int128)p.K[c] * p.L[a];
      });
    for (int n = 0; n < N; ++n) b.emit_chain(order, n);
  }
  for (const PlanNode& nd : p.nodes) {
    if (nd.label >= 0) {
      p.tree_macs += nd.macs;
      p.tree_elems += nd.in_elems + nd.out_elems;
    }
  }
  bool fuse = !(o.flags & TUCKER_PLAN_NO_FUSED_ROOT);
  bool sth_opt = (o.flags & TUCKER_PLAN_STHOSVD_ORDER) != 0;
  layout(p, fuse, sth_opt);
  // a workspace cap trades the fused root first, then the STHOSVD order
  if (o.ws_cap > 0 && p.ws_total > o.ws_cap && p.fused_u1 >= 0) layout(p, fuse = false, sth_opt);
  if (o.ws_cap > 0 && p.ws_total > o.ws_cap && sth_opt) layout(p, fuse, sth_opt = false);
  if (o.ws_cap > 0 && p.ws_total > o.ws_cap) {
    const std::string msg = "tucker_plan: the workspace needs " + std::to_string(p.ws_total) +
                            " bytes at least, above the cap of " + std::to_string(o.ws_cap);
    delete h;
    return fail(TUCKER_ERR_WORKSPACE, msg);
  }
  *out = h;
  return TUCKER_OK;
}

int tucker_plan_cost(tucker_plan_t plan, uint64_t* tree_macs, uint64_t* tree_elems,
                     uint64_t* core_macs, size_t* ws_bytes) {
  if (!plan) return fail(TUCKER_ERR_INVALID_ARG, "tucker_plan_cost: plan is NULL");
  const Plan& p = plan->p;
  if (tree_macs) *tree_macs = p.tree_macs;
  if (tree_elems) *tree_elems = p.tree_elems;
  if (core_macs) *core_macs = p.core_macs;
  if (ws_bytes) *ws_bytes = p.ws_total;
  return TUCKER_OK;
}

int tucker_plan_nodes(tucker_plan_t plan, tucker_node_t* nodes, int capacity, int* n_nodes) {
  if (!plan || !n_nodes) return fail(TUCKER_ERR_INVALID_ARG, "tucker_plan_nodes: NULL argument");
  const Plan& p = plan->p;
  *n_nodes = (int)p.nodes.size();
  if (nodes) {
    for (int i = 0; i < capacity && i < (int)p.nodes.size(); ++i) {
      const PlanNode& nd = p.nodes[(size_t)i];
      nodes[i].label = nd.label;
      nodes[i].parent = nd.parent;
      nodes[i].in_elems = nd.in_elems;
      nodes[i].out_elems = nd.out_elems;
      nodes[i].macs = nd.macs;
      nodes[i].ws_offset = nd.ws_off;
    }
  }
  return TUCKER_OK;
}

int tucker_plan_fused_root(tucker_plan_t plan, int* first, int* second) {
  if (!plan || !first || !second) return fail(TUCKER_ERR_INVALID_ARG, "tucker_plan_fused_root: NULL argument");
  *first = plan->p.fused_u1;
  *second = plan->p.fused_u2;
  return TUCKER_OK;
}

int tucker_plan_sthosvd(tucker_plan_t plan, int* order, uint64_t* cost) {
  if (!plan || !order) return fail(TUCKER_ERR_INVALID_ARG, "tucker_plan_sthosvd: NULL argument");
  for (int i = 0; i < plan->p.N; ++i) order[i] = plan->p.sth_order[(size_t)i];
  if (cost) *cost = plan->p.sth_cost;
  return TUCKER_OK;
}

void tucker_plan_destroy(tucker_plan_t plan) {
  if (!plan) return;
  destroy_profile(plan->p);
  delete plan;
}

size_t tucker_eig_ws_bytes(int batch, const int64_t* L, const int64_t* K) {
  if (batch <= 0 || !L || !K) return 0;
  return eig_ws_bytes(batch, L, K);
}

}  // extern "C"
