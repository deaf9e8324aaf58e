/*
 * planner_oracle.c -- brute-force and reference computations for TTM-trees
 * (Sec. 3 of the paper).
 *
 * TEST INFRASTRUCTURE ONLY (loaded by tests/ and bench.py's baseline leg);
 * shares no code with the library planner.
 *
 * Definitions followed:
 *   Sec. 3.1 "TTM-Trees": a rooted tree whose root is T, whose N leaves carry
 *     the new factors F~_n, whose internal nodes carry a mode, and where the
 *     root-to-leaf path of F~_n holds exactly the N-1 modes other than n.
 *   Sec. 3.1 "Computational Load": a node u labelled n costs K_n * |In(u)| and
 *     its output has |In(u)| * K_n / L_n elements; a tree costs the sum over
 *     its internal nodes.  |T[P]| = prod_{n in P} K_n * prod_{n not in P} L_n.
 *     The enumeration and the tree validator also take a second node cost,
 *     the elements a node moves (|In(u)| + |Out(u)|), summed the same way.
 *   Sec. 3.2: chain trees (N independent chains, a mode ordering), K-order,
 *     h-order and balanced trees (Kaya-Ucar divide and conquer).
 *   Sec. 3.3: the (P, Q, R) recurrence.  The printed split term is read as
 *     cost(P, Q1, R u Q2) + cost(P, Q2, R u Q1): inside the subtree for Q1 the
 *     modes of Q2 must still be multiplied, so they become reusable there.
 *
 * orc_tree_bruteforce enumerates every TTM-tree of any arity explicitly (not
 * only binary ones), so that it also checks Lemma 3.1 (an optimal binary tree
 * exists) against the DP, which only builds binary trees.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned long long u64;
#define ORC_INF 0xFFFFFFFFFFFFFFFFull

static int g_N;
static u64 g_L[16], g_K[16];
static unsigned g_full;

static void set_problem(int N, const int64_t* L, const int64_t* K) {
  g_N = N;
  for (int i = 0; i < N; ++i) { g_L[i] = (u64)L[i]; g_K[i] = (u64)K[i]; }
  g_full = (N >= 32) ? 0xFFFFFFFFu : ((1u << N) - 1u);
}

/* |T[P]|: T multiplied along every mode in P. */
static u64 tsize(unsigned P) {
  u64 s = 1;
  for (int n = 0; n < g_N; ++n) s *= ((P >> n) & 1u) ? g_K[n] : g_L[n];
  return s;
}

static int popc(unsigned x) { int c = 0; while (x) { x &= x - 1; ++c; } return c; }

/* Node cost of a TTM along mode m applied to T[P]: Sec. 3.1's multiply-adds
 * K_m * |T[P]|, or (g_cost_elems) the elements the node moves, its input read
 * and its output written, |T[P]| + |T[P + m]|. */
static int g_cost_elems;
static u64 node_cost(unsigned P, int m) {
  if (g_cost_elems) return tsize(P) + tsize(P | (1u << m));
  return g_K[m] * tsize(P);
}

/* ------------------------------------------------------------------------ */
/* Brute-force enumeration of all TTM-trees.                                 */
/* ------------------------------------------------------------------------ */
typedef struct { unsigned P, Q; } task_t;
static task_t g_tasks[256];
static u64 g_count, g_min, g_max;

static void enum_tasks(int nt, u64 cost);

/* Node with tensor T[P] must produce the leaves of Qrem (plus blocks already
 * chosen).  Children form a set partition of Q: the block holding the lowest
 * remaining mode is chosen first, so each partition is produced once.  A block
 * B is a leaf if B = {n} and P = all \ {n}; otherwise a child labelled m with
 * m outside P and outside B (mode m then lies on the path of every leaf in B). */
static void expand(unsigned P, unsigned Qrem, int nt, u64 cost) {
  if (Qrem == 0) { enum_tasks(nt, cost); return; }
  const unsigned low = Qrem & (~Qrem + 1u);
  const unsigned rest = Qrem & ~low;
  /* iterate over all subsets S of rest */
  unsigned S = 0;
  for (;;) {
    const unsigned B = low | S;
    const unsigned remain = rest & ~S;
    if (popc(B) == 1 && P == (g_full & ~B)) expand(P, remain, nt, cost);
    const unsigned avail = g_full & ~(P | B);
    for (int m = 0; m < g_N; ++m) {
      if (!((avail >> m) & 1u)) continue;
      g_tasks[nt].P = P | (1u << m);
      g_tasks[nt].Q = B;
      expand(P, remain, nt + 1, cost + node_cost(P, m));
    }
    if (S == rest) break;
    S = (S - rest) & rest; /* next subset of rest */
  }
}

static void enum_tasks(int nt, u64 cost) {
  if (nt == 0) {
    ++g_count;
    if (cost < g_min) g_min = cost;
    if (cost > g_max) g_max = cost;
    return;
  }
  const task_t t = g_tasks[nt - 1];
  expand(t.P, t.Q, nt - 1, cost);
  g_tasks[nt - 1] = t; /* expand() reuses this slot; the caller still needs it */
}

/* Enumerates every TTM-tree; returns the number of trees and the min / max
 * cost over them.  Feasible for N <= 5 (N = 5 has tens of millions). */
int orc_tree_bruteforce_model(int N, const int64_t* L, const int64_t* K, int elems, u64* n_trees,
                              u64* min_cost, u64* max_cost) {
  if (N < 2 || N > 6) return -1;
  set_problem(N, L, K);
  g_cost_elems = elems;
  g_count = 0; g_min = ORC_INF; g_max = 0;
  expand(0u, g_full, 0, 0);
  g_cost_elems = 0;
  *n_trees = g_count; *min_cost = g_min; *max_cost = g_max;
  return 0;
}

/* The same in multiply-adds (Sec. 3.1's cost). */
int orc_tree_bruteforce(int N, const int64_t* L, const int64_t* K, u64* n_trees, u64* min_cost,
                        u64* max_cost) {
  return orc_tree_bruteforce_model(N, L, K, 0, n_trees, min_cost, max_cost);
}

/* ------------------------------------------------------------------------ */
/* Top-down memoised recurrence of Sec. 3.3.                                 */
/* ------------------------------------------------------------------------ */
static u64* g_memo;
static int g_greedy; /* 1: "always reuse when R != {}" (the Remark's wrong rule) */

static u64 dp_rec(unsigned P, unsigned Q) {
  const size_t key = ((size_t)P << g_N) | Q;
  if (g_memo[key] != ORC_INF) return g_memo[key];
  const unsigned R = g_full & ~(P | Q);
  u64 best = ORC_INF;
  if (popc(Q) == 1 && R == 0) {
    best = 0; /* base case: the leaf F~_n */
  } else {
    for (int m = 0; m < g_N; ++m) { /* reuse */
      if (!((R >> m) & 1u)) continue;
      const u64 sub = dp_rec(P | (1u << m), Q);
      if (sub == ORC_INF) continue;
      const u64 c = g_K[m] * tsize(P) + sub;
      if (c < best) best = c;
    }
    if (popc(Q) >= 2 && !(g_greedy && R != 0)) { /* split */
      const unsigned low = Q & (~Q + 1u);
      const unsigned rest = Q & ~low;
      unsigned S = 0;
      for (;;) {
        const unsigned Q1 = low | S, Q2 = Q & ~Q1;
        if (Q2 != 0) {
          const u64 a = dp_rec(P, Q1), b = dp_rec(P, Q2);
          if (a != ORC_INF && b != ORC_INF && a + b < best) best = a + b;
        }
        if (S == rest) break;
        S = (S - rest) & rest;
      }
    }
  }
  g_memo[key] = best;
  return best;
}

/* Optimal tree cost by the recurrence; greedy != 0 forbids splitting while a
 * reusable mode exists (the rule the paper's Remark shows to be wrong). */
u64 orc_tree_dp(int N, const int64_t* L, const int64_t* K, int greedy) {
  if (N < 1 || N > 10) return ORC_INF;
  set_problem(N, L, K);
  g_greedy = greedy;
  const size_t sz = (size_t)1 << (2 * N);
  g_memo = (u64*)malloc(sizeof(u64) * sz);
  for (size_t i = 0; i < sz; ++i) g_memo[i] = ORC_INF;
  const u64 r = dp_rec(0u, g_full);
  free(g_memo);
  g_memo = NULL;
  return r;
}

/* ------------------------------------------------------------------------ */
/* Prior schemes of Sec. 3.2.                                                */
/* ------------------------------------------------------------------------ */
/* Chain tree with mode ordering `order` (a permutation of 0..N-1). */
u64 orc_chain_cost(int N, const int64_t* L, const int64_t* K, const int* order) {
  set_problem(N, L, K);
  u64 total = 0;
  for (int n = 0; n < N; ++n) {
    unsigned P = 0;
    for (int i = 0; i < N; ++i) {
      const int m = order[i];
      if (m == n) continue;
      total += g_K[m] * tsize(P);
      P |= 1u << m;
    }
  }
  return total;
}

/* Balanced tree: modes S (in the given order) split into the first floor(|S|/2)
 * and the rest; a chain of the first group then the recursive tree of the
 * second, and the same with the roles swapped. */
static u64 balanced_rec(unsigned P, const int* modes, int cnt) {
  if (cnt == 1) return 0;
  const int m = cnt / 2;
  u64 total = 0;
  for (int side = 0; side < 2; ++side) {
    const int* g1 = side == 0 ? modes : modes + m;
    const int n1 = side == 0 ? m : cnt - m;
    const int* g2 = side == 0 ? modes + m : modes;
    const int n2 = side == 0 ? cnt - m : m;
    unsigned Pc = P;
    for (int i = 0; i < n1; ++i) {
      total += g_K[g1[i]] * tsize(Pc);
      Pc |= 1u << g1[i];
    }
    total += balanced_rec(Pc, g2, n2);
  }
  return total;
}

u64 orc_balanced_cost(int N, const int64_t* L, const int64_t* K, const int* order) {
  set_problem(N, L, K);
  int modes[16];
  for (int i = 0; i < N; ++i) modes[i] = order ? order[i] : i;
  return balanced_rec(0u, modes, N);
}

/* Checks that a tree given as (label, parent) arrays is a TTM-tree per
 * Sec. 3.1 and returns its cost.  label[i] = mode for an internal node,
 * -1 for the root, -(n + 2) for the leaf of F~_n.  parent[i] = -1 for the root.
 * Returns ORC_INF if any property fails. */
static u64 tree_cost_impl(int N, const int64_t* L, const int64_t* K, int n_nodes, const int* label,
                          const int* parent) {
  set_problem(N, L, K);
  int root = -1, leaves = 0;
  unsigned leaf_seen = 0;
  for (int i = 0; i < n_nodes; ++i) {
    if (parent[i] < 0) {
      if (root >= 0 || label[i] != -1) return ORC_INF;
      root = i;
    } else if (parent[i] >= n_nodes || parent[i] == i) {
      return ORC_INF;
    }
  }
  if (root < 0) return ORC_INF;
  u64 total = 0;
  for (int i = 0; i < n_nodes; ++i) {
    if (i == root) continue;
    /* walk to the root collecting the modes on the path (excluding i) */
    unsigned P = 0;
    int steps = 0, cur = parent[i];
    while (cur != root) {
      if (cur < 0 || ++steps > n_nodes) return ORC_INF;
      const int lb = label[cur];
      if (lb < 0 || lb >= N) return ORC_INF; /* ancestors must be internal */
      if ((P >> lb) & 1u) return ORC_INF;    /* a mode twice on one path */
      P |= 1u << lb;
      cur = parent[cur];
    }
    if (label[i] >= 0) {
      const int m = label[i];
      if (m >= N || ((P >> m) & 1u)) return ORC_INF;
      total += node_cost(P, m);
    } else if (label[i] <= -2) {
      const int n = -label[i] - 2;
      if (n >= N || ((leaf_seen >> n) & 1u)) return ORC_INF;
      if (P != (g_full & ~(1u << n))) return ORC_INF;
      leaf_seen |= 1u << n;
      ++leaves;
    } else {
      return ORC_INF;
    }
  }
  /* leaves must be exactly N, and every internal node must lead to a leaf */
  if (leaves != N || leaf_seen != g_full) return ORC_INF;
  for (int i = 0; i < n_nodes; ++i) {
    if (label[i] < 0) continue;
    int has_child = 0;
    for (int j = 0; j < n_nodes; ++j) if (parent[j] == i) { has_child = 1; break; }
    if (!has_child) return ORC_INF;
  }
  return total;
}

u64 orc_tree_cost(int N, const int64_t* L, const int64_t* K, int n_nodes, const int* label,
                  const int* parent) {
  return tree_cost_impl(N, L, K, n_nodes, label, parent);
}

/* The cost of a given tree in elements moved (elems != 0) or multiply-adds. */
u64 orc_tree_cost_model(int N, const int64_t* L, const int64_t* K, int n_nodes, const int* label,
                        const int* parent, int elems) {
  g_cost_elems = elems;
  const u64 c = tree_cost_impl(N, L, K, n_nodes, label, parent);
  g_cost_elems = 0;
  return c;
}

/* ------------------------------------------------------------------------ */
/* STHOSVD mode order (Sec. 1 notes that the tree ideas carry over to it).  */
/* ------------------------------------------------------------------------ */
/* Cost of STHOSVD with the modes in `order`.  Step i takes mode m = order[i]
 * of the current tensor Y (modes order[0..i-1] already truncated to K):
 *   elems == 0: multiply-adds.  The Gram Y_(m) Y_(m)^T has L_m * L_m entries,
 *               each a sum of |Y| / L_m products: L_m * |Y|; the TTM
 *               Y x_m F_m^T costs K_m * |Y| (Sec. 3.1's node cost).
 *   elems != 0: elements moved.  The Gram reads Y (|Y|); the TTM reads Y and
 *               writes |Y| * K_m / L_m.
 * Returns ORC_INF when order is not a permutation of 0..N-1. */
u64 orc_sthosvd_order_cost(int N, const int64_t* L, const int64_t* K, const int* order, int elems) {
  set_problem(N, L, K);
  unsigned P = 0;
  u64 total = 0;
  for (int i = 0; i < N; ++i) {
    const int m = order[i];
    if (m < 0 || m >= N || ((P >> m) & 1u)) return ORC_INF;
    const u64 y = tsize(P);
    if (elems)
      total += y + y + tsize(P | (1u << m));
    else
      total += g_L[m] * y + g_K[m] * y;
    P |= 1u << m;
  }
  return total;
}

static int g_perm[16], g_best_perm[16];
static u64 g_best_cost, g_nat_cost;
static int g_elems;

static void perm_rec(int i, unsigned used) {
  if (i == g_N) {
    int64_t L[16], K[16];
    for (int n = 0; n < g_N; ++n) { L[n] = (int64_t)g_L[n]; K[n] = (int64_t)g_K[n]; }
    const u64 c = orc_sthosvd_order_cost(g_N, L, K, g_perm, g_elems);
    if (c < g_best_cost) {
      g_best_cost = c;
      memcpy(g_best_perm, g_perm, sizeof(int) * (size_t)g_N);
    }
    return;
  }
  for (int m = 0; m < g_N; ++m) {
    if ((used >> m) & 1u) continue;
    g_perm[i] = m;
    perm_rec(i + 1, used | (1u << m));
  }
}

/* Every order of the N modes (N! of them, lexicographic): the least cost, an
 * order reaching it (the lexicographically first), and the natural order's
 * cost. */
int orc_sthosvd_order_bruteforce(int N, const int64_t* L, const int64_t* K, int elems, int* best_order,
                                 u64* best_cost, u64* natural_cost) {
  if (N < 1 || N > 9) return -1;
  int nat[16];
  for (int n = 0; n < N; ++n) nat[n] = n;
  g_nat_cost = orc_sthosvd_order_cost(N, L, K, nat, elems);
  set_problem(N, L, K);
  g_elems = elems;
  g_best_cost = ORC_INF;
  perm_rec(0, 0u);
  memcpy(best_order, g_best_perm, sizeof(int) * (size_t)N);
  *best_cost = g_best_cost;
  *natural_cost = g_nat_cost;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* New-core chain order (Fig. 2 "New core": one chain over all N modes).    */
/* ------------------------------------------------------------------------ */
/* Multiply-adds of the chain T x_{order[0]} F^T x_{order[1]} F^T ...: step i
 * costs K_m * |T[P]| (Sec. 3.1's node cost), P the modes applied before it.
 * ORC_INF when order is not a permutation. */
u64 orc_core_chain_cost(int N, const int64_t* L, const int64_t* K, const int* order) {
  set_problem(N, L, K);
  unsigned P = 0;
  u64 total = 0;
  for (int i = 0; i < N; ++i) {
    const int m = order[i];
    if (m < 0 || m >= N || ((P >> m) & 1u)) return ORC_INF;
    total += g_K[m] * tsize(P);
    P |= 1u << m;
  }
  return total;
}

static u64 g_chain_best;

static void chain_perm_rec(int i, unsigned used, int* perm, const int64_t* L, const int64_t* K) {
  if (i == g_N) {
    const u64 c = orc_core_chain_cost(g_N, L, K, perm); /* re-sets the same problem */
    if (c < g_chain_best) g_chain_best = c;
    return;
  }
  for (int m = 0; m < g_N; ++m) {
    if ((used >> m) & 1u) continue;
    perm[i] = m;
    chain_perm_rec(i + 1, used | (1u << m), perm, L, K);
  }
}

/* Least chain cost over all N! orders. */
u64 orc_core_chain_bruteforce(int N, const int64_t* L, const int64_t* K) {
  if (N < 1 || N > 9) return ORC_INF;
  int perm[16];
  set_problem(N, L, K);
  g_chain_best = ORC_INF;
  chain_perm_rec(0, 0u, perm, L, K);
  return g_chain_best;
}
