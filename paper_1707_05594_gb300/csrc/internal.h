// internal.h -- host-side structures shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tucker.h"

namespace tk {

constexpr int kMaxModes = TUCKER_MAX_MODES;
constexpr size_t kAlign = 256;

inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

// One node of the TTM-tree (Sec. 3.1).  `P` is the set of modes multiplied on
// the path from the root down to and including this node, so Out(u) = T[P].
struct PlanNode {
  int label = -1;   // mode for internal nodes, -1 root, -(n+2) leaf of F~_n
  int parent = -1;
  unsigned P = 0;
  int64_t out_dims[kMaxModes] = {};
  uint64_t in_elems = 0, out_elems = 0, macs = 0;
  size_t ws_off = 0;  // byte offset of Out(u) in the workspace (internal nodes)
};

struct Plan {
  int N = 0;
  int64_t L[kMaxModes] = {}, K[kMaxModes] = {};
  int dtype = TUCKER_F32;
  int tree = TUCKER_TREE_OPTIMAL;
  int cost_model = TUCKER_COST_MACS;
  std::vector<PlanNode> nodes;  // depth-first pre-order, nodes[0] is the root
  // fused root: the first two root children (node indices, DFS order) are
  // computed together from one read of T when the first one is reached; the
  // second one's buffer is placed after the first one's whole subtree
  int fused_u1 = -1, fused_u2 = -1;
  uint64_t tree_macs = 0, tree_elems = 0;
  std::vector<int> core_order;  // mode order of the new-core chain
  uint64_t core_macs = 0;
  std::vector<int> sth_order;   // mode order of tucker_sthosvd
  uint64_t sth_cost = 0;        // its cost under cost_model (Gram + TTM per step)

  // workspace layout (byte offsets)
  size_t off_scratch = 0, bytes_scratch = 0;  // tree intermediates / chains
  size_t off_gram[kMaxModes] = {};            // FP64 L_n x L_n
  size_t off_eig = 0, bytes_eig = 0;          // eigensolver scratch
  size_t off_misc = 0;                        // small device scalars
  size_t ws_total = 0;

  // per-node CUDA-event timing (opaque cudaEvent_t pairs; see tucker_profile_*)
  int prof_cap = 0, prof_n = 0;
  std::vector<void*> prof_events;  // 2 * prof_cap events
  std::vector<int> prof_node, prof_label;

  size_t elem_bytes() const {  // bytes of T per element (hi + lo for the split type)
    return dtype == TUCKER_F64 ? 8 : (dtype == TUCKER_BF16 ? 2 : (dtype == TUCKER_FP8_E4M3 ? 1 : 4));
  }
  // tree intermediates: FP64 for FP64 tensors, BF16 for BF16 and FP8 tensors
  // (the precision forms), FP32 otherwise
  int inter_dtype() const {
    return dtype == TUCKER_F64 ? TUCKER_F64
                               : ((dtype == TUCKER_BF16 || dtype == TUCKER_FP8_E4M3) ? TUCKER_BF16
                                                                                     : TUCKER_F32);
  }
  size_t inter_bytes() const {
    return dtype == TUCKER_F64 ? 8 : ((dtype == TUCKER_BF16 || dtype == TUCKER_FP8_E4M3) ? 2 : 4);
  }
};

// whether the fused root TTM (ttm_fused_root.cu) takes the two root children of
// modes a < b of a tensor of this type and these lengths
bool fused_root_fits(int dtype, int N, const int64_t* L, const int64_t* K, int a, int b);
// whether a sweep computes the root children of modes a < b together: the
// fused kernel above, or (FP32 tensors, b = a + 2) the tensor-core pair that
// reads T once, blocked by mode a + 1 so that the second mode's tiles find
// each block in L2
bool root_pair_fits(int dtype, int N, const int64_t* L, const int64_t* K, int a, int b);

// byte offset of the lo half in a split BF16 tensor of n elements
inline size_t bf16_split_lo_offset(int64_t n) { return align_up((size_t)n * 2); }
// whether the tensor-core TTM reads a split BF16 tensor of this [R][L][C]
// view with K outputs (shape, alignment-free part, and shared memory)
bool ttm_tc_split_fits(int64_t R, int64_t L, int64_t C, int64_t K);

// thread-local error text
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

uint64_t tensor_size(const Plan& p, unsigned P);

// eigensolver scratch of one L x L matrix with K wanted vectors: V0 (L*K
// floats), theta (K floats), parked reflectors (L*L floats), Q, Y and the
// previous basis Qp (L*K doubles each), warm-start status (64 bytes)
constexpr size_t eig_bytes_per_matrix(size_t l, size_t k) {
  return ((l * k * 4 + kAlign - 1) / kAlign * kAlign) + ((k * 4 + kAlign - 1) / kAlign * kAlign) +
         ((l * l * 4 + kAlign - 1) / kAlign * kAlign) + 3 * ((l * k * 8 + kAlign - 1) / kAlign * kAlign) +
         kAlign;
}

// sizes of the eigensolver scratch for a batch of matrices (256 bytes for the
// list of matrices sent to the full path, then eig_bytes_per_matrix each)
size_t eig_ws_bytes(int batch, const int64_t* L, const int64_t* K);

// releases the plan's profiling events (defined with the executor)
void destroy_profile(Plan& p);

// number of kernels this library has launched (all threads)
void count_launches(uint64_t n);

}  // namespace tk

struct tucker_plan_s {
  tk::Plan p;
};
