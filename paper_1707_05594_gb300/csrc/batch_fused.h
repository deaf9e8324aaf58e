// batch_fused.h -- arguments of the fused batched sweep (batch_fused.cu),
// filled by the batch planner (batch.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace tk {

// One tensor's work in the fused tables (indices into them).
struct BFusedTensor {
  int32_t node0, nnodes;  // its tree nodes, parents before children
  int32_t gram0, ngram;   // its leaf Gram tiles
};

struct BFusedArgs {
  const BFusedTensor* work;  // [count]
  const int* order;          // tensors by decreasing size: the queue's order
  int count, N, KB;
  const void* nodes;         // tree nodes (BNode), staged flags set
  const void* cores;         // core node of each tensor (BNode) [count]
  const void* grams;         // leaf Gram tiles (BGram)
  const void* steps;         // reconstruction steps (BExp) [N][count]
  const EigDesc* eigs;       // [N][count], F / F0 as byte offsets
  char* f_base;              // F_out
  const char* f0_base;       // F_in
  const float* T;
  const float* F;            // F_in (element offsets of the nodes)
  float* inter;              // tree intermediates
  float* fit_inter;          // reconstruction intermediates (their own region)
  float* G;                  // cores of F_in
  double* gram;
  const double* normT2;
  double* fit;
  int* cold;                 // full-path list: cold[0] = count, cold[1 ..]
  int* queue;                // [0] next tensor, [1] CTAs done, [2] tensors done
  int* status;               // the library's device error word
  double tol;                // the warm start's subspace check
};

// Dynamic shared memory the fused kernel needs for matrices up to maxL x maxK.
size_t batch_fused_smem(int maxL, int maxK);
int launch_batch_fused(const BFusedArgs& a, int maxL, int maxK, cudaStream_t s);
// The full eigensolver path over the matrices the warm start's check listed
// in dev's cold list (no work when the list is empty).
int launch_eig_cold_path(const EigDesc* dev, int count, int maxL, int maxK, char* f_base,
                         const char* f0_base, int* cold, cudaStream_t s);

}  // namespace tk
