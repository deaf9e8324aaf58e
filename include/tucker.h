/*
 * tucker.h -- C ABI of the GB300 (sm_103a) dense Tucker / HOOI library.
 *
 * The library computes, on one GPU, the STHOSVD initial decomposition and the
 * HOOI procedure of Chakaravarthy et al., "On Optimizing Distributed Tucker
 * Decomposition for Dense Tensors" (arXiv 1707.05594), whose TTM component is
 * executed along the optimal TTM-tree of the paper's Sec. 3.3.
 *
 * Conventions shared by every call
 *   - A tensor of size L_0 x ... x L_{N-1} is dense, row-major (C order, mode
 *     N-1 fastest), contiguous, in device memory.  Modes are numbered from 0
 *     (the paper counts them 1..N).
 *   - Factor F_n is an L_n x K_n row-major matrix with orthonormal columns
 *     (Sec. 2.2); the core G is K_0 x ... x K_{N-1} row-major.
 *   - Element types: the plan's storage type fixes the type of T; factors and
 *     core are double for TUCKER_F64 and float otherwise.
 *   - Pointer arrays (F_in, F_out, ...) are HOST arrays of N DEVICE pointers.
 *   - Every call that takes a stream is asynchronous on it.  The caller owns
 *     all device buffers and the stream; the library owns plans.
 *   - The workspace `ws` is caller-provided device memory of at least
 *     tucker_plan_cost()'s ws_bytes, 256-byte aligned; one workspace must not
 *     be used by two calls that may overlap on the GPU.
 *   - Return value: TUCKER_OK (0) or a negative TUCKER_ERR_* code; the text of
 *     the last error of the calling thread is returned by tucker_last_error().
 *     No C++ exception crosses this boundary.  Arguments are validated on the
 *     host before anything is launched.
 */
#ifndef TUCKER_GB300_H
#define TUCKER_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TUCKER_OK 0
#define TUCKER_ERR_INVALID_ARG (-1)
#define TUCKER_ERR_UNSUPPORTED (-2)
#define TUCKER_ERR_WORKSPACE (-3)
#define TUCKER_ERR_CUDA (-4)
#define TUCKER_ERR_TIMEOUT (-5)
#define TUCKER_ERR_NONFINITE (-6)
#define TUCKER_ERR_INCOMPLETE (-7) /* device error word: a fused batched sweep ended with tensors untaken */

#define TUCKER_MAX_MODES 8

/* Storage type of the input tensor T. */
typedef enum {
  TUCKER_F32 = 0,  /* float32; factors/core float32                        */
  TUCKER_F64 = 1,  /* float64; factors/core float64                        */
  TUCKER_BF16 = 2, /* bfloat16 (raw uint16 bits); factors/core float32     */
  TUCKER_FP8_E4M3 = 3, /* FP8 E4M3 codes + one float32 scale per 64 elements */
                       /* (layout at tucker_fp8_bytes); factors/core float32 */
  TUCKER_BF16_SPLIT = 4 /* an FP32 tensor stored as two BF16 tensors hi + lo   */
                        /* (layout at tucker_bf16_split_bytes); factors/core   */
                        /* and tree intermediates float32                      */
} tucker_dtype_t;

/* Which TTM-tree the plan executes (Sec. 3.2 / 3.3). */
typedef enum {
  TUCKER_TREE_OPTIMAL = 0,  /* DP of Sec. 3.3 (min cost)                  */
  TUCKER_TREE_CHAIN = 1,    /* N independent chains, natural mode order  */
  TUCKER_TREE_CHAIN_K = 2,  /* chains, modes by increasing K_n           */
  TUCKER_TREE_CHAIN_H = 3,  /* chains, modes by increasing K_n / L_n     */
  TUCKER_TREE_BALANCED = 4  /* Kaya-Ucar balanced tree                   */
} tucker_tree_t;

/* Node cost the optimal-tree DP minimises. */
typedef enum {
  TUCKER_COST_MACS = 0,  /* the paper's computational load K_n*|In(u)|   */
  TUCKER_COST_ELEMS = 1  /* elements moved |In(u)| + |Out(u)|            */
} tucker_cost_t;

typedef struct {
  int32_t dtype;      /* tucker_dtype_t, storage type of T               */
  int32_t tree;       /* tucker_tree_t                                   */
  int32_t cost_model; /* tucker_cost_t (only for TUCKER_TREE_OPTIMAL)    */
  int32_t flags;      /* TUCKER_PLAN_* bits, 0 by default                */
  uint64_t ws_cap;    /* workspace cap in bytes, 0 for none (see below)  */
} tucker_plan_opts_t;
/* Workspace cap: when ws_cap > 0 and the plan's workspace would exceed it,
 * tucker_plan gives up, in this order, the fused root (the second root
 * child's buffer, live through the first child's subtree) and then the
 * least-cost STHOSVD order (TUCKER_PLAN_STHOSVD_ORDER; its ping-pong buffers
 * can be larger than the natural order's) -- tucker_plan_fused_root and
 * tucker_plan_sthosvd report what the plan kept -- and returns
 * TUCKER_ERR_WORKSPACE, with the smallest size it reached in the error text,
 * when the cap still cannot be met.  The tree itself (and so every sweep's
 * result) never changes with the cap.  Zero-initialise the whole struct. */

/* Plan flag: never fuse the root.  By default, when the first two root
 * children of the tree (modes a < b) are both TTM nodes, T is FP32 or BF16,
 * the trailing block of T from mode a on (L_a * ... * L_{N-1} elements) fits
 * in 8 KB and K_a, K_b <= 32, a sweep computes both children from one read of
 * T (one kernel that stages each block in shared memory and contracts it
 * along a and along b); when the plan is made under the kernel-policy bits
 * for the tensor-core pairs (see tucker_set_kernel_policy) and b = a + 2,
 * one tensor-core kernel computes both children of an FP32 or BF16 tensor,
 * running through T block by block of mode a + 1 (each block read from HBM
 * once and found in L2 by the second mode's tiles).  The second child's buffer then sits after the first
 * child's subtree (see ws_offset), which can enlarge the workspace.  Results
 * are those of the two separate TTMs (the same bits). */
#define TUCKER_PLAN_NO_FUSED_ROOT 1

/* Plan flag: let tucker_sthosvd take the modes in the order of least cost
 * instead of 0, 1, ..., N-1 (Sec. 1 notes that the tree ideas carry over to
 * STHOSVD).  The step on mode m of the current tensor Y costs L_m*|Y| (its
 * Gram) + K_m*|Y| (its TTM) multiply-adds, or 2*|Y| + |Y|*K_m/L_m elements
 * moved under TUCKER_COST_ELEMS; the order minimising the sum is found by a
 * DP over the set of modes already truncated, the natural order being kept
 * whenever it is optimal.  A different order gives different (equally valid)
 * STHOSVD factors; see tucker_plan_sthosvd. */
#define TUCKER_PLAN_STHOSVD_ORDER 2

typedef struct tucker_plan_s* tucker_plan_t;

/* One node of a plan's TTM-tree, in depth-first pre-order (root first).
 * label: mode n (0-based) for an internal node (Out = In x_n F_n^T), -1 for
 * the root, -(n+2) for the leaf that yields the new factor F~_n.
 * parent: index of the parent node, -1 for the root.
 * in_elems / out_elems: |In(u)|, |Out(u)|; macs: K_n*|In(u)| (0 for root and
 * leaves); ws_offset: byte offset of Out(u) inside the workspace (internal
 * nodes only, else 0). */
typedef struct {
  int32_t label;
  int32_t parent;
  uint64_t in_elems;
  uint64_t out_elems;
  uint64_t macs;
  uint64_t ws_offset;
} tucker_node_t;

/* Builds a plan for tensor lengths L[0..N-1] and core lengths K[0..N-1]
 * (Sec. 5: the planner needs only this metadata; the plan is reused by every
 * sweep).  Host only, no device work.  Validation: 2 <= N <= 8,
 * 1 <= K_n <= L_n, K_n <= prod_{j != n} K_j (else Z_(n) has rank < K_n),
 * prod L_n < 2^40.  opts may be NULL (F32, optimal tree, MAC cost, no cap). */
int tucker_plan(int N, const int64_t* L, const int64_t* K, const tucker_plan_opts_t* opts,
                tucker_plan_t* out);

/* Per-sweep figures of the plan.  tree_macs: cost of the TTM-tree in the
 * paper's unit (Sec. 3.1); tree_elems: elements read + written by its nodes;
 * core_macs: the new-core TTM chain; ws_bytes: workspace every call of this
 * plan needs.  Any output pointer may be NULL. */
int tucker_plan_cost(tucker_plan_t plan, uint64_t* tree_macs, uint64_t* tree_elems,
                     uint64_t* core_macs, size_t* ws_bytes);

/* Copies at most `capacity` nodes of the plan's tree (see tucker_node_t) and
 * sets *n_nodes to the total count.  nodes may be NULL to query the count. */
int tucker_plan_nodes(tucker_plan_t plan, tucker_node_t* nodes, int capacity, int* n_nodes);

/* The fused root of a plan: *first and *second = the node indices of the two
 * root children computed together (first in depth-first order), or -1 and -1
 * when the root is not fused.  Host only. */
int tucker_plan_fused_root(tucker_plan_t plan, int* first, int* second);

/* The mode order tucker_sthosvd takes (Sec. 1: the tree ideas carry over to
 * STHOSVD): writes N mode indices to order (caller-owned host array) and, if
 * cost is not NULL, the order's cost under the plan's cost model (see
 * TUCKER_PLAN_STHOSVD_ORDER).  Natural order unless the plan was made with
 * that flag.  Host only; TUCKER_ERR_INVALID_ARG if plan or order is NULL. */
int tucker_plan_sthosvd(tucker_plan_t plan, int* order, uint64_t* cost);

void tucker_plan_destroy(tucker_plan_t plan);

/* STHOSVD initial decomposition (Sec. 2.2 cites it): for n in the plan's
 * STHOSVD order (natural unless TUCKER_PLAN_STHOSVD_ORDER),
 * F_n <- leading K_n eigenvectors of Y_(n) Y_(n)^T and Y <- Y x_n F_n^T,
 * starting from Y = T; G <- Y (K_0 x ... x K_{N-1} whatever the order).
 * F: N device pointers. */
int tucker_sthosvd(tucker_plan_t plan, const void* T, void* const* F, void* G, void* ws,
                   size_t ws_bytes, void* stream);

/* One HOOI invocation (Fig. 2) along the plan's TTM-tree: for every mode n,
 * Z_n = T x_{j != n} F_in[j]^T (input factors for every chain), then
 * F_out[n] <- leading K_n left singular vectors of Z_(n), computed as the
 * leading eigenvectors of the Gram Z_(n) Z_(n)^T (Sec. 5).  Eigenvectors are
 * ordered by decreasing eigenvalue, and each column's entry of largest
 * magnitude is positive.  F_out may not alias F_in. */
int tucker_hooi_sweep(tucker_plan_t plan, const void* T, const void* const* F_in,
                      void* const* F_out, void* ws, size_t ws_bytes, void* stream);

/* tucker_hooi_sweep that also writes G_in = T x_0 F_in[0]^T ... x_{N-1}
 * F_in[N-1]^T, the core of the INPUT factors (Fig. 2's new core, formed for
 * F_in), at the cost of one small TTM: the input of the tree's smallest leaf
 * is already T x_{j != n} F_in[j]^T, so G_in = that x_n F_in[n]^T.  Run in a
 * loop, sweep s+1 therefore yields the core (and with tucker_fit the error) of
 * sweep s's factors; the last sweep's core needs one tucker_core.  G_in may be
 * NULL (then this is tucker_hooi_sweep). */
int tucker_hooi_sweep_core(tucker_plan_t plan, const void* T, const void* const* F_in,
                           void* const* F_out, void* G_in, void* ws, size_t ws_bytes,
                           void* stream);

/* One HOOI sweep in the Gauss-Seidel form (the standard HOOI of Kolda and
 * Bader, against which Sec. 3 describes its Jacobi form, Fig. 2): for
 * n = 0 .. N-1, Z_n = T x_{m != n} F_m^T with F_out[m] for m < n (already
 * updated this sweep) and F_in[m] for m > n, along the plan's core-chain order
 * without n; F_out[n] = the leading K_n eigenvectors of Z_(n) Z_(n)^T (warm-
 * started from F_in[n]).  No TTM-tree: each mode needs its own chain.  G_out
 * (if not NULL) receives the core of F_out.  F_out may not alias F_in. */
int tucker_hooi_sweep_gs(tucker_plan_t plan, const void* T, const void* const* F_in,
                         void* const* F_out, void* G_out, void* ws, size_t ws_bytes, void* stream);

/* New core (Fig. 2): G = T x_0 F_0^T ... x_{N-1} F_{N-1}^T, with the chain's
 * mode order chosen to minimise multiply-adds. */
int tucker_core(tucker_plan_t plan, const void* T, const void* const* F, void* G, void* ws,
                size_t ws_bytes, void* stream);

/* ||T||_F^2 accumulated in double, written to the device double *out. */
int tucker_norm2(tucker_plan_t plan, const void* T, double* out, void* stream);

/* Synchronous finiteness check of n elements of type dtype at X (a tensor,
 * factor or core): returns TUCKER_ERR_NONFINITE when any is NaN or Inf (their
 * sum of squares is not finite), TUCKER_OK otherwise.  Allocates nothing;
 * waits for `stream`.  Concurrent calls from several host threads run one
 * after another. */
int tucker_check_finite(const void* X, int dtype, int64_t n, void* stream);

/* Error metric of Sec. 2.2 ("normalized root mean square"), using
 * ||T - G x F||^2 = ||T||^2 - ||G||^2 for orthonormal factors:
 * out[0] = fit = 1 - sqrt(max(0, normT2 - ||G||^2)) / sqrt(normT2),
 * out[1] = ||G||^2.  normT2 and out are device pointers (out: 2 doubles). */
int tucker_fit(tucker_plan_t plan, const void* G, const double* normT2, double* out,
               void* stream);

/* Single mode-n TTM (Sec. 2.1) Y = X x_n F^T for an X of lengths dims[0..N-1]
 * of type x_dtype; F is dims[n] x K row-major (double for TUCKER_F64, else
 * float); Y has dims with dims[n] replaced by K and type double for
 * TUCKER_F64, else float.  Exposed for testing the TTM kernels. */
int tucker_ttm(int N, const int64_t* dims, const void* X, int x_dtype, int n, const void* F,
               int64_t K, void* Y, void* stream);

/* Two TTMs of one tensor from a single read of it (the fused root of a
 * sweep): Ya = X x_a Fa^T and Yb = X x_b Fb^T for modes a < b, with Fa
 * dims[a] x Ka and Fb dims[b] x Kb row-major float, Ya and Yb laid out as
 * X with dims[a] (dims[b]) replaced by Ka (Kb).  x_dtype TUCKER_F32 (y_dtype
 * TUCKER_F32) or TUCKER_BF16 (y_dtype TUCKER_BF16 or TUCKER_F32).  Each
 * output is summed over its contracted mode in increasing order with FP32
 * fused multiply-adds.  TUCKER_ERR_UNSUPPORTED unless the trailing block
 * dims[a] * ... * dims[N-1] fits in 8 KB, Ka, Kb <= 32 and the factors fit in
 * shared memory (the conditions of the plan's fused root). */
int tucker_ttm_pair(int N, const int64_t* dims, const void* X, int x_dtype, int a, const float* Fa,
                    int64_t Ka, int b, const float* Fb, int64_t Kb, void* Ya, void* Yb, int y_dtype,
                    void* stream);

/* Gram W = Z_(n) Z_(n)^T (Sec. 5) of a tensor Z of lengths dims[0..N-1] and
 * type z_dtype; W is a dims[n] x dims[n] device double matrix (overwritten). */
int tucker_gram(int N, const int64_t* dims, const void* Z, int z_dtype, int n, double* W,
                void* stream);

/* Leading-K eigenvectors of `batch` symmetric matrices (Sec. 5's EVD step).
 * W[b]: L[b] x L[b] device doubles (read only); F[b]: L[b] x K[b] row-major
 * output of type f_dtype (TUCKER_F64: double, else float), columns ordered by
 * decreasing eigenvalue, sign as in tucker_hooi_sweep.  ws: device scratch of
 * at least tucker_eig_ws_bytes(batch, L, K) bytes.  Requires L[b] <= 200 and
 * K[b] <= min(L[b], 64) (else TUCKER_ERR_UNSUPPORTED); f_dtype must be
 * TUCKER_F32 or TUCKER_F64 (else TUCKER_ERR_INVALID_ARG). */
int tucker_eig_topk(int batch, const int64_t* L, const int64_t* K, const double* const* W,
                    void* const* F, int f_dtype, void* ws, size_t ws_bytes, void* stream);
size_t tucker_eig_ws_bytes(int batch, const int64_t* L, const int64_t* K);

/* Allocation-free variant of tucker_eig_topk (the paper has no counterpart:
 * this serves callers that must not allocate device memory, e.g. when all
 * device memory belongs to another allocator, or where cudaMalloc/cudaFree
 * could synchronise the device).  Same arguments, results and ordering as
 * tucker_eig_topk, but no workspace: the scratch is a fixed array of about
 * 4 MiB compiled into the library, held on every GPU that loads it until the
 * process exits.  Limits: batch <= 8, every L <= 200 and K <= min(L, 64);
 * larger problems return TUCKER_ERR_UNSUPPORTED; an f_dtype other than
 * TUCKER_F32 or TUCKER_F64 returns TUCKER_ERR_INVALID_ARG.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current and keeps it for the life of the process; make that
 * first call before any stream capture.  A cudaDeviceReset (or any teardown of
 * the device's primary context) invalidates the kept address: do not call this
 * entry point on that device afterwards.  All calls share
 * the one array: calls that may overlap on the GPU (different streams, or
 * different host threads) race on it and must be serialised by the caller.
 * The call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine). */
int tucker_eig_topk_noalloc(int batch, const int64_t* L, const int64_t* K, const double* const* W,
                            void* const* F, int f_dtype, void* stream);

/* Per-node CUDA-event timing of a plan's calls (tracing).  While enabled,
 * tucker_hooi_sweep records a start/end event pair on its stream around each
 * tree node's launches (node = index in tucker_plan_nodes order, label = its
 * mode, or -(n+2) for the Gram of leaf n) and around the batched eigensolver
 * (node = -1), tucker_core around each chain step (node = -2, label =
 * mode) and tucker_hooi_sweep_gs around each step of its chains (node = -3,
 * label = mode).  With a fused root the first root child's record covers
 * both children and the second one's is empty.  Recording stops when
 * `capacity` pairs are used.  capacity = 0 disables profiling and frees the
 * events. */
typedef struct {
  int32_t node;
  int32_t label;
  float ms;
} tucker_prof_rec_t;
int tucker_profile_enable(tucker_plan_t plan, int capacity);
/* Waits for the recorded events, copies at most `capacity` records (in
 * recording order), sets *n_recs to the number recorded, and empties the
 * ring.  recs may be NULL. */
int tucker_profile_read(tucker_plan_t plan, tucker_prof_rec_t* recs, int capacity, int* n_recs);

/* Number of kernels this library has launched in this process (all threads,
 * all plans); a monotone counter for accounting. */
uint64_t tucker_launch_count(void);

/* Storage conversion for the precision form: hi[i] = bf16(x[i]) rounded to
 * nearest even and, if lo is not NULL, lo[i] = bf16(x[i] - hi[i]), so that
 * hi + lo holds x to ~16 significand bits.  n elements; all three device
 * buffers 16-byte aligned; BF16 values are raw uint16 bit patterns. */
int tucker_convert_bf16(const float* x, uint16_t* hi, uint16_t* lo, int64_t n, void* stream);

/* FP8 storage (the FP8 variant of the precision form).  An FP8 tensor of n
 * elements occupies tucker_fp8_bytes(n) bytes: n E4M3 codes, then, from the
 * next 256-byte boundary, ceil(n / 64) float scales; element i stands for
 * scale[i / 64] * E4M3(code[i]).  tucker_convert_fp8 fills such a buffer from
 * n floats: per slab of 64 consecutive elements, scale = amax / 448 (1 for an
 * all-zero slab) and code = E4M3(x / scale), rounded to nearest even and
 * saturated; out must be 256-byte aligned.  Plans of type TUCKER_FP8_E4M3 run
 * sweeps, cores and norms on such a tensor (BF16 tree intermediates, FP32
 * factors); their STHOSVD returns TUCKER_ERR_UNSUPPORTED (run it on the FP32
 * tensor). */
size_t tucker_fp8_bytes(int64_t n);
int tucker_convert_fp8(const float* x, void* out, int64_t n, void* stream);

/* Split BF16 storage (the optional split first TTM of the precision form):
 * an FP32 tensor x of n elements held as hi = bf16(x) and lo = bf16(x - hi)
 * (tucker_convert_bf16), which keeps ~16 significant bits (|x - hi - lo| <=
 * 2^-18 |x|) at the 4 bytes per element of FP32.  One buffer of
 * tucker_bf16_split_bytes(n) bytes holds the n hi values, then, from byte
 * offset tucker_bf16_split_lo_offset(n) (the first 256-byte boundary at or
 * after 2n), the n lo values; the buffer itself 256-byte aligned.  Plans of
 * type TUCKER_BF16_SPLIT read such a T in every TTM whose input is T (Sec.
 * 2.1): on the tensor cores, each k-step issuing A_hi [F_hi | F_lo] and
 * A_lo F_hi, FP32 accumulation; their tree intermediates, factors and core
 * are FP32.  tucker_plan returns TUCKER_ERR_UNSUPPORTED for such a plan
 * unless every mode's TTM of T takes the tensor-core tile (mode not last: the
 * product of the later lengths a multiple of 8 and >= 64; last mode: its
 * length a multiple of 8; K_n <= 64) and its factor fits in shared memory;
 * STHOSVD and the Gram of T are not offered for this type (run them on the
 * FP32 tensor). */
size_t tucker_bf16_split_bytes(int64_t n);
size_t tucker_bf16_split_lo_offset(int64_t n);

/* Kernel selection, a bit mask (process-wide; 0 is the default):
 *   bit 0 (1): every TTM on the CUDA-core kernels (otherwise BF16 and FP8
 *              tensors use the tensor-core TTMs, tcgen05 + TMA, where the
 *              shape allows and they are faster);
 *   bit 1 (2): HOOI sweeps always run the full eigensolver (otherwise they start
 *              from the input factors: two FP64 subspace-iteration steps and an
 *              a-posteriori check, falling back to the full path on the GPU
 *              when the check fails);
 *   bit 2 (4): FP32 TTMs of the column case (mode not last, C >= 64) on the
 *              tensor cores: tiles and factor split into three BF16 parts,
 *              six products accumulated in TMEM (off by default: the
 *              accumulation is not the CUDA cores' exactly rounded FMA, which
 *              moves the fit identity ||T||^2 - ||G||^2 by ~1e-5 relative on
 *              low-noise tensors);
 *   bit 3 (8): no short-row kernels (otherwise FP32 and BF16 TTMs with short
 *              rows after mode n -- C == 1 with 256 rows in 32 KB, or
 *              1 < C < 64 -- and no tensor-core tile copy runs of whole slabs
 *              into shared memory by cp.async and multiply from there);
 *   bit 4 (16): BF16 TTMs on the tensor cores wherever the shape allows
 *              (otherwise column shapes whose tensor-core tiles would be less
 *              than 60 % useful -- l in stages of 64, 128 positions per tile
 *              -- run on the CUDA cores, which are faster there);
 *   bit 5 (32): FP32 TTMs of the column case with C % 4 == 0, C >= 64 and
 *              K <= 32 on the tensor cores with exact integer slices: per
 *              64-l chunk each position's values and each factor column are
 *              scaled by a power of two and cut into three 8-bit integer
 *              slices held in BF16, whose products and sums the tensor core
 *              forms without rounding; only the slicing and an FP32 epilogue
 *              round, so the result is as accurate as an FP32 contraction
 *              and unbiased (slower than the CUDA cores at present);
 *   bit 6 (64): those FP32 TTMs on the tensor cores in TF32 with split
 *              operands instead (x_hi f_hi + x_hi f_lo + x_lo f_hi; less conversion
 *              work, but the tensor core's FP32 accumulation rounds toward
 *              zero, which biases every output by ~1e-7 relative and the
 *              fit identity by ~1e-5 on the 1e-2-noise workloads);
 *   bit 7 (128): with bit 6, one accumulator per tile instead of one per
 *              64-l chunk summed in registers;
 *   bit 8 (256): BF16 plans made while it is set compute their two root
 *              children (modes a, a + 2) with the L2-blocked tensor-core pair
 *              (see TUCKER_PLAN_NO_FUSED_ROOT; FP32 plans do so under bits 5
 *              or 6).  Off by default: measured slower than two separate
 *              tensor-core TTMs on the 64^5 workload.
 *   bit 9 (512): FP32 Grams on the CUDA cores (otherwise Grams of FP32
 *              unfoldings with C % 4 == 0, C >= 16 and L <= 512 run on the
 *              tensor cores: TF32 with split operands, x_hi y_hi + x_hi y_lo +
 *              x_lo y_hi, one 32-column stage per accumulator, the stage sums
 *              added in FP32 registers and the block sums in FP64 -- as
 *              accurate as FP32 arithmetic; bit 0 also selects the CUDA cores).
 *   bit 10 (1024): the warm-started eigensolver keeps each matrix's
 *              orthonormalisations and Rayleigh-Ritz in one CTA (otherwise a
 *              batch of at most 8 matrices with L >= 64, as in a sweep of
 *              one tensor, runs them on a cluster of 8 CTAs per matrix, each
 *              summing an eighth of the rows; the results agree to rounding).
 * Bits 5, 6 and 8 are read by tucker_plan (the pair changes the plan's
 * buffer layout) and by the calls.  TUCKER_ERR_INVALID_ARG outside 0..2047. */
int tucker_set_kernel_policy(int policy);

/* Debug build: the library compiled with -DTUCKER_DEBUG
 * (paper_1707_05594_gb300/build.py, build(debug=True), which writes
 * libtucker_gb300_debug.so).  There every kernel that forms global indices
 * from tensor shapes -- the TTMs on CUDA and tensor cores (their epilogue
 * stores), the CUDA-core Gram, the FP8 TTMs, the fused root, the short-row
 * kernels and the batched form's tree, Gram and expansion kernels -- checks,
 * per thread and per array, the first and last element it will touch (the
 * accesses are affine in the loop indices, so the two ends bound all of
 * them) against the array's length; a range outside it is recorded (the
 * first: offending index, length, source file and line) and its accesses are
 * skipped.  Kernels whose every access is guarded by `i < n` in its own loop
 * (norms, conversions, the eigensolver's L x L work) carry no check.
 * tucker_debug_build returns 1 in the debug build and 0 otherwise. */
int tucker_debug_build(void);

/* Synchronous (waits for the device): the number of out-of-range ranges
 * recorded since the last reset -- always 0 in the normal build -- and the
 * first one's index, length, source line and file (file: file_len bytes,
 * NUL-terminated).  Any pointer may be NULL; reset != 0 clears the records.
 * TUCKER_ERR_CUDA when a record cannot be read. */
int tucker_debug_check(int64_t* index, int64_t* bound, int* line, char* file, int file_len, int reset);

/* Device error word of the tensor-core kernels: 0, or TUCKER_ERR_TIMEOUT if a
 * pipeline wait gave up (the kernel then returned early and its output is not
 * valid).  Synchronous; reset != 0 clears the word. */
int tucker_device_status(int* status, int reset);

/* ---- Batched form: many small independent tensors ------------------------
 * A batch holds `count` FP32 tensors with the same order N but their own
 * lengths dims[i*N + n] and core lengths ranks[i*N + n] (i = tensor).  Each
 * tensor is planned with its own optimal TTM-tree (Sec. 3.3); a sweep runs the
 * trees level by level, so it is a fixed short sequence of launches, each over
 * every tensor of the batch, that can be recorded once in a CUDA graph.  The
 * method per tensor is tucker_hooi_sweep_core's (Fig. 2): the result equals
 * running that call on every tensor in turn.
 *
 * Data are packed back to back (offsets in elements, from
 * tucker_batch_offsets): T holds tensor i at t_off[i] (row-major), F holds
 * factor n of tensor i (dims x ranks, row-major) at f_off[i*N + n], G holds
 * core i at g_off[i].  Factors, cores and tensors are float; normT2 and fit
 * are `count` doubles.  All of them are device buffers owned by the caller.
 *
 * Limits: every dims <= 200, every ranks <= 32 and <= the product of the
 * other ranks of its tensor, count * N <= 65535. */
typedef struct tucker_batch_s* tucker_batch_t;
/* Plans the batch (host only). */
int tucker_batch_plan(int count, int N, const int64_t* dims, const int64_t* ranks,
                      tucker_batch_t* out);
/* Workspace bytes and the total element counts of T, F and G (any NULL). */
int tucker_batch_info(tucker_batch_t b, size_t* ws_bytes, int64_t* t_elems, int64_t* f_elems,
                      int64_t* g_elems);
/* Element offsets: t_off[count], f_off[count*N], g_off[count] (any NULL). */
int tucker_batch_offsets(tucker_batch_t b, int64_t* t_off, int64_t* f_off, int64_t* g_off);
void tucker_batch_destroy(tucker_batch_t b);
/* Uploads the batch's work tables into `ws` (synchronises `stream`).  Every
 * later call of this batch must pass the same workspace. */
int tucker_batch_prepare(tucker_batch_t b, void* ws, size_t ws_bytes, void* stream);
/* STHOSVD of every tensor (natural mode order, as tucker_sthosvd): writes F
 * and G. */
int tucker_batch_sthosvd(tucker_batch_t b, const float* T, float* F, float* G, void* ws,
                         size_t ws_bytes, void* stream);
/* One HOOI sweep of every tensor: F_out from F_in, and G_in (if not NULL) the
 * core of the input factors, as tucker_hooi_sweep_core.  F_out may not alias
 * F_in. */
int tucker_batch_sweep(tucker_batch_t b, const float* T, const float* F_in, float* F_out,
                       float* G_in, void* ws, size_t ws_bytes, void* stream);
/* normT2[i] = ||T_i||^2 (double accumulation). */
int tucker_batch_norm2(tucker_batch_t b, const float* T, double* normT2, void* ws,
                       size_t ws_bytes, void* stream);
/* fit[i] = 1 - ||T_i - G_i x_0 F_i0 ... x_{N-1} F_i,N-1|| / ||T_i|| (Sec. 2.2's
 * error metric) for the factors F and cores G, from the residual itself: the
 * reconstruction is formed mode by mode and its last step is compared with
 * T, the squared differences summed in double.  (With FP32 factors and cores
 * the shortcut ||T||^2 - ||G||^2 of tucker_fit cancels badly when the
 * residual is below about 1e-2 of ||T||.)  normT2 from tucker_batch_norm2. */
int tucker_batch_fit(tucker_batch_t b, const float* T, const float* F, const float* G,
                     const double* normT2, double* fit, void* ws, size_t ws_bytes, void* stream);
/* The same sweep and fit as one persistent, fused launch (Fig. 2 per
 * tensor): each CTA takes tensors from a device work queue (an atomic
 * counter, largest tensors first) and runs, for each, its TTM tree, leaf
 * Grams, the core of the input factors (G_in), the fit of F_in and G_in
 * (as tucker_batch_fit) and the eigensolver warm-started from F_in (F_out);
 * no CTA waits for another.  Matrices whose warm-start check fails are
 * listed and finished by the full eigensolver path in launches after it,
 * which do no work when the list is empty.  The results equal those of
 * tucker_batch_sweep + tucker_batch_fit (the fit's per-tensor sum of
 * squares is added in another order).  The last CTA verifies that every
 * tensor was taken, else it records TUCKER_ERR_INCOMPLETE in the device
 * error word (tucker_device_status), and resets the queue for the next
 * launch.  TUCKER_ERR_UNSUPPORTED under kernel policy bit 1 (full
 * eigensolver path). */
int tucker_batch_sweep_fused(tucker_batch_t b, const float* T, const float* F_in, float* F_out,
                             float* G_in, const double* normT2, double* fit, void* ws, size_t ws_bytes,
                             void* stream);
/* Byte offset in the workspace of the fused sweep's work queue (three ints:
 * next tensor, CTAs done, tensors done; all zero between launches).  Host
 * only; for tests that corrupt the queue to check the detection above. */
int tucker_batch_queue_offset(tucker_batch_t b, size_t* off);
/* on = 1: tucker_batch_graph_create records tucker_batch_sweep_fused (when
 * G_in, normT2 and fit are all non-NULL); on = 0: the per-site launches. */
int tucker_batch_set_fused(tucker_batch_t b, int on);
/* Records tucker_batch_sweep (and, when G_in, normT2 and fit are all non-NULL,
 * tucker_batch_fit of F_in and G_in; or the two as tucker_batch_sweep_fused
 * after tucker_batch_set_fused(b, 1)) with these buffers into an executable CUDA graph
 * (*graph_exec, a cudaGraphExec_t).  Nothing runs until
 * tucker_batch_graph_launch; each launch is one sweep of the whole batch on
 * the given stream.  The buffers must stay valid while the graph is used. */
int tucker_batch_graph_create(tucker_batch_t b, const float* T, const float* F_in, float* F_out,
                              float* G_in, const double* normT2, double* fit, void* ws,
                              size_t ws_bytes, void** graph_exec);
/* Launches a recorded sweep.  Fails with TUCKER_ERR_INVALID_ARG for a graph
 * not created from this batch, or recorded before a later
 * tucker_batch_autotune changed the batch's launch configurations (create it
 * again). */
int tucker_batch_graph_launch(tucker_batch_t b, void* graph_exec, void* stream);
void tucker_batch_graph_destroy(void* graph_exec);

/* Autotuner of the batched form's launch configurations (no paper
 * counterpart; the batched form runs many small tensors per launch).  Every
 * launch site of a sweep -- each tree level, the core step, each
 * reconstruction step of the fit -- is run with every candidate
 * configuration on these buffers and timed with CUDA events (one untimed
 * launch, then `reps` timed ones, 1 <= reps <= 1000); the fastest is kept
 * (another candidate replaces the default only when at least 2 % faster).
 * Candidates: positions per thread of the long-row TTM and reconstruction
 * tiles (256, 512 or 1024 consecutive positions per 256-thread tile; 1024
 * only when every rank <= 8), the row length below which a TTM tile stages
 * whole rows through shared memory (0, 16, 32 or 64), the order of the
 * site's nodes (tensor by tensor, or the nodes with the most tiles first),
 * and for long-row TTM tiles of one position per thread whether each chunk
 * of 32 input rows is copied into shared memory by cp.async first.
 * None of them changes the order in which the terms of any output are
 * summed: the tree's outputs, the factors and cores of a sweep are the same
 * bits tuned or not (the fit's per-tensor sums are added atomically and may
 * differ in the last bits).  STHOSVD keeps the default configuration.
 * The call runs the sites on the batch's data: it overwrites G with the core
 * of F (as tucker_batch_sweep with G_in) and the workspace's intermediates;
 * T and F are read only.  Synchronous.  Graphs recorded before it must be
 * created again.  F and G as in tucker_batch_sweep; needs a prepared `ws`. */
int tucker_batch_autotune(tucker_batch_t b, const float* T, const float* F, float* G, void* ws,
                          size_t ws_bytes, int reps, void* stream);
/* The batch's launch configuration per site (host only).  *n_sites = the
 * number of sites; for the first min(cap, *n_sites) sites, cfg[6i..6i+5] =
 * (kind: 0 tree level, 1 core step, 2 fit step; index within the kind;
 * positions per thread; staging row length; order 0/1; cp.async rows 0/1)
 * and ms[2i], ms[2i+1] = the default's and the chosen configuration's time
 * per launch in the last tucker_batch_autotune (-1 before one).  cfg and ms
 * may be NULL. */
int tucker_batch_tuning(tucker_batch_t b, int cap, int* n_sites, int* cfg, float* ms);
/* Sets every site's launch configuration from records in tucker_batch_tuning's
 * cfg format and order (to reuse an earlier tuning without timing again).
 * TUCKER_ERR_INVALID_ARG for a wrong site count or order, positions per
 * thread other than 1, 2 (or 4 when every rank <= 8), a staging length
 * outside 0..64, an order or cp.async flag other than 0/1, or the cp.async
 * flag with more than one position per thread or on a fit step (fit steps
 * ignore the staging length).  Host only; the batch must be prepared again
 * (tucker_batch_prepare) and its graphs created again. */
int tucker_batch_set_tuning(tucker_batch_t b, int n_sites, const int* cfg);

/* Self-test of the failure path (no paper counterpart): one thread waits,
 * through the same bounded wait the tensor-core pipelines use, on a barrier
 * that nothing completes.  The wait gives up after its limit (2 s), records
 * TUCKER_ERR_TIMEOUT in the device error word (read it with
 * tucker_device_status) and the kernel returns; *outcome is 2 when the wait
 * gave up, 1 if it completed.  Synchronous on `stream`. */
int tucker_selftest_wait_timeout(int* outcome, void* stream);

/* Text of the last error raised on the calling thread ("" if none). */
const char* tucker_last_error(void);

/* Library version as 10000*major + 100*minor + patch. */
int tucker_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TUCKER_GB300_H */
