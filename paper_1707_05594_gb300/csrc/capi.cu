// capi.cu -- the executor behind the C ABI: walks a plan's TTM-tree in
// depth-first order on a stream (Sec. 3.1 top-down execution, every node's
// output reused by all its children), forms the Gram of each leaf's input
// (Sec. 5), solves the N eigenproblems in one batched launch, and runs the
// new-core chain, STHOSVD, norms and fit.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "nvtx3/nvToolsExt.h"

#include <algorithm>

#include "common.cuh"

namespace tk {
namespace {

int factor_dtype(int dtype) { return dtype == TUCKER_F64 ? TUCKER_F64 : TUCKER_F32; }

// [R][L][C] view of a tensor with lengths `dims` along mode n
void view3(const int64_t* dims, int N, int n, int64_t* R, int64_t* L, int64_t* C) {
  *R = prod(dims, 0, n);
  *L = dims[n];
  *C = prod(dims, n + 1, N);
}

int check_ws(const Plan& p, void* ws, size_t ws_bytes, const char* who) {
  if (!ws) return fail(TUCKER_ERR_WORKSPACE, std::string(who) + ": workspace is NULL");
  if (ws_bytes < p.ws_total)
    return fail(TUCKER_ERR_WORKSPACE, std::string(who) + ": workspace smaller than ws_bytes");
  if ((uintptr_t)ws % kAlign != 0)
    return fail(TUCKER_ERR_WORKSPACE, std::string(who) + ": workspace not 256-byte aligned");
  return TUCKER_OK;
}

int check_ptrs(const void* const* F, int N, const char* who) {
  if (!F) return fail(TUCKER_ERR_INVALID_ARG, std::string(who) + ": factor array is NULL");
  for (int n = 0; n < N; ++n)
    if (!F[n]) return fail(TUCKER_ERR_INVALID_ARG, std::string(who) + ": a factor pointer is NULL");
  return TUCKER_OK;
}

// Per-node event timing: record a start event before a node's launches and
// an end event after them, while the ring has room.
struct ProfScope {
  Plan& p;
  cudaStream_t s;
  int slot = -1;
  bool nvtx = false;
  ProfScope(Plan& pp, cudaStream_t ss, int node, int label) : p(pp), s(ss) {
    if (p.prof_cap > 0) {
      // an NVTX range per node on the host timeline (for timeline tools)
      char name[64];
      snprintf(name, sizeof(name), "tucker node %d mode %d", node, label);
      nvtxRangePushA(name);
      nvtx = true;
    }
    if (p.prof_cap > 0 && p.prof_n < p.prof_cap) {
      slot = p.prof_n++;
      p.prof_node[(size_t)slot] = node;
      p.prof_label[(size_t)slot] = label;
      cudaEventRecord(static_cast<cudaEvent_t>(p.prof_events[2 * (size_t)slot]), s);
    }
  }
  ~ProfScope() {
    if (slot >= 0) cudaEventRecord(static_cast<cudaEvent_t>(p.prof_events[2 * (size_t)slot + 1]), s);
    if (nvtx) nvtxRangePop();
  }
};

std::atomic<uint64_t> g_launches{0};

// Both root children Ya = X x_a Fa^T, Yb = X x_b Fb^T (a < b): from one read
// of X by the fused kernel when the trailing block fits, else by a
// tensor-core pair that reads X once blocked by mode a + 1 (BF16 tensors; FP32
// tensors when a policy bit selects exact slices (32) or TF32 (64)), else as
// two TTMs.
int launch_root_pair(int dtype, const void* X, const int64_t* L, int N, int a, int b, const float* Fa,
                     int64_t Ka, const float* Fb, int64_t Kb, void* Ya, void* Yb, int y_dtype,
                     cudaStream_t s) {
  int64_t K[kMaxModes];
  for (int i = 0; i < N; ++i) K[i] = 1;
  K[a] = Ka;
  K[b] = Kb;
  if (fused_root_fits(dtype, N, L, K, a, b))
    return launch_ttm_fused_root(dtype, X, L, N, a, b, Fa, Ka, Fb, Kb, Ya, Yb, y_dtype, s);
  if (dtype == TUCKER_BF16 && (y_dtype == TUCKER_BF16 || y_dtype == TUCKER_F32) && (kernel_policy() & 1) == 0 &&
      ttm_tc_pair_supported(L, N, a, b, Ka, Kb, X))
    return launch_ttm_tc_pair(X, L, N, a, b, Fa, Ka, Fb, Kb, Ya, Yb, y_dtype == TUCKER_BF16, s);
  if (dtype == TUCKER_F32 && y_dtype == TUCKER_F32 && (kernel_policy() & 1) == 0) {
    const float* x = static_cast<const float*>(X);
    if ((kernel_policy() & 64) && ttm_tf32_pair_supported(L, N, a, b, Ka, Kb, X))
      return launch_ttm_tf32_pair(x, L, N, a, b, Fa, Ka, Fb, Kb, static_cast<float*>(Ya), static_cast<float*>(Yb), s);
    if ((kernel_policy() & (32 | 64)) == 32 && ttm_x3_pair_supported(L, N, a, b, Ka, Kb, X))
      return launch_ttm_x3_pair(x, L, N, a, b, Fa, Ka, Fb, Kb, static_cast<float*>(Ya), static_cast<float*>(Yb), s);
  }
  int64_t R, Ln, C;
  view3(L, N, a, &R, &Ln, &C);
  int rc = launch_ttm(dtype, X, R, Ln, C, Fa, Ka, Ya, y_dtype, s);
  if (rc) return rc;
  view3(L, N, b, &R, &Ln, &C);
  return launch_ttm(dtype, X, R, Ln, C, Fb, Kb, Yb, y_dtype, s);
}

}  // namespace

void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

#ifdef TUCKER_DEBUG
namespace dbg {
namespace {
struct Entry {
  Reader read;
  const char* file;
};
std::vector<Entry>& readers() {
  static std::vector<Entry> v;  // filled while the library loads
  return v;
}
}  // namespace
int add_reader(Reader r, const char* file) {
  readers().push_back({r, file});
  return (int)readers().size();
}
}  // namespace dbg
#endif

void destroy_profile(Plan& p) {
  for (void* e : p.prof_events)
    if (e) cudaEventDestroy(static_cast<cudaEvent_t>(e));
  p.prof_events.clear();
  p.prof_node.clear();
  p.prof_label.clear();
  p.prof_cap = p.prof_n = 0;
}

}  // namespace tk

using namespace tk;

extern "C" {

int tucker_debug_build(void) {
#ifdef TUCKER_DEBUG
  return 1;
#else
  return 0;
#endif
}

int tucker_debug_check(int64_t* index, int64_t* bound, int* line, char* file, int file_len, int reset) {
  if (index) *index = 0;
  if (bound) *bound = 0;
  if (line) *line = 0;
  if (file && file_len > 0) file[0] = 0;
#ifdef TUCKER_DEBUG
  TK_CUDA_TRY(cudaDeviceSynchronize());
  unsigned long long total = 0;
  for (const auto& e : dbg::readers()) {
    dbg::Record r{};
    if (e.read(&r, reset) != 0) return fail(TUCKER_ERR_CUDA, "tucker_debug_check: record not readable");
    if (r.count && !total) {
      if (index) *index = r.index;
      if (bound) *bound = r.bound;
      if (line) *line = r.line;
      if (file && file_len > 0) {
        std::strncpy(file, e.file, (size_t)file_len - 1);
        file[file_len - 1] = 0;
      }
    }
    total += r.count;
  }
  return total > (unsigned long long)INT32_MAX ? INT32_MAX : (int)total;
#else
  (void)reset;
  return 0;
#endif
}

int tucker_ttm(int N, const int64_t* dims, const void* X, int x_dtype, int n, const void* F,
               int64_t K, void* Y, void* stream) {
  if (N < 1 || N > kMaxModes || !dims || n < 0 || n >= N || K < 1 || !X || !F || !Y)
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_ttm: invalid argument");
  for (int i = 0; i < N; ++i)
    if (dims[i] < 1) return fail(TUCKER_ERR_INVALID_ARG, "tucker_ttm: lengths must be >= 1");
  int64_t R, L, C;
  view3(dims, N, n, &R, &L, &C);
  return launch_ttm(x_dtype, X, R, L, C, F, K, Y, factor_dtype(x_dtype),
                    static_cast<cudaStream_t>(stream));
}

int tucker_ttm_pair(int N, const int64_t* dims, const void* X, int x_dtype, int a, const float* Fa,
                    int64_t Ka, int b, const float* Fb, int64_t Kb, void* Ya, void* Yb, int y_dtype,
                    void* stream) {
  if (N < 2 || N > kMaxModes || !dims || !X || !Fa || !Fb || !Ya || !Yb || a < 0 || b <= a || b >= N ||
      Ka < 1 || Kb < 1 || Ka > dims[a] || Kb > dims[b])
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_ttm_pair: invalid argument");
  for (int i = 0; i < N; ++i)
    if (dims[i] < 1) return fail(TUCKER_ERR_INVALID_ARG, "tucker_ttm_pair: lengths must be >= 1");
  int64_t K[kMaxModes] = {};
  for (int i = 0; i < N; ++i) K[i] = 1;
  K[a] = Ka;
  K[b] = Kb;
  if (!root_pair_fits(x_dtype, N, dims, K, a, b))
    return fail(TUCKER_ERR_UNSUPPORTED, "tucker_ttm_pair: shape or type not supported");
  return launch_root_pair(x_dtype, X, dims, N, a, b, Fa, Ka, Fb, Kb, Ya, Yb, y_dtype,
                          static_cast<cudaStream_t>(stream));
}

int tucker_gram(int N, const int64_t* dims, const void* Z, int z_dtype, int n, double* W,
                void* stream) {
  if (N < 1 || N > kMaxModes || !dims || n < 0 || n >= N || !Z || !W)
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_gram: invalid argument");
  for (int i = 0; i < N; ++i)
    if (dims[i] < 1) return fail(TUCKER_ERR_INVALID_ARG, "tucker_gram: lengths must be >= 1");
  int64_t R, L, C;
  view3(dims, N, n, &R, &L, &C);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TK_CUDA_TRY(cudaMemsetAsync(W, 0, (size_t)L * (size_t)L * sizeof(double), s));
  return launch_gram(z_dtype, Z, R, L, C, W, s);
}

int tucker_eig_topk(int batch, const int64_t* L, const int64_t* K, const double* const* W,
                    void* const* F, int f_dtype, void* ws, size_t ws_bytes, void* stream) {
  if (batch < 1 || !L || !K || !W || !F)
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_eig_topk: invalid argument");
  if (f_dtype != TUCKER_F32 && f_dtype != TUCKER_F64)
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_eig_topk: f_dtype must be TUCKER_F32 or TUCKER_F64");
  std::vector<EigProblem> probs((size_t)batch);
  for (int b = 0; b < batch; ++b) {
    if (!W[b] || !F[b]) return fail(TUCKER_ERR_INVALID_ARG, "tucker_eig_topk: NULL matrix");
    probs[(size_t)b] = EigProblem{W[b], F[b], (int)L[b], (int)K[b]};
  }
  return launch_eig_topk(probs.data(), batch, f_dtype, ws, ws_bytes,
                         static_cast<cudaStream_t>(stream));
}

int tucker_hooi_sweep(tucker_plan_t plan, const void* T, const void* const* F_in,
                      void* const* F_out, void* ws, size_t ws_bytes, void* stream) {
  return tucker_hooi_sweep_core(plan, T, F_in, F_out, nullptr, ws, ws_bytes, stream);
}

int tucker_hooi_sweep_core(tucker_plan_t plan, const void* T, const void* const* F_in,
                           void* const* F_out, void* G_in, void* ws, size_t ws_bytes,
                           void* stream) {
  if (!plan || !T) return fail(TUCKER_ERR_INVALID_ARG, "tucker_hooi_sweep: NULL plan or T");
  const Plan& p = plan->p;
  int rc = check_ptrs(F_in, p.N, "tucker_hooi_sweep");
  if (rc) return rc;
  rc = check_ptrs(const_cast<const void* const*>(F_out), p.N, "tucker_hooi_sweep");
  if (rc) return rc;
  for (int n = 0; n < p.N; ++n)
    for (int j = 0; j < p.N; ++j)
      if (F_out[n] == F_in[j])
        return fail(TUCKER_ERR_INVALID_ARG, "tucker_hooi_sweep: F_out aliases F_in");
  rc = check_ws(p, ws, ws_bytes, "tucker_hooi_sweep");
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* wsb = static_cast<char*>(ws);
  const int fdt = factor_dtype(p.dtype);
  const int idt = p.inter_dtype();
  // the core of the input factors comes from the smallest leaf input:
  // G = Z_n x_n F_n^T with Z_n = T x_{j != n} F_j^T (Fig. 2 "New core" for F_in)
  int core_leaf = -1;
  if (G_in) {
    uint64_t best = ~0ull;
    for (size_t i = 1; i < p.nodes.size(); ++i)
      if (p.nodes[i].label < -1 && p.nodes[i].in_elems < best) {
        best = p.nodes[i].in_elems;
        core_leaf = (int)i;
      }
  }
  for (size_t i = 1; i < p.nodes.size(); ++i) {
    const PlanNode& nd = p.nodes[i];
    const PlanNode& par = p.nodes[(size_t)nd.parent];
    const bool from_root = nd.parent == 0;
    const void* in = from_root ? T : (const void*)(wsb + p.off_scratch + par.ws_off);
    const int in_dt = from_root ? p.dtype : idt;
    ProfScope prof(plan->p, s, (int)i, nd.label);
    if (nd.label >= 0 && (int)i == p.fused_u2) {
      // written together with the first root child
    } else if (nd.label >= 0 && (int)i == p.fused_u1) {
      // fused root: both root children from one read of T
      const PlanNode& n2 = p.nodes[(size_t)p.fused_u2];
      const int a = std::min(nd.label, n2.label), b = std::max(nd.label, n2.label);
      void* y1 = wsb + p.off_scratch + nd.ws_off;
      void* y2 = wsb + p.off_scratch + n2.ws_off;
      rc = launch_root_pair(p.dtype, T, p.L, p.N, a, b, static_cast<const float*>(F_in[a]), p.K[a],
                            static_cast<const float*>(F_in[b]), p.K[b], nd.label == a ? y1 : y2,
                            nd.label == a ? y2 : y1, idt, s);
      if (rc) return rc;
    } else if (nd.label >= 0) {
      int64_t R, L, C;
      view3(par.out_dims, p.N, nd.label, &R, &L, &C);
      rc = launch_ttm(in_dt, in, R, L, C, F_in[nd.label], p.K[nd.label],
                      wsb + p.off_scratch + nd.ws_off, idt, s);
      if (rc) return rc;
    } else {
      const int n = -nd.label - 2;
      int64_t R, L, C;
      view3(par.out_dims, p.N, n, &R, &L, &C);
      double* W = reinterpret_cast<double*>(wsb + p.off_gram[n]);
      TK_CUDA_TRY(cudaMemsetAsync(W, 0, (size_t)L * (size_t)L * sizeof(double), s));
      rc = launch_gram(in_dt, in, R, L, C, W, s);
      if (rc) return rc;
      if ((int)i == core_leaf) {
        rc = launch_ttm(in_dt, in, R, L, C, F_in[n], p.K[n], G_in, fdt, s);
        if (rc) return rc;
      }
    }
  }
  // the input factors start the eigensolver (warm start, checked on the GPU)
  EigProblem probs[kMaxModes];
  for (int n = 0; n < p.N; ++n)
    probs[n] = EigProblem{reinterpret_cast<const double*>(wsb + p.off_gram[n]), F_out[n],
                          (int)p.L[n], (int)p.K[n], F_in[n]};
  ProfScope prof(plan->p, s, -1, -1);
  return launch_eig_topk(probs, p.N, fdt, wsb + p.off_eig, p.bytes_eig, s);
}

int tucker_profile_enable(tucker_plan_t plan, int capacity) {
  if (!plan || capacity < 0) return fail(TUCKER_ERR_INVALID_ARG, "tucker_profile_enable");
  Plan& p = plan->p;
  destroy_profile(p);
  if (capacity == 0) return TUCKER_OK;
  p.prof_events.assign(2 * (size_t)capacity, nullptr);
  p.prof_node.assign((size_t)capacity, 0);
  p.prof_label.assign((size_t)capacity, 0);
  for (auto& e : p.prof_events) {
    cudaEvent_t ev;
    const cudaError_t err = cudaEventCreate(&ev);
    if (err != cudaSuccess) {
      destroy_profile(p);
      return fail(TUCKER_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(err));
    }
    e = ev;
  }
  p.prof_cap = capacity;
  p.prof_n = 0;
  return TUCKER_OK;
}

int tucker_profile_read(tucker_plan_t plan, tucker_prof_rec_t* recs, int capacity, int* n_recs) {
  if (!plan || !n_recs) return fail(TUCKER_ERR_INVALID_ARG, "tucker_profile_read");
  Plan& p = plan->p;
  int n = 0;
  for (int i = 0; i < p.prof_n; ++i) {
    cudaEvent_t a = static_cast<cudaEvent_t>(p.prof_events[2 * (size_t)i]);
    cudaEvent_t b = static_cast<cudaEvent_t>(p.prof_events[2 * (size_t)i + 1]);
    TK_CUDA_TRY(cudaEventSynchronize(b));
    float ms = 0.f;
    TK_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
    if (recs && n < capacity) {
      recs[n].node = p.prof_node[(size_t)i];
      recs[n].label = p.prof_label[(size_t)i];
      recs[n].ms = ms;
    }
    ++n;
  }
  *n_recs = n;
  p.prof_n = 0;
  return TUCKER_OK;
}

uint64_t tucker_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int tucker_core(tucker_plan_t plan, const void* T, const void* const* F, void* G, void* ws,
                size_t ws_bytes, void* stream) {
  if (!plan || !T || !G) return fail(TUCKER_ERR_INVALID_ARG, "tucker_core: NULL argument");
  const Plan& p = plan->p;
  int rc = check_ptrs(F, p.N, "tucker_core");
  if (rc) return rc;
  rc = check_ws(p, ws, ws_bytes, "tucker_core");
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* wsb = static_cast<char*>(ws) + p.off_scratch;
  const int fdt = factor_dtype(p.dtype);
  // ping-pong buffers sized for the largest intermediate of the chain
  size_t mx = 0;
  unsigned P = 0;
  for (int i = 0; i < p.N; ++i) {
    P |= 1u << p.core_order[(size_t)i];
    mx = std::max(mx, (size_t)tensor_size(p, P));
  }
  void* buf[2] = {wsb, wsb + align_up(mx * p.inter_bytes())};
  int64_t dims[kMaxModes];
  std::memcpy(dims, p.L, sizeof(int64_t) * (size_t)p.N);
  const void* cur = T;
  int cur_dt = p.dtype;
  for (int i = 0; i < p.N; ++i) {
    const int m = p.core_order[(size_t)i];
    void* out = (i == p.N - 1) ? G : buf[i & 1];
    int64_t R, L, C;
    view3(dims, p.N, m, &R, &L, &C);
    ProfScope prof(plan->p, s, -2, m);
    const int out_dt = (i == p.N - 1) ? fdt : p.inter_dtype();
    rc = launch_ttm(cur_dt, cur, R, L, C, F[m], p.K[m], out, out_dt, s);
    if (rc) return rc;
    dims[m] = p.K[m];
    cur = out;
    cur_dt = out_dt;
  }
  return TUCKER_OK;
}

int tucker_hooi_sweep_gs(tucker_plan_t plan, const void* T, const void* const* F_in,
                         void* const* F_out, void* G_out, void* ws, size_t ws_bytes, void* stream) {
  if (!plan || !T) return fail(TUCKER_ERR_INVALID_ARG, "tucker_hooi_sweep_gs: NULL plan or T");
  const Plan& p = plan->p;
  int rc = check_ptrs(F_in, p.N, "tucker_hooi_sweep_gs");
  if (rc) return rc;
  rc = check_ptrs(const_cast<const void* const*>(F_out), p.N, "tucker_hooi_sweep_gs");
  if (rc) return rc;
  for (int n = 0; n < p.N; ++n)
    for (int j = 0; j < p.N; ++j)
      if (F_out[n] == F_in[j])
        return fail(TUCKER_ERR_INVALID_ARG, "tucker_hooi_sweep_gs: F_out aliases F_in");
  rc = check_ws(p, ws, ws_bytes, "tucker_hooi_sweep_gs");
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* wsb = static_cast<char*>(ws);
  const int fdt = factor_dtype(p.dtype);
  const int idt = p.inter_dtype();
  // ping-pong buffers sized for the largest intermediate of any chain
  size_t mx = 1;
  for (int n = 0; n < p.N; ++n) {
    unsigned P = 0;
    for (int i = 0; i < p.N; ++i) {
      const int m = p.core_order[(size_t)i];
      if (m == n) continue;
      P |= 1u << m;
      mx = std::max(mx, (size_t)tensor_size(p, P));
    }
  }
  void* buf[2] = {wsb + p.off_scratch, wsb + p.off_scratch + align_up(mx * p.inter_bytes())};
  for (int n = 0; n < p.N; ++n) {
    // Z_n = T x_{m != n} F_m^T with the factors of this sweep for m < n
    // (the Gauss-Seidel form) along the core-chain order without n
    int64_t dims[kMaxModes];
    std::memcpy(dims, p.L, sizeof(int64_t) * (size_t)p.N);
    const void* cur = T;
    int cur_dt = p.dtype, step = 0;
    for (int i = 0; i < p.N; ++i) {
      const int m = p.core_order[(size_t)i];
      if (m == n) continue;
      int64_t R, L, C;
      view3(dims, p.N, m, &R, &L, &C);
      ProfScope prof(plan->p, s, -3, m);
      void* out = buf[step & 1];
      rc = launch_ttm(cur_dt, cur, R, L, C, m < n ? F_out[m] : F_in[m], p.K[m], out, idt, s);
      if (rc) return rc;
      dims[m] = p.K[m];
      cur = out;
      cur_dt = idt;
      ++step;
    }
    int64_t R, L, C;
    view3(dims, p.N, n, &R, &L, &C);
    double* W = reinterpret_cast<double*>(wsb + p.off_gram[n]);
    TK_CUDA_TRY(cudaMemsetAsync(W, 0, (size_t)L * (size_t)L * sizeof(double), s));
    rc = launch_gram(cur_dt, cur, R, L, C, W, s);
    if (rc) return rc;
    // the new F_n, warm-started from the input factor
    EigProblem prob{W, F_out[n], (int)p.L[n], (int)p.K[n], F_in[n]};
    rc = launch_eig_topk(&prob, 1, fdt, wsb + p.off_eig, p.bytes_eig, s);
    if (rc) return rc;
  }
  if (G_out) return tucker_core(plan, T, const_cast<const void* const*>(F_out), G_out, ws, ws_bytes, stream);
  return TUCKER_OK;
}

int tucker_sthosvd(tucker_plan_t plan, const void* T, void* const* F, void* G, void* ws,
                   size_t ws_bytes, void* stream) {
  if (!plan || !T || !G) return fail(TUCKER_ERR_INVALID_ARG, "tucker_sthosvd: NULL argument");
  const Plan& p = plan->p;
  int rc = check_ptrs(const_cast<const void* const*>(F), p.N, "tucker_sthosvd");
  if (rc) return rc;
  rc = check_ws(p, ws, ws_bytes, "tucker_sthosvd");
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* wsb = static_cast<char*>(ws);
  const int fdt = factor_dtype(p.dtype);
  size_t mx = 0;
  unsigned P = 0;
  for (int i = 0; i < p.N; ++i) {
    P |= 1u << p.sth_order[(size_t)i];
    mx = std::max(mx, (size_t)tensor_size(p, P));
  }
  void* buf[2] = {wsb + p.off_scratch, wsb + p.off_scratch + align_up(mx * p.inter_bytes())};
  int64_t dims[kMaxModes];
  std::memcpy(dims, p.L, sizeof(int64_t) * (size_t)p.N);
  const void* cur = T;
  int cur_dt = p.dtype;
  for (int i = 0; i < p.N; ++i) {
    const int n = p.sth_order[(size_t)i];
    int64_t R, L, C;
    view3(dims, p.N, n, &R, &L, &C);
    double* W = reinterpret_cast<double*>(wsb + p.off_gram[n]);
    TK_CUDA_TRY(cudaMemsetAsync(W, 0, (size_t)L * (size_t)L * sizeof(double), s));
    rc = launch_gram(cur_dt, cur, R, L, C, W, s);
    if (rc) return rc;
    EigProblem pr{W, F[n], (int)L, (int)p.K[n]};
    rc = launch_eig_topk(&pr, 1, fdt, wsb + p.off_eig, p.bytes_eig, s);
    if (rc) return rc;
    void* out = (i == p.N - 1) ? G : buf[i & 1];
    const int out_dt = (i == p.N - 1) ? fdt : p.inter_dtype();
    rc = launch_ttm(cur_dt, cur, R, L, C, F[n], p.K[n], out, out_dt, s);
    if (rc) return rc;
    dims[n] = p.K[n];
    cur = out;
    cur_dt = out_dt;
  }
  return TUCKER_OK;
}

int tucker_norm2(tucker_plan_t plan, const void* T, double* out, void* stream) {
  if (!plan || !T || !out) return fail(TUCKER_ERR_INVALID_ARG, "tucker_norm2: NULL argument");
  const Plan& p = plan->p;
  return launch_norm2(p.dtype, T, (int64_t)tensor_size(p, 0), out,
                      static_cast<cudaStream_t>(stream));
}

// ||X||^2 of the finiteness check: a device double of the library, so the
// check allocates nothing.  One check runs at a time (the check is
// synchronous anyway), so calls from several host threads or streams do not
// share the accumulator.
static __device__ double g_check_norm2;
static std::mutex g_check_mutex;

int tucker_check_finite(const void* X, int dtype, int64_t n, void* stream) {
  if (!X || n < 0) return fail(TUCKER_ERR_INVALID_ARG, "tucker_check_finite: invalid argument");
  if (n == 0) return TUCKER_OK;
  std::lock_guard<std::mutex> lock(g_check_mutex);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* d = nullptr;
  TK_CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void**>(&d), g_check_norm2));
  const int rc = launch_norm2(dtype, X, n, d, s);
  if (rc) return rc;
  double h = 0.0;
  TK_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, s));
  TK_CUDA_TRY(cudaStreamSynchronize(s));
  if (!std::isfinite(h))
    return fail(TUCKER_ERR_NONFINITE, "tucker_check_finite: the tensor holds NaN or Inf values");
  return TUCKER_OK;
}

int tucker_fit(tucker_plan_t plan, const void* G, const double* normT2, double* out,
               void* stream) {
  if (!plan || !G || !normT2 || !out)
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_fit: NULL argument");
  const Plan& p = plan->p;
  const unsigned full = (1u << p.N) - 1u;
  return launch_fit(factor_dtype(p.dtype), G, (int64_t)tensor_size(p, full), normT2, out,
                    static_cast<cudaStream_t>(stream));
}

}  // extern "C"
