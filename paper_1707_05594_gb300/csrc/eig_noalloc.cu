// eig_noalloc.cu -- tucker_eig_topk_noalloc: the leading-eigenvector solver of
// tucker_eig_topk with its scratch memory in a fixed array compiled into the
// library, for callers that must not allocate device memory.
//
// Who needs it: code that runs where a device allocation is not allowed or
// not wanted -- e.g. a process whose device memory is entirely handed to
// another allocator (a framework's caching pool or a fixed budget), or
// latency-sensitive code that cannot afford cudaMalloc / cudaFree, which may
// synchronise the device and stall other streams.  Such a caller passes only
// its inputs and outputs; the scratch comes from g_eig_scratch below.
//
// The array lives in every GPU that loads this library until the process
// exits (kNoallocScratchBytes, about 4 MiB).  Host code must not hand the
// symbol itself to a kernel (on the host it names a host-side stand-in); the
// device address is obtained once per device with cudaGetSymbolAddress.
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace tk {
namespace {

constexpr int kNoallocMaxBatch = 8;
constexpr int kNoallocMaxL = 200;
constexpr int kNoallocMaxK = 64;
// eig_ws_bytes() of kNoallocMaxBatch matrices with L = 200, K = 64 (~4 MiB):
// a 256-byte list head, then the per-matrix scratch
constexpr size_t kPerMatrix = eig_bytes_per_matrix(kNoallocMaxL, kNoallocMaxK);
constexpr size_t kNoallocScratchBytes = kAlign + kNoallocMaxBatch * kPerMatrix;

static __device__ __align__(256) unsigned char g_eig_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_eig_scratch on the current device (set-up on first use).
int scratch_address(void** out) {
  int dev = 0;
  TK_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(TUCKER_ERR_UNSUPPORTED, "tucker_eig_topk_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_eig_scratch);
    if (e != cudaSuccess || !p)
      return fail(TUCKER_ERR_CUDA, std::string("tucker_eig_topk_noalloc: cudaGetSymbolAddress: ") +
                                       cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return TUCKER_OK;
}

}  // namespace
}  // namespace tk

using namespace tk;

extern "C" int tucker_eig_topk_noalloc(int batch, const int64_t* L, const int64_t* K,
                                       const double* const* W, void* const* F, int f_dtype,
                                       void* stream) {
  if (batch < 1 || !L || !K || !W || !F)
    return fail(TUCKER_ERR_INVALID_ARG, "tucker_eig_topk_noalloc: invalid argument");
  if (f_dtype != TUCKER_F32 && f_dtype != TUCKER_F64)
    return fail(TUCKER_ERR_INVALID_ARG,
                "tucker_eig_topk_noalloc: f_dtype must be TUCKER_F32 or TUCKER_F64");
  if (batch > kNoallocMaxBatch)
    return fail(TUCKER_ERR_UNSUPPORTED,
                "tucker_eig_topk_noalloc: at most 8 matrices per call (fixed scratch)");
  EigProblem probs[kNoallocMaxBatch];
  for (int b = 0; b < batch; ++b) {
    if (!W[b] || !F[b]) return fail(TUCKER_ERR_INVALID_ARG, "tucker_eig_topk_noalloc: NULL matrix");
    if (L[b] < 1 || L[b] > kNoallocMaxL || K[b] < 1 || K[b] > L[b] || K[b] > kNoallocMaxK)
      return fail(TUCKER_ERR_UNSUPPORTED,
                  "tucker_eig_topk_noalloc: each matrix needs L <= 200 and 1 <= K <= min(L, 64) "
                  "to fit the fixed scratch");
    probs[b] = EigProblem{W[b], F[b], (int)L[b], (int)K[b]};
  }
  const size_t need = eig_ws_bytes(batch, L, K);
  if (need > kNoallocScratchBytes)
    return fail(TUCKER_ERR_UNSUPPORTED, "tucker_eig_topk_noalloc: problem exceeds the fixed scratch");
  void* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != TUCKER_OK) return rc;
  // every scratch word the solver reads it has written earlier in the same
  // call, so the previous call's contents need no clearing
  return launch_eig_topk(probs, batch, f_dtype, scratch, kNoallocScratchBytes,
                         static_cast<cudaStream_t>(stream));
}
