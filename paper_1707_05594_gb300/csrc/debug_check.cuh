// debug_check.cuh -- global-memory index checks of the debug build (the
// library compiled with -DTUCKER_DEBUG); in the normal build TK_DBG_IN is the
// constant true and costs nothing.
//
// A kernel states, per thread and per array, the first and last element it
// will read or write (the library's accesses are affine in their loop
// indices, so the two ends bound every access in between) together with the
// array's length: TK_DBG_IN(first, last, length).  When the range is not
// inside [0, length) the check records the offending index, the length and
// the source line in this translation unit's device record and yields false,
// and the kernel skips those accesses.  tucker_debug_check reads (and
// optionally clears) the records of every translation unit.
#pragma once

#ifdef TUCKER_DEBUG

#include <cuda_runtime.h>

namespace tk {
namespace dbg {

struct Record {
  unsigned long long count;  // out-of-range ranges seen since the last reset
  long long index;           // the first one's offending index
  long long bound;           // and the length it was checked against
  int line;                  // and its source line
  int pad;
};

// One record per translation unit (internal linkage).
static __device__ Record g_record;

static __device__ __noinline__ void record_bad(long long index, long long bound, int line) {
  if (atomicAdd(&g_record.count, 1ull) == 0ull) {
    g_record.index = index;
    g_record.bound = bound;
    g_record.line = line;
  }
}

static __device__ __forceinline__ bool in_range(long long first, long long last, long long n, int line) {
  if (last < first) return true;  // no access
  if (first >= 0 && last < n) return true;
  record_bad(first < 0 ? first : last, n, line);
  return false;
}

// Host: every translation unit registers a reader of its record at load time.
using Reader = int (*)(Record* out, int reset);
int add_reader(Reader r, const char* file);

static int read_record(Record* out, int reset) {
  if (cudaMemcpyFromSymbol(out, g_record, sizeof(Record)) != cudaSuccess) return -1;
  if (reset) {
    const Record z{};
    if (cudaMemcpyToSymbol(g_record, &z, sizeof(Record)) != cudaSuccess) return -1;
  }
  return 0;
}
static const int g_reader_id = add_reader(&read_record, __FILE__);

}  // namespace dbg
}  // namespace tk

#define TK_DBG_IN(first, last, n) \
  ::tk::dbg::in_range((long long)(first), (long long)(last), (long long)(n), __LINE__)

#else

#define TK_DBG_IN(first, last, n) true

#endif
