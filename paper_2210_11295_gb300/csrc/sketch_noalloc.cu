// bsrht_sketch_noalloc: the block SRHT sketch with library-owned fixed
// scratch, for callers that must not allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is off limits - for
// example a host that hands this library a stream inside a region where
// device allocation would synchronise the device or break its own memory
// accounting (a caching allocator that must see every byte, a real-time
// loop that may not block), or a plug-in whose host application owns all
// device memory.  Such a caller can pass A and the output, but cannot give
// the library scratch and cannot let it allocate any.
//
// The per-CTA partial sums of the sketch (the only scratch it needs) live in
// one file-scope device array of kNoAllocScratchBytes.  Every device that
// loads the library holds this array until the process exits.  All calls on
// a device share it and it keeps the last call's contents; the sketch writes
// every partial-sum slot before reading it and clears its one status word at
// the start of each call, so nothing else needs to start at zero.  Two calls whose kernels overlap on the GPU (different streams, or
// different host threads on one device) race on the array and give wrong
// results: serialise them on one stream.
#include <mutex>

#include "capi_internal.cuh"
#include "common.cuh"
#include "sketch.cuh"
#include "trace.cuh"

namespace bsrht {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {nullptr};

// Device address of g_noalloc_scratch on the current device.  In host code
// the array's name is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress, once per device, with that device current.
int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BSRHT_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return BSRHT_ECUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return BSRHT_OK;
}

}  // namespace
}  // namespace bsrht

using namespace bsrht;

extern "C" int bsrht_sketch_noalloc(const void* A, int64_t n, int64_t m, int32_t p, int64_t l, uint64_t seed,
                                    void* out, const bsrht_opts* opts) {
  bsrht_opts o;
  bsrht_opts_init(&o);
  if (opts) o = *opts;
  if ((!A && m > 0) || (!out && m > 0)) return BSRHT_EINVAL;
  int dt = 0;
  int st = plan_dtype(o, &dt);
  if (st != BSRHT_OK) return st;
  SketchPlan pl;
  st = sketch_make_plan(pl, dt, o.variant, n, m, o.lda, p, l, true, A);
  if (st != BSRHT_OK) return st;
  if (m == 0) return BSRHT_OK;
  if (pl.work_bytes > kNoAllocScratchBytes) return BSRHT_ENOMEM;
  void* scratch = nullptr;
  st = noalloc_scratch(&scratch);
  if (st != BSRHT_OK) return st;
  // Stage tracing (bsrht_profile_enable) starts afresh, as in bsrht_sketch.
  trace_begin(static_cast<cudaStream_t>(o.stream));
  return sketch_run(pl, A, seed, out, m, scratch, static_cast<cudaStream_t>(o.stream));
}
