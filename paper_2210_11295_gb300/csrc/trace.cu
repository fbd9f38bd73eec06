// Per-stage CUDA-event tracing: bsrht_profile_enable / bsrht_profile_stages.
#include <cstring>
#include <vector>

#include "common.cuh"
#include "trace.cuh"

namespace bsrht {
namespace {

struct Trace {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<const char*> names;
  size_t used = 0;
};
thread_local Trace g_trace;

cudaEvent_t next_event() {
  Trace& t = g_trace;
  if (t.used == t.pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    t.pool.push_back(e);
  }
  return t.pool[t.used++];
}

}  // namespace

void trace_begin(cudaStream_t s) {
  Trace& t = g_trace;
  if (!t.on) return;
  t.used = 0;
  t.names.clear();
  cudaEvent_t e = next_event();
  if (e) cudaEventRecord(e, s);
  t.names.push_back("begin");
}

void trace_mark(cudaStream_t s, const char* name) {
  Trace& t = g_trace;
  if (!t.on || t.used == 0) return;
  cudaEvent_t e = next_event();
  if (e) cudaEventRecord(e, s);
  t.names.push_back(name);
}

}  // namespace bsrht

using namespace bsrht;

extern "C" {

int bsrht_profile_enable(int on) {
  g_trace.on = on != 0;
  g_trace.used = 0;
  g_trace.names.clear();
  return BSRHT_OK;
}

int bsrht_profile_stages(char* names, double* ms, int cap, int* count) {
  if (!count) return BSRHT_EINVAL;
  Trace& t = g_trace;
  const int n = t.used > 1 ? (int)t.used - 1 : 0;
  *count = n;
  for (int i = 0; i < n && i < cap; ++i) {
    float f = 0.f;
    BSRHT_CUDA_TRY(cudaEventSynchronize(t.pool[i + 1]));
    BSRHT_CUDA_TRY(cudaEventElapsedTime(&f, t.pool[i], t.pool[i + 1]));
    if (ms) ms[i] = f;
    if (names) {
      std::strncpy(names + 32 * i, t.names[i + 1], 31);
      names[32 * i + 31] = 0;
    }
  }
  return BSRHT_OK;
}

}  // extern "C"
