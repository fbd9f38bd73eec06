// extern "C" entry points of libbsrht (declared in include/bsrht.h).
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "capi_internal.cuh"
#include "common.cuh"
#include "sketch.cuh"
#include "trace.cuh"

namespace bsrht {

// ------------------------------------------------------------ scratch pool
// One growing device buffer per device.  Growing frees the old buffer with
// cudaFree, which waits for the device, so a call still using it finishes
// first.  Concurrent calls on different streams must pass their own
// workspace (they would otherwise share this buffer).
namespace {
std::atomic<uint64_t> g_launches{0};
struct Pool {
  void* ptr = nullptr;
  size_t bytes = 0;
};
std::mutex g_pool_mu;
Pool g_pool[64];
}  // namespace

void note_launches(int k) { g_launches.fetch_add((uint64_t)k, std::memory_order_relaxed); }

int cuda_failure(cudaError_t e, const char* file, int line) {
  static const bool debug = std::getenv("BSRHT_DEBUG") != nullptr;
  if (debug) std::fprintf(stderr, "bsrht: %s at %s:%d\n", cudaGetErrorName(e), file, line);
  return BSRHT_ECUDA;
}

int pool_get(size_t bytes, void** out) {
  *out = nullptr;
  if (bytes == 0) return BSRHT_OK;
  int dev = 0;
  BSRHT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return BSRHT_EUNSUP;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  Pool& p = g_pool[dev];
  if (p.bytes < bytes) {
    if (p.ptr) cudaFree(p.ptr);
    p.ptr = nullptr;
    p.bytes = 0;
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      return BSRHT_ENOMEM;
    }
    p.ptr = ptr;
    p.bytes = bytes;
  }
  *out = p.ptr;
  return BSRHT_OK;
}

int workspace_for(const bsrht_opts* o, size_t need, void** out) {
  if (o && o->workspace) {
    if (o->workspace_bytes < need) return BSRHT_ENOMEM;
    *out = o->workspace;
    return BSRHT_OK;
  }
  return pool_get(need, out);
}

bsrht_opts opts_or_default(const bsrht_opts* o) {
  bsrht_opts d;
  bsrht_opts_init(&d);
  return o ? *o : d;
}

int plan_dtype(const bsrht_opts& o, int* dt) {
  if (o.precision != BSRHT_PREC_AUTO && o.precision != BSRHT_PREC_F64) return BSRHT_EINVAL;
  if (o.precision == BSRHT_PREC_AUTO || o.dtype == BSRHT_F64) {
    *dt = o.dtype;
    return BSRHT_OK;
  }
  if (o.dtype != BSRHT_F32) return o.dtype >= BSRHT_F64 && o.dtype <= BSRHT_F16 ? BSRHT_EUNSUP : BSRHT_EINVAL;
  *dt = kDtypeF32AsF64;
  return BSRHT_OK;
}

int precision_auto_only(const bsrht_opts& o) {
  if (o.precision == BSRHT_PREC_AUTO || (o.precision == BSRHT_PREC_F64 && o.dtype == BSRHT_F64)) return BSRHT_OK;
  return o.precision == BSRHT_PREC_F64 ? BSRHT_EUNSUP : BSRHT_EINVAL;
}

}  // namespace bsrht

using namespace bsrht;

extern "C" {

void bsrht_opts_init(bsrht_opts* o) {
  if (!o) return;
  o->dtype = BSRHT_F64;
  o->variant = BSRHT_VARIANT_AUTO;
  o->lda = 0;
  o->stream = nullptr;
  o->workspace = nullptr;
  o->workspace_bytes = 0;
  o->precision = BSRHT_PREC_AUTO;
}

const char* bsrht_strerror(int s) {
  switch (s) {
    case BSRHT_OK: return "success";
    case BSRHT_EINVAL: return "invalid argument";
    case BSRHT_ENOMEM: return "out of device memory or workspace too small";
    case BSRHT_EUNSUP: return "unsupported combination of arguments";
    case BSRHT_ETIMEDOUT: return "bounded wait timed out";
    case BSRHT_ENOTPD: return "matrix not positive definite after shifting";
    case BSRHT_ENOCONV: return "Jacobi SVD did not converge";
    case BSRHT_ECUDA: return "CUDA runtime error";
  }
  return "unknown status";
}

const char* bsrht_version(void) { return "0.1.0"; }

uint64_t bsrht_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int bsrht_sketch_workspace(int64_t n, int64_t m, int32_t p, int64_t l, const bsrht_opts* opts,
                           size_t* bytes) {
  if (!bytes) return BSRHT_EINVAL;
  const bsrht_opts o = opts_or_default(opts);
  int dt = 0;
  int st = plan_dtype(o, &dt);
  if (st != BSRHT_OK) return st;
  SketchPlan pl;
  st = sketch_make_plan(pl, dt, o.variant, n, m, o.lda, p, l, false);
  if (st != BSRHT_OK) return st;
  *bytes = pl.work_bytes;
  return BSRHT_OK;
}

int bsrht_sketch(const void* A, int64_t n, int64_t m, int32_t p, int64_t l, uint64_t seed, void* out,
                 const bsrht_opts* opts) {
  const bsrht_opts o = opts_or_default(opts);
  if ((!A && m > 0) || (!out && m > 0)) return BSRHT_EINVAL;
  int dt = 0;
  int st = plan_dtype(o, &dt);
  if (st != BSRHT_OK) return st;
  SketchPlan pl;
  st = sketch_make_plan(pl, dt, o.variant, n, m, o.lda, p, l, true, A);
  if (st != BSRHT_OK) return st;
  if (m == 0) return BSRHT_OK;
  void* work = nullptr;
  st = workspace_for(&o, pl.work_bytes, &work);
  if (st != BSRHT_OK) return st;
  // With bsrht_profile_enable on, the TMA / tensor-core paths record events
  // around their kernels (stages sketch_tables, sketch_kernel, sketch_reduce).
  trace_begin(static_cast<cudaStream_t>(o.stream));
  return sketch_run(pl, A, seed, out, m, work, static_cast<cudaStream_t>(o.stream));
}

int bsrht_sketch_autotune(const void* A, int64_t n, int64_t m, int32_t p, int64_t l, const bsrht_opts* opts,
                          int32_t* choice, double* best_ms) {
  const bsrht_opts o = opts_or_default(opts);
  if (!A || m < 1 || n < 1 || p < 1 || l < 1) return BSRHT_EINVAL;
  {
    const int ps = precision_auto_only(o);
    if (ps != BSRHT_OK) return ps;
  }
  const size_t wb = sketch_autotune_work_bytes(o.dtype, n, m, o.lda, p, l);
  const size_t ob = (size_t)l * (size_t)m * (o.dtype == BSRHT_F64 ? 8 : 4);
  const size_t wpad = (wb + 255) / 256 * 256;
  void* base = nullptr;
  int st = pool_get(wpad + ob, &base);
  if (st != BSRHT_OK) return st;
  int c = -1;
  double t = 0.0;
  st = sketch_autotune(A, o.dtype, n, m, o.lda, p, l, base, wb, static_cast<char*>(base) + wpad,
                       static_cast<cudaStream_t>(o.stream), &c, &t);
  if (st != BSRHT_OK) return st;
  if (choice) *choice = c;
  if (best_ms) *best_ms = t;
  return BSRHT_OK;
}

int bsrht_sketch_autotune_reset(void) {
  sketch_autotune_reset();
  return BSRHT_OK;
}

int bsrht_release_pool(void) {
  int dev = 0;
  BSRHT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return BSRHT_EUNSUP;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (g_pool[dev].ptr) cudaFree(g_pool[dev].ptr);
  g_pool[dev] = Pool();
  return BSRHT_OK;
}

}  // extern "C"
