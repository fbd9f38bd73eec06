// Host planning and launch of the block SRHT sketch.
#include <algorithm>
#include <atomic>

#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "sketch.cuh"
#include "sketch_kernels.cuh"

namespace bsrht {

int num_sms() {
  // Per-device cache; host threads may plan at the same time, so the
  // entries are atomics (every writer stores the same value).
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int v = cached[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 152;
    }
    cached[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static int ilog2_host(int64_t v) {
  int k = 0;
  while ((int64_t(1) << (k + 1)) <= v) ++k;
  return k;
}

// The TMA paths need 16-byte aligned rows: base address and row stride.
static bool tma_layout_ok(int dtype, const void* A, int64_t lda) {
  const size_t es = dtype_size(dtype);
  if ((lda * (int64_t)es) % 16 != 0) return false;
  return A == nullptr || (reinterpret_cast<uintptr_t>(A) % 16) == 0;
}

// 16-bit panels are 64-byte rows: pair the panels (TileSched) when there are
// at least two CTAs and two panels; sizes the partial-sum scratch.
static void set_pairing(SketchPlan& pl) {
  pl.paired = (pl.dtype == BSRHT_BF16 || pl.dtype == BSRHT_F16) && pl.G >= 2 && pl.P >= 2 ? 1 : 0;
  size_t slots = (size_t)(pl.G + pl.P);
  if (pl.paired) {
    pl.G &= ~1;
    slots = 2 * (size_t)(pl.G / 2 + (pl.P + 1) / 2);
  }
  pl.part_bytes = align_up(4 * slots * (size_t)pl.jgroup * pl.W, 256);
}

static int make_plan_tma(SketchPlan& pl, bool query_device) {
  pl.path = 2;
  pl.W = 32;
  pl.NT = 512;
  pl.R2 = 512;
  pl.JM = pl.l <= 512 ? 32 : pl.l <= 768 ? 48 : 64;
  pl.NRL = pl.NT / pl.W;
  pl.jgroup = std::min<int64_t>(pl.l, (int64_t)pl.JM * pl.NRL);
  pl.nch = (pl.rb + pl.R2 - 1) / pl.R2;
  pl.C = (int64_t)pl.p * pl.nch;
  pl.P = (pl.m + pl.W - 1) / pl.W;
  pl.T = pl.P * pl.C;
  int occ = query_device ? sketch_occupancy_tma(pl) : 0;
  if (occ <= 0) occ = 1;
  int64_t g = (int64_t)num_sms() * occ;
  pl.G = (int)std::max<int64_t>(1, std::min<int64_t>(g, std::max<int64_t>(pl.T, 1)));
  set_pairing(pl);
  pl.dtab_bytes = align_up(4 * (size_t)pl.p * (size_t)pl.nch * 16, 256);
  pl.dttab_bytes = align_up(8 * (size_t)pl.p * (size_t)((pl.jgroup + 63) / 64), 256);
  pl.work_bytes = pl.part_bytes + 256 + pl.dtab_bytes + pl.dttab_bytes;
  return BSRHT_OK;
}

// FP64 kernel with the exact integer transform: 16-column panels, 512-row
// chunks, sketch-row groups of 256 (l <= 256) or 512.
static int make_plan_f64x(SketchPlan& pl, bool query_device) {
  pl.path = 5;
  pl.W = 16;
  pl.NT = 512;
  pl.R2 = 512;
  pl.JM = pl.l <= 256 ? 8 : 16;
  pl.NRL = 32;
  pl.jgroup = std::min<int64_t>(pl.l, (int64_t)pl.JM * 32);
  pl.nch = (pl.rb + pl.R2 - 1) / pl.R2;
  pl.C = (int64_t)pl.p * pl.nch;
  pl.P = (pl.m + pl.W - 1) / pl.W;
  pl.T = pl.P * pl.C;
  int occ = query_device ? sketch_occupancy_f64x(pl) : 0;
  if (occ <= 0) occ = 1;
  const int64_t g = (int64_t)num_sms() * occ;
  pl.G = (int)std::max<int64_t>(1, std::min<int64_t>(g, std::max<int64_t>(pl.T, 1)));
  pl.paired = 0;
  pl.part_bytes = align_up(8 * (size_t)(pl.G + pl.P) * (size_t)pl.jgroup * pl.W, 256);
  pl.dtab_bytes = align_up(4 * (size_t)pl.p * (size_t)pl.nch * 32, 256);
  pl.dttab_bytes = align_up(8 * (size_t)pl.p * (size_t)((pl.jgroup + 63) / 64), 256);
  pl.work_bytes = pl.part_bytes + 256 + pl.dtab_bytes + pl.dttab_bytes;
  return BSRHT_OK;
}

// Tensor-core kernel (K2): 16-bit inputs, blocks of at least one 512-row
// chunk, TMA-compatible rows.
static bool tc_eligible(const SketchPlan& pl, const void* A) {
  return (pl.dtype == BSRHT_BF16 || pl.dtype == BSRHT_F16) && pl.r >= 512 && tma_layout_ok(pl.dtype, A, pl.lda);
}

static int make_plan_tc(SketchPlan& pl, bool query_device) {
  pl.path = 3;
  pl.variant = BSRHT_VARIANT_TENSOR;
  pl.W = 32;
  pl.NT = 512;
  pl.R2 = 512;
  pl.JM = pl.l <= 512 ? 32 : 64;
  pl.NRL = pl.NT / pl.W;
  pl.jgroup = std::min<int64_t>(pl.l, (int64_t)pl.JM * pl.NRL);
  pl.nch = (pl.rb + pl.R2 - 1) / pl.R2;
  pl.C = (int64_t)pl.p * pl.nch;
  pl.P = (pl.m + pl.W - 1) / pl.W;
  pl.T = pl.P * pl.C;
  int occ = query_device ? sketch_occupancy_tc(pl) : 0;
  if (occ <= 0) occ = 1;
  const int64_t g = (int64_t)num_sms() * occ;
  pl.G = (int)std::max<int64_t>(1, std::min<int64_t>(g, std::max<int64_t>(pl.T, 1)));
  set_pairing(pl);
  pl.dtab_bytes = pl.dttab_bytes = 0;
  pl.work_bytes = pl.part_bytes + 256;  // + the error word
  return BSRHT_OK;
}

// Fills the chunked-kernel fields of pl (common sizes already set) for
// kernel instance inst of the dtype family.
static void plan_chunked(SketchPlan& pl, int inst, bool query_device) {
  const bool f64 = pl.dtype == BSRHT_F64;
  pl.path = 0;
  pl.inst = inst;
  const K1Inst k = f64 ? kInstF64[inst] : kInstF32[inst];
  pl.W = f64 ? kW64 : kW32;
  pl.NT = k.NT;
  pl.R2 = k.R2;
  pl.JM = k.JM;
  pl.NRL = pl.NT / pl.W;
  const int64_t jg = (int64_t)pl.JM * pl.NRL;
  pl.jgroup = std::min<int64_t>(pl.l, jg);
  pl.nch = (pl.rb + pl.R2 - 1) / pl.R2;
  pl.C = (int64_t)pl.p * pl.nch;
  pl.P = (pl.m + pl.W - 1) / pl.W;
  pl.T = pl.P * pl.C;
  const size_t elem = f64 ? 8 : 4;
  pl.smem = elem * (size_t)pl.R2 * pl.W + 8 * (size_t)jg + 8 * (size_t)(jg / 64 + std::max(1, pl.R2 / 64));
  int occ = 0;
  if (query_device) occ = f64 ? sketch_occupancy_f64(pl) : sketch_occupancy_f32(pl);
  if (occ <= 0) {
    const size_t smem_sm = 228 * 1024;
    occ = (int)std::max<size_t>(1, std::min<size_t>(2048 / pl.NT, smem_sm / (pl.smem + 1024)));
  }
  int64_t g = (int64_t)num_sms() * occ;
  if (pl.T == 0) g = 1;
  pl.G = (int)std::max<int64_t>(1, std::min<int64_t>(g, std::max<int64_t>(pl.T, 1)));
  pl.part_bytes = align_up(elem * (size_t)(pl.G + pl.P) * (size_t)pl.jgroup * pl.W, 256);
  pl.work_bytes = pl.part_bytes;
}

static int n_instances(bool f64) {
  return f64 ? (int)(sizeof(kInstF64) / sizeof(kInstF64[0])) : (int)(sizeof(kInstF32) / sizeof(kInstF32[0]));
}

// ------------------------------------------------------------ tuned choices
namespace {
struct TuneKey {
  int dtype, log2r, log2m, big_l, tma_rows;
  bool operator<(const TuneKey& o) const {
    return std::tie(dtype, log2r, log2m, big_l, tma_rows) < std::tie(o.dtype, o.log2r, o.log2m, o.big_l, o.tma_rows);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;

TuneKey tune_key(int dtype, int64_t r, int64_t m, int64_t l, int64_t lda) {
  TuneKey k;
  k.dtype = dtype;
  k.log2r = ilog2_host(r);
  int lm = 0;
  while ((int64_t(1) << lm) < std::max<int64_t>(m, 1)) ++lm;
  k.log2m = lm;
  k.big_l = l > 512 ? 1 : 0;
  k.tma_rows = tma_layout_ok(dtype, nullptr, lda) ? 1 : 0;
  return k;
}
}  // namespace

// Built-in chunked instance: the largest chunk R2 <= min(r, 1024).
static int default_instance(bool f64, int64_t r, int64_t l) {
  const int64_t r2t = std::min<int64_t>(r, 1024);
  if (!f64) {
    if (r2t == 1024) return l <= 512 ? 0 : 1;
    return r2t == 512 ? 1 : r2t == 256 ? 2 : r2t == 128 ? 3 : r2t == 64 ? 4 : r2t == 32 ? 5 : 6;
  }
  return r2t == 1024 ? 0 : r2t == 512 ? 1 : r2t == 256 ? 2 : r2t == 128 ? 3 : 4;
}

// choice: -3 = tensor-core kernel, -2 = built-in rules, -1 = TMA-fed kernel,
// >= 0 = chunked instance.
static int make_plan_choice(SketchPlan& pl, int dtype, int64_t n, int64_t m, int64_t lda, int p, int64_t l,
                            bool query_device, const void* A, int choice) {
  pl = SketchPlan();
  pl.dtype = dtype;
  pl.variant = BSRHT_VARIANT_CUDACORE;
  pl.n = n;
  pl.m = m;
  pl.lda = lda;
  pl.p = p;
  pl.l = l;
  pl.rb = (n + p - 1) / p;
  pl.r = 1;
  while (pl.r < pl.rb) pl.r <<= 1;
  const bool f64 = dtype == BSRHT_F64;
  const int64_t rmin = f64 ? 64 : 16;
  if (pl.r < rmin) {
    pl.path = 1;
    pl.jgroup = l;
    pl.W = 32;
    pl.work_bytes = 0;
    return BSRHT_OK;
  }
  if (choice == -3) {
    if (!tc_eligible(pl, A)) return BSRHT_EINVAL;
    return make_plan_tc(pl, query_device);
  }
  int inst = default_instance(f64, pl.r, l);
  if (choice >= 0) {
    if (choice >= n_instances(f64)) return BSRHT_EINVAL;
    const K1Inst k = f64 ? kInstF64[choice] : kInstF32[choice];
    if (k.R2 > pl.r) return BSRHT_EINVAL;
    inst = choice;
  }
  plan_chunked(pl, inst, query_device);
  // Inputs with blocks of at least one 512-row chunk and TMA-compatible rows
  // take the TMA-fed kernel (FP64: the one with the integer transform)
  // unless a chunked instance was chosen; the plain kernel stays the
  // fallback, so a plan made without A reserves scratch for both.
  // (The TMA kernels count a panel's chunks in 32 bits.)
  const bool tma_ok = pl.r >= 512 && tma_layout_ok(dtype, A, lda) && (int64_t)p * ((pl.rb + 511) / 512) < INT32_MAX;
  if (choice == -1 && !(tma_ok || (A == nullptr && pl.r >= 512 && tma_layout_ok(dtype, nullptr, lda))))
    return BSRHT_EINVAL;
  if (tma_ok && choice < 0) {
    SketchPlan t = pl;
    if (f64)
      make_plan_f64x(t, query_device);
    else
      make_plan_tma(t, query_device);
    const size_t plain = pl.work_bytes;
    pl = t;
    if (A == nullptr) pl.work_bytes = std::max(pl.work_bytes, plain);
  }
  return BSRHT_OK;
}

int sketch_make_plan(SketchPlan& pl, int dtype, int variant, int64_t n, int64_t m, int64_t lda,
                     int p, int64_t l, bool query_device, const void* A) {
  if ((dtype < BSRHT_F64 || dtype > BSRHT_F16) && dtype != kDtypeF32AsF64) return BSRHT_EINVAL;
  if (n < 1 || m < 0 || p < 1 || (int64_t)p > n || l < 1 || l > n) return BSRHT_EINVAL;
  if (lda == 0) lda = m;
  if (lda < m) return BSRHT_EINVAL;
  if (dtype == kDtypeF32AsF64) {
    // FP32 A, FP64 arithmetic: only the TMA-fed integer-transform kernel
    // (blocks of at least one 512-row chunk, 16-byte aligned rows).
    if (variant != BSRHT_VARIANT_AUTO && variant != BSRHT_VARIANT_CUDACORE) return BSRHT_EUNSUP;
    const int st = make_plan_choice(pl, BSRHT_F64, n, m, lda, p, l, query_device, nullptr, -2);
    if (st != BSRHT_OK) return st;
    const bool tma_ok = pl.r >= 512 && tma_layout_ok(dtype, A, lda) && (int64_t)p * ((pl.rb + 511) / 512) < INT32_MAX;
    if (!tma_ok) return BSRHT_EUNSUP;
    pl.dtype = dtype;
    return make_plan_f64x(pl, query_device);
  }
  int64_t rb = (n + p - 1) / p, r = 1;
  while (r < rb) r <<= 1;
  if (variant == BSRHT_VARIANT_GAUSSIAN) return gaussian_plan(pl, dtype, n, m, lda, p, l);
  if (variant < BSRHT_VARIANT_AUTO || variant > BSRHT_VARIANT_GAUSSIAN) return BSRHT_EINVAL;
  if (variant == BSRHT_VARIANT_TENSOR) {
    // K2 only: 16-bit A, r >= 512, TMA-compatible rows.
    const int st = make_plan_choice(pl, dtype, n, m, lda, p, l, query_device, A, -3);
    return st == BSRHT_OK && pl.path == 3 ? BSRHT_OK : BSRHT_EUNSUP;
  }
  int choice = -2;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(tune_key(dtype, r, m, l, lda));
    if (it != g_tuned.end()) choice = it->second;
  }
  int st = make_plan_choice(pl, dtype, n, m, lda, p, l, query_device, A, choice);
  if (st != BSRHT_OK && choice != -2) st = make_plan_choice(pl, dtype, n, m, lda, p, l, query_device, A, -2);
  if (st == BSRHT_OK && A == nullptr && pl.path != 1) {
    // Scratch sized without A must also hold whatever plan the autotuner
    // records for this shape class before the run: reserve the largest.
    const bool f64 = dtype == BSRHT_F64;
    for (int c = -3; c < n_instances(f64); ++c) {
      SketchPlan alt;
      if (c != -2 && make_plan_choice(alt, dtype, n, m, lda, p, l, query_device, nullptr, c) == BSRHT_OK)
        pl.work_bytes = std::max(pl.work_bytes, alt.work_bytes);
    }
  }
  return st;
}

int sketch_autotune(const void* A, int dtype, int64_t n, int64_t m, int64_t lda, int p, int64_t l, void* work,
                    size_t work_bytes, void* out, cudaStream_t stream, int* choice_out, double* best_ms) {
  if (dtype < BSRHT_F64 || dtype > BSRHT_F16) return BSRHT_EINVAL;
  if (n < 1 || m < 1 || p < 1 || (int64_t)p > n || l < 1 || l > n) return BSRHT_EINVAL;
  if (lda == 0) lda = m;
  if (lda < m) return BSRHT_EINVAL;
  const bool f64 = dtype == BSRHT_F64;
  std::vector<int> cands;
  if (dtype == BSRHT_BF16 || dtype == BSRHT_F16) cands.push_back(-3);
  cands.push_back(-1);
  for (int i = 0; i < n_instances(f64); ++i) cands.push_back(i);
  cudaEvent_t e0, e1;
  BSRHT_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return BSRHT_ECUDA;
  }
  int best = -2;
  double best_t = 1e300;
  int st = BSRHT_OK;
  for (int c : cands) {
    SketchPlan pl;
    if (make_plan_choice(pl, dtype, n, m, lda, p, l, true, A, c) != BSRHT_OK) continue;
    if ((c == -1 && pl.path != 2 && pl.path != 5) || (c == -3 && pl.path != 3)) continue;
    if (pl.path == 1) {  // nothing to choose for tiny blocks
      best = -2;
      break;
    }
    if (pl.work_bytes > work_bytes) continue;
    double t_min = 1e300;
    for (int rep = 0; rep < 3 && st == BSRHT_OK; ++rep) {
      if (cudaEventRecord(e0, stream) != cudaSuccess) st = BSRHT_ECUDA;
      if (st == BSRHT_OK) st = sketch_run(pl, A, 0, out, m, work, stream);
      if (st == BSRHT_OK && cudaEventRecord(e1, stream) != cudaSuccess) st = BSRHT_ECUDA;
      if (st == BSRHT_OK && cudaEventSynchronize(e1) != cudaSuccess) st = BSRHT_ECUDA;
      float ms = 0.f;
      if (st == BSRHT_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = BSRHT_ECUDA;
      if (st == BSRHT_OK && rep > 0) t_min = std::min(t_min, (double)ms);  // rep 0 warms up
    }
    if (st != BSRHT_OK) break;
    if (t_min < best_t) {
      best_t = t_min;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BSRHT_OK) return st;
  int64_t rb = (n + p - 1) / p, r = 1;
  while (r < rb) r <<= 1;
  if (best != -2) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[tune_key(dtype, r, m, l, lda)] = best;
  }
  if (choice_out) *choice_out = best == -2 ? -1 : best;
  if (best_ms) *best_ms = best == -2 ? 0.0 : best_t;
  return BSRHT_OK;
}

size_t sketch_autotune_work_bytes(int dtype, int64_t n, int64_t m, int64_t lda, int p, int64_t l) {
  size_t w = 0;
  const bool f64 = dtype == BSRHT_F64;
  for (int c = -3; c < n_instances(f64); ++c) {
    SketchPlan pl;
    if (c != -2 && make_plan_choice(pl, dtype, n, m, lda == 0 ? m : lda, p, l, true, nullptr, c) == BSRHT_OK)
      w = std::max(w, pl.work_bytes);
  }
  return w;
}

void sketch_autotune_reset() {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned.clear();
}

int sketch_run(const SketchPlan& pl, const void* A, uint64_t seed, void* out, int64_t ldo, void* work,
               cudaStream_t stream) {
  if (pl.m == 0) return BSRHT_OK;
  if (pl.path == 4) return gaussian_run(pl, A, seed, out, ldo, work, stream);
  if (pl.path != 1 && pl.work_bytes > 0 && work == nullptr) return BSRHT_ENOMEM;
  for (int64_t j0 = 0; j0 < pl.l; j0 += pl.jgroup) {
    SketchArgs a;
    a.A = A;
    a.lda = pl.lda;
    a.n = pl.n;
    a.m = pl.m;
    a.rb = pl.rb;
    a.r = pl.r;
    a.p = pl.p;
    a.j0 = j0;
    a.jn = std::min<int64_t>(pl.jgroup, pl.l - j0);
    a.seed = seed;
    a.nch = pl.nch;
    a.C = pl.C;
    a.T = pl.T;
    a.G = pl.G;
    a.part = work;
    a.toff = 0;
    a.Tg = pl.T;
    a.Gg = pl.G;
    a.gfirst = 0;
    a.out = out;
    a.ldo = ldo;
    a.scale = 1.0 / std::sqrt((double)pl.l);
    a.paired = (pl.path == 2 || pl.path == 3) ? pl.paired : 0;
    a.P = pl.P;
    int st;
    if (pl.path == 3) {
      int* err = reinterpret_cast<int*>(static_cast<char*>(work) + pl.part_bytes);
      if (j0 == 0) BSRHT_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), stream));
      st = sketch_launch_tc(pl, a, out, ldo, err, stream);
    } else if (pl.path == 2 || pl.path == 5) {
      char* w = static_cast<char*>(work);
      int* err = reinterpret_cast<int*>(w + pl.part_bytes);
      uint64_t* dtab = reinterpret_cast<uint64_t*>(w + pl.part_bytes + 256);
      uint64_t* dttab = reinterpret_cast<uint64_t*>(w + pl.part_bytes + 256 + pl.dtab_bytes);
      if (j0 == 0) BSRHT_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), stream));
      st = pl.path == 5 ? sketch_launch_f64x(pl, a, out, ldo, err, dtab, dttab, stream)
                        : sketch_launch_tma(pl, a, out, ldo, err, dtab, dttab, stream);
    } else {
      st = pl.dtype == BSRHT_F64 ? sketch_launch_f64(pl, a, out, ldo, stream)
                                 : sketch_launch_f32(pl, a, out, ldo, stream);
    }
    if (st != BSRHT_OK) return st;
  }
  return BSRHT_OK;
}

// ------------------------------------------------------------ grouped launches
// A grouped sketch uses the plain chunked kernel (path 0) of its dtype family
// and must fit one sketch-row group (l <= jgroup).
int sketch_make_plan_grouped(SketchPlan& pl, int dtype, int64_t n, int64_t m, int64_t lda, int p, int64_t l) {
  // Planning without A keeps path 0 unless the TMA path applies; redo the
  // plan as the plain kernel in that case.
  int st = sketch_make_plan(pl, dtype, BSRHT_VARIANT_CUDACORE, n, m, lda, p, l, true, nullptr);
  if (st != BSRHT_OK) return st;
  if (pl.path == 2 || pl.path == 5) {
    // Same sizes through the plain kernel: plan with an address the TMA
    // rules reject (odd), which only steers the path choice.
    st = sketch_make_plan(pl, dtype, BSRHT_VARIANT_CUDACORE, n, m, lda, p, l, true,
                          reinterpret_cast<const void*>(uintptr_t(1)));
    if (st != BSRHT_OK) return st;
  }
  if (pl.path != 0 || pl.jgroup < pl.l) return BSRHT_EUNSUP;
  return BSRHT_OK;
}

size_t sketch_group_work_bytes(const SketchPlan& pl) {
  // A sketch in a grouped launch is touched by at most min(G_max, T + 1)
  // CTAs (G_max = the launch's CTA count, bounded by the SMs' residency).
  const int occ = pl.dtype == BSRHT_F64 ? sketch_occupancy_f64(pl) : sketch_occupancy_f32(pl);
  const int64_t gmax = (int64_t)num_sms() * std::max(occ, 1);
  const int64_t gq = std::min<int64_t>(gmax, pl.T + 1);
  const size_t elem = pl.dtype == BSRHT_F64 ? 8 : 4;
  return align_up(elem * (size_t)(gq + pl.P) * (size_t)pl.jgroup * pl.W, 256);
}

int sketch_group_run(const SketchPlan* const* plans, const void* const* A, const uint64_t* seeds, void* const* outs,
                     void* const* works, int nreq, cudaStream_t stream) {
  if (nreq < 1 || nreq > kMaxGroup) return BSRHT_EINVAL;
  const SketchPlan& p0 = *plans[0];
  for (int q = 0; q < nreq; ++q) {
    const SketchPlan& pl = *plans[q];
    if (pl.path != 0 || pl.dtype != p0.dtype || pl.inst != p0.inst || pl.jgroup < pl.l) return BSRHT_EINVAL;
  }
  SketchGroup grp;
  grp.nreq = nreq;
  int64_t Tg = 0;
  for (int q = 0; q < nreq; ++q) Tg += plans[q]->T;
  const int occ = p0.dtype == BSRHT_F64 ? sketch_occupancy_f64(p0) : sketch_occupancy_f32(p0);
  const int64_t Gg = std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * std::max(occ, 1), std::max<int64_t>(Tg, 1)));
  int64_t toff = 0;
  for (int q = 0; q < nreq; ++q) {
    const SketchPlan& pl = *plans[q];
    SketchArgs& a = grp.r[q];
    a.A = A[q];
    a.lda = pl.lda;
    a.n = pl.n;
    a.m = pl.m;
    a.rb = pl.rb;
    a.r = pl.r;
    a.p = pl.p;
    a.j0 = 0;
    a.jn = pl.l;
    a.seed = seeds[q];
    a.nch = pl.nch;
    a.C = pl.C;
    a.T = pl.T;
    a.G = pl.G;
    a.part = works[q];
    a.toff = toff;
    a.Tg = Tg;
    a.Gg = (int)Gg;
    // First CTA whose tile range reaches this sketch's first tile.
    int64_t c = toff * Gg / std::max<int64_t>(Tg, 1);
    while (c > 0 && c * Tg / Gg > toff) --c;
    while (c + 1 < Gg && (c + 1) * Tg / Gg <= toff) ++c;
    a.gfirst = (int)c;
    a.out = outs[q];
    a.ldo = pl.m;
    a.scale = 1.0 / std::sqrt((double)pl.l);
    a.paired = 0;
    a.P = pl.P;
    toff += pl.T;
  }
  int64_t maxel = 0;
  for (int q = 0; q < nreq; ++q) maxel = std::max<int64_t>(maxel, plans[q]->l * plans[q]->m);
  return p0.dtype == BSRHT_F64 ? sketch_group_launch_f64(p0, grp, (int)Gg, maxel, stream)
                               : sketch_group_launch_f32(p0, grp, (int)Gg, maxel, stream);
}

}  // namespace bsrht
