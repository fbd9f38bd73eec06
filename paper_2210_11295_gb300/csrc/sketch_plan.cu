// Host planning and launch of the block SRHT sketch.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "sketch.cuh"
#include "sketch_kernels.cuh"

namespace bsrht {

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 152;
    }
    cached[dev] = v;
  }
  return cached[dev];
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The TMA path needs 16-byte aligned rows: base address and row stride.
static bool tma_layout_ok(int dtype, const void* A, int64_t lda) {
  const size_t es = dtype == BSRHT_F32 ? 4 : 2;
  if ((lda * (int64_t)es) % 16 != 0) return false;
  return A == nullptr || (reinterpret_cast<uintptr_t>(A) % 16) == 0;
}

static int make_plan_tma(SketchPlan& pl, bool query_device) {
  pl.path = 2;
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
  int occ = query_device ? sketch_occupancy_tma(pl) : 0;
  if (occ <= 0) occ = 1;
  int64_t g = (int64_t)num_sms() * occ;
  pl.G = (int)std::max<int64_t>(1, std::min<int64_t>(g, std::max<int64_t>(pl.T, 1)));
  pl.part_bytes = align_up(4 * (size_t)(pl.G + pl.P) * (size_t)pl.jgroup * pl.W, 256);
  pl.dtab_bytes = align_up(4 * (size_t)pl.p * (size_t)pl.nch * 16, 256);
  pl.dttab_bytes = align_up(8 * (size_t)pl.p * (size_t)((pl.jgroup + 63) / 64), 256);
  pl.work_bytes = pl.part_bytes + 256 + pl.dtab_bytes + pl.dttab_bytes;
  return BSRHT_OK;
}

int sketch_make_plan(SketchPlan& pl, int dtype, int variant, int64_t n, int64_t m, int64_t lda,
                     int p, int64_t l, bool query_device, const void* A) {
  if (dtype < BSRHT_F64 || dtype > BSRHT_F16) return BSRHT_EINVAL;
  if (n < 1 || m < 0 || p < 1 || (int64_t)p > n || l < 1 || l > n) return BSRHT_EINVAL;
  if (lda == 0) lda = m;
  if (lda < m) return BSRHT_EINVAL;
  if (variant == BSRHT_VARIANT_TENSOR) return BSRHT_EUNSUP;
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
  const int64_t r2max = 1024;
  const int64_t r2t = std::min<int64_t>(pl.r, r2max);
  const int64_t rmin = f64 ? 64 : 16;
  if (pl.r < rmin) {
    pl.path = 1;
    pl.jgroup = l;
    pl.W = 32;
    pl.work_bytes = 0;
    return BSRHT_OK;
  }
  pl.path = 0;
  if (!f64) {
    pl.W = kW32;
    if (r2t == 1024)
      pl.inst = (l <= 512) ? 0 : 1;
    else
      pl.inst = r2t == 512 ? 1 : r2t == 256 ? 2 : r2t == 128 ? 3 : r2t == 64 ? 4 : r2t == 32 ? 5 : 6;
    const K1Inst k = kInstF32[pl.inst];
    pl.NT = k.NT;
    pl.R2 = k.R2;
    pl.JM = k.JM;
  } else {
    pl.W = kW64;
    pl.inst = r2t == 1024 ? 0 : r2t == 512 ? 1 : r2t == 256 ? 2 : r2t == 128 ? 3 : 4;
    const K1Inst k = kInstF64[pl.inst];
    pl.NT = k.NT;
    pl.R2 = k.R2;
    pl.JM = k.JM;
  }
  pl.NRL = pl.NT / pl.W;
  const int64_t jg = (int64_t)pl.JM * pl.NRL;
  pl.jgroup = std::min<int64_t>(l, jg);
  pl.nch = (pl.rb + pl.R2 - 1) / pl.R2;
  pl.C = (int64_t)p * pl.nch;
  pl.P = (m + pl.W - 1) / pl.W;
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
  // FP32-arithmetic inputs with blocks of at least one 512-row chunk and
  // TMA-compatible rows take the TMA-fed kernel; the plain kernel stays the
  // fallback, so a plan made without A reserves scratch for both.
  if (!f64 && pl.r >= 512 && tma_layout_ok(dtype, A, lda)) {
    SketchPlan t = pl;
    make_plan_tma(t, query_device);
    const size_t plain = pl.work_bytes;
    pl = t;
    if (A == nullptr) pl.work_bytes = std::max(pl.work_bytes, plain);
  }
  return BSRHT_OK;
}

int sketch_run(const SketchPlan& pl, const void* A, uint64_t seed, void* out, int64_t ldo, void* work,
               cudaStream_t stream) {
  if (pl.m == 0) return BSRHT_OK;
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
    int st;
    if (pl.path == 2) {
      char* w = static_cast<char*>(work);
      int* err = reinterpret_cast<int*>(w + pl.part_bytes);
      uint64_t* dtab = reinterpret_cast<uint64_t*>(w + pl.part_bytes + 256);
      uint64_t* dttab = reinterpret_cast<uint64_t*>(w + pl.part_bytes + 256 + pl.dtab_bytes);
      if (j0 == 0) BSRHT_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), stream));
      st = sketch_launch_tma(pl, a, out, ldo, err, dtab, dttab, stream);
    } else {
      st = pl.dtype == BSRHT_F64 ? sketch_launch_f64(pl, a, out, ldo, stream)
                                 : sketch_launch_f32(pl, a, out, ldo, stream);
    }
    if (st != BSRHT_OK) return st;
  }
  return BSRHT_OK;
}

}  // namespace bsrht
