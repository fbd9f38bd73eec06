// Gaussian-embedding sketch: the comparator the paper validates the block
// SRHT against (Sec. 4; Gaussian matrices are among the classical oblivious
// subspace embeddings of Sec. 1).  Omega_G (l x n) has independent N(0, 1/l)
// entries and the sketch is B = Omega_G A, a dense product of 2 l n m flops
// where the block SRHT needs n m (log2 R2 + l / R2) additions.
//
// Omega_G is generated into scratch by a counter-based kernel and the
// product runs on the tcgen05 3xTF32 GEMM (FP32 accuracy); A (n x m,
// row-major) is the GEMM's K x N operand, which the GEMM transposes (and
// splits into TF32 hi/lo) into scratch first: n m 8 bytes, the price of a
// dense Gaussian sketch on this layout.
//
// Entries: Philox4x64-10 (common.cuh) with key (seed, 0) and counter
// (k >> 1, j, 3, 0) gives four words for the column pair (2 (k >> 1),
// 2 (k >> 1) + 1) of row j: words 0, 1 for the even column, 2, 3 for the odd
// one.  A word w maps to u = (2 (w >> 41) + 1) 2^-24 in (0, 1), exact in
// FP32, and the Box-Muller transform (Box and Muller, 1958) of (u1, u2),
// z = sqrt(-2 ln u1) cos(2 pi u2), evaluated in FP32, is N(0, 1).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "dla.cuh"
#include "sketch.cuh"

namespace bsrht {
namespace {

constexpr uint64_t kStreamG = 3;

__device__ __forceinline__ float gauss_uniform(uint64_t w) {
  return (float)(2u * (uint32_t)(w >> 41) + 1u) * 0x1.0p-24f;
}

// Box-Muller in the output type: FP32 for the comparator's Omega_G, FP64
// where the map enters an FP64 computation.
__device__ __forceinline__ float box_muller(uint64_t a, uint64_t b, float) {
  const float u1 = gauss_uniform(a), u2 = gauss_uniform(b);
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}
__device__ __forceinline__ double box_muller(uint64_t a, uint64_t b, double) {
  const double u1 = (double)gauss_uniform(a), u2 = (double)gauss_uniform(b);
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// Om[j][k] (row stride ldo, ldo even) for j < l, k < n; columns [n, ldo)
// are zeroed.  One thread per column pair of a row: one Philox block, one
// paired store.
template <typename T>
__global__ void k_gaussian_omega(T* __restrict__ Om, int64_t l, int64_t n, int64_t ldo, uint64_t seed, T scale) {
  const int64_t npair = ldo / 2;
  const int64_t total = l * npair;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / npair, q = e - j * npair;
    T v0 = T(0), v1 = T(0);
    if (2 * q < n) {
      const U64x4 w = philox4x64_10(U64x4{(uint64_t)q, (uint64_t)j, kStreamG, 0}, seed, 0);
      v0 = scale * box_muller(w.x, w.y, T(0));
      if (2 * q + 1 < n) v1 = scale * box_muller(w.z, w.w, T(0));
    }
    Om[j * ldo + 2 * q] = v0;
    Om[j * ldo + 2 * q + 1] = v1;
  }
}

int64_t omega_ld(int64_t n) { return (n + 3) / 4 * 4; }

size_t omega_bytes(int64_t n, int64_t l) { return ((size_t)l * (size_t)omega_ld(n) * 4 + 255) / 256 * 256; }

}  // namespace

int gaussian_plan(SketchPlan& pl, int dtype, int64_t n, int64_t m, int64_t lda, int p, int64_t l) {
  if (dtype != BSRHT_F32) return BSRHT_EUNSUP;  // the comparator runs the FP32 benchmark data
  if (n < 8) return BSRHT_EUNSUP;                // the tensor-core product wants K >= 8
  pl = SketchPlan{};
  pl.dtype = dtype;
  pl.variant = BSRHT_VARIANT_GAUSSIAN;
  pl.path = 4;
  pl.n = n;
  pl.m = m;
  pl.lda = lda;
  pl.p = p;
  pl.l = l;
  pl.jgroup = l;
  Arena meas;
  meas.measure = true;
  const Dla d{nullptr, nullptr};
  const int st = gemm_tc(d, meas, l, m, n, nullptr, omega_ld(n), DT::F32, nullptr, lda, false, DT::F32, nullptr, m,
                         false);
  if (st != BSRHT_OK) return st;
  pl.part_bytes = omega_bytes(n, l);
  pl.work_bytes = pl.part_bytes + meas.high + 256;
  return BSRHT_OK;
}

int gaussian_run(const SketchPlan& pl, const void* A, uint64_t seed, void* out, int64_t ldo, void* work,
                 cudaStream_t stream) {
  if (pl.m == 0) return BSRHT_OK;
  if (work == nullptr) return BSRHT_ENOMEM;
  if (!gemm_tc_eligible(pl.l, pl.m, pl.n, work, omega_ld(pl.n))) return BSRHT_EUNSUP;
  float* om = static_cast<float*>(work);
  const int64_t ld = omega_ld(pl.n);
  const int64_t total = pl.l * (ld / 2);
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 16);
  k_gaussian_omega<float><<<blocks, 256, 0, stream>>>(om, pl.l, pl.n, ld, seed,
                                                      (float)(1.0 / std::sqrt((double)pl.l)));
  BSRHT_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  Arena ar;
  ar.base = static_cast<char*>(work) + pl.part_bytes;
  ar.cap = pl.work_bytes - pl.part_bytes;
  const Dla d{stream, nullptr};
  return gemm_tc(d, ar, pl.l, pl.m, pl.n, om, ld, DT::F32, A, pl.lda, false, DT::F32, out, ldo, false);
}

int gaussian_omega(cudaStream_t stream, DT t, void* out, int64_t rows, int64_t cols, int64_t ld, uint64_t seed,
                   double scale) {
  if (rows <= 0 || cols <= 0) return BSRHT_OK;
  if ((ld & 1) || ld < cols) return BSRHT_EINVAL;
  const int64_t total = rows * (ld / 2);
  const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 16);
  if (t == DT::F64)
    k_gaussian_omega<double><<<blocks, 256, 0, stream>>>(static_cast<double*>(out), rows, cols, ld, seed, scale);
  else if (t == DT::F32)
    k_gaussian_omega<float><<<blocks, 256, 0, stream>>>(static_cast<float*>(out), rows, cols, ld, seed,
                                                        (float)scale);
  else
    return BSRHT_EUNSUP;
  BSRHT_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return BSRHT_OK;
}

}  // namespace bsrht
