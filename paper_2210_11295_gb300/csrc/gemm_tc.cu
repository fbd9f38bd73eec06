// Host side of the tcgen05 3xTF32 GEMM (gemm_tc.cuh).
#include <algorithm>

#include "dla.cuh"
#include "gemm_tc.cuh"
#include "sketch.cuh"

namespace bsrht {

#define TRY_TC(expr)                   \
  do {                                 \
    const int st_ = (expr);            \
    if (st_ != BSRHT_OK) return st_;   \
  } while (0)

namespace {

// Bt[n][k] = B[k][n] in FP32 (B is K x N, FP32 or FP64, leading dimension
// ldb); columns k in [K, ldk) are zero.  With Blo != nullptr also
// Blo[n][k] = Bt[n][k] - (Bt[n][k] with the low 13 mantissa bits cleared),
// the lo part of the TF32 split.  64 x 64 tiles through shared memory (16
// elements per thread in flight), a 1-D grid of tiles (tiles_n per row of
// tiles).
template <typename TB>
__global__ void __launch_bounds__(256) k_transpose_f32(const TB* __restrict__ B, int64_t K, int64_t N, int64_t ldb,
                                                       float* __restrict__ Bt, int64_t ldk, float* __restrict__ Blo,
                                                       int64_t tiles_n) {
  __shared__ float tile[64][65];
  const int64_t tk = (int64_t)blockIdx.x / tiles_n, tnb = (int64_t)blockIdx.x - tk * tiles_n;
  const int64_t k0 = tk * 64, nb = tnb * 64;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
#pragma unroll
  for (int r = ty; r < 64; r += 8) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t k = k0 + r, n = nb + tx + 32 * h;
      tile[r][tx + 32 * h] = (k < K && n < N) ? (float)B[k * ldb + n] : 0.f;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = ty; r < 64; r += 8) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t n = nb + r, k = k0 + tx + 32 * h;
      if (n < N && k < ldk) {
        const float x = tile[tx + 32 * h][r];
        Bt[n * ldk + k] = x;
        if (Blo) Blo[n * ldk + k] = x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
      }
    }
  }
}

// Fixed-order sum of the split-K partials; for a Gram product the tiles
// skipped below the diagonal are read from their mirror images.
template <typename TC>
__global__ void k_tc_reduce(const float* __restrict__ P, TC* __restrict__ C, int64_t M, int64_t N, int64_t ldc,
                            int splits, int gram, int tile_n, float* __restrict__ Ct, int64_t ldct) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  const int64_t i = idx / N, j = idx - i * N;
  int64_t si = i, sj = j;
  if (gram && tc::tile_below_diagonal(i / tc::BM, j / tile_n, tile_n)) {
    si = j;
    sj = i;
  }
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += (double)P[(int64_t)z * M * N + si * N + sj];
  C[i * ldc + j] = (TC)s;
  if (Ct) Ct[j * ldct + i] = (float)(TC)s;
}

template <typename TC, bool PRE, int BNT>
int launch_tc(const Dla& d, const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mblo, tc::GemmTcArgs g,
              dim3 grid) {
  const size_t smem = tc::Cfg<BNT>::smem_bytes();
  auto kern = tc::k_gemm_tf32x3<TC, PRE, BNT>;
  BSRHT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, tc::Cfg<BNT>::THREADS, smem, d.s>>>(ma, mb, mblo, g);
  BSRHT_CUDA_TRY(cudaGetLastError());
  return BSRHT_OK;
}

template <int BNT>
int launch_tc_any(const Dla& d, bool pre, bool f32_out, const CUtensorMap& ma, const CUtensorMap& mb,
                  const CUtensorMap& mblo, tc::GemmTcArgs g, dim3 grid) {
  return pre ? (f32_out ? launch_tc<float, true, BNT>(d, ma, mb, mblo, g, grid)
                        : launch_tc<double, true, BNT>(d, ma, mb, mblo, g, grid))
             : (f32_out ? launch_tc<float, false, BNT>(d, ma, mb, mblo, g, grid)
                        : launch_tc<double, false, BNT>(d, ma, mb, mblo, g, grid));
}

// Tile width.  256 halves the shared-memory operand traffic per flop, but
// its 64-byte K rows suit only operands whose rows are close together:
// measured on GB300, A Q (K = 4096) 21.0 -> 17.9 ms, while the products
// with K = n (the Grams, the Gaussian sketch: K-major rows megabytes apart)
// slowed down (Gaussian sketch 53.6 -> 75.9 ms), and a Gram skips less work
// in wider tiles.  So 256 only for plain products with
// K <= 16384 and a full B (a triangular B skips less work in wide tiles: the
// tall QR's W R1^-1 measured no faster), and only if padding N to 256 wastes
// at most N / 8 columns.
int tile_width(int64_t N, int64_t K, bool gram, bool b_upper) {
  if (gram || b_upper || K > 16384 || N < 256) return 128;
  const int64_t pad256 = (N + 255) / 256 * 256 - N;
  return 8 * pad256 <= N ? 256 : 128;
}

}  // namespace

bool gemm_tc_eligible(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda) {
  return M >= 1 && N >= 1 && K >= 8 && (lda % 4) == 0 && (reinterpret_cast<uintptr_t>(A) % 16) == 0;
}

int transpose_to_f32(const Dla& d, DT tb, const void* B, int64_t K, int64_t N, int64_t ldb, float* Bt, int64_t ldk,
                     float* Blo) {
  const int64_t tiles_n = (N + 63) / 64, tiles = tiles_n * ((ldk + 63) / 64);
  if (tiles > 0x7FFFFFFF) return BSRHT_EUNSUP;
  const unsigned g = (unsigned)tiles;
  if (tb == DT::F32)
    k_transpose_f32<float><<<g, 256, 0, d.s>>>(static_cast<const float*>(B), K, N, ldb, Bt, ldk, Blo, tiles_n);
  else if (tb == DT::F64)
    k_transpose_f32<double><<<g, 256, 0, d.s>>>(static_cast<const double*>(B), K, N, ldb, Bt, ldk, Blo, tiles_n);
  else
    return BSRHT_EUNSUP;
  BSRHT_CUDA_TRY(cudaGetLastError());
  note_launches(1);
  return BSRHT_OK;
}

int gemm_tc(const Dla& d, Arena& ar, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, DT tb,
            const void* B, int64_t ldb, bool b_kmajor, DT tc_out, void* C, int64_t ldc, bool gram, bool b_upper,
            float* Ct) {
  if (M <= 0 || N <= 0) return BSRHT_OK;
  if (tc_out != DT::F32 && tc_out != DT::F64) return BSRHT_EUNSUP;
  if (Ct && (gram || tc_out != DT::F32)) return BSRHT_EINVAL;
  const float* Bt = static_cast<const float*>(B);
  const float* Btlo = nullptr;
  int64_t ldk = ldb;
  if (!b_kmajor) {
    ldk = (K + 3) / 4 * 4;
    float* bt = static_cast<float*>(ar.take(sizeof(float) * (size_t)N * ldk));
    float* btlo = static_cast<float*>(ar.take(sizeof(float) * (size_t)N * ldk));
    if (!ar.ok()) return BSRHT_ENOMEM;
    if (!ar.measure) TRY_TC(transpose_to_f32(d, tb, B, K, N, ldb, bt, ldk, btlo));
    Bt = bt;
    Btlo = btlo;
  } else if (tb != DT::F32 || (ldk % 4) != 0) {
    return BSRHT_EUNSUP;
  }
  const int tw = tile_width(N, K, gram, b_upper);
  const int tbk = tw == 128 ? tc::Cfg<128>::BK : tc::Cfg<256>::BK;
  const int64_t tm = (M + tc::BM - 1) / tc::BM, tn = (N + tw - 1) / tw;
  int64_t tiles = 0;
  for (int64_t bm = 0; bm < tm; ++bm)
    for (int64_t bn = 0; bn < tn; ++bn) tiles += (gram && tc::tile_below_diagonal(bm, bn, tw)) ? 0 : 1;
  const int64_t nkb = (K + tbk - 1) / tbk;
  // Split K when the tiles alone do not fill the GPU, and in any case so
  // that no CTA folds more than 256 K blocks into its FP32 running sums.
  int64_t splits = 1;
  const int64_t target = (int64_t)num_sms();
  if (tiles < target && nkb >= 16) splits = std::max<int64_t>(1, std::min<int64_t>((target + tiles - 1) / tiles, nkb / 8));
  splits = std::max<int64_t>(splits, (nkb + 255) / 256);
  if (gram && splits == 1) splits = 2;  // the mirror is applied by the reduce
  splits = std::min<int64_t>(splits, 65535);
  float* P = nullptr;
  if (splits > 1) {
    P = static_cast<float*>(ar.take(sizeof(float) * (size_t)splits * M * N));
    if (!ar.ok()) return BSRHT_ENOMEM;
  }
  int* err = static_cast<int*>(ar.take(256));
  if (!ar.ok()) return BSRHT_ENOMEM;
  if (ar.measure) return BSRHT_OK;
  CUtensorMap ma, mb, mblo;
  // Box: BK x 128 rows of A, BK x tw rows of B^T; rows of BK floats fill the
  // swizzle span (128 bytes for tw = 128, 64 bytes for tw = 256).
  const CUtensorMapSwizzle swz = tw == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  if (!make_tensor_map_2d(&ma, A, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (uint64_t)M, (uint64_t)K, (uint64_t)lda,
                          (uint32_t)tbk, tc::BM, swz) ||
      !make_tensor_map_2d(&mb, Bt, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (uint64_t)N, (uint64_t)K, (uint64_t)ldk,
                          (uint32_t)tbk, (uint32_t)tw, swz))
    return BSRHT_EUNSUP;
  const bool pre = Btlo != nullptr;
  mblo = mb;
  if (pre && !make_tensor_map_2d(&mblo, Btlo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (uint64_t)N, (uint64_t)K,
                                 (uint64_t)ldk, (uint32_t)tbk, (uint32_t)tw, swz))
    return BSRHT_EUNSUP;
  // A failed bounded wait sets kStatusTcWait in the caller's status word when
  // it has one (read back by the low-rank drivers), else in a word of its own.
  static_assert(tc::kErrWait == kStatusTcWait, "status bit");
  if (d.status) {
    err = d.status;
  } else {
    BSRHT_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), d.s));
  }
  if (tm * tn > 0x7FFFFFFF) return BSRHT_EUNSUP;
  dim3 grid((unsigned)(tm * tn), 1u, (unsigned)splits);
  tc::GemmTcArgs g{M,   N,   K,  splits > 1 ? (void*)P : C, ldc, gram ? 1 : 0, err, (b_upper && !gram) ? 1 : 0,
                   splits > 1 ? nullptr : Ct, M};
  const bool f32_out = tc_out == DT::F32 || splits > 1;
  const int st = tw == 128 ? launch_tc_any<128>(d, pre, f32_out, ma, mb, mblo, g, grid)
                           : launch_tc_any<256>(d, pre, f32_out, ma, mb, mblo, g, grid);
  if (st != BSRHT_OK) return st;
  int launches = 1;
  if (splits > 1) {
    const unsigned nb = (unsigned)((M * N + 255) / 256);
    if (tc_out == DT::F32)
      k_tc_reduce<float><<<nb, 256, 0, d.s>>>(P, static_cast<float*>(C), M, N, ldc, (int)splits, gram ? 1 : 0, tw,
                                              Ct, M);
    else
      k_tc_reduce<double><<<nb, 256, 0, d.s>>>(P, static_cast<double*>(C), M, N, ldc, (int)splits, gram ? 1 : 0,
                                               tw, nullptr, M);
    BSRHT_CUDA_TRY(cudaGetLastError());
    ++launches;
  }
  note_launches(launches);
  return BSRHT_OK;
}

}  // namespace bsrht
