// Tiled CUDA-core GEMM used by the low-rank drivers (tall-skinny products).
//
//   C[M x N] = alpha * op(A) * B  (+ beta * C)
//   op(A) = A  (A row-major M x K, element (i,k) at A[i*lda + k])   or
//   op(A) = A^T (A row-major K x M, element (i,k) at A[k*lda + i]);
//   B row-major K x N.  Accumulation in Tacc; with split-K the partial
//   products go to a [splits][M][N] Tacc buffer that k_gemm_splitk_reduce
//   sums in a fixed order (deterministic).
//   tri_b: B is upper triangular (B[k][n] = 0 for k > n): K is cut at the
//   tile's last column.  upper_c: only tiles with block row <= block column
//   are formed (for symmetric Gram matrices; the reduce mirrors them).
#pragma once

#include "common.cuh"

namespace bsrht {

struct GemmArgs {
  const void* A;
  const void* B;
  void* C;         // TC output (splits == 1) or Tacc partials (splits > 1)
  int64_t M, N, K;
  int64_t lda, ldb, ldc;
  int64_t tiles_n;  // column tiles: tile t of the 1-D grid is (t / tiles_n, t % tiles_n)
  double alpha, beta;
  int splits;      // split-K factor (gridDim.z)
  int a_trans;     // 1: op(A) = A^T
  int tri_b;       // B upper triangular
  int upper_c;     // only upper-triangle tiles (square C)
};

template <typename T>
__device__ __forceinline__ T to_acc(float v) { return (T)v; }

template <typename Tacc, typename Tin>
__device__ __forceinline__ Tacc cvt_in(const Tin* p) {
  if constexpr (sizeof(Tacc) == 8)
    return Elem<Tin>::to_f64(*p);
  else
    return Elem<Tin>::to_f32(*p);
}

// 256 threads as a 16 x 16 grid; each computes TM x TN outputs.
template <typename TA, typename TB, typename TC, typename Tacc, int TM, int TN, int BK>
__global__ void __launch_bounds__(256) k_gemm(GemmArgs g) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  __shared__ Tacc As[2][BK][BM + 4];
  __shared__ Tacc Bs[2][BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t bm = (int64_t)blockIdx.x / g.tiles_n, bn = (int64_t)blockIdx.x % g.tiles_n;
  if (g.upper_c && bm > bn) return;
  const int64_t m0 = bm * BM, n0 = bn * BN;
  int64_t kend = g.K;
  if (g.tri_b) kend = min(kend, n0 + BN);
  // split-K range (in units of BK tiles)
  const int64_t ktiles = (kend + BK - 1) / BK;
  const int64_t kt0 = ktiles * blockIdx.z / g.splits;
  const int64_t kt1 = ktiles * (blockIdx.z + 1) / g.splits;
  const TA* __restrict__ A = static_cast<const TA*>(g.A);
  const TB* __restrict__ B = static_cast<const TB*>(g.B);

  constexpr int A_ELEMS = BM * BK / 256;  // per thread
  constexpr int B_ELEMS = BN * BK / 256;
  Tacc ra[A_ELEMS], rb[B_ELEMS];

  auto load_tile = [&](int64_t kt) {
    const int64_t k0 = kt * BK;
#pragma unroll
    for (int e = 0; e < A_ELEMS; ++e) {
      const int idx = tid + 256 * e;
      int mi, ki;
      if (g.a_trans) {  // A is K x M: consecutive threads walk m
        mi = idx % BM;
        ki = idx / BM;
      } else {          // A is M x K: consecutive threads walk k
        ki = idx % BK;
        mi = idx / BK;
      }
      const int64_t gm = m0 + mi, gk = k0 + ki;
      Tacc v = Tacc(0);
      if (gm < g.M && gk < kend)
        v = g.a_trans ? cvt_in<Tacc>(A + gk * g.lda + gm) : cvt_in<Tacc>(A + gm * g.lda + gk);
      ra[e] = v;
    }
#pragma unroll
    for (int e = 0; e < B_ELEMS; ++e) {
      const int idx = tid + 256 * e;
      const int ni = idx % BN, ki = idx / BN;
      const int64_t gn = n0 + ni, gk = k0 + ki;
      Tacc v = Tacc(0);
      if (gn < g.N && gk < kend) v = cvt_in<Tacc>(B + gk * g.ldb + gn);
      rb[e] = v;
    }
  };
  auto store_tile = [&](int buf) {
#pragma unroll
    for (int e = 0; e < A_ELEMS; ++e) {
      const int idx = tid + 256 * e;
      int mi, ki;
      if (g.a_trans) {
        mi = idx % BM;
        ki = idx / BM;
      } else {
        ki = idx % BK;
        mi = idx / BK;
      }
      As[buf][ki][mi] = ra[e];
    }
#pragma unroll
    for (int e = 0; e < B_ELEMS; ++e) {
      const int idx = tid + 256 * e;
      Bs[buf][idx / BN][idx % BN] = rb[e];
    }
  };

  Tacc acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = Tacc(0);

  if (kt0 < kt1) {
    load_tile(kt0);
    store_tile(0);
    __syncthreads();
    int buf = 0;
    for (int64_t kt = kt0; kt < kt1; ++kt) {
      const bool more = kt + 1 < kt1;
      if (more) load_tile(kt + 1);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        Tacc a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      if (more) {
        store_tile(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
    }
  }

  if (g.splits > 1) {
    Tacc* P = static_cast<Tacc*>(g.C) + (int64_t)blockIdx.z * g.M * g.N;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t gm = m0 + ty + 16 * i;
      if (gm >= g.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t gn = n0 + tx + 16 * j;
        if (gn < g.N) P[gm * g.N + gn] = acc[i][j];
      }
    }
  } else {
    TC* C = static_cast<TC*>(g.C);
    const Tacc alpha = (Tacc)g.alpha, beta = (Tacc)g.beta;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t gm = m0 + ty + 16 * i;
      if (gm >= g.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t gn = n0 + tx + 16 * j;
        if (gn >= g.N) continue;
        Tacc v = alpha * acc[i][j];
        if (g.beta != 0.0) v += beta * (Tacc)C[gm * g.ldc + gn];
        C[gm * g.ldc + gn] = (TC)v;
      }
    }
  }
}

// Sums split-K partials in split order; optional mirror of the upper
// triangle (upper_c) into the lower one.
template <typename Tacc, typename TC>
__global__ void k_gemm_splitk_reduce(const Tacc* __restrict__ P, TC* __restrict__ C, int64_t M, int64_t N,
                                     int64_t ldc, int splits, double alpha, int mirror, int tile_m,
                                     int tile_n) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  int64_t i = idx / N, j = idx - i * N;
  int64_t si = i, sj = j;
  if (mirror && (i / tile_m) > (j / tile_n)) {  // tile below the diagonal: read the mirrored entry
    si = j;
    sj = i;
  }
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += (double)P[(int64_t)z * M * N + si * N + sj];
  C[i * ldc + j] = (TC)(alpha * s);
}

}  // namespace bsrht
