// Dense linear algebra for the low-rank drivers (device kernels + launchers).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "dla.cuh"
#include "trace.cuh"
#include "gemm.cuh"
#include "sketch.cuh"
#include "f32x2.cuh"

namespace cg = cooperative_groups;

namespace bsrht {

#define DLA_LAUNCH_CHECK()                                                   \
  do {                                                                       \
    const cudaError_t e_ = cudaGetLastError();                               \
    if (e_ != cudaSuccess) return ::bsrht::cuda_failure(e_, __FILE__, __LINE__); \
  } while (0)

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------ cooperative grids
// The kernels below with grid-wide barriers (grid.sync()) need every CTA of
// their grid resident at once.  One such grid, sized within the device's
// occupancy, is what cudaLaunchCooperativeKernel provides; but two of them
// enqueued on different streams (the server's executor streams, or callers
// of the library on several streams or host threads) could each hold part
// of the SMs while their barriers wait for CTAs that cannot start.  So every
// cooperative grid of this library runs on one stream per device: the
// caller's stream records an event, that stream waits for it, runs the grid
// and records an event that the caller's stream waits for, all under one
// host mutex.  Cooperative grids of different callers then run one after
// another; what runs beside them are ordinary kernels, which finish without
// waiting on any other grid (their own waits are bounded), so each
// cooperative grid finds its SMs as those kernels drain.
namespace {
std::mutex g_coop_mu;
cudaStream_t g_coop_stream[64] = {};
}  // namespace

static int launch_cooperative(const void* func, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t s) {
  int dev = 0;
  BSRHT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return BSRHT_EUNSUP;
  std::lock_guard<std::mutex> lock(g_coop_mu);
  if (!g_coop_stream[dev]) BSRHT_CUDA_TRY(cudaStreamCreateWithFlags(&g_coop_stream[dev], cudaStreamNonBlocking));
  cudaStream_t cs = g_coop_stream[dev];
  cudaEvent_t before = nullptr, after = nullptr;
  BSRHT_CUDA_TRY(cudaEventCreateWithFlags(&before, cudaEventDisableTiming));
  if (cudaEventCreateWithFlags(&after, cudaEventDisableTiming) != cudaSuccess) {
    cudaEventDestroy(before);
    return BSRHT_ECUDA;
  }
  cudaError_t e = cudaEventRecord(before, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, before, 0);
  if (e == cudaSuccess) e = cudaLaunchCooperativeKernel(func, grid, block, args, smem, cs);
  if (e == cudaSuccess) e = cudaEventRecord(after, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, after, 0);
  cudaEventDestroy(before);  // released once the recorded work completes
  cudaEventDestroy(after);
  return e == cudaSuccess ? BSRHT_OK : cuda_failure(e, __FILE__, __LINE__);
}

// ------------------------------------------------------------------ GEMM
namespace {

template <typename TA, typename TB, typename TC, typename Tacc, int TM>
int gemm_launch(const Dla& d, Arena& ar, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                bool a_trans, const void* B, int64_t ldb, void* C, int64_t ldc, double alpha, double beta,
                bool tri_b, bool gram) {
  constexpr int BM = 16 * TM, BN = 16 * TM, BK = 8;
  GemmArgs g;
  g.A = A;
  g.B = B;
  g.M = M;
  g.N = N;
  g.K = K;
  g.lda = lda;
  g.ldb = ldb;
  g.ldc = ldc;
  g.alpha = alpha;
  g.beta = beta;
  g.a_trans = a_trans ? 1 : 0;
  g.tri_b = tri_b ? 1 : 0;
  g.upper_c = gram ? 1 : 0;
  const int64_t tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  const int64_t tiles = gram ? tm * (tm + 1) / 2 : tm * tn;
  // Split K when the tiles alone leave SMs idle.  FP64 FMAs run at 1/64 of
  // the FP32 rate on this GPU (about two per SM and clock): one 64 x 64 tile
  // over K = 256 keeps an SM busy for a quarter of a millisecond, so FP64
  // products split K down to 32-deep ranges; FP32 ones keep ranges of at
  // least 256.
  constexpr bool kF64 = std::is_same<Tacc, double>::value;
  constexpr int64_t kMinRange = kF64 ? 4 * BK : 32 * BK, kMinK = kF64 ? 8 * BK : 64 * BK;
  int splits = 1;
  const int64_t target = 2 * (int64_t)num_sms();
  if (tiles < target && K > kMinK) {
    splits = (int)std::min<int64_t>((target + tiles - 1) / tiles, K / kMinRange);
    splits = std::max(1, std::min(splits, 64));
  }
  // Row and column tiles on one grid dimension (the y dimension's 65535
  // would cap M at about 4 million rows).
  g.tiles_n = tn;
  if (tm * tn > (int64_t)INT32_MAX) return BSRHT_EUNSUP;
  dim3 grid((unsigned)(tm * tn), 1u, (unsigned)splits);
  if (splits > 1 || gram) {
    Tacc* P = static_cast<Tacc*>(ar.take(sizeof(Tacc) * (size_t)splits * M * N));
    if (!ar.ok()) return BSRHT_ENOMEM;
    if (ar.measure) return BSRHT_OK;
    g.C = P;
    g.splits = splits;
    k_gemm<TA, TB, Tacc, Tacc, TM, TM, BK><<<grid, 256, 0, d.s>>>(g);
    DLA_LAUNCH_CHECK();
    k_gemm_splitk_reduce<Tacc, TC><<<blocks_for(M * N, 256), 256, 0, d.s>>>(
        P, static_cast<TC*>(C), M, N, ldc, splits, alpha, gram ? 1 : 0, BM, BN);
    DLA_LAUNCH_CHECK();
    note_launches(2);
    return BSRHT_OK;
  }
  if (ar.measure) return BSRHT_OK;
  g.C = C;
  g.splits = 1;
  k_gemm<TA, TB, TC, Tacc, TM, TM, BK><<<grid, 256, 0, d.s>>>(g);
  DLA_LAUNCH_CHECK();
  note_launches(1);
  return BSRHT_OK;
}

}  // namespace

int gemm(const Dla& d, Arena& ar, DT ta, DT tb, DT tc, bool acc64, int64_t M, int64_t N, int64_t K,
         const void* A, int64_t lda, bool a_trans, const void* B, int64_t ldb, void* C, int64_t ldc,
         double alpha, double beta, bool tri_b, bool gram) {
  if (M <= 0 || N <= 0) return BSRHT_OK;
  if ((gram) && beta != 0.0) return BSRHT_EINVAL;
  if (acc64) {
    if (ta == DT::F64 && tb == DT::F64 && tc == DT::F64)
      return gemm_launch<double, double, double, double, 4>(d, ar, M, N, K, A, lda, a_trans, B, ldb, C, ldc,
                                                            alpha, beta, tri_b, gram);
    if (ta == DT::F32 && tb == DT::F32 && tc == DT::F64)  // FP64 accumulation of FP32 data
      return gemm_launch<float, float, double, double, 4>(d, ar, M, N, K, A, lda, a_trans, B, ldb, C, ldc, alpha,
                                                          beta, tri_b, gram);
    return BSRHT_EUNSUP;
  }
  if (tb != DT::F32) return BSRHT_EUNSUP;
#define GEMM32(TAT, TCT)                                                                                   \
  return gemm_launch<TAT, float, TCT, float, 8>(d, ar, M, N, K, A, lda, a_trans, B, ldb, C, ldc, alpha, beta, \
                                                tri_b, gram)
  if (tc == DT::F32) {
    if (ta == DT::F32) GEMM32(float, float);
    if (ta == DT::BF16) GEMM32(__nv_bfloat16, float);
    if (ta == DT::F16) GEMM32(__half, float);
  } else if (tc == DT::F64) {
    if (ta == DT::F32) GEMM32(float, double);
  }
#undef GEMM32
  return BSRHT_EUNSUP;
}

// ------------------------------------------------------------ Cholesky
constexpr int kNB = 32;

__global__ void k_chol_diag(double* g, int64_t l, int64_t k0, int nb, int* status) {
  __shared__ double a[kNB][kNB + 1];
  const int tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    a[i][j] = (j <= i) ? g[(k0 + i) * l + k0 + j] : 0.0;
  }
  for (int j = 0; j < nb; ++j) {
    __syncthreads();
    if (tid == 0) {
      double dj = a[j][j];
      if (!(dj > 0.0)) {
        atomicOr(status, kStatusNotPD);
        dj = 1.0;
      }
      a[j][j] = sqrt(dj);
    }
    __syncthreads();
    const double piv = a[j][j];
    for (int i = j + 1 + tid; i < nb; i += blockDim.x) a[i][j] /= piv;
    __syncthreads();
    const int rem = nb - j - 1;
    for (int e = tid; e < rem * rem; e += blockDim.x) {
      const int i = j + 1 + e / rem, c = j + 1 + e % rem;
      if (c <= i) a[i][c] -= a[i][j] * a[c][j];
    }
  }
  __syncthreads();
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    g[(k0 + i) * l + k0 + j] = (j <= i) ? a[i][j] : 0.0;
  }
}

// Rows below the diagonal block: L[i, k0:k0+nb] = A[i, k0:k0+nb] L_kk^-T.
__global__ void k_chol_panel(double* g, int64_t l, int64_t k0, int nb) {
  __shared__ double lkk[kNB][kNB + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    lkk[i][j] = g[(k0 + i) * l + k0 + j];
  }
  __syncthreads();
  const int64_t i = k0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= l) return;
  double x[kNB];
#pragma unroll
  for (int c = 0; c < kNB; ++c) x[c] = c < nb ? g[i * l + k0 + c] : 0.0;
#pragma unroll
  for (int c = 0; c < kNB; ++c) {
    if (c < nb) {
      double v = x[c];
#pragma unroll
      for (int e = 0; e < kNB; ++e)
        if (e < c) v -= x[e] * lkk[c][e];
      x[c] = v / lkk[c][c];
    }
  }
#pragma unroll
  for (int c = 0; c < kNB; ++c)
    if (c < nb) g[i * l + k0 + c] = x[c];
}

// Trailing update of the lower triangle: A[i][j] -= sum_c L[i][k0+c] L[j][k0+c].
__global__ void k_chol_update(double* g, int64_t l, int64_t k0, int nb) {
  __shared__ double li[32][kNB + 1];
  __shared__ double lj[32][kNB + 1];
  const int64_t t0 = k0 + nb;
  const int64_t bi = t0 + (int64_t)blockIdx.y * 32, bj = t0 + (int64_t)blockIdx.x * 32;
  if (bj > bi) return;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8 threads
  for (int r = ty; r < 32; r += 8) {
    const int64_t ri = bi + r, rj = bj + r;
    li[r][tx] = (ri < l && tx < nb) ? g[ri * l + k0 + tx] : 0.0;
    lj[r][tx] = (rj < l && tx < nb) ? g[rj * l + k0 + tx] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = bi + r, j = bj + tx;
    if (i >= l || j >= l || j > i) continue;
    double s = 0.0;
#pragma unroll 8
    for (int c = 0; c < nb; ++c) s += li[r][c] * lj[tx][c];
    g[i * l + j] -= s;
  }
}

__global__ void k_zero_upper(double* g, int64_t l) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= l * l) return;
  const int64_t i = idx / l, j = idx % l;
  if (j > i) g[idx] = 0.0;
}

int cholesky(const Dla& d, double* g, int64_t l) {
  int launches = 0;
  for (int64_t k0 = 0; k0 < l; k0 += kNB) {
    const int nb = (int)std::min<int64_t>(kNB, l - k0);
    k_chol_diag<<<1, 256, 0, d.s>>>(g, l, k0, nb, d.status);
    DLA_LAUNCH_CHECK();
    const int64_t below = l - k0 - nb;
    launches += 1;
    if (below > 0) {
      k_chol_panel<<<blocks_for(below, 128), 128, 0, d.s>>>(g, l, k0, nb);
      DLA_LAUNCH_CHECK();
      const unsigned tb = (unsigned)((below + 31) / 32);
      k_chol_update<<<dim3(tb, tb), 256, 0, d.s>>>(g, l, k0, nb);
      DLA_LAUNCH_CHECK();
      launches += 2;
    }
  }
  k_zero_upper<<<blocks_for(l * l, 256), 256, 0, d.s>>>(g, l);
  DLA_LAUNCH_CHECK();
  note_launches(launches + 1);
  return BSRHT_OK;
}

// ------------------------------------------------------ triangular inverse
__global__ void k_transpose_sq(const double* in, double* out, int64_t l) {
  __shared__ double t[32][33];
  const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = by + r, j = bx + tx;
    t[r][tx] = (i < l && j < l) ? in[i * l + j] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = bx + r, j = by + tx;
    if (i < l && j < l) out[i * l + j] = t[tx][r];
  }
}

// Column j of L^-1 by forward substitution; written as row j of R^-1 = L^-T.
// LT = L^T (row k of LT is column k of L).
__global__ void k_trinv(const double* __restrict__ LT, double* __restrict__ Rinv, int64_t l) {
  extern __shared__ double x[];
  const int64_t j = blockIdx.x;
  for (int64_t i = threadIdx.x; i < l; i += blockDim.x) x[i] = (i == j) ? 1.0 : 0.0;
  for (int64_t k = j; k < l; ++k) {
    __syncthreads();
    if (threadIdx.x == 0) x[k] /= LT[k * l + k];
    __syncthreads();
    const double xk = x[k];
    for (int64_t i = k + 1 + threadIdx.x; i < l; i += blockDim.x) x[i] -= LT[k * l + i] * xk;
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < l; i += blockDim.x) Rinv[j * l + i] = x[i];
}

int tri_inverse(const Dla& d, const double* L, double* LT, double* Rinv, int64_t l) {
  const unsigned t = (unsigned)((l + 31) / 32);
  k_transpose_sq<<<dim3(t, t), 256, 0, d.s>>>(L, LT, l);
  DLA_LAUNCH_CHECK();
  k_trinv<<<(unsigned)l, 256, sizeof(double) * l, d.s>>>(LT, Rinv, l);
  DLA_LAUNCH_CHECK();
  note_launches(2);
  return BSRHT_OK;
}

// ------------------------------------------- fused Cholesky and inverse
// One cooperative kernel: right-looking blocked Cholesky G = L L^T with
// 32 x 32 blocks, and the same block eliminations applied to an identity
// matrix T, which turns T into L^-1.  Step kb:
//   (a) L_kk = chol(A_kk) and X_kk = L_kk^-1 (one CTA, shared memory);
//   (b) panel L_ik = A_ik X_kk^T (one warp per row i > kb) and the final
//       block row X_kb,c = X_kk T_kb,c of L^-1 (c < kb);
//   (c) trailing update A_ij -= L_ik L_jk^T (kb < j <= i) and
//       T_ic -= L_ik X_kb,c (c <= kb < i), one 32 x 32 tile per CTA; the CTA
//       holding tile (kb+1, kb+1) then factors it, which is (a) of the next
//       step.
// Two grid barriers per block step.  Outputs: L in the lower triangle of g
// (upper zeroed), LT = L^T and Rinv = L^-T (row-major, upper triangular).
// T and X are l x l scratch.  A pivot <= 0 sets kStatusNotPD (and is
// replaced by 1 so the kernel runs to the end).
constexpr int kCB = 32;

struct CholInvArgs {
  double* g;
  double* LT;
  double* Rinv;
  double* T;
  double* X;
  int l;
  int nblk;
  int* status;
};

// 1/d for a pivot d > 0: FP32 seed on d scaled by a power of two into
// [1, 2), then two Newton steps y <- y + y (1 - d y) (relative error 2^-23 ->
// 2^-46 -> rounding).  A dependent FP64 operation costs about 60 cycles on
// this GPU (measured), so this chain of six is what one column of the
// diagonal factorisation waits for.
__device__ __forceinline__ double ci_rcp(double d) {
  if (d > 0x1.0p-1000 && d < 0x1.0p1000) {
    const long long bits = __double_as_longlong(d);
    const int e = (int)((bits >> 52) & 0x7FF) - 1023;                       // d = f 2^e, f in [1, 2)
    const double f = __longlong_as_double(bits - ((long long)e << 52));     // f in [1, 2)
    double y = (double)__frcp_rn((float)f);
    y = fma(y, fma(-f, y, 1.0), y);
    y = fma(y, fma(-f, y, 1.0), y);
    return y * __longlong_as_double((long long)(1023 - e) << 52);          // times 2^-e
  }
  return 1.0 / d;
}

// (a): factor the diagonal block kb (already updated), G_kk = L D L^T with
// unit lower L, and form its inverse alongside: the eliminations of column j
// (row i -= l_ij row j, l_ij = s_ij / d_j) are applied to the trailing part
// of s and to an identity block t, which ends as L^-1.  Thread 0 applies
// column j's elimination to the next pivot first and forms its reciprocal
// while threads 1..255 apply the rest, so one barrier per column; the
// square roots come at the end, all at once: L_kk = L D^1/2 and
// X_kk = L_kk^-1 = D^-1/2 L^-1.
__device__ void ci_factor_diag(const CholInvArgs& a, int kb, double (*s)[kCB + 1], double (*t)[kCB + 1],
                               double* dinv, double* dd) {
  const int tid = threadIdx.x, l = a.l, k0 = kb * kCB;
  const int nb = min(kCB, l - k0);
  for (int e = tid; e < kCB * kCB; e += blockDim.x) {
    const int i = e / kCB, j = e % kCB;
    double v = (i == j) ? 1.0 : 0.0;
    if (i < nb && j < nb && j <= i) v = a.g[(int64_t)(k0 + i) * l + k0 + j];
    s[i][j] = v;
    t[i][j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    double p = s[0][0];
    if (!(p > 0.0)) {
      atomicOr(a.status, kStatusNotPD);
      p = 1.0;
    }
    dd[0] = p;
    dinv[0] = ci_rcp(p);
  }
  __syncthreads();
  for (int j = 0; j < kCB; ++j) {
    const double ij = dinv[j];
    if (tid == 0) {
      if (j + 1 < kCB) {
        const double x = s[j + 1][j];
        double p = fma(-x * ij, x, s[j + 1][j + 1]);
        if (!(p > 0.0)) {
          atomicOr(a.status, kStatusNotPD);
          p = 1.0;
        }
        dd[j + 1] = p;
        dinv[j + 1] = ci_rcp(p);
      }
    } else {
      // Trailing entries (i, c), j < c <= i, except the next pivot; item e ->
      // row offset u with u (u + 1) / 2 <= e < (u + 1) (u + 2) / 2.  Then the
      // entries (i, c), i > j, c <= j of t.
      const int rem = kCB - 1 - j;
      const int n_tr = rem * (rem + 1) / 2;
      const int n_items = n_tr + rem * (j + 1);
      for (int e = tid - 1; e < n_items; e += blockDim.x - 1) {
        if (e < n_tr) {
          if (e == 0) continue;  // (j+1, j+1): thread 0
          int u = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
          while ((u + 1) * (u + 2) / 2 <= e) ++u;
          while (u * (u + 1) / 2 > e) --u;
          const int i = j + 1 + u, c = j + 1 + (e - u * (u + 1) / 2);
          s[i][c] = fma(-s[i][j] * ij, s[c][j], s[i][c]);
        } else {
          const int q = e - n_tr, i = j + 1 + q / (j + 1), c = q % (j + 1);
          t[i][c] = fma(-s[i][j] * ij, t[j][c], t[i][c]);
        }
      }
    }
    __syncthreads();
  }
  // D^1/2: sqrt(d_j) and 1/sqrt(d_j), all columns at once.
  if (tid < kCB) {
    const double r = sqrt(dd[tid]);
    dd[tid] = r;
    dinv[tid] = 1.0 / r;
  }
  __syncthreads();
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    // L_kk[i][j] = (s_ij / d_j) sqrt(d_j) = s_ij / sqrt(d_j);  X_kk[i][j] = t_ij / sqrt(d_i).
    a.g[(int64_t)(k0 + i) * l + k0 + j] = (j < i) ? s[i][j] * dinv[j] : (i == j ? dd[j] : 0.0);
    a.X[(int64_t)(k0 + i) * l + k0 + j] = (j <= i) ? t[i][j] * dinv[i] : 0.0;
  }
}

__global__ void __launch_bounds__(256) k_chol_inv(CholInvArgs a) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double s0[kCB][kCB + 1];
  __shared__ double s1[kCB][kCB + 1];
  __shared__ double dinv[kCB];
  __shared__ double dd[kCB];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int l = a.l, nblk = a.nblk;
  const int64_t ll = (int64_t)l * l;
  // T = I (only its lower block triangle is ever read).
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + tid; e < ll; e += (int64_t)gridDim.x * blockDim.x)
    a.T[e] = (e / l == e % l) ? 1.0 : 0.0;
  if (blockIdx.x == 0) ci_factor_diag(a, 0, s0, s1, dinv, dd);
  grid.sync();
  const int gw = blockIdx.x * (blockDim.x >> 5) + w, nwg = gridDim.x * (blockDim.x >> 5);
  for (int kb = 0; kb < nblk; ++kb) {
    const int k0 = kb * kCB, nb = min(kCB, l - k0);
    const int rows_below = l - k0 - nb;
    // (b) X_kk into shared memory (every CTA), then panel rows and X row block.
    for (int e = tid; e < kCB * kCB; e += blockDim.x) {
      const int i = e / kCB, j = e % kCB;
      s1[i][j] = (i < nb && j < nb) ? a.X[(int64_t)(k0 + i) * l + k0 + j] : 0.0;
    }
    __syncthreads();
    const int xrow_items = kb * kCB;  // rows r < 32 of block kb times column blocks c < kb
    for (int it = gw; it < rows_below + xrow_items; it += nwg) {
      if (it < rows_below) {
        const int64_t i = k0 + nb + it;
        const double v = lane < nb ? a.g[i * l + k0 + lane] : 0.0;
        double out = 0.0;
        for (int e = 0; e < kCB; ++e) out = fma(__shfl_sync(0xffffffffu, v, e), s1[lane][e], out);
        if (lane < nb) a.g[i * l + k0 + lane] = out;
      } else {
        const int q = it - rows_below, r = q / kb, c = q % kb;
        if (r < nb) {
          // X[k0+r][c*32+lane] = sum_{e<=r} X_kk[r][e] T[k0+e][c*32+lane]
          double out = 0.0;
          for (int e = 0; e <= r; ++e) out = fma(s1[r][e], a.T[(int64_t)(k0 + e) * l + c * kCB + lane], out);
          a.X[(int64_t)(k0 + r) * l + c * kCB + lane] = out;
        }
      }
    }
    grid.sync();
    if (kb + 1 == nblk) break;
    // (c) trailing tiles (bi >= bj > kb) and T tiles (bi > kb >= c).
    const int rem = nblk - kb - 1;
    const int n_trail = rem * (rem + 1) / 2, n_t = rem * (kb + 1);
    const int tx = tid & 31, ty = tid >> 5;
    for (int item = blockIdx.x; item < n_trail + n_t; item += gridDim.x) {
      int bi, bj;
      bool trail = item < n_trail;
      if (trail) {
        // item 0 is the diagonal tile (kb+1, kb+1); then the rest row by row.
        int q = item, row = 0;
        while (q > row) {
          q -= row + 1;
          ++row;
        }
        bi = kb + 1 + row;
        bj = kb + 1 + q;
      } else {
        const int q = item - n_trail;
        bi = kb + 1 + q / (kb + 1);
        bj = q % (kb + 1);
      }
      __syncthreads();
      // s0 = L rows of block bi (panel of block kb); s1 = L rows of block bj or X row block kb.
      for (int r = ty; r < kCB; r += 8) {
        const int64_t ri = (int64_t)bi * kCB + r;
        s0[r][tx] = (ri < l && tx < nb) ? a.g[ri * l + k0 + tx] : 0.0;
        if (trail) {
          const int64_t rj = (int64_t)bj * kCB + r;
          s1[r][tx] = (rj < l && tx < nb) ? a.g[rj * l + k0 + tx] : 0.0;
        } else {
          s1[r][tx] = (r < nb) ? a.X[(int64_t)(k0 + r) * l + bj * kCB + tx] : 0.0;
        }
      }
      __syncthreads();
      const int64_t col = (int64_t)bj * kCB + tx;
      for (int r = ty; r < kCB; r += 8) {
        const int64_t row = (int64_t)bi * kCB + r;
        if (row >= l || col >= l) continue;
        double acc = 0.0;
        if (trail) {
#pragma unroll 8
          for (int e = 0; e < kCB; ++e) acc = fma(s0[r][e], s1[tx][e], acc);
          a.g[row * l + col] -= acc;
        } else {
#pragma unroll 8
          for (int e = 0; e < kCB; ++e) acc = fma(s0[r][e], s1[e][tx], acc);
          a.T[row * l + col] -= acc;
        }
      }
      if (item == 0) {
        __syncthreads();
        ci_factor_diag(a, kb + 1, s0, s1, dinv, dd);
      }
    }
    grid.sync();
  }
  // Outputs: zero the upper triangle of g, LT = L^T, Rinv = X^T.
  grid.sync();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + tid; e < ll; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / l, j = e % l;  // element (i, j) of the outputs
    if (j > i) a.g[e] = 0.0;
    a.LT[e] = (j >= i) ? a.g[j * l + i] : 0.0;
    a.Rinv[e] = (j >= i) ? a.X[j * l + i] : 0.0;
  }
}

int chol_inv(const Dla& d, double* g, double* LT, double* Rinv, double* T, double* X, int64_t l) {
  if (l <= 0) return BSRHT_OK;
  CholInvArgs a{g, LT, Rinv, T, X, (int)l, (int)((l + kCB - 1) / kCB), d.status};
  int occ = 0;
  BSRHT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_chol_inv, 256, 0));
  const int blocks = num_sms() * std::max(1, std::min(occ, 1));
  void* args[] = {&a};
  const int st = launch_cooperative((const void*)k_chol_inv, dim3(blocks), dim3(256), args, 0, d.s);
  if (st != BSRHT_OK) return st;
  note_launches(1);
  return BSRHT_OK;
}

// ------------------------------------------------------- Jacobi SVD
__device__ __forceinline__ int rr_player(int pos, int round, int lp) {
  if (pos == 0) return 0;
  return 1 + (pos - 1 + round) % (lp - 1);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One-sided (Hestenes) Jacobi on the l columns (each of `rows` entries,
// stored contiguously) of M with round-robin pairs, the same rotations
// applied to the columns of V (also `rows` entries each); one block of WP
// warps per column pair, a grid-wide barrier between rounds.
// Warp w of the block holds rows w*32*JR .. (w+1)*32*JR-1 of the two columns
// of M and of V in registers (JR values per lane), the block sums the
// partial inner products in shared memory, every warp derives the rotation
// from the sum and rotates its rows in registers, so each round costs one
// round trip to L2 and one block barrier.  A pair is rotated while
// |x.y| > tol sqrt(x.x y.y); the sweeps stop after one in which no rotation
// exceeded tol_stop (>= tol), i.e. once only rounding-level rotations are
// left.  Two columns that are both numerically zero (norm at most
// tiny_rel ||M||_F, *fnorm = ||M||_F) are left alone: rounding keeps their
// directions random and rotating them would never converge.
// `status` (may be null) gets kStatusNoConv if max_sweeps ran out.
// Column norms: nrm[c] = |M_c|^2 is formed exactly at the start of every
// sweep and then carried through the rotations as alpha - t gamma and
// beta + t gamma (what the rotation makes of them in exact arithmetic), so a
// pair needs one inner product instead of three.
// Rotation: t = tan(theta) is the smaller root of gamma t^2 + (beta - alpha)
// t - gamma = 0; c = 1/sqrt(1 + t^2), s = c t.  The rotation is orthogonal
// for any t, and a relative error delta in t leaves a cosine of about delta
// times the old one, so in FP64 t comes from an FP32 evaluation of the root
// (the FP64 units of this GPU run at 1/64 of the FP32 rate) while c and s
// are formed in FP64 from that t.
__device__ __forceinline__ double jac_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float jac_rsqrt(float x) { return rsqrtf(x); }

// tan(theta) for the pair (alpha, beta, gamma), gamma != 0, with
// zeta = (beta - alpha) / (2 gamma).  For |zeta| > 2^60 the root is
// 1 / (2 zeta) to relative 2^-122, which also keeps zeta^2 in FP32 range.
__device__ __forceinline__ float jac_tangent(float alpha, float beta, float gamma) {
  const float zeta = (beta - alpha) / (2.0f * gamma);
  if (fabsf(zeta) > 0x1.0p60f) return 0.5f / zeta;
  return (zeta >= 0.0f ? 1.0f : -1.0f) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
}
__device__ __forceinline__ double jac_tangent(double alpha, double beta, double gamma) {
  const double d = beta - alpha, g2 = 2.0 * gamma;
  if (fabs(d) > 0x1.0p60 * fabs(g2)) return gamma / d;  // 1 / (2 zeta), in FP64
  // |zeta| <= 2^60: scale d and 2 gamma by the same power of two so that
  // 2 gamma lands in [1, 2); zeta is unchanged and both values are in FP32
  // range.  Subnormal gamma (biased exponent 0) is scaled as if its
  // exponent were -1022; its FP32 value is then below 1 but not zero.
  int e = (int)((__double_as_longlong(g2) >> 52) & 0x7FF) - 1023;
  e = e < -1022 ? -1022 : e;
  const double sc = __longlong_as_double((long long)(1023 - e) << 52);  // 2^-e, e in [-1022, 1023]
  const float zeta = __double2float_rn(d * sc) / __double2float_rn(g2 * sc);
  return (double)((zeta >= 0.0f ? 1.0f : -1.0f) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta)));
}

template <typename T, int JR, int WP>
__global__ void __launch_bounds__(32 * WP) k_jacobi(T* __restrict__ M, T* __restrict__ V, T* __restrict__ nrm,
                                                    int l, int lp, int rows, double tol, double tol_stop,
                                                    const double* __restrict__ fnorm, double tiny_rel,
                                                    int max_sweeps, int* __restrict__ rot_counts,
                                                    int* __restrict__ status) {
  cg::grid_group grid = cg::this_grid();
  __shared__ T part[2][WP];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gwarp = blockIdx.x * WP + w, nwarps = gridDim.x * WP;
  const T ttol2 = (T)(tol * tol), tstop2 = (T)(tol_stop * tol_stop);
  const T ttol = (T)tol, tstop = (T)tol_stop;
  const double tiny = tiny_rel * fnorm[0];
  const T tiny2 = (T)(tiny * tiny);
  const int row0 = w * 32 * JR + lane;
  int sweep = 0, it = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int c = gwarp; c < l; c += nwarps) {
      const T* __restrict__ col = M + (int64_t)c * rows;
      T sq = 0;
      for (int r = lane; r < rows; r += 32) sq = fma(col[r], col[r], sq);
      sq = warp_sum(sq);
      if (lane == 0) nrm[c] = sq;
    }
    grid.sync();
    for (int round = 0; round < lp - 1; ++round) {
      for (int k = blockIdx.x; k < lp / 2; k += gridDim.x) {
        int p = rr_player(k, round, lp), q = rr_player(lp - 1 - k, round, lp);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        if (q >= l) continue;  // padding column (block-uniform)
        T* __restrict__ a = M + (int64_t)p * rows;
        T* __restrict__ b = M + (int64_t)q * rows;
        T* __restrict__ va = V + (int64_t)p * rows;
        T* __restrict__ vb = V + (int64_t)q * rows;
        T x[JR], y[JR], vx[JR], vy[JR];
#pragma unroll
        for (int e = 0; e < JR; ++e) {
          const int r = row0 + 32 * e;
          const bool in = r < rows;
          x[e] = in ? a[r] : (T)0;
          y[e] = in ? b[r] : (T)0;
          vx[e] = in ? va[r] : (T)0;
          vy[e] = in ? vb[r] : (T)0;
        }
        // Four independent partial sums: a dependent FP64 FMA costs about 60
        // cycles on this GPU.
        T g4[4] = {0, 0, 0, 0};
#pragma unroll
        for (int e = 0; e < JR; ++e) g4[e & 3] = fma(x[e], y[e], g4[e & 3]);
        T ga = warp_sum((g4[0] + g4[1]) + (g4[2] + g4[3]));
        const T alpha = nrm[p], beta = nrm[q];  // read before thread 0 updates them
        if (WP > 1) {
          // Double-buffered: a warp can be one pair ahead, never two (the
          // barrier of the next pair waits for the slowest warp).
          if (lane == 0) part[it & 1][w] = ga;
          __syncthreads();
          ga = 0;
#pragma unroll
          for (int u = 0; u < WP; ++u) ga += part[it & 1][u];
          ++it;
        }
        const T gamma = ga;
        if (alpha <= tiny2 && beta <= tiny2) continue;
        if (gamma == (T)0) continue;
        bool rotate, significant;
        if constexpr (sizeof(T) == 8) {
          const T g2 = gamma * gamma, ab = alpha * beta;
          rotate = g2 > ttol2 * ab;
          significant = g2 > tstop2 * ab;
        } else {
          const T gnorm = sqrt(alpha) * sqrt(beta);  // alpha * beta may overflow FP32
          rotate = fabs(gamma) > ttol * gnorm;
          significant = fabs(gamma) > tstop * gnorm;
        }
        if (!rotate) continue;
        const T t = jac_tangent(alpha, beta, gamma);
        const T c = jac_rsqrt((T)1 + t * t), s = c * t;
#pragma unroll
        for (int e = 0; e < JR; ++e) {
          const int r = row0 + 32 * e;
          if (r < rows) {
            a[r] = c * x[e] - s * y[e];
            b[r] = s * x[e] + c * y[e];
            va[r] = c * vx[e] - s * vy[e];
            vb[r] = s * vx[e] + c * vy[e];
          }
        }
        if (threadIdx.x == 0) {
          nrm[p] = alpha - t * gamma;
          nrm[q] = beta + t * gamma;
          if (significant) atomicAdd(&rot_counts[sweep], 1);
        }
      }
      grid.sync();
    }
    if (*((volatile int*)&rot_counts[sweep]) == 0) break;
  }
  if (status && sweep >= max_sweeps && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kStatusNoConv);
}

template <typename T>
__global__ void k_init_identity_cols(T* V, int64_t l) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < l * l) V[idx] = (idx / l == idx % l) ? (T)1 : (T)0;
}

__global__ void k_col_norms(const double* __restrict__ M, double* __restrict__ sigma, int64_t l) {
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (c >= l) return;
  double s = 0.0;
  for (int64_t i = lane; i < l; i += 32) s = fma(M[c * l + i], M[c * l + i], s);
  s = warp_sum(s);
  if (lane == 0) sigma[c] = sqrt(s);
}

// perm[rank] = c with ranks by descending sigma (ties: lower index first).
__global__ void k_rank_desc(const double* __restrict__ sigma, int* __restrict__ perm, int64_t l) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= l) return;
  const double v = sigma[c];
  int64_t rank = 0;
  for (int64_t e = 0; e < l; ++e) {
    const double w = sigma[e];
    rank += (w > v) || (w == v && e < c);
  }
  perm[rank] = (int)c;
}

// U[i][r] = M[perm[r]][i] / sigma, Vout[i][r] = Vcols[perm[r]][i], sig_out[r].
__global__ void k_svd_finish(const double* __restrict__ M, const double* __restrict__ Vc,
                             const double* __restrict__ sigma, const int* __restrict__ perm,
                             double* __restrict__ U, double* __restrict__ Vout, double* __restrict__ sig_out,
                             int64_t l) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= l * l) return;
  const int64_t i = idx / l, r = idx % l;
  const int c = perm[r];
  const double s = sigma[c];
  U[i * l + r] = s > 0.0 ? M[(int64_t)c * l + i] / s : 0.0;
  Vout[i * l + r] = Vc[(int64_t)c * l + i];
  if (i == 0) sig_out[r] = s;
}

#define TRY_DLA(expr)                   \
  do {                                  \
    const int st_ = (expr);             \
    if (st_ != BSRHT_OK) return st_;    \
  } while (0)

// The mixed-precision path (FP32 Jacobi, FP64 polish) above this order.
constexpr int64_t kJacobiMixedMin = 64;

// sigma[c] = ||column c||_2 (FP64 sums) of the ncols columns of `rows`
// entries stored contiguously in M.
template <typename T>
__global__ void k_col_norms_t(const T* __restrict__ M, double* __restrict__ sigma, int64_t ncols, int64_t rows) {
  const int64_t c = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (c >= ncols) return;
  double sq = 0.0;
  for (int64_t i = lane; i < rows; i += 32) {
    const double v = (double)M[c * rows + i];
    sq = fma(v, v, sq);
  }
  sq = warp_sum(sq);
  if (lane == 0) sigma[c] = sqrt(sq);
}

// Vr[i][r] = V32 column perm[r], entry i (row-major l x s, FP64).
__global__ void k_gather_cols_t(const float* __restrict__ V32, const int* __restrict__ perm, int64_t l, int64_t s,
                                double* __restrict__ Vr) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= l * s) return;
  const int64_t i = idx / s, r = idx - i * s;
  Vr[idx] = (double)V32[(int64_t)perm[r] * l + i];
}

// Outputs of the partly polished SVD: ranks r < s from the s polished
// columns (Ysc, Vsc in column storage of l entries, norms sigS, ranks
// permS), ranks r >= s from the FP32 phase (M32, V32, norms sig, ranks
// perm, whose first s entries are the columns that were polished).
__global__ void k_svd_finish_part(const double* __restrict__ Ysc, const double* __restrict__ Vsc,
                                  const double* __restrict__ sigS, const int* __restrict__ permS, int64_t s,
                                  const float* __restrict__ M32, const float* __restrict__ V32,
                                  const double* __restrict__ sig, const int* __restrict__ perm, int64_t l,
                                  double* __restrict__ U, double* __restrict__ Vout, double* __restrict__ sig_out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= l * l) return;
  const int64_t i = idx / l, r = idx - i * l;
  double u, v, sv;
  if (r < s) {
    const int64_t c = permS[r];
    sv = sigS[c];
    u = sv > 0.0 ? Ysc[c * l + i] / sv : 0.0;
    v = Vsc[c * l + i];
  } else {
    const int64_t c = perm[r];
    sv = sig[c];
    u = sv > 0.0 ? (double)M32[c * l + i] / sv : 0.0;
    v = (double)V32[c * l + i];
  }
  U[idx] = u;
  Vout[idx] = v;
  if (i == 0) sig_out[r] = sv;
}

// *flag = 1 when some pair i < j of the columns whose Gram is G (n x n,
// FP64) has |G_ij| > tol sqrt(G_ii G_jj), pairs whose squared norms are both
// at most (tiny_rel ||M||_F)^2 left out: the test by which a further Jacobi
// sweep would rotate a pair (k_jacobi, tol_stop).
__global__ void k_offdiag_exceeds(const double* __restrict__ G, int64_t n, const double* __restrict__ fnorm,
                                  double tiny_rel, double tol, int* __restrict__ flag) {
  const double tiny = tiny_rel * fnorm[0], tiny2 = tiny * tiny, tol2 = tol * tol;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * n;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / n, j = idx - i * n;
    if (i >= j) continue;
    const double a = G[i * n + i], b = G[j * n + j], g = G[idx];
    if (a <= tiny2 && b <= tiny2) continue;
    if (g * g > tol2 * a * b) *flag = 1;
  }
}

__global__ void k_or_status(int* __restrict__ status, int v) { atomicOr(status, v); }

__global__ void k_ns_coeff(double* __restrict__ G, int64_t l) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < l * l) G[idx] = (idx / l == idx % l ? 1.5 : 0.0) - 0.5 * G[idx];
}

namespace {

// WP warps per column pair (measured on GB300 at l = 128 .. 1024): two for
// FP64, where the rotations load the FP64 units and every warp of a pair
// repeats the scalar work (four above l = 1024, to stay within 16 values per
// lane); four for FP32 at l >= 512 and two below, where a round is
// latency-bound and shorter per-warp chains help.
template <typename T, int WP>
int launch_jacobi_wp(const Dla& d, T* cols, T* Vc, T* nrm, int64_t l, int64_t rows, double tol, double tol_stop,
                     const double* fnorm, double tiny_rel, int max_sweeps, int* rot, int* status) {
  int li = (int)l, lp = (int)(l + (l & 1)), ri = (int)rows, msw = max_sweeps;
  const int threads = 32 * WP;
  const int pairs = lp / 2;
  void* args[] = {&cols, &Vc, &nrm, &li, &lp, &ri, &tol, &tol_stop, &fnorm, &tiny_rel, &msw, &rot, &status};
  auto launch = [&](auto kern) -> int {
    int occ = 0;
    BSRHT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, 0));
    const int blocks = std::max(1, std::min(pairs, num_sms() * std::max(occ, 1)));
    const int st = launch_cooperative((const void*)kern, dim3(blocks), dim3(threads), args, 0, d.s);
    if (st != BSRHT_OK) return st;
    note_launches(1);
    return BSRHT_OK;
  };
  if (l <= 1) return BSRHT_OK;
  const int64_t per = (rows + 32 * WP - 1) / (32 * WP);  // values per lane and column
  if (per <= 1) return launch(k_jacobi<T, 1, WP>);
  if (per <= 2) return launch(k_jacobi<T, 2, WP>);
  if (per <= 4) return launch(k_jacobi<T, 4, WP>);
  if (per <= 8) return launch(k_jacobi<T, 8, WP>);
  if (per <= 16) return launch(k_jacobi<T, 16, WP>);
  if constexpr (sizeof(T) == 4) {
    if (per <= 32) return launch(k_jacobi<T, 32, WP>);
  }
  return BSRHT_EUNSUP;
}

// l columns of `rows` entries each (rows = l for a square matrix).
template <typename T>
int launch_jacobi(const Dla& d, T* cols, T* Vc, T* nrm, int64_t l, int64_t rows, double tol, double tol_stop,
                  const double* fnorm, double tiny_rel, int max_sweeps, int* rot, int* status) {
  if constexpr (sizeof(T) == 8) {
    if (rows <= 1024)
      return launch_jacobi_wp<T, 2>(d, cols, Vc, nrm, l, rows, tol, tol_stop, fnorm, tiny_rel, max_sweeps, rot,
                                    status);
    return launch_jacobi_wp<T, 4>(d, cols, Vc, nrm, l, rows, tol, tol_stop, fnorm, tiny_rel, max_sweeps, rot,
                                  status);
  } else if (rows >= 512)
    return launch_jacobi_wp<T, 4>(d, cols, Vc, nrm, l, rows, tol, tol_stop, fnorm, tiny_rel, max_sweeps, rot,
                                  status);
  else
    return launch_jacobi_wp<T, 2>(d, cols, Vc, nrm, l, rows, tol, tol_stop, fnorm, tiny_rel, max_sweeps, rot,
                                  status);
}

// Block one-sided Jacobi (FP32 phase of the mixed SVD).  The columns are cut
// into nblk blocks of B (the last ones padded with absent columns); CTA c
// holds the block pair of round-robin position c in shared memory (M and V
// columns), so a grid barrier is needed only between block rounds.  In the
// first block round of a sweep the pairs inside each of the two blocks are
// treated (B - 1 rounds of round-robin), in every block round the B x B cross
// pairs (B rounds, warp w pairs column w of the first block with column
// (w + r) mod B of the second): over a sweep every pair of columns is
// rotated exactly once, as in the scalar kernel, with the same rotation and
// stopping rules.  Column norms are formed exactly when a block pair is
// loaded and carried through the rotations in between.
template <int B, int JR, bool VEC, int WP>
__global__ void __launch_bounds__(32 * B * WP) k_jacobi_blk(float* __restrict__ M, float* __restrict__ V, int l, int nblk,
                                                       double tol, double tol_stop, const double* __restrict__ fnorm,
                                                       double tiny_rel, int max_sweeps,
                                                       int* __restrict__ rot_counts) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ float jsm[];
  float* Ms = jsm;
  float* Vs = jsm + (size_t)2 * B * l;
  float* nrm = Vs + (size_t)2 * B * l;
  float* part = nrm + 2 * B;  // [B][WP]: the pair's warps' partial inner products (WP > 1)
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pw = w / WP, hw = w % WP;  // pair slot and half of the warp
  const float ttol = (float)tol, tstop = (float)tol_stop;
  const double tiny = tiny_rel * fnorm[0];
  const float tiny2 = (float)(tiny * tiny);
  auto gcol = [&](int P, int Q, int j) { return j < B ? P * B + j : Q * B + (j - B); };
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int R = 0; R < nblk - 1; ++R) {
      const int P = rr_player(blockIdx.x, R, nblk), Q = rr_player(nblk - 1 - blockIdx.x, R, nblk);
      // The B columns of a block are one contiguous run of B l floats (16-byte
      // aligned: B is a multiple of 4); copy both runs with float4 accesses,
      // all in flight at once.  Absent columns (>= l) read as zero.
      for (int h = 0; h < 2; ++h) {
        const int blk = h ? Q : P;
        const int64_t valid = (int64_t)max(0, min(B, l - blk * B)) * l;  // floats present
        const float4* gm = reinterpret_cast<const float4*>(M + (int64_t)blk * B * l);
        const float4* gv = reinterpret_cast<const float4*>(V + (int64_t)blk * B * l);
        float4* sm4 = reinterpret_cast<float4*>(Ms + (size_t)h * B * l);
        float4* sv4 = reinterpret_cast<float4*>(Vs + (size_t)h * B * l);
        const int n4 = B * l / 4;
#pragma unroll 4
        for (int i = threadIdx.x; i < n4; i += blockDim.x) {
          float4 xm = make_float4(0.f, 0.f, 0.f, 0.f), xv = xm;
          if (4 * (int64_t)i + 3 < valid) {
            xm = gm[i];
            xv = gv[i];
          } else if (4 * (int64_t)i < valid) {
            const float* m1 = reinterpret_cast<const float*>(gm + i);
            const float* v1 = reinterpret_cast<const float*>(gv + i);
            const int64_t left = valid - 4 * (int64_t)i;
            xm.x = m1[0]; xv.x = v1[0];
            if (left > 1) { xm.y = m1[1]; xv.y = v1[1]; }
            if (left > 2) { xm.z = m1[2]; xv.z = v1[2]; }
          }
          sm4[i] = xm;
          sv4[i] = xv;
        }
      }
      __syncthreads();
      for (int j = w; j < 2 * B; j += B * WP) {
        const float* col = Ms + (size_t)j * l;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        int r = lane;
        for (; r + 96 < l; r += 128) {
          s0 = fmaf(col[r], col[r], s0);
          s1 = fmaf(col[r + 32], col[r + 32], s1);
          s2 = fmaf(col[r + 64], col[r + 64], s2);
          s3 = fmaf(col[r + 96], col[r + 96], s3);
        }
        for (; r < l; r += 32) s0 = fmaf(col[r], col[r], s0);
        const float sq = warp_sum((s0 + s1) + (s2 + s3));
        if (lane == 0) nrm[j] = sq;
      }
      __syncthreads();
      const int nr = (R == 0 ? B - 1 : 0) + B;
      for (int ir = 0; ir < nr; ++ir) {
        int p, q;
        if (R == 0 && ir < B - 1) {  // inside block 0 (pair slots 0..B/2-1) or block 1
          const int half = pw / (B / 2), k = pw % (B / 2);
          p = half * B + rr_player(k, ir, B);
          q = half * B + rr_player(B - 1 - k, ir, B);
        } else {
          const int cr = ir - (R == 0 ? B - 1 : 0);
          p = pw;
          q = B + (pw + cr) % B;
        }
        const int gp = gcol(P, Q, p), gq = gcol(P, Q, q);
        float* a = Ms + (size_t)p * l;
        float* b = Ms + (size_t)q * l;
        float* va = Vs + (size_t)p * l;
        float* vb = Vs + (size_t)q * l;
        const float alpha = nrm[p], beta = nrm[q];
        bool skip = gp >= l || gq >= l || (alpha <= tiny2 && beta <= tiny2);
        if constexpr (VEC) {
          if (!skip) {
          // l % 4 == 0: the lane holds rows 128 e + 4 lane + j (j < 4) of the
          // two columns of M and V, moved with 16-byte shared-memory accesses,
          // and rotates them as packed pairs (rows j = 0, 1 and 2, 3).  With
          // WP > 1 the pair's WP warps take the chunks e = WP e' + hw and add
          // their partial inner products through shared memory (a named
          // barrier of 32 WP threads per pair), in the same order in every
          // warp, so all derive the same rotation.
          constexpr int JQ = JR / 4 / WP;
          const ulonglong2* a2 = reinterpret_cast<const ulonglong2*>(a);
          const ulonglong2* b2 = reinterpret_cast<const ulonglong2*>(b);
          const ulonglong2* va2 = reinterpret_cast<const ulonglong2*>(va);
          const ulonglong2* vb2 = reinterpret_cast<const ulonglong2*>(vb);
          ulonglong2 x[JQ], y[JQ], vx[JQ], vy[JQ];
          const ulonglong2 z2 = make_ulonglong2(0ull, 0ull);
#pragma unroll
          for (int e = 0; e < JQ; ++e) {
            const int c4 = 32 * (WP * e + hw) + lane;  // 16-byte chunk: rows 4 c4 .. 4 c4 + 3
            const bool in = 4 * c4 < l;
            x[e] = in ? a2[c4] : z2;
            y[e] = in ? b2[c4] : z2;
            vx[e] = in ? va2[c4] : z2;
            vy[e] = in ? vb2[c4] : z2;
          }
          f2 g2[2] = {0ull, 0ull};
#pragma unroll
          for (int e = 0; e < JQ; ++e) {
            g2[e & 1] = f2_fma(x[e].x, y[e].x, g2[e & 1]);
            g2[e & 1] = f2_fma(x[e].y, y[e].y, g2[e & 1]);
          }
          const float2 gp = f2_to_float2(f2_add(g2[0], g2[1]));
          float gamma = warp_sum(gp.x + gp.y);
          if constexpr (WP > 1) {
            if (lane == 0) part[WP * pw + hw] = gamma;
            asm volatile("bar.sync %0, %1;" ::"r"(1 + pw), "r"(32 * WP) : "memory");
            gamma = part[WP * pw];
#pragma unroll
            for (int h = 1; h < WP; ++h) gamma += part[WP * pw + h];
          }
          const float gnorm = sqrtf(alpha) * sqrtf(beta);
          if (gamma != 0.f && fabsf(gamma) > ttol * gnorm) {
            const float t = jac_tangent(alpha, beta, gamma);
            const float c = rsqrtf(1.f + t * t), sn = c * t;
            const f2 C2 = f2_splat(c), S2 = f2_splat(sn), NS2 = f2_splat(-sn);
            // new p = c x - s y = (-s) y + c x, new q = s x + c y = c y + s x
#pragma unroll
            for (int e = 0; e < JQ; ++e) {
              const int c4 = 32 * (WP * e + hw) + lane;
              if (4 * c4 < l) {
                ulonglong2 na, nb, nva, nvb;
                na.x = f2_fma(y[e].x, NS2, f2_mul(x[e].x, C2));
                na.y = f2_fma(y[e].y, NS2, f2_mul(x[e].y, C2));
                nb.x = f2_fma(y[e].x, C2, f2_mul(x[e].x, S2));
                nb.y = f2_fma(y[e].y, C2, f2_mul(x[e].y, S2));
                nva.x = f2_fma(vy[e].x, NS2, f2_mul(vx[e].x, C2));
                nva.y = f2_fma(vy[e].y, NS2, f2_mul(vx[e].y, C2));
                nvb.x = f2_fma(vy[e].x, C2, f2_mul(vx[e].x, S2));
                nvb.y = f2_fma(vy[e].y, C2, f2_mul(vx[e].y, S2));
                reinterpret_cast<ulonglong2*>(a)[c4] = na;
                reinterpret_cast<ulonglong2*>(b)[c4] = nb;
                reinterpret_cast<ulonglong2*>(va)[c4] = nva;
                reinterpret_cast<ulonglong2*>(vb)[c4] = nvb;
              }
            }
            if (hw == 0 && lane == 0) {
              nrm[p] = alpha - t * gamma;
              nrm[q] = beta + t * gamma;
              if (fabsf(gamma) > tstop * gnorm) atomicAdd(&rot_counts[sweep], 1);
            }
          }
          }
        } else if (!skip) {
          // The warp's two columns of M and of V in registers (JR values per
          // lane; rows lane + 32 e), loaded back to back.
          float x[JR], y[JR], vx[JR], vy[JR];
#pragma unroll
          for (int e = 0; e < JR; ++e) {
            const int r = lane + 32 * e;
            const bool in = r < l;
            x[e] = in ? a[r] : 0.f;
            y[e] = in ? b[r] : 0.f;
            vx[e] = in ? va[r] : 0.f;
            vy[e] = in ? vb[r] : 0.f;
          }
          float g4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int e = 0; e < JR; ++e) g4[e & 3] = fmaf(x[e], y[e], g4[e & 3]);
          const float gamma = warp_sum((g4[0] + g4[1]) + (g4[2] + g4[3]));
          const float gnorm = sqrtf(alpha) * sqrtf(beta);
          if (gamma != 0.f && fabsf(gamma) > ttol * gnorm) {
            const float t = jac_tangent(alpha, beta, gamma);
            const float c = rsqrtf(1.f + t * t), s = c * t;
#pragma unroll
            for (int e = 0; e < JR; ++e) {
              const int r = lane + 32 * e;
              if (r < l) {
                a[r] = c * x[e] - s * y[e];
                b[r] = s * x[e] + c * y[e];
                va[r] = c * vx[e] - s * vy[e];
                vb[r] = s * vx[e] + c * vy[e];
              }
            }
            if (lane == 0) {
              nrm[p] = alpha - t * gamma;
              nrm[q] = beta + t * gamma;
              if (fabsf(gamma) > tstop * gnorm) atomicAdd(&rot_counts[sweep], 1);
            }
          }
        }
        __syncthreads();
      }
      for (int h = 0; h < 2; ++h) {
        const int blk = h ? Q : P;
        const int64_t valid = (int64_t)max(0, min(B, l - blk * B)) * l;
        float4* gm = reinterpret_cast<float4*>(M + (int64_t)blk * B * l);
        float4* gv = reinterpret_cast<float4*>(V + (int64_t)blk * B * l);
        const float4* sm4 = reinterpret_cast<const float4*>(Ms + (size_t)h * B * l);
        const float4* sv4 = reinterpret_cast<const float4*>(Vs + (size_t)h * B * l);
        const int n4 = B * l / 4;
#pragma unroll 4
        for (int i = threadIdx.x; i < n4; i += blockDim.x) {
          if (4 * (int64_t)i + 3 < valid) {
            gm[i] = sm4[i];
            gv[i] = sv4[i];
          } else if (4 * (int64_t)i < valid) {
            float* m1 = reinterpret_cast<float*>(gm + i);
            float* v1 = reinterpret_cast<float*>(gv + i);
            const float4 xm = sm4[i], xv = sv4[i];
            const int64_t left = valid - 4 * (int64_t)i;
            m1[0] = xm.x; v1[0] = xv.x;
            if (left > 1) { m1[1] = xm.y; v1[1] = xv.y; }
            if (left > 2) { m1[2] = xm.z; v1[2] = xv.z; }
          }
        }
      }
      grid.sync();
    }
    if (*((volatile int*)&rot_counts[sweep]) == 0) break;
  }
}

// Two warps per column pair (each on half the rows) in the 16-byte form
// when a lane holds at least two 16-byte chunks: four warps per scheduler
// instead of two hide the shared-memory and FMA latencies of a round.
template <int B, int JR, bool VEC>
int launch_jacobi_blk_v(const Dla& d, float* M, float* V, int64_t l, double tol, double tol_stop,
                        const double* fnorm, double tiny_rel, int max_sweeps, int* rot) {
  constexpr int WP = (VEC && JR >= 8) ? 2 : 1;
  constexpr int NT = 32 * B * WP;
  auto kern = k_jacobi_blk<B, JR, VEC, WP>;
  int li = (int)l, nblk = (int)((l + B - 1) / B), msw = max_sweeps;
  nblk += nblk & 1;
  const size_t smem = sizeof(float) * ((size_t)4 * B * l + (2 + WP) * B);
  // One instance serves every l up to 32 JR, and host threads (the server's
  // executors) launch it concurrently: the attribute is always set to the
  // largest of them, so no thread lowers it below another one's launch.
  const size_t smem_max = sizeof(float) * ((size_t)4 * B * 32 * JR + (2 + WP) * B);
  BSRHT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
  int occ = 0;
  BSRHT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem));
  if ((int64_t)(nblk / 2) > (int64_t)occ * num_sms()) return BSRHT_EUNSUP;  // not co-resident: caller falls back
  void* args[] = {&M, &V, &li, &nblk, &tol, &tol_stop, &fnorm, &tiny_rel, &msw, &rot};
  const int st = launch_cooperative((const void*)kern, dim3(nblk / 2), dim3(NT), args, smem, d.s);
  if (st != BSRHT_OK) return st;
  note_launches(1);
  return BSRHT_OK;
}

// The 16-byte form when the columns (and so the blocks) start on 16 bytes.
template <int B, int JR>
int launch_jacobi_blk_b(const Dla& d, float* M, float* V, int64_t l, double tol, double tol_stop,
                        const double* fnorm, double tiny_rel, int max_sweeps, int* rot) {
  if (l % 4 == 0)
    return launch_jacobi_blk_v<B, JR, true>(d, M, V, l, tol, tol_stop, fnorm, tiny_rel, max_sweeps, rot);
  return launch_jacobi_blk_v<B, JR, false>(d, M, V, l, tol, tol_stop, fnorm, tiny_rel, max_sweeps, rot);
}

template <int B>
int launch_jacobi_blk_jr(const Dla& d, float* M, float* V, int64_t l, double tol, double tol_stop,
                         const double* fnorm, double tiny_rel, int max_sweeps, int* rot) {
  if (l <= 128) return launch_jacobi_blk_b<B, 4>(d, M, V, l, tol, tol_stop, fnorm, tiny_rel, max_sweeps, rot);
  if (l <= 256) return launch_jacobi_blk_b<B, 8>(d, M, V, l, tol, tol_stop, fnorm, tiny_rel, max_sweeps, rot);
  if (l <= 512) return launch_jacobi_blk_b<B, 16>(d, M, V, l, tol, tol_stop, fnorm, tiny_rel, max_sweeps, rot);
  if constexpr (B <= 8) {
    if (l <= 1024) return launch_jacobi_blk_b<B, 32>(d, M, V, l, tol, tol_stop, fnorm, tiny_rel, max_sweeps, rot);
  }
  return BSRHT_EUNSUP;
}

// Blocks of 8 columns, for l <= 1024.  Only l / 16 CTAs work, and a block
// round is bound by their instruction issue and latency (ncu at l = 512,
// B = 16: 43 % issue-active), so the block form wins only while the grid
// barriers it saves outweigh the SMs it leaves idle.  Measured on GB300,
// FP32 phase of the benchmark's rSVD (16-byte accesses, packed rotations
// and two warps per pair when l % 4 == 0): l = 512 7.3 ms (B = 8, one warp
// per pair 7.9; scalar kernel 11.6 ms, B = 4 10.4 ms, B = 16 13.3 ms),
// l = 600 11.1 ms (one warp 12.3, scalar 14.1), l = 1024 22.9 ms (one warp
// 28.4, scalar 34.9).  BSRHT_EUNSUP sends the caller to the
// scalar kernel (also when the block pairs cannot all be resident at once).
int launch_jacobi_blk(const Dla& d, float* M, float* V, int64_t l, double tol, double tol_stop, const double* fnorm,
                      double tiny_rel, int max_sweeps, int* rot) {
  if (l <= 1 || l > 1024) return BSRHT_EUNSUP;
  return launch_jacobi_blk_jr<8>(d, M, V, l, tol, tol_stop, fnorm, tiny_rel, max_sweeps, rot);
}

}  // namespace

int jacobi_svd(const Dla& d, Arena& ar, double* colsM, int64_t l, double* U, double* sigma, double* Vout,
               double polish_tol, double zero_rel, int64_t ktop, double keep_rel) {
  if (l > 2048) return BSRHT_EUNSUP;
  const int max_sweeps = 40;
  // Rotate only while the cosine of the pair exceeds sqrt(l) eps (the usual
  // one-sided Jacobi threshold); a tighter one keeps rotating at noise level.
  const double tol = polish_tol > 0.0 ? polish_tol : std::max(1e-15, std::sqrt((double)l) * 0x1.0p-52);
  const bool mixed = l > kJacobiMixedMin;
  // Callers at FP32-data accuracy that use only the leading ktop triplets
  // polish the s leading columns of the FP32 phase (a margin of
  // max(16, ktop / 4) beyond ktop) and keep the FP32 phase's estimates for
  // the rest.
  // With keep_rel > 0 instead, the leading columns are those whose FP32
  // norm exceeds keep_rel times the largest (counted after the FP32 phase),
  // with the same margin; the workspace is sized for all l.
  auto with_margin = [&](int64_t c) { return std::min<int64_t>(l, c + std::max<int64_t>(16, c / 4)); };
  const bool part_mode = mixed && polish_tol > 0.0 && (ktop > 0 || keep_rel > 0.0);
  int64_t s = part_mode ? (ktop > 0 ? with_margin(ktop) : l) : l;
  const bool part = part_mode && (s < l || keep_rel > 0.0);
  double* Vc = static_cast<double*>(ar.take(sizeof(double) * l * l));
  double* sig = static_cast<double*>(ar.take(sizeof(double) * l));
  int* perm = static_cast<int*>(ar.take(sizeof(int) * l));
  int* rot = static_cast<int*>(ar.take(sizeof(int) * 2 * max_sweeps));
  double* fnorm = static_cast<double*>(ar.take(sizeof(double)));
  double* nrm64 = static_cast<double*>(ar.take(sizeof(double) * l));
  float* nrm32 = static_cast<float*>(ar.take(sizeof(float) * l));
  double* Yt = static_cast<double*>(ar.take(sizeof(double) * l * l));  // convergence test: columns, row-major
  double* Gc = static_cast<double*>(ar.take(sizeof(double) * l * l));  // and their Gram
  int* cflag = static_cast<int*>(ar.take(sizeof(int)));
  double* sigS = static_cast<double*>(ar.take(sizeof(double) * l));
  int* permS = static_cast<int*>(ar.take(sizeof(int) * l));
  float *M32 = nullptr, *V32 = nullptr;
  double *S2 = nullptr, *G = nullptr, *Y = nullptr;
  if (mixed) {
    M32 = static_cast<float*>(ar.take(sizeof(float) * l * l));
    V32 = static_cast<float*>(ar.take(sizeof(float) * l * l));
    S2 = static_cast<double*>(ar.take(sizeof(double) * l * l));
    G = static_cast<double*>(ar.take(sizeof(double) * l * l));
    Y = static_cast<double*>(ar.take(sizeof(double) * l * l));
  }
  if (!ar.ok()) return BSRHT_ENOMEM;
  // FP64 products (row-major operands); each releases its split-K scratch.
  auto gemm_f64 = [&](int64_t Mm, int64_t Nn, int64_t Kk, const double* A, int64_t lda, bool a_trans,
                      const double* B, int64_t ldb, double* C, int64_t ldc, bool gram) -> int {
    const size_t mk = ar.mark();
    const int st = gemm(d, ar, DT::F64, DT::F64, DT::F64, true, Mm, Nn, Kk, A, lda, a_trans, B, ldb, C, ldc, 1.0,
                        0.0, false, gram);
    ar.release(mk);
    return st;
  };
  auto gemm64 = [&](const double* A, bool a_trans, const double* B, double* C, bool gram) -> int {
    return gemm_f64(l, l, l, A, l, a_trans, B, l, C, l, gram);
  };
  {
    const size_t mk = ar.mark();
    const int st = frob_norm(d, ar, DT::F64, colsM, l * l, fnorm);
    ar.release(mk);
    if (st != BSRHT_OK) return st;
  }
  if (ar.measure) {  // every product below
    TRY_DLA(gemm_f64(s, s, l, nullptr, s, true, nullptr, s, nullptr, s, true));
    if (mixed) {
      TRY_DLA(gemm64(nullptr, true, nullptr, nullptr, true));
      TRY_DLA(gemm64(nullptr, false, nullptr, nullptr, false));
    }
    if (part) {
      TRY_DLA(gemm_f64(l, s, s, nullptr, s, false, nullptr, s, nullptr, s, false));
      TRY_DLA(gemm_f64(l, s, l, nullptr, l, true, nullptr, s, nullptr, s, false));
    }
    return BSRHT_OK;
  }
  BSRHT_CUDA_TRY(cudaMemsetAsync(rot, 0, sizeof(int) * 2 * max_sweeps, d.s));

  // FP64 one-sided Jacobi of nc columns of `rows` entries (pc, the same
  // rotations on pv), one sweep per launch.  A sweep without a significant
  // rotation ends it.  After a sweep that rotated at most 1/16 of the pairs,
  // the cosines of all pairs come from the Gram of the columns (one FP64
  // product) instead of a further sweep, and the sweeps stop once none
  // exceeds the stopping threshold 16 tol: the test that sweep would make
  // pair by pair.  (Clustered singular values keep the rotation angles
  // large while the cosines shrink, so the last rotating sweep is not known
  // in advance.)
  auto polish = [&](double* pc, double* pv, int64_t nc, int64_t rows) -> int {
    const double tiny_rel = std::max((double)l * 0x1.0p-53, zero_rel);
    const unsigned cblocks = (unsigned)std::min<int64_t>(blocks_for(nc * nc, 256), 4096);
    bool converged = false;
    for (int sw = 0; sw < max_sweeps && !converged; ++sw) {
      TRY_DLA(launch_jacobi<double>(d, pc, pv, nrm64, nc, rows, tol, 16.0 * tol, fnorm, tiny_rel, 1, rot + sw,
                                    nullptr));
      int cnt = 0;
      BSRHT_CUDA_TRY(cudaMemcpyAsync(&cnt, rot + sw, sizeof(int), cudaMemcpyDeviceToHost, d.s));
      BSRHT_CUDA_TRY(cudaStreamSynchronize(d.s));
      if (cnt == 0) {
        converged = true;
        break;
      }
      if ((int64_t)cnt * 16 > nc * (nc - 1) / 2) continue;
      TRY_DLA(transpose_cast(d, DT::F64, pc, nc, rows, rows, DT::F64, Yt, nc));  // rows x nc
      TRY_DLA(gemm_f64(nc, nc, rows, Yt, nc, true, Yt, nc, Gc, nc, true));
      BSRHT_CUDA_TRY(cudaMemsetAsync(cflag, 0, sizeof(int), d.s));
      k_offdiag_exceeds<<<cblocks, 256, 0, d.s>>>(Gc, nc, fnorm, tiny_rel, 16.0 * tol, cflag);
      DLA_LAUNCH_CHECK();
      note_launches(1);
      int h = 1;
      BSRHT_CUDA_TRY(cudaMemcpyAsync(&h, cflag, sizeof(int), cudaMemcpyDeviceToHost, d.s));
      BSRHT_CUDA_TRY(cudaStreamSynchronize(d.s));
      converged = h == 0;
    }
    if (!converged) {
      k_or_status<<<1, 1, 0, d.s>>>(d.status, kStatusNoConv);
      DLA_LAUNCH_CHECK();
      note_launches(1);
    }
    return BSRHT_OK;
  };

  double* cols = colsM;
  if (mixed) {
    // 1. FP32 one-sided Jacobi on a copy of M: V32 ~ the right singular
    //    vectors to FP32 accuracy, at 64x the FP64 rate of this GPU (block
    //    Jacobi in shared memory: one grid barrier per block round).
    TRY_DLA(cast_copy(d, DT::F64, colsM, DT::F32, M32, l * l));
    k_init_identity_cols<float><<<blocks_for(l * l, 256), 256, 0, d.s>>>(V32, l);
    DLA_LAUNCH_CHECK();
    const double tol32 = 16.0 * std::sqrt((double)l) * 0x1.0p-24;
    // With the partial FP64 polish behind it, the FP32 phase ends after the
    // first sweep whose rotations all stayed below 8 tol32 (they are still
    // applied down to tol32): the sweeps after it only confirm what the
    // polish's Rayleigh-Ritz step settles anyway (measured at l = 512: one
    // FP32 sweep less, the same number of FP64 sweeps, sigma_k equal to
    // 5e-13 relative).  A full FP64 polish keeps the tight stop.
    const double tstop32 = part ? 8.0 * tol32 : tol32;
    const int bst =
        launch_jacobi_blk(d, M32, V32, l, tol32, tstop32, fnorm, (double)l * 0x1.0p-24, 20, rot + max_sweeps);
    if (bst == BSRHT_EUNSUP)
      TRY_DLA(launch_jacobi<float>(d, M32, V32, nrm32, l, l, tol32, tstop32, fnorm, (double)l * 0x1.0p-24, 20,
                                   rot + max_sweeps, nullptr));
    else if (bst != BSRHT_OK)
      return bst;
    trace_mark(d.s, "svd_jacobi_fp32");
    if (part) {
      // 2'. The s leading columns by the FP32 norms: their V32 columns made
      //     orthonormal in FP64 (Vr, l x s row-major: two Newton-Schulz
      //     steps Vr <- Vr (1.5 I - 0.5 Vr^T Vr)), Y_S = M Vr, then the FP64
      //     Jacobi on the s columns of Y_S.  In exact arithmetic this is the
      //     SVD of M restricted to span(Vr) (Rayleigh-Ritz); it differs from
      //     the leading triplets of M by terms of second order in the FP32
      //     phase's residual cosines between the s columns and the rest.
      k_col_norms_t<float><<<blocks_for(l, 8), 256, 0, d.s>>>(M32, sig, l, l);
      DLA_LAUNCH_CHECK();
      k_rank_desc<<<blocks_for(l, 256), 256, 0, d.s>>>(sig, perm, l);
      DLA_LAUNCH_CHECK();
      if (ktop <= 0) {
        std::vector<double> sh((size_t)l);
        BSRHT_CUDA_TRY(cudaMemcpyAsync(sh.data(), sig, sizeof(double) * l, cudaMemcpyDeviceToHost, d.s));
        BSRHT_CUDA_TRY(cudaStreamSynchronize(d.s));
        const double smax = *std::max_element(sh.begin(), sh.end());
        int64_t c = 0;
        for (double v : sh) c += v > keep_rel * smax;
        s = with_margin(std::max<int64_t>(c, 1));
      }
      double* Vr = S2;
      double* Vn = Vc;
      k_gather_cols_t<<<blocks_for(l * s, 256), 256, 0, d.s>>>(V32, perm, l, s, Vr);
      DLA_LAUNCH_CHECK();
      note_launches(3);
      for (int it = 0; it < 2; ++it) {
        TRY_DLA(gemm_f64(s, s, l, Vr, s, true, Vr, s, G, s, true));  // G = Vr^T Vr
        k_ns_coeff<<<blocks_for(s * s, 256), 256, 0, d.s>>>(G, s);   // G <- 1.5 I - 0.5 G
        DLA_LAUNCH_CHECK();
        note_launches(1);
        TRY_DLA(gemm_f64(l, s, s, Vr, s, false, G, s, Vn, s, false));
        std::swap(Vr, Vn);
      }
      TRY_DLA(gemm_f64(l, s, l, colsM, l, true, Vr, s, Y, s, false));  // Y_S = M Vr (colsM row-major is M^T)
      double* Ysc = colsM;                                               // column storage: s x l
      double* Vsc = G;
      TRY_DLA(transpose_cast(d, DT::F64, Y, l, s, s, DT::F64, Ysc, l));
      TRY_DLA(transpose_cast(d, DT::F64, Vr, l, s, s, DT::F64, Vsc, l));
      trace_mark(d.s, "svd_orthogonalize");
      TRY_DLA(polish(Ysc, Vsc, s, l));
      k_col_norms_t<double><<<blocks_for(s, 8), 256, 0, d.s>>>(Ysc, sigS, s, l);
      DLA_LAUNCH_CHECK();
      k_rank_desc<<<blocks_for(s, 256), 256, 0, d.s>>>(sigS, permS, s);
      DLA_LAUNCH_CHECK();
      k_svd_finish_part<<<blocks_for(l * l, 256), 256, 0, d.s>>>(Ysc, Vsc, sigS, permS, s, M32, V32, sig, perm, l,
                                                                  U, Vout, sigma);
      DLA_LAUNCH_CHECK();
      note_launches(3);
      return BSRHT_OK;
    }
    // 2. Make it orthogonal in FP64: with S = V0^T (the column storage),
    //    two Newton-Schulz steps S <- 1.5 S - 0.5 S (S^T S) take the
    //    orthogonality error from that of the accumulated FP32 rotations
    //    to rounding level.
    TRY_DLA(cast_copy(d, DT::F32, V32, DT::F64, Vc, l * l));
    for (int it = 0; it < 2; ++it) {
      TRY_DLA(gemm64(Vc, true, Vc, G, true));  // G = S^T S
      k_ns_coeff<<<blocks_for(l * l, 256), 256, 0, d.s>>>(G, l);  // G <- 1.5 I - 0.5 G
      DLA_LAUNCH_CHECK();
      note_launches(1);
      TRY_DLA(gemm64(Vc, false, G, S2, false));
      std::swap(Vc, S2);
    }
    // 3. Y = (M V0)^T in column storage: Y = S T with T = M^T the column
    //    storage of M.  The FP64 Jacobi below starts from V = V0, so its
    //    rotations compose onto V0 and M V = U Sigma holds for the result.
    TRY_DLA(gemm64(Vc, false, colsM, Y, false));
    cols = Y;
    trace_mark(d.s, "svd_orthogonalize");
  } else {
    k_init_identity_cols<double><<<blocks_for(l * l, 256), 256, 0, d.s>>>(Vc, l);
    DLA_LAUNCH_CHECK();
  }
  // 4. FP64 one-sided Jacobi (from V0 it converges in a few sweeps).
  TRY_DLA(polish(cols, Vc, l, l));
  k_col_norms<<<blocks_for(l, 8), 256, 0, d.s>>>(cols, sig, l);
  DLA_LAUNCH_CHECK();
  k_rank_desc<<<blocks_for(l, 256), 256, 0, d.s>>>(sig, perm, l);
  DLA_LAUNCH_CHECK();
  k_svd_finish<<<blocks_for(l * l, 256), 256, 0, d.s>>>(cols, Vc, sig, perm, U, Vout, sigma, l);
  DLA_LAUNCH_CHECK();
  note_launches(4);
  return BSRHT_OK;
}

// ------------------------------------------------------------ helpers
// 64 x 64 tiles through shared memory (TS: float unless a side is double;
// one padding column keeps both passes free of bank conflicts), 16 elements
// per thread in flight.  A 1-D grid of tile indices, so any row count fits.
template <typename TI, typename TO, typename TS>
__global__ void __launch_bounds__(256) k_transpose_cast(const TI* __restrict__ in, int64_t rows, int64_t cols,
                                                        int64_t ldin, TO* __restrict__ out, int64_t ldout,
                                                        int64_t tiles_c) {
  __shared__ TS t[64][65];
  const int64_t tr = (int64_t)blockIdx.x / tiles_c, tcol = (int64_t)blockIdx.x - tr * tiles_c;
  const int64_t br = tr * 64, bc = tcol * 64;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
#pragma unroll
  for (int r = ty; r < 64; r += 8) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t i = br + r, j = bc + tx + 32 * h;
      t[r][tx + 32 * h] = (i < rows && j < cols) ? (TS)in[i * ldin + j] : (TS)0;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = ty; r < 64; r += 8) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t j = bc + r, i = br + tx + 32 * h;
      if (i < rows && j < cols) out[j * ldout + i] = (TO)t[tx + 32 * h][r];
    }
  }
}

int transpose_cast(const Dla& d, DT tin, const void* in, int64_t rows, int64_t cols, int64_t ldin, DT tout,
                   void* out, int64_t ldout) {
  if (rows <= 0 || cols <= 0) return BSRHT_OK;
  const int64_t tiles_c = (cols + 63) / 64, tiles = tiles_c * ((rows + 63) / 64);
  if (tiles > 0x7FFFFFFF) return BSRHT_EUNSUP;
  const unsigned grid = (unsigned)tiles;
#define TC_CASE(TIT, TOT, TST)                                                                           \
  k_transpose_cast<TIT, TOT, TST><<<grid, 256, 0, d.s>>>(static_cast<const TIT*>(in), rows, cols, ldin, \
                                                         static_cast<TOT*>(out), ldout, tiles_c)
  if (tin == DT::F64 && tout == DT::F64) TC_CASE(double, double, double);
  else if (tin == DT::F32 && tout == DT::F64) TC_CASE(float, double, float);
  else if (tin == DT::F32 && tout == DT::F32) TC_CASE(float, float, float);
  else if (tin == DT::F64 && tout == DT::F32) TC_CASE(double, float, double);
  else return BSRHT_EUNSUP;
#undef TC_CASE
  DLA_LAUNCH_CHECK();
  note_launches(1);
  return BSRHT_OK;
}

template <typename TI, typename TO>
__global__ void k_cast(const TI* __restrict__ in, TO* __restrict__ out, int64_t count) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < count) out[idx] = (TO)in[idx];
}

int cast_copy(const Dla& d, DT tin, const void* in, DT tout, void* out, int64_t count) {
  if (count <= 0) return BSRHT_OK;
  if (tin == DT::F64 && tout == DT::F32)
    k_cast<double, float><<<blocks_for(count, 256), 256, 0, d.s>>>(static_cast<const double*>(in),
                                                                    static_cast<float*>(out), count);
  else if (tin == DT::F32 && tout == DT::F64)
    k_cast<float, double><<<blocks_for(count, 256), 256, 0, d.s>>>(static_cast<const float*>(in),
                                                                    static_cast<double*>(out), count);
  else if (tin == DT::F64 && tout == DT::F64)
    k_cast<double, double><<<blocks_for(count, 256), 256, 0, d.s>>>(static_cast<const double*>(in),
                                                                     static_cast<double*>(out), count);
  else
    return BSRHT_EUNSUP;
  DLA_LAUNCH_CHECK();
  note_launches(1);
  return BSRHT_OK;
}

int transpose_lower_to_upper(const Dla& d, const double* Li, double* R, int64_t l) {
  const unsigned t = (unsigned)((l + 31) / 32);
  k_transpose_sq<<<dim3(t, t), 256, 0, d.s>>>(Li, R, l);
  DLA_LAUNCH_CHECK();
  note_launches(1);
  return BSRHT_OK;
}

__global__ void k_scale_cols(double* X, int64_t rows, int64_t cols, int64_t ld, const double* sc, int inv) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int64_t i = idx / cols, j = idx % cols;
  const double s = sc[j];
  X[i * ld + j] = inv ? (s != 0.0 ? X[i * ld + j] / s : 0.0) : X[i * ld + j] * s;
}

int scale_columns(const Dla& d, double* X, int64_t rows, int64_t cols, int64_t ld, const double* scale,
                  bool invert) {
  if (rows * cols <= 0) return BSRHT_OK;
  k_scale_cols<<<blocks_for(rows * cols, 256), 256, 0, d.s>>>(X, rows, cols, ld, scale, invert ? 1 : 0);
  DLA_LAUNCH_CHECK();
  note_launches(1);
  return BSRHT_OK;
}

// Column argmax of |U| per row chunk: partial (value, index) per chunk.
__global__ void k_colargmax_partial(const double* __restrict__ U, int64_t n, int64_t k, int64_t rows_per,
                                    double* __restrict__ pv, int64_t* __restrict__ pi) {
  const int64_t c = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per, r1 = min(n, r0 + rows_per);
  double best = -1.0;
  int64_t bi = r0;
  for (int64_t i = r0; i < r1; ++i) {
    const double v = fabs(U[i * k + c]);
    if (v > best) {
      best = v;
      bi = i;
    }
  }
  pv[(int64_t)blockIdx.x * k + c] = best;
  pi[(int64_t)blockIdx.x * k + c] = bi;
}

__global__ void k_colargmax_final(const double* __restrict__ U, int64_t k, int nchunks, const double* pv,
                                  const int64_t* pi, double* __restrict__ sgn) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  double best = -1.0;
  int64_t bi = 0;
  for (int b = 0; b < nchunks; ++b) {
    const double v = pv[(int64_t)b * k + c];
    if (v > best) {
      best = v;
      bi = pi[(int64_t)b * k + c];
    }
  }
  sgn[c] = (U[bi * k + c] < 0.0) ? -1.0 : 1.0;
}

int sign_normalize(const Dla& d, Arena& ar, double* U, int64_t n, int64_t k, double* V, int64_t m) {
  const int nchunks = (int)std::min<int64_t>(1024, std::max<int64_t>(1, n / 256));
  const int64_t rows_per = (n + nchunks - 1) / nchunks;
  double* pv = static_cast<double*>(ar.take(sizeof(double) * nchunks * k));
  int64_t* pi = static_cast<int64_t*>(ar.take(sizeof(int64_t) * nchunks * k));
  double* sg = static_cast<double*>(ar.take(sizeof(double) * k));
  if (!ar.ok()) return BSRHT_ENOMEM;
  if (ar.measure) return BSRHT_OK;
  const int tb = (int)std::min<int64_t>(256, k);
  k_colargmax_partial<<<dim3(nchunks, blocks_for(k, tb)), tb, 0, d.s>>>(U, n, k, rows_per, pv, pi);
  DLA_LAUNCH_CHECK();
  k_colargmax_final<<<blocks_for(k, 128), 128, 0, d.s>>>(U, k, nchunks, pv, pi, sg);
  DLA_LAUNCH_CHECK();
  note_launches(2);
  int st = scale_columns(d, U, n, k, k, sg, false);
  if (st != BSRHT_OK) return st;
  if (V) st = scale_columns(d, V, m, k, k, sg, false);
  return st;
}

template <typename T>
__global__ void k_sumsq_partial(const T* __restrict__ X, int64_t count, double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)Elem<T>::to_f64(X[i]);
    s = fma(v, v, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_sqrt(const double* part, int count, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < count; ++i) s += part[i];
    *out = sqrt(s);
  }
}

int frob_norm(const Dla& d, Arena& ar, DT t, const void* X, int64_t count, double* out) {
  const int nb = 1024;
  double* part = static_cast<double*>(ar.take(sizeof(double) * nb));
  if (!ar.ok()) return BSRHT_ENOMEM;
  if (ar.measure) return BSRHT_OK;
  if (t == DT::F64)
    k_sumsq_partial<double><<<nb, 256, 0, d.s>>>(static_cast<const double*>(X), count, part);
  else if (t == DT::F32)
    k_sumsq_partial<float><<<nb, 256, 0, d.s>>>(static_cast<const float*>(X), count, part);
  else
    return BSRHT_EUNSUP;
  DLA_LAUNCH_CHECK();
  k_sum_sqrt<<<1, 32, 0, d.s>>>(part, nb, out);
  DLA_LAUNCH_CHECK();
  note_launches(2);
  return BSRHT_OK;
}

}  // namespace bsrht

namespace bsrht {

// ------------------------------------------------ Householder QR (FP64)
// Cooperative kernel: the rows of X are split into contiguous block ranges;
// every column step needs grid-wide sums, taken as per-block partials that
// every block then adds in block order (deterministic).
__global__ void k_house_qr(double* __restrict__ X, int64_t rows, int64_t l, double* __restrict__ tau,
                           double* __restrict__ part) {
  cg::grid_group grid = cg::this_grid();
  const int64_t nb = gridDim.x;
  const int64_t per = (rows + nb - 1) / nb;
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(rows, r0 + per);
  __shared__ double red[256];
  __shared__ double s_beta, s_v0, s_tau;
  for (int64_t j = 0; j < l; ++j) {
    // (1) sum of squares of X[i][j], i > j, per block
    double acc = 0.0;
    for (int64_t i = max(r0, j + 1) + threadIdx.x; i < r1; i += blockDim.x) acc = fma(X[i * l + j], X[i * l + j], acc);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
    grid.sync();
    // (2) reflector: every block derives the same scalars
    if (threadIdx.x == 0) {
      double sigma = 0.0;
      for (int64_t b = 0; b < nb; ++b) sigma += part[b];
      const double x0 = (j < rows) ? X[j * l + j] : 0.0;
      if (sigma == 0.0 || j >= rows) {
        s_beta = x0;
        s_v0 = 1.0;
        s_tau = 0.0;
      } else {
        const double alpha = sqrt(x0 * x0 + sigma);
        const double beta = x0 <= 0.0 ? alpha : -alpha;
        s_beta = beta;
        s_v0 = x0 - beta;
        s_tau = (beta - x0) / beta;
      }
    }
    __syncthreads();
    const double v0 = s_v0, tj = s_tau;
    for (int64_t i = max(r0, j + 1) + threadIdx.x; i < r1; i += blockDim.x) X[i * l + j] /= v0;
    grid.sync();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (j < rows) X[j * l + j] = s_beta;
      tau[j] = tj;
    }
    // (3) w_c = v^T X[j:, c] for c > j, per block (v_j = 1 implicit)
    for (int64_t c = j + 1 + threadIdx.x; c < l; c += blockDim.x) {
      double w = 0.0;
      if (j >= r0 && j < r1) w = X[j * l + c];
      for (int64_t i = max(r0, j + 1); i < r1; ++i) w = fma(X[i * l + j], X[i * l + c], w);
      part[(int64_t)blockIdx.x * l + c] = w;
    }
    grid.sync();
    // (4) X[i][c] -= tau v_i w_c
    if (tj != 0.0) {
      for (int64_t c = j + 1 + threadIdx.x; c < l; c += blockDim.x) {
        double w = 0.0;
        for (int64_t b = 0; b < nb; ++b) w += part[b * l + c];
        w *= tj;
        if (j >= r0 && j < r1) X[j * l + c] -= w;
        for (int64_t i = max(r0, j + 1); i < r1; ++i) X[i * l + c] -= X[i * l + j] * w;
      }
    }
    grid.sync();
  }
}

// Q = H_0 ... H_{l-1} [I; 0] by backward accumulation.
__global__ void k_house_formq(const double* __restrict__ X, int64_t rows, int64_t l, const double* __restrict__ tau,
                              double* __restrict__ Q, double* __restrict__ part) {
  cg::grid_group grid = cg::this_grid();
  const int64_t nb = gridDim.x;
  const int64_t per = (rows + nb - 1) / nb;
  const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(rows, r0 + per);
  for (int64_t i = r0; i < r1; ++i)
    for (int64_t c = threadIdx.x; c < l; c += blockDim.x) Q[i * l + c] = (i == c) ? 1.0 : 0.0;
  grid.sync();
  for (int64_t j = min(l, rows) - 1; j >= 0; --j) {
    const double tj = tau[j];
    if (tj == 0.0) continue;  // uniform across the grid
    for (int64_t c = j + threadIdx.x; c < l; c += blockDim.x) {
      double w = 0.0;
      if (j >= r0 && j < r1) w = Q[j * l + c];
      for (int64_t i = max(r0, j + 1); i < r1; ++i) w = fma(X[i * l + j], Q[i * l + c], w);
      part[(int64_t)blockIdx.x * l + c] = w;
    }
    grid.sync();
    for (int64_t c = j + threadIdx.x; c < l; c += blockDim.x) {
      double w = 0.0;
      for (int64_t b = 0; b < nb; ++b) w += part[b * l + c];
      w *= tj;
      if (j >= r0 && j < r1) Q[j * l + c] -= w;
      for (int64_t i = max(r0, j + 1); i < r1; ++i) Q[i * l + c] -= X[i * l + j] * w;
    }
    grid.sync();
  }
}

int householder_q(const Dla& d, Arena& ar, double* X, int64_t rows, int64_t l, double* Q) {
  int occ1 = 0, occ2 = 0;
  const int threads = 256;
  if (!ar.measure) {
    BSRHT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, k_house_qr, threads, 0));
    BSRHT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_house_formq, threads, 0));
  }
  const int64_t want = std::max<int64_t>(1, (rows + 31) / 32);
  const int64_t cap = (int64_t)num_sms() * std::max(1, std::min(occ1, occ2));
  const int nb = (int)std::max<int64_t>(1, std::min(want, std::min<int64_t>(cap, 1024)));
  double* tau = static_cast<double*>(ar.take(sizeof(double) * l));
  double* part = static_cast<double*>(ar.take(sizeof(double) * 1024 * std::max<int64_t>(l, 1)));
  if (!ar.ok()) return BSRHT_ENOMEM;
  if (ar.measure) return BSRHT_OK;
  void* a1[] = {&X, &rows, &l, &tau, &part};
  int st = launch_cooperative((const void*)k_house_qr, dim3(nb), dim3(threads), a1, 0, d.s);
  if (st != BSRHT_OK) return st;
  void* a2[] = {&X, &rows, &l, &tau, &Q, &part};
  st = launch_cooperative((const void*)k_house_formq, dim3(nb), dim3(threads), a2, 0, d.s);
  if (st != BSRHT_OK) return st;
  note_launches(2);
  return BSRHT_OK;
}

}  // namespace bsrht
