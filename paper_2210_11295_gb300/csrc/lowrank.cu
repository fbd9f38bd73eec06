// Randomized SVD (Algorithm 1, Sec. 3.1) and randomized Nystrom (Algorithm 2,
// Sec. 3.2) on the block SRHT sketch, one GPU, one stream.
//
// Precision: the tall products run in the arithmetic of A (FP64 for FP64
// input, FP32 otherwise); the QR of the l x m sketch, the Cholesky factors,
// the triangular inverses and the small SVD are FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "capi_internal.cuh"
#include "common.cuh"
#include "dla.cuh"
#include "sketch.cuh"
#include "trace.cuh"

namespace bsrht {

namespace {

DT dt_of(int d) {
  switch (d) {
    case BSRHT_F64: return DT::F64;
    case BSRHT_F32: return DT::F32;
    case BSRHT_BF16: return DT::BF16;
    default: return DT::F16;
  }
}

#define TRY(expr)                 \
  do {                            \
    const int st_ = (expr);       \
    if (st_ != BSRHT_OK) return st_; \
  } while (0)

// R = L2^T L1^T and friends: small FP64 products through the GEMM.
int gemm64(const Dla& d, Arena& ar, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
           bool a_trans, const double* B, int64_t ldb, double* C, int64_t ldc, bool tri_b = false,
           bool gram = false) {
  const size_t mk = ar.mark();
  const int st = gemm(d, ar, DT::F64, DT::F64, DT::F64, true, M, N, K, A, lda, a_trans, B, ldb, C, ldc, 1.0, 0.0,
                      tri_b, gram);
  ar.release(mk);
  return st;
}

// Tall product in the compute type tc (F32 or F64): C = op(A) B.
int gemm_c(const Dla& d, Arena& ar, DT ta, DT tc, DT tout, int64_t M, int64_t N, int64_t K, const void* A,
           int64_t lda, bool a_trans, const void* B, int64_t ldb, void* C, int64_t ldc, bool tri_b, bool gram) {
  const size_t mk = ar.mark();
  const int st = gemm(d, ar, ta, tc, tout, tc == DT::F64, M, N, K, A, lda, a_trans, B, ldb, C, ldc, 1.0, 0.0,
                      tri_b, gram);
  ar.release(mk);
  return st;
}

// Tall product on tensor cores (FP32 data, FP32 accuracy) when the layout
// allows it: C (M x N, tout) = A (M x K, FP32) * B (K x N, B64 in FP64 or B32
// in FP32).  Falls back to the CUDA-core GEMM with B32.
bool use_tc(DT tc, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda) {
  return tc == DT::F32 && M >= 256 && gemm_tc_eligible(M, N, K, A, lda);
}

// With Ct (FP32 output only) the tensor-core path also writes C^T (N x M)
// there and sets *ct_done; the CUDA-core path leaves *ct_done false.
int tall_gemm(const Dla& d, Arena& ar, DT ta, DT tc, DT tout, int64_t M, int64_t N, int64_t K, const void* A,
              int64_t lda, const double* B64, const void* B32, int64_t ldb, void* C, int64_t ldc, bool tri_b,
              float* Ct = nullptr, bool* ct_done = nullptr) {
  if (ct_done) *ct_done = false;
  if (ar.measure) {
    // Which form runs depends on pointers and on column counts that a
    // rank-revealing basis can lower at run time: size every form the call
    // could take (tensor cores with N columns and with N rounded down to a
    // multiple of 4, and the CUDA-core GEMM); the arena keeps the largest.
    const size_t mk = ar.mark();
    if (ta == DT::F32 && tc == DT::F32 && M >= 256) {
      for (int64_t nn : {N, N - N % 4}) {
        if (nn < 1) continue;
        const int st = gemm_tc(d, ar, M, nn, K, nullptr, lda, DT::F64, nullptr, ldb, false, tout, nullptr, ldc,
                               false, tri_b, tout == DT::F32 ? Ct : nullptr);
        ar.release(mk);
        if (st != BSRHT_OK && st != BSRHT_EUNSUP) return st;
      }
    }
    const int st = gemm_c(d, ar, ta, tc, tout, M, N, K, A, lda, false, tc == DT::F64 ? (const void*)B64 : B32, ldb,
                          C, ldc, tri_b, false);
    ar.release(mk);
    return st;
  }
  if (ta == DT::F32 && use_tc(tc, M, N, K, A, lda) && B64 != nullptr) {
    if (tout != DT::F32) Ct = nullptr;
    const size_t mk = ar.mark();
    const int st = gemm_tc(d, ar, M, N, K, static_cast<const float*>(A), lda, DT::F64, B64, ldb, false, tout, C, ldc,
                           false, tri_b, Ct);
    ar.release(mk);
    if (st == BSRHT_OK && ct_done) *ct_done = Ct != nullptr;
    return st;
  }
  return gemm_c(d, ar, ta, tc, tout, M, N, K, A, lda, false, tc == DT::F64 ? (const void*)B64 : B32, ldb, C, ldc,
                tri_b, false);
}

// G (l x l, FP64) = X^T X for the tall X (rows x l, type tc); the tensor-core
// path writes X^T into `scratch` (rows x l elements) first, unless have_t
// says the product that formed X already left X^T (FP32) there.
int tall_gram(const Dla& d, Arena& ar, bool dry, DT tc, const void* X, int64_t rows, int64_t l, void* scratch,
              double* G, bool have_t = false) {
  if (ar.measure) {
    // As in tall_gemm: size the tensor-core form at l and at l rounded down
    // to a multiple of 4 (a lower run-time rank may select it) and the
    // CUDA-core form.
    const size_t mk = ar.mark();
    if (tc == DT::F32 && l >= 256 && (rows % 4) == 0) {
      for (int64_t ll : {l, l - l % 4}) {
        if (ll < 4 || (ll % 4) != 0) continue;
        const int st = gemm_tc(d, ar, ll, ll, rows, nullptr, rows, DT::F32, nullptr, rows, true, DT::F64, G, ll,
                               true);
        ar.release(mk);
        if (st != BSRHT_OK && st != BSRHT_EUNSUP) return st;
      }
    }
    const int st = gemm_c(d, ar, tc, tc, DT::F64, l, l, rows, X, l, true, X, l, G, l, false, true);
    ar.release(mk);
    return st;
  }
  if (use_tc(tc, l, l, rows, scratch, rows) && (rows % 4) == 0 && (l % 4) == 0) {
    if (!dry && !have_t) {
      const int st = transpose_to_f32(d, DT::F32, X, rows, l, l, static_cast<float*>(scratch), rows);
      if (st != BSRHT_OK) return st;
    }
    const size_t mk = ar.mark();
    const int st = gemm_tc(d, ar, l, l, rows, static_cast<const float*>(scratch), rows, DT::F32, scratch, rows, true,
                           DT::F64, G, l, true);
    ar.release(mk);
    return st;
  }
  return gemm_c(d, ar, tc, tc, DT::F64, l, l, rows, X, l, true, X, l, G, l, false, true);
}

int read_status(const Dla& d, int* host) {
  BSRHT_CUDA_TRY(cudaMemcpyAsync(host, d.status, sizeof(int), cudaMemcpyDeviceToHost, d.s));
  BSRHT_CUDA_TRY(cudaStreamSynchronize(d.s));
  return BSRHT_OK;
}

int status_to_code(int s) {
  if (s & kStatusTcWait) return BSRHT_ETIMEDOUT;
  if (s & kStatusNotPD) return BSRHT_ENOTPD;
  if (s & kStatusNoConv) return BSRHT_ENOCONV;
  return BSRHT_OK;
}

// Seeded fill of the columns c with scale[c] == 0 (directions dropped as
// numerically null) by uniform values in [-1, 1): they complete the basis the
// way Householder QR does for a rank-deficient input.
template <typename T>
__global__ void k_fill_null_cols(T* __restrict__ X, int64_t rows, int64_t l, const double* __restrict__ scale,
                                 uint64_t seed) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * l) return;
  const int64_t i = idx / l, c = idx - i * l;
  if (scale[c] != 0.0) return;
  U64x4 ctr{(uint64_t)i, (uint64_t)c, 3, 0};
  const uint64_t w = philox4x64_10(ctr, seed, 0x5eed).x;
  X[idx] = (T)((double)(int64_t)w * 0x1.0p-63);
}

// Keep column c (scale 1/sqrt(lambda_c)) when lambda_c > tau * lambda_0.
__global__ void k_svqb_scale(const double* __restrict__ lam, double* __restrict__ scale, int64_t l, double tau) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= l) return;
  const double l0 = lam[0], v = lam[c];
  scale[c] = (l0 > 0.0 && v > tau * l0) ? 1.0 / sqrt(v) : 0.0;
}

// min / max of the squared diagonal of the Cholesky factor L (l x l).
__global__ void k_pivot_ratio(const double* __restrict__ L, int64_t l, double* __restrict__ out) {
  __shared__ double mn[256], mx[256];
  double a = INFINITY, b = 0.0;
  for (int64_t i = threadIdx.x; i < l; i += blockDim.x) {
    const double v = L[i * l + i] * L[i * l + i];
    a = fmin(a, v);
    b = fmax(b, v);
  }
  mn[threadIdx.x] = a;
  mx[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      mn[threadIdx.x] = fmin(mn[threadIdx.x], mn[threadIdx.x + o]);
      mx[threadIdx.x] = fmax(mx[threadIdx.x], mx[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = mx[0] > 0.0 ? mn[0] / mx[0] : 0.0;
}

struct OrthBufs {
  double* G;      // l x l
  double* LT1;    // l x l
  double* LT2;    // l x l
  double* Rinv;   // l x l
  void* Rinv_c;   // l x l in tc
  double* Ug;     // l x l (fallback)
  double* Vg;     // l x l (fallback)
  double* lam;    // l (fallback)
  double* sc;     // l (fallback)
  double* ratio;  // 1: min / max squared Cholesky pivot (pivot check)
};

OrthBufs take_orth_bufs(Arena& ar, int64_t l, size_t cs) {
  OrthBufs b;
  b.G = static_cast<double*>(ar.take(8 * l * l));
  b.LT1 = static_cast<double*>(ar.take(8 * l * l));
  b.LT2 = static_cast<double*>(ar.take(8 * l * l));
  b.Rinv = static_cast<double*>(ar.take(8 * l * l));
  b.Rinv_c = ar.take(cs * l * l);
  b.Ug = static_cast<double*>(ar.take(8 * l * l));
  b.Vg = static_cast<double*>(ar.take(8 * l * l));
  b.lam = static_cast<double*>(ar.take(8 * l));
  b.sc = static_cast<double*>(ar.take(8 * l));
  b.ratio = static_cast<double*>(ar.take(8));
  return b;
}

// Smallest accepted ratio of squared Cholesky pivots (min / max) on the
// CholeskyQR2 path of FP64 data.  CholeskyQR2 is accurate while the
// condition number of X stays below about u^-1/2 (u = 2^-53); a Gram whose
// pivots spread by more than 2^44 is past that, or numerically singular
// (its smallest eigenvalues are then rounding noise, and a Cholesky factor
// that happens to exist is meaningless).  Such inputs take the Householder /
// rank-revealing paths instead.
constexpr double kCholQrPivotMin64 = 0x1.0p-44;
// The same for products and Grams at FP32 accuracy (u = 2^-24): condition
// numbers up to about 10^3.
constexpr double kCholQrPivotMin32 = 0x1.0p-20;

// Orthonormal basis Q (rows x l, type tc) of the tall X, robust to rank
// deficiency, and R (l x l FP64) with X = Q R when R != nullptr.
// Fast path: CholeskyQR2 (R upper triangular).  If a Cholesky factorization
// fails (X numerically rank deficient), fallback: eigen-decomposition of
// X^T X by the Jacobi SVD, directions with lambda <= tau lambda_0 replaced by
// seeded random ones, CholeskyQR2 of that full-rank basis, R = Q^T X.
// Buffers: X (input), Y and Z (rows x l scratch). On return *Qout points to
// the buffer holding Q; X is left intact when keep_x (then Q is not formed
// on the fast path unless need_q).
// With Rinv_out != nullptr the fast path may return Q in factored form,
// Q = Q1 R2^{-1}: then *Qout holds the first-pass basis Q1 and *Rinv_out the
// upper-triangular FP64 R2^{-1} (l x l), and the caller applies R2^{-1} to its
// small right-hand factor instead of forming Q (one rows x l x l product
// less).  *Rinv_out is nullptr when Q is explicit.
// With declined != nullptr only the fast path runs: when it cannot be used
// (a Cholesky factorization fails, or for FP64 data the pivot check above),
// *declined is set and nothing else is done.
int orth_robust(const Dla& d, Arena& ar, bool dry, DT tc, void* X, void* Y, void* Z, int64_t rows, int64_t l,
                uint64_t seed, const OrthBufs& b, double* R, bool need_q, bool keep_x, void** Qout,
                const double** Rinv_out = nullptr, bool x_t_in_z = false, bool* declined = nullptr) {
  const void* RinvB = (tc == DT::F32) ? b.Rinv_c : (const void*)b.Rinv;
  if (Rinv_out) *Rinv_out = nullptr;
  if (declined) *declined = false;
  // ---- fast path: CholeskyQR2 (Z serves as scratch for the transposed Grams)
  bool fast = true;
  // (b.Ug and b.Vg, used only by the fallback, are the scratch of chol_inv.)
  TRY(tall_gram(d, ar, dry, tc, X, rows, l, Z, b.G, x_t_in_z));
  if (!dry) {
    TRY(chol_inv(d, b.G, b.LT1, b.Rinv, b.Ug, b.Vg, l));
    // FP64 data: the squared pivots of the first factor must stay above
    // kCholQrPivotMin64 of the largest (see there); FP32 data, when the
    // caller has a fallback (declined), above kCholQrPivotMin32.
    double ratio = 1.0;
    const double pivot_min = tc == DT::F64 ? kCholQrPivotMin64 : kCholQrPivotMin32;
    if (tc == DT::F64 || declined) {
      k_pivot_ratio<<<1, 256, 0, d.s>>>(b.G, l, b.ratio);
      BSRHT_CUDA_TRY(cudaGetLastError());
      note_launches(1);
      BSRHT_CUDA_TRY(cudaMemcpyAsync(&ratio, b.ratio, sizeof(double), cudaMemcpyDeviceToHost, d.s));
    }
    int hs = 0;
    TRY(read_status(d, &hs));
    if (hs & kStatusTcWait) return BSRHT_ETIMEDOUT;
    if (hs || !(ratio > pivot_min)) {
      fast = false;
      BSRHT_CUDA_TRY(cudaMemsetAsync(d.status, 0, sizeof(int), d.s));
      if (declined) {
        *declined = true;
        return BSRHT_OK;
      }
    }
  }
  if (fast || dry) {
    if (!dry && tc == DT::F32) TRY(cast_copy(d, DT::F64, b.Rinv, DT::F32, b.Rinv_c, l * l));
    // Y = X R1^-1, leaving Y^T in Z (the first Gram is done with it) for the
    // second Gram.
    bool y_t = false;
    TRY(tall_gemm(d, ar, tc, tc, tc, rows, l, l, X, l, b.Rinv, RinvB, l, Y, l, true,
                  tc == DT::F32 ? static_cast<float*>(Z) : nullptr, &y_t));
    TRY(tall_gram(d, ar, dry, tc, Y, rows, l, Z, b.G, y_t));
    if (!dry) {
      TRY(chol_inv(d, b.G, b.LT2, b.Rinv, b.Ug, b.Vg, l));
      int hs = 0;
      TRY(read_status(d, &hs));
      if (hs & kStatusTcWait) return BSRHT_ETIMEDOUT;
      if (hs) {
        fast = false;
        BSRHT_CUDA_TRY(cudaMemsetAsync(d.status, 0, sizeof(int), d.s));
        if (declined) {
          *declined = true;
          return BSRHT_OK;
        }
      }
    }
    if (fast || dry) {
      if (!dry && tc == DT::F32) TRY(cast_copy(d, DT::F64, b.Rinv, DT::F32, b.Rinv_c, l * l));
      void* dst = keep_x ? Z : X;
      if (Rinv_out) {
        *Rinv_out = b.Rinv;
        dst = Y;
      } else if (need_q || !keep_x) {
        TRY(tall_gemm(d, ar, tc, tc, tc, rows, l, l, Y, l, b.Rinv, RinvB, l, dst, l, true));
      }
      if (R) TRY(gemm64(d, ar, l, l, l, b.LT2, l, false, b.LT1, l, R, l, true, false));
      *Qout = dst;
      if (!dry) return BSRHT_OK;
    }
  }
  // ---- fallback for moderate FP64 inputs: Householder QR of a copy of X.
  if (tc == DT::F64 && rows <= (int64_t(1) << 17)) {
    if (!dry) BSRHT_CUDA_TRY(cudaMemcpyAsync(Z, X, sizeof(double) * rows * l, cudaMemcpyDeviceToDevice, d.s));
    {
      const size_t mk = ar.mark();
      TRY(householder_q(d, ar, static_cast<double*>(Z), rows, l, static_cast<double*>(Y)));
      ar.release(mk);
    }
    if (R) TRY(gemm_c(d, ar, tc, tc, DT::F64, l, l, rows, Y, l, true, X, l, R, l, false, false));
    *Qout = Y;
    if (!dry) return BSRHT_OK;
  }
  // ---- fallback: eigen-based basis with random completion.  The Gram is
  // accumulated in FP64 (also for FP32 data) so that small directions are
  // resolved to FP64 accuracy before they are dropped or kept.
  {
    const size_t mk = ar.mark();
    TRY(gemm(d, ar, tc, tc, DT::F64, true, l, l, rows, X, l, true, X, l, b.G, l, 1.0, 0.0, false, true));
    ar.release(mk);
  }
  {
    const size_t mk = ar.mark();
    TRY(jacobi_svd(d, ar, b.G, l, b.Ug, b.lam, b.Vg));
    ar.release(mk);
  }
  const double tau = (double)l * 10.0 * 0x1.0p-52;
  if (!dry) {
    k_svqb_scale<<<(unsigned)((l + 127) / 128), 128, 0, d.s>>>(b.lam, b.sc, l, tau);
    BSRHT_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    TRY(scale_columns(d, b.Vg, l, l, l, b.sc, false));
    if (tc == DT::F32) TRY(cast_copy(d, DT::F64, b.Vg, DT::F32, b.Rinv_c, l * l));
  }
  const void* Bv = (tc == DT::F32) ? b.Rinv_c : (const void*)b.Vg;
  TRY(gemm_c(d, ar, tc, tc, tc, rows, l, l, X, l, false, Bv, l, Y, l, false, false));
  if (!dry) {
    const unsigned nb = (unsigned)((rows * l + 255) / 256);
    if (tc == DT::F64)
      k_fill_null_cols<double><<<nb, 256, 0, d.s>>>(static_cast<double*>(Y), rows, l, b.sc, seed);
    else
      k_fill_null_cols<float><<<nb, 256, 0, d.s>>>(static_cast<float*>(Y), rows, l, b.sc, seed);
    BSRHT_CUDA_TRY(cudaGetLastError());
    note_launches(1);
  }
  // CholeskyQR2 of the completed basis: Y -> Z -> Y.
  for (int pass = 0; pass < 2; ++pass) {
    void* src = pass == 0 ? Y : Z;
    void* dst = pass == 0 ? Z : Y;
    TRY(gemm_c(d, ar, tc, tc, DT::F64, l, l, rows, src, l, true, src, l, b.G, l, false, true));
    if (!dry) {
      TRY(chol_inv(d, b.G, b.LT1, b.Rinv, b.Ug, b.Vg, l));
      int hs = 0;
      TRY(read_status(d, &hs));
      if (hs) return status_to_code(hs) != BSRHT_OK ? status_to_code(hs) : BSRHT_ENOTPD;
      if (tc == DT::F32) TRY(cast_copy(d, DT::F64, b.Rinv, DT::F32, b.Rinv_c, l * l));
    }
    TRY(gemm_c(d, ar, tc, tc, tc, rows, l, l, src, l, false, RinvB, l, dst, l, true, false));
  }
  if (R) TRY(gemm_c(d, ar, tc, tc, DT::F64, l, l, rows, Y, l, true, X, l, R, l, false, false));
  *Qout = Y;
  return BSRHT_OK;
}

// cols[c * l + i] = R[i][c] for the upper triangle R of the first l rows of
// the Householder output Z (rows x l): the column storage of R for the
// Jacobi SVD.
__global__ void k_upper_to_cols(const double* __restrict__ Z, int64_t l, double* __restrict__ cols) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= l * l) return;
  const int64_t c = idx / l, i = idx - c * l;
  cols[idx] = i <= c ? Z[i * l + c] : 0.0;
}

// Rank rule of the basis of range(Y): directions with sigma <= tau sigma_1
// are numerically absent, tau = l 2^-44: l times the relative precision of
// the FP64 sketch (its transform is exact on fixed-point values with at
// least 45 fraction bits below each column's largest magnitude), so that
// directions that vanish in exact arithmetic are dropped.
double range_tol(int64_t l) { return (double)l * 0x1.0p-44; }

// Orthonormal basis Q of the numerical range of the FP64 sketch matrix X
// (rows x l), Algorithm 1 step 2: range(Q) = range(Y).  Sampling with
// replacement (Sec. 2) lets Omega repeat a row up to sign in every block;
// range(Y) then has dimension r' < l, and Q must not be completed with
// arbitrary directions (the result would depend on them).  Rule: keep the
// left singular directions of X with sigma > range_tol(l) sigma_1.
// Fast path: CholeskyQR2 with the pivot check of kCholQrPivotMin64, which
// accepts only inputs whose smallest singular value is far above the rule's
// cutoff (every direction kept, r' = l).  Otherwise: Householder QR
// X = Qh R, one-sided Jacobi SVD R = Ur S Vr^T (FP64), and
// Q = Qh Ur[:, :r'] with r' the count of sigma > tau sigma_1.
// Buffers: X (input, overwritten), Y and Z (rows x l scratch).  On return
// *Qout (rows x r', leading dimension r') and *rank = r'; reads r' back on
// the stream.  In dry mode both paths are measured and r' = l.
int range_basis(const Dla& d, Arena& ar, bool dry, double* X, double* Y, double* Z, int64_t rows, int64_t l,
                uint64_t seed, const OrthBufs& b, double** Qout, int64_t* rank) {
  *rank = l;
  void* Qv = nullptr;
  bool declined = false;
  TRY(orth_robust(d, ar, dry, DT::F64, X, Y, Z, rows, l, seed, b, nullptr, true, false, &Qv, nullptr, false,
                  &declined));
  if (!dry && !declined) {
    *Qout = static_cast<double*>(Qv);
    return BSRHT_OK;
  }
  // Householder QR of a copy of X: Z holds R (upper triangle of its first
  // l rows) and the reflectors, Y = Qh.
  if (!dry) BSRHT_CUDA_TRY(cudaMemcpyAsync(Z, X, sizeof(double) * rows * l, cudaMemcpyDeviceToDevice, d.s));
  {
    const size_t mk = ar.mark();
    TRY(householder_q(d, ar, Z, rows, l, Y));
    ar.release(mk);
  }
  if (!dry) {
    k_upper_to_cols<<<(unsigned)((l * l + 255) / 256), 256, 0, d.s>>>(Z, l, b.G);
    BSRHT_CUDA_TRY(cudaGetLastError());
    note_launches(1);
  }
  {
    const size_t mk = ar.mark();
    // R V = U S: b.Ug = Ur (l x l), b.lam = S.  Columns whose norm is below
    // the rank rule's tau (against ||R||_F) are numerically zero for the
    // Jacobi too: they hold the rounding of the sketch (about 2^-45 of its
    // scale for FP64 data) and would otherwise keep the sweeps going.
    TRY(jacobi_svd(d, ar, b.G, l, b.Ug, b.lam, b.Vg, 0.0, range_tol(l)));
    ar.release(mk);
  }
  int64_t r = l;
  if (!dry) {
    std::vector<double> sig((size_t)l);
    BSRHT_CUDA_TRY(cudaMemcpyAsync(sig.data(), b.lam, sizeof(double) * l, cudaMemcpyDeviceToHost, d.s));
    int hs = 0;
    TRY(read_status(d, &hs));
    if (hs) return status_to_code(hs) != BSRHT_OK ? status_to_code(hs) : BSRHT_ENOCONV;
    r = 0;
    const double cut = range_tol(l) * sig[0];
    for (int64_t c = 0; c < l; ++c)
      if (sig[0] > 0.0 && sig[c] > cut) ++r;
  }
  // Q = Qh Ur[:, :r'] into X (rows x r').
  if (r > 0) TRY(gemm64(d, ar, rows, r, l, Y, l, false, b.Ug, l, X, r));
  *Qout = X;
  *rank = r;
  return BSRHT_OK;
}

// Cosine threshold of the FP64 Jacobi polish for FP32 data: 16 sqrt(l) 2^-40
// (sweeps stop once none exceeds 16 times that), about 3.3e-10 at l = 512:
// far below the FP32 accuracy of the tall factors it is combined with, and
// reached in one rotating sweep from the FP32 Jacobi's 16 sqrt(l) 2^-24.
double polish_tol_fp32(int64_t l) { return 16.0 * std::sqrt((double)l) * 0x1.0p-40; }

// ---------------------------------------------------------------- RSVD
int rsvd_impl(const bsrht_opts& o, const void* A, int64_t n, int64_t m, int k, int64_t l, int p, uint64_t seed,
              double* U, double* S, double* V, Arena& ar, bool dry) {
  const DT ta = dt_of(o.dtype);
  const DT tc = (ta == DT::F64) ? DT::F64 : DT::F32;
  const size_t cs = dt_size(tc);
  const int64_t lda = o.lda ? o.lda : m;
  SketchPlan sp;
  TRY(sketch_make_plan(sp, o.dtype, o.variant, n, m, lda, p, l, !dry, dry ? nullptr : A));
  Dla d{static_cast<cudaStream_t>(o.stream), nullptr};
  d.status = static_cast<int*>(ar.take(sizeof(int)));
  void* sk_ws = ar.take(sp.work_bytes);
  void* B = ar.take(cs * l * m);
  double* X1 = static_cast<double*>(ar.take(8 * m * l));
  double* X2 = static_cast<double*>(ar.take(8 * m * l));
  double* X3 = static_cast<double*>(ar.take(8 * m * l));
  void* Qc = ar.take(cs * m * l);
  void* W1 = ar.take(cs * n * l);
  void* W2 = ar.take(cs * n * l);
  void* W3 = ar.take(cs * n * l);
  double* R = static_cast<double*>(ar.take(8 * l * l));
  double* Us = static_cast<double*>(ar.take(8 * l * l));
  double* Vs = static_cast<double*>(ar.take(8 * l * l));
  double* sig = static_cast<double*>(ar.take(8 * l));
  double* Vp = static_cast<double*>(ar.take(8 * l * k));
  double* RT = static_cast<double*>(ar.take(8 * l * l));
  void* Vs_c = ar.take(cs * l * l);
  const OrthBufs ob = take_orth_bufs(ar, l, cs);
  if (!ar.ok()) return BSRHT_ENOMEM;
  if (!dry) BSRHT_CUDA_TRY(cudaMemsetAsync(d.status, 0, sizeof(int), d.s));

  // Step 1: B = Omega A (l x m); the paper's Y is B^T.
  if (!dry) trace_begin(d.s);
  if (!dry) TRY(sketch_run(sp, A, seed, B, m, sk_ws, d.s));
  if (!dry) trace_mark(d.s, "sketch");
  // Step 2: Q = orth(B^T) (m x lq, lq = dim range(Y) <= l).  FP32 data:
  // the second pass reads Q in FP32, so a well-conditioned sketch takes
  // CholeskyQR2 at FP32 accuracy on the tensor cores (pivot check
  // kCholQrPivotMin32) and only V = Q U~_k is made orthonormal in FP64 at
  // the end (an m x k CholeskyQR2).  Otherwise, and for FP64 data: the
  // rank-revealing FP64 basis (range_basis).
  double* Q = nullptr;
  int64_t lq = l;
  const void* Qa = nullptr;
  bool q32 = false;
  if (tc == DT::F32) {
    float* Y32 = reinterpret_cast<float*>(X2);
    if (!dry) TRY(transpose_cast(d, DT::F32, B, l, m, m, DT::F32, Y32, l));
    void* Qv = nullptr;
    bool declined = false;
    TRY(orth_robust(d, ar, dry, DT::F32, Y32, X3, Qc, m, l, seed ^ 0x51ull, ob, nullptr, true, false, &Qv, nullptr,
                    false, &declined));
    if (!dry && !declined) {
      TRY(cast_copy(d, DT::F32, Qv, DT::F64, X1, m * l));
      Q = X1;
      Qa = Qv;
      q32 = true;
    }
  }
  if (!q32) {
    if (!dry) TRY(transpose_cast(d, tc, B, l, m, m, DT::F64, X1, l));
    TRY(range_basis(d, ar, dry, X1, X2, X3, m, l, seed ^ 0x51ull, ob, &Q, &lq));
  }
  if (!dry) trace_mark(d.s, "orth_sketch");
  // Below the numerical rank of Y the factors are zero (lq < k).
  const int64_t kk = std::min<int64_t>(k, lq);
  if (!dry && kk < k) {
    BSRHT_CUDA_TRY(cudaMemsetAsync(U, 0, sizeof(double) * n * k, d.s));
    BSRHT_CUDA_TRY(cudaMemsetAsync(S, 0, sizeof(double) * k, d.s));
    BSRHT_CUDA_TRY(cudaMemsetAsync(V, 0, sizeof(double) * m * k, d.s));
  }
  if (!dry && lq == 0) {  // Y = 0: A Omega^T vanishes, the approximation is 0
    int hs = 0;
    TRY(read_status(d, &hs));
    return status_to_code(hs);
  }
  if (!q32) {
    Qa = Q;
    if (tc == DT::F32) {
      if (!dry) TRY(cast_copy(d, DT::F64, Q, DT::F32, Qc, m * lq));
      Qa = Qc;
    }
  }
  // Step 3: the paper's Z = Q^T A_paper, i.e. Z^T = A Q (n x lq): second pass over A.
  bool w_t = false;  // W1^T left in W3, the Gram scratch of the QR below
  TRY(tall_gemm(d, ar, ta, tc, tc, n, lq, m, A, lda, Q, Qa, lq, W1, lq, false,
                tc == DT::F32 ? static_cast<float*>(W3) : nullptr, &w_t));
  if (!dry) trace_mark(d.s, "second_pass");
  // Step 4: Z^T = P R (CholeskyQR2, rank-robust).  On the CholeskyQR2 path P
  // stays factored, P = P1 R2^{-1} (Rinv2 != nullptr).
  void* Pv = nullptr;
  const double* Rinv2 = nullptr;
  TRY(orth_robust(d, ar, dry, tc, W1, W2, W3, n, lq, seed ^ 0x52ull, ob, R, true, false, &Pv, &Rinv2, w_t));
  if (!dry) trace_mark(d.s, "tall_qr");
  // Step 5: SVD of R^T = U~ Sigma~ V~^T.  FP64 data: Jacobi on the columns
  // of R^T (the rows of R) to FP64 tolerance.  FP32 data: Jacobi on the
  // columns of R (R = V~ Sigma~ U~^T), so that the accumulated rotations,
  // orthogonal to FP64 rounding, give U~ (multiplied by the FP64 Q below),
  // and the polish stops at cosines of polish_tol_fp32(lq): the other factor
  // V~ meets P, itself orthogonal only to FP32 accuracy.
  {
    const size_t mk = ar.mark();
    if (tc == DT::F32) {
      if (!dry) TRY(transpose_lower_to_upper(d, R, RT, lq));
      TRY(jacobi_svd(d, ar, RT, lq, Vs, sig, Us, polish_tol_fp32(lq), 0.0, k));
    } else {
      TRY(jacobi_svd(d, ar, R, lq, Us, sig, Vs));
    }
    ar.release(mk);
  }
  if (!dry) trace_mark(d.s, "small_svd");
  // Step 6: U = P V~_k, V = Q U~_k, S = Sigma~_k.  With P factored, U =
  // P1 (R2^{-1} V~_k): the lq x k factor is formed in FP64 first.
  const double* Vk64 = Vs;
  int64_t ldv = lq;
  if (Rinv2) {
    TRY(gemm64(d, ar, lq, kk, lq, Rinv2, lq, false, Vs, lq, Vp, kk));
    Vk64 = Vp;
    ldv = kk;
  }
  const void* Vk = Vk64;
  if (tc == DT::F32) {
    if (!dry) TRY(cast_copy(d, DT::F64, Vk64, DT::F32, Vs_c, lq * ldv));
    Vk = Vs_c;
  }
  TRY(tall_gemm(d, ar, tc, tc, DT::F64, n, kk, lq, Pv, lq, Vk64, Vk, ldv, U, k, false));
  if (q32 || (dry && tc == DT::F32)) {
    // FP32-accuracy Q: V = Q U~_k on the tensor cores (FP32 accuracy, that
    // of Q itself; U~_k also in FP32 for the CUDA-core form).
    if (!dry) TRY(cast_copy(d, DT::F64, Us, DT::F32, Vs_c, lq * lq));
    TRY(tall_gemm(d, ar, DT::F32, DT::F32, DT::F64, m, kk, lq, Qa, lq, Us, Vs_c, lq, V, k, false));
  }
  if (!q32) TRY(gemm64(d, ar, m, kk, lq, Q, lq, false, Us, lq, V, k));
  if (!dry) BSRHT_CUDA_TRY(cudaMemcpyAsync(S, sig, sizeof(double) * kk, cudaMemcpyDeviceToDevice, d.s));
  // With the FP32-accuracy Q, V is orthonormal to FP32 accuracy: one FP64
  // CholeskyQR pass (V^T V = I + O(1e-6), so one pass reaches FP64 rounding)
  // makes it orthonormal while moving it by about 1e-6, the accuracy of
  // FP32 data; CholeskyQR2 with its fallbacks if that Cholesky fails.
  if ((q32 || dry) && kk == k && tc == DT::F32) {
    bool done = false;
    TRY(tall_gram(d, ar, dry, DT::F64, V, m, k, X3, ob.G));
    if (!dry) {
      TRY(chol_inv(d, ob.G, ob.LT1, ob.Rinv, ob.Ug, ob.Vg, k));
      int hs = 0;
      TRY(read_status(d, &hs));
      if (hs & kStatusTcWait) return BSRHT_ETIMEDOUT;
      if (hs)
        BSRHT_CUDA_TRY(cudaMemsetAsync(d.status, 0, sizeof(int), d.s));
      else
        done = true;
    }
    if (done || dry) {
      TRY(gemm64(d, ar, m, k, k, V, k, false, ob.Rinv, k, X2, k, true, false));
      if (!dry) BSRHT_CUDA_TRY(cudaMemcpyAsync(V, X2, sizeof(double) * m * k, cudaMemcpyDeviceToDevice, d.s));
    }
    if (!done) {
      void* Vv = nullptr;
      TRY(orth_robust(d, ar, dry, DT::F64, V, X2, X3, m, k, seed ^ 0x54ull, ob, nullptr, true, false, &Vv));
      if (!dry && Vv != static_cast<void*>(V))
        BSRHT_CUDA_TRY(cudaMemcpyAsync(V, Vv, sizeof(double) * m * k, cudaMemcpyDeviceToDevice, d.s));
    }
  }
  {
    const size_t mk = ar.mark();
    TRY(sign_normalize(d, ar, U, n, k, V, m));
    ar.release(mk);
  }
  if (!dry) trace_mark(d.s, "factors");
  if (dry) return BSRHT_OK;
  int hs = 0;
  TRY(read_status(d, &hs));
  return status_to_code(hs);
}

// ------------------------------------------------------ single-view RSVD
// Algorithm 3 (Sec. 3.3) for the tall n x m A (the paper's m x n matrix is
// A^T = A_p).  Sketching maps, keys seed + 0..3: Omega (l x n, p blocks),
// Phi (s x m, one block) and Psi (s x n, p blocks) are block SRHTs (eq. 2.3);
// Gamma (l x m), the short side's range sketch, is the Gaussian map of the
// comparator (N(0, 1/l), Philox / Box-Muller, in FP64): an SRHT row sample
// of l out of r ~ m draws repeated rows (with replacement, about l^2 / 2r of
// them), which would make X exactly rank deficient.  Step 1 forms the three
// sketches, each a linear function of A alone: Y = A_p Omega^T =
// (Omega A)^T, X = A_p^T Gamma^T = A Gamma^T (a tall product) and
// Z = Phi A_p Psi^T = (Psi (A Phi^T))^T, A Phi^T through the sketch kernels
// on an on-device transpose of A.
// Step 2: Q = orth(Y) (FP64, m x l), P = orth(X) (n x l).  Steps 3-4:
// C = (Phi Q)^+ Z ((Psi P)^T)^+, by the normal equations
// C = G1^-1 (Phi Q)^T Z (Psi P) G2^-1, G1 = (Phi Q)^T (Phi Q),
// G2 = (Psi P)^T (Psi P): Phi and Psi embed range(Q) and range(P), so G1 and
// G2 have condition numbers near 1 (Sec. 2, OSE property) and their fused
// Cholesky inverses are accurate.  Steps 5-6: C = U~ S~ V~^T (Jacobi), and
// A ~ (P V~_k) S~_k (Q U~_k)^T, i.e. U = P V~_k, V = Q U~_k.
int srsvd_impl(const bsrht_opts& o, const void* A, int64_t n, int64_t m, int k, int64_t l, int64_t s, int p,
               uint64_t seed, double* U, double* S, double* V, Arena& ar, bool dry) {
  const DT ta = dt_of(o.dtype);  // F32 or F64 (validated)
  const DT tc = ta;
  const size_t cs = dt_size(tc);
  const int64_t lda = o.lda ? o.lda : m;
  const uint64_t s_om = seed, s_ga = seed + 1, s_ph = seed + 2, s_ps = seed + 3;
  Dla d{static_cast<cudaStream_t>(o.stream), nullptr};
  d.status = static_cast<int*>(ar.take(sizeof(int)));
  void* At = ar.take(cs * m * n);
  void* Yb = ar.take(cs * l * m);
  const int64_t ldg = m + (m & 1);
  double* Gm = static_cast<double*>(ar.take(8 * l * ldg));   // Gamma (l x m, FP64)
  double* GT = static_cast<double*>(ar.take(8 * m * l));     // Gamma^T (m x l, FP64)
  void* GTc = ar.take(cs * m * l);                            // Gamma^T in the type of A
  void* Ws = ar.take(cs * s * n);
  void* Wn = ar.take(cs * n * s);
  void* Zs = ar.take(cs * s * s);
  double* Zp = static_cast<double*>(ar.take(8 * s * s));
  double* Y1 = static_cast<double*>(ar.take(8 * m * l));
  double* Y2 = static_cast<double*>(ar.take(8 * m * l));
  double* Y3 = static_cast<double*>(ar.take(8 * m * l));
  void* X1 = ar.take(cs * n * l);
  void* X2 = ar.take(cs * n * l);
  void* X3 = ar.take(cs * n * l);
  double* PhQ = static_cast<double*>(ar.take(8 * s * l));
  void* PsPc = ar.take(cs * s * l);
  double* PsP = static_cast<double*>(ar.take(8 * s * l));
  double* G1 = static_cast<double*>(ar.take(8 * l * l));
  double* G2 = static_cast<double*>(ar.take(8 * l * l));
  double* LT = static_cast<double*>(ar.take(8 * l * l));
  double* Ri1 = static_cast<double*>(ar.take(8 * l * l));
  double* Ri2 = static_cast<double*>(ar.take(8 * l * l));
  double* RiT = static_cast<double*>(ar.take(8 * l * l));
  double* Gi1 = static_cast<double*>(ar.take(8 * l * l));
  double* Gi2 = static_cast<double*>(ar.take(8 * l * l));
  double* T1 = static_cast<double*>(ar.take(8 * l * s));
  double* Mm = static_cast<double*>(ar.take(8 * l * l));
  double* T2 = static_cast<double*>(ar.take(8 * l * l));
  double* C = static_cast<double*>(ar.take(8 * l * l));
  double* CT = static_cast<double*>(ar.take(8 * l * l));
  double* Uc = static_cast<double*>(ar.take(8 * l * l));
  double* Vc = static_cast<double*>(ar.take(8 * l * l));
  double* sig = static_cast<double*>(ar.take(8 * l));
  void* Vc_c = ar.take(cs * l * l);
  const OrthBufs ob = take_orth_bufs(ar, l, 8);
  // Sketch plans; the scratch is shared (the sketches run one after another).
  SketchPlan sp_y, sp_w, sp_z, sp_q, sp_p;
  TRY(sketch_make_plan(sp_y, o.dtype, BSRHT_VARIANT_AUTO, n, m, lda, p, l, !dry, dry ? nullptr : A));
  TRY(sketch_make_plan(sp_w, o.dtype, BSRHT_VARIANT_AUTO, m, n, n, 1, s, !dry, dry ? nullptr : At));
  TRY(sketch_make_plan(sp_z, o.dtype, BSRHT_VARIANT_AUTO, n, s, s, p, s, !dry, dry ? nullptr : Wn));
  TRY(sketch_make_plan(sp_q, BSRHT_F64, BSRHT_VARIANT_AUTO, m, l, l, 1, s, !dry, nullptr));
  TRY(sketch_make_plan(sp_p, o.dtype, BSRHT_VARIANT_AUTO, n, l, l, p, s, !dry, nullptr));
  const size_t skb = std::max({sp_y.work_bytes, sp_w.work_bytes, sp_z.work_bytes, sp_q.work_bytes,
                               sp_p.work_bytes});
  void* sk_ws = ar.take(skb);
  if (!ar.ok()) return BSRHT_ENOMEM;
  if (!dry) BSRHT_CUDA_TRY(cudaMemsetAsync(d.status, 0, sizeof(int), d.s));

  // Step 1: the three sketches.
  if (!dry) {
    trace_begin(d.s);
    TRY(sketch_run(sp_y, A, s_om, Yb, m, sk_ws, d.s));                      // Omega A (l x m)
    TRY(transpose_cast(d, ta, A, n, m, lda, ta, At, n));                   // A^T (m x n)
    TRY(sketch_run(sp_w, At, s_ph, Ws, n, sk_ws, d.s));                    // Phi A^T (s x n)
    TRY(transpose_cast(d, tc, Ws, s, n, n, tc, Wn, s));                    // A Phi^T (n x s)
    TRY(sketch_run(sp_z, Wn, s_ps, Zs, s, sk_ws, d.s));                    // Psi A Phi^T = Z^T (s x s)
    TRY(transpose_cast(d, tc, Zs, s, s, s, DT::F64, Zp, s));               // Z (s x s, FP64)
    trace_mark(d.s, "sketches");
    TRY(transpose_cast(d, tc, Yb, l, m, m, DT::F64, Y1, l));               // Y (m x l, FP64)
    TRY(gaussian_omega(d.s, DT::F64, Gm, l, m, ldg, s_ga, 1.0 / std::sqrt((double)l)));
    TRY(transpose_cast(d, DT::F64, Gm, l, m, ldg, DT::F64, GT, l));        // Gamma^T (m x l)
    if (tc == DT::F32) TRY(cast_copy(d, DT::F64, GT, DT::F32, GTc, m * l));
  }
  bool x_t = false;  // X^T left in X3, the Gram scratch of orth(X)
  TRY(tall_gemm(d, ar, ta, tc, tc, n, l, m, A, lda, GT, tc == DT::F32 ? GTc : (const void*)GT, l, X1, l,
                false, tc == DT::F32 ? static_cast<float*>(X3) : nullptr, &x_t));  // X = A Gamma^T (n x l)
  // Step 2: Q = orth(Y) in FP64 (m x rq), P = orth(X) (n x rp), rank
  // revealing as in Algorithm 1 (range_basis) for FP64 bases; FP32 data
  // keep the rank-robust CholeskyQR2 basis of X (rp = l).
  double* Q = nullptr;
  int64_t rq = l, rp = l;
  TRY(range_basis(d, ar, dry, Y1, Y2, Y3, m, l, seed ^ 0x61ull, ob, &Q, &rq));
  void* Pv = nullptr;
  if (tc == DT::F64) {
    double* P64 = nullptr;
    TRY(range_basis(d, ar, dry, static_cast<double*>(X1), static_cast<double*>(X2), static_cast<double*>(X3), n, l,
                    seed ^ 0x62ull, ob, &P64, &rp));
    Pv = P64;
  } else {
    TRY(orth_robust(d, ar, dry, tc, X1, X2, X3, n, l, seed ^ 0x62ull, ob, nullptr, true, false, &Pv, nullptr, x_t));
  }
  if (!dry) trace_mark(d.s, "orth");
  const int64_t L = std::max(rq, rp);              // the core is zero-padded to L x L
  const int64_t kk = std::min<int64_t>(k, std::min(rq, rp));
  if (!dry && kk < k) {
    BSRHT_CUDA_TRY(cudaMemsetAsync(U, 0, sizeof(double) * n * k, d.s));
    BSRHT_CUDA_TRY(cudaMemsetAsync(S, 0, sizeof(double) * k, d.s));
    BSRHT_CUDA_TRY(cudaMemsetAsync(V, 0, sizeof(double) * m * k, d.s));
  }
  if (!dry && kk == 0) {
    int hs = 0;
    TRY(read_status(d, &hs));
    return status_to_code(hs);
  }
  // Step 3: Phi Q (s x rq) and Psi P (s x rp).
  if (!dry) {
    SketchPlan pq = sp_q, pp = sp_p;
    if (rq != l) TRY(sketch_make_plan(pq, BSRHT_F64, BSRHT_VARIANT_AUTO, m, rq, rq, 1, s, true, nullptr));
    if (rp != l) TRY(sketch_make_plan(pp, o.dtype, BSRHT_VARIANT_AUTO, n, rp, rp, p, s, true, nullptr));
    if (pq.work_bytes > skb || pp.work_bytes > skb) return BSRHT_ENOMEM;
    TRY(sketch_run(pq, Q, s_ph, PhQ, rq, sk_ws, d.s));
    TRY(sketch_run(pp, Pv, s_ps, PsPc, rp, sk_ws, d.s));
    if (tc == DT::F32)
      TRY(cast_copy(d, DT::F32, PsPc, DT::F64, PsP, s * rp));
    else
      BSRHT_CUDA_TRY(cudaMemcpyAsync(PsP, PsPc, 8 * s * rp, cudaMemcpyDeviceToDevice, d.s));
  }
  // Step 4: C = G1^-1 (Phi Q)^T Z (Psi P) G2^-1 (rq x rp, in an L x L zero frame).
  TRY(gemm64(d, ar, rq, rq, s, PhQ, rq, true, PhQ, rq, G1, rq, false, true));  // G1 = (Phi Q)^T (Phi Q)
  TRY(gemm64(d, ar, rp, rp, s, PsP, rp, true, PsP, rp, G2, rp, false, true));  // G2 = (Psi P)^T (Psi P)
  if (!dry) {
    TRY(chol_inv(d, G1, LT, Ri1, ob.Ug, ob.Vg, rq));                        // Ri1 = L1^-T
    TRY(chol_inv(d, G2, LT, Ri2, ob.Ug, ob.Vg, rp));
    TRY(transpose_lower_to_upper(d, Ri1, RiT, rq));
  }
  TRY(gemm64(d, ar, rq, rq, rq, RiT, rq, true, RiT, rq, Gi1, rq));       // G1^-1 = Ri1 Ri1^T
  if (!dry) TRY(transpose_lower_to_upper(d, Ri2, RiT, rp));
  TRY(gemm64(d, ar, rp, rp, rp, RiT, rp, true, RiT, rp, Gi2, rp));       // G2^-1
  TRY(gemm64(d, ar, rq, s, s, PhQ, rq, true, Zp, s, T1, s));             // (Phi Q)^T Z
  TRY(gemm64(d, ar, rq, rp, s, T1, s, false, PsP, rp, Mm, rp));          // ... (Psi P)
  TRY(gemm64(d, ar, rq, rp, rq, Gi1, rq, false, Mm, rp, T2, rp));
  if (!dry && L != rq) BSRHT_CUDA_TRY(cudaMemsetAsync(C, 0, sizeof(double) * L * L, d.s));
  if (!dry && L != rp) BSRHT_CUDA_TRY(cudaMemsetAsync(C, 0, sizeof(double) * L * L, d.s));
  TRY(gemm64(d, ar, rq, rp, rp, T2, rp, false, Gi2, rp, C, L));
  if (!dry) trace_mark(d.s, "core");
  // Step 5: SVD of C = U~ Sigma~ V~^T; the zero frame leaves the nonzero
  // singular triplets unchanged.  FP64 data: Jacobi on the columns of C (the
  // rows of C^T).  FP32 data: Jacobi on the columns of C^T (C's row-major
  // storage), polished to FP32-data accuracy on the k leading triplets, so
  // that the accumulated rotations, orthogonal to FP64 rounding, give U~,
  // which multiplies the FP64 basis Q below; the other factor meets P.
  {
    const size_t mk = ar.mark();
    if (tc == DT::F32) {
      TRY(jacobi_svd(d, ar, C, L, Vc, sig, Uc, polish_tol_fp32(L), 0.0, k));
    } else {
      if (!dry) TRY(transpose_lower_to_upper(d, C, CT, L));
      TRY(jacobi_svd(d, ar, CT, L, Uc, sig, Vc));
    }
    ar.release(mk);
  }
  if (!dry) trace_mark(d.s, "small_svd");
  // Step 6: U = P V~_k, V = Q U~_k, S = S~_k (the first rp / rq rows of the
  // L x L factors).
  const void* Vk = Vc;
  if (tc == DT::F32) {
    if (!dry) TRY(cast_copy(d, DT::F64, Vc, DT::F32, Vc_c, L * L));
    Vk = Vc_c;
  }
  TRY(tall_gemm(d, ar, tc, tc, DT::F64, n, kk, rp, Pv, rp, Vc, Vk, L, U, k, false));
  TRY(gemm64(d, ar, m, kk, rq, Q, rq, false, Uc, L, V, k));
  if (!dry) BSRHT_CUDA_TRY(cudaMemcpyAsync(S, sig, sizeof(double) * kk, cudaMemcpyDeviceToDevice, d.s));
  {
    const size_t mk = ar.mark();
    TRY(sign_normalize(d, ar, U, n, k, V, m));
    ar.release(mk);
  }
  if (!dry) trace_mark(d.s, "factors");
  if (dry) return BSRHT_OK;
  int hs = 0;
  TRY(read_status(d, &hs));
  return status_to_code(hs);
}

// ---------------------------------------------------------------- Nystrom
struct OmegaTables {
  uint32_t* s;      // l samples s_j (mod r)
  uint64_t* dbits;  // p * ceil(r/64) words of D signs
  uint64_t* dtbits; // p * ceil(l/64) words of Dt signs
};

__global__ void k_omega_tables(OmegaTables t, uint64_t seed, int64_t l, int p, int64_t r) {
  const int64_t dw = (r + 63) / 64, tw = (l + 63) / 64;
  const int64_t total = l + (int64_t)p * dw + (int64_t)p * tw;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < l) {
      t.s[idx] = (uint32_t)(sample_word(seed, (uint64_t)idx) & (uint64_t)(r - 1));
    } else if (idx < l + (int64_t)p * dw) {
      const int64_t e = idx - l, i = e / dw, w = e % dw;
      t.dbits[e] = sign_word(seed, kStreamD, (uint64_t)i, (uint64_t)w);
    } else {
      const int64_t e = idx - l - (int64_t)p * dw, i = e / tw, w = e % tw;
      t.dtbits[e] = sign_word(seed, kStreamDt, (uint64_t)i, (uint64_t)w);
    }
  }
}

// Ynu[row][j] = Y[row][j] + nu * Omega[j][row], Omega[j][i*rb+k] =
// Dt_jj^(i) H_r[s_j, k] D_kk^(i) / sqrt(l); nu = factor * sqrt(n) eps ||Y||_F.
template <typename TI, typename TO>
__global__ void k_add_omega_t(const TI* __restrict__ Y, TO* __restrict__ Ynu, int64_t n, int64_t l, int64_t rb,
                              int64_t r, OmegaTables t, const double* __restrict__ ynorm, double factor,
                              double* __restrict__ nu_out) {
  const double nu = factor * sqrt((double)n) * 2.220446049250313e-16 * (*ynorm);
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx == 0) *nu_out = nu;
  if (idx >= n * l) return;
  const int64_t row = idx / l, j = idx - row * l;
  const int64_t i = row / rb, kk = row - i * rb;
  const int64_t dw = (r + 63) / 64, tw = (l + 63) / 64;
  const uint32_t neg = (uint32_t)((__popcll((unsigned long long)t.s[j] & (unsigned long long)kk) +
                                   (int)((t.dbits[i * dw + (kk >> 6)] >> (kk & 63)) & 1ull) +
                                   (int)((t.dtbits[i * tw + (j >> 6)] >> (j & 63)) & 1ull)) & 1);
  const double om = (neg ? -1.0 : 1.0) / sqrt((double)l);
  Ynu[idx] = (TO)((double)Y[idx] + nu * om);
}

// Gs = (G + G^T)/2 in FP64.
template <typename T>
__global__ void k_symmetrize(const T* __restrict__ G, double* __restrict__ Gs, int64_t l) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= l * l) return;
  const int64_t i = idx / l, j = idx % l;
  Gs[idx] = 0.5 * ((double)G[i * l + j] + (double)G[j * l + i]);
}

__global__ void k_lambda(const double* __restrict__ sig, const double* __restrict__ nu, double* __restrict__ lam,
                         int k) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < k) lam[c] = fmax(sig[c] * sig[c] - *nu, 0.0);
}

// Matrix-free source of Algorithm 2: the kernel matrix
// A_ij = exp(-|x_i - x_j|^2 / (2 h^2)) of the points x_i (rows of X, n x dim,
// FP32, row stride ldx), generated a column panel at a time and sketched
// right away, so the n x n matrix is never stored.
struct RbfSource {
  const float* X = nullptr;  // nullptr: A is a stored matrix
  int64_t dim = 0, ldx = 0;
  double h = 0.0;
};

// sq[i] = |x_i|^2, summed in FP64 and rounded to FP32.
__global__ void k_row_sqnorm(const float* __restrict__ X, int64_t n, int64_t dim, int64_t ldx,
                             float* __restrict__ sq) {
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t c = threadIdx.x & 31; c < dim; c += 32) {
    const double v = X[i * ldx + c];
    s = fma(v, v, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sq[i] = (float)s;
}

// Panel of columns [j0, j0 + w) in place: G[i][j] = x_i . x_{j0+j} (FP32
// accuracy) becomes exp(-max(|x_i|^2 + |x_j|^2 - 2 G, 0) / (2 h^2)) in FP32
// arithmetic (the entries are FP32 values; the FP64 units of this GPU run
// at 1/64 of the FP32 rate), with the diagonal exactly 1.
__global__ void k_rbf_panel(float* __restrict__ P, int64_t n, int64_t w, int64_t j0, const float* __restrict__ sq,
                            float inv2h2) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * w) return;
  const int64_t i = idx / w, j = idx - i * w;
  const float d2 = fmaxf(sq[i] + sq[j0 + j] - 2.0f * P[idx], 0.0f);
  P[idx] = (i == j0 + j) ? 1.0f : expf(-d2 * inv2h2);
}

// Column-panel width of the matrix-free sketch: about 1 GiB of FP32 panel,
// a multiple of 64 columns, at most n.
int64_t rbf_panel_width(int64_t n) {
  int64_t w = ((int64_t)1 << 28) / std::max<int64_t>(n, 1);
  w = std::max<int64_t>(64, std::min<int64_t>(8192, w / 64 * 64));
  return std::min(w, n);
}

// B (l x n, row stride n) = Omega A for the kernel matrix of src: per panel,
// the Gram of the points on the tensor cores (3xTF32), the RBF map, and the
// sketch of the panel into B's columns.
int rbf_sketch(const Dla& d, Arena& ar, bool dry, const RbfSource& src, int64_t n, int p, int64_t l, int variant,
               uint64_t seed, float* B, void* sk_ws, size_t sk_bytes) {
  const int64_t w = rbf_panel_width(n);
  float* panel = static_cast<float*>(ar.take(sizeof(float) * (size_t)n * w));
  float* sq = static_cast<float*>(ar.take(sizeof(float) * (size_t)n));
  if (!ar.ok()) return BSRHT_ENOMEM;
  if (!dry) {
    k_row_sqnorm<<<(unsigned)((n + 7) / 8), 256, 0, d.s>>>(src.X, n, src.dim, src.ldx, sq);
    BSRHT_CUDA_TRY(cudaGetLastError());
    note_launches(1);
  }
  for (int64_t j0 = 0; j0 < n; j0 += w) {
    const int64_t wj = std::min(w, n - j0);
    {
      const size_t mk = ar.mark();
      const int st = gemm_tc(d, ar, n, wj, src.dim, src.X, src.ldx, DT::F32, src.X + j0 * src.ldx, src.ldx, true,
                             DT::F32, panel, wj, false);
      ar.release(mk);
      if (st != BSRHT_OK) return st;
    }
    if (!dry) trace_mark(d.s, "rbf_gram");
    SketchPlan sp;
    TRY(sketch_make_plan(sp, BSRHT_F32, variant, n, wj, wj, p, l, !dry, dry ? nullptr : panel));
    if (sp.work_bytes > sk_bytes) return BSRHT_ENOMEM;
    if (dry) break;  // every panel but the last has the same plan; the last one is narrower
    k_rbf_panel<<<(unsigned)((n * wj + 255) / 256), 256, 0, d.s>>>(panel, n, wj, j0, sq,
                                                                   (float)(0.5 / (src.h * src.h)));
    BSRHT_CUDA_TRY(cudaGetLastError());
    note_launches(1);
    trace_mark(d.s, "rbf_map");
    TRY(sketch_run(sp, panel, seed, B + j0, n, sk_ws, d.s));
  }
  return BSRHT_OK;
}

int nystrom_impl(const bsrht_opts& o, const void* A, int64_t n, int k, int64_t l, int p, uint64_t seed, double* U,
                 double* Lam, Arena& ar, bool dry, const RbfSource& src = RbfSource()) {
  // FP64 arithmetic for FP64 data and for FP32 data with precision
  // BSRHT_PREC_F64 (then Y is the FP64 sketch of the FP32 values).
  const bool f64 = o.dtype == BSRHT_F64 || o.precision == BSRHT_PREC_F64;
  const DT tc = f64 ? DT::F64 : DT::F32;
  const size_t cs = dt_size(tc);
  const int64_t lda = o.lda ? o.lda : n;
  SketchPlan sp_a, sp_y;
  const bool rbf = src.X != nullptr;
  int a_dt = o.dtype;
  if (!rbf) TRY(plan_dtype(o, &a_dt));
  if (rbf) {
    // The panels' plan (the widest panel) sizes the sketch scratch.
    const int64_t w = rbf_panel_width(n);
    TRY(sketch_make_plan(sp_a, BSRHT_F32, o.variant, n, w, w, p, l, !dry, nullptr));
  } else {
    TRY(sketch_make_plan(sp_a, a_dt, o.variant, n, n, lda, p, l, !dry, dry ? nullptr : A));
  }
  // The l x l core Omega Y_nu is formed in FP64 whatever the type of A, with
  // the FP64-add kernel: the shift nu of Remark 3.1 is a few FP64 units of
  // ||Y||, below the precision of the fixed-point FP64 sketch (an address
  // the TMA rules reject steers the plan to it, as for grouped sketches).
  TRY(sketch_make_plan(sp_y, BSRHT_F64, BSRHT_VARIANT_CUDACORE, n, l, l, p, l, !dry,
                       reinterpret_cast<const void*>(uintptr_t(1))));
  const int64_t rb = sp_a.rb, r = sp_a.r;
  Dla d{static_cast<cudaStream_t>(o.stream), nullptr};
  d.status = static_cast<int*>(ar.take(sizeof(int)));
  void* sk_ws = ar.take(std::max(sp_a.work_bytes, sp_y.work_bytes));
  void* B = ar.take(cs * l * n);     // sketch, later Y_nu in tc, later scratch
  void* Y = ar.take(cs * n * l);     // Y, later Z
  double* Y64 = static_cast<double*>(ar.take(8 * n * l));  // Y_nu in FP64
  void* Z3 = ar.take(cs * n * l);
  double* G = static_cast<double*>(ar.take(8 * l * l));
  double* LT1 = static_cast<double*>(ar.take(8 * l * l));
  double* Cinv = static_cast<double*>(ar.take(8 * l * l));
  void* Cinv_c = ar.take(cs * l * l);
  double* R = static_cast<double*>(ar.take(8 * l * l));
  double* RT = static_cast<double*>(ar.take(8 * l * l));
  double* Us = static_cast<double*>(ar.take(8 * l * l));
  double* Vs = static_cast<double*>(ar.take(8 * l * l));
  double* sig = static_cast<double*>(ar.take(8 * l));
  void* Vs_c = ar.take(cs * l * l);
  double* ynorm = static_cast<double*>(ar.take(8));
  double* nu = static_cast<double*>(ar.take(8));
  OmegaTables t;
  const int64_t dw = (r + 63) / 64, tw = (l + 63) / 64;
  t.s = static_cast<uint32_t*>(ar.take(4 * l));
  t.dbits = static_cast<uint64_t*>(ar.take(8 * p * dw));
  t.dtbits = static_cast<uint64_t*>(ar.take(8 * p * tw));
  const OrthBufs ob = take_orth_bufs(ar, l, cs);
  if (!ar.ok()) return BSRHT_ENOMEM;
  if (!dry) {
    BSRHT_CUDA_TRY(cudaMemsetAsync(d.status, 0, sizeof(int), d.s));
    // Step 1: Y = A Omega^T = (Omega A)^T for symmetric A.
    trace_begin(d.s);
    if (rbf) {
      const size_t mk = ar.mark();
      TRY(rbf_sketch(d, ar, false, src, n, p, l, o.variant, seed, static_cast<float*>(B), sk_ws,
                     std::max(sp_a.work_bytes, sp_y.work_bytes)));
      ar.release(mk);
    } else {
      TRY(sketch_run(sp_a, A, seed, B, n, sk_ws, d.s));
    }
    trace_mark(d.s, "sketch");
    TRY(transpose_cast(d, tc, B, l, n, n, tc, Y, l));
    {
      const size_t mk = ar.mark();
      TRY(frob_norm(d, ar, tc, Y, n * l, ynorm));
      ar.release(mk);
    }
    const int64_t ttot = l + (int64_t)p * dw + (int64_t)p * tw;
    k_omega_tables<<<(unsigned)std::min<int64_t>((ttot + 255) / 256, 4096), 256, 0, d.s>>>(t, seed, l, p, r);
    BSRHT_CUDA_TRY(cudaGetLastError());
    note_launches(1);
  } else {
    size_t mk = ar.mark();
    TRY(frob_norm(d, ar, tc, Y, n * l, ynorm));
    ar.release(mk);
    if (rbf) {
      mk = ar.mark();
      TRY(rbf_sketch(d, ar, true, src, n, p, l, o.variant, seed, nullptr, nullptr,
                     std::max(sp_a.work_bytes, sp_y.work_bytes)));
      ar.release(mk);
    }
  }
  // Steps 1b-2 (Remark 3.1): Y_nu = Y + nu Omega^T, core = sym(Omega Y_nu) in
  // FP64 and its Cholesky factor C (C^T C = core).  When the factorization
  // fails or its pivots show that the core is numerically rank deficient
  // (repeated rows of Omega, which sampling with replacement allows, or a
  // low-rank A), C is replaced by the SVD square root of Remark 3.1: the
  // core's eigenvectors V_r scaled by lambda_r^-1/2, lambda below
  // tau lambda_max dropped, i.e. the pseudo-inverse of the definition.
  const double tau_core = (double)l * (tc == DT::F64 ? 0x1.0p-52 : 0x1.0p-23);
  bool use_eig = dry;
  double* pr = static_cast<double*>(ar.take(8));
  if (!ar.ok()) return BSRHT_ENOMEM;
  if (!dry) {
    const unsigned nb = (unsigned)((n * l + 255) / 256);
    if (tc == DT::F64)
      k_add_omega_t<double, double><<<nb, 256, 0, d.s>>>(static_cast<const double*>(Y), Y64, n, l, rb, r, t, ynorm,
                                                          1.0, nu);
    else
      k_add_omega_t<float, double><<<nb, 256, 0, d.s>>>(static_cast<const float*>(Y), Y64, n, l, rb, r, t, ynorm,
                                                         1.0, nu);
    BSRHT_CUDA_TRY(cudaGetLastError());
    TRY(sketch_run(sp_y, Y64, seed, R, l, sk_ws, d.s));
    k_symmetrize<double><<<(unsigned)((l * l + 255) / 256), 256, 0, d.s>>>(R, G, l);
    BSRHT_CUDA_TRY(cudaGetLastError());
    TRY(chol_inv(d, G, LT1, Cinv, ob.Ug, ob.Vg, l));  // C^-1 = L^-T, used unless the eig path is taken
    k_pivot_ratio<<<1, 256, 0, d.s>>>(G, l, pr);
    BSRHT_CUDA_TRY(cudaGetLastError());
    note_launches(3);
    double ratio = 0.0;
    BSRHT_CUDA_TRY(cudaMemcpyAsync(&ratio, pr, sizeof(double), cudaMemcpyDeviceToHost, d.s));
    int hs = 0;
    TRY(read_status(d, &hs));
    if (hs & kStatusTcWait) return BSRHT_ETIMEDOUT;
    if ((hs & kStatusNotPD) || !(ratio > tau_core)) {
      use_eig = true;
      BSRHT_CUDA_TRY(cudaMemsetAsync(d.status, 0, sizeof(int), d.s));
    }
  }
  if (!dry) trace_mark(d.s, "core");
  // Step 3: Z = Y_nu C^-1 in the arithmetic of A (C^-1 = L^-T, or V_r lambda_r^-1/2).
  const void* Ynu = Y64;
  if (!dry && tc == DT::F32) TRY(cast_copy(d, DT::F64, Y64, DT::F32, B, n * l));
  if (tc == DT::F32) Ynu = B;
  void* Z = Y;
  bool z_t = false;  // Z^T left in Z3, the Gram scratch of the QR of step 4
  float* const Zt = tc == DT::F32 ? static_cast<float*>(Z3) : nullptr;
  if (!use_eig || dry) {
    if (!dry && tc == DT::F32) TRY(cast_copy(d, DT::F64, Cinv, DT::F32, Cinv_c, l * l));
    TRY(tall_gemm(d, ar, tc, tc, tc, n, l, l, Ynu, l, Cinv, tc == DT::F32 ? Cinv_c : (const void*)Cinv, l, Z, l,
                  true, Zt, &z_t));
  }
  int64_t lr = l;  // columns of Z (the kept rank on the SVD square root path)
  if (use_eig) {
    if (!dry) {
      k_symmetrize<double><<<(unsigned)((l * l + 255) / 256), 256, 0, d.s>>>(R, G, l);
      BSRHT_CUDA_TRY(cudaGetLastError());
      note_launches(1);
    }
    {
      // FP32 data: only eigenvalues above tau_core lambda_max are kept, so
      // only those columns (with a margin) are polished in FP64.
      const size_t mk = ar.mark();
      if (tc == DT::F32)
        TRY(jacobi_svd(d, ar, G, l, ob.Ug, ob.lam, Cinv, polish_tol_fp32(l), 0.0, 0, 0.5 * tau_core));
      else
        TRY(jacobi_svd(d, ar, G, l, ob.Ug, ob.lam, Cinv));
      ar.release(mk);
    }
    if (!dry) {
      std::vector<double> lam_h((size_t)l);
      BSRHT_CUDA_TRY(cudaMemcpyAsync(lam_h.data(), ob.lam, sizeof(double) * l, cudaMemcpyDeviceToHost, d.s));
      BSRHT_CUDA_TRY(cudaStreamSynchronize(d.s));
      lr = 0;
      for (int64_t c = 0; c < l; ++c)
        if (lam_h[0] > 0.0 && lam_h[c] > tau_core * lam_h[0]) ++lr;
      if (lr == 0) return BSRHT_ENOTPD;  // A Omega^T vanishes
      k_svqb_scale<<<(unsigned)((l + 127) / 128), 128, 0, d.s>>>(ob.lam, ob.sc, l, tau_core);
      BSRHT_CUDA_TRY(cudaGetLastError());
      note_launches(1);
      TRY(scale_columns(d, Cinv, l, l, l, ob.sc, false));
      if (tc == DT::F32) TRY(cast_copy(d, DT::F64, Cinv, DT::F32, Cinv_c, l * l));
    }
    // Z = Y_nu V_r lambda_r^-1/2, n x lr (contiguous, leading dimension lr).
    TRY(tall_gemm(d, ar, tc, tc, tc, n, lr, l, Ynu, l, Cinv, tc == DT::F32 ? Cinv_c : (const void*)Cinv, l, Z, lr,
                  false, Zt, &z_t));
  }
  if (!dry) trace_mark(d.s, "z");
  // Step 4: R factor of Z (CholeskyQR2, rank-robust); Z itself is kept for step 6.
  {
    void* scratch = (tc == DT::F32) ? B : (void*)Y64;
    void* Qv = nullptr;
    TRY(orth_robust(d, ar, dry, tc, Z, scratch, Z3, n, lr, seed ^ 0x53ull, ob, R, false, true, &Qv, nullptr, z_t));
  }
  if (!dry) trace_mark(d.s, "tall_qr");
  // Step 5: SVD of R = U~ Sigma~ V~^T (Jacobi on the columns of R, i.e. rows of R^T).
  if (!dry) {
    TRY(transpose_lower_to_upper(d, R, RT, lr));
    BSRHT_CUDA_TRY(cudaMemsetAsync(sig, 0, sizeof(double) * l, d.s));
    BSRHT_CUDA_TRY(cudaMemsetAsync(U, 0, sizeof(double) * n * k, d.s));
  }
  {
    const size_t mk = ar.mark();
    TRY(jacobi_svd(d, ar, RT, lr, Us, sig, Vs, tc == DT::F32 ? polish_tol_fp32(lr) : 0.0, 0.0,
                   tc == DT::F32 ? k : 0));
    ar.release(mk);
  }
  if (!dry) trace_mark(d.s, "small_svd");
  // Step 6: U^ = (Z V~_k) Sigma~_k^-1; step 7: Lambda = max(Sigma~_k^2 - nu, 0).
  const int64_t kk = std::min<int64_t>(k, lr);
  const void* Vk = Vs;
  if (tc == DT::F32) {
    if (!dry) TRY(cast_copy(d, DT::F64, Vs, DT::F32, Vs_c, lr * lr));
    Vk = Vs_c;
  }
  TRY(tall_gemm(d, ar, tc, tc, DT::F64, n, kk, lr, Z, lr, Vs, Vk, lr, U, k, false));
  if (!dry) {
    TRY(scale_columns(d, U, n, k, k, sig, true));
    k_lambda<<<(unsigned)((k + 127) / 128), 128, 0, d.s>>>(sig, nu, Lam, k);
    BSRHT_CUDA_TRY(cudaGetLastError());
    note_launches(1);
  }
  {
    const size_t mk = ar.mark();
    TRY(sign_normalize(d, ar, U, n, k, nullptr, 0));
    ar.release(mk);
  }
  if (!dry) trace_mark(d.s, "factors");
  if (dry) return BSRHT_OK;
  int hs = 0;
  TRY(read_status(d, &hs));
  return status_to_code(hs);
}

int validate_rsvd(const bsrht_opts& o, int64_t n, int64_t m, int k, int64_t l, int p) {
  if (o.dtype < BSRHT_F64 || o.dtype > BSRHT_F16) return BSRHT_EINVAL;
  TRY(precision_auto_only(o));
  if (n < 1 || m < 1 || k < 1 || l < k || l > m || l > n || p < 1 || p > n) return BSRHT_EINVAL;
  if (o.lda != 0 && o.lda < m) return BSRHT_EINVAL;
  return BSRHT_OK;
}

int validate_srsvd(const bsrht_opts& o, int64_t n, int64_t m, int k, int64_t l, int64_t s, int p) {
  if (o.dtype != BSRHT_F64 && o.dtype != BSRHT_F32) return o.dtype >= BSRHT_F64 && o.dtype <= BSRHT_F16
                                                               ? BSRHT_EUNSUP : BSRHT_EINVAL;
  TRY(precision_auto_only(o));
  if (o.variant != BSRHT_VARIANT_AUTO && o.variant != BSRHT_VARIANT_CUDACORE) return BSRHT_EUNSUP;
  if (n < 1 || m < 1 || k < 1 || l < k || s < l || s > m || s > n || p < 1 || p > n) return BSRHT_EINVAL;
  if (o.lda != 0 && o.lda < m) return BSRHT_EINVAL;
  return BSRHT_OK;
}

int validate_nystrom(const bsrht_opts& o, int64_t n, int k, int64_t l, int p) {
  if (o.dtype < BSRHT_F64 || o.dtype > BSRHT_F16) return BSRHT_EINVAL;
  {
    int dt = 0;
    TRY(plan_dtype(o, &dt));  // FP64 arithmetic on FP32 storage, or the dtype's
  }
  // The shift of Remark 3.1 adds nu Omega^T entry by entry from the block
  // SRHT definition; the Gaussian comparator is a sketch / rSVD option only.
  if (o.variant == BSRHT_VARIANT_GAUSSIAN) return BSRHT_EUNSUP;
  if (n < 1 || k < 1 || l < k || l > n || p < 1 || p > n) return BSRHT_EINVAL;
  if (o.lda != 0 && o.lda < n) return BSRHT_EINVAL;
  return BSRHT_OK;
}

int validate_nystrom_rbf(const bsrht_opts& o, const float* X, int64_t n, int64_t dim, double h, int k, int64_t l,
                         int p) {
  if (o.dtype != BSRHT_F32) return o.dtype >= BSRHT_F64 && o.dtype <= BSRHT_F16 ? BSRHT_EUNSUP : BSRHT_EINVAL;
  TRY(precision_auto_only(o));
  if (o.variant == BSRHT_VARIANT_GAUSSIAN || o.variant == BSRHT_VARIANT_TENSOR) return BSRHT_EUNSUP;
  if (dim < 1 || !(h > 0.0) || !std::isfinite(h)) return BSRHT_EINVAL;
  const int64_t ldx = o.lda ? o.lda : dim;
  if (ldx < dim) return BSRHT_EINVAL;
  if ((ldx % 4) != 0 || (reinterpret_cast<uintptr_t>(X) % 16) != 0) return BSRHT_EUNSUP;
  bsrht_opts on = o;
  on.lda = 0;  // opts->lda is the stride of X here, not of an n x n matrix
  return validate_nystrom(on, n, k, l, p);
}

}  // namespace
}  // namespace bsrht

using namespace bsrht;

extern "C" {

int bsrht_rsvd_workspace(int64_t n, int64_t m, int32_t k, int64_t l, int32_t p, const bsrht_opts* opts,
                         size_t* bytes) {
  if (!bytes) return BSRHT_EINVAL;
  const bsrht_opts o = opts_or_default(opts);
  TRY(validate_rsvd(o, n, m, k, l, p));
  Arena ar;
  ar.measure = true;
  TRY(rsvd_impl(o, nullptr, n, m, k, l, p, 0, nullptr, nullptr, nullptr, ar, true));
  *bytes = ar.high + 256;
  return BSRHT_OK;
}

int bsrht_rsvd(const void* A, int64_t n, int64_t m, int32_t k, int64_t l, int32_t p, uint64_t seed, double* U,
               double* S, double* V, const bsrht_opts* opts) {
  const bsrht_opts o = opts_or_default(opts);
  TRY(validate_rsvd(o, n, m, k, l, p));
  if (!A || !U || !S || !V) return BSRHT_EINVAL;
  size_t need = 0;
  TRY(bsrht_rsvd_workspace(n, m, k, l, p, &o, &need));
  void* ws = nullptr;
  TRY(workspace_for(&o, need, &ws));
  Arena ar;
  ar.base = static_cast<char*>(ws);
  ar.cap = need;
  return rsvd_impl(o, A, n, m, k, l, p, seed, U, S, V, ar, false);
}

int bsrht_srsvd_workspace(int64_t n, int64_t m, int32_t k, int64_t l, int64_t s, int32_t p, const bsrht_opts* opts,
                          size_t* bytes) {
  if (!bytes) return BSRHT_EINVAL;
  const bsrht_opts o = opts_or_default(opts);
  TRY(validate_srsvd(o, n, m, k, l, s, p));
  Arena ar;
  ar.measure = true;
  TRY(srsvd_impl(o, nullptr, n, m, k, l, s, p, 0, nullptr, nullptr, nullptr, ar, true));
  *bytes = ar.high + 256;
  return BSRHT_OK;
}

int bsrht_srsvd(const void* A, int64_t n, int64_t m, int32_t k, int64_t l, int64_t s, int32_t p, uint64_t seed,
                double* U, double* S, double* V, const bsrht_opts* opts) {
  const bsrht_opts o = opts_or_default(opts);
  TRY(validate_srsvd(o, n, m, k, l, s, p));
  if (!A || !U || !S || !V) return BSRHT_EINVAL;
  size_t need = 0;
  TRY(bsrht_srsvd_workspace(n, m, k, l, s, p, &o, &need));
  void* ws = nullptr;
  TRY(workspace_for(&o, need, &ws));
  Arena ar;
  ar.base = static_cast<char*>(ws);
  ar.cap = need;
  return srsvd_impl(o, A, n, m, k, l, s, p, seed, U, S, V, ar, false);
}

int bsrht_nystrom_workspace(int64_t n, int32_t k, int64_t l, int32_t p, const bsrht_opts* opts, size_t* bytes) {
  if (!bytes) return BSRHT_EINVAL;
  const bsrht_opts o = opts_or_default(opts);
  TRY(validate_nystrom(o, n, k, l, p));
  Arena ar;
  ar.measure = true;
  TRY(nystrom_impl(o, nullptr, n, k, l, p, 0, nullptr, nullptr, ar, true));
  *bytes = ar.high + 256;
  return BSRHT_OK;
}


int bsrht_nystrom_rbf_workspace(int64_t n, int64_t dim, int32_t k, int64_t l, int32_t p, const bsrht_opts* opts,
                                size_t* bytes) {
  if (!bytes) return BSRHT_EINVAL;
  bsrht_opts o = opts_or_default(opts);
  TRY(validate_nystrom_rbf(o, nullptr, n, dim, 1.0, k, l, p));
  RbfSource src;
  src.X = reinterpret_cast<const float*>(uintptr_t(256));  // marks the source; never read in a dry run
  src.dim = dim;
  src.ldx = o.lda ? o.lda : dim;
  src.h = 1.0;
  o.lda = 0;
  Arena ar;
  ar.measure = true;
  TRY(nystrom_impl(o, nullptr, n, k, l, p, 0, nullptr, nullptr, ar, true, src));
  *bytes = ar.high + 256;
  return BSRHT_OK;
}

int bsrht_nystrom_rbf(const float* X, int64_t n, int64_t dim, double h, int32_t k, int64_t l, int32_t p,
                      uint64_t seed, double* U, double* Lambda, const bsrht_opts* opts) {
  bsrht_opts o = opts_or_default(opts);
  if (!X || !U || !Lambda) return BSRHT_EINVAL;
  TRY(validate_nystrom_rbf(o, X, n, dim, h, k, l, p));
  size_t need = 0;
  TRY(bsrht_nystrom_rbf_workspace(n, dim, k, l, p, &o, &need));
  void* ws = nullptr;
  TRY(workspace_for(&o, need, &ws));
  RbfSource src;
  src.X = X;
  src.dim = dim;
  src.ldx = o.lda ? o.lda : dim;
  src.h = h;
  o.lda = 0;
  Arena ar;
  ar.base = static_cast<char*>(ws);
  ar.cap = need;
  return nystrom_impl(o, nullptr, n, k, l, p, seed, U, Lambda, ar, false, src);
}

int bsrht_nystrom(const void* A, int64_t n, int32_t k, int64_t l, int32_t p, uint64_t seed, double* U,
                  double* Lambda, const bsrht_opts* opts) {
  const bsrht_opts o = opts_or_default(opts);
  TRY(validate_nystrom(o, n, k, l, p));
  if (!A || !U || !Lambda) return BSRHT_EINVAL;
  size_t need = 0;
  TRY(bsrht_nystrom_workspace(n, k, l, p, &o, &need));
  void* ws = nullptr;
  TRY(workspace_for(&o, need, &ws));
  Arena ar;
  ar.base = static_cast<char*>(ws);
  ar.cap = need;
  return nystrom_impl(o, A, n, k, l, p, seed, U, Lambda, ar, false);
}

}  // extern "C"
