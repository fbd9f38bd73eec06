// Dense linear algebra for the low-rank drivers (host interface).
//
// Tall-skinny products run on the tiled CUDA-core GEMM (gemm.cuh); the small
// l x l factorizations (Cholesky, triangular inverse, one-sided Jacobi SVD)
// run in FP64 on the device.  Everything is enqueued on one stream; scratch
// comes from a caller-provided arena.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace bsrht {

enum class DT { F64, F32, BF16, F16 };

inline size_t dt_size(DT t) { return t == DT::F64 ? 8 : (t == DT::F32 ? 4 : 2); }

// Bump allocator over a caller buffer (256-byte aligned slices).
struct Arena {
  char* base = nullptr;
  size_t cap = 0, used = 0, high = 0;
  bool measure = false;  // only count bytes (no pointers handed out)
  void* take(size_t bytes) {
    used = (used + 255) / 256 * 256;
    void* p = measure ? nullptr : base + used;
    used += bytes;
    if (used > high) high = used;
    return p;
  }
  // Scratch taken after mark() may be handed out again after release():
  // every user is stream-ordered on the same stream.
  size_t mark() const { return used; }
  void release(size_t m) { used = m; }
  bool ok() const { return measure || used <= cap; }
};

struct Dla {
  cudaStream_t s;
  int* status;  // device int: 0 ok, else first failure code (see kStatus*)
};

constexpr int kStatusNotPD = 1;
constexpr int kStatusNoConv = 2;
// A tensor-core product (gemm_tc) gave up one of its bounded waits; its
// output is not valid.
constexpr int kStatusTcWait = 8;

// C[M x N] = alpha * op(A) B + beta C.  op(A) = A (M x K, lda) or A^T (A is
// K x M, lda).  B is K x N (ldb).  Accumulation in FP64 when acc64, else
// FP32.  tri_b: B upper triangular.  gram: C is the symmetric M x M product
// A^T A (a_trans, B == A), only the upper tiles are formed and mirrored.
// splitk scratch is taken from the arena when needed.
int gemm(const Dla& d, Arena& ar, DT ta, DT tb, DT tc, bool acc64, int64_t M, int64_t N, int64_t K,
         const void* A, int64_t lda, bool a_trans, const void* B, int64_t ldb, void* C, int64_t ldc,
         double alpha, double beta, bool tri_b, bool gram);

// Lower Cholesky factor L (G = L L^T) of the symmetric l x l FP64 matrix g
// (lower triangle read; ldg = l); L overwrites g's lower triangle, the strict
// upper triangle is zeroed.  Sets *status |= kStatusNotPD on a non-positive
// pivot.
int cholesky(const Dla& d, double* g, int64_t l);

// Rinv = L^-T (upper triangular, row-major) for the lower-triangular l x l
// L; LT receives L^T (the upper Cholesky factor R = L^T).
int tri_inverse(const Dla& d, const double* L, double* LT, double* Rinv, int64_t l);

// cholesky followed by tri_inverse in one cooperative kernel: L in the lower
// triangle of g (upper zeroed), LT = L^T, Rinv = L^-T; T and X are l x l
// FP64 scratch.  Sets *status |= kStatusNotPD on a non-positive pivot (the
// outputs are then meaningless).
int chol_inv(const Dla& d, double* g, double* LT, double* Rinv, double* T, double* X, int64_t l);

// One-sided Jacobi SVD of the l x l FP64 matrix given by its COLUMNS:
// colsM[c*l + i] = M[i][c].  The singular triplets, sorted by descending
// sigma, go to U (l x l row-major, U[i][c]), sigma and Vout (row-major).
// polish_tol > 0 replaces the FP64 rotation threshold sqrt(l) 2^-52 on the
// cosine of a pair: Vout (accumulated rotations) stays orthogonal to FP64
// rounding whatever the threshold, the columns of U to about polish_tol.
// Two columns whose norms are both at most zero_rel ||M||_F (at least
// l 2^-53) count as numerically zero and are not rotated against each other:
// a caller that drops directions below a rank threshold passes it here, so
// that columns made of rounding noise at that level do not keep the sweeps
// going.
// ktop > 0 with polish_tol > 0 (a caller at FP32-data accuracy that uses
// only the leading ktop triplets, l > 64): only the s = min(l, ktop +
// max(16, ktop / 4)) leading columns of the FP32 phase are polished in FP64
// (the SVD of M restricted to their span, which differs from the leading
// triplets of M in second order of the FP32 phase's residual cosines);
// ranks s and beyond hold the FP32 phase's estimates.  keep_rel > 0 with
// polish_tol > 0 and ktop = 0 (a caller that keeps the triplets with
// sigma > keep_rel sigma_1): s = c + max(16, c / 4) with c the FP32 phase's
// count above that threshold.  colsM is overwritten in every case.
int jacobi_svd(const Dla& d, Arena& ar, double* colsM, int64_t l, double* U, double* sigma, double* Vout,
               double polish_tol = 0.0, double zero_rel = 0.0, int64_t ktop = 0, double keep_rel = 0.0);

// Tensor-core (tcgen05) GEMM in FP32 accuracy (three TF32 products):
// C (M x N, FP32 or FP64 in tc_out, ldc) = A (M x K, FP32, lda) * B, with B
// either K x N (FP32 or FP64, ldb; transposed into scratch) or, when
// b_kmajor, given as Bt = B^T (N x K, FP32, ldb).  gram: C = A A^T (B = A^T),
// only tiles on or above the diagonal are formed and the rest mirrored.
// A and Bt need 16-byte aligned rows (gemm_tc_eligible).
// b_upper: B is upper triangular (B[k][n] = 0 for k > n); the zero K blocks
// of each N tile are skipped.  Ct (optional, FP32 output, not gram): also
// Ct[j * M + i] = C[i][j], the transposed copy (N x M) that tall Gram
// products read.
int gemm_tc(const Dla& d, Arena& ar, int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, DT tb,
            const void* B, int64_t ldb, bool b_kmajor, DT tc_out, void* C, int64_t ldc, bool gram,
            bool b_upper = false, float* Ct = nullptr);
bool gemm_tc_eligible(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda);
// Bt (N x ldk, FP32) = B^T for B K x N (FP32 or FP64, ldb); Bt[:, K:ldk] = 0.
int transpose_to_f32(const Dla& d, DT tb, const void* B, int64_t K, int64_t N, int64_t ldb, float* Bt, int64_t ldk,
                     float* Blo = nullptr);

// Householder QR of the tall FP64 X (rows x l, rows >= l), X overwritten by
// the reflectors; Q (rows x l, orthonormal columns) is formed explicitly.
// Robust to rank deficiency (a zero column gives an identity reflector).
int householder_q(const Dla& d, Arena& ar, double* X, int64_t rows, int64_t l, double* Q);

// Elementwise helpers.
int transpose_cast(const Dla& d, DT tin, const void* in, int64_t rows, int64_t cols, int64_t ldin, DT tout,
                   void* out, int64_t ldout);  // out[c][r] = in[r][c]
int cast_copy(const Dla& d, DT tin, const void* in, DT tout, void* out, int64_t count);
int transpose_lower_to_upper(const Dla& d, const double* Li, double* R, int64_t l);  // R = Li^T
int scale_columns(const Dla& d, double* X, int64_t rows, int64_t cols, int64_t ld, const double* scale,
                  bool invert);
int sign_normalize(const Dla& d, Arena& ar, double* U, int64_t n, int64_t k, double* V, int64_t m);
int frob_norm(const Dla& d, Arena& ar, DT t, const void* X, int64_t count, double* out);

}  // namespace bsrht
