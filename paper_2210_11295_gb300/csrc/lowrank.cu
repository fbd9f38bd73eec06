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

// One CholeskyQR pass on the tall X (rows x l, type tc):
// G = X^T X (FP64), L = chol(G), Rinv = L^-T, Xout = X Rinv; LT = L^T.
int cholqr_pass(const Dla& d, Arena& ar, bool dry, DT tc, const void* X, void* Xout, int64_t rows, int64_t l,
                double* G, double* LT, double* Rinv, void* Rinv_c) {
  TRY(gemm_c(d, ar, tc, tc, DT::F64, l, l, rows, X, l, true, X, l, G, l, false, true));
  if (!dry) {
    TRY(cholesky(d, G, l));
    TRY(tri_inverse(d, G, LT, Rinv, l));
    if (tc == DT::F32) TRY(cast_copy(d, DT::F64, Rinv, DT::F32, Rinv_c, l * l));
  }
  const void* Rb = (tc == DT::F32) ? Rinv_c : (const void*)Rinv;
  TRY(gemm_c(d, ar, tc, tc, tc, rows, l, l, X, l, false, Rb, l, Xout, l, true, false));
  return BSRHT_OK;
}

int read_status(const Dla& d, int* host) {
  BSRHT_CUDA_TRY(cudaMemcpyAsync(host, d.status, sizeof(int), cudaMemcpyDeviceToHost, d.s));
  BSRHT_CUDA_TRY(cudaStreamSynchronize(d.s));
  return BSRHT_OK;
}

int status_to_code(int s) {
  if (s & kStatusNotPD) return BSRHT_ENOTPD;
  if (s & kStatusNoConv) return BSRHT_ENOCONV;
  return BSRHT_OK;
}

// ---------------------------------------------------------------- RSVD
int rsvd_impl(const bsrht_opts& o, const void* A, int64_t n, int64_t m, int k, int64_t l, int p, uint64_t seed,
              double* U, double* S, double* V, Arena& ar, bool dry) {
  const DT ta = dt_of(o.dtype);
  const DT tc = (ta == DT::F64) ? DT::F64 : DT::F32;
  const size_t cs = dt_size(tc);
  const int64_t lda = o.lda ? o.lda : m;
  SketchPlan sp;
  TRY(sketch_make_plan(sp, o.dtype, o.variant, n, m, lda, p, l, !dry));
  Dla d{static_cast<cudaStream_t>(o.stream), nullptr};
  d.status = static_cast<int*>(ar.take(sizeof(int)));
  void* sk_ws = ar.take(sp.work_bytes);
  void* B = ar.take(cs * l * m);
  double* X = static_cast<double*>(ar.take(8 * m * l));
  double* X2 = static_cast<double*>(ar.take(8 * m * l));
  double* G = static_cast<double*>(ar.take(8 * l * l));
  double* LT1 = static_cast<double*>(ar.take(8 * l * l));
  double* LT2 = static_cast<double*>(ar.take(8 * l * l));
  double* Rinv = static_cast<double*>(ar.take(8 * l * l));
  void* Rinv_c = ar.take(cs * l * l);
  void* Qc = ar.take(cs * m * l);
  void* W = ar.take(cs * n * l);
  void* P = ar.take(cs * n * l);
  double* R = static_cast<double*>(ar.take(8 * l * l));
  double* Us = static_cast<double*>(ar.take(8 * l * l));
  double* Vs = static_cast<double*>(ar.take(8 * l * l));
  double* sig = static_cast<double*>(ar.take(8 * l));
  void* Vs_c = ar.take(cs * l * l);
  if (!ar.ok()) return BSRHT_ENOMEM;
  if (!dry) BSRHT_CUDA_TRY(cudaMemsetAsync(d.status, 0, sizeof(int), d.s));

  // Step 1: B = Omega A (l x m); the paper's Y is B^T.
  if (!dry) TRY(sketch_run(sp, A, seed, B, m, sk_ws, d.s));
  // Step 2: Q = orth(B^T) by FP64 CholeskyQR2 on X = B^T (m x l).
  if (!dry) TRY(transpose_cast(d, tc, B, l, m, m, DT::F64, X, l));
  TRY(cholqr_pass(d, ar, dry, DT::F64, X, X2, m, l, G, LT1, Rinv, nullptr));
  TRY(cholqr_pass(d, ar, dry, DT::F64, X2, X, m, l, G, LT2, Rinv, nullptr));
  double* Q = X;  // m x l, FP64
  const void* Qa = Q;
  if (tc == DT::F32) {
    if (!dry) TRY(cast_copy(d, DT::F64, Q, DT::F32, Qc, m * l));
    Qa = Qc;
  }
  // Step 3: the paper's Z = Q^T A_paper, i.e. Z^T = A Q (n x l): second pass over A.
  TRY(gemm_c(d, ar, ta, tc, tc, n, l, m, A, lda, false, Qa, l, W, l, false, false));
  // Step 4: Z^T = P R by CholeskyQR2 (R = R2 R1, R_i = L_i^T).
  TRY(cholqr_pass(d, ar, dry, tc, W, P, n, l, G, LT1, Rinv, Rinv_c));
  TRY(cholqr_pass(d, ar, dry, tc, P, W, n, l, G, LT2, Rinv, Rinv_c));
  void* Pf = W;  // final P (n x l)
  TRY(gemm64(d, ar, l, l, l, LT2, l, false, LT1, l, R, l, true, false));
  // Step 5: SVD of R^T; the columns of R^T are the rows of R.
  {
    const size_t mk = ar.mark();
    TRY(jacobi_svd(d, ar, R, l, Us, sig, Vs));
    ar.release(mk);
  }
  // Step 6: U = P V~_k, V = Q U~_k, S = Sigma~_k.
  const void* Vk = Vs;
  if (tc == DT::F32) {
    if (!dry) TRY(cast_copy(d, DT::F64, Vs, DT::F32, Vs_c, l * l));
    Vk = Vs_c;
  }
  TRY(gemm_c(d, ar, tc, tc, DT::F64, n, k, l, Pf, l, false, Vk, l, U, k, false, false));
  TRY(gemm64(d, ar, m, k, l, Q, l, false, Us, l, V, k));
  if (!dry) BSRHT_CUDA_TRY(cudaMemcpyAsync(S, sig, sizeof(double) * k, cudaMemcpyDeviceToDevice, d.s));
  {
    const size_t mk = ar.mark();
    TRY(sign_normalize(d, ar, U, n, k, V, m));
    ar.release(mk);
  }
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
template <typename T>
__global__ void k_add_omega_t(const T* __restrict__ Y, T* __restrict__ Ynu, int64_t n, int64_t l, int64_t rb,
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
  Ynu[idx] = (T)((double)Y[idx] + nu * om);
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

int nystrom_impl(const bsrht_opts& o, const void* A, int64_t n, int k, int64_t l, int p, uint64_t seed, double* U,
                 double* Lam, Arena& ar, bool dry) {
  const DT ta = dt_of(o.dtype);
  const DT tc = (ta == DT::F64) ? DT::F64 : DT::F32;
  const size_t cs = dt_size(tc);
  const int64_t lda = o.lda ? o.lda : n;
  SketchPlan sp_a, sp_y;
  TRY(sketch_make_plan(sp_a, o.dtype, o.variant, n, n, lda, p, l, !dry));
  TRY(sketch_make_plan(sp_y, tc == DT::F64 ? BSRHT_F64 : BSRHT_F32, BSRHT_VARIANT_CUDACORE, n, l, l, p, l, !dry));
  const int64_t rb = sp_a.rb, r = sp_a.r;
  Dla d{static_cast<cudaStream_t>(o.stream), nullptr};
  d.status = static_cast<int*>(ar.take(sizeof(int)));
  void* sk_ws = ar.take(std::max(sp_a.work_bytes, sp_y.work_bytes));
  void* B = ar.take(cs * l * n);
  void* Y = ar.take(cs * n * l);
  void* Ynu = ar.take(cs * n * l);
  void* Gc = ar.take(cs * l * l);
  double* G = static_cast<double*>(ar.take(8 * l * l));
  double* LT1 = static_cast<double*>(ar.take(8 * l * l));
  double* LT2 = static_cast<double*>(ar.take(8 * l * l));
  double* Cinv = static_cast<double*>(ar.take(8 * l * l));
  double* Rinv = static_cast<double*>(ar.take(8 * l * l));
  void* Rinv_c = ar.take(cs * l * l);
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
  if (!ar.ok()) return BSRHT_ENOMEM;
  if (!dry) {
    BSRHT_CUDA_TRY(cudaMemsetAsync(d.status, 0, sizeof(int), d.s));
    // Step 1: Y = A Omega^T = (Omega A)^T for symmetric A.
    TRY(sketch_run(sp_a, A, seed, B, n, sk_ws, d.s));
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
    const size_t mk = ar.mark();
    TRY(frob_norm(d, ar, tc, Y, n * l, ynorm));
    ar.release(mk);
  }
  // Steps 1b-2: shifted core and its Cholesky factor, doubling the shift on failure.
  bool ok = dry;
  for (int attempt = 0; attempt <= 10 && !ok; ++attempt) {
    const double factor = std::ldexp(1.0, attempt);
    const unsigned nb = (unsigned)((n * l + 255) / 256);
    if (tc == DT::F64)
      k_add_omega_t<double><<<nb, 256, 0, d.s>>>(static_cast<const double*>(Y), static_cast<double*>(Ynu), n, l, rb,
                                                 r, t, ynorm, factor, nu);
    else
      k_add_omega_t<float><<<nb, 256, 0, d.s>>>(static_cast<const float*>(Y), static_cast<float*>(Ynu), n, l, rb, r,
                                                t, ynorm, factor, nu);
    BSRHT_CUDA_TRY(cudaGetLastError());
    TRY(sketch_run(sp_y, Ynu, seed, Gc, l, sk_ws, d.s));
    if (tc == DT::F64)
      k_symmetrize<double><<<(unsigned)((l * l + 255) / 256), 256, 0, d.s>>>(static_cast<const double*>(Gc), G, l);
    else
      k_symmetrize<float><<<(unsigned)((l * l + 255) / 256), 256, 0, d.s>>>(static_cast<const float*>(Gc), G, l);
    BSRHT_CUDA_TRY(cudaGetLastError());
    note_launches(2);
    TRY(cholesky(d, G, l));
    int hs = 0;
    TRY(read_status(d, &hs));
    if (hs & kStatusNotPD) {
      BSRHT_CUDA_TRY(cudaMemsetAsync(d.status, 0, sizeof(int), d.s));
      continue;
    }
    ok = true;
  }
  if (!ok) return BSRHT_ENOTPD;
  // Step 3: Z = Y_nu C^-1 with C = L^T (so C^-1 = L^-T), into Y's buffer.
  void* Z = Y;
  if (!dry) {
    TRY(tri_inverse(d, G, LT1, Cinv, l));
    if (tc == DT::F32) TRY(cast_copy(d, DT::F64, Cinv, DT::F32, Rinv_c, l * l));
  }
  TRY(gemm_c(d, ar, tc, tc, tc, n, l, l, Ynu, l, false, tc == DT::F32 ? Rinv_c : (const void*)Cinv, l, Z, l,
             true, false));
  // Step 4: R factor of Z by CholeskyQR2; the second pass only needs its Gram.
  TRY(cholqr_pass(d, ar, dry, tc, Z, Ynu, n, l, G, LT1, Rinv, Rinv_c));
  TRY(gemm_c(d, ar, tc, tc, DT::F64, l, l, n, Ynu, l, true, Ynu, l, G, l, false, true));
  if (!dry) {
    TRY(cholesky(d, G, l));
    TRY(tri_inverse(d, G, LT2, Rinv, l));
  }
  TRY(gemm64(d, ar, l, l, l, LT2, l, false, LT1, l, R, l, true, false));
  // Step 5: SVD of R = U~ Sigma~ V~^T (Jacobi on the columns of R, i.e. rows of R^T).
  if (!dry) TRY(transpose_lower_to_upper(d, R, RT, l));
  {
    const size_t mk = ar.mark();
    TRY(jacobi_svd(d, ar, RT, l, Us, sig, Vs));
    ar.release(mk);
  }
  // Step 6: U^ = (Z V~_k) Sigma~_k^-1; step 7: Lambda = max(Sigma~_k^2 - nu, 0).
  const void* Vk = Vs;
  if (tc == DT::F32) {
    if (!dry) TRY(cast_copy(d, DT::F64, Vs, DT::F32, Vs_c, l * l));
    Vk = Vs_c;
  }
  TRY(gemm_c(d, ar, tc, tc, DT::F64, n, k, l, Z, l, false, Vk, l, U, k, false, false));
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
  if (dry) return BSRHT_OK;
  int hs = 0;
  TRY(read_status(d, &hs));
  return status_to_code(hs);
}

int validate_rsvd(const bsrht_opts& o, int64_t n, int64_t m, int k, int64_t l, int p) {
  if (o.dtype < BSRHT_F64 || o.dtype > BSRHT_F16) return BSRHT_EINVAL;
  if (n < 1 || m < 1 || k < 1 || l < k || l > m || l > n || p < 1 || p > n) return BSRHT_EINVAL;
  if (o.lda != 0 && o.lda < m) return BSRHT_EINVAL;
  return BSRHT_OK;
}

int validate_nystrom(const bsrht_opts& o, int64_t n, int k, int64_t l, int p) {
  if (o.dtype < BSRHT_F64 || o.dtype > BSRHT_F16) return BSRHT_EINVAL;
  if (n < 1 || k < 1 || l < k || l > n || p < 1 || p > n) return BSRHT_EINVAL;
  if (o.lda != 0 && o.lda < n) return BSRHT_EINVAL;
  return BSRHT_OK;
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
