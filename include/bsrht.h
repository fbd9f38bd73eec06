/*
 * bsrht.h - C ABI of the block SRHT sketching library (sm_103a, one GPU).
 *
 * Method: Balabanov, Beaupere, Grigori, Lederer, "Block subsampled randomized
 * Hadamard transform for low-rank approximation on distributed
 * architectures".  Orientation used by every call: A is n x m and tall, the
 * sketching matrix Omega is l x n, and the sketch is B = Omega A (l x m).
 * The paper writes the same quantities for the transposed m x n matrix, so
 * its Y = A Omega^T is B^T here.
 *
 * Omega (Sec. 2, eq. 2.3) = [Omega^(1) ... Omega^(p)],
 *   Omega^(i) = sqrt(r/l) Dt^(i) R H D^(i),
 * with one sampling matrix R (uniform, with replacement) shared by all p
 * blocks, independent Rademacher diagonals D^(i) (r x r) and Dt^(i) (l x l),
 * and H the r x r Walsh-Hadamard matrix (Sylvester/natural order) scaled by
 * 1/sqrt(r); every entry of Omega is +-1/sqrt(l).  Block i holds rows
 * [i*rb, min(n,(i+1)*rb)) of A with rb = ceil(n/p); r is the next power of
 * two >= rb and the missing rows count as zero (the partial SRHT / zero
 * padding of Sec. 2).
 *
 * Randomness: Philox4x64-10 (Salmon et al., SC'11) with key (seed, 0).
 *   D^(i)_kk  : counter (k>>8, i, 0, 0), output word (k>>6)&3, bit k&63
 *   Dt^(i)_jj : counter (j>>8, i, 1, 0), output word (j>>6)&3, bit j&63
 *               (a set bit means -1)
 *   R row j   : counter (j>>2, 0, 2, 0), output word j&3, s_j = word mod r
 * so a given (seed, n, p, l) defines the same Omega on every device.
 *
 * Memory: every matrix is row-major.  Unless noted, pointers are DEVICE
 * pointers owned by the caller; the library never frees them and never
 * writes to A.  Calls are asynchronous and stream-ordered on opts->stream
 * (NULL = the legacy default stream); a non-zero return means nothing was
 * enqueued, except BSRHT_ECUDA (a launch failed) and the numerical statuses
 * of bsrht_rsvd / bsrht_nystrom, which are read back on the stream and so
 * make those two calls synchronous with it.
 *
 * Scratch: if opts->workspace is NULL the library allocates scratch from its
 * own per-device pool (cudaMalloc, kept for reuse, released by
 * bsrht_release_pool); otherwise it uses the caller's buffer, which must hold
 * at least the bytes that the matching *_workspace query reports.
 */
#ifndef BSRHT_H_
#define BSRHT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes (0 = success, negative = failure) ------------------- */
#define BSRHT_OK 0
#define BSRHT_EINVAL (-22)     /* bad size, pointer, dtype, stride or option   */
#define BSRHT_ENOMEM (-12)     /* scratch allocation failed / workspace short  */
#define BSRHT_EUNSUP (-95)     /* valid but unsupported combination            */
#define BSRHT_ETIMEDOUT (-110) /* a bounded wait gave up                       */
#define BSRHT_ENOTPD (-1001)   /* a Gram or core matrix numerically singular
                                  where no remedy applies (e.g. the Nystrom
                                  sketch A Omega^T is zero, or Phi Q / Psi P of
                                  Algorithm 3 lose rank)                        */
#define BSRHT_ENOCONV (-1002)  /* Jacobi SVD hit its sweep limit               */
#define BSRHT_ECUDA (-1003)    /* a CUDA runtime call or launch failed          */

/* ---- element types of A ----------------------------------------------- */
typedef enum bsrht_dtype {
  BSRHT_F64 = 0,  /* double: sketch computed and returned in FP64           */
  BSRHT_F32 = 1,  /* float : FP32 arithmetic, FP32 sketch                   */
  BSRHT_BF16 = 2, /* bfloat16 storage, FP32 arithmetic, FP32 sketch         */
  BSRHT_F16 = 3   /* IEEE half storage, FP32 arithmetic, FP32 sketch        */
} bsrht_dtype;

/* ---- kernel variant of the sketch ------------------------------------- */
typedef enum bsrht_variant {
  BSRHT_VARIANT_AUTO = 0,     /* library choice                             */
  BSRHT_VARIANT_CUDACORE = 1, /* radix-2 butterflies on CUDA cores (K1)     */
  BSRHT_VARIANT_TENSOR = 2,   /* Kronecker H16 factors on tensor cores (K2)  */
  BSRHT_VARIANT_GAUSSIAN = 3  /* not a block SRHT: the Gaussian embedding the
                                 paper compares against (Sec. 4), see below  */
} bsrht_variant;

/*
 * BSRHT_VARIANT_GAUSSIAN (bsrht_sketch, bsrht_rsvd; BSRHT_F32 only, n >= 8;
 * bsrht_nystrom returns BSRHT_EUNSUP): Omega is replaced by Omega_G (l x n)
 * with independent N(0, 1/l) entries -- the comparator of Sec. 4, where the
 * paper reports the same approximation quality and a block SRHT up to 2.5x
 * faster to apply.  p is validated but unused.  Entries: Philox4x64-10 with
 * key (seed, 0) and counter (k>>1, j, 3, 0) for row j, column k (words 0, 1
 * for even k, 2, 3 for odd k); a word w gives u = (2 (w >> 41) + 1) 2^-24 and
 * the pair (u1, u2) gives z = sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller,
 * evaluated in FP32); the entry is z / sqrt(l).  B = Omega_G A is a dense
 * product (2 l n m flops, tcgen05 tensor cores at FP32 accuracy); its
 * scratch holds Omega_G and a transposed, TF32-split copy of A (about
 * 4 l n + 8 n m bytes; the *_workspace queries report it).  The product's
 * waits are bounded: a tile whose wait gives up is written as NaN (the
 * low-rank calls see it in their status word and return BSRHT_ETIMEDOUT).
 */

/* ---- arithmetic precision ---------------------------------------------- */
typedef enum bsrht_precision {
  BSRHT_PREC_AUTO = 0, /* the arithmetic the dtype names (bsrht_dtype)        */
  BSRHT_PREC_F64 = 1   /* FP64 arithmetic on FP32 storage (bsrht_sketch and
                          bsrht_nystrom only; a no-op for BSRHT_F64 data):
                          the sketch is the exact integer Walsh-Hadamard
                          transform of the FP32 values widened to FP64 (the
                          FP64 kernel), written in FP64, and everything after
                          it runs as for FP64 data.  A is still read as FP32
                          (half the bytes of FP64 storage).  Needs blocks of
                          at least 512 rows (r >= 512) and 16-byte aligned
                          rows; otherwise, and for 16-bit data, any variant
                          but AUTO / CUDACORE and the other calls:
                          BSRHT_EUNSUP.                                        */
} bsrht_precision;

typedef struct bsrht_opts {
  int32_t dtype;          /* bsrht_dtype of A                                */
  int32_t variant;        /* bsrht_variant                                   */
  int64_t lda;            /* elements between consecutive rows of A; 0 means
                             the row length (m, or n for bsrht_nystrom)      */
  void* stream;           /* cudaStream_t, NULL = legacy default stream      */
  void* workspace;        /* device scratch or NULL (library pool)           */
  size_t workspace_bytes; /* size of opts->workspace in bytes                */
  int32_t precision;      /* bsrht_precision                                 */
} bsrht_opts;

/* Fills *opts with dtype F64, variant AUTO, lda 0, NULL stream/workspace,
 * precision AUTO. */
void bsrht_opts_init(bsrht_opts* opts);

/* Short English description of a status code (static storage). */
const char* bsrht_strerror(int status);

/*
 * bsrht_sketch - B = Omega A (eq. 2.3 applied as the block sum of eq. 2.4).
 *   A    : n x m, row stride opts->lda (>= m), element type opts->dtype.
 *   n, m : n >= 1, m >= 0.  p: number of blocks, 1 <= p <= n.
 *   l    : sketch rows, 1 <= l <= n (Thm 2.1 assumes n >= l); l > r is
 *          allowed because R samples with replacement.
 *   out  : l x m, row stride m; double for BSRHT_F64 input or precision
 *          BSRHT_PREC_F64, float otherwise.
 * One pass over A: Philox signs, the Walsh-Hadamard butterflies, the row
 * sample and the sum over the p blocks all run inside the kernels; the block
 * sum is reduced in a fixed order, so repeated calls give identical bits.
 * Returns BSRHT_EINVAL on bad arguments (nothing enqueued).
 */
int bsrht_sketch(const void* A, int64_t n, int64_t m, int32_t p, int64_t l,
                 uint64_t seed, void* out, const bsrht_opts* opts);

/* Scratch bytes bsrht_sketch needs for these sizes (host only, no GPU work). */
int bsrht_sketch_workspace(int64_t n, int64_t m, int32_t p, int64_t l,
                           const bsrht_opts* opts, size_t* bytes);

/*
 * bsrht_sketch_noalloc - bsrht_sketch for callers that cannot allocate
 * device memory.  The paper has no counterpart; this is a deployment aid.
 * Some callers may not call cudaMalloc at all: a host whose own caching
 * allocator must account for every device byte, a loop that may not block on
 * the implicit device synchronisation an allocation can cause, or a plug-in
 * whose host application owns all device memory.  They still pass A and out
 * exactly as for bsrht_sketch (same arguments, same result bits), but the
 * sketch's scratch comes from one fixed 32 MiB array that the library keeps
 * in device memory on every device that loads it, until the process exits.
 *   - opts->workspace is ignored; nothing is allocated or freed.
 *   - Returns BSRHT_ENOMEM, with nothing enqueued, when the sizes need more
 *     than 32 MiB of scratch (bsrht_sketch_workspace reports the need;
 *     n = 2^20, m = 4096, l = 512 needs about 19 MB in FP32, 27 MB in FP64).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls on one device share the array: calls whose kernels overlap on
 *     the GPU (other streams, other host threads) race and corrupt each
 *     other's results, so serialise them on one stream.  The array keeps the
 *     last call's contents; the sketch overwrites every slot it reads and
 *     clears its status word at the start of each call.
 */
int bsrht_sketch_noalloc(const void* A, int64_t n, int64_t m, int32_t p,
                         int64_t l, uint64_t seed, void* out,
                         const bsrht_opts* opts);

/*
 * bsrht_rsvd - rank-k randomized SVD, Algorithm 1 of Sec. 3.1, on the sketch.
 *   A (n x m) ~ U diag(S) V^T with U n x k, S k (descending), V m x k, all
 *   double, U and V with orthonormal columns.  Requires 1 <= k <= l <= m and
 *   l <= n.  Steps: B = Omega A; Q = an orthonormal basis of range(B^T), FP64
 *   and rank revealing: m x l' with l' <= l the number of singular values of
 *   B above l 2^-44 sigma_1 (l times the relative precision of the FP64
 *   sketch) (CholeskyQR2 when B is well conditioned, else
 *   Householder QR and a Jacobi SVD of its R factor; l' < l when Omega
 *   repeats a row up to sign in every block, which sampling with replacement
 *   allows, or when rank(A) < l); W = A Q (second pass over A, in the
 *   arithmetic of A: FP64 for F64, FP32 otherwise); W = P R (CholeskyQR2;
 *   Householder QR for ill-conditioned FP64 W up to 2^17 rows, else an
 *   eigen-based basis); SVD of R^T (one-sided Jacobi);
 *   U = P V~_k, S = Sigma~_k, V = Q U~_k.  If l' < k the trailing k - l'
 *   singular values and the matching columns of U and V are zero.  Each
 *   column of U is flipped so its largest-magnitude entry is positive (V gets
 *   the same flip).
 *   Synchronises opts->stream to read the status of the small factorizations;
 *   returns BSRHT_ENOTPD if a Gram matrix is numerically singular,
 *   BSRHT_ENOCONV if the Jacobi SVD does not converge, BSRHT_ETIMEDOUT if a
 *   tensor-core product gave up one of its bounded waits.
 */
int bsrht_rsvd(const void* A, int64_t n, int64_t m, int32_t k, int64_t l,
               int32_t p, uint64_t seed, double* U, double* S, double* V,
               const bsrht_opts* opts);

int bsrht_rsvd_workspace(int64_t n, int64_t m, int32_t k, int64_t l, int32_t p,
                         const bsrht_opts* opts, size_t* bytes);

/*
 * bsrht_srsvd - rank-k single-view randomized SVD, Algorithm 3 of Sec. 3.3:
 * every sketch of A is a linear function of A alone (no second product with
 * a basis, unlike Algorithm 1), so A could be streamed once.
 *   A (n x m, BSRHT_F64 or BSRHT_F32, row stride opts->lda) ~ U diag(S) V^T,
 *   U n x k, S k (descending), V m x k, all double, orthonormal columns.
 *   Requires 1 <= k <= l <= s <= min(n, m), 1 <= p <= n; variant AUTO or
 *   CUDACORE (BSRHT_EUNSUP otherwise and for 16-bit A).
 * In the paper's orientation A_p = A^T (m x n).  Sketching maps: block
 * SRHTs (eq. 2.3, the same Philox rules as bsrht_sketch) Omega (l x n,
 * p blocks, key seed), Phi (s x m, one block, key seed+2), Psi (s x n,
 * p blocks, key seed+3); Gamma (l x m, key seed+1) is the Gaussian map of
 * BSRHT_VARIANT_GAUSSIAN evaluated in FP64 (an SRHT sample of l rows out of
 * r ~ m repeats rows and would make X rank deficient).  Steps:
 * Y = A_p Omega^T, X = A_p^T Gamma^T = A Gamma^T, Z = Phi A_p Psi^T (A Phi^T
 * through an on-device transpose of A: scratch n m size(A) bytes);
 * Q = orth(Y) (FP64, rank revealing as in bsrht_rsvd: m x rq),
 * P = orth(X) (FP64 data: rank revealing, n x rp; FP32: rank-robust
 * CholeskyQR2, rp = l); C = (Phi Q)^+ Z ((Psi P)^T)^+ (rq x rp) by the
 * normal equations of the well-conditioned Phi Q and Psi P; C = U~ S~ V~^T
 * (FP64 Jacobi on C in a zero-padded square frame); U = P V~_k, S = S~_k,
 * V = Q U~_k (signs as bsrht_rsvd; zero beyond min(rq, rp)).
 * Synchronises opts->stream like bsrht_rsvd; BSRHT_ENOTPD if Phi Q or Psi P
 * is numerically rank deficient, BSRHT_ETIMEDOUT as for bsrht_rsvd.
 */
int bsrht_srsvd(const void* A, int64_t n, int64_t m, int32_t k, int64_t l,
                int64_t s, int32_t p, uint64_t seed, double* U, double* S,
                double* V, const bsrht_opts* opts);

int bsrht_srsvd_workspace(int64_t n, int64_t m, int32_t k, int64_t l, int64_t s,
                          int32_t p, const bsrht_opts* opts, size_t* bytes);

/*
 * bsrht_nystrom - rank-k randomized Nystrom approximation, Algorithm 2 of
 * Sec. 3.2, of a symmetric positive semi-definite n x n matrix A (row stride
 * opts->lda >= n; symmetry is assumed, not checked).
 *   A ~ U diag(Lambda) U^T with U n x k (orthonormal columns), Lambda k
 *   (descending, >= 0), both double.  Requires 1 <= k <= l <= n.
 *   Steps: Y = (Omega A)^T; shift nu = sqrt(n) 2^-52 ||Y||_F,
 *   Y_nu = Y + nu Omega^T; core = sym(Omega Y_nu) and its Cholesky factor C
 *   in FP64 (Remark 3.1); if the factorization fails or its squared pivots
 *   fall below l*eps of the largest (eps of the arithmetic of A), C^-1 is
 *   replaced by the SVD square root's pseudo-inverse (Remark 3.1);
 *   Z = Y_nu C^-1; R factor of Z (CholeskyQR2, rank-robust); SVD
 *   R = U~ Sigma~ V~^T; U = Z V~_k Sigma~_k^-1; Lambda = max(Sigma~_k^2 - nu, 0).
 *   With BSRHT_F32 data and opts->precision = BSRHT_PREC_F64, Y is the FP64
 *   sketch of the FP32 values and every step after it runs in FP64 (eps
 *   2^-52): the result of the same matrix stored in FP64.
 *   Synchronises opts->stream; status codes as for bsrht_rsvd.
 */
int bsrht_nystrom(const void* A, int64_t n, int32_t k, int64_t l, int32_t p,
                  uint64_t seed, double* U, double* Lambda,
                  const bsrht_opts* opts);

int bsrht_nystrom_workspace(int64_t n, int32_t k, int64_t l, int32_t p,
                            const bsrht_opts* opts, size_t* bytes);

/*
 * bsrht_nystrom_rbf - bsrht_nystrom on the kernel matrix of a point set,
 * without storing the matrix (Sec. 4.1 applies Algorithm 2 to such RBF
 * kernel matrices; step 1 only needs Omega A, which is built from column
 * panels of A):
 *   A_ij = exp(-|x_i - x_j|^2 / (2 h^2)),  x_i the rows of X.
 *   X    : device, n x dim, FP32, row stride opts->lda (0 = dim; a multiple
 *          of 4, X 16-byte aligned: BSRHT_EUNSUP otherwise); h > 0.
 *   opts->dtype must be BSRHT_F32 (the matrix is formed in FP32 arithmetic).
 * Each panel of about 2^28 entries (a multiple of 64 columns) is formed as
 * the Gram of the points on the tensor cores (FP32 accuracy: three TF32
 * products), mapped through the exponential in FP32 (the diagonal is
 * exactly 1), and sketched into Omega A before the next panel is formed;
 * steps 1b-7 are those of bsrht_nystrom (same shift, thresholds, status
 * codes; synchronous with opts->stream).  A panel holds n * w FP32 values
 * of scratch, reported by bsrht_nystrom_rbf_workspace, instead of the n x n
 * matrix.  Entries differ from a stored FP32 kernel matrix by rounding (A is
 * symmetric to FP32 accuracy, not bitwise).
 */
int bsrht_nystrom_rbf(const float* X, int64_t n, int64_t dim, double h,
                      int32_t k, int64_t l, int32_t p, uint64_t seed,
                      double* U, double* Lambda, const bsrht_opts* opts);

int bsrht_nystrom_rbf_workspace(int64_t n, int64_t dim, int32_t k, int64_t l,
                                int32_t p, const bsrht_opts* opts,
                                size_t* bytes);

/* Frees the library's scratch pool on the current device (no-op if empty).
 * The caller must make sure no call that uses the pool is still running. */
int bsrht_release_pool(void);

/* Stage tracing of bsrht_sketch / bsrht_rsvd / bsrht_nystrom for the calling
 * host thread: when enabled, each call records CUDA events between its stages
 * on its stream (sketch, orthogonalisation of the sketch, second pass, tall
 * QR, small SVD, output factors; Nystrom: sketch, core, Z, tall QR, small
 * SVD, factors; inside a sketch on the TMA / tensor-core kernels:
 * sketch_tables, sketch_kernel, sketch_reduce, i.e. the sign tables, the
 * transform kernel and the block-sum reduce, each timed on its own).
 * bsrht_profile_stages waits for those events and returns up to
 * cap stage names (32 bytes each, NUL-terminated, in names) and durations in
 * milliseconds (ms); *count receives the number of stages of the last call. */
int bsrht_profile_enable(int on);
int bsrht_profile_stages(char* names, double* ms, int cap, int* count);

/* Number of CUDA kernels the library has launched in this process (all
 * devices, all threads).  Diagnostic counter for benchmarks and tests. */
uint64_t bsrht_kernel_launches(void);

/* Library version, e.g. "0.1.0" (static storage). */
const char* bsrht_version(void);

/* ---- sketch autotuner -------------------------------------------------
 * Times every kernel instance that can run the sketch of these sizes (the
 * TMA-fed kernel and the chunked kernels with each chunk length R2 <= r,
 * i.e. tile shape and FWHT split) on A itself, two runs each after one
 * warm-up, with CUDA events on opts->stream, and records the fastest for the
 * shape class (dtype, r, ceil(log2 m), l <= 512 or not, TMA-compatible rows).
 * Later plans of that class (bsrht_sketch, the *_workspace queries, the
 * server) use the recorded choice.  Writes only library scratch; A is read.
 * *choice: the instance picked (-1 = the TMA-fed kernel, else the chunked
 * instance index); *best_ms: its time.  Synchronous with opts->stream.
 * Returns EINVAL on bad sizes, ENOMEM if scratch cannot be allocated.      */
int bsrht_sketch_autotune(const void* A, int64_t n, int64_t m, int32_t p, int64_t l, const bsrht_opts* opts,
                          int32_t* choice, double* best_ms);
/* Forgets every recorded choice (plans fall back to the built-in rules).   */
int bsrht_sketch_autotune_reset(void);

/* ---- serving loop -----------------------------------------------------
 * A server owns a device pool of hbm_budget bytes for request scratch and a
 * set of executor threads, each with its own CUDA stream.  Requests (sketch,
 * Algorithm 1 RSVD, Algorithm 2 Nystrom) are submitted at any time and run
 * as soon as an executor is free and their scratch fits in the free part of
 * the pool (first fit; requests that fit may pass one that does not yet, up
 * to a bounded number of times, so a large request is not starved).  Work of
 * different requests overlaps on the device through the executors' streams.
 * Small sketches (too few tiles to fill the GPU alone) of the same kernel
 * instance are packed, up to max_group at a time, into one persistent
 * grouped FWHT launch; sketch launches are replayed from captured CUDA
 * graphs (one executable graph per shape, updated in place for new
 * pointers).  A and all outputs are caller-owned device buffers that must
 * stay valid until the request completes; the server never writes to A.
 * The executors' streams are not ordered after the caller's streams: A must
 * be completely written (its producer synchronized) before bsrht_submit,
 * and the outputs may be read once bsrht_poll / bsrht_wait report the
 * request done.
 * Latency = submit to observed completion on the host.                     */
typedef struct bsrht_server bsrht_server;

typedef enum bsrht_request_kind {
  BSRHT_REQ_SKETCH = 0,  /* out = Omega A (l x m; F64 if A is F64, else F32) */
  BSRHT_REQ_RSVD = 1,    /* U (n x k), S (k), V (m x k), FP64 (bsrht_rsvd)  */
  BSRHT_REQ_NYSTROM = 2  /* U (n x k), S = Lambda (k), FP64; A is n x n     */
} bsrht_request_kind;

typedef struct bsrht_request {
  int32_t kind;     /* bsrht_request_kind                                  */
  int32_t dtype;    /* bsrht_dtype of A                                    */
  const void* A;    /* device, n x m row-major (n x n for Nystrom)         */
  int64_t n, m;     /* m is ignored for Nystrom                            */
  int64_t lda;      /* 0 = dense rows                                      */
  int32_t p;        /* number of blocks                                    */
  int32_t k;        /* target rank (RSVD, Nystrom)                         */
  int64_t l;        /* sketch rows                                         */
  uint64_t seed;
  void* out;        /* sketch output                                       */
  double* U;
  double* S;        /* singular values (RSVD) or Lambda (Nystrom)          */
  double* V;        /* RSVD only                                           */
  int32_t precision;/* bsrht_precision (sketch, Nystrom)                    */
} bsrht_request;

typedef struct bsrht_server_opts {
  size_t hbm_budget;      /* bytes of the scratch pool (cudaMalloc'ed once) */
  int32_t executors;      /* executor threads / streams (default 4)         */
  int32_t max_group;      /* sketches per grouped launch, 1..32 (default 16)*/
  int32_t use_graphs;     /* replay sketch launches from CUDA graphs (1)    */
  int32_t autotune;       /* autotune each new sketch shape class (1)       */
  int64_t exec_timeout_ms;/* bounded wait of an executor for its work; on
                             expiry the request fails with ETIMEDOUT and its
                             scratch stays reserved (default 600000)         */
} bsrht_server_opts;

typedef struct bsrht_server_stats {
  int64_t submitted, completed, failed, pending;
  int64_t grouped_launches;  /* grouped FWHT launches                       */
  int64_t grouped_requests;  /* sketches that ran inside them               */
  int64_t graph_launches;    /* launches replayed from CUDA graphs          */
  int64_t tuned_classes;     /* shape classes the server autotuned          */
  double p50_ms, p99_ms, mean_ms, max_ms;  /* latency of completed requests */
  size_t pool_high_bytes;    /* high-water mark of the scratch pool         */
} bsrht_server_stats;

void bsrht_server_opts_init(bsrht_server_opts* o);
/* Server with default options and the given budget on the current device. */
int bsrht_server_create(size_t hbm_budget, bsrht_server** out);
int bsrht_server_create_ex(const bsrht_server_opts* o, bsrht_server** out);
/* Validates and queues a request; *ticket identifies it.  EINVAL on bad
 * arguments, ENOMEM if its scratch exceeds the whole budget.               */
int bsrht_submit(bsrht_server* s, const bsrht_request* r, uint64_t* ticket);
/* *done = 1 once the request finished; the return value is then its status
 * (BSRHT_OK or the library status of the call), else BSRHT_OK with *done = 0.
 * EINVAL for an unknown ticket.                                            */
int bsrht_poll(bsrht_server* s, uint64_t ticket, int* done);
/* Blocks until the request finished or timeout_us elapsed: its status, or
 * ETIMEDOUT (the request keeps running).                                   */
int bsrht_wait(bsrht_server* s, uint64_t ticket, int64_t timeout_us);
int bsrht_server_stats_get(bsrht_server* s, bsrht_server_stats* out);
/* Submit and completion times of a request in seconds of the host's
 * monotonic clock (CLOCK_MONOTONIC); *done_s = -1 while it is pending.     */
int bsrht_request_times(bsrht_server* s, uint64_t ticket, double* submit_s, double* done_s);
/* Lets queued and running requests finish, joins the executors, frees the
 * pool and the graphs.  The server must not be used afterwards.            */
int bsrht_server_destroy(bsrht_server* s);

/* Host-only self-test of the server's first-fit pool allocator (no GPU):
 * random allocate / free sequences checked against a reference model.
 * Returns 0 when every invariant held, else the number of violations.     */
int bsrht_selftest_pool_allocator(uint64_t seed, int32_t steps);

#ifdef __cplusplus
} /* extern "C" */
#endif

#endif /* BSRHT_H_ */
