// Internal interface of the sketch kernels (host side).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace bsrht {

// Upper bound on the sketches of one grouped launch (a kernel parameter).
constexpr int kMaxGroup = 32;

struct SketchPlan {
  int dtype = 0;      // bsrht_dtype of A
  int variant = 1;    // 1 = CUDA-core butterflies (K1), 2 = tensor cores (K2)
  int path = 0;       // 0 = chunked FWHT kernel, 1 = small-r direct kernel, 2 = TMA-fed chunked kernel,
                      // 3 = tensor-core kernel (K2, 16-bit inputs), 4 = Gaussian comparator (gaussian.cu),
                      // 5 = TMA-fed FP64 kernel with the exact integer transform (sketch_f64x.cu)
  int inst = 0;       // kernel instance id within the dtype family
  int W = 0, NT = 0, R2 = 0, JM = 0, NRL = 0;
  int64_t n = 0, m = 0, lda = 0, l = 0;
  int p = 0;
  int64_t rb = 0, r = 0;
  int64_t nch = 0;    // chunks per block
  int64_t C = 0;      // chunks per column panel (p * nch)
  int64_t P = 0;      // column panels
  int64_t T = 0;      // tiles = P * C
  int G = 0;          // CTAs of the chunked kernel (persistent, one wave)
  int paired = 0;     // TMA-fed paths: CTA pairs share panel pairs (16-bit inputs)
  int64_t jgroup = 0; // sketch rows handled per launch
  size_t smem = 0;    // dynamic shared memory per CTA
  size_t part_bytes = 0;  // partial-sum scratch (paths 2, 5 then: status word, D and Dt sign tables)
  size_t dtab_bytes = 0;  // paths 2, 5: D^(i) sign table
  size_t dttab_bytes = 0; // paths 2, 5: Dt^(i) sign table (one sketch-row group)
  size_t work_bytes = 0;  // total scratch
};

// Fills plan for the given sizes; returns a bsrht status. When
// query_device is false, no CUDA call is made and G is an upper bound.
// A (may be null) decides whether the TMA path's alignment rules hold; with
// A null the plan's work_bytes covers both the TMA and the plain path.
int sketch_make_plan(SketchPlan& plan, int dtype, int variant, int64_t n, int64_t m,
                     int64_t lda, int p, int64_t l, bool query_device, const void* A = nullptr);

// Enqueues the sketch on stream; work must hold plan.work_bytes.
int sketch_run(const SketchPlan& plan, const void* A, uint64_t seed, void* out, int64_t ldo,
               void* work, cudaStream_t stream);

int num_sms();

// Gaussian-embedding comparator (gaussian.cu): plan (path 4; part_bytes =
// the Omega_G scratch) and run.
int gaussian_plan(SketchPlan& plan, int dtype, int64_t n, int64_t m, int64_t lda, int p, int64_t l);
int gaussian_run(const SketchPlan& plan, const void* A, uint64_t seed, void* out, int64_t ldo, void* work,
                 cudaStream_t stream);
// Gaussian map on its own (gaussian.cu): out[j][k] = scale * z(j, k) for
// j < rows, k < cols (row stride ld, even; columns [cols, ld) zeroed), z the
// comparator's Philox / Box-Muller normal evaluated in the type t (F32/F64).
enum class DT;
int gaussian_omega(cudaStream_t stream, DT t, void* out, int64_t rows, int64_t cols, int64_t ld, uint64_t seed,
                   double scale);

// Autotuner: times every candidate instance on A (scratch work, output out
// of l x m) and records the fastest for the shape class; see
// bsrht_sketch_autotune.  work must hold sketch_autotune_work_bytes.
int sketch_autotune(const void* A, int dtype, int64_t n, int64_t m, int64_t lda, int p, int64_t l, void* work,
                    size_t work_bytes, void* out, cudaStream_t stream, int* choice, double* best_ms);
size_t sketch_autotune_work_bytes(int dtype, int64_t n, int64_t m, int64_t lda, int p, int64_t l);
void sketch_autotune_reset();

// Grouped launches: several sketches of one dtype family in one persistent
// launch of the chunked kernel.  The plan is the plain-kernel plan of the
// sizes; EUNSUP if they need more than one sketch-row group.
int sketch_make_plan_grouped(SketchPlan& plan, int dtype, int64_t n, int64_t m, int64_t lda, int p, int64_t l);
// Scratch of one sketch inside a grouped launch.
size_t sketch_group_work_bytes(const SketchPlan& plan);
// Enqueues nreq (<= kMaxGroup) sketches with equal dtype and kernel
// instance; outs[q] is l x m row-major, works[q] holds
// sketch_group_work_bytes(*plans[q]).
int sketch_group_run(const SketchPlan* const* plans, const void* const* A, const uint64_t* seeds, void* const* outs,
                     void* const* works, int nreq, cudaStream_t stream);

}  // namespace bsrht

namespace bsrht {

// Kernel instances of the chunked CUDA-core sketch (K1).
struct K1Inst {
  int NT, R2, JM;
};
// FP32 arithmetic (A in f32 / bf16 / f16), panels of 32 columns.
constexpr int kW32 = 32;
constexpr K1Inst kInstF32[] = {{512, 1024, 32}, {512, 512, 64}, {512, 256, 64}, {128, 128, 64},
                               {128, 64, 64},   {128, 32, 64},  {128, 16, 64}};
// FP64 arithmetic, panels of 16 columns (128-byte rows).
constexpr int kW64 = 16;
constexpr K1Inst kInstF64[] = {{512, 1024, 16}, {256, 512, 16}, {256, 256, 32}, {128, 128, 32},
                               {128, 64, 32}};

struct SketchArgs;
struct SketchGroup;
// Per-family launchers (sketch_f32.cu / sketch_f64.cu).
int sketch_group_launch_f32(const SketchPlan& plan, const SketchGroup& grp, int G, int64_t max_out,
                            cudaStream_t stream);
int sketch_group_launch_f64(const SketchPlan& plan, const SketchGroup& grp, int G, int64_t max_out,
                            cudaStream_t stream);
int sketch_launch_f32(const SketchPlan& plan, const SketchArgs& a, void* out, int64_t ldo,
                      cudaStream_t stream);
int sketch_launch_f64(const SketchPlan& plan, const SketchArgs& a, void* out, int64_t ldo,
                      cudaStream_t stream);
int sketch_occupancy_f32(const SketchPlan& plan);
int sketch_occupancy_f64(const SketchPlan& plan);
// TMA-fed path (sketch_tma.cu): W = 32, NT = 512, R2 = 512, JM in {32, 48, 64}.
int sketch_occupancy_tma(const SketchPlan& plan);
int sketch_launch_tma(const SketchPlan& plan, const SketchArgs& a, void* out, int64_t ldo, int* err,
                      uint64_t* dtab, uint64_t* dttab, cudaStream_t stream);
// FP64 path with the exact integer transform (sketch_f64x.cu): W = 16,
// NT = 512, R2 = 512, JM (sketch rows per thread) in {8, 16}.
int sketch_occupancy_f64x(const SketchPlan& plan);
int sketch_launch_f64x(const SketchPlan& plan, const SketchArgs& a, void* out, int64_t ldo, int* err,
                       uint64_t* dtab, uint64_t* dttab, cudaStream_t stream);
// Tensor-core path (sketch_tc.cu, K2): BF16 / F16, W = 32, R2 = 512.
int sketch_occupancy_tc(const SketchPlan& plan);
int sketch_launch_tc(const SketchPlan& plan, const SketchArgs& a, void* out, int64_t ldo, int* err,
                     cudaStream_t stream);

}  // namespace bsrht
