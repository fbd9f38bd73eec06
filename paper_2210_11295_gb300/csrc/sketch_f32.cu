// K1 sketch instances with FP32 arithmetic: A in f32, bf16 or f16.
#include <algorithm>

#include "sketch.cuh"
#include "sketch_kernels.cuh"

namespace bsrht {
namespace {

template <typename Tin, int NT, int R2, int JM>
int launch_chunked(const SketchPlan& plan, const SketchArgs& a, void* out, int64_t ldo,
                   cudaStream_t stream) {
  using S = K1Shape<Tin, float, kW32, NT, R2, JM>;
  auto kern = k_sketch_chunked<Tin, float, kW32, NT, R2, JM>;
  const size_t smem = S::smem_bytes();
  BSRHT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<plan.G, NT, smem, stream>>>(a);
  BSRHT_CUDA_TRY(cudaGetLastError());
  note_launches(2);
  const int64_t total = a.jn * a.m;
  const float scale = (float)(1.0 / sqrt((double)plan.l));
  k_sketch_reduce<float, float, kW32><<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(
      a, static_cast<float*>(out), ldo, scale);
  BSRHT_CUDA_TRY(cudaGetLastError());
  return BSRHT_OK;
}

template <typename Tin>
int launch_typed(const SketchPlan& plan, const SketchArgs& a, void* out, int64_t ldo,
                 cudaStream_t stream) {
  if (plan.path == 1) {
    dim3 grid((unsigned)((a.m + 31) / 32), (unsigned)((a.jn + 7) / 8));
    const float scale = (float)(1.0 / sqrt((double)plan.l));
    k_sketch_small_r<Tin, float, float><<<grid, 256, 0, stream>>>(a, static_cast<float*>(out), ldo, scale);
    BSRHT_CUDA_TRY(cudaGetLastError());
    return BSRHT_OK;
  }
  switch (plan.inst) {
    case 0: return launch_chunked<Tin, 512, 1024, 32>(plan, a, out, ldo, stream);
    case 1: return launch_chunked<Tin, 512, 512, 64>(plan, a, out, ldo, stream);
    case 2: return launch_chunked<Tin, 512, 256, 64>(plan, a, out, ldo, stream);
    case 3: return launch_chunked<Tin, 128, 128, 64>(plan, a, out, ldo, stream);
    case 4: return launch_chunked<Tin, 128, 64, 64>(plan, a, out, ldo, stream);
    case 5: return launch_chunked<Tin, 128, 32, 64>(plan, a, out, ldo, stream);
    case 6: return launch_chunked<Tin, 128, 16, 64>(plan, a, out, ldo, stream);
  }
  return BSRHT_EUNSUP;
}

template <typename Tin, int NT, int R2, int JM>
int occ_of() {
  using S = K1Shape<Tin, float, kW32, NT, R2, JM>;
  auto kern = k_sketch_chunked<Tin, float, kW32, NT, R2, JM>;
  const size_t smem = S::smem_bytes();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem) != cudaSuccess) return 0;
  return occ;
}

template <typename Tin>
int occ_typed(int inst) {
  switch (inst) {
    case 0: return occ_of<Tin, 512, 1024, 32>();
    case 1: return occ_of<Tin, 512, 512, 64>();
    case 2: return occ_of<Tin, 512, 256, 64>();
    case 3: return occ_of<Tin, 128, 128, 64>();
    case 4: return occ_of<Tin, 128, 64, 64>();
    case 5: return occ_of<Tin, 128, 32, 64>();
    case 6: return occ_of<Tin, 128, 16, 64>();
  }
  return 0;
}


template <typename Tin, int NT, int R2, int JM>
int launch_grouped(const SketchGroup& grp, int G, int64_t max_out, cudaStream_t stream) {
  using S = K1Shape<Tin, float, kW32, NT, R2, JM>;
  auto kern = k_sketch_grouped<Tin, float, kW32, NT, R2, JM>;
  const size_t smem = S::smem_bytes();
  BSRHT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<G, NT, smem, stream>>>(grp);
  BSRHT_CUDA_TRY(cudaGetLastError());
  const unsigned bx = (unsigned)std::min<int64_t>((max_out + 255) / 256, 1024);
  k_sketch_reduce_grouped<float, float, kW32><<<dim3(bx, (unsigned)grp.nreq), 256, 0, stream>>>(grp);
  BSRHT_CUDA_TRY(cudaGetLastError());
  note_launches(2);
  return BSRHT_OK;
}
}  // namespace

int sketch_launch_f32(const SketchPlan& plan, const SketchArgs& a, void* out, int64_t ldo,
                      cudaStream_t stream) {
  switch (plan.dtype) {
    case BSRHT_F32: return launch_typed<float>(plan, a, out, ldo, stream);
    case BSRHT_BF16: return launch_typed<__nv_bfloat16>(plan, a, out, ldo, stream);
    case BSRHT_F16: return launch_typed<__half>(plan, a, out, ldo, stream);
  }
  return BSRHT_EINVAL;
}

int sketch_occupancy_f32(const SketchPlan& plan) {
  switch (plan.dtype) {
    case BSRHT_F32: return occ_typed<float>(plan.inst);
    case BSRHT_BF16: return occ_typed<__nv_bfloat16>(plan.inst);
    case BSRHT_F16: return occ_typed<__half>(plan.inst);
  }
  return 0;
}


namespace {
template <typename Tin>
int group_typed(const SketchPlan& plan, const SketchGroup& grp, int G, int64_t max_out, cudaStream_t stream) {
  switch (plan.inst) {
    case 0: return launch_grouped<Tin, 512, 1024, 32>(grp, G, max_out, stream);
    case 1: return launch_grouped<Tin, 512, 512, 64>(grp, G, max_out, stream);
    case 2: return launch_grouped<Tin, 512, 256, 64>(grp, G, max_out, stream);
    case 3: return launch_grouped<Tin, 128, 128, 64>(grp, G, max_out, stream);
    case 4: return launch_grouped<Tin, 128, 64, 64>(grp, G, max_out, stream);
    case 5: return launch_grouped<Tin, 128, 32, 64>(grp, G, max_out, stream);
    case 6: return launch_grouped<Tin, 128, 16, 64>(grp, G, max_out, stream);
  }
  return BSRHT_EUNSUP;
}
}  // namespace

int sketch_group_launch_f32(const SketchPlan& plan, const SketchGroup& grp, int G, int64_t max_out,
                            cudaStream_t stream) {
  switch (plan.dtype) {
    case BSRHT_F32: return group_typed<float>(plan, grp, G, max_out, stream);
    case BSRHT_BF16: return group_typed<__nv_bfloat16>(plan, grp, G, max_out, stream);
    case BSRHT_F16: return group_typed<__half>(plan, grp, G, max_out, stream);
  }
  return BSRHT_EINVAL;
}

}  // namespace bsrht
