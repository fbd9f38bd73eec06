// K1 sketch instances with FP64 arithmetic (A in f64).
#include <algorithm>

#include "sketch.cuh"
#include "sketch_kernels.cuh"

namespace bsrht {
namespace {

template <int NT, int R2, int JM>
int launch_chunked(const SketchPlan& plan, const SketchArgs& a, void* out, int64_t ldo,
                   cudaStream_t stream) {
  using S = K1Shape<double, double, kW64, NT, R2, JM>;
  auto kern = k_sketch_chunked<double, double, kW64, NT, R2, JM>;
  const size_t smem = S::smem_bytes();
  BSRHT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<plan.G, NT, smem, stream>>>(a);
  BSRHT_CUDA_TRY(cudaGetLastError());
  note_launches(2);
  const int64_t total = a.jn * a.m;
  const double scale = 1.0 / sqrt((double)plan.l);
  k_sketch_reduce<double, double, kW64><<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(
      a, static_cast<double*>(out), ldo, scale);
  BSRHT_CUDA_TRY(cudaGetLastError());
  return BSRHT_OK;
}

template <int NT, int R2, int JM>
int occ_of() {
  using S = K1Shape<double, double, kW64, NT, R2, JM>;
  auto kern = k_sketch_chunked<double, double, kW64, NT, R2, JM>;
  const size_t smem = S::smem_bytes();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem) != cudaSuccess) return 0;
  return occ;
}


template <int NT, int R2, int JM>
int launch_grouped(const SketchGroup& grp, int G, int64_t max_out, cudaStream_t stream) {
  using S = K1Shape<double, double, kW64, NT, R2, JM>;
  auto kern = k_sketch_grouped<double, double, kW64, NT, R2, JM>;
  const size_t smem = S::smem_bytes();
  BSRHT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<G, NT, smem, stream>>>(grp);
  BSRHT_CUDA_TRY(cudaGetLastError());
  const unsigned bx = (unsigned)std::min<int64_t>((max_out + 255) / 256, 1024);
  k_sketch_reduce_grouped<double, double, kW64><<<dim3(bx, (unsigned)grp.nreq), 256, 0, stream>>>(grp);
  BSRHT_CUDA_TRY(cudaGetLastError());
  note_launches(2);
  return BSRHT_OK;
}
}  // namespace

int sketch_launch_f64(const SketchPlan& plan, const SketchArgs& a, void* out, int64_t ldo,
                      cudaStream_t stream) {
  if (plan.dtype != BSRHT_F64) return BSRHT_EINVAL;
  if (plan.path == 1) {
    dim3 grid((unsigned)((a.m + 31) / 32), (unsigned)((a.jn + 7) / 8));
    const double scale = 1.0 / sqrt((double)plan.l);
    k_sketch_small_r<double, double, double><<<grid, 256, 0, stream>>>(a, static_cast<double*>(out), ldo, scale);
    BSRHT_CUDA_TRY(cudaGetLastError());
    return BSRHT_OK;
  }
  switch (plan.inst) {
    case 0: return launch_chunked<512, 1024, 16>(plan, a, out, ldo, stream);
    case 1: return launch_chunked<256, 512, 16>(plan, a, out, ldo, stream);
    case 2: return launch_chunked<256, 256, 32>(plan, a, out, ldo, stream);
    case 3: return launch_chunked<128, 128, 32>(plan, a, out, ldo, stream);
    case 4: return launch_chunked<128, 64, 32>(plan, a, out, ldo, stream);
  }
  return BSRHT_EUNSUP;
}

int sketch_occupancy_f64(const SketchPlan& plan) {
  switch (plan.inst) {
    case 0: return occ_of<512, 1024, 16>();
    case 1: return occ_of<256, 512, 16>();
    case 2: return occ_of<256, 256, 32>();
    case 3: return occ_of<128, 128, 32>();
    case 4: return occ_of<128, 64, 32>();
  }
  return 0;
}


int sketch_group_launch_f64(const SketchPlan& plan, const SketchGroup& grp, int G, int64_t max_out,
                            cudaStream_t stream) {
  if (plan.dtype != BSRHT_F64) return BSRHT_EINVAL;
  switch (plan.inst) {
    case 0: return launch_grouped<512, 1024, 16>(grp, G, max_out, stream);
    case 1: return launch_grouped<256, 512, 16>(grp, G, max_out, stream);
    case 2: return launch_grouped<256, 256, 32>(grp, G, max_out, stream);
    case 3: return launch_grouped<128, 128, 32>(grp, G, max_out, stream);
    case 4: return launch_grouped<128, 64, 32>(grp, G, max_out, stream);
  }
  return BSRHT_EUNSUP;
}

}  // namespace bsrht
