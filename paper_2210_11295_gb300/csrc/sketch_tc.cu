// Block SRHT sketch, tensor-core variant (K2) for 16-bit inputs (BF16, FP16).
//
// Same result as the K1 kernels (eq. 2.3-2.4, R2 = 512-row chunks, the outer
// Kronecker factor collapsed to a sign per sampled row), with the chunk
// transform split by the tensor form of H (Sec. 2):
//     H_512 = H_4 (x) H_128,   H_128 = H_8 (x) H_16,
// and H_128 applied on the tensor cores as one dense +-1 operand: per
// 128-row block of the chunk, D = H_128 X_blk (M = 128, N = 32 columns,
// K = 128) with tcgen05.mma kind::f16.  +-1 and the 16-bit inputs are exact
// in the operand type and the products accumulate in FP32 in TMEM, so the
// result is the FP32 transform of the stored values.  The remaining H_4
// across the four blocks, the sampled rows and their signs run on the CUDA
// cores as in K1.
//
// Per chunk (32 columns of one panel): a TMA load into a 2-stage ring; all
// threads apply the D^(i) signs while transposing the chunk into the
// K-major, 128-byte-swizzled B operand; one thread issues 32 MMAs (4 blocks
// x 8 K-steps of 16) into a double-buffered TMEM accumulator; the previous
// chunk's accumulator is read back (tcgen05.ld), combined by the radix-4
// stage into an FP32 tile and gathered into per-thread accumulators while
// the tensor cores work on the current one.  Waits are bounded; on a failed
// wait the CTA raises the error word (the reduce then writes NaN), drains
// its copies and MMAs and frees TMEM.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "gemm_tc.cuh"
#include "sketch.cuh"
#include "sketch_kernels.cuh"
#include "tma.cuh"

namespace bsrht {
namespace {

constexpr uint32_t kTcWait = 1u << 22;

constexpr int kW = 32, kNT = 512, kR2 = 512, kNRL = 16;
constexpr int kTStride = 36;                       // FP32 tile row stride (floats): conflict-free float4 stores
constexpr uint32_t kHBytes = 2 * 128 * 128;        // H_128, 16-bit, K-major SW128 (2 K-blocks of 64)
constexpr uint32_t kBtBytes = 8 * kW * 128;        // chunk^T: 8 K-blocks x 32 rows x 128 B
constexpr uint32_t kXBytes = kR2 * kW * 2;         // one staged chunk (row-major, 64-byte rows)
constexpr uint32_t kTBytes = kR2 * kTStride * 4;   // FP32 transform of the chunk
constexpr uint32_t kTmemCols = 256;                // 2 buffers x 4 blocks x 32 columns

template <int JM>
struct TcShape {
  static constexpr int JG = JM * kNRL;
  static constexpr size_t meta_bytes = 2 * 4 * (size_t)JG + 2 * 8 * 8 + 8 * 8 + 16;
  static constexpr size_t smem_bytes() {
    return 1024 + kHBytes + kBtBytes + 2 * (size_t)kXBytes + kTBytes + meta_bytes;
  }
};

template <typename Tin>
constexpr uint32_t idesc_16() {
  // D FP32, A = B = F16 (0) or BF16 (1), both K-major, N = 32, M = 128.
  constexpr uint32_t f = sizeof(Tin) == 2 && std::is_same<Tin, __nv_bfloat16>::value ? 1u : 0u;
  return (1u << 4) | (f << 7) | (f << 10) | ((uint32_t)(kW >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

// 4 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row n, k) in a K-major operand of 128-byte rows
// (64 16-bit values) with the 128-byte swizzle; K-blocks of 64 are
// rows_per_kblock * 128 bytes apart.
__device__ __forceinline__ uint32_t sw128_off(uint32_t n, uint32_t k, uint32_t rows_per_kblock) {
  const uint32_t kb = k >> 6, kk = k & 63;
  return kb * rows_per_kblock * 128u + n * 128u + ((((kk >> 3) ^ (n & 7u)) & 7u) << 4) + (kk & 7u) * 2u;
}

template <typename Tin, int JM>
__global__ void __launch_bounds__(kNT, 1)
    k_sketch_tc(const __grid_constant__ CUtensorMap tmap, SketchArgs g, int* __restrict__ err) {
  using S = TcShape<JM>;
  constexpr int JG = S::JG;
  constexpr uint32_t idesc = idesc_16<Tin>();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (reinterpret_cast<uintptr_t>(smem_raw) & 1023)) & 1023);
  unsigned char* Hs = base;                                   // H_128 operand
  unsigned char* Bt = Hs + kHBytes;                           // chunk^T operand
  unsigned char* Xs = Bt + kBtBytes;                          // [2][R2][W] staged chunks
  float* T = reinterpret_cast<float*>(Xs + 2 * kXBytes);      // [R2][kTStride]
  uint32_t* s_off = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(T) + kTBytes);  // [rl][u]
  uint32_t* s_hi = s_off + JG;
  uint64_t* s_d = reinterpret_cast<uint64_t*>(s_hi + JG);     // [2][8] D^(i) words of a chunk
  uint64_t* full = s_d + 16;                                  // [2] TMA
  uint64_t* mmad = full + 2;                                  // [2] MMA done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mmad + 2);

  const int tid = threadIdx.x;
  const int cg = tid % kW;
  const int rl = tid / kW;  // == warp
  const int jn = (int)g.jn;
  const int64_t t_begin = (int64_t)blockIdx.x * g.T / g.G;
  const int64_t t_end = (int64_t)(blockIdx.x + 1) * g.T / g.G;
  const int64_t ntiles = t_end - t_begin;

  struct TileIt {  // 32-bit fields: panels, blocks and chunks all fit
    int pc, i, a;
    __device__ void next(int64_t nch, int p) {
      if (++a == nch) {
        a = 0;
        if (++i == p) {
          i = 0;
          ++pc;
        }
      }
    }
  };
  auto tile_at = [&](int64_t t) {
    TileIt it;
    const int64_t pc = t / g.C;
    const int64_t c = t - pc * g.C;
    it.pc = (int)pc;
    it.i = (int)(c / g.nch);
    it.a = (int)(c - (int64_t)it.i * g.nch);
    return it;
  };

  // ---- setup: barriers, TMEM, H_128, sample tables
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&mmad[s], 1);
    }
    fence_mbar_init();
  }
  if (rl == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
  {
    const uint16_t pos = sizeof(Tin) == 2 && std::is_same<Tin, __nv_bfloat16>::value ? 0x3F80u : 0x3C00u;
    for (int e = tid; e < 128 * 128; e += kNT) {
      const uint32_t m = (uint32_t)e >> 7, k = (uint32_t)e & 127u;
      const uint16_t v = (uint16_t)(pos | ((__popc(m & k) & 1) ? 0x8000u : 0u));
      *reinterpret_cast<uint16_t*>(Hs + sw128_off(m, k, 128)) = v;
    }
  }
  for (int jl = tid; jl < JG; jl += kNT) {
    uint32_t off = 0, hi = 0;
    if (jl < jn) {
      const uint64_t sv = sample_word(g.seed, (uint64_t)(g.j0 + jl)) & (uint64_t)(g.r - 1);
      off = (uint32_t)(sv & (kR2 - 1)) * kTStride;
      hi = (uint32_t)(sv >> 9);
    }
    s_off[(jl % kNRL) * JM + jl / kNRL] = off;
    s_hi[jl] = hi;
  }
  TileIt iss = tile_at(t_begin);
  int64_t issued = 0;
  auto issue_next = [&]() {
    const int s = (int)(issued & 1);
    unsigned char* dst = Xs + (size_t)s * kXBytes;
    mbar_arrive_expect_tx(&full[s], kXBytes);
    const int32_t x = (int32_t)(iss.pc * kW);
    const int64_t y0 = (int64_t)iss.i * g.rb + (int64_t)iss.a * kR2;
    tma_load_2d(dst, &tmap, &full[s], x, (int32_t)y0);
    tma_load_2d(dst + kXBytes / 2, &tmap, &full[s], x, (int32_t)(y0 + 256));
    iss.next(g.nch, g.p);
    ++issued;
  };
  auto d_words = [&](int buf, const TileIt& t) {  // threads 0..7
    if (tid < 8) s_d[buf * 8 + tid] = sign_word(g.seed, kStreamD, (uint64_t)t.i, (uint64_t)(t.a * 8 + tid));
  };
  if (ntiles > 0) d_words(0, tile_at(t_begin));
  fence_proxy_async_smem();  // H_128 written by the generic proxy, read by the MMAs
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (tid == 0)
    for (int64_t k = 0; k < 2 && k < ntiles; ++k) issue_next();

  uint32_t my_hi[JM / 32];
  uint64_t my_dt[JM / 32];
  int64_t dt_block = -1;
#pragma unroll
  for (int h = 0; h < JM / 32; ++h) {
    my_hi[h] = s_hi[rl + kNRL * (32 * h + cg)];
    my_dt[h] = 0;
  }
  float acc[JM];
#pragma unroll
  for (int u = 0; u < JM; ++u) acc[u] = 0.f;
  int64_t cur_pc = -1;
  float* part = static_cast<float*>(g.part);
  auto flush = [&](int64_t pc) {
    float* dst = part + ((int64_t)blockIdx.x + pc) * (int64_t)jn * kW + cg;
#pragma unroll
    for (int u = 0; u < JM; ++u) {
      const int jl = rl + kNRL * u;
      if (jl < jn) dst[(int64_t)jl * kW] = acc[u];
    }
  };

  // Epilogue of chunk `t` (accumulator buffer buf): T = (H_4 (x) I) D.
  // Warp w reads TMEM lanes 32 (w % 4) .. + 31 (H_128 output rows b) and
  // columns 8 (w / 4) .. + 7 of each of the four 128-row blocks.
  const int quarter = rl & 3, cgrp = rl >> 2;
  auto epilogue = [&](int buf) {
    const int b = 32 * quarter + (tid & 31);
#pragma unroll
    for (int half = 0; half < 2; ++half) {  // 4 columns at a time keeps registers low
      float v[4][4];
#pragma unroll
      for (int blk = 0; blk < 4; ++blk)
        tmem_ld4(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(buf * 128 + blk * 32 + cgrp * 8 + half * 4),
                 v[blk]);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float x0 = v[0][c], x1 = v[1][c], x2 = v[2][c], x3 = v[3][c];
        const float s01 = x0 + x1, d01 = x0 - x1, s23 = x2 + x3, d23 = x2 - x3;
        v[0][c] = s01 + s23;
        v[1][c] = d01 + d23;
        v[2][c] = s01 - s23;
        v[3][c] = d01 - d23;
      }
#pragma unroll
      for (int blk = 0; blk < 4; ++blk)
        *reinterpret_cast<float4*>(T + (size_t)(blk * 128 + b) * kTStride + cgrp * 8 + half * 4) =
            make_float4(v[blk][0], v[blk][1], v[blk][2], v[blk][3]);
    }
  };
  // Gather of chunk tile `t` (block i, chunk a) from T.
  auto gather = [&](const TileIt& t) {
    if (t.pc != cur_pc) {
      if (cur_pc >= 0) flush(cur_pc);
#pragma unroll
      for (int u = 0; u < JM; ++u) acc[u] = 0.f;
      cur_pc = t.pc;
    }
    if (t.i != dt_block) {
#pragma unroll
      for (int h = 0; h < JM / 32; ++h) {
        const int jl = rl + kNRL * (32 * h + cg);
        my_dt[h] = jl < jn ? sign_word(g.seed, kStreamDt, (uint64_t)t.i, (uint64_t)((g.j0 + jl) >> 6)) : 0ull;
      }
      dt_block = t.i;
    }
    uint32_t gmask[JM / 32];
#pragma unroll
    for (int h = 0; h < JM / 32; ++h) {
      const int jl = rl + kNRL * (32 * h + cg);
      const uint32_t sg =
          (uint32_t)((__popc(my_hi[h] & (uint32_t)t.a) + (int)((my_dt[h] >> ((g.j0 + jl) & 63)) & 1ull)) & 1);
      gmask[h] = __ballot_sync(0xffffffffu, jl < jn ? sg : 0u);
    }
    const uint4* offv = reinterpret_cast<const uint4*>(s_off + rl * JM);
    const float* tcol = T + cg;
#pragma unroll
    for (int u4 = 0; u4 < JM / 4; ++u4) {
      const uint4 o = offv[u4];
      const uint32_t oo[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int u = 4 * u4 + q;
        const float tv = tcol[oo[q]];
        const uint32_t sb = (gmask[u >> 5] << (31 - (u & 31))) & 0x80000000u;
        acc[u] += __int_as_float(__float_as_int(tv) ^ (int)sb);
      }
    }
  };

  TileIt cur = tile_at(t_begin), prev = cur;
  uint32_t mma_issued = 0;  // MMA batches committed (thread 0)
  bool failed = false;
  for (int64_t k = 0; k < ntiles; ++k) {
    const int s = (int)(k & 1);
    const int64_t rows_i = min(g.rb, g.n - (int64_t)cur.i * g.rb);
    const int nvalid = (int)min((int64_t)kR2, rows_i - (int64_t)cur.a * kR2);
    bool ok = mbar_wait_bounded(&full[s], (uint32_t)((k >> 1) & 1), kTcWait);
    if (k >= 1) ok = ok && mbar_wait_bounded(&mmad[(k - 1) & 1], (uint32_t)(((k - 1) >> 1) & 1), kTcWait);
    // D^(i) signs and transpose into the K-major B operand: item = (4
    // columns, 8 consecutive rows); lanes 8-15 / 24-31 walk their rows in a
    // rotated order so a half-warp's two rows sit in different bank halves.
    if (ok) {
      const unsigned char* X = Xs + (size_t)s * kXBytes;
      const uint64_t* dw = s_d + s * 8;
      const int q4 = tid & 7;                  // columns 4 q4 .. 4 q4 + 3
      const int g8 = (tid >> 3);               // rows 8 g8 .. 8 g8 + 7 (64 groups)
      const int rot = (tid >> 3) & 1;
#pragma unroll
      for (int pair = 0; pair < 2; ++pair) {  // columns (4 q4, 4 q4 + 1), then (4 q4 + 2, 4 q4 + 3)
        uint32_t w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int jj = (j + rot) & 7;
          const int row = 8 * g8 + jj;
          uint32_t x = 0u;
          if (row < nvalid) x = *reinterpret_cast<const uint32_t*>(X + (size_t)row * (kW * 2) + q4 * 8 + pair * 4);
          w[jj] = x ^ (((dw[row >> 6] >> (row & 63)) & 1ull) ? 0x80008000u : 0u);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t sel = h ? 0x7632u : 0x5410u;  // high or low halves of two words
          uint4 o;
          o.x = __byte_perm(w[0], w[1], sel);
          o.y = __byte_perm(w[2], w[3], sel);
          o.z = __byte_perm(w[4], w[5], sel);
          o.w = __byte_perm(w[6], w[7], sel);
          const uint32_t n = (uint32_t)(4 * q4 + 2 * pair + h);
          *reinterpret_cast<uint4*>(Bt + sw128_off(n, (uint32_t)(8 * g8), kW)) = o;
        }
      }
    }
    fence_proxy_async_smem();
    tc::tc_fence_before();
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::tc_fence_after();
    if (tid == 0) {
      // MMAs of chunk k into accumulator buffer s: 4 blocks x 8 K-steps.
      const uint32_t hb = smem_u32(Hs), bb = smem_u32(Bt);
#pragma unroll
      for (int blk = 0; blk < 4; ++blk) {
        const uint32_t d = tmem + (uint32_t)(s * 128 + blk * 32);
#pragma unroll
        for (int ks = 0; ks < 8; ++ks) {
          const uint32_t koff = (uint32_t)(ks & 3) * 32u;
          const uint64_t ad = tc::desc_sw128(hb + (uint32_t)(ks >> 2) * (128u * 128u) + koff);
          const uint64_t bd = tc::desc_sw128(bb + (uint32_t)(2 * blk + (ks >> 2)) * (kW * 128u) + koff);
          mma_f16(d, ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
      }
      tc::mma_commit(&mmad[s]);
      ++mma_issued;
      if (issued < ntiles) issue_next();  // stage s was consumed by the transpose above
    }
    TileIt nx = cur;
    nx.next(g.nch, g.p);
    if (k + 1 < ntiles) d_words((int)((k + 1) & 1), nx);
    if (k >= 1) epilogue((int)((k - 1) & 1));
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (k >= 1) gather(prev);
    prev = cur;
    cur = nx;
  }
  if (!failed && ntiles > 0) {
    const int64_t k = ntiles - 1;
    const bool ok = mbar_wait_bounded(&mmad[k & 1], (uint32_t)((k >> 1) & 1), kTcWait);
    if (__syncthreads_or(!ok)) {
      failed = true;
    } else {
      tc::tc_fence_after();
      epilogue((int)(k & 1));
      tc::tc_fence_before();
      __syncthreads();
      gather(prev);
    }
  }
  if (failed) {
    if (tid == 0) {
      atomicOr(err, 1);
      // Let copies and MMAs in flight land before shared memory and TMEM go.
      for (int64_t kk = (issued > 2 ? issued - 2 : 0); kk < issued; ++kk)
        mbar_wait_bounded(&full[kk & 1], (uint32_t)((kk >> 1) & 1), kTcWait);
      if (mma_issued > 0) {
        const uint32_t kk = mma_issued - 1;
        mbar_wait_bounded(&mmad[kk & 1], (kk >> 1) & 1u, kTcWait);
      }
    }
  } else if (cur_pc >= 0) {
    flush(cur_pc);
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (rl == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

template <typename Tin, int JM>
int launch_tc(const SketchPlan& plan, const SketchArgs& a, int* err, void* out, int64_t ldo, cudaStream_t stream) {
  using S = TcShape<JM>;
  auto kern = k_sketch_tc<Tin, JM>;
  const size_t smem = S::smem_bytes();
  CUtensorMap map;
  const CUtensorMapDataType dt =
      std::is_same<Tin, __nv_bfloat16>::value ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  if (!make_tensor_map_2d(&map, a.A, dt, 2, (uint64_t)a.n, (uint64_t)a.m, (uint64_t)a.lda, kW, 256))
    return BSRHT_EUNSUP;
  BSRHT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<plan.G, kNT, smem, stream>>>(map, a, err);
  BSRHT_CUDA_TRY(cudaGetLastError());
  const int64_t total = a.jn * a.m;
  const float scale = (float)(1.0 / sqrt((double)plan.l));
  k_sketch_reduce_checked<kW><<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(a, static_cast<float*>(out), ldo,
                                                                                   scale, err);
  BSRHT_CUDA_TRY(cudaGetLastError());
  note_launches(2);
  return BSRHT_OK;
}

template <typename Tin, int JM>
int occ_tc() {
  auto kern = k_sketch_tc<Tin, JM>;
  const size_t smem = TcShape<JM>::smem_bytes();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kNT, smem) != cudaSuccess) return 0;
  return occ;
}

}  // namespace

int sketch_occupancy_tc(const SketchPlan& plan) {
  switch (plan.dtype) {
    case BSRHT_BF16: return plan.JM == 32 ? occ_tc<__nv_bfloat16, 32>() : occ_tc<__nv_bfloat16, 64>();
    case BSRHT_F16: return plan.JM == 32 ? occ_tc<__half, 32>() : occ_tc<__half, 64>();
  }
  return 0;
}

int sketch_launch_tc(const SketchPlan& plan, const SketchArgs& a, void* out, int64_t ldo, int* err,
                     cudaStream_t stream) {
  switch (plan.dtype) {
    case BSRHT_BF16:
      return plan.JM == 32 ? launch_tc<__nv_bfloat16, 32>(plan, a, err, out, ldo, stream)
                           : launch_tc<__nv_bfloat16, 64>(plan, a, err, out, ldo, stream);
    case BSRHT_F16:
      return plan.JM == 32 ? launch_tc<__half, 32>(plan, a, err, out, ldo, stream)
                           : launch_tc<__half, 64>(plan, a, err, out, ldo, stream);
  }
  return BSRHT_EUNSUP;
}

}  // namespace bsrht
