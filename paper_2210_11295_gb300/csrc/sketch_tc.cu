// Block SRHT sketch, tensor-core variant (K2) for 16-bit inputs (BF16, FP16).
//
// Same result as the K1 kernels (eq. 2.3-2.4, R2 = 512-row chunks, the outer
// Kronecker factor collapsed to a sign per sampled row), with the chunk
// transform split by the tensor form of H (Sec. 2):
//     H_512 = H_4 (x) H_128,   H_128 = H_8 (x) H_16,
// and H_128 applied on the tensor cores as one dense +-1 operand: the four
// 128-row blocks of a chunk sit side by side as the columns of one product,
// D = H_128 [X_0 X_1 X_2 X_3] (M = 128, N = 4 x 32, K = 128), with
// tcgen05.mma kind::f16.  +-1 and the 16-bit inputs are exact
// in the operand type and the products accumulate in FP32 in TMEM, so the
// result is the FP32 transform of the stored values.  The remaining H_4
// across the four blocks, the sampled rows and their signs run on the CUDA
// cores as in K1.
//
// Per chunk (32 columns of one panel): a TMA load (64-byte swizzle) into a
// 2-stage ring; all threads apply the D^(i) signs while transposing the
// chunk (ldmatrix.trans) into the K-major, 128-byte-swizzled B operand; one thread issues 8 MMAs (K-steps of
// 16) into a double-buffered TMEM accumulator; the previous
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
#include "trace.cuh"
#include "sketch_kernels.cuh"
#include "tma.cuh"

namespace bsrht {
namespace {

constexpr uint32_t kTcWait = 1u << 22;

constexpr int kW = 32, kNT = 512, kR2 = 512, kNRL = 16;
constexpr int kTStride = 36;                       // FP32 tile row stride (floats): conflict-free float4 stores
constexpr uint32_t kHBytes = 2 * 128 * 128;        // H_128, 16-bit, K-major SW128 (2 K-blocks of 64)
constexpr uint32_t kBtBytes = 2 * 128 * 128;       // chunk^T: 2 K-blocks x 128 rows (block, column) x 128 B
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
  // D FP32, A = B = F16 (0) or BF16 (1), both K-major, N = 128 (the four
  // 128-row blocks' 32 columns side by side), M = 128.
  constexpr uint32_t f = std::is_same<Tin, __nv_bfloat16>::value ? 1u : 0u;
  return (1u << 4) | (f << 7) | (f << 10) | ((uint32_t)(128 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
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
  TileSched sched;
  sched.init(g, (int)blockIdx.x);
  const int64_t t_begin = sched.begin;
  const int64_t ntiles = sched.end - sched.begin;

  const int pstep = sched.step;
  struct TileIt {  // 32-bit fields: panels, blocks and chunks all fit
    int pc, i, a;
    __device__ void next(int64_t nch, int p, int step) {
      if (++a == nch) {
        a = 0;
        if (++i == p) {
          i = 0;
          pc += step;
        }
      }
    }
  };
  auto tile_at = [&](int64_t t) {  // unit t of the schedule
    TileIt it;
    const int64_t u = t / g.C;
    const int64_t c = t - u * g.C;
    it.pc = (int)(u * pstep + sched.half);
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
    iss.next(g.nch, g.p, pstep);
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
    float* dst = part + sched.slot(pc) * (int64_t)jn * kW + cg;
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
  // Columns per pass: fewer live registers beside 64 accumulators.
  constexpr int EC = JM == 64 ? 2 : 4;
  auto epilogue = [&](int buf) {
    const int b = 32 * quarter + (tid & 31);
    const uint32_t tbase = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(buf * 128 + cgrp * 8);
    float* trow = T + (size_t)b * kTStride + cgrp * 8;
#pragma unroll
    for (int pass = 0; pass < 8 / EC; ++pass) {
      uint32_t r[4][EC];
#pragma unroll
      for (int blk = 0; blk < 4; ++blk) {
        const uint32_t ta = tbase + (uint32_t)(blk * 32 + pass * EC);
        if constexpr (EC == 4) {
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(r[blk][0]), "=r"(r[blk][1]), "=r"(r[blk][2]), "=r"(r[blk][3])
                       : "r"(ta)
                       : "memory");
        } else {
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                       : "=r"(r[blk][0]), "=r"(r[blk][1])
                       : "r"(ta)
                       : "memory");
        }
      }
      tc::tmem_wait_ld();
#pragma unroll
      for (int c = 0; c < EC; ++c) {
        const float x0 = __uint_as_float(r[0][c]), x1 = __uint_as_float(r[1][c]);
        const float x2 = __uint_as_float(r[2][c]), x3 = __uint_as_float(r[3][c]);
        const float s01 = x0 + x1, d01 = x0 - x1, s23 = x2 + x3, d23 = x2 - x3;
        r[0][c] = __float_as_uint(s01 + s23);
        r[1][c] = __float_as_uint(d01 + d23);
        r[2][c] = __float_as_uint(s01 - s23);
        r[3][c] = __float_as_uint(d01 - d23);
      }
#pragma unroll
      for (int blk = 0; blk < 4; ++blk) {
        float* dst = trow + (size_t)blk * 128 * kTStride + pass * EC;
        if constexpr (EC == 4)
          *reinterpret_cast<uint4*>(dst) = make_uint4(r[blk][0], r[blk][1], r[blk][2], r[blk][3]);
        else
          *reinterpret_cast<uint2*>(dst) = make_uint2(r[blk][0], r[blk][1]);
      }
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
        const uint32_t tv = __float_as_uint(tcol[oo[q]]);
        acc[u] += __uint_as_float(tv ^ ((gmask[u >> 5] << (31 - (u & 31))) & 0x80000000u));
      }
    }
  };

  TileIt cur = tile_at(t_begin), prev = cur;
  uint32_t mma_issued = 0;  // MMA batches committed (thread 0)
  bool failed = false;
  // Only thread 0 waits on the mbarriers (chunk k + 1 landed, MMA k done);
  // the CTA barrier that follows releases the others, so 511 threads do not
  // poll.  Its result rides on __syncthreads_or.
  {
    const bool ok0 = tid != 0 || ntiles == 0 || mbar_wait_bounded(&full[0], 0u, kTcWait);
    if (__syncthreads_or(!ok0)) failed = true;
  }
  for (int64_t k = 0; k < ntiles && !failed; ++k) {
    const int s = (int)(k & 1);
    const int64_t rows_i = min(g.rb, g.n - (int64_t)cur.i * g.rb);
    const int nvalid = (int)min((int64_t)kR2, rows_i - (int64_t)cur.a * kR2);
    const bool ok = true;  // chunk k landed and MMA k - 1 finished (checked by thread 0 below)
    // D^(i) signs and transpose into the K-major B operand with
    // ldmatrix.trans: warp w takes 8-row groups q = 4w .. 4w + 3; one x4 load
    // covers the group's four 8 x 8 tiles (columns 8i .. 8i + 7), and lane t
    // then holds rows 8q + 2(t % 4), +1 of column 8i + t / 4 as one 32-bit
    // word, which is that column's K-pair in the operand.
    if (ok) {
      const uint32_t X = smem_u32(Xs + (size_t)s * kXBytes);
      const uint64_t* dw = s_d + s * 8;
      const int lane = tid & 31;
      const uint32_t kp = (uint32_t)(2 * (lane & 3));  // row pair within the 8-row group
      // Operand address of (column n0 = block * 32 + lane / 4, K-pair kp): the
      // four tiles' columns n0 + 8i share the swizzle phase (n & 7), so they
      // are 8 rows = 1024 bytes apart.
      unsigned char* bt_lane = Bt + (size_t)(((rl >> 2) * kW + (lane >> 2)) * 128 + 2 * kp);
      const bool full_chunk = nvalid >= kR2;
#pragma unroll
      for (int gq = 0; gq < 4; ++gq) {
        const int q = 4 * rl + gq;  // 8-row group 0..63
        uint32_t r0, r1, r2, r3;
        // The chunk is staged with the 64-byte swizzle: 16-byte unit u of row r
        // sits at unit u ^ ((r >> 1) & 3), so the 8 rows of a tile hit 8 banks.
        const int r8 = 8 * q + (lane & 7);
        const uint32_t addr = X + (uint32_t)(r8 * (kW * 2) + (((lane >> 3) ^ ((r8 >> 1) & 3)) << 4));
        asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                     : "r"(addr)
                     : "memory");
        const uint32_t db = (uint32_t)(dw[q >> 3] >> ((q & 7) * 8 + kp));  // bit 0: row kp, bit 1: row kp + 1
        uint32_t flip = ((db & 1u) << 15) | ((db & 2u) << 30);
        if (!full_chunk) {  // rows past the block's end read as zero
          const int row = 8 * q + (int)kp;
          const uint32_t keep = row >= nvalid ? 0u : (row + 1 >= nvalid ? 0x0000FFFFu : 0xFFFFFFFFu);
          r0 &= keep;
          r1 &= keep;
          r2 &= keep;
          r3 &= keep;
          flip &= keep;
        }
        uint32_t* dst = reinterpret_cast<uint32_t*>(bt_lane + ((q >> 3) & 1) * 16384 +
                                                    ((((uint32_t)q & 7u) ^ (uint32_t)(lane >> 2)) << 4));
        dst[0] = r0 ^ flip;
        dst[256] = r1 ^ flip;  // + 1024 bytes: column + 8
        dst[512] = r2 ^ flip;
        dst[768] = r3 ^ flip;
      }
    }
    fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (tid == 0) {
      // MMAs of chunk k into accumulator buffer s: 8 K-steps of 16, all four
      // blocks at once (N = 128).
      const uint32_t hb = smem_u32(Hs), bb = smem_u32(Bt);
      const uint32_t d = tmem + (uint32_t)(s * 128);
#pragma unroll
      for (int ks = 0; ks < 8; ++ks) {
        const uint32_t koff = (uint32_t)(ks & 3) * 32u + (uint32_t)(ks >> 2) * (128u * 128u);
        mma_f16(d, tc::desc_sw128(hb + koff), tc::desc_sw128(bb + koff), idesc, ks > 0 ? 1u : 0u);
      }
      tc::mma_commit(&mmad[s]);
      ++mma_issued;
      if (issued < ntiles) issue_next();  // stage s was consumed by the transpose above
    }
    TileIt nx = cur;
    nx.next(g.nch, g.p, pstep);
    if (k + 1 < ntiles) d_words((int)((k + 1) & 1), nx);
    if (k >= 1) epilogue((int)((k - 1) & 1));
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (k >= 1) gather(prev);
    bool ok0 = true;
    if (tid == 0) {
      if (k + 1 < ntiles) ok0 = mbar_wait_bounded(&full[(k + 1) & 1], (uint32_t)(((k + 1) >> 1) & 1), kTcWait);
      ok0 = ok0 && mbar_wait_bounded(&mmad[s], (uint32_t)((k >> 1) & 1), kTcWait);
    }
    tc::tc_fence_before();
    if (__syncthreads_or(!ok0)) failed = true;
    tc::tc_fence_after();
    prev = cur;
    cur = nx;
  }
  if (!failed && ntiles > 0) {  // MMA of the last chunk: waited at the end of the loop
    epilogue((int)((ntiles - 1) & 1));
    tc::tc_fence_before();
    __syncthreads();
    gather(prev);
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
  if (!make_tensor_map_2d(&map, a.A, dt, 2, (uint64_t)a.n, (uint64_t)a.m, (uint64_t)a.lda, kW, 256,
                          CU_TENSOR_MAP_SWIZZLE_64B))
    return BSRHT_EUNSUP;
  BSRHT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<plan.G, kNT, smem, stream>>>(map, a, err);
  BSRHT_CUDA_TRY(cudaGetLastError());
  trace_mark(stream, "sketch_kernel");
  const int64_t total = (a.jn + kReduceRows - 1) / kReduceRows * a.P * 32;  // one warp per (row group, panel)
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
