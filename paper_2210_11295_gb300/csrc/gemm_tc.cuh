// Tensor-core GEMM for the tall products of the low-rank drivers:
//   C[M x N] = A[M x K] * B[K x N]  in FP32 accuracy on tcgen05 (TF32 MMAs).
//
// A (M x K) and Bt = B^T (N x K) are FP32 with K contiguous (K-major) and
// are read by TMA with the 128- or 64-byte swizzle.  Each tile is split in shared
// memory into a TF32-exact hi part (low 13 mantissa bits cleared; the TF32
// MMA reads the staged x as exactly that) and lo = x - hi, and the product
// is accumulated in TMEM as
//   A_hi B_hi + A_hi B_lo + A_lo B_hi
// (three TF32 MMAs; the dropped A_lo B_lo term and the TF32 truncation of the
// lo parts leave a relative error of about 2^-21 per product, FP32 level).
//
// The tensor core's FP32 accumulation rounds toward zero, so an accumulator
// that runs over all of K drifts by about (number of MMAs) x 2^-24 of its
// value (1e-4 at K = 4096, worse on the all-positive sums of a Gram
// diagonal).  Each K block (32 or 16 deep, 12 or 6 MMAs) is therefore
// accumulated into a fresh TMEM buffer (two buffers, ping-pong) and the
// epilogue warps add it into an FP32 running sum held in registers, rounding
// to nearest.
//
// The small right-hand operand of a tall product (B given K x N) is split
// once in global memory while it is transposed, and both halves come in by
// TMA; only the Gram product, whose B is the tall matrix itself, splits B
// in shared memory too.  (Shared-memory bandwidth, shared by the split and
// the MMA operand reads, is what bounds this kernel.)
//
// CTA: warp 0 allocates TMEM and issues the TMA loads (one thread), warp 1
// issues the MMAs (one thread), warps 4 and up split the tiles, fold the
// finished K blocks (tcgen05.ld of their 32 TMEM lanes, 128 columns per
// warp) and store the rows.  Tiles 128 x 128 (UMMA M=128, N=128, K=8; K
// blocks of 32, a 3-stage ring, 256 threads) or 128 x 256 (UMMA N=256; K
// blocks of 16, a 4-stage ring, 384 threads), see Cfg below.  gridDim.z > 1
// splits K: CTA z writes an FP32 partial to
// C + z * M * N (leading dimension N) for a fixed-order FP64 reduce.  With
// `gram` set (C = A A^T) tiles entirely below the diagonal are skipped.
// With Ct set the epilogue also stores C^T in FP32 (the operand layout of a
// following Gram product, which then needs no transpose pass).
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "common.cuh"
#include "tma.cuh"
#include "tmem.cuh"

namespace bsrht {

namespace tc {

// Two tile shapes.  Cfg<128>: 128 x 128 tiles, K blocks of 32 (128-byte
// rows, 128-byte swizzle), a 3-stage ring, 4 epilogue warps.  Cfg<256>:
// 128 x 256 tiles (one UMMA N = 256 per staged A tile, so the A operand is
// read from shared memory half as often per flop), K blocks of 16 (64-byte
// rows, 64-byte swizzle) so that a 4-stage ring still fits, 8 epilogue
// warps (two per TMEM lane quarter, 128 columns each).
template <int BNT>
struct Cfg {
  static constexpr int BM = 128, BN = BNT;
  static constexpr int BK = BNT == 128 ? 32 : 16;
  static constexpr int STAGES = BNT == 128 ? 3 : 4;
  static constexpr int EPI_WARPS = BN / 32;           // 4 or 8
  static constexpr int THREADS = 128 + 32 * EPI_WARPS;  // warps 0-3: TMA, MMA, 2 idle
  static constexpr int ROW_BYTES = BK * 4;             // 128 or 64: the swizzle span
  static constexpr uint32_t A_BYTES = BM * BK * 4;
  static constexpr uint32_t B_BYTES = BN * BK * 4;
  static constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // A_hi, A_lo, B_hi, B_lo
  static constexpr uint32_t TMEM_COLS = 2 * BN;                        // two accumulator buffers
  static constexpr size_t smem_bytes() { return 1024 + (size_t)STAGES * STAGE_BYTES + 256; }
  static_assert(BNT == 128 || BNT == 256, "tile width");
  static_assert(STAGES * STAGE_BYTES + 1024 + 256 <= 227 * 1024, "shared memory");
  static_assert(TMEM_COLS <= 512, "tensor memory");
};
constexpr int BM = 128;  // both shapes
constexpr uint32_t kWait = 1u << 24;
constexpr int kErrWait = 8;  // the status bit a failed wait sets (kStatusTcWait of dla.cuh)

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes in 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

// The same for rows of 64 bytes (64-byte swizzle): 8-row atoms 512 bytes
// apart, layout type 4.
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}
template <int ROW_BYTES>
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr) {
  if constexpr (ROW_BYTES == 128)
    return desc_sw128(saddr);
  else
    return desc_sw64(saddr);
}

// Instruction descriptor: D FP32, A/B TF32, both K-major, M = BM, N = bn.
template <int bn>
constexpr uint32_t idesc_tf32() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

struct GemmTcArgs {
  int64_t M, N, K;
  void* C;      // TC output, or FP32 partials when gridDim.z > 1
  int64_t ldc;
  int gram;
  int* err;
  int b_upper;  // B[k][n] = 0 for k > n: the N tile at n0 stops at K = n0 + BN
  float* Ct;    // optional FP32 copy of C transposed (N x M, leading dimension ldct)
  int64_t ldct;
};

__host__ __device__ __forceinline__ bool tile_below_diagonal(int64_t bm, int64_t bn, int tile_n) {
  return bm * BM >= (bn + 1) * tile_n;
}

// Split of n16 16-byte groups: lo = x - hi with hi = x with the low 13
// mantissa bits cleared.  The staged x itself serves as the hi operand: the
// TF32 MMA reads only the top 19 bits of each 32-bit operand, which is hi.
template <int NTH>
__device__ __forceinline__ void split_tf32(const uint4* __restrict__ hi, uint4* __restrict__ lo, int t, int n16) {
  for (int idx = t; idx < n16; idx += NTH) {
    const uint4 x = hi[idx];
    uint4 l;
    l.x = __float_as_uint(__uint_as_float(x.x) - __uint_as_float(x.x & 0xFFFFE000u));
    l.y = __float_as_uint(__uint_as_float(x.y) - __uint_as_float(x.y & 0xFFFFE000u));
    l.z = __float_as_uint(__uint_as_float(x.z) - __uint_as_float(x.z & 0xFFFFE000u));
    l.w = __float_as_uint(__uint_as_float(x.w) - __uint_as_float(x.w & 0xFFFFE000u));
    lo[idx] = l;
  }
}

// PRE: B arrives already split (mapB its FP32 values, mapBlo the lo parts,
// both by TMA), and the epilogue warps split only the A tile; without PRE
// they split both tiles in shared memory.
template <typename TC, bool PRE, int BNT>
__global__ void __launch_bounds__(Cfg<BNT>::THREADS, 1)
    k_gemm_tf32x3(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                  const __grid_constant__ CUtensorMap mapBlo, GemmTcArgs g) {
  using C_ = Cfg<BNT>;
  constexpr int BN = C_::BN, BK = C_::BK, STAGES = C_::STAGES, EPI = C_::EPI_WARPS;
  constexpr uint32_t A_BYTES = C_::A_BYTES, B_BYTES = C_::B_BYTES, STAGE_BYTES = C_::STAGE_BYTES;
  constexpr int NSPLIT = 32 * EPI;  // threads of the epilogue warps
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (reinterpret_cast<uintptr_t>(smem_raw) & 1023)) & 1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
  uint64_t* ready = full + STAGES;
  uint64_t* empty = ready + STAGES;
  uint64_t* accf = empty + STAGES;    // [2] K block finished in buffer b
  uint64_t* accfree = accf + 2;       // [2] buffer b folded by the epilogue
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accfree + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // blockIdx.x enumerates tiles row-major, so the N tiles of one row band run
  // side by side and share its A tile through L2.
  const int64_t tn = (g.N + BN - 1) / BN;
  const int64_t bm = (int64_t)blockIdx.x / tn, bn = (int64_t)blockIdx.x - bm * tn;
  const int64_t m0 = bm * BM, n0 = bn * BN;
  if (g.gram && tile_below_diagonal(bm, bn, BN)) return;  // uniform: before any barrier
  const int64_t kmax = g.b_upper ? (g.K < n0 + BN ? g.K : n0 + BN) : g.K;
  const int nkb_all = (int)((kmax + BK - 1) / BK);
  const int kb0 = (int)((int64_t)nkb_all * blockIdx.z / gridDim.z);
  const int kb1 = (int)((int64_t)nkb_all * (blockIdx.z + 1) / gridDim.z);
  const int nkb = kb1 - kb0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&ready[s], NSPLIT);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&accfree[b], EPI);
    }
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, C_::TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool failed = false;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int issued = 0;
      for (int kb = 0; kb < nkb && !failed; ++kb) {
        const int s = kb % STAGES, u = kb / STAGES;
        if (u > 0 && !mbar_wait_bounded(&empty[s], (uint32_t)((u - 1) & 1), kWait)) {
          failed = true;
          break;
        }
        unsigned char* st = base + (size_t)s * STAGE_BYTES;
        mbar_arrive_expect_tx(&full[s], A_BYTES + (PRE ? 2 : 1) * B_BYTES);
        const int32_t kx = (kb0 + kb) * BK;
        tma_load_2d(st, &mapA, &full[s], kx, (int32_t)m0);
        tma_load_2d(st + 2 * A_BYTES, &mapB, &full[s], kx, (int32_t)n0);
        if (PRE) tma_load_2d(st + 2 * A_BYTES + B_BYTES, &mapBlo, &full[s], kx, (int32_t)n0);
        issued = kb + 1;
      }
      if (failed) {
        // Shared memory must not be released under copies still landing.
        for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
          if (!mbar_wait_bounded(&full[kb % STAGES], (uint32_t)((kb / STAGES) & 1), kWait)) atomicOr(g.err, kErrWait);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      constexpr uint32_t idesc = idesc_tf32<BN>();
      int issued = 0;
      for (int kb = 0; kb < nkb && !failed; ++kb) {
        const int s = kb % STAGES, u = kb / STAGES, b = kb & 1;
        if (!mbar_wait_bounded(&ready[s], (uint32_t)(u & 1), kWait) ||
            (kb >= 2 && !mbar_wait_bounded(&accfree[b], (uint32_t)(((kb >> 1) - 1) & 1), kWait))) {
          failed = true;
          break;
        }
        tc_fence_after();
        const uint32_t a_hi = smem_u32(base + (size_t)s * STAGE_BYTES);
        const uint32_t a_lo = a_hi + A_BYTES;
        const uint32_t b_hi = a_hi + 2 * A_BYTES;
        const uint32_t b_lo = b_hi + B_BYTES;
        const uint32_t d = tmem + (uint32_t)(b * BN);
#pragma unroll
        for (int kk = 0; kk < BK / 8; ++kk) {
          const uint32_t off = kk * 32;  // 8 TF32 values along K
          mma_tf32(d, desc_kmajor<C_::ROW_BYTES>(a_hi + off), desc_kmajor<C_::ROW_BYTES>(b_hi + off), idesc,
                   kk > 0 ? 1u : 0u);
          mma_tf32(d, desc_kmajor<C_::ROW_BYTES>(a_hi + off), desc_kmajor<C_::ROW_BYTES>(b_lo + off), idesc, 1u);
          mma_tf32(d, desc_kmajor<C_::ROW_BYTES>(a_lo + off), desc_kmajor<C_::ROW_BYTES>(b_hi + off), idesc, 1u);
        }
        mma_commit(&empty[s]);
        mma_commit(&accf[b]);
        issued = kb + 1;
      }
      // Never free TMEM under MMAs that may still be running: the last
      // commit covers every MMA this thread issued (on the normal path its
      // phase has already completed and the wait returns at once).
      if (issued > 0) {
        const int kb = issued - 1;
        if (!mbar_wait_bounded(&accf[kb & 1], (uint32_t)((kb >> 1) & 1), kWait)) atomicOr(g.err, kErrWait);
      }
    }
  } else if (warp >= 4) {
    const int t = threadIdx.x - 128;  // 0 .. NSPLIT - 1
    const int ew = warp - 4;
    const int wq = warp & 3;         // TMEM lane quarter this warp may access
    const int ch = ew >> 2;          // column half of a 256-wide tile (0 for 128)
    const uint32_t lane_base = tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(128 * ch);
    float run[128];
#pragma unroll
    for (int i = 0; i < 128; ++i) run[i] = 0.f;
    // Adds the finished K block kb (TMEM buffer kb & 1) into run[] and hands
    // the buffer back to the MMA issuer.
    // Waits are made warp-uniform: tcgen05.ld is a warp-collective.
    auto fold = [&](int kb) -> bool {
      const bool ok = mbar_wait_bounded(&accf[kb & 1], (uint32_t)((kb >> 1) & 1), kWait);
      if (!__all_sync(0xffffffffu, ok)) return false;
      tc_fence_after();
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float v[32];
        tmem_ld32(lane_base + (uint32_t)((kb & 1) * BN + 32 * c), v);
#pragma unroll
        for (int q = 0; q < 32; ++q) run[32 * c + q] += v[q];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accfree[kb & 1]);
      return true;
    };
    for (int kb = 0; kb < nkb && !failed; ++kb) {
      const int s = kb % STAGES, u = kb / STAGES;
      const bool ok = mbar_wait_bounded(&full[s], (uint32_t)(u & 1), kWait);
      if (!__all_sync(0xffffffffu, ok)) {
        failed = true;
        break;
      }
      unsigned char* st = base + (size_t)s * STAGE_BYTES;
      split_tf32<NSPLIT>(reinterpret_cast<uint4*>(st), reinterpret_cast<uint4*>(st + A_BYTES), t,
                         (int)(A_BYTES / 16));
      if (!PRE)
        split_tf32<NSPLIT>(reinterpret_cast<uint4*>(st + 2 * A_BYTES),
                           reinterpret_cast<uint4*>(st + 2 * A_BYTES + B_BYTES), t, (int)(B_BYTES / 16));
      fence_proxy_async_smem();
      mbar_arrive(&ready[s]);
      if (kb > 0 && !fold(kb - 1)) failed = true;
    }
    if (!failed && nkb > 0 && !fold(nkb - 1)) failed = true;
    // A warp that gave up a wait writes NaN over its rows, so a caller that
    // does not read the status word still cannot take the tile for a result.
    if (failed) {
#pragma unroll
      for (int i = 0; i < 128; ++i) run[i] = __int_as_float(0x7fc00000);
    }
    // This warp's 32 TMEM lanes are tile rows 32 * wq + lane; its columns
    // are 128 ch .. 128 ch + 127 of the tile.
    const int64_t row = m0 + 32 * wq + lane;
    const int64_t c0 = n0 + 128 * ch;
    const int64_t ncol = g.N - c0;
    if (row < g.M && ncol > 0) {
      if (gridDim.z > 1) {
        float* dst = static_cast<float*>(g.C) + (int64_t)blockIdx.z * g.M * g.N + row * g.N + c0;
        if (ncol >= 128 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
          for (int q = 0; q < 32; ++q)
            reinterpret_cast<float4*>(dst)[q] = make_float4(run[4 * q], run[4 * q + 1], run[4 * q + 2], run[4 * q + 3]);
        } else {
#pragma unroll
          for (int q = 0; q < 128; ++q)
            if (q < ncol) dst[q] = run[q];
        }
      } else {
        TC* dst = static_cast<TC*>(g.C) + row * g.ldc + c0;
        if (sizeof(TC) == 4 && ncol >= 128 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
#pragma unroll
          for (int q = 0; q < 32; ++q)
            reinterpret_cast<float4*>(dst)[q] = make_float4(run[4 * q], run[4 * q + 1], run[4 * q + 2], run[4 * q + 3]);
        } else {
#pragma unroll
          for (int q = 0; q < 128; ++q)
            if (q < ncol) dst[q] = (TC)run[q];
        }
        if (g.Ct != nullptr) {
          // Column q of the tile is row c0 + q of C^T; lane = row of C, so
          // each store of the warp covers 32 consecutive floats.
          float* ct = g.Ct + c0 * g.ldct + row;
#pragma unroll
          for (int q = 0; q < 128; ++q)
            if (q < ncol) ct[(int64_t)q * g.ldct] = run[q];
        }
      }
    }
  }
  if (failed) atomicOr(g.err, kErrWait);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, C_::TMEM_COLS);
}

}  // namespace tc
}  // namespace bsrht
