// Block SRHT sketch, CUDA-core variant with a TMA-fed shared-memory ring
// (the streaming form of K1 used when A's layout allows 2-D TMA).
//
// Same arithmetic as k_sketch_chunked (see sketch_kernels.cuh): per R2-row
// chunk of a W-column panel, D^(i) signs, the R2-point Walsh-Hadamard
// transform (tensor form of H, Sec. 2) and the sampled rows with the outer
// Kronecker-factor and Dt^(i) signs, accumulated over the chunks a CTA owns
// (eq. 2.4 block sum), partials reduced in a fixed order.  The register
// phase (high five row bits) gives each thread one column of 32 rows; the
// exchange phase (low four bits) and the gather give it two adjacent columns
// and use 64-bit shared-memory accesses, the exchange phase as packed FP32
// pairs.  For 512 < l <= 768 a 256-thread form (k_sketch_tma256) holds
// 2 x 32 rows in the register phase and 4 columns in the exchange phase and
// gather; above that the 512-thread kernel keeps half of its 1024-row
// group's accumulators in tensor memory.  Here one thread
// streams the chunks with cp.async.bulk.tensor into a STAGES-deep ring
// guarded by mbarriers, so HBM reads of later chunks overlap the butterflies
// and the gather of the current one.  FP32 inputs are transformed in place
// in the staged chunk; 16-bit inputs are widened into a separate FP32 tile.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "sketch.cuh"
#include "trace.cuh"
#include "sketch_kernels.cuh"
#include "tma.cuh"
#include "f32x2.cuh"
#include "tmem.cuh"

namespace bsrht {

namespace {

constexpr uint32_t kWaitLimit = 1u << 22;  // bounded mbarrier waits (each try_wait may sleep)

// Ring depth: three 64 KB FP32 stages, or four 32 KB 16-bit stages plus the
// 64 KB FP32 tile.
template <typename Tin>
constexpr int stages_for() {
  return sizeof(Tin) == 4 ? 3 : 4;
}

template <typename Tin, int W, int NT, int R2, int JM, int STAGES>
struct TmaShape {
  static constexpr int NRL = NT / W;
  static constexpr int E = R2 / NRL;
  static constexpr int LOG_R2 = ilog2c(R2);
  static constexpr int JG = JM * NRL;
  static constexpr bool kInPlace = sizeof(Tin) == 4;
  static constexpr int BOXR = R2 < 256 ? R2 : 256;
  static constexpr size_t stage_bytes = sizeof(Tin) * (size_t)R2 * W;
  static constexpr size_t tile_bytes = kInPlace ? 0 : sizeof(float) * (size_t)R2 * W;
  static constexpr size_t meta_bytes = 2 * sizeof(uint32_t) * JG + sizeof(uint64_t) * STAGES + 16;
  static constexpr size_t smem_bytes() { return STAGES * stage_bytes + tile_bytes + meta_bytes + 128; }
  static_assert(NT % W == 0 && E >= NRL && E % NRL == 0, "thread layout");
  static_assert(R2 >= 64 && R2 % BOXR == 0, "chunk rows");
  static_assert(JG % 64 == 0, "sketch-row groups on 64-bit words");
};

// Chunk geometry: R2 = 512 rows x W = 32 columns, 256 threads (so each may
// hold 64 values in registers).  Register phase (row bits 4-8): 16 row
// lanes x 16 column pairs, rows rl + 16 e; exchange phase (bits 0-3) and
// gather: 32 row groups x 8 column quads.  JU sketch rows per thread (32 JU
// per launch).
template <typename Tin, int JU, int STAGES>
struct TmaShape256 {
  static constexpr int W = 32, NT = 256, R2 = 512;
  static constexpr int JG = 32 * JU;
  static constexpr bool kInPlace = sizeof(Tin) == 4;
  static constexpr int BOXR = 256;
  static constexpr size_t stage_bytes = sizeof(Tin) * (size_t)R2 * W;
  static constexpr size_t tile_bytes = kInPlace ? 0 : sizeof(float) * (size_t)R2 * W;
  static constexpr size_t meta_bytes = 2 * sizeof(uint32_t) * JG + sizeof(uint64_t) * STAGES;
  static constexpr size_t smem_bytes() { return STAGES * stage_bytes + tile_bytes + meta_bytes + 128; }
  static_assert(JG % 64 == 0 && JU % 8 == 0, "sketch-row groups on 64-bit words");
};

template <typename Tin>
__device__ __forceinline__ float widen(Tin v) {
  if constexpr (sizeof(Tin) == 4)
    return v;
  else
    return Elem<Tin>::to_f32(v);
}

// Sign tables for the TMA path.  dmtab[(i*nch + a)*16 + rl] holds, at bit e,
// the D^(i) sign of row rl + 16e of chunk a of block i (the 32 rows a thread
// of row lane rl owns); dttab holds the Dt^(i) words of the launch's sketch
// rows.
__global__ void k_sign_tables(uint64_t seed, int p, int64_t nch, int64_t j0, int64_t tw, uint32_t* __restrict__ dmtab,
                              uint64_t* __restrict__ dttab) {
  const int64_t nm = (int64_t)p * nch * 16;
  const int64_t total = nm + (int64_t)p * tw;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < nm) {
      const int rl = (int)(idx & 15);
      const int64_t ia = idx >> 4, i = ia / nch, a = ia - i * nch;
      uint32_t m = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) {  // rows 64w + 16q + rl, q < 4
        const uint64_t x = (sign_word(seed, kStreamD, (uint64_t)i, (uint64_t)(a * 8 + w)) >> rl) & 0x0001000100010001ull;
        m |= ((uint32_t)(x | (x >> 15) | (x >> 30) | (x >> 45)) & 0xFu) << (4 * w);
      }
      dmtab[idx] = m;
    } else {
      const int64_t e = idx - nm, i = e / tw, w = e - i * tw;
      dttab[e] = sign_word(seed, kStreamDt, (uint64_t)i, (uint64_t)((j0 >> 6) + w));
    }
  }
}

template <typename Tin, int W, int NT, int R2, int JM, int STAGES>
__global__ void __launch_bounds__(NT, 1)
    k_sketch_tma(const __grid_constant__ CUtensorMap tmap, SketchArgs g, const uint32_t* __restrict__ dmtab,
                 const uint64_t* __restrict__ dttab, int64_t tw, int* __restrict__ err) {
  using S = TmaShape<Tin, W, NT, R2, JM, STAGES>;
  constexpr int NRL = S::NRL, E = S::E, JG = S::JG, BOXR = S::BOXR;
  static_assert(W == 32 && NRL == 16 && E == 32 && R2 == 512, "sign masks assume 16 row lanes x 32 rows");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((128 - (reinterpret_cast<uintptr_t>(smem_raw) & 127)) & 127);
  Tin* stage = reinterpret_cast<Tin*>(base);                                   // [STAGES][R2][W]
  float* tile_sep = reinterpret_cast<float*>(base + STAGES * S::stage_bytes);  // [R2][W] (16-bit inputs)
  uint32_t* s_off = reinterpret_cast<uint32_t*>(base + STAGES * S::stage_bytes + S::tile_bytes);  // s_lo * W
  uint32_t* s_hi = s_off + JG;
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_hi + JG);
  uint32_t* tm_slot = reinterpret_cast<uint32_t*>(bar + STAGES);  // TMEM base address (JM = 64)

  const int tid = threadIdx.x;
  const int cg = tid % W;  // == lane
  const int rl = tid / W;  // == warp
  const int jn = (int)g.jn;
  TileSched sched;
  sched.init(g, (int)blockIdx.x);
  const int64_t t_begin = sched.begin;
  const int64_t ntiles = sched.end - sched.begin;

  // Tile t = (panel pc, block i, chunk a) in panel-major order; iterators
  // advance without divisions.
  struct TileIt {
    int64_t pc, i, a;
    int step;
    __device__ void next(int64_t nch, int p) {
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
    it.pc = u * sched.step + sched.half;
    it.i = c / g.nch;
    it.a = c - it.i * g.nch;
    it.step = sched.step;
    return it;
  };
  TileIt iss = tile_at(t_begin);  // next tile to issue (thread 0 only)
  int64_t issued = 0;
  auto issue_next = [&]() {  // TMA for the CTA's next tile into stage issued % STAGES
    const int s = (int)(issued % STAGES);
    Tin* dst = stage + (size_t)s * R2 * W;
    mbar_arrive_expect_tx(&bar[s], (uint32_t)S::stage_bytes);
    const int32_t x = (int32_t)(iss.pc * W);
    const int64_t y0 = iss.i * g.rb + iss.a * R2;
#pragma unroll
    for (int h = 0; h < R2 / BOXR; ++h)
      tma_load_2d(dst + (size_t)h * BOXR * W, &tmap, &bar[s], x, (int32_t)(y0 + h * BOXR));
    iss.next(g.nch, g.p);
    ++issued;
  };

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  for (int jl = tid; jl < JG; jl += NT) {
    uint32_t off = 0, hi = 0;
    if (jl < jn) {
      const uint64_t sv = sample_word(g.seed, (uint64_t)(g.j0 + jl)) & (uint64_t)(g.r - 1);
      off = (uint32_t)(sv & (R2 - 1)) * W;
      hi = (uint32_t)(sv >> S::LOG_R2);
    }
    s_off[(jl % 32) * (JM / 2) + jl / 32] = off;  // [row lane rg][u]: jl = rg + 32 u
    s_hi[jl] = hi;
  }
  // Sketch-row groups of 1024 (JU = 32 rows per thread, 64 accumulators):
  // the 128-register budget of 512 threads holds half of them, and the
  // other half waits in TMEM (unused by this kernel otherwise).  Each warp
  // owns two 32-column slots of its lane quarter; per chunk the gather
  // works through the half in registers, swaps it with the half in TMEM
  // (one tcgen05.st and one tcgen05.ld of 32 values per thread) and works
  // through that one; the next chunk starts with the half now in registers.
  constexpr int JU = JM / 2, NH = JU / 16;
  constexpr bool kTm = JU > 16;
  constexpr int JR = kTm ? 16 : JU;  // sketch rows whose accumulators are in registers
  constexpr uint32_t kTmCols = 256;
  if constexpr (kTm) {
    if (tid < 32) tc::tmem_alloc(tm_slot, kTmCols);
    tc::tc_fence_before();
  }
  __syncthreads();
  uint32_t tm_addr = 0;  // this thread's slot 0; slot 1 is 32 columns on
  if constexpr (kTm) {
    tc::tc_fence_after();
    tm_addr = *tm_slot + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16) + 64u * (uint32_t)(tid >> 7);
  }
  if (tid == 0)
    for (int64_t k = 0; k < STAGES && k < ntiles; ++k) issue_next();

  // Exchange phase and gather: thread = (row lane rg = tid / 16, column
  // pair cp = tid % 16); sketch rows jl = rg + 32 u, u < JM / 2, two columns
  // each.  The 16 lanes of a row lane share its sketch rows: lane cp
  // evaluates the outer-factor x Dt^(i) sign of u = 16 h + cp and a warp
  // ballot hands each lane its row lane's 16 bits.  s_hi never changes; the
  // Dt word only with the block.
  const int cp = tid & 15, rg = tid >> 4;
  uint32_t my_hi[NH];
#pragma unroll
  for (int h = 0; h < NH; ++h) my_hi[h] = s_hi[rg + 32 * (16 * h + cp)];  // 0 for jl >= jn

  float acc[JR][2];
  float(&accv)[2 * JR] = reinterpret_cast<float(&)[2 * JR]>(acc);
#pragma unroll
  for (int u = 0; u < JR; ++u) acc[u][0] = acc[u][1] = 0.f;
  int hcur = 0;  // (JM = 64) the half of the sketch rows whose accumulators are in registers
  int64_t cur_pc = -1;
  float* part = static_cast<float*>(g.part);
  auto flush_rows = [&](int64_t pc, int ubase) {  // sketch rows rg + 32 (ubase + u)
    float* dst = part + sched.slot(pc) * (int64_t)jn * W + 2 * cp;
#pragma unroll
    for (int u = 0; u < JR; ++u) {
      const int jl = rg + 32 * (ubase + u);
      if (jl < jn) *reinterpret_cast<float2*>(dst + (int64_t)jl * W) = make_float2(acc[u][0], acc[u][1]);
    }
  };
  auto flush = [&](int64_t pc) {
    if constexpr (kTm) {
      flush_rows(pc, JR * hcur);
      tc::tmem_ld32(tm_addr + 32u * (uint32_t)(1 - hcur), accv);
      flush_rows(pc, JR * (1 - hcur));
    } else {
      flush_rows(pc, 0);
    }
  };

  // Chunk coordinates within the panel in 32-bit registers, advanced
  // incrementally: block i, chunk a of the block, c = i nch + a (the plan
  // keeps p nch below 2^31).  Every chunk is full unless the blocks are
  // ragged.
  const int nch = (int)g.nch, C = (int)g.C;
  const bool all_full = g.rb % R2 == 0 && g.n == (int64_t)g.p * g.rb;
  int64_t pc;
  int i, a, c;
  {
    const TileIt t0 = tile_at(t_begin);
    pc = t0.pc;
    i = (int)t0.i;
    a = (int)t0.a;
    c = i * nch + a;
  }
  const uint32_t* dm_row = dmtab + rl;
  uint32_t dmask_next = ntiles > 0 ? __ldg(dm_row + (size_t)c * 16) : 0u;
  bool new_panel = true, new_block = true;
  uint32_t my_dtbit[NH];
  int s = 0;
  uint32_t parity = 0;
  for (int64_t k = 0; k < ntiles; ++k) {
    if (new_panel) {
      if (cur_pc >= 0) flush(cur_pc);
#pragma unroll
      for (int u = 0; u < JR; ++u) acc[u][0] = acc[u][1] = 0.f;
      if constexpr (kTm) tc::tmem_st32(tm_addr + 32u * (uint32_t)(1 - hcur), accv);
      cur_pc = pc;
    }
    int nvalid = R2;
    if (!all_full) {
      const int64_t rows_i = min(g.rb, g.n - (int64_t)i * g.rb);
      nvalid = (int)min((int64_t)R2, rows_i - (int64_t)a * R2);
    }
    // The next chunk's coordinates (a wraps at the block end, c and i at the
    // panel end).
    int a_n = a + 1, i_n = i, c_n = c + 1;
    bool wrap = false;
    if (a_n == nch) {
      a_n = 0;
      ++i_n;
      if (c_n == C) {
        c_n = 0;
        i_n = 0;
        wrap = true;
      }
    }
    // This thread's 32 D^(i) signs (rows rl + 16e) and, by a warp ballot, the
    // outer-factor x Dt^(i) signs of its row lane's sketch rows jl = rl + 16u.
    const uint32_t dmask = dmask_next;
    if (k + 1 < ntiles) dmask_next = __ldg(dm_row + (size_t)c_n * 16);  // prefetch the next chunk's D mask
    if (new_block) {
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        const int jl = rg + 32 * (16 * h + cp);
        my_dtbit[h] = jl < jn ? (uint32_t)(__ldg(dttab + (int64_t)i * tw + (jl >> 6)) >> (jl & 63)) & 1u : 0u;
      }
    }
    uint32_t gmask[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      const uint32_t sg = (uint32_t)(__popc(my_hi[h] & (uint32_t)a) + my_dtbit[h]) & 1u;  // my_hi = 0 for jl >= jn
      gmask[h] = (__ballot_sync(0xffffffffu, sg) >> (16 * ((tid >> 4) & 1))) & 0xFFFFu;
    }
    const bool ok = mbar_wait_bounded(&bar[s], parity, kWaitLimit);

    Tin* st = stage + (size_t)s * R2 * W;
    float* tile = S::kInPlace ? reinterpret_cast<float*>(st) : tile_sep;
    // Register phase: rows rl + NRL*e, D^(i) signs, high log2(E) bits.
    float v[E];
    if (nvalid == R2) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const float x = widen<Tin>(st[(rl + NRL * e) * W + cg]);
        v[e] = __int_as_float(__float_as_int(x) ^ (int)((dmask << (31 - e)) & 0x80000000u));
      }
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int rr = rl + NRL * e;
        const float x = rr < nvalid ? widen<Tin>(st[rr * W + cg]) : 0.f;
        v[e] = __int_as_float(__float_as_int(x) ^ (int)((dmask << (31 - e)) & 0x80000000u));
      }
    }
    fwht_regs<float, E>(v);
#pragma unroll
    for (int e = 0; e < E; ++e) tile[(rl + NRL * e) * W + cg] = v[e];
    // One barrier both publishes the register phase and makes a failed
    // (bounded) wait CTA-uniform: data read after a failed wait is garbage
    // but nothing reaches global memory before this check.
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(err, 1);
        for (int64_t kk = (issued - STAGES < k ? k : issued - STAGES); kk < issued; ++kk)
          mbar_wait_bounded(&bar[kk % STAGES], (uint32_t)((kk / STAGES) & 1), kWaitLimit);
      }
      if constexpr (kTm) tc::tc_fence_before();
      __syncthreads();
      if constexpr (kTm) {
        if (tid < 32) {
          tc::tc_fence_after();
          tc::tmem_dealloc(*tm_slot, kTmCols);
        }
      }
      return;
    }
    // In place (FP32): every thread has finished the previous chunk, so its
    // stage is free; refill it (the 16-bit path refills at the chunk end).
    if constexpr (S::kInPlace) {
      if (tid == 0 && k >= 1 && issued < ntiles) {
        fence_proxy_async_smem();
        issue_next();
      }
    }
    // Exchange phase: rows 16 rg + b (low four bits), columns 2 cp, 2 cp + 1
    // as packed pairs (one instruction per butterfly for both columns; the
    // pairs load and store without re-pairing registers).
    {
      f2 w[NRL];
      float* tp = tile + (NRL * rg) * W + 2 * cp;
#pragma unroll
      for (int b = 0; b < NRL; ++b) w[b] = *reinterpret_cast<const f2*>(tp + b * W);
      fwht_regs2<NRL>(w);
#pragma unroll
      for (int b = 0; b < NRL; ++b) *reinterpret_cast<f2*>(tp + b * W) = w[b];
    }
    __syncthreads();
    // Sampled rows (offsets s_lo * W) with the signs of gmask, two columns per load.
    const float* tq = tile + 2 * cp;
    auto gather = [&](int hs) {  // sketch rows rg + 32 (JR hs + u), u < JR
      const uint4* offv = reinterpret_cast<const uint4*>(s_off + rg * JU + JR * hs);
      const uint32_t gm = (NH > 1 && hs) ? gmask[NH - 1] : gmask[0];
#pragma unroll
      for (int u4 = 0; u4 < JR / 4; ++u4) {
        // Groups of four sketch rows all at or past jn hold nothing (uniform).
        if constexpr (kTm) {
          if (32 * (JR * hs + 4 * u4) >= jn) break;
        }
        const uint4 o = offv[u4];
        const uint32_t oo[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int u = 4 * u4 + q;
          const float2 tv = *reinterpret_cast<const float2*>(tq + oo[q]);
          // +-1.0f from the sign bit: the product is exact, so the FMA adds
          // exactly +-tv, one instruction per column.
          const float sg = __uint_as_float((((NH > 1 ? gm : gmask[u >> 4]) << (31 - (u & 15))) & 0x80000000u) |
                                           0x3f800000u);
          acc[u][0] = fmaf(tv.x, sg, acc[u][0]);
          acc[u][1] = fmaf(tv.y, sg, acc[u][1]);
        }
      }
    };
    if constexpr (kTm) {
      gather(hcur);
      tc::tmem_st32(tm_addr + 32u * (uint32_t)hcur, accv);
      tc::tmem_ld32(tm_addr + 32u * (uint32_t)(1 - hcur), accv);
      hcur ^= 1;
      gather(hcur);
    } else {
      gather(0);
    }
    if constexpr (!S::kInPlace) {
      __syncthreads();  // stage s and the separate tile are free again
      if (tid == 0 && issued < ntiles) {
        fence_proxy_async_smem();
        issue_next();
      }
    }
    if (++s == STAGES) {
      s = 0;
      parity ^= 1u;
    }
    new_block = a_n == 0;
    new_panel = wrap;
    a = a_n;
    i = i_n;
    c = c_n;
    if (wrap) pc += sched.step;
  }
  if (cur_pc >= 0) flush(cur_pc);
  if constexpr (kTm) {
    tc::tc_fence_before();
    __syncthreads();
    if (tid < 32) {
      tc::tc_fence_after();
      tc::tmem_dealloc(*tm_slot, kTmCols);
    }
  }
}

template <typename Tin, int JU, int STAGES>
__global__ void __launch_bounds__(256, 1)
    k_sketch_tma256(const __grid_constant__ CUtensorMap tmap, SketchArgs g, const uint32_t* __restrict__ dmtab,
                 const uint64_t* __restrict__ dttab, int64_t tw, int* __restrict__ err) {
  using S = TmaShape256<Tin, JU, STAGES>;
  constexpr int W = S::W, NT = S::NT, R2 = S::R2, JG = S::JG, BOXR = S::BOXR;
  static_assert(JU <= 24, "32 sketch rows per thread: k_sketch_tma with JM = 64");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((128 - (reinterpret_cast<uintptr_t>(smem_raw) & 127)) & 127);
  Tin* stage = reinterpret_cast<Tin*>(base);                                   // [STAGES][R2][W]
  float* tile_sep = reinterpret_cast<float*>(base + STAGES * S::stage_bytes);  // [R2][W] (16-bit inputs)
  uint32_t* s_off = reinterpret_cast<uint32_t*>(base + STAGES * S::stage_bytes + S::tile_bytes);  // s_lo * W
  uint32_t* s_hi = s_off + JG;
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_hi + JG);

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int rl = tid >> 4, cp = tid & 15;  // register phase: row lane, column pair
  const int rg = tid >> 3, c4 = tid & 7;   // exchange phase and gather: row group, column quad
  const int jn = (int)g.jn;
  TileSched sched;
  sched.init(g, (int)blockIdx.x);
  const int64_t t_begin = sched.begin;
  const int64_t ntiles = sched.end - sched.begin;

  // Tile t = (panel pc, block i, chunk a) in panel-major order; iterators
  // advance without divisions.
  struct TileIt {
    int64_t pc, i, a;
    int step;
    __device__ void next(int64_t nch, int p) {
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
    it.pc = u * sched.step + sched.half;
    it.i = c / g.nch;
    it.a = c - it.i * g.nch;
    it.step = sched.step;
    return it;
  };
  TileIt iss = tile_at(t_begin);  // next tile to issue (thread 0 only)
  int64_t issued = 0;
  auto issue_next = [&]() {  // TMA for the CTA's next tile into stage issued % STAGES
    const int s = (int)(issued % STAGES);
    Tin* dst = stage + (size_t)s * R2 * W;
    mbar_arrive_expect_tx(&bar[s], (uint32_t)S::stage_bytes);
    const int32_t x = (int32_t)(iss.pc * W);
    const int64_t y0 = iss.i * g.rb + iss.a * R2;
#pragma unroll
    for (int h = 0; h < R2 / BOXR; ++h)
      tma_load_2d(dst + (size_t)h * BOXR * W, &tmap, &bar[s], x, (int32_t)(y0 + h * BOXR));
    iss.next(g.nch, g.p);
    ++issued;
  };

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  for (int jl = tid; jl < JG; jl += NT) {
    uint32_t off = 0, hi = 0;
    if (jl < jn) {
      const uint64_t sv = sample_word(g.seed, (uint64_t)(g.j0 + jl)) & (uint64_t)(g.r - 1);
      off = (uint32_t)(sv & (R2 - 1)) * W;
      hi = (uint32_t)(sv >> 9);  // R2 = 512
    }
    s_off[(jl % 32) * JU + jl / 32] = off;  // [row group rg][u]: jl = rg + 32 u
    s_hi[jl] = hi;
  }
  __syncthreads();
  if (tid == 0)
    for (int64_t k = 0; k < STAGES && k < ntiles; ++k) issue_next();

  // Gather: sketch rows jl = rg + 32 u, u < JU, four columns each.  The 8
  // lanes of a row group share its sketch rows: lane c4 evaluates the
  // outer-factor x Dt^(i) sign of u = 8 h + c4 and a warp ballot hands each
  // lane its row group's byte.  s_hi never changes; the Dt word only with
  // the block.
  constexpr int NH = JU / 8;
  uint32_t my_hi[NH];
#pragma unroll
  for (int h = 0; h < NH; ++h) my_hi[h] = s_hi[rg + 32 * (8 * h + c4)];  // 0 for jl >= jn

  float acc[JU][4];
#pragma unroll
  for (int u = 0; u < JU; ++u) acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = 0.f;
  int64_t cur_pc = -1;
  float* part = static_cast<float*>(g.part);
  auto flush = [&](int64_t pc) {
    float* dst = part + sched.slot(pc) * (int64_t)jn * W + 4 * c4;
#pragma unroll
    for (int u = 0; u < JU; ++u) {
      const int jl = rg + 32 * u;
      if (jl < jn)
        *reinterpret_cast<float4*>(dst + (int64_t)jl * W) = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
    }
  };

  // Chunk coordinates as in k_sketch_tma: 32-bit, advanced incrementally.
  const int nch = (int)g.nch, C = (int)g.C;
  const bool all_full = g.rb % R2 == 0 && g.n == (int64_t)g.p * g.rb;
  int64_t pc;
  int i, a, c;
  {
    const TileIt t0 = tile_at(t_begin);
    pc = t0.pc;
    i = (int)t0.i;
    a = (int)t0.a;
    c = i * nch + a;
  }
  const uint32_t* dm_row = dmtab + rl;  // rows rl + 16 e
  uint32_t dmask_next = ntiles > 0 ? __ldg(dm_row + (size_t)c * 16) : 0u;
  bool new_panel = true, new_block = true;
  uint32_t my_dtbit[NH];
  int s = 0;
  uint32_t parity = 0;
  for (int64_t k = 0; k < ntiles; ++k) {
    if (new_panel) {
      if (cur_pc >= 0) flush(cur_pc);
#pragma unroll
      for (int u = 0; u < JU; ++u) acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = 0.f;
      cur_pc = pc;
    }
    int nvalid = R2;
    if (!all_full) {
      const int64_t rows_i = min(g.rb, g.n - (int64_t)i * g.rb);
      nvalid = (int)min((int64_t)R2, rows_i - (int64_t)a * R2);
    }
    int a_n = a + 1, i_n = i, c_n = c + 1;
    bool wrap = false;
    if (a_n == nch) {
      a_n = 0;
      ++i_n;
      if (c_n == C) {
        c_n = 0;
        i_n = 0;
        wrap = true;
      }
    }
    // This thread's 32 D^(i) signs (rows rl + 16e) and, by a warp ballot, the
    // outer-factor x Dt^(i) signs of its row group's sketch rows.
    const uint32_t dmask = dmask_next;
    if (k + 1 < ntiles) dmask_next = __ldg(dm_row + (size_t)c_n * 16);  // prefetch the next chunk's D mask
    if (new_block) {
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        const int jl = rg + 32 * (8 * h + c4);
        my_dtbit[h] = jl < jn ? (uint32_t)(__ldg(dttab + (int64_t)i * tw + (jl >> 6)) >> (jl & 63)) & 1u : 0u;
      }
    }
    uint32_t gmask[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      const uint32_t sg = (uint32_t)(__popc(my_hi[h] & (uint32_t)a) + my_dtbit[h]) & 1u;  // my_hi = 0 for jl >= jn
      gmask[h] = (__ballot_sync(0xffffffffu, sg) >> (8 * (lane >> 3))) & 0xFFu;
    }
    const bool ok = mbar_wait_bounded(&bar[s], parity, kWaitLimit);

    Tin* st = stage + (size_t)s * R2 * W;
    float* tile = S::kInPlace ? reinterpret_cast<float*>(st) : tile_sep;
    // Register phase: rows rl + 16 e (high five row bits), columns 2 cp,
    // 2 cp + 1, D^(i) signs (one per row for both columns).
    // Both columns of a row travel as one packed pair (one instruction per
    // butterfly for both).
    {
      f2 v[32];
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        const int rr = rl + 16 * e;
        f2 x = 0ull;
        if (nvalid == R2 || rr < nvalid) {
          if constexpr (sizeof(Tin) == 4) {
            x = *reinterpret_cast<const f2*>(reinterpret_cast<const float*>(st) + rr * W + 2 * cp);
          } else {
            const uint32_t raw = *reinterpret_cast<const uint32_t*>(st + rr * W + 2 * cp);
            const Tin* h2 = reinterpret_cast<const Tin*>(&raw);
            x = ((f2)__float_as_uint(widen<Tin>(h2[1])) << 32) | __float_as_uint(widen<Tin>(h2[0]));
          }
        }
        const uint32_t sb = (dmask << (31 - e)) & 0x80000000u;
        v[e] = x ^ (((f2)sb << 32) | sb);
      }
      fwht_regs2<32>(v);
      if constexpr (!S::kInPlace) __syncthreads();  // the previous chunk's gather is done with the tile
#pragma unroll
      for (int e = 0; e < 32; ++e) *reinterpret_cast<f2*>(tile + (rl + 16 * e) * W + 2 * cp) = v[e];
    }
    // One barrier both publishes the register phase and makes a failed
    // (bounded) wait CTA-uniform: data read after a failed wait is garbage
    // but nothing reaches global memory before this check.
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(err, 1);
        for (int64_t kk = (issued - STAGES < k ? k : issued - STAGES); kk < issued; ++kk)
          mbar_wait_bounded(&bar[kk % STAGES], (uint32_t)((kk / STAGES) & 1), kWaitLimit);
      }
      __syncthreads();
      return;
    }
    // Every thread has finished the previous chunk's gather (FP32: its stage,
    // which is its tile, is free) or this chunk's widening (16-bit: this
    // stage is free): refill it.
    if (tid == 0 && issued < ntiles && (!S::kInPlace || k >= 1)) {
      fence_proxy_async_smem();
      issue_next();
    }
    // Exchange phase: rows 16 rg + b (low four bits), columns 4 c4 .. 4 c4 + 3.
    // (Packed column pairs (4 c4, 4 c4 + 1) and (4 c4 + 2, 4 c4 + 3).)
    {
      f2 w[2][16];
      float* tp = tile + (16 * rg) * W + 4 * c4;
#pragma unroll
      for (int b = 0; b < 16; ++b) {
        const ulonglong2 t4 = *reinterpret_cast<const ulonglong2*>(tp + b * W);
        w[0][b] = t4.x;
        w[1][b] = t4.y;
      }
      fwht_regs2<16>(w[0]);
      fwht_regs2<16>(w[1]);
#pragma unroll
      for (int b = 0; b < 16; ++b) *reinterpret_cast<ulonglong2*>(tp + b * W) = make_ulonglong2(w[0][b], w[1][b]);
    }
    __syncthreads();
    // Sampled rows (offsets s_lo * W) with the signs of gmask, four columns
    // per load; +-1.0f from the sign bit makes the FMA add exactly +-t.
    const uint4* offv = reinterpret_cast<const uint4*>(s_off + rg * JU);
    const float* tq = tile + 4 * c4;
#pragma unroll
    for (int u4 = 0; u4 < JU / 4; ++u4) {
      const uint4 o = offv[u4];
      const uint32_t oo[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int u = 4 * u4 + q;
        const float4 tv = *reinterpret_cast<const float4*>(tq + oo[q]);
        const float sg = __uint_as_float(((gmask[u >> 3] << (31 - (u & 7))) & 0x80000000u) | 0x3f800000u);
        acc[u][0] = fmaf(tv.x, sg, acc[u][0]);
        acc[u][1] = fmaf(tv.y, sg, acc[u][1]);
        acc[u][2] = fmaf(tv.z, sg, acc[u][2]);
        acc[u][3] = fmaf(tv.w, sg, acc[u][3]);
      }
    }
    if (++s == STAGES) {
      s = 0;
      parity ^= 1u;
    }
    new_block = a_n == 0;
    new_panel = wrap;
    a = a_n;
    i = i_n;
    c = c_n;
    if (wrap) pc += sched.step;
  }
  if (cur_pc >= 0) flush(cur_pc);
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static std::once_flag once;
  static EncodeFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
    cudaGetLastError();
  });
  return fn;
}

// l <= 512 (JM = 32) and l > 768 (JM = 64, sketch-row groups of 1024, half
// the accumulators in TMEM): 512 threads of 32 values (more warps hide the
// shared-memory latency); 512 < l <= 768 (JM = 48): 256 threads of 64
// values, whose 255-register budget holds 96 accumulators (packed
// butterflies).
template <typename Tin, int JM>
struct TmaKernel {
  static constexpr int STAGES = stages_for<Tin>();
  static constexpr bool k256 = JM == 48;
  static constexpr int NT = k256 ? 256 : 512;
  static size_t smem() {
    if constexpr (k256)
      return TmaShape256<Tin, JM / 2, STAGES>::smem_bytes();
    else
      return TmaShape<Tin, 32, 512, 512, JM, STAGES>::smem_bytes();
  }
  static auto fn() {
    if constexpr (k256)
      return k_sketch_tma256<Tin, JM / 2, STAGES>;
    else
      return k_sketch_tma<Tin, 32, 512, 512, JM, STAGES>;
  }
};

template <typename Tin, int JM>
int launch_tma(const SketchPlan& plan, const SketchArgs& a, const CUtensorMap& map, int* err, uint64_t* dtab,
               uint64_t* dttab, void* out, int64_t ldo, cudaStream_t stream) {
  constexpr int W = 32;
  constexpr int NT = TmaKernel<Tin, JM>::NT;
  auto kern = TmaKernel<Tin, JM>::fn();
  const size_t smem = TmaKernel<Tin, JM>::smem();
  BSRHT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t tw = (a.jn + 63) / 64;
  const int64_t tot = (int64_t)plan.p * (plan.nch * 16 + tw);
  uint32_t* dmtab = reinterpret_cast<uint32_t*>(dtab);
  k_sign_tables<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, stream>>>(a.seed, plan.p, plan.nch,
                                                                                          a.j0, tw, dmtab, dttab);
  BSRHT_CUDA_TRY(cudaGetLastError());
  trace_mark(stream, "sketch_tables");
  kern<<<plan.G, NT, smem, stream>>>(map, a, dmtab, dttab, tw, err);
  BSRHT_CUDA_TRY(cudaGetLastError());
  trace_mark(stream, "sketch_kernel");
  const int64_t total = (a.jn + kReduceRows - 1) / kReduceRows * a.P * 32;  // one warp per (row group, panel)
  const float scale = (float)(1.0 / sqrt((double)plan.l));
  k_sketch_reduce_checked<W><<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(a, static_cast<float*>(out), ldo,
                                                                                  scale, err);
  BSRHT_CUDA_TRY(cudaGetLastError());
  trace_mark(stream, "sketch_reduce");
  note_launches(3);
  return BSRHT_OK;
}

template <typename Tin, int JM>
int occ_tma() {
  constexpr int NT = TmaKernel<Tin, JM>::NT;
  auto kern = TmaKernel<Tin, JM>::fn();
  const size_t smem = TmaKernel<Tin, JM>::smem();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem) != cudaSuccess) return 0;
  return occ;
}

template <typename Tin>
int occ_tma_jm(int jm) {
  switch (jm) {
    case 32: return occ_tma<Tin, 32>();
    case 48: return occ_tma<Tin, 48>();
    case 64: return occ_tma<Tin, 64>();
  }
  return 0;
}

template <typename Tin>
int launch_tma_jm(const SketchPlan& plan, const SketchArgs& a, const CUtensorMap& map, int* err, uint64_t* dtab,
                  uint64_t* dttab, void* out, int64_t ldo, cudaStream_t stream) {
  switch (plan.JM) {
    case 32: return launch_tma<Tin, 32>(plan, a, map, err, dtab, dttab, out, ldo, stream);
    case 48: return launch_tma<Tin, 48>(plan, a, map, err, dtab, dttab, out, ldo, stream);
    case 64: return launch_tma<Tin, 64>(plan, a, map, err, dtab, dttab, out, ldo, stream);
  }
  return BSRHT_EINVAL;
}

}  // namespace

bool make_tensor_map_2d(CUtensorMap* map, const void* base, CUtensorMapDataType dtype, size_t elem_bytes,
                        uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_cols, uint32_t box_rows,
                        CUtensorMapSwizzle swizzle) {
  EncodeFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {ld * elem_bytes};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, dtype, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swizzle, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


int sketch_occupancy_tma(const SketchPlan& plan) {
  switch (plan.dtype) {
    case BSRHT_F32: return occ_tma_jm<float>(plan.JM);
    case BSRHT_BF16: return occ_tma_jm<__nv_bfloat16>(plan.JM);
    case BSRHT_F16: return occ_tma_jm<__half>(plan.JM);
  }
  return 0;
}

int sketch_launch_tma(const SketchPlan& plan, const SketchArgs& a, void* out, int64_t ldo, int* err,
                      uint64_t* dtab, uint64_t* dttab, cudaStream_t stream) {
  CUtensorMap map;
  const CUtensorMapDataType dt = plan.dtype == BSRHT_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : plan.dtype == BSRHT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                            : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const size_t es = plan.dtype == BSRHT_F32 ? 4 : 2;
  if (!make_tensor_map_2d(&map, a.A, dt, es, (uint64_t)plan.n, (uint64_t)plan.m, (uint64_t)plan.lda, 32,
                          256))
    return BSRHT_EUNSUP;
  switch (plan.dtype) {
    case BSRHT_F32: return launch_tma_jm<float>(plan, a, map, err, dtab, dttab, out, ldo, stream);
    case BSRHT_BF16: return launch_tma_jm<__nv_bfloat16>(plan, a, map, err, dtab, dttab, out, ldo, stream);
    case BSRHT_F16: return launch_tma_jm<__half>(plan, a, map, err, dtab, dttab, out, ldo, stream);
  }
  return BSRHT_EINVAL;
}

}  // namespace bsrht
