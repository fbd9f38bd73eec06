// Block SRHT sketch of FP64 data with an exact integer Walsh-Hadamard
// transform (the TMA-fed K1 form for FP64 inputs).
//
// Same method as the other K1 kernels (sketch_kernels.cuh): per R2 = 512-row
// chunk of a W = 16-column panel, the D^(i) signs, the R2-point transform of
// the tensor form of H (Sec. 2), the sampled rows with the outer
// Kronecker-factor and Dt^(i) signs, the block sum of eq. 2.4 over the
// chunks a CTA owns, and per-(CTA, panel) partials reduced in a fixed order.
//
// Why integers: the FP64 units of this GPU run at 1/64 of the FP32 rate, and
// the transform needs log2 R2 adds per element, so FP64 butterflies cannot
// keep up with HBM.  H has entries +-1, so the transform is exact in integer
// arithmetic: each value is converted to 64-bit fixed point at a scale
// shared by its column, the butterflies and the gather of the sampled rows
// run on 64-bit integers (exact), and the integer sums are converted to FP64
// and added into the CTA's partial sums every kFlushChunks chunks, when a
// column's scale grows, and at the end of a panel.
//
// Fixed point: a column keeps a scale exponent S (IEEE biased exponent,
// S >= the biased exponent of every value of the column seen so far, raised
// kScaleMargin above the largest one when it grows); a value
// x = M 2^(e - 1075) (M the 53-bit significand, e its biased exponent, e >= 1
// for subnormals) becomes q = trunc(M / 2^(5 + S - e)) with the sign of x
// times its D^(i) sign, i.e. x = q 2^(S - 1070) up to less than one unit of
// 2^(S - 1070): |q| < 2^48, 48 fraction bits below the column's scale.
// Nine butterfly stages keep |T| < 2^57, and kFlushChunks = 32 chunks of
// sums stay below 2^62, so nothing overflows.  A column that holds Inf or NaN
// gets the scale kNonFinite (every value then converts to 0) and its sketch
// entries are NaN.
//
// Thread layout (512 threads, cg = tid % 16 the column in every phase):
// register phase rows rl + 32 e (rl = tid / 16, e < 16): row bits 5-8 in
// registers, then row bit 0 (= bit 0 of rl = lane bit 4) with one warp
// shuffle; exchange phase rows (g & 1) + 2 b + 32 (g >> 1) (g = tid / 16,
// b < 16): bits 1-4 in registers.  The gather then reads the transformed
// row s_j of each sampled row.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "sketch.cuh"
#include "sketch_kernels.cuh"
#include "tma.cuh"
#include "trace.cuh"

namespace bsrht {

namespace {

constexpr uint32_t kWaitLimit64 = 1u << 22;  // bounded mbarrier waits
constexpr int kW = 16, kNT = 512, kR2 = 512, kBoxR = 256, kStages = 3;
constexpr int kFlushChunks = 32;
constexpr int kScaleMargin = 2;
constexpr int kNonFinite = 4096;  // scale of a column that holds Inf or NaN
constexpr size_t kStageBytes = sizeof(double) * (size_t)kR2 * kW;  // 64 KB

template <int JU>
struct F64xShape {
  static constexpr int JG = 32 * JU;  // sketch rows per launch
  static constexpr size_t meta_bytes = sizeof(uint32_t) * JG + sizeof(uint32_t) * JG + sizeof(int) * kW +
                                       sizeof(uint64_t) * kStages;
  static constexpr size_t smem_bytes() { return kStages * kStageBytes + meta_bytes + 128; }
  static_assert(JU % 8 == 0 && JU <= 16, "sketch-row groups of 256 or 512 on 64-bit sign words");
};

// D^(i) masks: dmtab[(i * nch + a) * 32 + rl] holds at bit e the sign of row
// rl + 32 e of chunk a of block i (16 bits used); dttab the Dt^(i) words of
// the launch's sketch rows (as in the FP32 TMA path).
__global__ void k_sign_tables64(uint64_t seed, int p, int64_t nch, int64_t j0, int64_t tw,
                                uint32_t* __restrict__ dmtab, uint64_t* __restrict__ dttab) {
  const int64_t nm = (int64_t)p * nch * 32;
  const int64_t total = nm + (int64_t)p * tw;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    if (idx < nm) {
      const int rl = (int)(idx & 31);
      const int64_t ia = idx >> 5, i = ia / nch, a = ia - i * nch;
      uint32_t msk = 0;
#pragma unroll
      for (int w = 0; w < 8; ++w) {  // rows 64 w + rl (e = 2 w) and 64 w + 32 + rl (e = 2 w + 1)
        const uint64_t x = sign_word(seed, kStreamD, (uint64_t)i, (uint64_t)(a * 8 + w));
        msk |= (uint32_t)((x >> rl) & 1ull) << (2 * w);
        msk |= (uint32_t)((x >> (rl + 32)) & 1ull) << (2 * w + 1);
      }
      dmtab[idx] = msk;
    } else {
      const int64_t e = idx - nm, i = e / tw, w = e - i * tw;
      dttab[e] = sign_word(seed, kStreamDt, (uint64_t)i, (uint64_t)((j0 >> 6) + w));
    }
  }
}

// Butterflies on 64-bit integers (wrap-around unsigned arithmetic; the
// magnitudes stay below 2^62, so the signed values are exact).
template <int N>
__device__ __forceinline__ void fwht_u64(uint64_t (&v)[N]) {
#pragma unroll
  for (int h = 1; h < N; h <<= 1) {
#pragma unroll
    for (int e = 0; e < N; ++e) {
      if ((e & h) == 0) {
        const uint64_t x = v[e], y = v[e + h];
        v[e] = x + y;
        v[e + h] = x - y;
      }
    }
  }
}

// Fixed-point value of the FP64 bits `raw` at column scale S, negated when
// the sign of x differs from the D sign bit dneg.
__device__ __forceinline__ uint64_t to_fixed(uint64_t raw, int S, uint32_t dneg) {
  const uint32_t hi = (uint32_t)(raw >> 32);
  const int ex = (int)((hi >> 20) & 0x7FFu);
  const uint64_t mant = (raw & 0x000FFFFFFFFFFFFFull) | ((uint64_t)(ex != 0) << 52);
  const int sh = min(5 + S - max(ex, 1), 63);
  const uint64_t q = mant >> sh;
  const uint64_t sm = 0ull - (uint64_t)(((hi >> 31) ^ dneg) & 1u);
  return (q ^ sm) - sm;
}

// The same conversion for columns with S >= 48, where zero and subnormal
// values convert to 0 with or without the subnormal rules (the shift then
// exceeds the 53 significand bits): no implicit-bit test, no exponent clamp.
// c0 = 5 + S; bit 31 of dsign is the D sign.
__device__ __forceinline__ uint64_t to_fixed_fast(uint64_t raw, int c0, uint32_t dsign) {
  const uint32_t hi = (uint32_t)(raw >> 32);
  const int sh = min(c0 - (int)((hi >> 20) & 0x7FFu), 63);
  const uint64_t mant = ((uint64_t)((hi & 0xFFFFFu) | 0x100000u) << 32) | (uint32_t)raw;
  const uint64_t q = mant >> sh;
  const uint64_t sm = (uint64_t)(int64_t)((int32_t)(hi ^ dsign) >> 31);
  return (q ^ sm) - sm;
}

// The FP64 bits of an input value: FP64 as stored, FP32 widened (exactly).
__device__ __forceinline__ uint64_t raw64(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ uint64_t raw64(float x) { return (uint64_t)__double_as_longlong((double)x); }

// Tin: FP64 A, or FP32 A with FP64 arithmetic (each value widened to FP64
// at the load; a 64 KB stage slot then receives a 32 KB chunk and, after
// the register phase, its 64-bit fixed-point transform).
template <int JU, typename Tin>
__global__ void __launch_bounds__(kNT, 1)
    k_sketch_f64x(const __grid_constant__ CUtensorMap tmap, SketchArgs g, const uint32_t* __restrict__ dmtab,
                  const uint64_t* __restrict__ dttab, int64_t tw, int* __restrict__ err) {
  using S = F64xShape<JU>;
  constexpr int JG = S::JG, NH = JU / 16 > 0 ? JU / 16 : 1;
  constexpr uint32_t kChunkBytes = (uint32_t)(sizeof(Tin) * kR2 * kW);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((128 - (reinterpret_cast<uintptr_t>(smem_raw) & 127)) & 127);
  uint32_t* s_off = reinterpret_cast<uint32_t*>(base + kStages * kStageBytes);  // [rg][u]: (s_j & 511) * kW
  uint32_t* s_hi = s_off + JG;                                                  // s_j >> 9
  int* s_scale = reinterpret_cast<int*>(s_hi + JG);                            // column scales S
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_scale + kW);

  const int tid = threadIdx.x;
  const int cg = tid & 15, rl = tid >> 4, lane = tid & 31;
  const int jn = (int)g.jn;
  TileSched sched;
  sched.init(g, (int)blockIdx.x);
  const int64_t t_begin = sched.begin;
  const int64_t ntiles = sched.end - sched.begin;

  struct TileIt {
    int64_t pc, i, a;
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
    it.pc = t / g.C;
    const int64_t c = t - it.pc * g.C;
    it.i = c / g.nch;
    it.a = c - it.i * g.nch;
    return it;
  };
  TileIt iss = tile_at(t_begin);
  int64_t issued = 0;
  auto issue_next = [&]() {
    const int s = (int)(issued % kStages);
    Tin* dst = reinterpret_cast<Tin*>(base + (size_t)s * kStageBytes);
    mbar_arrive_expect_tx(&bar[s], kChunkBytes);
    const int32_t x = (int32_t)(iss.pc * kW);
    const int64_t y0 = iss.i * g.rb + iss.a * kR2;
#pragma unroll
    for (int h = 0; h < kR2 / kBoxR; ++h)
      tma_load_2d(dst + (size_t)h * kBoxR * kW, &tmap, &bar[s], x, (int32_t)(y0 + h * kBoxR));
    iss.next(g.nch, g.p);
    ++issued;
  };

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  for (int jl = tid; jl < JG; jl += kNT) {
    uint32_t off = 0, hi = 0;
    if (jl < jn) {
      const uint64_t sv = sample_word(g.seed, (uint64_t)(g.j0 + jl)) & (uint64_t)(g.r - 1);
      off = (uint32_t)(sv & (kR2 - 1)) * kW;
      hi = (uint32_t)(sv >> 9);
    }
    s_off[(jl & 31) * JU + (jl >> 5)] = off;  // [rg][u]: jl = rg + 32 u
    s_hi[jl] = hi;
  }
  if (tid < kW) s_scale[tid] = 0;
  __syncthreads();
  if (tid == 0)
    for (int64_t k = 0; k < kStages && k < ntiles; ++k) issue_next();

  // Gather: sketch rows jl = rl + 32 u (u < JU), column cg.  The 16 lanes
  // of a row lane share its rows: lane cg evaluates the outer-factor x
  // Dt^(i) sign of u = 16 h + cg, a ballot hands each lane its row lane's
  // 16 bits.
  uint32_t my_hi[NH];
  uint64_t my_dt[NH];
  int64_t dt_block = -1;
#pragma unroll
  for (int h = 0; h < NH; ++h) {
    const int u = 16 * h + cg;
    my_hi[h] = u < JU ? s_hi[rl + 32 * u] : 0u;
    my_dt[h] = 0;
  }
  // Shuffle stage on row bit 0: this thread holds the rows with bit 0 =
  // rl & 1; the partner (lane ^ 16) the others.  Bit 0 clear: own + other;
  // set: other - own = other + (own ^ -1) + 1.
  const uint32_t hbit = (uint32_t)(rl & 1);
  const uint64_t hmask = 0ull - hbit;

  uint64_t acc[JU];
#pragma unroll
  for (int u = 0; u < JU; ++u) acc[u] = 0;
  int scale = 0;       // this thread's copy of s_scale[cg]
  int nacc = 0;        // chunks summed into acc since the last flush (CTA-uniform)
  bool written = false;  // the partial slot of the current panel holds data
  int64_t cur_pc = -1;
  double* part = static_cast<double*>(g.part);

  // Adds the integer sums, at the current scale, into the CTA's partial
  // slot of panel pc (the first flush of a panel stores) and clears them.
  auto flush = [&](int64_t pc) {
    double* dst = part + sched.slot(pc) * (int64_t)jn * kW + cg;
    const double f = ldexp(1.0, scale - 1070);
    const bool bad = scale >= kNonFinite;
#pragma unroll
    for (int u = 0; u < JU; ++u) {
      const int jl = rl + 32 * u;
      if (jl < jn) {
        double v = bad ? __longlong_as_double(0x7ff8000000000000ll) : (double)(long long)acc[u] * f;
        if (written) v += dst[(int64_t)jl * kW];
        dst[(int64_t)jl * kW] = v;
      }
      acc[u] = 0;
    }
    written = true;
    nacc = 0;
  };

  TileIt cur = tile_at(t_begin);
  uint32_t dmask_next = ntiles > 0 ? __ldg(dmtab + (cur.i * g.nch + cur.a) * 32 + rl) : 0u;
  int s = 0;
  uint32_t parity = 0;
  for (int64_t k = 0; k < ntiles; ++k, cur.next(g.nch, g.p)) {
    const int64_t pc = cur.pc, i = cur.i, a = cur.a;
    if (pc != cur_pc) {
      if (cur_pc >= 0) flush(cur_pc);
      written = false;
      scale = 0;  // s_scale is reset below, before the barrier that publishes raises
      cur_pc = pc;
    }
    const bool new_panel = scale == 0;
    const int64_t rows_i = min(g.rb, g.n - i * g.rb);
    const int64_t row0 = a * kR2;
    const int nvalid = (int)max((int64_t)0, min((int64_t)kR2, rows_i - row0));
    const uint32_t dmask = dmask_next;
    {
      TileIt nx = cur;
      nx.next(g.nch, g.p);
      if (k + 1 < ntiles) dmask_next = __ldg(dmtab + (nx.i * g.nch + nx.a) * 32 + rl);
    }
    if (i != dt_block) {
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        const int jl = rl + 32 * (16 * h + cg);
        my_dt[h] = (16 * h + cg < JU && jl < jn) ? __ldg(dttab + i * tw + (jl >> 6)) : 0ull;
      }
      dt_block = i;
    }
    uint32_t gmask[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      const int u = 16 * h + cg;
      const int jl = rl + 32 * u;
      const uint32_t sg = (uint32_t)((__popc(my_hi[h] & (uint32_t)a) + (int)((my_dt[h] >> (jl & 63)) & 1ull)) & 1);
      gmask[h] = (__ballot_sync(0xffffffffu, (u < JU && jl < jn) ? sg : 0u) >> (16 * (lane >> 4))) & 0xFFFFu;
    }
    const bool ok = mbar_wait_bounded(&bar[s], parity, kWaitLimit64);
    // The chunk as loaded (Tin) and, from the register phase's store on,
    // its 64-bit fixed-point transform in the same slot.
    const Tin* st_in = reinterpret_cast<const Tin*>(base + (size_t)s * kStageBytes);
    uint64_t* st = reinterpret_cast<uint64_t*>(base + (size_t)s * kStageBytes);

    // Register phase: raw bits of rows rl + 32 e, their largest exponent
    // (kept in place in bits 20-30 of the high word).
    uint64_t v[16];
    uint32_t mex = 0x00100000u;  // exponent field 1 (the subnormal floor)
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int rr = rl + 32 * e;
      const uint64_t raw = rr < nvalid ? raw64(st_in[rr * kW + cg]) : 0ull;
      v[e] = raw;
      mex = max(mex, (uint32_t)(raw >> 32) & 0x7FF00000u);
    }
    const int me = (int)(mex >> 20);
    if (new_panel && tid < kW) s_scale[tid] = 0;
    const bool raise = scale < kNonFinite && me > scale;
    // One barrier checks the (bounded) TMA wait and whether any column's
    // scale must grow; both are rare, and then handled CTA-uniformly.
    if (__syncthreads_or(!ok || raise)) {
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicOr(err, 1);
          for (int64_t kk = (issued - kStages < k ? k : issued - kStages); kk < issued; ++kk)
            mbar_wait_bounded(&bar[kk % kStages], (uint32_t)((kk / kStages) & 1), kWaitLimit64);
        }
        __syncthreads();
        return;
      }
      if (raise) atomicMax(&s_scale[cg], me == 2047 ? kNonFinite : me + kScaleMargin);
      __syncthreads();
      const int ns = s_scale[cg];
      if (nacc > 0) flush(pc);  // sums so far belong to the old scales
      scale = ns;
    }
    // Every thread is past the previous chunk's gather: refill its stage.
    if (tid == 0 && k >= 1 && issued < ntiles) {
      fence_proxy_async_smem();
      issue_next();
    }
    if (scale >= 48) {
      const int c0 = 5 + scale;
#pragma unroll
      for (int e = 0; e < 16; ++e) v[e] = to_fixed_fast(v[e], c0, dmask << (31 - e));
    } else {
#pragma unroll
      for (int e = 0; e < 16; ++e) v[e] = to_fixed(v[e], scale, (dmask >> e) & 1u);
    }
    fwht_u64<16>(v);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const uint64_t other = __shfl_xor_sync(0xffffffffu, v[e], 16);
      v[e] = other + (v[e] ^ hmask) + hbit;
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) st[(rl + 32 * e) * kW + cg] = v[e];
    __syncthreads();
    // Exchange phase: rows (g & 1) + 2 b + 32 (g >> 1), g = rl.
    const int xr0 = (rl & 1) + 32 * (rl >> 1);
#pragma unroll
    for (int b = 0; b < 16; ++b) v[b] = st[(xr0 + 2 * b) * kW + cg];
    fwht_u64<16>(v);
#pragma unroll
    for (int b = 0; b < 16; ++b) st[(xr0 + 2 * b) * kW + cg] = v[b];
    __syncthreads();
    // Gather: T[s_j] with the outer-factor x Dt^(i) sign.
    const uint4* offv = reinterpret_cast<const uint4*>(s_off + rl * JU);
    const uint64_t* tq = st + cg;
#pragma unroll
    for (int u4 = 0; u4 < JU / 4; ++u4) {
      const uint4 o = offv[u4];
      const uint32_t oo[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int u = 4 * u4 + q;
        const uint64_t x = tq[oo[q]];
        const uint64_t m = (uint64_t)(int64_t)((int32_t)(gmask[u >> 4] << (31 - (u & 15))) >> 31);
        acc[u] += (x ^ m) - m;
      }
    }
    if (++nacc == kFlushChunks) flush(pc);
    if (++s == kStages) {
      s = 0;
      parity ^= 1u;
    }
  }
  if (cur_pc >= 0) flush(cur_pc);
}

// Fixed-order sum of the FP64 partials (one thread per output entry), NaN
// if any CTA reported a failed wait.
__global__ void k_sketch_reduce_checked64(SketchArgs g, double* __restrict__ out, int64_t ldo, double scale,
                                          const int* __restrict__ err) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.jn * g.P * kW) return;
  const int cw = (int)(idx % kW);
  const int64_t jl = (idx / kW) % g.jn;
  const int64_t pc = idx / (kW * g.jn);
  const int64_t col = pc * kW + cw;
  if (col >= g.m) return;
  double* o = out + (g.j0 + jl) * ldo + col;
  if (*err) {
    *o = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  const double* part = static_cast<const double*>(g.part);
  double sum = 0.0;
  for_panel_slots(g, pc, [&](int64_t slot) { sum += part[(slot * g.jn + jl) * kW + cw]; });
  *o = sum * scale;
}

template <int JU, typename Tin>
int launch_f64x(const SketchPlan& plan, const SketchArgs& a, const CUtensorMap& map, int* err, uint32_t* dmtab,
                uint64_t* dttab, void* out, int64_t ldo, cudaStream_t stream) {
  auto kern = k_sketch_f64x<JU, Tin>;
  const size_t smem = F64xShape<JU>::smem_bytes();
  BSRHT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t tw = (a.jn + 63) / 64;
  const int64_t tot = (int64_t)plan.p * (plan.nch * 32 + tw);
  k_sign_tables64<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, stream>>>(a.seed, plan.p,
                                                                                            plan.nch, a.j0, tw,
                                                                                            dmtab, dttab);
  BSRHT_CUDA_TRY(cudaGetLastError());
  trace_mark(stream, "sketch_tables");
  kern<<<plan.G, kNT, smem, stream>>>(map, a, dmtab, dttab, tw, err);
  BSRHT_CUDA_TRY(cudaGetLastError());
  trace_mark(stream, "sketch_kernel");
  const int64_t total = a.jn * a.P * kW;
  k_sketch_reduce_checked64<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(
      a, static_cast<double*>(out), ldo, 1.0 / std::sqrt((double)plan.l), err);
  BSRHT_CUDA_TRY(cudaGetLastError());
  trace_mark(stream, "sketch_reduce");
  note_launches(3);
  return BSRHT_OK;
}

template <int JU>
int occ_f64x() {
  auto kern = k_sketch_f64x<JU, double>;
  const size_t smem = F64xShape<JU>::smem_bytes();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kNT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}

}  // namespace

int sketch_occupancy_f64x(const SketchPlan& plan) { return plan.JM == 8 ? occ_f64x<8>() : occ_f64x<16>(); }

int sketch_launch_f64x(const SketchPlan& plan, const SketchArgs& a, void* out, int64_t ldo, int* err,
                       uint64_t* dtab, uint64_t* dttab, cudaStream_t stream) {
  CUtensorMap map;
  const bool in32 = plan.dtype == kDtypeF32AsF64;
  if (!make_tensor_map_2d(&map, a.A, in32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                          in32 ? 4 : 8, (uint64_t)plan.n, (uint64_t)plan.m, (uint64_t)plan.lda, kW, kBoxR))
    return BSRHT_EUNSUP;
  uint32_t* dmtab = reinterpret_cast<uint32_t*>(dtab);
  if (in32)
    return plan.JM == 8 ? launch_f64x<8, float>(plan, a, map, err, dmtab, dttab, out, ldo, stream)
                        : launch_f64x<16, float>(plan, a, map, err, dmtab, dttab, out, ldo, stream);
  if (plan.JM == 8) return launch_f64x<8, double>(plan, a, map, err, dmtab, dttab, out, ldo, stream);
  return launch_f64x<16, double>(plan, a, map, err, dmtab, dttab, out, ldo, stream);
}

}  // namespace bsrht
