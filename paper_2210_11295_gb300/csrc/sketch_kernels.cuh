// Block SRHT sketch kernels, CUDA-core variant (K1).
//
// B = Omega A with Omega = [Omega^(1) ... Omega^(p)] (eq. 2.3) is formed as the
// block sum of eq. 2.4 in one pass over A.  H_r of each block is split with
// its tensor form (Sec. 2): for r = r1 * R2,
//     H_r[s, a*R2 + b] = H_{r1}[s >> log2 R2, a] * H_{R2}[s & (R2-1), b],
// so a chunk a of R2 rows only needs its own R2-point transform T_a; the
// r1-point outer factor collapses to a sign per sampled row,
//     (R H_r D x)_j = sum_a (-1)^popc((s_j >> log2 R2) & a) * T_a[s_j & (R2-1)].
// A CTA streams chunks of one column panel (W columns): D^(i) signs and the
// high log2(E) butterfly stages run in registers on a column held by one
// thread, one shared-memory exchange gives the low log2(NRL) stages, and the
// sampled rows are gathered from shared memory into per-thread accumulators
// with the outer-factor and Dt^(i) signs.  Partial sums are written per
// (CTA, panel) and summed in a fixed order by the reduce kernel, which also
// applies the 1/sqrt(l) scale (every entry of Omega is +-1/sqrt(l)).
#pragma once

#include "common.cuh"
#include "sketch.cuh"

namespace bsrht {

struct SketchArgs {
  const void* A;
  int64_t lda, n, m;
  int64_t rb, r;
  int p;
  int64_t j0, jn;  // sketch rows [j0, j0 + jn) handled by this launch
  uint64_t seed;
  int64_t nch, C, T;
  int G;
  void* part;      // Tc [(G + P) * jn * W]; slot of (CTA g, panel pc) = g + pc
  // Grouped launches (several sketches in one persistent launch): this
  // sketch owns the global tiles [toff, toff + T) of a launch of Gg CTAs over
  // Tg tiles (CTA c takes [c Tg / Gg, (c + 1) Tg / Gg)), and CTA c writes
  // partial slot (c - gfirst + pc).  A launch of one sketch has toff = 0,
  // Tg = T, Gg = G and gfirst = 0.
  int64_t toff, Tg;
  int Gg, gfirst;
  void* out;       // grouped reduce only: output, leading dimension, scale
  int64_t ldo;
  double scale;
  // TMA-fed kernels: with `paired` set (16-bit inputs, 64-byte panel rows)
  // CTAs 2q and 2q + 1 walk the same (panel pair, block, chunk) units on the
  // two panels of each pair (see TileSched).  P = number of column panels.
  int paired;
  int64_t P;
};

// Tile schedule of the TMA-fed kernels.  Plain: CTA c takes tiles
// [c T / G, (c + 1) T / G) of the panel-major order (panel, block, chunk)
// and writes partial slot c + panel.  Paired: units are (panel pair, block,
// chunk), U = ceil(P / 2) C of them; CTA pair q = c / 2 takes units
// [q U / Gp, (q + 1) U / Gp) (Gp = G / 2) on panel 2 pp + (c & 1), so the two
// 64-byte halves of each 128-byte line are fetched at about the same time
// and one of the two reads hits L2 instead of DRAM; slot = half (Gp + Pp) +
// q + pp.  (An odd P gives the last pair's second CTA a panel past the end:
// its loads read zeros and its slots are never reduced.)
struct TileSched {
  int64_t begin, end;  // unit range of this CTA
  int half, step;      // panel = step * (unit / C) + half
  int64_t slot0;       // slot of panel pc: slot0 + pc / step
  __device__ __forceinline__ void init(const SketchArgs& g, int cta) {
    if (!g.paired) {
      begin = (int64_t)cta * g.T / g.G;
      end = (int64_t)(cta + 1) * g.T / g.G;
      half = 0;
      step = 1;
      slot0 = cta;
    } else {
      const int64_t gp = g.G / 2, pp = (g.P + 1) / 2, u = pp * g.C, q = cta >> 1;
      half = cta & 1;
      step = 2;
      begin = q < gp ? q * u / gp : 0;
      end = q < gp ? (q + 1) * u / gp : 0;
      slot0 = half * (gp + pp) + q;
    }
  }
  __device__ __forceinline__ int64_t slot(int64_t pc) const { return slot0 + pc / step; }
};

// Partial-slot range of panel pc for the reduce: calls f(slot) for every CTA
// whose units touch the panel, in CTA order.
template <typename F>
__device__ __forceinline__ void for_panel_slots(const SketchArgs& g, int64_t pc, F&& f) {
  int64_t lo, hi, G, U, base;
  if (!g.paired) {
    lo = pc * g.C;
    G = g.G;
    U = g.T;
    base = pc;
  } else {
    const int64_t pp = (g.P + 1) / 2;
    lo = (pc >> 1) * g.C;
    G = g.G / 2;
    U = pp * g.C;
    base = (pc & 1) * (G + pp) + (pc >> 1);
  }
  hi = lo + g.C;
  int64_t c = lo * G / U;
  if (c > 0) --c;
  while (c < G && (c + 1) * U / G <= lo) ++c;
  for (; c < G && c * U / G < hi; ++c) f(base + c);
}

struct SketchGroup {
  int nreq;
  SketchArgs r[kMaxGroup];
};

// Walsh-Hadamard butterflies over the index of a register array:
// stage h pairs v[e] with v[e + h] for every e with (e & h) == 0.
template <typename Tc, int N>
__device__ __forceinline__ void fwht_regs(Tc (&v)[N]) {
#pragma unroll
  for (int h = 1; h < N; h <<= 1) {
#pragma unroll
    for (int e = 0; e < N; ++e) {
      if ((e & h) == 0) {
        const Tc x = v[e], y = v[e + h];
        v[e] = x + y;
        v[e + h] = x - y;
      }
    }
  }
}

template <typename Tin, typename Tc, int W, int NT, int R2, int JM>
struct K1Shape {
  static constexpr int NRL = NT / W;          // rows handled in parallel (row lanes)
  static constexpr int E = R2 / NRL;          // rows per thread in the register phase
  static constexpr int Q = E / NRL;           // high parts per thread in the exchange phase
  static constexpr int LOG_R2 = ilog2c(R2);
  static constexpr int JG = JM * NRL;         // sketch rows per launch
  static constexpr int DW = R2 >= 64 ? R2 / 64 : 1;  // D-sign words per chunk
  static_assert(NT % W == 0, "NT multiple of W");
  static_assert((R2 & (R2 - 1)) == 0 && R2 % NRL == 0, "R2 power of two");
  static_assert(E >= NRL && E % NRL == 0, "exchange phase needs E >= NRL");
  static_assert(JG % 64 == 0, "sketch-row groups start on 64-bit sign words");
  static constexpr size_t smem_bytes() {
    return sizeof(Tc) * R2 * W + 2 * sizeof(uint32_t) * JG + sizeof(uint64_t) * (JG / 64 + DW);
  }
};

// The tiles of sketch g that CTA `cta` owns (see SketchArgs), with shared
// memory smem_raw of K1Shape::smem_bytes().
template <typename Tin, typename Tc, int W, int NT, int R2, int JM>
__device__ __forceinline__ void sketch_chunked_body(const SketchArgs& g, int cta, unsigned char* smem_raw) {
  using S = K1Shape<Tin, Tc, W, NT, R2, JM>;
  constexpr int NRL = S::NRL, E = S::E, Q = S::Q, JG = S::JG, DW = S::DW;
  const int64_t t_begin = max((int64_t)cta * g.Tg / g.Gg - g.toff, (int64_t)0);
  const int64_t t_end = min((int64_t)(cta + 1) * g.Tg / g.Gg - g.toff, g.T);
  if (t_begin >= t_end) return;
  __syncthreads();  // a previous sketch of this CTA is done with shared memory
  Tc* tile = reinterpret_cast<Tc*>(smem_raw);                        // [R2][W]
  uint32_t* s_lo = reinterpret_cast<uint32_t*>(tile + R2 * W);        // s_j & (R2-1)
  uint32_t* s_hi = s_lo + JG;                                         // s_j >> log2 R2
  uint64_t* s_dt = reinterpret_cast<uint64_t*>(s_hi + JG);            // Dt^(i) bits
  uint64_t* s_d = s_dt + JG / 64;                                     // D^(i) bits of the chunk

  const int tid = threadIdx.x;
  const int cg = tid % W;
  const int rl = tid / W;
  const int jn = (int)g.jn;
  const Tin* __restrict__ A = static_cast<const Tin*>(g.A);

  for (int jl = tid; jl < jn; jl += NT) {
    const uint64_t s = sample_word(g.seed, (uint64_t)(g.j0 + jl)) & (uint64_t)(g.r - 1);
    s_lo[jl] = (uint32_t)(s & (R2 - 1));
    s_hi[jl] = (uint32_t)(s >> S::LOG_R2);
  }

  Tc acc[JM];
#pragma unroll
  for (int u = 0; u < JM; ++u) acc[u] = Tc(0);
  int64_t cur_pc = -1, cur_block = -1;
  Tc* part = static_cast<Tc*>(g.part);

  auto flush = [&](int64_t pc) {
    Tc* dst = part + ((int64_t)(cta - g.gfirst) + pc) * (int64_t)jn * W + cg;
#pragma unroll
    for (int u = 0; u < JM; ++u) {
      const int jl = rl + NRL * u;
      if (jl < jn) dst[(int64_t)jl * W] = acc[u];
    }
  };

  for (int64_t t = t_begin; t < t_end; ++t) {
    const int64_t pc = t / g.C;
    const int64_t c = t - pc * g.C;
    const int64_t i = c / g.nch;
    const int64_t a = c - i * g.nch;
    if (pc != cur_pc) {
      if (cur_pc >= 0) flush(cur_pc);
#pragma unroll
      for (int u = 0; u < JM; ++u) acc[u] = Tc(0);
      cur_pc = pc;
    }
    const int64_t rows_i = min(g.rb, g.n - i * g.rb);
    const int64_t row0 = a * R2;
    if (row0 >= rows_i) continue;  // all-padding chunk: contributes zero

    __syncthreads();  // previous chunk's gather is done with tile / tables
    if (i != cur_block) {
      for (int w = tid; w < (jn + 63) / 64; w += NT)
        s_dt[w] = sign_word(g.seed, kStreamDt, (uint64_t)i, (uint64_t)(g.j0 >> 6) + w);
      cur_block = i;
    }
    for (int w = tid; w < DW; w += NT)
      s_d[w] = sign_word(g.seed, kStreamD, (uint64_t)i, (uint64_t)(row0 >> 6) + w);
    __syncthreads();

    // Register phase: rows rl + NRL*e of column cg; D^(i) signs; stages on
    // the high log2(E) bits of the in-chunk row index.
    Tc v[E];
    const int64_t col = pc * W + cg;
    const bool col_ok = col < g.m;
    const int64_t nvalid = min((int64_t)R2, rows_i - row0);
    const Tin* src = A + (i * g.rb + row0) * g.lda + col;
    const int dshift = R2 >= 64 ? 0 : (int)(row0 & 63);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int rr = rl + NRL * e;
      Tc x = Tc(0);
      if (col_ok && rr < nvalid) x = load_as<Tc>(src + (int64_t)rr * g.lda);
      const uint32_t neg = (uint32_t)((s_d[rr >> 6] >> ((rr & 63) + dshift)) & 1ull);
      v[e] = flip(x, neg);
    }
    fwht_regs<Tc, E>(v);
#pragma unroll
    for (int e = 0; e < E; ++e) tile[(rl + NRL * e) * W + cg] = v[e];
    __syncthreads();

    // Exchange phase: rows NRL*h + b (b < NRL) of Q high parts h; stages on
    // the low log2(NRL) bits.
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      Tc w2[NRL];
      const int h = rl * Q + q;
#pragma unroll
      for (int b = 0; b < NRL; ++b) w2[b] = tile[(NRL * h + b) * W + cg];
      fwht_regs<Tc, NRL>(w2);
#pragma unroll
      for (int b = 0; b < NRL; ++b) tile[(NRL * h + b) * W + cg] = w2[b];
    }
    __syncthreads();

    // Sampled rows with the outer-factor sign H_{r1}[s_hi, a] and Dt^(i).
#pragma unroll
    for (int u = 0; u < JM; ++u) {
      const int jl = rl + NRL * u;
      if (jl < jn) {
        const uint32_t neg =
            (uint32_t)((__popcll((unsigned long long)s_hi[jl] & (unsigned long long)a) +
                        (int)((s_dt[jl >> 6] >> (jl & 63)) & 1ull)) & 1);
        acc[u] += flip(tile[s_lo[jl] * W + cg], neg);
      }
    }
  }
  if (cur_pc >= 0) flush(cur_pc);
}

template <typename Tin, typename Tc, int W, int NT, int R2, int JM>
__global__ void __launch_bounds__(NT, 1) k_sketch_chunked(SketchArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  sketch_chunked_body<Tin, Tc, W, NT, R2, JM>(g, (int)blockIdx.x, smem_raw);
}

// Several sketches of one kernel instance in one persistent launch: the
// tiles of all of them are laid end to end and cut evenly over the CTAs.
template <typename Tin, typename Tc, int W, int NT, int R2, int JM>
__global__ void __launch_bounds__(NT, 1) k_sketch_grouped(const __grid_constant__ SketchGroup grp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int q = 0; q < grp.nreq; ++q)
    sketch_chunked_body<Tin, Tc, W, NT, R2, JM>(grp.r[q], (int)blockIdx.x, smem_raw);
}

// Fixed-order sum of the per-(CTA, panel) partials and the 1/sqrt(l) scale.
template <typename Tc, int W>
__device__ __forceinline__ Tc sketch_reduce_entry(const SketchArgs& g, int64_t jl, int64_t col) {
  const int64_t pc = col / W;
  const int cw = (int)(col - pc * W);
  const int64_t lo = g.toff + pc * g.C, hi = lo + g.C;  // global tile range of panel pc
  int64_t cta = lo * g.Gg / g.Tg;
  if (cta > 0) --cta;
  while (cta < g.Gg && (cta + 1) * g.Tg / g.Gg <= lo) ++cta;
  const Tc* part = static_cast<const Tc*>(g.part);
  Tc s = Tc(0);
  for (; cta < g.Gg && cta * g.Tg / g.Gg < hi; ++cta)
    s += part[((cta - g.gfirst + pc) * g.jn + jl) * W + cw];
  return s;
}

template <typename Tc, typename Tout, int W>
__global__ void k_sketch_reduce(SketchArgs g, Tout* __restrict__ out, int64_t ldo, Tc scale) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = g.jn * g.m;
  if (idx >= total) return;
  const int64_t jl = idx / g.m;
  const int64_t col = idx - jl * g.m;
  out[(g.j0 + jl) * ldo + col] = (Tout)(sketch_reduce_entry<Tc, W>(g, jl, col) * scale);
}

// Reduce of a grouped launch: blockIdx.y selects the sketch.
template <typename Tc, typename Tout, int W>
__global__ void k_sketch_reduce_grouped(const __grid_constant__ SketchGroup grp) {
  const SketchArgs& g = grp.r[blockIdx.y];
  const int64_t total = g.jn * g.m;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t jl = idx / g.m;
    const int64_t col = idx - jl * g.m;
    Tout* out = static_cast<Tout*>(g.out);
    out[(g.j0 + jl) * g.ldo + col] = (Tout)(sketch_reduce_entry<Tc, W>(g, jl, col) * (Tc)g.scale);
  }
}

// Fixed-order reduce of the TMA-fed kernels' partials; NaN output if any CTA
// reported a failed wait.  One warp per (column panel, group of kReduceRows
// sketch rows), lane = column of the panel (W = 32): every slot row read and
// every output row written is one contiguous 128-byte run, and the panel's
// slot range (64-bit divisions) is found once per warp.  Each entry is summed
// over the slots in CTA order.  Launch with
// ceil(jn / kReduceRows) * P * 32 threads.
constexpr int kReduceRows = 8;
template <int W>
__global__ void k_sketch_reduce_checked(SketchArgs g, float* __restrict__ out, int64_t ldo, float scale,
                                        const int* __restrict__ err) {
  static_assert(W == 32, "one lane per panel column");
  constexpr int RG = kReduceRows;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nrg = (g.jn + RG - 1) / RG;
  if (gw >= nrg * g.P) return;  // warp-uniform
  const int64_t pc = gw / nrg;
  const int64_t jb = (gw - pc * nrg) * RG;
  const int nr = (int)(g.jn - jb < RG ? g.jn - jb : RG);
  const int64_t col = pc * W + lane;
  const bool colok = col < g.m;
  float* o = out + (g.j0 + jb) * ldo + col;
  if (*err) {
    for (int r = 0; r < nr; ++r)
      if (colok) o[(int64_t)r * ldo] = __int_as_float(0x7fc00000);
    return;
  }
  float s[RG];
#pragma unroll
  for (int r = 0; r < RG; ++r) s[r] = 0.f;
  const float* part = static_cast<const float*>(g.part);
  for_panel_slots(g, pc, [&](int64_t slot) {
    const float* v = part + (slot * g.jn + jb) * W + lane;
#pragma unroll
    for (int r = 0; r < RG; ++r)
      if (r < nr) s[r] += v[(int64_t)r * W];
  });
  if (colok) {
#pragma unroll
    for (int r = 0; r < RG; ++r)
      if (r < nr) o[(int64_t)r * ldo] = s[r] * scale;
  }
}

// Direct kernel for tiny blocks (r below the smallest chunk): each thread
// forms one output entry as the explicit +-1 combination of its column.
template <typename Tin, typename Tc, typename Tout>
__global__ void __launch_bounds__(256) k_sketch_small_r(SketchArgs g, Tout* __restrict__ out,
                                                        int64_t ldo, Tc scale) {
  constexpr int JT = 8, CT = 32;
  __shared__ uint64_t s_dw;
  __shared__ uint64_t s_dtw[2];
  const int cw = threadIdx.x % CT;
  const int jt = threadIdx.x / CT;
  const int64_t col = (int64_t)blockIdx.x * CT + cw;
  const int64_t jbase = g.j0 + (int64_t)blockIdx.y * JT;
  const int64_t j = jbase + jt;
  const bool ok = col < g.m && j < g.j0 + g.jn;
  const uint64_t s = ok ? (sample_word(g.seed, (uint64_t)j) & (uint64_t)(g.r - 1)) : 0;
  const Tin* __restrict__ A = static_cast<const Tin*>(g.A);
  Tc acc = Tc(0);
  for (int64_t i = 0; i < g.p; ++i) {
    __syncthreads();
    if (threadIdx.x == 0) s_dw = sign_word(g.seed, kStreamD, (uint64_t)i, 0);
    if (threadIdx.x == 32) s_dtw[0] = sign_word(g.seed, kStreamDt, (uint64_t)i, (uint64_t)(jbase >> 6));
    if (threadIdx.x == 64)
      s_dtw[1] = sign_word(g.seed, kStreamDt, (uint64_t)i, (uint64_t)((jbase + JT - 1) >> 6));
    __syncthreads();
    const int64_t rows_i = min(g.rb, g.n - i * g.rb);
    if (!ok || rows_i <= 0) continue;
    Tc part = Tc(0);
    for (int64_t k = 0; k < rows_i; ++k) {
      const Tc x = load_as<Tc>(A + (i * g.rb + k) * g.lda + col);
      const uint32_t neg = (uint32_t)((__popcll((unsigned long long)(s & (uint64_t)k)) +
                                       (int)((s_dw >> k) & 1ull)) & 1);
      part += flip(x, neg);
    }
    const uint64_t dtw = ((j >> 6) == (jbase >> 6)) ? s_dtw[0] : s_dtw[1];
    acc += flip(part, (uint32_t)((dtw >> (j & 63)) & 1ull));
  }
  if (ok) out[j * ldo + col] = (Tout)(acc * scale);
}

}  // namespace bsrht
