// Shared device helpers: Philox4x64-10, element-type traits, status macros.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bsrht.h"

namespace bsrht {

// ---------------------------------------------------------------- Philox
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 64x64->128-bit multiplications whose halves are xored with the other
// counter words and the key; the key is bumped by two Weyl constants
// between rounds.
struct U64x4 {
  uint64_t x, y, z, w;
};

constexpr uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t kPhiloxM1 = 0xCA5A826395121157ull;
constexpr uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kPhiloxW1 = 0xBB67AE8584CAA73Bull;

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ U64x4 philox4x64_10(U64x4 c, uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    const uint64_t hi0 = mulhi64(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint64_t hi1 = mulhi64(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    U64x4 o;
    o.x = hi1 ^ c.y ^ k0;
    o.y = lo1;
    o.z = hi0 ^ c.w ^ k1;
    o.w = lo0;
    c = o;
  }
  return c;
}

// Streams of the block SRHT randomness (third counter word).
constexpr uint64_t kStreamD = 0;   // D^(i) signs, indexed by local row k
constexpr uint64_t kStreamDt = 1;  // Dt^(i) signs, indexed by sketch row j
constexpr uint64_t kStreamR = 2;   // shared row samples s_j

__host__ __device__ __forceinline__ uint64_t pick(const U64x4& v, int w) {
  return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
}

// 64 sign bits (bit b set = -1) of indices [64*word, 64*word+64) of one
// (stream, block) pair: counter (word>>2, block, stream, 0), output word&3.
__host__ __device__ __forceinline__ uint64_t sign_word(uint64_t seed, uint64_t stream,
                                                       uint64_t block, uint64_t word) {
  U64x4 c{word >> 2, block, stream, 0};
  return pick(philox4x64_10(c, seed, 0), (int)(word & 3));
}

// Row sample s_j of the shared R (before reduction mod r).
__host__ __device__ __forceinline__ uint64_t sample_word(uint64_t seed, uint64_t j) {
  U64x4 c{j >> 2, 0, kStreamR, 0};
  return pick(philox4x64_10(c, seed, 0), (int)(j & 3));
}

// ---------------------------------------------------------------- types
template <typename T>
struct Elem;
template <>
struct Elem<double> {
  __device__ __forceinline__ static double to_f64(double v) { return v; }
  __device__ __forceinline__ static float to_f32(double v) { return (float)v; }
};
template <>
struct Elem<float> {
  __device__ __forceinline__ static double to_f64(float v) { return v; }
  __device__ __forceinline__ static float to_f32(float v) { return v; }
};
template <>
struct Elem<__nv_bfloat16> {
  __device__ __forceinline__ static double to_f64(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ __forceinline__ static float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
};
template <>
struct Elem<__half> {
  __device__ __forceinline__ static double to_f64(__half v) { return __half2float(v); }
  __device__ __forceinline__ static float to_f32(__half v) { return __half2float(v); }
};

template <typename Tc, typename Tin>
__device__ __forceinline__ Tc load_as(const Tin* p) {
  Tin v = __ldg(p);
  if constexpr (sizeof(Tc) == 8)
    return Elem<Tin>::to_f64(v);
  else
    return Elem<Tin>::to_f32(v);
}
template <typename Tc>
__device__ __forceinline__ Tc flip(Tc v, uint32_t neg) {
  return neg ? -v : v;
}

__host__ __device__ constexpr int ilog2c(long long x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }

// Adds k to the library's kernel-launch counter (bsrht_kernel_launches).
void note_launches(int k);

// Internal element-type code for FP32 storage with FP64 arithmetic
// (bsrht_opts.precision = BSRHT_PREC_F64 on BSRHT_F32 data): the sketch runs
// the FP64 integer-transform kernel on FP32 input and writes FP64.
constexpr int kDtypeF32AsF64 = 16;

inline size_t dtype_size(int dt) {
  return dt == BSRHT_F64 ? 8 : (dt == BSRHT_F32 || dt == kDtypeF32AsF64 ? 4 : 2);
}

}  // namespace bsrht

namespace bsrht {
// Reports a failed CUDA call on stderr (file, line, error name) when the
// environment variable BSRHT_DEBUG is set; returns BSRHT_ECUDA.
int cuda_failure(cudaError_t e, const char* file, int line);
}  // namespace bsrht

#define BSRHT_CUDA_TRY(expr)                                                \
  do {                                                                      \
    cudaError_t e_ = (expr);                                                \
    if (e_ != cudaSuccess) return ::bsrht::cuda_failure(e_, __FILE__, __LINE__); \
  } while (0)
