// Packed FP32 pairs (sm_100 family): two IEEE single-precision lanes in one
// 64-bit register, added, subtracted, multiplied or fused-multiply-added lane
// by lane with round-to-nearest-even by one instruction.  Each lane rounds exactly like the scalar
// instruction, so results are bit-identical to scalar code performing the
// same operations.  The low 32 bits hold the element at the lower address:
// a 64-bit shared-memory load of two adjacent floats yields the packed pair,
// and the pair is stored back from the same register pair.
#pragma once

namespace bsrht {

using f2 = unsigned long long;

__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// a * b + c, lane by lane, one rounding.
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ float2 f2_to_float2(f2 v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}

// Both lanes set to v.
__device__ __forceinline__ f2 f2_splat(float v) {
  f2 d;
  asm("mov.b64 %0, {%1, %1};" : "=l"(d) : "f"(v));
  return d;
}

// In-register Walsh-Hadamard transform of N packed pairs (natural order,
// unnormalised): the butterflies of the scalar transform, in the same
// order, on both lanes at once.
template <int N>
__device__ __forceinline__ void fwht_regs2(f2 (&v)[N]) {
#pragma unroll
  for (int h = 1; h < N; h <<= 1) {
#pragma unroll
    for (int e = 0; e < N; ++e) {
      if ((e & h) == 0) {
        const f2 x = v[e], y = v[e + h];
        v[e] = f2_add(x, y);
        v[e + h] = f2_sub(x, y);
      }
    }
  }
}

}  // namespace bsrht
