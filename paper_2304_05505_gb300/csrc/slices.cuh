// Fixed-point bf16 slices of the tensor-core operands (shared by the operand
// preparation and by the k-convolution, which writes M directly as slices).
//
// A value x of a row with exponent e (|x| <= 2^e) is written as
//   x = 2^(e - 7) (P0 + P1 + P2 + P3),  P_s = 2^(-8 s) S_s,
//   y0 = 2^(7 - e) x,  S_s = rint(y_s),  y_{s+1} = 2^8 (y_s - S_s)
// with integer S_s in [-128, 128] (|S_0| may reach 255 when |x| slightly
// exceeds 2^e, which stays exact in bf16).  Every step is exact in the
// working precision.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

__device__ __forceinline__ void slice4(double x, int e, uint16_t* s) {
  double y = ldexp(x, 7 - e);
#pragma unroll
  for (int p = 0; p < 4; p++) {
    const double sp = rint(y);
    s[p] = __bfloat16_as_ushort(__float2bfloat16_rn(ldexpf((float)sp, -8 * p)));   // exact, |sp| <= 255
    y = (y - sp) * 256.0;
  }
}

__device__ __forceinline__ void slice4(float x, int e, uint16_t* s) {
  float y = ldexpf(x, 7 - e);
#pragma unroll
  for (int p = 0; p < 4; p++) {
    const float sp = rintf(y);
    s[p] = __bfloat16_as_ushort(__float2bfloat16_rn(ldexpf(sp, -8 * p)));
    y = (y - sp) * 256.0f;
  }
}

// The smallest e with m < 2^e (0 for m = 0).
__device__ __forceinline__ int row_exponent(double m) {
  if (!(m > 0.0)) return 0;
  int e;
  frexp(m, &e);
  return e;
}

// Plane p of a complex element at base + p * plane + off: (re, im) as one word.
__device__ __forceinline__ void store4(uint16_t* base, long plane, long off, const uint16_t* re,
                                       const uint16_t* im) {
#pragma unroll
  for (int p = 0; p < 4; p++)
    *reinterpret_cast<uint32_t*>(base + p * plane + off) = (uint32_t)re[p] | ((uint32_t)im[p] << 16);
}
