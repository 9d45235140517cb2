// Fixed-point bf16 slices of the tensor-core operands (the operand
// preparation kernels: rows of X, Psi and M, and the embedded B operands).
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

// FP32 form.  The scale 2^(7 - e) is an exact power of two built from its
// exponent bits, and slice p, rint(y_p) 2^-8p, is the remainder rounded to a
// multiple of 2^-8p by adding and subtracting 1.5 * 2^(23 - 8p) (to nearest,
// ties to even, exact for |y| <= 255); each remainder is exact.  These are
// the slices of the steps above, bit for bit, without rint, ldexp or a bf16
// conversion: a slice of at most 8 significant bits is its FP32 top half.
__device__ __forceinline__ void slice4(float x, int e, uint16_t* s) {
  const int sh = 7 - e;
  float y = (sh >= -126 && sh <= 127) ? x * __int_as_float((sh + 127) << 23) : ldexpf(x, sh);
  const float magic[4] = {0x1.8p23f, 0x1.8p15f, 0x1.8p7f, 0x1.8p-1f};
#pragma unroll
  for (int p = 0; p < 4; p++) {
    const float sp = __fsub_rn(__fadd_rn(y, magic[p]), magic[p]);
    s[p] = (uint16_t)(__float_as_uint(sp) >> 16);
    y = __fsub_rn(y, sp);
  }
}

// The slices of -x, from those of x (rint is odd: only the signs flip).
__device__ __forceinline__ void negate4(const uint16_t* s, uint16_t* n) {
#pragma unroll
  for (int p = 0; p < 4; p++) n[p] = s[p] ^ 0x8000u;
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
