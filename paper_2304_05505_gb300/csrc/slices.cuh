// Fixed-point fp16 slices of the tensor-core operands (the operand
// preparation kernels and the converter warps of the GEMM).
//
// A value x of a row with exponent e (|x| <= 2^e) is written as
//   x = 2^(e - 7) (S0 + 2^-11 S1 + 2^-22 S2),
//   y = 2^(7 - e) x,  S0 = rint(y),  S1 = rint(2^11 (y - S0)),  S2 = rint(2^22 (y - S0) - 2^11 S1)
// with integers S0 in [-128, 128] (|S0| may reach 255 when |x| slightly exceeds
// 2^e) and S1, S2 in [-1024, 1024].  The planes hold P0 = 2^8 S0, P1 = 2^-3 S1
// and P2 = 2^-14 S2: each is zero or a normal fp16 number (at most 65280, at
// least 2^-14 in magnitude) with at most 11 significant bits, so exact.  Every
// step is exact in FP32 for |y| <= 2^22.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

// The three planes of y = 2^(7 - e) x as FP32 values P0, P1, P2 (exact fp16
// numbers).  Each rounding to a multiple of 2^-11 k is an add and a subtract
// of 1.5 * 2^(23 - 11 k) (to nearest, ties to even, exact for these
// magnitudes), and each remainder is exact.
__device__ __forceinline__ void slice3_planes(float y, float* p) {
  const float s0 = __fsub_rn(__fadd_rn(y, 0x1.8p23f), 0x1.8p23f);   // rint(y)
  float r = __fsub_rn(y, s0);                                         // |r| <= 1/2
  const float s1 = __fsub_rn(__fadd_rn(r, 0x1.8p12f), 0x1.8p12f);   // r to a multiple of 2^-11
  r = __fsub_rn(r, s1);                                               // |r| <= 2^-12
  const float s2 = __fsub_rn(__fadd_rn(r, 0x1.8p1f), 0x1.8p1f);     // r to a multiple of 2^-22
  p[0] = s0 * 256.0f;
  p[1] = s1 * 256.0f;
  p[2] = s2 * 256.0f;
}

// The same for y + l with |l| far below the leading slice's unit: the
// leading slice is rint(y), and l joins the first remainder before it is
// rounded to the second and third slices.
__device__ __forceinline__ void slice3_planes_x(float y, float l, float* p) {
  const float s0 = __fsub_rn(__fadd_rn(y, 0x1.8p23f), 0x1.8p23f);
  float r = __fadd_rn(__fsub_rn(y, s0), l);
  const float s1 = __fsub_rn(__fadd_rn(r, 0x1.8p12f), 0x1.8p12f);
  r = __fsub_rn(r, s1);
  const float s2 = __fsub_rn(__fadd_rn(r, 0x1.8p1f), 0x1.8p1f);
  p[0] = s0 * 256.0f;
  p[1] = s1 * 256.0f;
  p[2] = s2 * 256.0f;
}

// The fp16 bits of the three planes of x with row exponent e.  The scale
// 2^(7 - e) is an exact power of two built from its exponent bits.
__device__ __forceinline__ void slice3(float x, int e, uint16_t* s) {
  const int sh = 7 - e;
  const float y = (sh >= -126 && sh <= 127) ? x * __int_as_float((sh + 127) << 23) : ldexpf(x, sh);
  float p[3];
  slice3_planes(y, p);
#pragma unroll
  for (int k = 0; k < 3; k++) s[k] = __half_as_ushort(__float2half_rn(p[k]));
}

// The slices of -x, from those of x (rint is odd: only the signs flip).
__device__ __forceinline__ void negate3(const uint16_t* s, uint16_t* n) {
#pragma unroll
  for (int p = 0; p < 3; p++) n[p] = s[p] ^ 0x8000u;
}

// The smallest e with m < 2^e (0 for m = 0).
__device__ __forceinline__ int row_exponent(double m) {
  if (!(m > 0.0)) return 0;
  int e;
  frexp(m, &e);
  return e;
}

// Plane p of a complex element at base + p * plane + off: (re, im) as one word.
__device__ __forceinline__ void store3(uint16_t* base, long plane, long off, const uint16_t* re,
                                       const uint16_t* im) {
#pragma unroll
  for (int p = 0; p < 3; p++)
    *reinterpret_cast<uint32_t*>(base + p * plane + off) = (uint32_t)re[p] | ((uint32_t)im[p] << 16);
}
