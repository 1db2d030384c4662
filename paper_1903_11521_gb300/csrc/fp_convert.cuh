// binary32 <-> binary64 conversions on the integer units.
//
// On GB300 a float <-> double conversion issues on the FP64 pipe (2 operations per clock
// per SM, the rate of a DFMA), so the reduced-precision kernels, which convert every
// operand entering or leaving their binary64 accumulations, spend a large share of their
// FP64 budget on conversions.  These helpers do the same conversions with integer
// operations from the IEEE 754 layouts (sign | exponent | fraction; binary32 bias 127,
// binary64 bias 1023):
//   f2d: exact for normal floats: the fraction is widened by 29 bits and the exponent
//        re-biased (+896); zeros stay signed zeros, infinities and NaNs keep their class;
//        subnormal floats (below 2^-126) flush to a signed zero.
//   d2f: round to nearest, ties to even, on the 29 dropped fraction bits; results whose
//        magnitude is below the smallest normal float flush to a signed zero, overflow
//        gives infinity, NaN stays NaN.
// Both are branch-free (selects only): they sit in fully unrolled kernel code, where a
// branch would split the schedule.  The kernels' values never come near 2^-126 (their
// magnitudes follow the DOFs, the flush matches flush-to-zero arithmetic).  Both are
// checked against the hardware conversions by yt_selftest_conversions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace yt {

__device__ __forceinline__ double f2d_int(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t a = u & 0x7FFFFFFFu;
  const uint32_t s = u ^ a;
  uint32_t hi = s | ((a >> 3) + (896u << 20));
  uint32_t lo = a << 29;
  hi = (a >= 0x7F800000u) ? (hi | 0x7FF00000u) : hi;     // infinity, NaN
  hi = (a < 0x00800000u) ? s : hi;                        // zero, subnormal: signed zero
  lo = (a < 0x00800000u) ? 0u : lo;
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float d2f_int(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  const uint32_t ah = hi & 0x7FFFFFFFu;
  const uint32_t s = hi ^ ah;
  const int e = (int)(ah >> 20) - 896;                    // binary32 biased exponent
  const uint32_t m = ((ah & 0xFFFFFu) << 3) | (lo >> 29);
  const uint32_t r = lo & 0x1FFFFFFFu;                    // dropped bits; half = 0x10000000
  uint32_t u = ((uint32_t)e << 23) + m;
  u += (r > 0x10000000u || (r == 0x10000000u && (m & 1u))) ? 1u : 0u;
  const bool nan = ah > 0x7FF00000u || (ah == 0x7FF00000u && lo != 0u);
  u = (e >= 255) ? (nan ? 0x7FC00000u : 0x7F800000u) : u;
  u = (e <= 0) ? 0u : u;
  return __uint_as_float(s | u);
}

}  // namespace yt
