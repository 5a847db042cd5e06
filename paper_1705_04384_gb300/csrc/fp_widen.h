// Exact widening of an IEEE-754 binary32 value to binary64 with integer operations.
//
// On GB300 the conversion instruction from FP32 to FP64 runs on the FP64 unit, whose
// rate (about 0.5 operations per clock per SM sub-partition) is the bottleneck of the
// kernels that read the precision form's FP32 vectors; the same result can be formed
// from the bit fields on the integer units.  From the binary32 layout (sign s, biased
// exponent e in 8 bits, fraction f in 23 bits) and the binary64 layout (exponent bias 1023
// instead of 127, 52 fraction bits):
//   normal     (0 < e < 255):  exponent e + 896, fraction f << 29;
//   zero       (e = 0, f = 0): a signed zero;
//   subnormal  (e = 0, f > 0): value f 2^-149 = 1.g 2^(t - 149) with t the position of
//                              f's leading one: exponent t + 874, fraction f << (52 - t)
//                              with the leading one removed;
//   inf / NaN  (e = 255):      exponent 2047, fraction f << 29.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define IGA_HD __host__ __device__ __forceinline__
#else
#define IGA_HD inline
#endif

namespace iga {

IGA_HD int leading_one_position(uint32_t x) {  // x != 0
#ifdef __CUDA_ARCH__
  return 31 - __clz(x);
#else
  int t = 31;
  while (!((x >> t) & 1u)) --t;
  return t;
#endif
}

IGA_HD uint64_t widen_f32_bits(uint32_t u) {
  const uint64_t sign = (uint64_t)(u >> 31) << 63;
  const uint32_t e = (u >> 23) & 0xffu, f = u & 0x7fffffu;
  if (e != 0 && e != 0xffu) return sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)f << 29);
  if (e == 0xffu) return sign | (0x7ffull << 52) | ((uint64_t)f << 29);
  if (f == 0) return sign;
  const int t = leading_one_position(f);  // 0 .. 22
  const uint64_t frac = ((uint64_t)f << (52 - t)) & ((1ull << 52) - 1);
  return sign | ((uint64_t)(t + 874) << 52) | frac;
}

IGA_HD double widen_f32(float x) {
  uint32_t u;
  uint64_t d;
  double r;
#ifdef __CUDA_ARCH__
  u = __float_as_uint(x);
  d = widen_f32_bits(u);
  r = __longlong_as_double((long long)d);
#else
  std::memcpy(&u, &x, 4);
  d = widen_f32_bits(u);
  std::memcpy(&r, &d, 8);
#endif
  return r;
}

}  // namespace iga
