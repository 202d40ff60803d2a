// Exact conversions between IEEE 754 binary32 and binary64 with integer operations only. On this
// part a hardware conversion between FP32 and FP64 issues at the FP64 pipe's rate (1/64 of FP32),
// so the kernels widen and narrow on the integer pipe instead. Both functions restate the formats'
// definitions (sign, biased exponent, mantissa) and build for the host too, where a test compares
// them bit for bit with the host's own conversions.
#pragma once

#include <cstring>

#ifndef __CUDACC__  // a host-only build (the conversion test)
#define __host__
#define __device__
#endif

namespace mdk {

__host__ __device__ inline unsigned fc_f2u(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  std::memcpy(&u, &f, sizeof u);
  return u;
#endif
}

__host__ __device__ inline float fc_u2f(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, sizeof f);
  return f;
#endif
}

__host__ __device__ inline unsigned fc_hi(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2hiint(d);
#else
  unsigned long long b;
  std::memcpy(&b, &d, sizeof b);
  return (unsigned)(b >> 32);
#endif
}

__host__ __device__ inline unsigned fc_lo(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2loint(d);
#else
  unsigned long long b;
  std::memcpy(&b, &d, sizeof b);
  return (unsigned)b;
#endif
}

__host__ __device__ inline double fc_hilo(unsigned hi, unsigned lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const unsigned long long b = ((unsigned long long)hi << 32) | lo;
  double d;
  std::memcpy(&d, &b, sizeof d);
  return d;
#endif
}

// leading zeros of a nonzero 32-bit word
__host__ __device__ inline int fc_clz(unsigned m) {
#ifdef __CUDA_ARCH__
  return __clz(m);
#else
  return __builtin_clz(m);
#endif
}

// FP32 -> FP64, exact: sign kept, exponent rebiased by 1023 - 127 = 896, mantissa moved up by 29
// bits; zero, subnormals (renormalised), infinities and NaNs by their own cases
__host__ __device__ inline double widen_f32(float f) {
  const unsigned u = fc_f2u(f);
  const unsigned sgn = u & 0x80000000u, m = u & 0x7fffffffu;
  unsigned hi, lo;
  if (m - 0x00800000u < 0x7f000000u) {  // normal: biased exponent in [1, 254]
    hi = sgn | ((m >> 3) + (896u << 20));
    lo = m << 29;
  } else if (m == 0u) {
    hi = sgn;
    lo = 0u;
  } else if (m >= 0x7f800000u) {        // infinity or NaN: all-ones exponent
    hi = sgn | 0x7ff00000u | ((m & 0x007fffffu) >> 3);
    lo = m << 29;
  } else {                              // subnormal: m * 2^-149, normalised
    const int sh = fc_clz(m) - 8;       // moves the leading bit to bit 23
    const unsigned mn = (m << sh) & 0x007fffffu;
    hi = sgn | ((unsigned)(897 - sh) << 20) | (mn >> 3);
    lo = mn << 29;
  }
  return fc_hilo(hi, lo);
}

// FP64 -> FP32, rounded to nearest, ties to even: the 23 leading mantissa bits, plus one unit when
// the 29 dropped bits are above half a unit, or exactly half with the kept last bit odd (a carry out
// of the mantissa raises the exponent, as it should). Results below the FP32 normal range (zero
// among them) or in the top two binades go to the built-in conversion: never for the cell-local
// offsets the kernels narrow, except an exact zero.
__host__ __device__ inline float narrow_f64(double d) {
  const unsigned hi = fc_hi(d), lo = fc_lo(d);
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;  // the FP32 biased exponent
  if (e <= 0 || e >= 254) return (float)d;
  const unsigned m = ((hi & 0x000fffffu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1fffffffu, half = 0x10000000u;
  unsigned bits = ((unsigned)e << 23) + m;
  if (rest > half || (rest == half && (m & 1u))) bits += 1u;
  return fc_u2f((hi & 0x80000000u) | bits);
}

}  // namespace mdk
