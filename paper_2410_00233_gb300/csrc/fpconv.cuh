// Exact IEEE-754 binary32 <-> binary64 conversions in integer arithmetic.
//
// On GB300 a float <-> double conversion instruction issues to the FP64 pipe and costs as
// much as a DADD (measured with dependent chains: FMUL + convert + DADD runs at half the
// rate of FMUL + DADD fed by a bit-built double).  The split Bregman vector kernels are
// bound by that pipe, so the conversions they make per element (the FP32 apply outputs
// widened to FP64, the FP64 vectors rounded to FP32 for their TF32 split planes) are done
// here on the integer pipes.  Both functions return exactly the bits of the hardware
// conversions (round to nearest, ties to even, for binary64 -> binary32; subnormals, signed
// zeros and infinities included; NaN maps to a NaN), which kpsb_conversion_check verifies
// on the device over every binary32 value and over random and tie-case binary64 values.
#pragma once

#include <cuda_runtime.h>
#ifndef __CUDA_ARCH__
#include <string.h>
#endif

namespace kpsb {

// Bit moves: the device intrinsics, or byte copies on the host (where the same functions
// are compiled to check them against the host's IEEE conversions).
__host__ __device__ __forceinline__ unsigned fpc_f2u(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ float fpc_u2f(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, sizeof f);
  return f;
#endif
}
__host__ __device__ __forceinline__ double fpc_hilo2d(unsigned hi, unsigned lo) {
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const unsigned long long b = ((unsigned long long)hi << 32) | lo;
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
#endif
}
__host__ __device__ __forceinline__ unsigned fpc_d2hi(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2hiint(d);
#else
  unsigned long long b;
  memcpy(&b, &d, sizeof b);
  return (unsigned)(b >> 32);
#endif
}
__host__ __device__ __forceinline__ unsigned fpc_d2lo(double d) {
#ifdef __CUDA_ARCH__
  return (unsigned)__double2loint(d);
#else
  unsigned long long b;
  memcpy(&b, &d, sizeof b);
  return (unsigned)b;
#endif
}
__host__ __device__ __forceinline__ int fpc_clz(unsigned x) {  // x != 0
#ifdef __CUDA_ARCH__
  return __clz((int)x);
#else
  int n = 0;
  while (!(x & 0x80000000u)) {
    x <<= 1;
    ++n;
  }
  return n;
#endif
}

// binary32 -> binary64, exact.
__host__ __device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = fpc_f2u(f);
  const unsigned s = u & 0x80000000u;
  const unsigned ex = (u >> 23) & 0xffu;
  const unsigned m = u & 0x7fffffu;
  if (ex - 1u < 254u)  // normal: rebias the exponent (1023 - 127 = 896), widen the fraction
    return fpc_hilo2d(s | ((ex + 896u) << 20) | (m >> 3), m << 29);
  if (ex == 0xffu)  // infinity or NaN (payload kept)
    return fpc_hilo2d(s | 0x7ff00000u | (m >> 3), m << 29);
  if (m == 0u) return fpc_hilo2d(s, 0u);  // signed zero
  // subnormal m * 2^-149: leading bit at position p (0..22) -> value 2^(p-149) * 1.f
  const int p = 31 - fpc_clz(m);
  const unsigned long long fr = ((unsigned long long)m << (52 - p)) & 0xfffffffffffffull;
  return fpc_hilo2d(s | ((unsigned)(p + 874) << 20) | (unsigned)(fr >> 32), (unsigned)fr);
}

// binary64 -> binary32, round to nearest, ties to even.
__host__ __device__ __forceinline__ float d2f_rn_bits(double d) {
  const unsigned hi = fpc_d2hi(d), lo = fpc_d2lo(d);
  const unsigned s = hi & 0x80000000u;
  const int ex = (int)((hi >> 20) & 0x7ffu);
  const int e = ex - 896;  // binary32 biased exponent of the value
  if (e > 0 && e < 255) {
    // 23 kept fraction bits: the high word's 20 and the low word's top 3; 29 dropped bits
    const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    unsigned r = ((unsigned)e << 23) | mant;
    r += (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) ? 1u : 0u;  // carry may reach inf
    return fpc_u2f(s | r);
  }
  if (ex == 0x7ff) {
    const bool nan = (hi & 0xfffffu) != 0u || lo != 0u;
    return fpc_u2f(s | 0x7f800000u | (nan ? 0x00400000u | ((hi & 0xfffffu) << 3) | (lo >> 29) : 0u));
  }
  if (e >= 255) return fpc_u2f(s | 0x7f800000u);  // overflow
  if (e < -23) return fpc_u2f(s);  // below half the smallest subnormal (or zero)
  // binary32 subnormal: the 53-bit significand shifted right by 30 - e, rounded
  const unsigned long long sig = (((unsigned long long)(hi & 0xfffffu) << 32) | lo) | (1ull << 52);
  const int sh = 30 - e;  // 30 .. 53
  const unsigned long long q = sig >> sh, rem = sig & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  const unsigned r = (unsigned)q + ((rem > half || (rem == half && (q & 1ull))) ? 1u : 0u);
  return fpc_u2f(s | r);  // a carry into bit 23 gives the smallest normal
}

}  // namespace kpsb
