// Conversions between IEEE 754 binary32 and binary64, done as integer
// arithmetic on the two encodings (sign bit, biased exponent: 8 bits with bias
// 127 / 11 bits with bias 1023, fraction: 23 / 52 bits).
//
// GB300 executes the FP32 <-> FP64 conversion instructions on its FP64 pipe,
// which runs at about 1/64 of the FP32 rate. The FP64 tail of the M-step
// (finalize, start) converts about 60 values per superpixel, so these
// conversions take an important part of that pipe. The integer forms below
// run on the integer pipes and give the same bits as the hardware:
//  * widen_bits: exact. Every binary32 value is a binary64 value. Subnormal
//    inputs are left to the caller (false).
//  * narrow_bits: rounds to nearest, ties to even. It handles zeros and
//    magnitudes in [2^-126, 2^128), including a rounding carry into the
//    exponent (which takes magnitudes just below 2^128 to infinity). It
//    returns false for other nonzero magnitudes and for infinities and NaNs,
//    which the caller converts with the hardware instruction.
//
// Pure integer code: the host test suite checks both against the C casts.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define GMMSP_FPCONV_FN __host__ __device__ __forceinline__
#else
#define GMMSP_FPCONV_FN inline
#endif

namespace gmmsp {

// binary32 encoding b -> binary64 encoding (hi, lo words).
GMMSP_FPCONV_FN bool widen_bits(uint32_t b, uint32_t& hi, uint32_t& lo) {
  const uint32_t e = (b >> 23) & 0xffu, f = b & 0x7fffffu;
  if (e == 0u && f != 0u) return false;  // subnormal
  const uint32_t ed = e == 0u ? 0u : (e == 0xffu ? 0x7ffu : e + 896u);  // 1023 - 127 = 896
  hi = (b & 0x80000000u) | (ed << 20) | (f >> 3);
  lo = f << 29;
  return true;
}

// binary64 encoding (hi, lo words) -> binary32 encoding, nearest even;
// false outside zero and [2^-126, 2^128) in magnitude.
GMMSP_FPCONV_FN bool narrow_bits(uint32_t hi, uint32_t lo, uint32_t& out) {
  const uint32_t sign = hi & 0x80000000u, e = (hi >> 20) & 0x7ffu;
  if (e == 0u && ((hi & 0xfffffu) | lo) == 0u) {  // +-0
    out = sign;
    return true;
  }
  if (e - 897u > 253u) return false;  // binary32 exponent field 1..254 before rounding
  // exponent and the top 23 fraction bits; the 29 dropped bits decide the rounding
  uint32_t r = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1fffffffu, half = 0x10000000u;
  r += (rest > half || (rest == half && (r & 1u))) ? 1u : 0u;
  out = sign | r;
  return true;
}

#if defined(__CUDACC__)
__device__ __forceinline__ double widen(float x) {
  uint32_t hi, lo;
  if (!widen_bits(__float_as_uint(x), hi, lo)) return double(x);
  return __hiloint2double(int(hi), int(lo));
}

__device__ __forceinline__ float narrow(double x) {
  uint32_t out;
  if (!narrow_bits(uint32_t(__double2hiint(x)), uint32_t(__double2loint(x)), out)) return __double2float_rn(x);
  return __uint_as_float(out);
}

// The conversions of the templated M-step arithmetic: identity for float.
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(double x) { return narrow(x); }
template <typename T> __device__ __forceinline__ T from_f32(float x);
template <> __device__ __forceinline__ float from_f32<float>(float x) { return x; }
template <> __device__ __forceinline__ double from_f32<double>(float x) { return widen(x); }
#endif

}  // namespace gmmsp
