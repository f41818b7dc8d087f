// FP64 <-> FP32 conversions by integer operations, and double-single (FP32 pair) arithmetic.
//
// On this GPU every FP64 instruction, the FP64 <-> FP32 conversions included, issues on the narrow FP64 pipe,
// while the integer and FP32 pipes are ~30-75 times wider.  The kernels of the mixed-precision inner solves move
// FP64 data into FP32 pairs and back on every pass, so the conversions are written here with integer operations
// on the IEEE 754 bit fields: a FP64 value is sign | 11-bit exponent (bias 1023) | 52-bit fraction, a FP32 value
// sign | 8-bit exponent (bias 127) | 23-bit fraction, both with an implicit leading 1 for normal numbers.
//
// The header is plain C++ as well (host bit casts through memcpy), so the conversions are tested on the host.
#pragma once
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define FETIRP_HD __host__ __device__ __forceinline__
#else
#define FETIRP_HD inline
#endif

namespace fetirp {

FETIRP_HD uint64_t bits64(double v) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t b;
  std::memcpy(&b, &v, 8);
  return b;
#endif
}
FETIRP_HD double from_bits64(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double v;
  std::memcpy(&v, &b, 8);
  return v;
#endif
}
FETIRP_HD uint32_t bits32(float v) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(v);
#else
  uint32_t b;
  std::memcpy(&b, &v, 4);
  return b;
#endif
}
FETIRP_HD float from_bits32(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float v;
  std::memcpy(&v, &b, 4);
  return v;
#endif
}

// FP64 -> FP32 with rounding to nearest, ties to even (the conversion instruction's rounding), integer operations
// only.  Values whose magnitude is in the FP32 normal range give the same result as the conversion instruction;
// smaller magnitudes (zeros, FP32-subnormal and FP64-subnormal values) give a zero of the same sign, larger ones
// (and those that round up past FLT_MAX) the infinity of that sign; NaN gives a quiet NaN.
FETIRP_HD float d2f_rn(double v) {
  const uint64_t b = bits64(v);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t sign = hi & 0x80000000u;
  const uint32_t ex = (hi >> 20) & 0x7ffu;                          // FP64 biased exponent
  // exponent rebiased to FP32 (1023 - 127 = 896) and the top 23 fraction bits: 20 from hi, 3 from lo
  uint32_t mag = (((hi & 0x7fffffffu) - (896u << 20)) << 3) | (lo >> 29);
  // the 29 dropped fraction bits decide the rounding; a carry out of the fraction moves into the exponent
  const uint32_t dropped = lo & 0x1fffffffu, half = 0x10000000u;
  mag += (dropped > half || (dropped == half && (mag & 1u))) ? 1u : 0u;
  uint32_t f = sign | mag;
  if (ex <= 896u) f = sign;                                           // below the FP32 normal range
  if (ex >= 1151u) f = sign | 0x7f800000u;                            // above it (and infinities)
  if (ex == 0x7ffu && ((hi & 0xfffffu) | lo) != 0u) f = 0x7fc00000u;  // NaN
  return from_bits32(f);
}

// FP32 -> FP64, exact.  Normal values and zeros by integer operations; FP32-subnormal values, infinities and
// NaN (rare here) through the conversion instruction.
FETIRP_HD double f2d(float f) {
  const uint32_t b = bits32(f);
  const uint32_t ex = (b >> 23) & 0xffu;
  if (ex == 0u || ex == 0xffu) {
    if ((b & 0x7fffffffu) == 0u) return from_bits64((uint64_t)(b & 0x80000000u) << 32);
    return (double)f;
  }
  // exponent rebiased to FP64 (+896), 23 fraction bits moved to the top of the 52
  const uint32_t hi = (b & 0x80000000u) | (((b & 0x7fffffffu) >> 3) + (896u << 20));
  return from_bits64(((uint64_t)hi << 32) | ((uint64_t)(b & 7u) << 29));
}

// FP64 -> unevaluated FP32 pair, v ~ h + l: h = d2f_rn(v), l = d2f_rn(v - h) with the difference formed exactly
// in FP64 (one FP64 add, the only FP64 instruction); the same pair as the conversion instructions give.
// |v - (h + l)| <= 2^-48 |v| while l stays in the FP32 normal range (|v| >= 2^-78 or so); below that l is
// flushed to zero and the pair keeps h's 2^-24.
FETIRP_HD void d2ds(double v, float& h, float& l) {
  h = d2f_rn(v);
  l = d2f_rn(v - f2d(h));
}

// -v when neg, v otherwise, by flipping the sign bit (no FP64 instruction)
FETIRP_HD double neg_if(double v, bool neg) { return from_bits64(bits64(v) ^ ((uint64_t)neg << 63)); }
FETIRP_HD float neg_if(float v, bool neg) { return from_bits32(bits32(v) ^ ((uint32_t)neg << 31)); }
// v == +0 or -0, tested on the bits (no FP64 instruction)
FETIRP_HD bool is_zero(double v) { return (bits64(v) << 1) == 0u; }

// FP32 pair -> FP64 (one FP64 add)
FETIRP_HD double ds2d(float h, float l) { return f2d(h) + f2d(l); }

// Conversions for code templated on FP32 / FP64 storage: FP64 -> T and T -> FP64
template <typename T>
FETIRP_HD T from_f64(double v) {
  if constexpr (sizeof(T) == 4) return d2f_rn(v);
  else return v;
}
FETIRP_HD double to_f64(float v) { return f2d(v); }
FETIRP_HD double to_f64(double v) { return v; }

}  // namespace fetirp
