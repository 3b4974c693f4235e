// Conversions to IEEE 754 binary64 assembled from bit patterns with integer
// operations, for host and device code.  On this GPU the FP64 and conversion
// units run at a small fraction of the integer rate, so the per-atom output
// kernels build their doubles this way.  The results are those of the
// round-to-nearest-even conversions (the format's definition: sign, biased
// exponent, 52-bit fraction); tests/test_host_bits.py compares them with the
// host's own conversions.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define RELRES_HD __host__ __device__ __forceinline__
#else
#define RELRES_HD inline
#endif

namespace relres {

RELRES_HD int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll(static_cast<long long>(x));
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

RELRES_HD double double_from_bits(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(static_cast<long long>(b));
#else
  double d;
  std::memcpy(&d, &b, sizeof d);
  return d;
#endif
}

RELRES_HD uint64_t bits_of_double(double d) {
#ifdef __CUDA_ARCH__
  return static_cast<uint64_t>(__double_as_longlong(d));
#else
  uint64_t b;
  std::memcpy(&b, &d, sizeof b);
  return b;
#endif
}

RELRES_HD uint32_t bits_of_float(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(f);
#else
  uint32_t b;
  std::memcpy(&b, &f, sizeof b);
  return b;
#endif
}

// The binary64 nearest to u (ties to even).  The leading one of u is moved
// to bit 63; its top 53 bits are the significand q (the implicit one at bit
// 52) and the 11 below are rounded away.  With q in [2^52, 2^53] the pattern
// is (E - 1) 2^52 + q for the biased exponent E = 1086 - lz: a q rounded up
// to 2^53 carries into the exponent, which is what that value needs.
RELRES_HD uint64_t double_bits_of_u64(uint64_t u) {
  if (u == 0) return 0;
  const int lz = clz64(u);
  const uint64_t m = u << lz;
  uint64_t q = m >> 11;
  const uint64_t rest = m & 0x7ffu;
  if (rest > 0x400u || (rest == 0x400u && (q & 1u))) q += 1u;
  return (static_cast<uint64_t>(1085 - lz) << 52) + q;
}

RELRES_HD double double_of_u64(uint64_t u) { return double_from_bits(double_bits_of_u64(u)); }

// A float as a double (exact): the exponent rebiased (127 -> 1023) and the
// fraction moved up 29 bits; a zero keeps its sign.  Subnormal, infinite and
// NaN inputs take the conversion instruction.
RELRES_HD double double_of_float(float f) {
  const uint32_t b = bits_of_float(f);
  const uint32_t e = (b >> 23) & 0xffu;
  if (e == 0u && (b & 0x7fffffu) == 0u) return double_from_bits(static_cast<uint64_t>(b) << 32);
  if (e == 0u || e == 0xffu) return static_cast<double>(f);
  return double_from_bits((static_cast<uint64_t>(b & 0x80000000u) << 32) | (static_cast<uint64_t>(e + 896u) << 52) |
                          (static_cast<uint64_t>(b & 0x7fffffu) << 29));
}

}  // namespace relres
