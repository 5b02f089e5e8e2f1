// Integer helpers of the FP64-accurate tensor-core GEMM (ec_oz.cu), written for
// both host and device so that the host can check them bit for bit.
//
// On GB300 the FP64 pipe (and every conversion to or from a 64-bit type) retires
// about two results per SM per clock, so the GEMM's epilogue and operand split do
// their exact integer work, and the assembly of IEEE binary64 results, with 32- and
// 64-bit integer instructions instead.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define OZ_HD __host__ __device__ __forceinline__
#else
#define OZ_HD inline
#endif

namespace ec {
namespace oz {

OZ_HD int clz64(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)u);
#else
  return u ? __builtin_clzll(u) : 64;
#endif
}

// Bits of the binary64 nearest to X * 2^sc (round to nearest, ties to even), for
// |X| < 2^63.  Returns false when the result would be subnormal or overflow (the
// caller then takes a slow path); true otherwise with the bits in *out.
OZ_HD bool i64_scaled_to_f64_bits(int64_t X, int sc, uint64_t* out) {
  if (X == 0) {
    *out = 0;
    return true;
  }
  const uint64_t sign = X < 0 ? (1ull << 63) : 0ull;
  const uint64_t u = X < 0 ? (uint64_t)0 - (uint64_t)X : (uint64_t)X;
  int p = 63 - clz64(u);                       // position of the leading one
  uint64_t mant;
  if (p <= 52) {
    mant = u << (52 - p);
  } else {
    const int sh = p - 52;
    uint64_t q = u >> sh;
    const uint64_t rem = u & ((1ull << sh) - 1);
    const uint64_t half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (q & 1ull))) {
      ++q;
      if (q >> 53) {
        q >>= 1;
        ++p;
      }
    }
    mant = q;
  }
  const int be = p + 1023 + sc;
  if (be <= 0 || be >= 2047) return false;
  *out = sign | ((uint64_t)be << 52) | (mant & ((1ull << 52) - 1));
  return true;
}

// Same result without branches on the common path: normalise u = |X| so that its
// leading one sits at bit 63, keep 53 bits, round to nearest even from the 11 bits
// below, and add the biased exponent one below its final value so that a mantissa
// that rounds up to 2^53 carries into the exponent.  Requires X != 0 and a normal
// result; returns false otherwise (the caller then takes a slow path).
OZ_HD bool i64_scaled_to_f64_bits_fast(int64_t X, int sc, uint64_t* out) {
  const uint64_t sign = (uint64_t)X & (1ull << 63);
  const uint64_t u = X < 0 ? (uint64_t)0 - (uint64_t)X : (uint64_t)X;
  const int lz = clz64(u);
  const uint64_t nu = u << (lz & 63);          // leading one at bit 63 (u != 0)
  uint64_t mant = nu >> 11;                    // 53 bits, implicit one at bit 52
  const uint32_t low = (uint32_t)(nu & 0x7FFull);
  mant += (low > 0x400u || (low == 0x400u && (mant & 1ull))) ? 1ull : 0ull;
  const int be = 63 - lz + 1023 + sc;          // biased exponent before a rounding carry
  *out = sign | (((uint64_t)(be - 1) << 52) + mant);
  return u != 0 && be > 0 && be < 2046;
}

// Fixed-point image of a binary64 value against a power-of-two scale: the integer
// F = round(a * 2^(64 - e)) for |a| < 2^(e-1), so |F| < 2^63 (ties away from zero;
// exact whenever a carries no bits below 2^(e-64)).  Returns F.
OZ_HD int64_t f64_to_fixed64(uint64_t bits, int e) {
  const int E = (int)((bits >> 52) & 0x7FF);
  uint64_t m = bits & ((1ull << 52) - 1);
  if (E == 0 && m == 0) return 0;
  int ex;                                     // a = m * 2^ex
  if (E == 0) {
    ex = -1074;
  } else {
    m |= (1ull << 52);
    ex = E - 1075;
  }
  const int shift = ex + 64 - e;              // F = m * 2^shift
  uint64_t mag;
  if (shift >= 0) {
    // |a| < 2^(e-1) keeps shift <= 10 for a normal a (m >= 2^52) and <= 11 for a
    // subnormal one (m < 2^52, a row whose largest entry is subnormal): |F| < 2^63 either way
    mag = shift > 11 ? 0 : (m << shift);
  } else if (shift <= -64) {
    mag = 0;
  } else {
    const int r = -shift;
    mag = (m >> r) + ((m >> (r - 1)) & 1ull);
  }
  return (bits >> 63) ? -(int64_t)mag : (int64_t)mag;
}

// Balanced base-256 digits of a fixed-point value |F| < 2^63:
//   F = sum_{s=0}^{7} d_s 256^(7-s),  |d_s| <= 128  (d_0 carries the top bits).
OZ_HD void digits8(int64_t F, int* d) {
  const bool neg = F < 0;
  uint64_t u = neg ? (uint64_t)0 - (uint64_t)F : (uint64_t)F;
  for (int s = 7; s >= 1; --s) {
    const int low = (int)(u & 255u);
    u >>= 8;
    int v = low;
    if (low > 128) {
      v = low - 256;
      ++u;
    }
    d[s] = neg ? -v : v;
  }
  d[0] = neg ? -(int)u : (int)u;
}

// Exponent e with |a| < 2^(e-1) for the largest magnitude of a row (0 for a zero row),
// from the bits of that magnitude (a non-negative binary64).
OZ_HD int row_exponent(uint64_t maxbits) {
  if (maxbits == 0) return 0;
  const int E = (int)((maxbits >> 52) & 0x7FF);
  // value < 2^(E - 1022) for normals (mantissa < 2), < 2^-1022 for subnormals
  const int top = (E == 0) ? -1022 : E - 1022;
  return top + 1;
}

}  // namespace oz
}  // namespace ec
