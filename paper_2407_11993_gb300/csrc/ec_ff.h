// Compensated FP32 ("float-float") helpers shared by the kernels that move FP64 work
// onto GB300's FP32 pipe: an FP64 value is carried as an unevaluated sum hi + lo of two
// FP32 numbers (about 48 significant bits), products are formed exactly in their
// leading part with an FMA, and sums keep their rounding errors in the low part.
//
// Every operation uses rounded intrinsics so that the compiler cannot contract an
// error-free transformation into an FMA.  On GB300 every conversion to or from FP64
// costs a slot of the slow FP64 pipe, so the split of an FP64 value is done with
// integer operations.
#pragma once

#include <cstdint>

namespace ec {
namespace ff {

// The same split with fewer integer operations: lo is the 29 bits below hi converted
// by one integer-to-float instruction (rounded to 24 bits) and scaled by a power of two
// built from the exponent.  a = hi + lo + r, |r| < 2^-47 |a|; lo is 0 when its scale
// would leave FP32's normal range (|a| below about 2^-74); other cases as split().
__device__ __forceinline__ float2 split_fast(double a) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
  const unsigned sgn = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7FFu);
  const int eh = e - 896;
  const unsigned mh = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  const int es = e - 948;                                // biased exponent of 2^(e - 1075)
  const float scale = es >= 1 ? __int_as_float((int)(sgn | ((unsigned)es << 23))) : 0.f;
  float2 r;
  r.x = __int_as_float((int)(sgn | ((unsigned)eh << 23) | mh));
  r.y = __fmul_rn(__uint2float_rn(lw & 0x1FFFFFFFu), scale);
  if (eh < 1 || eh > 254) {
    r.x = e == 2047 ? __int_as_float((int)(sgn | 0x7FC00000u))
                    : (eh > 254 ? __int_as_float((int)(sgn | 0x7F800000u)) : 0.f);
    r.y = 0.f;
  }
  return r;
}

// a = hi + lo + r with |r| < 2^-47 |a|: hi is a truncated to 24 significant bits, lo
// the next 24 bits (truncated).  Magnitudes below FP32's normal range contribute 0; a
// non-finite or out-of-range a gives hi = NaN / +-inf.
__device__ __forceinline__ float2 split(double a) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
  const unsigned sgn = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7FFu);
  const int eh = e - 896;                               // FP32 biased exponent of hi
  const unsigned mh = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  const unsigned rem = lw & 0x1FFFFFFFu;                 // the 29 bits below hi
  const int p = 31 - __clz((int)rem);                    // leading one of rem (-1: none)
  const int el = eh - 52 + p;                            // FP32 biased exponent of lo
  const unsigned ml = p >= 23 ? (rem >> (p - 23)) : (rem << (23 - p));
  float2 r;
  if (eh >= 1 && eh <= 254) {
    r.x = __int_as_float((int)(sgn | ((unsigned)eh << 23) | mh));
    r.y = (rem != 0u && el >= 1) ? __int_as_float((int)(sgn | ((unsigned)el << 23) | (ml & 0x7FFFFFu)))
                                 : 0.f;
  } else if (e == 2047) {
    r.x = __int_as_float((int)(sgn | 0x7FC00000u));
    r.y = 0.f;
  } else if (eh > 254) {
    r.x = __int_as_float((int)(sgn | 0x7F800000u));
    r.y = 0.f;
  } else {
    r.x = 0.f;
    r.y = 0.f;
  }
  return r;
}

// (sh, sl) += (ah + al)(bh + bl), dropping al*bl (2^-48 relative); sl accumulates the
// rounding errors of the high sum and the product's low part.
__device__ __forceinline__ void madd(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);                 // exact rounding error of p
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float t = __fadd_rn(sh, p);
  const float bp = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  sl = __fadd_rn(sl, __fadd_rn(err, e));
  sh = t;
}

// (sh, sl) += (bh, bl)
__device__ __forceinline__ void add(float& sh, float& sl, float bh, float bl) {
  const float t = __fadd_rn(sh, bh);
  const float bp = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(bh, bp));
  sl = __fadd_rn(sl, __fadd_rn(err, bl));
  sh = t;
}

}  // namespace ff
}  // namespace ec
