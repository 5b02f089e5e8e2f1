// Host driver for the compensated-FP32 helpers (paper_2407_11993_gb300/csrc/ec_ff.h): the
// same source the kernels compile, built with the host compiler over a shim that gives the
// CUDA intrinsics it uses their documented meaning (round-to-nearest FP32 operations,
// bit casts, count of leading zeros).  Build with -ffp-contract=off so that no product and
// sum are fused behind the helpers' back.  tests/test_ff_host.py drives it.
//
// One request per line on stdin, one answer line per request (binary64 / binary32 values
// as their bit patterns, unsigned decimal):
//   P <bits64>                         -> "<hi> <lo> <hi_fast> <lo_fast>"   split, split_fast
//   A <sh> <sl> <bh> <bl>              -> "<sh'> <sl'>"                     add
//   M <sh> <sl> <ah> <al> <bh> <bl>    -> "<sh'> <sl'>"                     madd
//   X <n> <a_1> <b_1> ... <a_n> <b_n>  -> "<sh> <sl>"   sum of a_i b_i: each operand cut by
//                                                       split_fast, products added by madd
#include <cinttypes>
#include <cmath>
#include <cstdio>
#include <cstring>

struct float2 {
  float x, y;
};
#define __device__
#define __forceinline__ inline

static inline long long __double_as_longlong(double a) {
  long long r;
  std::memcpy(&r, &a, sizeof r);
  return r;
}
static inline float __int_as_float(int a) {
  float r;
  std::memcpy(&r, &a, sizeof r);
  return r;
}
static inline int __clz(int a) { return a ? __builtin_clz((unsigned)a) : 32; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __uint2float_rn(unsigned a) { return (float)a; }
using std::fmaf;

#include "ec_ff.h"

static float f32(uint32_t b) {
  float r;
  std::memcpy(&r, &b, sizeof r);
  return r;
}
static uint32_t b32(float f) {
  uint32_t r;
  std::memcpy(&r, &f, sizeof r);
  return r;
}
static double f64(uint64_t b) {
  double r;
  std::memcpy(&r, &b, sizeof r);
  return r;
}

int main() {
  char op[4];
  while (std::scanf("%3s", op) == 1) {
    if (!std::strcmp(op, "P")) {
      uint64_t a;
      if (std::scanf("%" SCNu64, &a) != 1) return 2;
      const float2 s = ec::ff::split(f64(a)), t = ec::ff::split_fast(f64(a));
      std::printf("%u %u %u %u\n", b32(s.x), b32(s.y), b32(t.x), b32(t.y));
    } else if (!std::strcmp(op, "A")) {
      uint32_t v[4];
      if (std::scanf("%u %u %u %u", &v[0], &v[1], &v[2], &v[3]) != 4) return 2;
      float sh = f32(v[0]), sl = f32(v[1]);
      ec::ff::add(sh, sl, f32(v[2]), f32(v[3]));
      std::printf("%u %u\n", b32(sh), b32(sl));
    } else if (!std::strcmp(op, "M")) {
      uint32_t v[6];
      if (std::scanf("%u %u %u %u %u %u", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]) != 6)
        return 2;
      float sh = f32(v[0]), sl = f32(v[1]);
      ec::ff::madd(sh, sl, f32(v[2]), f32(v[3]), f32(v[4]), f32(v[5]));
      std::printf("%u %u\n", b32(sh), b32(sl));
    } else if (!std::strcmp(op, "X")) {
      int n;
      if (std::scanf("%d", &n) != 1 || n < 0) return 2;
      float sh = 0.f, sl = 0.f;
      for (int i = 0; i < n; ++i) {
        uint64_t a, b;
        if (std::scanf("%" SCNu64 " %" SCNu64, &a, &b) != 2) return 2;
        const float2 x = ec::ff::split_fast(f64(a)), y = ec::ff::split_fast(f64(b));
        ec::ff::madd(sh, sl, x.x, x.y, y.x, y.y);
      }
      std::printf("%u %u\n", b32(sh), b32(sl));
    } else {
      return 3;
    }
  }
  return 0;
}
