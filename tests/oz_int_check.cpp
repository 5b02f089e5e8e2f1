// Host driver for the integer helpers of the FP64-accurate tensor-core GEMM
// (paper_2407_11993_gb300/csrc/ec_oz_int.h): the same source the kernels compile,
// built here with the host compiler so that tests/test_oz_int_host.py can compare every
// helper bit for bit with exact integer arithmetic.
//
// Reads one request per line from stdin and writes one answer line per request:
//   S <X> <sc>      -> "<ok> <bits> <ok_fast> <bits_fast>"   i64_scaled_to_f64_bits(_fast)
//   F <bits> <e>    -> "<F>"                                 f64_to_fixed64
//   D <F>           -> "<d_0> ... <d_7>"                     digits8
//   E <bits>        -> "<e>"                                 row_exponent
// Integers are decimal; binary64 bit patterns are unsigned decimal.
#include <cinttypes>
#include <cstdio>
#include <cstring>

#include "ec_oz_int.h"

int main() {
  char op[4];
  while (std::scanf("%3s", op) == 1) {
    if (!std::strcmp(op, "S")) {
      int64_t X;
      int sc;
      if (std::scanf("%" SCNd64 " %d", &X, &sc) != 2) return 2;
      uint64_t b = 0, bf = 0;
      const bool ok = ec::oz::i64_scaled_to_f64_bits(X, sc, &b);
      const bool okf = ec::oz::i64_scaled_to_f64_bits_fast(X, sc, &bf);
      std::printf("%d %" PRIu64 " %d %" PRIu64 "\n", ok ? 1 : 0, ok ? b : 0, okf ? 1 : 0,
                  okf ? bf : 0);
    } else if (!std::strcmp(op, "F")) {
      uint64_t bits;
      int e;
      if (std::scanf("%" SCNu64 " %d", &bits, &e) != 2) return 2;
      std::printf("%" PRId64 "\n", ec::oz::f64_to_fixed64(bits, e));
    } else if (!std::strcmp(op, "D")) {
      int64_t F;
      if (std::scanf("%" SCNd64, &F) != 1) return 2;
      int d[8];
      ec::oz::digits8(F, d);
      for (int s = 0; s < 8; ++s) std::printf(s ? " %d" : "%d", d[s]);
      std::printf("\n");
    } else if (!std::strcmp(op, "E")) {
      uint64_t bits;
      if (std::scanf("%" SCNu64, &bits) != 1) return 2;
      std::printf("%d\n", ec::oz::row_exponent(bits));
    } else {
      return 3;
    }
  }
  return 0;
}
