// Compares lv::i128_to_double (csrc/exact.cuh, used by the device-side
// tolerance test) with the host compiler's 128-bit to double conversion on
// values at every bit length, including exact ties at the rounding position.
#include "exact.cuh"
#include <cstdio>
#include <random>
typedef __int128 i128;
int main() {
  std::mt19937_64 r(1);
  long bad = 0, n = 0;
  auto check = [&](i128 v) {
    const double want = (double)v;
    const double got = lv::i128_to_double((int64_t)(v >> 64), (uint64_t)v);
    ++n;
    if (got != want) { if (bad < 5) printf("mismatch %.17g %.17g\n", got, want); ++bad; }
  };
  for (int b = 0; b < 127; ++b) {
    for (int k = 0; k < 2000; ++k) {
      i128 v = ((i128)r() << 64) | r();
      v &= (((i128)1) << b) - 1;  // below 2^b
      v |= ((i128)1) << b;        // top bit b
      check(v); check(-v);
      // ties and near-ties at every rounding position
      if (b > 53) {
        i128 m = v & ~((((i128)1) << (b - 52)) - 1);
        i128 half = ((i128)1) << (b - 53);
        check(m + half); check(m + half - 1); check(m + half + 1); check(m); check(m + 2 * half - 1);
      }
    }
  }
  check(0); check(1); check(-1);
  printf("%ld checked, %ld mismatches\n", n, bad);
  return bad != 0;
}
