// Host check of the integer float32 <-> float64 conversions of csrc/fp_bits.cuh against
// the host's IEEE 754 conversions (exact widening, round-to-nearest-even narrowing).
// Widening: every float32 bit pattern.  Narrowing: random doubles, doubles with the
// exponent forced into and around the float32 range, and for each of those the exact
// ties, their neighbours and the other boundary fractions, plus special values.
// Prints "ok" and exits 0 when every result matches bit for bit.
#include "fp_bits.cuh"

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <random>

using agents::narrow;
using agents::widen;

static uint64_t b64(double x) { uint64_t b; std::memcpy(&b, &x, 8); return b; }
static uint32_t b32(float x) { uint32_t b; std::memcpy(&b, &x, 4); return b; }
static double d_from(uint64_t b) { double x; std::memcpy(&x, &b, 8); return x; }

int main(int argc, char** argv) {
  const long samples = argc > 1 ? std::atol(argv[1]) : 20000000L;
  long bad = 0;
  for (uint64_t u = 0; u <= 0xffffffffull; ++u) {
    const uint32_t b = (uint32_t)u;
    float f;
    std::memcpy(&f, &b, 4);
    const double a = widen(f), r = (double)f;
    if (b64(a) != b64(r) && !(std::isnan(a) && std::isnan(r))) {
      if (bad < 5) std::printf("widen %08x\n", b);
      ++bad;
    }
  }
  auto check = [&](double x) {
    const float a = narrow(x), r = (float)x;
    if (b32(a) != b32(r) && !(std::isnan(a) && std::isnan(r))) {
      if (bad < 5) std::printf("narrow %016llx\n", (unsigned long long)b64(x));
      ++bad;
    }
  };
  std::mt19937_64 g(20251016);
  for (long i = 0; i < samples; ++i) {
    const uint64_t b = g();
    check(d_from(b));
    const uint64_t e = 860 + g() % 310;           // around [897, 1150], the normal range
    const uint64_t bb = (b & 0x800fffffffffffffull) | (e << 52);
    check(d_from(bb));
    const uint64_t t = bb & ~0x1fffffffull;
    const uint64_t low[6] = {0x10000000ull, 0x0fffffffull, 0x10000001ull, 0ull, 0x1fffffffull, 1ull};
    for (uint64_t l : low) check(d_from(t | l));
  }
  const double specials[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, 3.4028234663852886e38,
                             3.4028235677973366e38, 3.4028235677973362e38,
                             1.1754943508222875e-38, 1.1754942e-38, 1.401298464324817e-45,
                             7.006492321624085e-46, 7.006492321624087e-46, 1e-300, -1e-300,
                             1.0, -1.0, 0.1, 2.5e-39};
  for (double x : specials) check(x);
  if (bad) {
    std::printf("%ld mismatches\n", bad);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
