// Host check of the integer binary64 <-> binary32 conversions (fconv.h)
// against the host's own conversions (C casts: round to nearest, ties to
// even).  Prints the number of mismatches; exit status 1 on any.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <limits>
#include <random>
#include "fconv.h"

static uint64_t bits(double x) { uint64_t u; std::memcpy(&u, &x, 8); return u; }
static uint32_t bitsf(float x) { uint32_t u; std::memcpy(&u, &x, 4); return u; }
static double from(uint64_t u) { double x; std::memcpy(&x, &u, 8); return x; }

int main() {
  long bad = 0, n = 0;
  auto check_d = [&](double x) {
    const float a = mabd::d2f(x), b = (float)x;
    ++n;
    if (bitsf(a) != bitsf(b) && !(std::isnan(a) && std::isnan(b))) {
      if (bad < 10) std::printf("d2f %.17g: %08x vs %08x\n", x, bitsf(a), bitsf(b));
      ++bad;
    }
  };
  auto check_f = [&](float x) {
    const double a = mabd::f2d(x), b = (double)x;
    ++n;
    if (bits(a) != bits(b) && !(std::isnan(a) && std::isnan(b))) {
      if (bad < 10) std::printf("f2d %.9g: %016llx vs %016llx\n", x, (unsigned long long)bits(a),
                                (unsigned long long)bits(b));
      ++bad;
    }
  };
  std::mt19937_64 rng(12345);
  // random bit patterns over the whole binary64 range
  for (int i = 0; i < 2000000; ++i) check_d(from(rng()));
  // values near 1 with random low bits (the rounding decision)
  std::uniform_real_distribution<double> U(-4.0, 4.0);
  for (int i = 0; i < 2000000; ++i) check_d(U(rng));
  // exact ties and neighbours: a binary32 value plus half an ulp (+-1 binary64 ulp)
  for (int i = 0; i < 1000000; ++i) {
    uint64_t u = bits(U(rng)) & ~((uint64_t)0x1fffffff);
    for (uint64_t low : {(uint64_t)0x10000000, (uint64_t)0x0fffffff, (uint64_t)0x10000001,
                         (uint64_t)0x1fffffff, (uint64_t)0})
      check_d(from(u | low));
  }
  // edges: zeros, binary32 range limits, subnormals, overflow, specials
  const double edges[] = {0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38,
                          3.4028236e38, 1e39, -1e39, 1.1754943508222875e-38, 1.1754942e-38,
                          5.877471754111438e-39, 1.401298464324817e-45, 7e-46, 1e-300, -1e-300,
                          std::numeric_limits<double>::infinity(), -std::numeric_limits<double>::infinity(),
                          std::numeric_limits<double>::quiet_NaN(), std::numeric_limits<double>::denorm_min()};
  for (double x : edges) check_d(x);
  // every binary32 exponent with random fractions and signs
  for (uint32_t e = 0; e < 256; ++e)
    for (int i = 0; i < 4000; ++i) {
      uint32_t u = (uint32_t)(rng() & 0x807fffffu) | (e << 23);
      float x;
      std::memcpy(&x, &u, 4);
      check_f(x);
    }
  std::printf("checked %ld, mismatches %ld\n", n, bad);
  return bad ? 1 : 0;
}
