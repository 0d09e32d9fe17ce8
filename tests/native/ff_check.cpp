// Host check of the double-float arithmetic (ff.h) against long double:
// the binary64 -> double-float split and the sum back, and the relative
// (sums: absolute, against the operands' size) error of each operation on
// random operands over a wide range of magnitudes.  Prints the worst error
// of each, in units of 2^-44, and "failures N"; exit status 1 on any.
#include <cmath>
#include <cstdio>
#include <random>
#include "ff.h"

using mabd::ff;
typedef long double LD;

static LD val(ff a) { return (LD)a.h + (LD)a.l; }

int main() {
  std::mt19937_64 rng(2024);
  std::uniform_real_distribution<double> U(-1.0, 1.0), E(-30.0, 30.0);
  auto rnd = [&]() { return U(rng) * std::ldexp(1.0, (int)E(rng)); };
  const LD unit = std::ldexp((LD)1, -44);
  long fails = 0;
  double worst[7] = {0, 0, 0, 0, 0, 0, 0};
  const char *names[7] = {"split", "to_f64", "add", "mul", "fma", "rcp", "mulf"};
  auto note = [&](int i, LD err, LD scale, LD bound_units) {
    const double u = (double)(err / (scale * unit));
    if (u > worst[i]) worst[i] = u;
    if (!(u <= (double)bound_units)) {
      if (fails < 10) std::printf("%s: error %.3g units\n", names[i], u);
      ++fails;
    }
  };
  for (int it = 0; it < 1000000; ++it) {
    const double x = rnd(), y = rnd(), z = rnd();
    const ff a = mabd::ff_from(x), b = mabd::ff_from(y), c = mabd::ff_from(z);
    // the split keeps 48 of the 53 bits: error below 2^-46 |x|
    note(0, std::fabs(val(a) - (LD)x), std::fabs((LD)x), 0.25L);
    if (!(std::fabs(a.l) <= std::fabs(a.h) * std::ldexp(1.0f, -23))) ++fails;
    note(1, std::fabs((LD)mabd::ff_to(a) - val(a)), std::fabs(val(a)), 1.0L / 512);
    const LD A = val(a), B = val(b), Cc = val(c);
    note(2, std::fabs(val(mabd::ff_add(a, b)) - (A + B)), std::fabs(A) + std::fabs(B), 1.0L);
    note(3, std::fabs(val(mabd::ff_mul(a, b)) - A * B), std::fabs(A * B), 1.0L);
    note(4, std::fabs(val(mabd::ff_fma(a, b, c)) - (A * B + Cc)), std::fabs(A * B) + std::fabs(Cc), 1.0L);
    note(5, std::fabs(val(mabd::ff_rcp(a)) - 1.0L / A), std::fabs(1.0L / A), 1.0L);
    const float f = (float)y;
    note(6, std::fabs(val(mabd::ff_mulf(a, f)) - A * (LD)f), std::fabs(A * (LD)f), 1.0L);
  }
  // special values of the split
  const double sp[] = {0.0, -0.0, 1.0, -1.0, 1e-30, 1e30, 5e-324, 1e300, INFINITY, -INFINITY};
  for (double x : sp) {
    const ff a = mabd::ff_from(x);
    if (std::isinf(x) ? !(a.h == (float)x && a.l == 0.0f) : (x != 0 && std::fabs(x) > 1e-38 &&
                                                              std::fabs(x) < 1e38 &&
                                                              !(std::fabs(val(a) - (LD)x) <=
                                                                std::fabs((LD)x) * unit))) {
      std::printf("split of %g wrong\n", x);
      ++fails;
    }
  }
  for (int i = 0; i < 7; ++i) std::printf("%s worst %.3g units of 2^-44\n", names[i], worst[i]);
  std::printf("failures %ld\n", fails);
  return fails ? 1 : 0;
}
