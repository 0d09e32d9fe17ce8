// Prints the library's structured inverse of Hbar_A (csrc/hbar_inv.h) for
// bodies read from stdin, one per line: "m s0 s1 s2 V E nu h" -> 16 numbers
// (or "fail" when the function refuses the body).
#include <cstdio>

#include "hbar_inv.h"

int main() {
  double m, s[3], V, E, nu, h;
  while (std::scanf("%lf %lf %lf %lf %lf %lf %lf %lf", &m, s, s + 1, s + 2, &V, &E, &nu, &h) == 8) {
    double out[16];
    if (!mabd::hbar_inverse(m, s, V, E, nu, h, out)) {
      std::printf("fail\n");
      continue;
    }
    for (int i = 0; i < 16; ++i) std::printf("%.17g%c", out[i], i == 15 ? '\n' : ' ');
  }
  return 0;
}
