// Host check of the fixed-point FP64 arithmetic of csrc/fx64.h against
// references that use other means: exact power-of-two scaling plus trunc() for
// the fixed-point conversion, the compiler's int64 to FP64 conversion plus
// ldexp for the rounding back, and a 128-bit fixed point with 40 more fraction
// bits for the error of a group sum.  Prints one line per
// check and exits nonzero on the first failure.
#include <cinttypes>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "fx64.h"

using namespace sr;

static double rnd_double(std::mt19937_64& g, int e_lo, int e_hi) {
  std::uniform_real_distribution<double> u(1.0, 2.0);
  std::uniform_int_distribution<int> e(e_lo, e_hi), sg(0, 1);
  const double v = std::ldexp(u(g), e(g));
  return sg(g) ? -v : v;
}

int main() {
  std::mt19937_64 g(12345);
  // 1. fx_of: v * 2^(1078 - em) truncated toward zero
  for (int i = 0; i < 200000; ++i) {
    const double v = rnd_double(g, -60, 10);
    const int em = fx_exp(v) + (int)(g() % 70);
    const double want = std::trunc(std::ldexp(v, 1078 - em));  // |.| < 2^56: exact
    const int64_t got = fx_of(v, em);
    if ((double)got != want) {
      std::printf("fx_of FAIL v=%.17g em=%d got=%" PRId64 " want=%.17g\n", v, em, got, want);
      return 1;
    }
  }
  std::printf("fx_of ok\n");
  // 2. fx_value: t * 2^(em - 1078), one rounding (the compiler's int64 to
  //    FP64 conversion rounds to nearest even; ldexp is exact in range)
  for (int i = 0; i < 400000; ++i) {
    int64_t t;
    const int kind = (int)(g() % 3);
    if (kind == 0) t = (int64_t)(g() >> (g() % 63));     // any width
    else if (kind == 1) t = (int64_t)(g() % 1000000);      // small
    else t = (int64_t)((g() >> 11) << 11);                  // ties and exact cases
    if (g() & 1) t = -t;
    const int em = 40 + (int)(g() % 1200);
    const double want = std::ldexp((double)t, em - 1078);
    const double got = fx_value(t, em);
    if (got != want) {
      std::printf("fx_value FAIL t=%" PRId64 " em=%d got=%.17g want=%.17g\n", t, em, got, want);
      return 1;
    }
  }
  std::printf("fx_value ok\n");
  // 3. a group of up to 65 values: the fixed-point total is within
  //    65 * 2^(em - 1078) of the exact sum
  double worst = 0.0;
  for (int i = 0; i < 20000; ++i) {
    const int n = 1 + (int)(g() % 65);
    double v[65];
    int em = 0;
    const int ehi = -(int)(g() % 40);
    for (int q = 0; q < n; ++q) {
      v[q] = (g() % 8 == 0) ? 0.0 : rnd_double(g, ehi - 60, ehi);
      if (fx_exp(v[q]) > em) em = fx_exp(v[q]);
    }
    int64_t t = 0;
    __int128 ref = 0;  // the exact sum in units of 2^(em - 1118)
    for (int q = 0; q < n; ++q) {
      t += fx_of(v[q], em);
      if (v[q] != 0.0) ref += (__int128)std::ldexp(v[q], 1118 - em);  // to 2^-40 of a unit
    }
    if (em == 0) continue;
    const double err = std::fabs((double)((__int128)t * ((__int128)1 << 40) - ref));
    const double bound = 65.0 * std::ldexp(1.0, 40);
    if (err > bound) {
      std::printf("sum FAIL n=%d em=%d err=%.6g units > %.6g\n", n, em, err, bound);
      return 1;
    }
    if (err / bound > worst) worst = err / bound;
  }
  std::printf("group sums ok (largest error %.3f of the bound)\n", worst);
  return 0;
}
