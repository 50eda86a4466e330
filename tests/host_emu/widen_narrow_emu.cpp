// Host check of the integer-pipe FP32 <-> FP64 conversions (widen, narrow) of
// paper_1607_03252_gb300/csrc/widen.cuh, compiled from that file's text (see the test):
// against the C conversions, which round to nearest even, on random values and on the
// halfway, carry, overflow, zero and subnormal cases.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

static unsigned __float_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
static float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
static int __double2hiint(double d) { uint64_t b; std::memcpy(&b, &d, 8); return (int)(uint32_t)(b >> 32); }
static int __double2loint(double d) { uint64_t b; std::memcpy(&b, &d, 8); return (int)(uint32_t)b; }
static double __hiloint2double(int hi, int lo) {
  uint64_t b = ((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo;
  double d;
  std::memcpy(&d, &b, 8);
  return d;
}

#include "widen_narrow.inc"

static int fails = 0;
static void check_narrow(double d) {
  float want = (float)d;
  if (std::fabs(want) < 1.1754943508222875e-38f) want = std::signbit(d) ? -0.0f : 0.0f;  // flush
  const float got = narrow(d);
  if (__float_as_uint(got) != __float_as_uint(want)) {
    if (fails++ < 20) std::printf("narrow(%a) = %a, want %a\n", d, (double)got, (double)want);
  }
}
static void check_widen(float f) {
  double want = (double)f;
  if (std::fpclassify(f) == FP_SUBNORMAL) want = std::signbit(f) ? -0.0 : 0.0;
  const double got = widen(f);
  uint64_t a, b;
  std::memcpy(&a, &got, 8);
  std::memcpy(&b, &want, 8);
  if (a != b && !(std::isnan(got) && std::isnan(want))) {
    if (fails++ < 20) std::printf("widen(%a) = %a, want %a\n", (double)f, got, want);
  }
}

int main() {
  std::mt19937_64 rng(12345);
  // random bit patterns over the binary32 exponent range and beyond
  for (int i = 0; i < 2000000; ++i) {
    uint64_t b = rng();
    const int e = 1023 - 140 + (int)(rng() % 300);
    b = (b & 0x800fffffffffffffull) | ((uint64_t)e << 52);
    double d;
    std::memcpy(&d, &b, 8);
    check_narrow(d);
  }
  // ties: the 29 dropped bits exactly half, both parities; carries into the exponent
  for (int i = 0; i < 200000; ++i) {
    const uint64_t e = 1023 - 120 + rng() % 240;
    const uint64_t keep = rng() & 0x7fffffull;
    const uint64_t tail[4] = {0x10000000ull, 0x0fffffffull, 0x10000001ull, 0x1fffffffull};
    for (uint64_t t : tail) {
      const uint64_t b = ((rng() & 1) << 63) | (e << 52) | (keep << 29) | t;
      double d;
      std::memcpy(&d, &b, 8);
      check_narrow(d);
    }
    const uint64_t ones = (e << 52) | (0x7fffffull << 29) | 0x10000000ull;
    double d;
    std::memcpy(&d, &ones, 8);
    check_narrow(d);
  }
  const double special[] = {0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38, 3.5e38, -3.5e38,
                            1.1754943508222875e-38, 1.1754942e-38, 1e-300, -1e-300, 1e300, 0.1, 1.0 / 3.0};
  for (double d : special) check_narrow(d);
  for (int i = 0; i < 2000000; ++i) check_widen(__uint_as_float((unsigned)rng()));
  const float fs[] = {0.0f, -0.0f, 1.0f, INFINITY, -INFINITY, 1e-45f, -1e-40f, 3.4028235e38f};
  for (float f : fs) check_widen(f);
  std::printf("%d mismatches\n", fails);
  return fails ? 1 : 0;
}
