// Host build of the SPDE sampler's device normals (log_series, unit_pm, octant_normal and
// the Philox round function, from the CUDA sources' own text; see the test): the _rn
// intrinsics become the IEEE operations they denote (the build forbids contraction).
// Prints the bit pattern of the normal of octants first .. first + count - 1.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

static unsigned __float_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
static float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
static float __fmul_rn(float a, float b) { return a * b; }
static float __fadd_rn(float a, float b) { return a + b; }
static float __fsub_rn(float a, float b) { return a - b; }
static float __fdiv_rn(float a, float b) { return a / b; }
static float __fsqrt_rn(float a) { return std::sqrt(a); }
static float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
static uint32_t __umulhi(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }

#include "spde_normals.inc"

int main(int argc, char** argv) {
  const uint64_t seed = std::strtoull(argv[1], nullptr, 10), id = std::strtoull(argv[2], nullptr, 10);
  const uint64_t first = std::strtoull(argv[3], nullptr, 10), count = std::strtoull(argv[4], nullptr, 10);
  for (uint64_t o = first; o < first + count; ++o)
    std::printf("%08x\n", __float_as_uint(octant_normal((uint32_t)seed, (uint32_t)(seed >> 32), id, o)));
  return 0;
}
