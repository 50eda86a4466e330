// Host runs of barrier-free CUDA kernels (their text extracted from the sources; see
// tests/test_kernels_host.py): the launch is a loop over every block and thread, with
// blockIdx / threadIdx / blockDim / gridDim as globals. Modes:
//   noise seed id n n_noise         -> the SPDE right-hand side of one sample (hex doubles)
//   faces n in.bin out.bin          -> k_faces_fe<double> on an n^3 field (st0 = 1)
//   prolong nf in.bin out.bin       -> k_prolong_p1<double> of a coarse correction into zeros
//   restrict nf in.bin out.bin      -> k_restrict_p1<double> of a fine residual
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

struct dim3 {
  unsigned x = 1, y = 1, z = 1;
  dim3(unsigned a = 1, unsigned b = 1, unsigned c = 1) : x(a), y(b), z(c) {}
};
static dim3 blockIdx, threadIdx, blockDim, gridDim;

static unsigned __float_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
static float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
static float __fmul_rn(float a, float b) { return a * b; }
static float __fadd_rn(float a, float b) { return a + b; }
static float __fsub_rn(float a, float b) { return a - b; }
static float __fdiv_rn(float a, float b) { return a / b; }
static float __fsqrt_rn(float a) { return std::sqrt(a); }
static float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
static uint32_t __umulhi(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }

#include "kernels.inc"

template <typename F>
static void launch(dim3 grid, dim3 block, F body) {
  gridDim = grid;
  blockDim = block;
  for (unsigned bz = 0; bz < grid.z; ++bz)
    for (unsigned by = 0; by < grid.y; ++by)
      for (unsigned bx = 0; bx < grid.x; ++bx)
        for (unsigned t = 0; t < block.x; ++t) {
          blockIdx = dim3(bx, by, bz);
          threadIdx = dim3(t, 0, 0);
          body();
        }
}

static std::vector<double> readf(const char* p, size_t n) {
  std::vector<double> v(n);
  FILE* f = std::fopen(p, "rb");
  if (!f || std::fread(v.data(), 8, n, f) != n) std::exit(3);
  std::fclose(f);
  return v;
}
static void writef(const char* p, const std::vector<double>& v) {
  FILE* f = std::fopen(p, "wb");
  std::fwrite(v.data(), 8, v.size(), f);
  std::fclose(f);
}

int main(int argc, char** argv) {
  const std::string mode = argv[1];
  const unsigned T = 64;
  if (mode == "noise") {
    const uint64_t seed = std::strtoull(argv[2], nullptr, 10), id = std::strtoull(argv[3], nullptr, 10);
    const int n = std::atoi(argv[4]), n_noise = std::atoi(argv[5]);
    const int C = 2 * (n - 1), r = (n_noise - 1) / (n - 1);
    int lc = 0;
    while ((1 << lc) < C) ++lc;
    const double h = 1.0 / (double)(n - 1), hf = 1.0 / (double)(n_noise - 1), v = 0.5 * hf;
    const double scale = std::sqrt(v * v * v) / h;
    const uint64_t Mo = 4 * (uint64_t)(n_noise - 1) + 1;
    const size_t C3 = (size_t)C * C * C;
    std::vector<double> g(C3, -1.0);
    uint64_t ids[1] = {id};
    launch(dim3((unsigned)((C3 + T - 1) / T), 1), dim3(T), [&] {
      k_spde_noise(ids, 1, lc, r, Mo, (uint32_t)seed, (uint32_t)(seed >> 32), scale, g.data());
    });
    for (double x : g) {
      uint64_t b;
      std::memcpy(&b, &x, 8);
      std::printf("%016llx\n", (unsigned long long)b);
    }
    return 0;
  }
  const int n = std::atoi(argv[2]);
  if (mode == "faces") {
    const size_t n3 = (size_t)n * n * n;
    auto k = readf(argv[3], n3);
    std::vector<double> out(3 * n3, -7.0);
    launch(dim3((unsigned)((n * n + T - 1) / T), (unsigned)n), dim3(T), [&] {
      k_faces_fe<double>(k.data(), n, 1, n, 1, out.data(), out.data() + n3, out.data() + 2 * n3);
    });
    writef(argv[4], out);
  } else if (mode == "prolong") {
    const int nf = n, nc = (nf + 1) / 2, m = nf - 2;
    auto ec = readf(argv[3], (size_t)nc * nc * nc);
    std::vector<double> u((size_t)nf * nf * nf, 0.0);
    launch(dim3((unsigned)((m * m + T - 1) / T), (unsigned)m), dim3(T), [&] {
      k_prolong_p1<double>(nf, 1, ec.data(), u.data(), nullptr);
    });
    writef(argv[4], u);
  } else if (mode == "restrict") {
    const int nf = n, nc = (nf + 1) / 2, mc = nc - 2;
    auto r = readf(argv[3], (size_t)nf * nf * nf);
    std::vector<double> gc((size_t)nc * nc * nc, 0.0);
    launch(dim3((unsigned)((mc * mc + T - 1) / T), (unsigned)mc), dim3(T), [&] {
      k_restrict_p1<double>(nf, 1, r.data(), gc.data(), nullptr);
    });
    writef(argv[4], gc);
  }
  return 0;
}
