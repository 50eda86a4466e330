// Host run of the SPDE sampler (the kernels' own text from paper_1607_03252_gb300/csrc/
// spde.cu and widen.cuh; see tests/test_spde_solve_host.py): the noise, the FP64 residual,
// the FP32 V(2,2) correction cycle on the cell grids, the update, the convergence test and
// the extraction, launched as loops over blocks and threads (a block's threads in reverse
// order, so that thread 0, which writes a block's reduction, sees the whole sum), driven by
// the same refinement loop as spde_field_dev. Prints k at the n^3 nodes (hex doubles).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "mlmc.h"

struct dim3 {
  unsigned x = 1, y = 1, z = 1;
  dim3(unsigned a = 1, unsigned b = 1, unsigned c = 1) : x(a), y(b), z(c) {}
};
static dim3 blockIdx, threadIdx, blockDim, gridDim;
using std::min;

static unsigned __float_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
static float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
static float __fmul_rn(float a, float b) { return a * b; }
static float __fadd_rn(float a, float b) { return a + b; }
static float __fsub_rn(float a, float b) { return a - b; }
static float __fdiv_rn(float a, float b) { return a / b; }
static float __fsqrt_rn(float a) { return std::sqrt(a); }
static float __fmaf_rn(float a, float b, float c) { return std::fmaf(a, b, c); }
static uint32_t __umulhi(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }
static int __double2hiint(double d) { uint64_t b; std::memcpy(&b, &d, 8); return (int)(uint32_t)(b >> 32); }
static int __double2loint(double d) { uint64_t b; std::memcpy(&b, &d, 8); return (int)(uint32_t)b; }
static double __hiloint2double(int hi, int lo) {
  uint64_t b = ((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo;
  double d;
  std::memcpy(&d, &b, 8);
  return d;
}
static int __popc(unsigned v) { return __builtin_popcount(v); }
static int atomicOr(int* p, int v) {
  const int o = *p;
  *p |= v;
  return o;
}

// block reduction stand-in: the threads of a block run from the last to thread 0
static double g_block_acc = 0.0;
template <int THREADS>
static double block_sum(double v) {
  if (threadIdx.x == blockDim.x - 1) g_block_acc = 0.0;
  g_block_acc += v;
  return g_block_acc;
}
static double warp_partial_sum(const double* part, int NB) {
  double a = 0.0;
  for (int b = 0; b < NB; ++b) a += part[b];
  return a;
}

#include "spde_kernels.inc"

template <typename F>
static void launch(dim3 grid, dim3 block, F body) {
  gridDim = grid;
  blockDim = block;
  for (unsigned bz = 0; bz < grid.z; ++bz)
    for (unsigned by = 0; by < grid.y; ++by)
      for (unsigned bx = 0; bx < grid.x; ++bx)
        for (int t = (int)block.x - 1; t >= 0; --t) {
          blockIdx = dim3(bx, by, bz);
          threadIdx = dim3((unsigned)t, 0, 0);
          body();
        }
}

struct Lv {
  int C;
  std::vector<float> e, g, r;
};

static void vcycle32(std::vector<Lv>& L, size_t l, double kappa, double h0, const int* active) {
  const int C = L[l].C, lc = log2i(C);
  const double hl = h0 * (double)(1 << l), ch2d = kappa * kappa * hl * hl;
  const float ch2 = (float)ch2d;
  if (C == 2) {
    launch(dim3(1), dim3(128), [&] { k_cc_coarse<float>(1, ch2, L[l].g.data(), L[l].e.data(), active); });
    return;
  }
  const float i3 = (float)(1.0 / (ch2d + 3.0)), i4 = (float)(1.0 / (ch2d + 4.0)), i5 = (float)(1.0 / (ch2d + 5.0)),
              i6 = (float)(1.0 / (ch2d + 6.0));
  auto sweep = [&]() {
    for (int colour = 0; colour < 2; ++colour)
      launch(cell_grid((size_t)C * C * C / 2, 1), dim3(kT), [&] {
        k_cc_rbgs<float>(colour, lc, 1, i3, i4, i5, i6, L[l].g.data(), L[l].e.data(), active);
      });
  };
  sweep();
  sweep();
  int zs = 0;
  const int slabs = zslabs(C, &zs);
  launch(dim3(col_blocks(C), slabs, 1), dim3(128), [&] {
    k_cc_residual<float, float>(lc, zs, ch2, L[l].g.data(), L[l].e.data(), L[l].r.data(), nullptr, active);
  });
  const int Cc = L[l + 1].C;
  launch(cell_grid((size_t)Cc * Cc * Cc, 1), dim3(kT),
         [&] { k_cc_restrict<float>(lc - 1, 1, L[l].r.data(), L[l + 1].g.data(), active); });
  std::fill(L[l + 1].e.begin(), L[l + 1].e.end(), 0.0f);
  vcycle32(L, l + 1, kappa, h0, active);
  launch(cell_grid((size_t)C * C * C, 1), dim3(kT),
         [&] { k_cc_prolong<float>(lc, 1, L[l + 1].e.data(), L[l].e.data(), active); });
  sweep();
  sweep();
}

int main(int argc, char** argv) {
  const uint64_t seed = std::strtoull(argv[1], nullptr, 10), id = std::strtoull(argv[2], nullptr, 10);
  const int n = std::atoi(argv[3]), n_noise = std::atoi(argv[4]);
  const double sigma2 = std::atof(argv[5]), ell = std::atof(argv[6]);
  const int C = 2 * (n - 1), lc = log2i(C), r = (n_noise - 1) / (n - 1);
  const size_t C3 = (size_t)C * C * C;
  const double h = 1.0 / (double)(n - 1), hf = 1.0 / (double)(n_noise - 1), v = 0.5 * hf;
  const double scale = std::sqrt(v * v * v) / h;
  const uint64_t Mo = 4 * (uint64_t)(n_noise - 1) + 1;
  std::vector<double> g64(C3), Z64(C3, 0.0);
  uint64_t ids[1] = {id};
  launch(cell_grid(C3, 1), dim3(kT), [&] {
    k_spde_noise(ids, 1, lc, r, Mo, (uint32_t)seed, (uint32_t)(seed >> 32), scale, g64.data());
  });
  std::vector<Lv> L;
  for (int c = C; c >= 2; c /= 2) L.push_back(Lv{c, std::vector<float>((size_t)c * c * c), std::vector<float>((size_t)c * c * c),
                                                 std::vector<float>((size_t)c * c * c)});
  int active[1] = {1}, cycles[1] = {0}, flag = 0;
  int zs = 0;
  const int slabs = zslabs(C, &zs), NB = col_blocks(C) * slabs;
  std::vector<double> partial(NB), g2(1);
  launch(dim3(col_blocks(C), slabs, 1), dim3(128), [&] {
    k_cc_residual<double, float>(lc, zs, 0.0, g64.data(), nullptr, nullptr, partial.data(), active);
  });
  launch(dim3(1), dim3(128), [&] { k_cc_sum(1, NB, partial.data(), g2.data(), active); });
  const double kappa = 1.0 / ell, ch2 = kappa * kappa * h * h;
  for (int c = 0; c <= kSpdeMaxCycles; ++c) {
    launch(dim3(col_blocks(C), slabs, 1), dim3(128), [&] {
      k_cc_residual64(lc, zs, ch2 + 3.0, ch2 + 4.0, ch2 + 5.0, ch2 + 6.0, g64.data(), Z64.data(), L[0].g.data(),
                      partial.data(), active);
    });
    flag = 0;
    launch(dim3(1), dim3(128), [&] {
      k_cc_check(1, NB, c, partial.data(), g2.data(), kSpdeRtol, kSpdeMaxCycles, active, cycles, &flag);
    });
    if (!(flag & 1)) break;
    std::fill(L[0].e.begin(), L[0].e.end(), 0.0f);
    vcycle32(L, 0, kappa, h, active);
    launch(cell_grid(C3, 1), dim3(kT), [&] { k_cc_update(lc, 1, L[0].e.data(), Z64.data(), active); });
  }
  std::fprintf(stderr, "cycles %d flag %d\n", cycles[0], flag);
  const int off = (n - 1) / 2;
  const double a = std::sqrt(8.0 * 3.14159265358979323846 * kappa * sigma2);
  const size_t nodes = (size_t)n * n * n;
  std::vector<double> k(nodes);
  launch(dim3((unsigned)((nodes + kT - 1) / kT)), dim3(kT), [&] {
    k_spde_extract(n, C, off, 1, a, Z64.data(), MLMC_F64, k.data());
  });
  for (double x : k) {
    uint64_t b;
    std::memcpy(&b, &x, 8);
    std::printf("%016llx\n", (unsigned long long)b);
  }
  return (flag & 2) ? 2 : 0;
}
