// Host run of the warp-level tensor-core field's data path (tests/test_tc_layout_host.py): the
// kernels' own text for the feature draw, the phasor tables, the x-phasor slice fragments
// (k_xslices) and the staging of the line factors' slices (tc_stage, q_slices, pack_bf16x2),
// with the launch emulated as a loop; the mma.sync m16n8k16 products are emulated from the
// PTX fragment layout (A: rows g, g + 8 and k pairs 2c, 2c + 8; B: column g and the same k;
// D: rows g, g + 8, columns 2c, 2c + 1; the lower half of a register holds the even k) in
// exact double arithmetic, one sum per slice group. Writes, for every sample, line (y, z) and
// x < n - 1, the sum over the groups, i.e. log k / scale, then the same on the face x = n - 1
// for every z and y < n - 1 (the face factors by k_face_factors).
//   tc_emu seed M n ell cov out.bin id0 id1 ...
#define _GNU_SOURCE 1
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

struct dim3 {
  unsigned x = 1, y = 1, z = 1;
  dim3(unsigned a = 1, unsigned b = 1, unsigned c = 1) : x(a), y(b), z(c) {}
};
static dim3 blockIdx, threadIdx, blockDim, gridDim;
struct float4 { float x, y, z, w; };
struct uint4 { unsigned x, y, z, w; };
struct uint2 { unsigned x, y; };
struct int4 { int x, y, z, w; };
struct double2 { double x, y; };
static float4 make_float4(float a, float b, float c, float d) { return {a, b, c, d}; }
static uint4 make_uint4(unsigned a, unsigned b, unsigned c, unsigned d) { return {a, b, c, d}; }
static double2 make_double2(double a, double b) { return {a, b}; }
struct __nv_bfloat162 { uint16_t x, y; };
static uint16_t bf16_rn(float f) {  // round to nearest even (every slice is exact in bf16)
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t r = u + 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(r >> 16);
}
static __nv_bfloat162 __floats2bfloat162_rn(float a, float b) { return {bf16_rn(a), bf16_rn(b)}; }
static int __double2hiint(double d) { uint64_t u; std::memcpy(&u, &d, 8); return (int)(u >> 32); }
static int __double2loint(double d) { uint64_t u; std::memcpy(&u, &d, 8); return (int)(uint32_t)u; }
static double __hiloint2double(int hi, int lo) {
  const uint64_t u = ((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo;
  double d;
  std::memcpy(&d, &u, 8);
  return d;
}
static unsigned __float_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
static float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
static uint32_t __umulhi(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }
#define MLMC_COV_EXP 1

#include "dfloat.cuh"

namespace mlmc {
#include "kernels.inc"
}  // namespace mlmc

using namespace mlmc;

static float bf(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
static double lo16(unsigned r) { return (double)bf((uint16_t)(r & 0xffffu)); }
static double hi16(unsigned r) { return (double)bf((uint16_t)(r >> 16)); }

// The volume x < n - 1 (rows x, lines (y, z)) or the face x = n - 1 (rows y < n - 1, lines z;
// FACE) with RX row tiles per block: every block's line slots as the kernel fills them, the
// staged chunks by tc_stage, the products of every warp emulated. S[s][line][row].
template <int RX, bool FACE>
static void run_volume(int B, int M, int n, const float4* xs, const float4* pt, const uint4* Xf, double* S) {
  using Sh = TcShape<RX>;
  const int KS = (M + 7) / 8, RT = (n - 1) / 16;
  const size_t nl = FACE ? (size_t)n : (size_t)n * n;
  const int lgps = (int)((nl + 31) / 32);
  const int gy = (B * lgps + 8 / RX - 1) / (8 / RX);
  std::vector<int4> sline(Sh::LQ);
  std::vector<uint2> sq((size_t)Sh::BUF);
  std::vector<double> acc((size_t)8 * kTcSlices * 16 * 32);
  for (int by = 0; by < gy; ++by)
    for (int bx = 0; bx < RT / RX; ++bx) {
      blockIdx = dim3(bx, by, 0);
      for (int t = 0; t < Sh::LQ; ++t) {
        const int lg = by * (8 / RX) + t / 32, ls = lg / lgps, line = (lg % lgps) * 32 + t % 32;
        const bool ok = ls < B && (size_t)line < nl;
        sline[t] = FACE ? int4{ls, line, 0, ok ? 1 : 0} : int4{ls, line % n, line / n, ok ? 1 : 0};
      }
      std::fill(acc.begin(), acc.end(), 0.0);
      for (int m0 = 0; m0 < M; m0 += Sh::KCF) {
        std::fill(sq.begin(), sq.end(), uint2{0x7fc07fc0u, 0x7fc07fc0u});  // NaN if read unstaged
        for (int it = 0; it < Sh::LQ * Sh::KCF; ++it)
          tc_stage<RX, FACE>(it, m0, M, n, xs, pt, sline.data(), sq.data());
        const int ksn = std::min(RX, KS - m0 / 8);
        for (int warp = 0; warp < 8; ++warp) {
          const int rt = bx * RX + warp % RX, ct0 = (warp / RX) * 4;
          const int glg = by * (8 / RX) + warp / RX;
          const int s = std::min(glg / lgps, B - 1);
          for (int ksl = 0; ksl < ksn; ++ksl) {
            const int ks = m0 / 8 + ksl;
            for (int j = 0; j < kTcSlices; ++j)
              for (int i = 0; i + j < kTcSlices; ++i)
                for (int ct = 0; ct < 4; ++ct) {
                  // the 16 x 16 A and 16 x 8 B of this product, from the lanes' registers
                  double A[16][16], Bm[16][8];
                  for (int lane = 0; lane < 32; ++lane) {
                    const int g = lane >> 2, c = lane & 3;
                    const uint4 a = Xf[(((size_t)(s * RT + rt) * KS + ks) * kTcSlices + i) * 32 + lane];
                    A[g][2 * c] = lo16(a.x), A[g][2 * c + 1] = hi16(a.x);
                    A[g + 8][2 * c] = lo16(a.y), A[g + 8][2 * c + 1] = hi16(a.y);
                    A[g][2 * c + 8] = lo16(a.z), A[g][2 * c + 9] = hi16(a.z);
                    A[g + 8][2 * c + 8] = lo16(a.w), A[g + 8][2 * c + 9] = hi16(a.w);
                    const uint2 b = sq[((size_t)(ksl * kTcSlices + j) * Sh::CT + ct0 + ct) * 32 + lane];
                    Bm[2 * c][g] = lo16(b.x), Bm[2 * c + 1][g] = hi16(b.x);
                    Bm[2 * c + 8][g] = lo16(b.y), Bm[2 * c + 9][g] = hi16(b.y);
                  }
                  double* D = &acc[((size_t)warp * kTcSlices + (i + j)) * 16 * 32];
                  for (int r = 0; r < 16; ++r)
                    for (int col = 0; col < 8; ++col) {
                      double d = 0.0;
                      for (int k = 0; k < 16; ++k) d += A[r][k] * Bm[k][col];
                      D[r * 32 + ct * 8 + col] += d;
                    }
                }
          }
        }
      }
      for (int warp = 0; warp < 8; ++warp) {
        const int rt = bx * RX + warp % RX;
        const int glg = by * (8 / RX) + warp / RX;
        const int s = glg / lgps;
        if (s >= B) continue;
        for (int r = 0; r < 16; ++r)
          for (int l = 0; l < 32; ++l) {
            const size_t line = (size_t)(glg % lgps) * 32 + l;
            if (line >= nl) continue;
            double sum = 0.0;
            for (int gi = kTcSlices - 1; gi >= 0; --gi)
              sum += acc[(((size_t)warp * kTcSlices + gi) * 16 + r) * 32 + l];
            S[((size_t)s * nl + line) * (n - 1) + 16 * rt + r] = sum;
          }
      }
    }
}

int main(int argc, char** argv) {
  if (argc < 8) return 2;
  const uint64_t seed = strtoull(argv[1], nullptr, 10);
  const int M = atoi(argv[2]), n = atoi(argv[3]);
  const double ell = atof(argv[4]);
  const int cov = atoi(argv[5]);
  const char* outp = argv[6];
  const int B = argc - 7;
  std::vector<uint64_t> ids(B);
  for (int s = 0; s < B; ++s) ids[s] = strtoull(argv[7 + s], nullptr, 10);
  blockDim = dim3(1);
  threadIdx = dim3(0, 0, 0);
  // features: one thread per (sample, feature)
  std::vector<double> w((size_t)B * M * 3), bph((size_t)B * M);
  gridDim = dim3((unsigned)((size_t)B * M));
  for (unsigned b = 0; b < gridDim.x; ++b) {
    blockIdx = dim3(b);
    k_features(ids.data(), B, M, seed, ell, cov, w.data(), bph.data());
  }
  // phasor tables and x-slice fragments: grid-stride loops, one thread covers all
  gridDim = dim3(1);
  blockIdx = dim3(0);
  const double h = 1.0 / (double)(n - 1);
  std::vector<double2> tab((size_t)B * 3 * M * n);
  std::vector<float4> xs((size_t)B * 3 * M * n);
  k_phasors(w.data(), bph.data(), B, M, n, h, tab.data(), xs.data());
  const int KS = (M + 7) / 8, RT = (n - 1) / 16;
  std::vector<uint4> Xf(2 * tc_xslice_bytes(B, M, n) / sizeof(uint4));
  std::vector<float> e2(64);
  k_xslices(xs.data(), B, M, n, KS, 0, Xf.data(), e2.data());
  std::vector<float4> pt((size_t)B * M * n);
  k_face_factors(xs.data(), B, M, n, pt.data());
  const uint4* Xy = Xf.data() + Xf.size() / 2;  // the y-phasor fragments (axis 1)
  std::vector<double> S((size_t)B * n * n * (n - 1), NAN), Sf((size_t)B * n * (n - 1), NAN);
  if (RT % 8 == 0) {
    run_volume<8, false>(B, M, n, xs.data(), pt.data(), Xf.data(), S.data());
    run_volume<8, true>(B, M, n, xs.data(), pt.data(), Xy, Sf.data());
  } else if (RT % 4 == 0) {
    run_volume<4, false>(B, M, n, xs.data(), pt.data(), Xf.data(), S.data());
    run_volume<4, true>(B, M, n, xs.data(), pt.data(), Xy, Sf.data());
  } else if (RT % 2 == 0) {
    run_volume<2, false>(B, M, n, xs.data(), pt.data(), Xf.data(), S.data());
    run_volume<2, true>(B, M, n, xs.data(), pt.data(), Xy, Sf.data());
  } else {
    run_volume<1, false>(B, M, n, xs.data(), pt.data(), Xf.data(), S.data());
    run_volume<1, true>(B, M, n, xs.data(), pt.data(), Xy, Sf.data());
  }
  FILE* f = std::fopen(outp, "wb");
  if (!f) return 3;
  std::fwrite(S.data(), sizeof(double), S.size(), f);
  std::fwrite(Sf.data(), sizeof(double), Sf.size(), f);
  std::fclose(f);
  return 0;
}
