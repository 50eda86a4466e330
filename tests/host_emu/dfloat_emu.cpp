// Host checks of the double-float helpers of the tensor-core field (dfloat.cuh, built with
// g++ -ffp-contract=off) and a host model of the tensor-core field evaluation.
//
//   dfloat_emu slices N seed   : slice7 on N random double-floats of every magnitude; prints the
//                                worst |v - sum t| and the number of violated slice properties
//   dfloat_emu exp N seed      : exp_df against expl on N random arguments in [-80, 80];
//                                prints the worst relative error
//   dfloat_emu field in out    : the field of one sample from its features (in: M n sigma_scale,
//                                then w[M][3], b[M] as doubles) by the tensor-core scheme: every
//                                phasor split into slices, the 28 slice pairs summed per group
//                                (exactly, as the tensor cores do within 2^24 grid steps), folded
//                                every 256 features, exp in double-float; writes n^3 doubles
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <random>
#include <vector>

#include "dfloat.cuh"

using namespace mlmc;

static int sig_bits(float v) {
  if (v == 0.f) return 0;
  int e;
  double m = frexp((double)fabsf(v), &e);  // m in [0.5, 1)
  uint64_t q = (uint64_t)ldexp(m, 53);
  int b = 53;
  while (b > 0 && (q & 1u) == 0) {
    q >>= 1;
    --b;
  }
  return b;
}

static int run_slices(long N, unsigned seed) {
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::uniform_int_distribution<int> E(0, 30);
  long double worst = 0;
  long bad = 0;
  for (long it = 0; it < N; ++it) {
    double v = U(rng);
    if (it % 3 == 1) v = ldexp(v, -E(rng));          // small magnitudes
    if (it % 97 == 0) v = (it % 2 ? 1.0 : -1.0);       // the ends of the range
    const float h = (float)v, l = (float)(v - (double)h);
    float t[7];
    df::slice7(h, l, t);
    long double sum = 0;
    for (int i = 0; i < 7; ++i) {
      const long double step = ldexpl(1.0L, -7 * (i + 1));
      const long double q = (long double)t[i] / step;
      if (q != floorl(q)) ++bad;                                       // on its grid
      const long double lim = i == 0 ? 128.0L : (i == 3 ? 72.0L : 64.0L);
      if (fabsl(q) > lim) ++bad;                                        // bounded
      if (sig_bits(t[i]) > 8) ++bad;                                    // exact in bf16
      sum += t[i];
    }
    const long double err = fabsl(((long double)h + (long double)l) - sum);
    if (err > worst) worst = err;
  }
  printf("slices worst_abs_err %.6Le bad %ld\n", worst, bad);
  return 0;
}

static void e2tab(float* th, float* tl) {
  for (int j = 0; j < 32; ++j) {
    const long double v = exp2l((long double)j / 32.0L);
    th[j] = (float)v;
    tl[j] = (float)(v - (long double)th[j]);
  }
}

static int run_exp(long N, unsigned seed) {
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> U(-80.0, 80.0);
  float th[32], tl[32];
  e2tab(th, tl);
  long double worst = 0;
  for (long it = 0; it < N; ++it) {
    double y = U(rng);
    if (it % 4 == 1) y *= 1e-3;
    if (it % 4 == 2) y *= 0.05;
    const float yh = (float)y, yl = (float)(y - (double)yh);
    float eh, el;
    int m;
    df::exp_df(yh, yl, th, tl, eh, el, m);
    const long double got = ldexpl((long double)eh + (long double)el, m);
    const long double ref = expl((long double)yh + (long double)yl);
    const long double rel = fabsl(got - ref) / ref;
    if (rel > worst) worst = rel;
  }
  printf("exp worst_rel_err %.6Le\n", worst);
  return 0;
}

// One sample's field by the tensor-core scheme on the host.
static int run_field(const char* in, const char* outp) {
  FILE* f = fopen(in, "rb");
  if (!f) return 2;
  int hdr[2];
  double scale;
  if (fread(hdr, sizeof(int), 2, f) != 2 || fread(&scale, sizeof(double), 1, f) != 1) return 2;
  const int M = hdr[0], n = hdr[1];
  std::vector<double> w((size_t)M * 3), b(M);
  if (fread(w.data(), sizeof(double), w.size(), f) != w.size() || fread(b.data(), sizeof(double), M, f) != (size_t)M)
    return 2;
  fclose(f);
  const double h = 1.0 / (n - 1);
  // slices of A[x][2m] = Re X, A[x][2m+1] = -Im X and of the double-float Y, Z phasors
  std::vector<float> As((size_t)n * 2 * M * 7);
  std::vector<float> Yd((size_t)M * n * 4), Zd((size_t)M * n * 4);
  for (int m = 0; m < M; ++m)
    for (int i = 0; i < n; ++i) {
      double px = w[3 * m] * (i * h) + b[m];
      const double cx = cos(px), sx = sin(px);
      float t[7];
      float xh = (float)cx, xl = (float)(cx - xh);
      df::slice7(xh, xl, t);
      for (int q = 0; q < 7; ++q) As[(((size_t)i * M + m) * 2 + 0) * 7 + q] = t[q];
      xh = (float)-sx;
      xl = (float)(-sx - xh);
      df::slice7(xh, xl, t);
      for (int q = 0; q < 7; ++q) As[(((size_t)i * M + m) * 2 + 1) * 7 + q] = t[q];
      const double py = w[3 * m + 1] * (i * h), pz = w[3 * m + 2] * (i * h);
      const double v[4] = {cos(py), sin(py), cos(pz), sin(pz)};
      float* yd = &Yd[((size_t)m * n + i) * 4];
      float* zd = &Zd[((size_t)m * n + i) * 4];
      yd[0] = (float)v[0]; yd[1] = (float)(v[0] - yd[0]); yd[2] = (float)v[1]; yd[3] = (float)(v[1] - yd[2]);
      zd[0] = (float)v[2]; zd[1] = (float)(v[2] - zd[0]); zd[2] = (float)v[3]; zd[3] = (float)(v[3] - zd[2]);
    }
  float th[32], tl[32];
  e2tab(th, tl);
  const float sch = (float)scale, scl = (float)(scale - sch);
  std::vector<double> out((size_t)n * n * n);
  std::vector<float> Bs((size_t)2 * M * 7);
  for (int z = 0; z < n; ++z)
    for (int y = 0; y < n; ++y) {
      for (int m = 0; m < M; ++m) {
        const float* b4 = &Yd[((size_t)m * n + y) * 4];
        const float* d4 = &Zd[((size_t)m * n + z) * 4];
        float t1h, t1l, t2h, t2l, rh, rl, ih, il;
        df::mul(b4[0], b4[1], d4[0], d4[1], t1h, t1l);
        df::mul(b4[2], b4[3], d4[2], d4[3], t2h, t2l);
        df::add(t1h, t1l, -t2h, -t2l, rh, rl);
        df::mul(b4[0], b4[1], d4[2], d4[3], t1h, t1l);
        df::mul(b4[2], b4[3], d4[0], d4[1], t2h, t2l);
        df::add(t1h, t1l, t2h, t2l, ih, il);
        df::slice7(rh, rl, &Bs[(size_t)(2 * m) * 7]);
        df::slice7(ih, il, &Bs[(size_t)(2 * m + 1) * 7]);
      }
      for (int x = 0; x < n; ++x) {
        float Th = 0.f, Tl = 0.f;
        for (int f0 = 0; f0 < M; f0 += 256) {
          const int f1 = f0 + 256 < M ? f0 + 256 : M;
          double g[7] = {0, 0, 0, 0, 0, 0, 0};  // exact: every product and partial sum fits
          for (int k = 2 * f0; k < 2 * f1; ++k) {
            const float* a = &As[(((size_t)x * M) * 2 + k) * 7];
            const float* bb = &Bs[(size_t)k * 7];
            for (int i = 0; i < 7; ++i)
              for (int j = 0; i + j < 7; ++j) g[i + j] += (double)a[i] * (double)bb[j];
          }
          float gf[7], sh, sl;
          for (int q = 0; q < 7; ++q) gf[q] = (float)g[q];
          df::sum7(gf, sh, sl);
          df::add(Th, Tl, sh, sl, Th, Tl);
        }
        float yh, yl, eh, el;
        int m;
        df::mul(Th, Tl, sch, scl, yh, yl);
        df::exp_df(yh, yl, th, tl, eh, el, m);
        out[((size_t)z * n + y) * n + x] = ldexp((double)eh + (double)el, m);
      }
    }
  FILE* o = fopen(outp, "wb");
  if (!o) return 2;
  fwrite(out.data(), sizeof(double), out.size(), o);
  fclose(o);
  return 0;
}

int main(int argc, char** argv) {
  if (argc < 4) return 2;
  if (!strcmp(argv[1], "slices")) return run_slices(atol(argv[2]), (unsigned)atol(argv[3]));
  if (!strcmp(argv[1], "exp")) return run_exp(atol(argv[2]), (unsigned)atol(argv[3]));
  if (!strcmp(argv[1], "field")) return run_field(argv[2], argv[3]);
  return 2;
}
