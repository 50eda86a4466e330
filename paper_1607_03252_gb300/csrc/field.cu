// Lognormal random-field evaluation (K1 feature draw, K2 field evaluation).
//
// The coefficient of one realisation omega (one sample of Algorithm 1; lognormal k =
// exp(Z) of Sec. 3.2) is log k(x) = sigma sqrt(2/M) sum_m cos(w_m . x + b_m).
// On the structured grid every node is x = (i h, j h, k h), so each term factorises:
//   cos(w.x + b) = Re( e^{i(w_1 x_i + b)} e^{i w_2 y_j} e^{i w_3 z_k} ).
// The kernels tabulate the three per-axis phasors once per (sample, feature, index)
// and evaluate the sum as Re(A_m[i] * Q_m[j,k]) with Q_m[j,k] = B_m[j] C_m[k]:
// two FP64 FMAs per node and feature instead of one FP64 cos (about 20x fewer FP64
// instructions; FP64 throughput is the binding resource of this kernel on GB300).
#include <math.h>

#include <cstdlib>

#include "common.cuh"
#include "field.cuh"
#include "philox.cuh"
#include "prof.cuh"
#include "widen.cuh"

namespace mlmc {

__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) * (1.0 / 9007199254740992.0);
}

// One thread per (sample, feature): w (B x M x 3), b (B x M).
// cov = MLMC_COV_EXP divides the Gaussian vector by |g4| (fourth Box-Muller normal), which
// turns N(0, I/ell^2) into the multivariate Cauchy law of the exponential covariance.
__global__ void k_features(const uint64_t* __restrict__ ids, int B, int M, uint64_t seed, double ell, int cov,
                           double* __restrict__ w, double* __restrict__ bph) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (size_t)B * M) return;
  const int s = (int)(t / M), m = (int)(t - (size_t)s * M);
  const uint64_t id = ids[s];
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  uint32_t wd[12];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    uint32_t c0 = (uint32_t)id, c1 = (uint32_t)(id >> 32), c2 = (uint32_t)m, c3 = (uint32_t)c;
    philox10(c0, c1, c2, c3, k0, k1);
    wd[4 * c + 0] = c0;
    wd[4 * c + 1] = c1;
    wd[4 * c + 2] = c2;
    wd[4 * c + 3] = c3;
  }
  const double U1 = u53(wd[0], wd[1]), U2 = u53(wd[2], wd[3]);
  const double U3 = u53(wd[4], wd[5]), U4 = u53(wd[6], wd[7]);
  const double U5 = u53(wd[8], wd[9]);
  const double two_pi = 6.283185307179586476925286766559;
  const double r1 = sqrt(-2.0 * log(U1)), r2 = sqrt(-2.0 * log(U3));
  const double g1 = r1 * cos(two_pi * U2);
  const double g2 = r1 * sin(two_pi * U2);
  const double g3 = r2 * cos(two_pi * U4);
  double scale = 1.0 / ell;
  if (cov == MLMC_COV_EXP) scale = 1.0 / (ell * fabs(r2 * sin(two_pi * U4)));
  w[3 * t + 0] = g1 * scale;
  w[3 * t + 1] = g2 * scale;
  w[3 * t + 2] = g3 * scale;
  bph[t] = two_pi * U5;
}

// Phasor tables tab[s][axis][m][i] = (cos, sin) of (w_axis x_i (+ b_m on axis 0)), and
// the same pre-split for the double-float kernels, xs = (Re hi, Re lo, Im hi, Im lo). A
// thread fills a run of kPhRun consecutive i of one (sample, axis, feature) row: the first
// entry by sincos of its phase, the next ones by multiplying by the step e^{i w h} (one
// sincos per run), so each entry costs one complex product instead of a sincos on the FP64
// unit; over a run the products add a few ulps (below 2e-15 relative). The split is done
// by the integer-pipe narrowing (hi = fl32(v), lo = fl32(v - hi), the difference exact in
// FP64).
constexpr int kPhRun = 8;
__global__ void k_phasors(const double* __restrict__ w, const double* __restrict__ bph, int B, int M, int n,
                          double h, double2* __restrict__ tab, float4* __restrict__ xs) {
  const int runs = (n + kPhRun - 1) / kPhRun;
  const size_t total = (size_t)B * 3 * M * runs;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int run = (int)(t % runs);
    const size_t r = t / runs;  // row (s, axis, m)
    const int m = (int)(r % M);
    const size_t r2 = r / M;
    const int axis = (int)(r2 % 3);
    const int s = (int)(r2 / 3);
    const size_t f = (size_t)s * M + m;
    const double wa = w[3 * f + axis];
    const int i0 = run * kPhRun;
    double ph = wa * ((double)i0 * h);
    if (axis == 0) ph += bph[f];
    double sn, cs, ds, dc;
    sincos(ph, &sn, &cs);
    sincos(wa * h, &ds, &dc);
    const int i1 = i0 + kPhRun < n ? i0 + kPhRun : n;
    for (int i = i0; i < i1; ++i) {
      const size_t o = r * n + i;
      tab[o] = make_double2(cs, sn);
      const float ch = narrow(cs), sh = narrow(sn);
      xs[o] = make_float4(ch, narrow(cs - widen(ch)), sh, narrow(sn - widen(sh)));
      const double c2 = cs * dc - sn * ds, s2 = sn * dc + cs * ds;
      cs = c2;
      sn = s2;
    }
  }
}

constexpr int kFieldThreads = 256;
constexpr int kFieldOut = 8;  // outputs per thread

// One block: sample blockIdx.y, lines [L0, L0 + LT) of the flattened (z, y) index,
// all n x-values: LT * n <= 2048 outputs. Features are staged MC at a time in shared
// memory: the x-phasors A[m][0..n) and the line factors Q[m][l] = B[m][y] C[m][z].
template <typename TOut>
__global__ void __launch_bounds__(kFieldThreads) k_field(const double2* __restrict__ tab, int M, int n, int LT, int MC,
                                                          double scale, TOut* __restrict__ kout) {
  extern __shared__ double2 sm[];
  double2* sA = sm;
  double2* sQ = sm + (size_t)MC * n;
  const int s = blockIdx.y;
  const size_t n2 = (size_t)n * n;
  const size_t L0 = (size_t)blockIdx.x * LT;
  const int nl = (int)((n2 - L0) < (size_t)LT ? (n2 - L0) : (size_t)LT);
  const int nout = nl * n;
  const double2* Tx = tab + (size_t)s * 3 * M * n;
  const double2* Ty = Tx + (size_t)M * n;
  const double2* Tz = Ty + (size_t)M * n;
  int xo[kFieldOut], lo[kFieldOut];
  double acc[kFieldOut];
#pragma unroll
  for (int q = 0; q < kFieldOut; ++q) {
    const int o = threadIdx.x + q * kFieldThreads;
    lo[q] = o < nout ? o / n : -1;
    xo[q] = o < nout ? o - lo[q] * n : 0;
    acc[q] = 0.0;
  }
  for (int m0 = 0; m0 < M; m0 += MC) {
    const int mc = min(MC, M - m0);
    __syncthreads();
    for (int t = threadIdx.x; t < mc * n; t += kFieldThreads) sA[t] = Tx[(size_t)m0 * n + t];
    for (int t = threadIdx.x; t < mc * nl; t += kFieldThreads) {
      const int mm = t / nl, l = t - mm * nl;
      const size_t line = L0 + l;
      const int y = (int)(line % n), z = (int)(line / n);
      const double2 b = Ty[(size_t)(m0 + mm) * n + y], c = Tz[(size_t)(m0 + mm) * n + z];
      sQ[mm * LT + l] = make_double2(b.x * c.x - b.y * c.y, b.x * c.y + b.y * c.x);
    }
    __syncthreads();
    for (int mm = 0; mm < mc; ++mm) {
#pragma unroll
      for (int q = 0; q < kFieldOut; ++q) {
        if (lo[q] >= 0) {
          const double2 a = sA[mm * n + xo[q]];
          const double2 qq = sQ[mm * LT + lo[q]];
          acc[q] = fma(a.x, qq.x, fma(-a.y, qq.y, acc[q]));
        }
      }
    }
  }
  TOut* out = kout + (size_t)s * n2 * n + L0 * n;
#pragma unroll
  for (int q = 0; q < kFieldOut; ++q) {
    const int o = threadIdx.x + q * kFieldThreads;
    if (o < nout) out[o] = (TOut)exp(scale * acc[q]);
  }
}

static size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

// The same sum in double-float arithmetic on the FP32 pipe (GB300 runs FP32 at 64x the
// FP64 rate). Every FP64 factor f is split into f = hi + lo (two floats, hi = fl32(f));
// a term Re(A Q) = Ar Qr - Ai Qi becomes the exact FP32 products Arh Qrh and Aih Qih
// (their rounding errors recovered by FMA), an exact TwoSum of the two, the four cross
// terms hi x lo, and a TwoSum into the (hi, lo) accumulator. The relative error of the
// sum is ~2^-44 of the magnitudes involved, far below what the FP64 solve can resolve
// (parity against the FP64 oracle is checked at 1e-12 relative in k).
__device__ __forceinline__ float4 split2(double2 v) {
  const float xh = (float)v.x, yh = (float)v.y;
  return make_float4(xh, (float)(v.x - (double)xh), yh, (float)(v.y - (double)yh));
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bv = s - a;
  e = (a - (s - bv)) + (b - bv);
}

template <typename TOut>
__global__ void __launch_bounds__(kFieldThreads) k_field_df(const double2* __restrict__ tab,
                                                             const float4* __restrict__ xsplit, int M, int n, int LT,
                                                             int MC, double scale, TOut* __restrict__ kout) {
  extern __shared__ float4 smf[];
  float4* sA = smf;
  float4* sQ = smf + (size_t)MC * n;
  const int s = blockIdx.y;
  const size_t n2 = (size_t)n * n;
  const size_t L0 = (size_t)blockIdx.x * LT;
  const int nl = (int)((n2 - L0) < (size_t)LT ? (n2 - L0) : (size_t)LT);
  const int nout = nl * n;
  const double2* Ty = tab + (size_t)s * 3 * M * n + (size_t)M * n;
  const double2* Tz = Ty + (size_t)M * n;
  const float4* Xs = xsplit + (size_t)s * 3 * M * n;
  int xo[kFieldOut], lo[kFieldOut];
  float ah[kFieldOut], al[kFieldOut];
#pragma unroll
  for (int q = 0; q < kFieldOut; ++q) {
    const int o = threadIdx.x + q * kFieldThreads;
    lo[q] = o < nout ? o / n : -1;
    xo[q] = o < nout ? o - lo[q] * n : 0;
    ah[q] = 0.f;
    al[q] = 0.f;
  }
  for (int m0 = 0; m0 < M; m0 += MC) {
    const int mc = min(MC, M - m0);
    __syncthreads();
    for (int t = threadIdx.x; t < mc * n; t += kFieldThreads) sA[t] = Xs[(size_t)m0 * n + t];
    for (int t = threadIdx.x; t < mc * nl; t += kFieldThreads) {
      const int mm = t / nl, l = t - mm * nl;
      const size_t line = L0 + l;
      const int y = (int)(line % n), z = (int)(line / n);
      const double2 b = Ty[(size_t)(m0 + mm) * n + y], c = Tz[(size_t)(m0 + mm) * n + z];
      sQ[mm * LT + l] = split2(make_double2(b.x * c.x - b.y * c.y, b.x * c.y + b.y * c.x));
    }
    __syncthreads();
    for (int mm = 0; mm < mc; ++mm) {
#pragma unroll
      for (int q = 0; q < kFieldOut; ++q) {
        if (lo[q] >= 0) {
          const float4 a = sA[mm * n + xo[q]];   // (Re hi, Re lo, Im hi, Im lo)
          const float4 b = sQ[mm * LT + lo[q]];
          const float p1 = a.x * b.x, e1 = fmaf(a.x, b.x, -p1);
          const float p2 = a.z * b.z, e2 = fmaf(a.z, b.z, -p2);
          float th, tl;
          two_sum(p1, -p2, th, tl);
          float lw = (e1 - e2) + tl;
          lw = fmaf(a.x, b.y, lw);
          lw = fmaf(a.y, b.x, lw);
          lw = fmaf(-a.z, b.w, lw);
          lw = fmaf(-a.w, b.z, lw);
          float sh, se;
          two_sum(ah[q], th, sh, se);
          ah[q] = sh;
          al[q] += se + lw;
        }
      }
    }
  }
  TOut* out = kout + (size_t)s * n2 * n + L0 * n;
#pragma unroll
  for (int q = 0; q < kFieldOut; ++q) {
    const int o = threadIdx.x + q * kFieldThreads;
    if (o < nout) out[o] = (TOut)exp(scale * ((double)ah[q] + (double)al[q]));
  }
}

// Double-float sum with one (y, z) line and XC consecutive x-values per thread: the
// line factor Q_m = B_m[y] C_m[z] is formed once per feature in double-float complex
// arithmetic and reused for the XC x-phasors, which every lane of a warp reads at the
// same shared-memory address (broadcast). No FP64 instruction remains in the loop. A grid
// of n = 2^p + 1 nodes per line runs as tiles of 8 x-values over x < n - 1 (8 divides
// n - 1 from n = 9) and one of a single x-value for x = n - 1, so no thread computes
// x-values past the line's end; every node's sum is the same whatever its tile.
constexpr int kXC = 8;

__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
  ph = ah * bh;
  pl = fmaf(ah, bh, -ph);
  pl = fmaf(ah, bl, pl);
  pl = fmaf(al, bh, pl);
}
// (sh, sl) = (ah, al) + (bh, bl), renormalised
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& sh, float& sl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e += al + bl;
  sh = s + e;
  sl = e - (sh - s);
}

template <typename TOut, int XC>
__global__ void __launch_bounds__(kFieldThreads) k_field_line(const float4* __restrict__ tsplit, int M, int n, int MC,
                                                               int xbase, double scale, TOut* __restrict__ kout) {
  extern __shared__ float4 sml[];
  float4* sA = sml;  // [MC][XC]
  const int s = blockIdx.z;
  const int x0 = xbase + (int)blockIdx.x * XC;
  const size_t n2 = (size_t)n * n;
  const size_t line = (size_t)blockIdx.y * kFieldThreads + threadIdx.x;
  const bool valid = line < n2;
  const int y = valid ? (int)(line % n) : 0, z = valid ? (int)(line / n) : 0;
  const float4* Tx = tsplit + (size_t)s * 3 * M * n;
  const float4* Ty = Tx + (size_t)M * n;
  const float4* Tz = Ty + (size_t)M * n;
  float ah[XC], al[XC];
#pragma unroll
  for (int q = 0; q < XC; ++q) {
    ah[q] = 0.f;
    al[q] = 0.f;
  }
  for (int m0 = 0; m0 < M; m0 += MC) {
    const int mc = min(MC, M - m0);
    __syncthreads();
    for (int t = threadIdx.x; t < mc * XC; t += kFieldThreads) {
      const int mm = t / XC, xi = t - mm * XC;
      const int x = x0 + xi;
      sA[t] = x < n ? Tx[(size_t)(m0 + mm) * n + x] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    for (int mm = 0; mm < mc; ++mm) {
      const float4 b = Ty[(size_t)(m0 + mm) * n + y];
      const float4 c = Tz[(size_t)(m0 + mm) * n + z];
      // Q = b c (complex, double-float)
      float rh, rl, ih, il, t1h, t1l, t2h, t2l;
      df_mul(b.x, b.y, c.x, c.y, t1h, t1l);
      df_mul(b.z, b.w, c.z, c.w, t2h, t2l);
      df_add(t1h, t1l, -t2h, -t2l, rh, rl);
      df_mul(b.x, b.y, c.z, c.w, t1h, t1l);
      df_mul(b.z, b.w, c.x, c.y, t2h, t2l);
      df_add(t1h, t1l, t2h, t2l, ih, il);
#pragma unroll
      for (int q = 0; q < XC; ++q) {
        const float4 a = sA[mm * XC + q];  // same address in every lane: broadcast
        const float p1 = a.x * rh, e1 = fmaf(a.x, rh, -p1);
        const float p2 = a.z * ih, e2 = fmaf(a.z, ih, -p2);
        float th, tl;
        two_sum(p1, -p2, th, tl);
        float lw = (e1 - e2) + tl;
        lw = fmaf(a.x, rl, lw);
        lw = fmaf(a.y, rh, lw);
        lw = fmaf(-a.z, il, lw);
        lw = fmaf(-a.w, ih, lw);
        float sh, se;
        two_sum(ah[q], th, sh, se);
        ah[q] = sh;
        al[q] += se + lw;
      }
    }
  }
  if (!valid) return;
  TOut* out = kout + (size_t)s * n2 * n + line * n + x0;
#pragma unroll
  for (int q = 0; q < XC; ++q)
    if (x0 + q < n) out[q] = (TOut)exp(scale * ((double)ah[q] + (double)al[q]));
}

// One launch of k_field_line<., XC> over `tiles` x-tiles from x = xbase; `share` is the
// fraction of the field's nodes it evaluates (for the launch accounting).
template <int XC>
int field_line_launch(const float4* xsplit, int M, int n, int MC, int xbase, unsigned tiles, unsigned lines, int B,
                      double scale, int dtype, void* kout, double bytes, double flops, cudaStream_t st,
                      double share) {
  const dim3 gl(tiles, lines, (unsigned)B);
  const size_t sml = (size_t)MC * XC * sizeof(float4);
  if (dtype == MLMC_F64)
    MLMC_LAUNCH("field_df32", bytes * share, flops * share, st,
                (k_field_line<double, XC><<<gl, kFieldThreads, sml, st>>>(xsplit, M, n, MC, xbase, scale,
                                                                           (double*)kout)));
  else
    MLMC_LAUNCH("field_df32", bytes * share, flops * share, st,
                (k_field_line<float, XC><<<gl, kFieldThreads, sml, st>>>(xsplit, M, n, MC, xbase, scale,
                                                                          (float*)kout)));
  return MLMC_OK;
}

size_t field_scratch_bytes(int B, int M, int n) {
  return a256((size_t)B * M * 3 * sizeof(double)) + a256((size_t)B * M * sizeof(double)) +
         a256((size_t)B * 3 * M * n * sizeof(double2)) + a256((size_t)B * 3 * M * n * sizeof(float4));
}

int field_arith_default() {
  static const int a = [] {
    const char* e = getenv("MLMC_FIELD_ARITH");
    const int v = e ? atoi(e) : (int)kFieldDF32Line;
    return v >= kFieldDF32Line && v <= kFieldDF32 ? v : (int)kFieldDF32Line;
  }();
  return a;
}

int field_eval_dev(const mlmc_field_cfg& cfg, const uint64_t* ids_dev, int B, int n, int dtype, void* kout,
                   void* scratch, cudaStream_t st, int arith) {
  if (arith < 0) arith = field_arith_default();
  char* p = (char*)scratch;
  auto carve = [&](size_t bytes) {
    void* r = p;
    p += a256(bytes);
    return r;
  };
  double* w = (double*)carve((size_t)B * cfg.M * 3 * sizeof(double));
  double* bph = (double*)carve((size_t)B * cfg.M * sizeof(double));
  double2* tab = (double2*)carve((size_t)B * 3 * cfg.M * n * sizeof(double2));
  float4* xsplit = (float4*)carve((size_t)B * 3 * cfg.M * n * sizeof(float4));
  const size_t nf = (size_t)B * cfg.M;
  MLMC_LAUNCH("features", nf * 40.0, nf * 200.0, st,
              (k_features<<<(unsigned)((nf + 255) / 256), 256, 0, st>>>(ids_dev, B, cfg.M, cfg.run_seed,
                                                                          cfg.ell, cfg.cov, w, bph)));
  const double h = 1.0 / (double)(n - 1);
  const size_t nt = (size_t)B * 3 * cfg.M * n;
  MLMC_LAUNCH("phasors", nt * 32.0, nt * 12.0, st,
              (k_phasors<<<blocks_for(nt / kPhRun + 1, 256), 256, 0, st>>>(w, bph, B, cfg.M, n, h, tab, xsplit)));
  int LT = 2048 / n;
  if (LT < 1) LT = 1;
  if ((size_t)LT > (size_t)n * n) LT = n * n;
  int MC = 3072 / (n + LT);
  if (MC > 32) MC = 32;
  if (MC < 1) MC = 1;
  const size_t smem = (size_t)MC * (n + LT) * sizeof(double2);  // double2 and float4 are both 16 B
  dim3 grid((unsigned)(((size_t)n * n + LT - 1) / LT), (unsigned)B);
  const double scale = sqrt(cfg.sigma2) * sqrt(2.0 / (double)cfg.M);
  // algorithmic work: 2 FMA (4 flops) per node and feature, plus one complex product
  // (6 flops) per line and feature; bytes: the tables once and the output once
  const double flops = (double)B * cube(n) * cfg.M * 4.0 + (double)B * n * n * cfg.M * 6.0;
  const double bytes = (double)B * cube(n) * (dtype == MLMC_F64 ? 8.0 : 4.0) + (double)nt * 16.0;
  // double-float form: the same algorithmic flops, executed as ~24 FP32 operations per
  // node and feature; its roofline is the FP32 pipe
  if (arith == kFieldFP64) {
    if (dtype == MLMC_F64)
      MLMC_LAUNCH("field_f64", bytes, flops, st,
                  (k_field<double><<<grid, kFieldThreads, smem, st>>>(tab, cfg.M, n, LT, MC, scale, (double*)kout)));
    else
      MLMC_LAUNCH("field_f64", bytes, flops, st,
                  (k_field<float><<<grid, kFieldThreads, smem, st>>>(tab, cfg.M, n, LT, MC, scale, (float*)kout)));
  } else if (arith == kFieldDF32Line) {
    const int MCl = cfg.M < 64 ? cfg.M : 64;
    const unsigned lines = (unsigned)(((size_t)n * n + kFieldThreads - 1) / kFieldThreads);
    // x < n - 1 in tiles of 8 (of 4 on the 5-node grid), then x = n - 1
    const int xt = (n - 1) % kXC == 0 ? kXC : 4;
    const unsigned tiles = (unsigned)((n - 1) / xt);
    if (xt == kXC)
      MLMC_TRY(field_line_launch<kXC>(xsplit, cfg.M, n, MCl, 0, tiles, lines, B, scale, dtype, kout, bytes, flops, st,
                                     (double)(n - 1) / n));
    else
      MLMC_TRY(field_line_launch<4>(xsplit, cfg.M, n, MCl, 0, tiles, lines, B, scale, dtype, kout, bytes, flops, st,
                                   (double)(n - 1) / n));
    MLMC_TRY(field_line_launch<1>(xsplit, cfg.M, n, MCl, n - 1, 1, lines, B, scale, dtype, kout, bytes, flops, st,
                                 1.0 / n));
  } else {
    if (dtype == MLMC_F64)
      MLMC_LAUNCH("field_df32", bytes, flops, st,
                  (k_field_df<double><<<grid, kFieldThreads, smem, st>>>(tab, xsplit, cfg.M, n, LT, MC, scale,
                                                                         (double*)kout)));
    else
      MLMC_LAUNCH("field_df32", bytes, flops, st,
                  (k_field_df<float><<<grid, kFieldThreads, smem, st>>>(tab, xsplit, cfg.M, n, LT, MC, scale,
                                                                        (float*)kout)));
  }
  MLMC_CUDA_TRY(cudaGetLastError());
  return MLMC_OK;
}

}  // namespace mlmc
