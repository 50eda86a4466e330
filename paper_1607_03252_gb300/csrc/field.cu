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
#include <cuda_bf16.h>
#include <math.h>

#include <atomic>
#include <cstdlib>

#include "bulk.cuh"
#include "common.cuh"
#include "dfloat.cuh"
#include "field.cuh"
#include "philox.cuh"
#include "prof.cuh"
#include "umma.cuh"
#include "umma_layout.h"
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

// The phasor sum on the tensor cores. For one sample, log k / scale at node (x, l) (l the
// (y, z) line) is the product of an x-by-2M matrix and a 2M-by-line matrix: A[x][2m] = Re X_m[x],
// A[x][2m+1] = -Im X_m[x], B[2m][l] = Re Q_m[l], B[2m+1][l] = Im Q_m[l], Q_m[l] = Y_m[y] Z_m[z],
// every entry in [-1, 1]. Each entry is split (df::slice7) into seven bf16 slices on the fixed
// grids 2^-7, ..., 2^-49, so slice i of A times slice j of B is an integer multiple of
// 2^(-7(i+j+2)): the bf16 products are exact, and an FP32 sum of them is exact while it stays
// below 2^24 grid steps. The 28 pairs i + j <= 6 go into seven FP32 group sums (group i + j);
// over 256 features (512 terms) the groups i + j <= 4 are exact in the worst case and the
// groups 5 and 6 round by at most 4e-13 in all; the groups are folded into a double-float
// sum every 256 features. The dropped pairs and the slices' remainders leave below 3e-12 of
// the sum (worst case; 1e-13 for random-signed terms), against the 1e-11 that k's 1e-12
// relative accuracy allows at sigma sqrt(2/M) = 0.09. This is the splitting of Ozaki, Ogita,
// Oishi and Rump (Numer. Algorithms 59, 2012) on a fixed grid, which suffices because every
// entry is bounded by 1. The final exp is Tang's double-float exp on the FP32 pipe (dfloat.cuh).
//
// Fragments follow the register layout of mma.m16n8k16 with bf16 operands: A is 16 x-values by
// 16 k (8 features), B is 16 k by 8 lines; lane (g = lane / 4, c = lane % 4) holds A rows g and
// g + 8 at the feature pairs c and c + 4, B column g at the same features, and D rows g, g + 8
// at the columns 2c, 2c + 1. A (the x-phasors) is the same for every line of a sample and is
// sliced once per sample into Xf[s][rt][ks][slice][lane] (one uint4 of four bf16 pairs per
// lane); B is sliced per block into shared memory.
constexpr int kTcSlices = 7;
constexpr int kTcThreads = 256;
constexpr int kTcFold = 256;  // features per exact FP32 group sum

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // exact: every slice fits in bf16
  return *reinterpret_cast<const uint32_t*>(&v);
}

// The seven bf16 pairs (Re, Im) of the slices of Q = Y Z, Y and Z double-float complex
// (Re hi, Re lo, Im hi, Im lo): Re Q = Re Y Re Z - Im Y Im Z, Im Q = Re Y Im Z + Im Y Re Z.
// (The paired FP32 instructions, f32x2, with Re and Im as the two lanes measured slower here:
// the packing of the lanes costs more integer instructions than the pairing saves.)
__device__ __forceinline__ void q_slices(const float4& y, const float4& z, uint32_t (&q)[kTcSlices]) {
  float t1h, t1l, t2h, t2l, rh, rl, ih, il, qr[kTcSlices], qi[kTcSlices];
  df::mul(y.x, y.y, z.x, z.y, t1h, t1l);
  df::mul(y.z, y.w, z.z, z.w, t2h, t2l);
  df::add(t1h, t1l, -t2h, -t2l, rh, rl);
  df::mul(y.x, y.y, z.z, z.w, t1h, t1l);
  df::mul(y.z, y.w, z.x, z.y, t2h, t2l);
  df::add(t1h, t1l, t2h, t2l, ih, il);
  df::slice7(rh, rl, qr);
  df::slice7(ih, il, qi);
#pragma unroll
  for (int j = 0; j < kTcSlices; ++j) q[j] = pack_bf16x2(qr[j], qi[j]);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint4& a, const uint2& b) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y));
}

size_t tc_xslice_bytes(int B, int M, int n) {
  return (size_t)B * ((n - 1) / 16) * ((M + 7) / 8) * kTcSlices * 32 * sizeof(uint4);
}

// One thread per (axis, sample, row tile, k-step, lane): the lane's four A registers of every
// slice, for the x-phasors (axis 0, into Xf) and the y-phasors (axis 1, into Xf + the size of
// one axis: the A operand of the x = n - 1 face). Threads 0..31 also write 2^(j/32) as
// double-floats (e2tab[j], e2tab[32 + j]) for the exp.
__global__ void k_xslices(const float4* __restrict__ xsplit, int B, int M, int n, int KS, int axis0,
                          uint4* __restrict__ Xf, float* __restrict__ e2tab) {
  const int RT = (n - 1) / 16;
  const size_t per_axis = (size_t)B * RT * KS * 32;
  const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 < 32) {
    const double v = exp2((double)t0 / 32.0);
    const float h = narrow(v);
    e2tab[t0] = h;
    e2tab[32 + t0] = narrow(v - widen(h));
  }
  for (size_t t = t0 + axis0 * per_axis; t < 2 * per_axis; t += (size_t)gridDim.x * blockDim.x) {
    const int axis = t < per_axis ? 0 : 1;
    const size_t ta = t - axis * per_axis;
    const int lane = (int)(ta & 31);
    size_t r = ta >> 5;
    const int ks = (int)(r % KS);
    r /= KS;
    const int rt = (int)(r % RT);
    const int s = (int)(r / RT);
    const int g = lane >> 2, c = lane & 3;
    uint32_t reg[4][kTcSlices];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int x = 16 * rt + g + (q & 1) * 8;
      const int f = 8 * ks + c + (q >> 1) * 4;
      float re[kTcSlices], im[kTcSlices];
      if (f < M) {
        const float4 v = xsplit[(((size_t)s * 3 + axis) * M + f) * n + x];
        df::slice7(v.x, v.y, re);
        df::slice7(-v.z, -v.w, im);
      } else {
#pragma unroll
        for (int i = 0; i < kTcSlices; ++i) re[i] = im[i] = 0.f;
      }
#pragma unroll
      for (int i = 0; i < kTcSlices; ++i) reg[q][i] = pack_bf16x2(re[i], im[i]);
    }
    uint4* o = Xf + axis * per_axis * kTcSlices + ((size_t)(s * RT + rt) * KS + ks) * kTcSlices * 32 + lane;
#pragma unroll
    for (int i = 0; i < kTcSlices; ++i) o[i * 32] = make_uint4(reg[0][i], reg[1][i], reg[2][i], reg[3][i]);
  }
}

// The line factors of the x = n - 1 face: P_m[z] = X_m[n - 1] Z_m[z] in double-float, laid out
// as the tables (pt[s][m][z] = (Re hi, Re lo, Im hi, Im lo)). On that face log k / scale is
// sum_m Re(Y_m[y] P_m[z]): the same product as the volume with y for x and z for the line.
__global__ void k_face_factors(const float4* __restrict__ xsplit, int B, int M, int n, float4* __restrict__ pt) {
  const size_t total = (size_t)B * M * n;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int z = (int)(t % n);
    const size_t sm = t / n;  // s * M + m
    const int m = (int)(sm % M);
    const int s = (int)(sm / M);
    const float4 a = xsplit[((size_t)s * 3 * M + m) * n + (n - 1)];
    const float4 d = xsplit[(((size_t)s * 3 + 2) * M + m) * n + z];
    float t1h, t1l, t2h, t2l, rh, rl, ih, il;
    df::mul(a.x, a.y, d.x, d.y, t1h, t1l);
    df::mul(a.z, a.w, d.z, d.w, t2h, t2l);
    df::add(t1h, t1l, -t2h, -t2l, rh, rl);
    df::mul(a.x, a.y, d.z, d.w, t1h, t1l);
    df::mul(a.z, a.w, d.x, d.y, t2h, t2l);
    df::add(t1h, t1l, t2h, t2l, ih, il);
    pt[t] = make_float4(rh, rl, ih, il);
  }
}

// The edge x = y = n - 1 in FP64 (n nodes per sample): one warp per (sample, z), lanes over the
// features, log k / scale = sum_m Re(X_m[n - 1] Y_m[n - 1] Z_m[z]), a butterfly sum over the lanes.
template <typename TOut>
__global__ void k_field_edge(const double2* __restrict__ tab, int B, int M, int n, double scale,
                             TOut* __restrict__ kout) {
  const size_t gw = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= (size_t)B * n) return;
  const int s = (int)(gw / n), z = (int)(gw % n);
  const double2* Tx = tab + (size_t)s * 3 * M * n;
  const double2* Ty = Tx + (size_t)M * n;
  const double2* Tz = Ty + (size_t)M * n;
  double acc = 0.0;
  for (int m = lane; m < M; m += 32) {
    const double2 x = Tx[(size_t)m * n + n - 1], y = Ty[(size_t)m * n + n - 1], zz = Tz[(size_t)m * n + z];
    const double cr = x.x * y.x - x.y * y.y, ci = x.x * y.y + x.y * y.x;
    acc = fma(cr, zz.x, fma(-ci, zz.y, acc));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) kout[(size_t)s * n * n * n + ((size_t)z * n + n - 1) * n + n - 1] = (TOut)exp(scale * acc);
}

// Block: RX row tiles (16 rows each, from row 16 RX blockIdx.x) by 256 / RX lines (from
// blockIdx.y * 256 / RX) of sample blockIdx.z; warp w takes row tile w % RX and the 32 lines
// (four column tiles) of line group w / RX. Features come in chunks of 8 RX (RX k-steps): every
// thread forms double-float Q_m[l] of 8 (line, feature) pairs of a chunk, slices it and stores
// the bf16 pairs (Re, Im) of each slice in the B-fragment order sq[k-step][slice][column
// tile][lane]. The chunks are double-buffered: a warp stages its items of the next chunk
// between the k-steps of the current one (8 / RX items after each k-step), so the FP32 work of
// the staging and the tensor-core work of the products overlap; one barrier per chunk. The
// double-float running sums of the group folds live in shared memory (used every 256
// features only). FACE = false: the volume x < n - 1 (rows x, lines (y, z), Q_m = Y_m[y] Z_m[z]
// from the tables); FACE = true: the face x = n - 1, y < n - 1 (rows y, lines z, Q_m = P_m[z]
// from k_face_factors, A from the y-phasor slices).
template <int RX>
struct TcShape {
  static constexpr int LQ = 256 / RX;                        // lines per block
  static constexpr int CT = LQ / 8;                          // column tiles per block
  static constexpr int KCF = 8 * RX;                         // features per chunk
  static constexpr int BUF = KCF / 8 * kTcSlices * CT * 32;  // uint2 per chunk buffer
  static constexpr size_t smem =
      (2 * (size_t)BUF) * sizeof(uint2) + 32 * kTcThreads * sizeof(float) + (size_t)LQ * sizeof(int4);
};

// Q_m[line] of item `it` (of LQ * KCF) of the chunk at feature m0, sliced into buffer buf.
template <int RX, bool FACE>
__device__ __forceinline__ void tc_stage(int it, int m0, int M, int n, const float4* tsplit, const float4* pt,
                                         const int4* sline, uint2* buf) {
  using S = TcShape<RX>;
  const int cc = it & 3, gg = (it >> 2) & 7, half = (it >> 5) & 1;
  const int rest = it >> 6;
  const int ctl = rest % S::CT, ksl = rest / S::CT;
  const int f = m0 + ksl * 8 + half * 4 + cc;
  const int4 L = sline[ctl * 8 + gg];  // (sample, y or z, z, valid) of the block's line slot
  const bool valid = L.w != 0;
  const int si = L.x;
  uint32_t q[kTcSlices];
  if (valid && f < M) {
    if (FACE) {
      const float4 p = pt[((size_t)si * M + f) * n + L.y];
      float qr[kTcSlices], qi[kTcSlices];
      df::slice7(p.x, p.y, qr);
      df::slice7(p.z, p.w, qi);
#pragma unroll
      for (int j = 0; j < kTcSlices; ++j) q[j] = pack_bf16x2(qr[j], qi[j]);
    } else {
      const float4* Ty = tsplit + ((size_t)si * 3 + 1) * M * n;
      q_slices(Ty[(size_t)f * n + L.y], Ty[((size_t)M + f) * n + L.z], q);
    }
  } else {
#pragma unroll
    for (int j = 0; j < kTcSlices; ++j) q[j] = 0u;
  }
  uint32_t* dst =
      reinterpret_cast<uint32_t*>(buf) + ((size_t)(ksl * kTcSlices * S::CT + ctl) * 32 + gg * 4 + cc) * 2 + half;
#pragma unroll
  for (int j = 0; j < kTcSlices; ++j) dst[j * S::CT * 64] = q[j];
}

template <typename TOut, int RX, bool FACE>
__global__ void __launch_bounds__(kTcThreads, 1) k_field_tc(const float4* __restrict__ tsplit,
                                                             const float4* __restrict__ pt,
                                                             const uint4* __restrict__ Xf,
                                                             const float* __restrict__ e2tab, int B, int M, int n,
                                                             int KS, double scale, TOut* __restrict__ kout) {
  using S = TcShape<RX>;
  constexpr int IPK = 8 / RX;  // staged items per thread after each k-step
  extern __shared__ uint2 sq[];
  float* sacc = reinterpret_cast<float*>(sq + 2 * S::BUF);  // [32][kTcThreads]: th[16], tl[16]
  int4* sline = reinterpret_cast<int4*>(sacc + 32 * kTcThreads);  // [LQ]
  __shared__ float se2[64];
  const int RT = (n - 1) / 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, c = lane & 3;
  const int rt = blockIdx.x * RX + warp % RX;
  const int ct0 = (warp / RX) * 4;  // its column tiles in the block's staged chunk
  // the warp's line group: 32 consecutive lines of one sample (ceil(lines / 32) groups per
  // sample, 8 / RX groups per block; the last group of a sample is partly empty)
  const size_t nl = FACE ? (size_t)n : (size_t)n * n;
  const int lgps = (int)((nl + 31) / 32);
  const int glg = (int)blockIdx.y * (8 / RX) + warp / RX;
  int s = glg / lgps;
  const size_t wline0 = (size_t)(glg % lgps) * 32;
  const bool wvalid = s < B;
  if (!wvalid) s = B - 1;  // its products are computed and dropped
  const uint4* xa = Xf + (size_t)(s * RT + rt) * KS * kTcSlices * 32 + lane;
  if (threadIdx.x < 64) se2[threadIdx.x] = e2tab[threadIdx.x];
  for (int t = threadIdx.x; t < S::LQ; t += kTcThreads) {  // line slot t: column tile t / 8, lane row t % 8
    const int lg = (int)blockIdx.y * (8 / RX) + t / 32;
    const int ls = lg / lgps;
    const int line = (lg % lgps) * 32 + t % 32;
    const bool ok = ls < B && (size_t)line < nl;
    sline[t] = FACE ? make_int4(ls, line, 0, ok) : make_int4(ls, line % n, line / n, ok);
  }
#pragma unroll
  for (int q = 0; q < 32; ++q) sacc[q * kTcThreads + threadIdx.x] = 0.f;
  float acc[kTcSlices][4][4];
#pragma unroll
  for (int q = 0; q < kTcSlices; ++q)
#pragma unroll
    for (int ct = 0; ct < 4; ++ct)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[q][ct][e] = 0.f;
  uint4 a[kTcSlices];
#pragma unroll
  for (int i = 0; i < kTcSlices; ++i) a[i] = xa[i * 32];
  __syncthreads();  // the line table
#pragma unroll 1
  for (int r = 0; r < 8; ++r) tc_stage<RX, FACE>(threadIdx.x + r * kTcThreads, 0, M, n, tsplit, pt, sline, sq);
  __syncthreads();
  for (int m0 = 0, cb = 0; m0 < M; m0 += S::KCF, cb ^= 1) {
    const uint2* cur = sq + cb * S::BUF;
    uint2* nxt = sq + (cb ^ 1) * S::BUF;
    const bool more = m0 + S::KCF < M;
    const int ksb = m0 / 8;
    const int ksn = min(RX, KS - ksb);
    for (int ksl = 0; ksl < ksn; ++ksl) {
      const int ks = ksb + ksl;
      uint4 an[kTcSlices];
      if (ks + 1 < KS) {
#pragma unroll
        for (int i = 0; i < kTcSlices; ++i) an[i] = xa[((size_t)(ks + 1) * kTcSlices + i) * 32];
      } else {
#pragma unroll
        for (int i = 0; i < kTcSlices; ++i) an[i] = a[i];
      }
#pragma unroll
      for (int j = 0; j < kTcSlices; ++j) {
        uint2 b[4];
#pragma unroll
        for (int ct = 0; ct < 4; ++ct) b[ct] = cur[((ksl * kTcSlices + j) * S::CT + ct0 + ct) * 32 + lane];
#pragma unroll
        for (int i = kTcSlices - 1 - j; i >= 0; --i)  // the highest group first: its chain is the longest
#pragma unroll
          for (int ct = 0; ct < 4; ++ct) mma_bf16_16816(acc[i + j][ct], a[i], b[ct]);
      }
#pragma unroll
      for (int i = 0; i < kTcSlices; ++i) a[i] = an[i];
      if (more) {
#pragma unroll
        for (int r = 0; r < IPK; ++r)
          tc_stage<RX, FACE>(threadIdx.x + (ksl * IPK + r) * kTcThreads, m0 + S::KCF, M, n, tsplit, pt, sline, nxt);
      }
    }
    if ((m0 + S::KCF) % kTcFold == 0 || !more) {
#pragma unroll
      for (int ct = 0; ct < 4; ++ct)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float gs[kTcSlices], sh, sl;
#pragma unroll
          for (int q = 0; q < kTcSlices; ++q) {
            gs[q] = acc[q][ct][e];
            acc[q][ct][e] = 0.f;
          }
          df::sum7(gs, sh, sl);
          float* th = sacc + (ct * 4 + e) * kTcThreads + threadIdx.x;
          float* tl = th + 16 * kTcThreads;
          float h, l;
          df::add(*th, *tl, sh, sl, h, l);
          *th = h;
          *tl = l;
        }
    }
    __syncthreads();
  }
  const float sch = narrow(scale), scl = narrow(scale - widen(sch));
  TOut* out = kout + (size_t)s * n * n * n;
#pragma unroll
  for (int ct = 0; ct < 4; ++ct)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = 16 * rt + g + (e >> 1) * 8;
      const size_t line = wline0 + ct * 8 + 2 * c + (e & 1);
      if (!wvalid || line >= nl) continue;
      float yh, yl, eh, el;
      int m;
      const float* th = sacc + (ct * 4 + e) * kTcThreads + threadIdx.x;
      df::mul(th[0], th[16 * kTcThreads], sch, scl, yh, yl);
      df::exp_df(yh, yl, se2, se2 + 32, eh, el, m);
      const size_t o = FACE ? ((size_t)line * n + r) * n + (n - 1) : line * n + r;
      if constexpr (sizeof(TOut) == 8)
        out[o] = (widen(eh) + widen(el)) * __hiloint2double((m + 1023) << 20, 0);
      else
        out[o] = (m > -126 && m < 128) ? __fmul_rn(eh, __int_as_float((m + 127) << 23)) : ldexpf(eh, m);
    }
}

template <typename TOut, int RX, bool FACE>
int field_tc_launch(const float4* xsplit, const float4* pt, const uint4* Xf, const float* e2tab, int M, int n, int KS,
                    int B, double scale, void* kout, double bytes, double flops, cudaStream_t st, double share) {
  const size_t smem = TcShape<RX>::smem;
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_field_tc<TOut, RX, FACE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  MLMC_CUDA_TRY(attr);
  // line groups of 32 lines, ceil(lines / 32) per sample, 8 / RX per block; samples in
  // chunks that keep the grid's y-extent within 65535
  const size_t nl = FACE ? (size_t)n : (size_t)n * n;
  const size_t lgps = (nl + 31) / 32;
  const int per_chunk = (int)(65535 * (size_t)(8 / RX) / lgps);
  if (per_chunk < 1) {
    set_error("field: grid too large for the tensor-core form (n = %d)", n);
    return MLMC_ERR_INVALID;
  }
  const int RT = (n - 1) / 16;
  for (int s0 = 0; s0 < B; s0 += per_chunk) {
    const int b = B - s0 < per_chunk ? B - s0 : per_chunk;
    const dim3 grid((unsigned)(RT / RX), (unsigned)(((size_t)b * lgps + 8 / RX - 1) / (8 / RX)), 1u);
    MLMC_LAUNCH(FACE ? "field_tc_face" : "field_tc", bytes * share * b / B, flops * share * b / B, st,
                (k_field_tc<TOut, RX, FACE><<<grid, kTcThreads, smem, st>>>(
                    xsplit + (size_t)s0 * 3 * M * n, pt + (size_t)s0 * M * n,
                    Xf + (size_t)s0 * RT * KS * kTcSlices * 32, e2tab, b, M, n, KS, scale,
                    (TOut*)kout + (size_t)s0 * n * n * n)));
  }
  return MLMC_OK;
}

template <typename TOut, bool FACE>
int field_tc_dispatch(const float4* xsplit, const float4* pt, const uint4* Xf, const float* e2tab, int M, int n,
                      int KS, int B, double scale, void* kout, double bytes, double flops, cudaStream_t st,
                      double share) {
  const int rts = (n - 1) / 16;
  if (rts % 8 == 0)
    return field_tc_launch<TOut, 8, FACE>(xsplit, pt, Xf, e2tab, M, n, KS, B, scale, kout, bytes, flops, st, share);
  if (rts % 4 == 0)
    return field_tc_launch<TOut, 4, FACE>(xsplit, pt, Xf, e2tab, M, n, KS, B, scale, kout, bytes, flops, st, share);
  if (rts % 2 == 0)
    return field_tc_launch<TOut, 2, FACE>(xsplit, pt, Xf, e2tab, M, n, KS, B, scale, kout, bytes, flops, st, share);
  return field_tc_launch<TOut, 1, FACE>(xsplit, pt, Xf, e2tab, M, n, KS, B, scale, kout, bytes, flops, st, share);
}

// The volume product on the fifth-generation tensor cores (grids from n = 65): one block
// computes 128 lines by 64 x-values with tcgen05.mma (M = 128, N = 64, K = 16, bf16 operands
// from shared memory, FP32 accumulators in tensor memory: the seven slice groups take 7 x 64
// of the 512 columns). The A operand (the line factors' slices) is staged by all 256 threads
// into K-major core matrices; the B operand (the x-phasors' slices, the same for every line
// of a sample) is laid out in that form once per sample (k_uxslices) and brought in by one
// bulk copy per chunk. Chunks of two k-steps are double-buffered: one thread issues the 56
// products of a chunk and commits them to the buffer's mbarrier while the block stages the
// next chunk, so the staging's FP32 work runs under the tensor cores' work. Every 256
// features (and at the end) the group sums are read from tensor memory and folded into a
// double-float; the next product overwrites them. Every wait is bounded: a block whose wait
// runs out records *err, drains its copies and products, writes NaN to its nodes and frees
// its tensor memory.
constexpr int kUmM = 128, kUmN = 64, kUmKC = 2;

// Set to 1 by a tensor-core field block whose bounded wait ran out (field_wait_error_take).
__device__ int g_field_wait_err = 0;

static std::atomic<int> g_inject_wait{0};
void field_inject_wait_failure(int launches) { g_inject_wait.store(launches); }

int field_wait_error_take(cudaStream_t st) {
  int v = 0;
  if (cudaMemcpyFromSymbolAsync(&v, g_field_wait_err, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return 0;
  if (v) {
    static const int zero = 0;
    cudaMemcpyToSymbolAsync(g_field_wait_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
  }
  return v;
}
constexpr unsigned kUmCols = 512;
constexpr int kUmATile = kUmM * 32, kUmBTile = kUmN * 32;  // bytes of one (k-step, slice) tile
constexpr int kUmAChunk = kUmKC * kTcSlices * kUmATile, kUmBChunk = kUmKC * kTcSlices * kUmBTile;
constexpr int kUmStage = kUmAChunk + kUmBChunk;
constexpr size_t kUmSmem = 2 * (size_t)kUmStage + 128 + kUmM * sizeof(int2) + 64 * sizeof(float) + 64;

static bool umma_applies(int n) { return n >= 65 && (n - 1) % kUmN == 0; }

size_t tc_uxslice_bytes(int B, int M, int n) {
  return umma_applies(n) ? (size_t)B * ((n - 1) / kUmN) * ((M + 7) / 8) * kTcSlices * kUmBTile : 0;
}

// XU[s][x block][k-step][slice]: 64 x-rows by 16 k in K-major core matrices, (Re X, -Im X) of
// feature 8 ks + fl at k = 2 fl, 2 fl + 1. One thread per (sample, x block, k-step, x, feature).
__global__ void k_uxslices(const float4* __restrict__ xsplit, int B, int M, int n, int KS,
                           unsigned char* __restrict__ XU) {
  const int XB = (n - 1) / kUmN;
  const size_t total = (size_t)B * XB * KS * kUmN * 8;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int fl = (int)(t & 7);
    size_t r = t >> 3;
    const int xr = (int)(r % kUmN);
    r /= kUmN;
    const int ks = (int)(r % KS);
    r /= KS;
    const int xb = (int)(r % XB);
    const int s = (int)(r / XB);
    const int f = ks * 8 + fl;
    float re[kTcSlices], im[kTcSlices];
    if (f < M) {
      const float4 v = xsplit[((size_t)s * 3 * M + f) * n + xb * kUmN + xr];
      df::slice7(v.x, v.y, re);
      df::slice7(-v.z, -v.w, im);
    } else {
#pragma unroll
      for (int i = 0; i < kTcSlices; ++i) re[i] = im[i] = 0.f;
    }
    unsigned char* o = XU + (((size_t)(s * XB + xb) * KS + ks) * kTcSlices) * kUmBTile + umma::pair_offset(xr, fl);
#pragma unroll
    for (int i = 0; i < kTcSlices; ++i)
      *reinterpret_cast<uint32_t*>(o + (size_t)i * kUmBTile) = pack_bf16x2(re[i], im[i]);
  }
}

template <typename TOut, bool MULTI, int SW>
__global__ void __launch_bounds__(32 * (SW + 1), 1) k_field_umma(const float4* __restrict__ tsplit,
                                                               const unsigned char* __restrict__ XU,
                                                               const float* __restrict__ e2tab, int M, int n, int KS,
                                                               double scale, long long budget, int inject, int* err,
                                                               TOut* __restrict__ kout) {
  extern __shared__ unsigned char um_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)um_raw + 127) & ~(uintptr_t)127);
  int2* sline = reinterpret_cast<int2*>(sm + 2 * kUmStage);  // (y, z) of line slot l, y = -1: none
  float* se2 = reinterpret_cast<float*>(sline + kUmM);
  uint64_t* bfull = reinterpret_cast<uint64_t*>(se2 + 64);  // [2]: B chunk landed
  uint64_t* mdone = bfull + 2;                               // [2]: the chunk's products done
  uint64_t* never = mdone + 2;                               // fault injection: nothing arrives
  uint32_t* tslot = reinterpret_cast<uint32_t*>(never + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int s = blockIdx.z, xb = blockIdx.x, XB = (n - 1) / kUmN;
  const size_t n2 = (size_t)n * n, L0 = (size_t)blockIdx.y * kUmM;
  if (tid < kUmM) {
    const size_t line = L0 + tid;
    sline[tid] = line < n2 ? make_int2((int)(line % n), (int)(line / n)) : make_int2(-1, 0);
  }
  if (tid < 64) se2[tid] = e2tab[tid];
  if (tid == 0) {
    for (int q = 0; q < 2; ++q) {
      mbar_init(&bfull[q], 1);
      mbar_init(&mdone[q], 1);
    }
    mbar_init(never, 1);
    mbar_fence_init();
  }
  if (warp == 0) umma::alloc(tslot, kUmCols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = *tslot;
  const float4* Ty = tsplit + ((size_t)s * 3 + 1) * M * n;
  const float4* Tz = Ty + (size_t)M * n;
  const unsigned char* xu = XU + ((size_t)(s * XB + xb) * KS) * kTcSlices * kUmBTile;
  const uint32_t idesc = umma::idesc_bf16_f32(kUmM, kUmN);
  const int nchunks = (KS + kUmKC - 1) / kUmKC;
  // the thread's outputs: tensor-memory lane 32 (warp % 4) + lane, XW x-values from XW (warp / 4)
  // SW staging warps (they also read the accumulators out) and one issuing warp, warp SW
  constexpr int STAGERS = 32 * SW;
  const bool stager = warp < SW;
  const int issuer = STAGERS;  // the thread that issues the copies and the products
  constexpr int XW = kUmN / (SW / 4);
  const int myl = 32 * (warp & 3) + lane, xh = XW * (warp >> 2);
  const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)xh;
  // MULTI (more than 256 features): the double-float running sums of the folds
  float th[MULTI ? XW : 1], tl[MULTI ? XW : 1];
#pragma unroll
  for (int q = 0; q < (MULTI ? XW : 1); ++q) th[q] = tl[q] = 0.f;
  int last_commit = -1, last_copy = -1;  // (thread 0's) the last chunk whose products / copy were issued
  bool bad = false;                       // a bounded wait of this thread ran out
  auto wait = [&](uint64_t* mb, int chunk, long long bud) {
    if (!mbar_wait_bounded(mb, (unsigned)((chunk >> 1) & 1), bud)) {
      bad = true;
      atomicExch(err, 1);
    }
  };
  const float sch = narrow(scale), scl = narrow(scale - widen(sch));
  const size_t myline = L0 + myl;
  TOut* out = kout + (size_t)s * n2 * n + myline * n + xb * kUmN + xh;
  // the groups' current sums of the thread's 32 x-values: folded into (th, tl) (last = false)
  // or, with the earlier folds, turned into k and stored (last = true)
  auto fold = [&](bool last) {
#pragma unroll
    for (int c0 = 0; c0 < XW; c0 += 8) {
      float v[kTcSlices][8];
#pragma unroll
      for (int g = 0; g < kTcSlices; ++g) umma::ld8(trow + (uint32_t)(g * kUmN + c0), v[g]);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float gs[kTcSlices], sh, sl;
#pragma unroll
        for (int g = 0; g < kTcSlices; ++g) gs[g] = v[g][q];
        df::sum7(gs, sh, sl);
        if (MULTI) df::add(th[c0 + q], tl[c0 + q], sh, sl, sh, sl);
        if (!last) {
          if (MULTI) {
            th[c0 + q] = sh;
            tl[c0 + q] = sl;
          }
          continue;
        }
        if (myline >= n2) continue;
        float yh, yl, eh, el;
        int m;
        df::mul(sh, sl, sch, scl, yh, yl);
        df::exp_df(yh, yl, se2, se2 + 32, eh, el, m);
        if constexpr (sizeof(TOut) == 8)
          out[c0 + q] = (widen(eh) + widen(el)) * __hiloint2double((m + 1023) << 20, 0);
        else
          out[c0 + q] = (m > -126 && m < 128) ? __fmul_rn(eh, __int_as_float((m + 127) << 23)) : ldexpf(eh, m);
      }
    }
  };
  // (thread 0) the bulk copy of chunk cc's x-slices into its buffer
  auto issue_copy = [&](int cc) {
    const int k0 = cc * kUmKC, kk = min(kUmKC, KS - k0);
    const unsigned bytes = (unsigned)(kk * kTcSlices * kUmBTile);
    mbar_arrive_expect_tx(&bfull[cc & 1], bytes);
    bulk_g2s(sm + (size_t)(cc & 1) * kUmStage + kUmAChunk, xu + (size_t)k0 * kTcSlices * kUmBTile, bytes,
             &bfull[cc & 1]);
    last_copy = cc;
  };
  if (tid == issuer) {
    issue_copy(0);
    if (inject) wait(never, 0, budget);  // injected failure: runs out after the budget
  }
  for (int c = 0; c < nchunks; ++c) {
    const int b = c & 1;
    const int ks0 = c * kUmKC, kn = min(kUmKC, KS - ks0);
    unsigned char* sA = sm + (size_t)b * kUmStage;
    unsigned char* sB = sA + kUmAChunk;
    // the buffer is free once the products of chunk c - 2 are done
    if (c >= 2) wait(&mdone[b], c - 2, budget);
    umma::fence_after_sync();
    // staging: 2048 / STAGERS (line, feature) items per staging thread, their table loads
    // issued four at a time
#pragma unroll 1
    for (int h = 0; h < 2048 / STAGERS / 4 && stager && !bad; ++h) {
      float4 bq[4], dq[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int it = tid + (4 * h + r) * STAGERS;
        const int fl4 = it & 3, rr = (it >> 2) & 7, kg = (it >> 5) & 1, rg = (it >> 6) & 15, ksl = it >> 10;
        const int f = (ks0 + ksl) * 8 + kg * 4 + fl4;
        const int2 yz = sline[rg * 8 + rr];
        if (ksl < kn && yz.x >= 0 && f < M) {
          bq[r] = Ty[(size_t)f * n + yz.x];
          dq[r] = Tz[(size_t)f * n + yz.y];
        } else {
          bq[r] = dq[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int it = tid + (4 * h + r) * STAGERS;
        const int fl4 = it & 3, rr = (it >> 2) & 7, kg = (it >> 5) & 1, rg = (it >> 6) & 15, ksl = it >> 10;
        if (ksl >= kn) continue;
        uint32_t q[kTcSlices];
        q_slices(bq[r], dq[r], q);  // zero tables give zero slices
        unsigned char* dst = sA + (size_t)ksl * kTcSlices * kUmATile + umma::pair_offset(rg * 8 + rr, kg * 4 + fl4);
#pragma unroll
        for (int j = 0; j < kTcSlices; ++j) *reinterpret_cast<uint32_t*>(dst + (size_t)j * kUmATile) = q[j];
      }
    }
    fence_proxy_async();
    umma::fence_before_sync();
    bad = __syncthreads_or(bad);
    if (bad) break;
    if (tid == issuer) {
      // the x-slices of chunk c + 1 go to the other buffer once the products of chunk c - 1,
      // its last readers, are done (they are by now as a rule), a chunk ahead of their use
      if (c + 1 < nchunks) {
        if (c >= 1) wait(&mdone[b ^ 1], c - 1, budget);
        if (!bad) issue_copy(c + 1);
      }
      if (!bad) wait(&bfull[b], c, budget);
      if (!bad) {
        umma::fence_after_sync();
        const bool fresh = (ks0 * 8) % kTcFold == 0;  // the first chunk of a fold period
        // a tile's descriptor is the chunk base's plus its byte offset / 16 (shared-memory
        // addresses stay below 2^18, so the 14-bit address field does not carry)
        const uint64_t ad0 = umma::smem_desc(smem_addr(sA), umma::kLeadingBytes, umma::kStrideBytes);
        const uint64_t bd0 = umma::smem_desc(smem_addr(sB), umma::kLeadingBytes, umma::kStrideBytes);
#pragma unroll
        for (int ksl = 0; ksl < kUmKC; ++ksl) {
          if (ksl >= kn) break;
#pragma unroll
          for (int j = 0; j < kTcSlices; ++j)
#pragma unroll
            for (int i = kTcSlices - 1 - j; i >= 0; --i)
              umma::mma_bf16(tmem + (uint32_t)((i + j) * kUmN),
                             ad0 + (uint64_t)(((ksl * kTcSlices + i) * kUmATile) >> 4),
                             bd0 + (uint64_t)(((ksl * kTcSlices + j) * kUmBTile) >> 4), idesc,
                             (fresh && ksl == 0 && j == 0) ? 0u : 1u);
        }
        umma::commit(&mdone[b]);
        last_commit = c;
      }
    }
    // every 256 features, before the next chunk overwrites the groups: fold them
    if (((ks0 + kn) * 8) % kTcFold == 0 && c + 1 < nchunks) {
      bad = __syncthreads_or(bad);
      if (bad) break;
      wait(&mdone[b], c, budget);
      umma::fence_after_sync();
      bad = __syncthreads_or(bad);
      if (bad) break;
      if (stager) fold(false);
      umma::fence_before_sync();
      __syncthreads();
    }
  }
  bad = __syncthreads_or(bad);
  if (!bad) wait(&mdone[(nchunks - 1) & 1], nchunks - 1, budget);
  bad = __syncthreads_or(bad);
  if (bad && tid == issuer) {
    // drain: the last issued products and copy land before the block leaves
    if (last_commit >= 0) mbar_wait_bounded(&mdone[last_commit & 1], (unsigned)((last_commit >> 1) & 1), kDrainBudget);
    for (int cc = last_copy - 1; cc <= last_copy; ++cc)  // the copies run up to one chunk ahead
      if (cc >= 0) mbar_wait_bounded(&bfull[cc & 1], (unsigned)((cc >> 1) & 1), kDrainBudget);
  }
  umma::fence_after_sync();
  if (!stager) {
  } else if (!bad) {
    fold(true);
  } else if (myline < n2) {
#pragma unroll 4
    for (int q = 0; q < XW; ++q) out[q] = (TOut)__int_as_float(0x7fc00000);
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::dealloc(tmem, kUmCols);
}

template <typename TOut>
int field_umma_launch(const float4* xsplit, const unsigned char* XU, const float* e2tab, int M, int n,
                      int KS, int B, double scale, void* kout, double bytes, double flops, cudaStream_t st,
                      double share) {
  // one fold (up to 256 features): 16 staging warps at 120 registers; more: 8, which also hold
  // the running double-float sums; and the issuing warp
  static const cudaError_t attr1 = cudaFuncSetAttribute(k_field_umma<TOut, false, 16>,
                                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUmSmem);
  static const cudaError_t attr2 = cudaFuncSetAttribute(k_field_umma<TOut, true, 8>,
                                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUmSmem);
  MLMC_CUDA_TRY(attr1);
  MLMC_CUDA_TRY(attr2);
  const dim3 grid((unsigned)((n - 1) / kUmN), (unsigned)(((size_t)n * n + kUmM - 1) / kUmM), (unsigned)B);
  const long long budget = wait_budget_clocks();
  int inject = 0;
  for (int left = g_inject_wait.load(); left > 0; left = g_inject_wait.load())
    if (g_inject_wait.compare_exchange_weak(left, left - 1)) {
      inject = 1;
      break;
    }
  static int* const err = [] {
    void* p = nullptr;
    return cudaGetSymbolAddress(&p, g_field_wait_err) == cudaSuccess ? (int*)p : nullptr;
  }();
  if (!err) {
    set_error("field: no address for the wait-error flag");
    return MLMC_ERR_CUDA;
  }
  if (M > kTcFold)
    MLMC_LAUNCH("field_tc", bytes * share, flops * share, st,
                (k_field_umma<TOut, true, 8><<<grid, 32 * 9, kUmSmem, st>>>(xsplit, XU, e2tab, M, n, KS, scale, budget,
                                                                             inject, err, (TOut*)kout)));
  else
    MLMC_LAUNCH("field_tc", bytes * share, flops * share, st,
                (k_field_umma<TOut, false, 16><<<grid, 32 * 17, kUmSmem, st>>>(xsplit, XU, e2tab, M, n, KS, scale,
                                                                                budget, inject, err, (TOut*)kout)));
  return MLMC_OK;
}

// All of the tensor-core form: slices of the x- and y-phasors, the face factors, the volume
// x < n - 1 (tcgen05 from n = 65 unless warp_mma, warp-level mma.sync otherwise), the face
// x = n - 1 (y < n - 1), the edge x = y = n - 1.
template <typename TOut>
int field_tc_all(const double2* tab, const float4* xsplit, float4* pt, uint4* Xf, unsigned char* XU, float* e2tab, int M, int n, int B, double scale, void* kout, double bytes, double flops,
                 cudaStream_t st, bool warp_mma) {
  const int KS = (M + 7) / 8;
  const size_t nxs = (size_t)B * ((n - 1) / 16) * KS * 32;
  const bool umma_volume = !warp_mma && umma_applies(n);
  const int axis0 = umma_volume ? 1 : 0;  // the tcgen05 volume takes its x-slices from k_uxslices
  MLMC_LAUNCH("xslices", (double)nxs * (2 - axis0) * 112.0, (double)nxs * (2 - axis0) * 500.0, st,
              (k_xslices<<<blocks_for((2 - axis0) * nxs, 256), 256, 0, st>>>(xsplit, B, M, n, KS, axis0, Xf,
                                                                               e2tab)));
  const size_t nf = (size_t)B * M * n;
  MLMC_LAUNCH("face_factors", (double)nf * 48.0, (double)nf * 40.0, st,
              (k_face_factors<<<blocks_for(nf, 256), 256, 0, st>>>(xsplit, B, M, n, pt)));
  const double n3 = (double)n * n * n;
  const double vshare = (double)(n - 1) * n * n / n3;
  if (umma_volume) {
    const size_t nux = (size_t)B * ((n - 1) / kUmN) * KS * kUmN * 8;
    MLMC_LAUNCH("xslices", (double)nux * 28.0, (double)nux * 250.0, st,
                (k_uxslices<<<blocks_for(nux, 256), 256, 0, st>>>(xsplit, B, M, n, KS, XU)));
    MLMC_TRY(field_umma_launch<TOut>(xsplit, XU, e2tab, M, n, KS, B, scale, kout, bytes, flops, st, vshare));
  } else {
    MLMC_TRY((field_tc_dispatch<TOut, false>(xsplit, pt, Xf, e2tab, M, n, KS, B, scale, kout, bytes, flops, st,
                                             vshare)));
  }
  MLMC_TRY((field_tc_dispatch<TOut, true>(xsplit, pt, Xf + nxs * kTcSlices, e2tab, M, n, KS, B, scale, kout, bytes,
                                          flops, st, (double)(n - 1) * n / n3)));
  MLMC_LAUNCH("field_edge", bytes * n / n3, flops * n / n3, st,
              (k_field_edge<TOut><<<(unsigned)(((size_t)B * n + 3) / 4), 128, 0, st>>>(tab, B, M, n, scale,
                                                                                       (TOut*)kout)));
  return MLMC_OK;
}

// The tensor-core form applies where the x-values below n - 1 make whole row tiles.
static bool tc_applies(int n) { return n >= 17 && (n - 1) % 16 == 0; }

size_t field_scratch_bytes(int B, int M, int n) {
  return a256((size_t)B * M * 3 * sizeof(double)) + a256((size_t)B * M * sizeof(double)) +
         a256((size_t)B * 3 * M * n * sizeof(double2)) + a256((size_t)B * 3 * M * n * sizeof(float4)) +
         (tc_applies(n) ? a256(2 * tc_xslice_bytes(B, M, n)) + a256(64 * sizeof(float)) +
                              a256((size_t)B * M * n * sizeof(float4)) + a256(tc_uxslice_bytes(B, M, n))
                        : 0);
}

int field_arith_default() {
  static const int a = [] {
    const char* e = getenv("MLMC_FIELD_ARITH");
    const int v = e ? atoi(e) : (int)kFieldTC;
    return v >= kFieldDF32Line && v <= kFieldTCWarp ? v : (int)kFieldTC;
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
  uint4* Xf = tc_applies(n) ? (uint4*)carve(2 * tc_xslice_bytes(B, cfg.M, n)) : nullptr;
  float* e2tab = tc_applies(n) ? (float*)carve(64 * sizeof(float)) : nullptr;
  float4* pt = tc_applies(n) ? (float4*)carve((size_t)B * cfg.M * n * sizeof(float4)) : nullptr;
  unsigned char* XU = tc_applies(n) ? (unsigned char*)carve(tc_uxslice_bytes(B, cfg.M, n)) : nullptr;
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
  } else if (arith == kFieldDF32Line || arith == kFieldTC || arith == kFieldTCWarp) {
    const int MCl = cfg.M < 64 ? cfg.M : 64;
    const unsigned lines = (unsigned)(((size_t)n * n + kFieldThreads - 1) / kFieldThreads);
    if ((arith == kFieldTC || arith == kFieldTCWarp) && tc_applies(n)) {
      const bool warp_mma = arith == kFieldTCWarp;
      if (dtype == MLMC_F64)
        MLMC_TRY(field_tc_all<double>(tab, xsplit, pt, Xf, XU, e2tab, cfg.M, n, B, scale, kout, bytes, flops, st,
                                      warp_mma));
      else
        MLMC_TRY(field_tc_all<float>(tab, xsplit, pt, Xf, XU, e2tab, cfg.M, n, B, scale, kout, bytes, flops, st,
                                     warp_mma));
    } else {
      // x < n - 1 in tiles of 8 (of 4 on the 5-node grid), then x = n - 1
      const int xt = (n - 1) % kXC == 0 ? kXC : 4;
      const unsigned tiles = (unsigned)((n - 1) / xt);
      if (xt == kXC)
        MLMC_TRY(field_line_launch<kXC>(xsplit, cfg.M, n, MCl, 0, tiles, lines, B, scale, dtype, kout, bytes, flops,
                                       st, (double)(n - 1) / n));
      else
        MLMC_TRY(field_line_launch<4>(xsplit, cfg.M, n, MCl, 0, tiles, lines, B, scale, dtype, kout, bytes, flops, st,
                                     (double)(n - 1) / n));
      MLMC_TRY(field_line_launch<1>(xsplit, cfg.M, n, MCl, n - 1, 1, lines, B, scale, dtype, kout, bytes, flops, st,
                                   1.0 / n));
    }
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
