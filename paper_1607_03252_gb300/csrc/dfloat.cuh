// Double-float arithmetic (a value is the unevaluated sum hi + lo of two binary32 numbers,
// |lo| <= ulp(hi) / 2) for the tensor-core field evaluation, and the two steps that bracket
// its tensor-core sum: the split of a double-float into seven bf16 slices on fixed grids,
// and exp of a double-float.
//
// The functions are plain C++ on the host (the host tests build them with g++ and
// -ffp-contract=off) and use the round-to-nearest intrinsics on the device, which the
// compiler never fuses into an FMA: the error-free transformations below rely on every
// product and sum being rounded once, as written.
#pragma once

#if defined(__CUDACC__)
#include <cuda_runtime.h>
#define MLMC_DF_HD __host__ __device__ __forceinline__
#else
#include <math.h>
#define MLMC_DF_HD static inline
#endif

namespace mlmc {
namespace df {

#if defined(__CUDA_ARCH__)
MLMC_DF_HD float add(float a, float b) { return __fadd_rn(a, b); }
MLMC_DF_HD float sub(float a, float b) { return __fsub_rn(a, b); }
MLMC_DF_HD float mul(float a, float b) { return __fmul_rn(a, b); }
MLMC_DF_HD float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
MLMC_DF_HD float rint(float a) { return rintf(a); }
#else
MLMC_DF_HD float add(float a, float b) { return a + b; }
MLMC_DF_HD float sub(float a, float b) { return a - b; }
MLMC_DF_HD float mul(float a, float b) { return a * b; }
MLMC_DF_HD float fma(float a, float b, float c) { return fmaf(a, b, c); }
MLMC_DF_HD float rint(float a) { return rintf(a); }
#endif

// s + e = a + b exactly, s = fl(a + b) (Knuth's TwoSum, no condition on the magnitudes)
MLMC_DF_HD void two_sum(float a, float b, float& s, float& e) {
  s = add(a, b);
  const float bv = sub(s, a);
  e = add(sub(a, sub(s, bv)), sub(b, bv));
}
// the same for |a| >= |b| or a == 0 (Dekker's FastTwoSum)
MLMC_DF_HD void fast_two_sum(float a, float b, float& s, float& e) {
  s = add(a, b);
  e = sub(b, sub(s, a));
}
// (ph, pl) = (ah + al)(bh + bl), renormalised; relative error below 2^-45
MLMC_DF_HD void mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
  const float p = mul(ah, bh);
  float e = fma(ah, bh, -p);
  e = fma(ah, bl, e);
  e = fma(al, bh, e);
  fast_two_sum(p, e, ph, pl);
}
// (sh, sl) = (ah + al) + (bh + bl), renormalised
MLMC_DF_HD void add(float ah, float al, float bh, float bl, float& sh, float& sl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e = add(e, add(al, bl));
  fast_two_sum(s, e, sh, sl);
}

// Seven slices of v = h + l (|v| <= 1 + 2^-20, |l| <= ulp(h)): t[i] is an integer multiple of
// 2^(-7(i+1)) with |t[0]| <= 1, |t[3]| <= 72 * 2^-28 and |t[i]| <= 64 * 2^(-7(i+1)) otherwise, so
// every slice has at most 8 significant bits (exact in bf16), and |v - sum t| <= 2^-50 + 2^-60.
// A slice is v rounded to its grid by adding and subtracting 1.5 * 2^23 times the grid step
// (the sum lands in the binade whose ulp is the step); the remainder is exact. The first three
// come from h alone; l is added before the fourth, that sum's error before the sixth. Both
// additions are FastTwoSum: the remainder is a multiple of the ulp of the value it came from
// (h, then the first sum), so it is zero or at least as large as the addend (at most half that
// ulp), which makes FastTwoSum exact.
MLMC_DF_HD void slice7(float h, float l, float t[7]) {
  const float C0 = 98304.f;                     // 1.5 * 2^16: step 2^-7
  const float C1 = 768.f;                       // 1.5 * 2^9: 2^-14
  const float C2 = 6.f;                         // 1.5 * 2^2: 2^-21
  const float C3 = 0.046875f;                   // 1.5 * 2^-5: 2^-28
  const float C4 = 3.662109375e-4f;             // 1.5 * 2^-12: 2^-35
  const float C5 = 2.86102294921875e-6f;        // 1.5 * 2^-19: 2^-42
  const float C6 = 2.2351741790771484375e-8f;   // 1.5 * 2^-26: 2^-49
  float r = h, e, e2;
  t[0] = sub(add(r, C0), C0);
  r = sub(r, t[0]);
  t[1] = sub(add(r, C1), C1);
  r = sub(r, t[1]);
  t[2] = sub(add(r, C2), C2);
  r = sub(r, t[2]);
  fast_two_sum(r, l, r, e);
  t[3] = sub(add(r, C3), C3);
  r = sub(r, t[3]);
  t[4] = sub(add(r, C4), C4);
  r = sub(r, t[4]);
  fast_two_sum(r, e, r, e2);
  t[5] = sub(add(r, C5), C5);
  r = sub(r, t[5]);
  t[6] = sub(add(r, C6), C6);
  (void)e2;  // below 2^-60, dropped
}

// Sum of the seven slice-group sums g[0..6] (largest first) as a renormalised double-float.
MLMC_DF_HD void sum7(const float g[7], float& sh, float& sl) {
  float h = g[0], l = 0.f, e;
#pragma unroll
  for (int i = 1; i < 7; ++i) {
    two_sum(h, g[i], h, e);
    l = add(l, e);
  }
  fast_two_sum(h, l, sh, sl);
}

// exp(yh + yl) = (eh + el) * 2^m for |yh| < 88 (|N| below 2^12 keeps N * L1 exact), by Tang's
// table-driven method (P. T. P. Tang, ACM Trans. Math. Softw. 15(2), 1989): with N the integer
// nearest to y 32/ln2, j = N mod 32 and m = (N - j) / 32, exp(y) = 2^m 2^(j/32) exp(r) with
// r = y - N ln2/32, |r| <= ln2/64 (+ rounding). ln2/32 is carried as L1 + L2 + L3 (L1 with 12
// significant bits, so N L1 and yh - N L1 are exact; the three agree with ln2/32 to 4e-22).
// exp(r) is its Taylor polynomial to r^6 (remainder below 4e-18) by Horner's rule, the inner
// factor 1/24 + r/120 + r^2/720 in binary32, the outer three steps in double-float. tab_h/tab_l
// hold 2^(j/32), j = 0..31, as double-floats. Relative error below ~1e-14.
MLMC_DF_HD void exp_df(float yh, float yl, const float* tab_h, const float* tab_l, float& eh, float& el, int& m) {
  const float kInvL = 46.16624069213867f;        // 32 / ln2 (only the choice of N depends on it)
  const float L1 = 0.02165985107421875f;         // 0x1.62ep-6
  const float L2 = 9.983182280848268e-07f;       // 0x1.0bfbe8p-20
  const float L3 = 5.14560928046269e-14f;        // 0x1.cf79acp-45
  const float Nf = rint(mul(yh, kInvL));
  const int N = (int)Nf;
  const int j = N & 31;
  m = (N - j) / 32;
  // r = y - N (L1 + L2 + L3)
  const float a = sub(yh, mul(Nf, L1));          // exact (Sterbenz, or N = 0)
  const float p2 = mul(Nf, L2);
  const float p2e = fma(Nf, L2, -p2);
  float rh, rl, e;
  two_sum(a, -p2, rh, rl);
  two_sum(rh, yl, rh, e);  // yl reaches 4e-6 at |y| = 80: it must not be rounded to rl's ulp
  rl = add(add(rl, e), -add(p2e, mul(Nf, L3)));
  fast_two_sum(rh, rl, rh, rl);
  // Horner: e^r = 1 + r (1 + r (1/2 + r (1/6 + r (1/24 + r/120 + r^2/720))))
  const float q = fma(rh, fma(rh, 1.3888889225e-3f, 8.3333337680e-3f), 4.1666667908e-2f);
  float th, tl;
  fast_two_sum(0.16666667163372040f, mul(rh, q), th, tl);   // 1/6 = 0x1.555556p-3 - 0x1.555556p-28
  tl = add(tl, -4.9670538793e-09f);
  float ph, pl;
  mul(rh, rl, th, tl, ph, pl);
  float uh, ul;
  fast_two_sum(0.5f, ph, uh, ul);
  ul = add(ul, pl);
  mul(rh, rl, uh, ul, ph, pl);
  fast_two_sum(1.f, ph, uh, ul);
  ul = add(ul, pl);
  mul(rh, rl, uh, ul, ph, pl);
  fast_two_sum(1.f, ph, uh, ul);
  ul = add(ul, pl);
  mul(tab_h[j], tab_l[j], uh, ul, eh, el);
}

}  // namespace df

}  // namespace mlmc
