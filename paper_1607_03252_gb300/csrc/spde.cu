// SPDE field sampler (Sec. 3.2): the lognormal coefficient k = exp(Z) with Z the solution
// of (kappa^2 - Laplace) Z = W, W Gaussian white noise, whose covariance in R^3 is
// (8 pi kappa)^-1 exp(-kappa r) (Whittle): kappa = 1 / ell and log k =
// sqrt(8 pi kappa sigma^2) Z give the exponential covariance sigma^2 exp(-r / ell).
//
// Discretisation: cell-centred finite volumes on the zero-flux box of C = 2(n-1) cells of
// side h = 1/(n-1) per axis around D, cell i centred at -1/2 + i h (D's node j is cell
// j + (n-1)/2). Scaled by 1/h, cell p reads (kappa^2 h^2 + n_p) Z_p - sum_q Z_q =
// W(cell p) / h (n_p face neighbours inside the box). W(cell) is exact white noise over
// the cell: a sum of the standard normals of the octants (cubes of side h_f / 2 of the
// pair's fine spacing h_f) that tile it, times (h_f / 2)^(3/2), so the fine and the
// coarse grid of one sample share one realisation of W.
//
// Normals: Marsaglia's polar method on Philox4x32-10 words in FP32, every operation a
// correctly rounded one (the _rn intrinsics: no contraction, no approximate division),
// with the logarithm written out below, so the normals are reproducible bit for bit.
//
// Solver: iterative refinement. Each step computes the FP64 residual r = g - A Z (also the
// convergence test), and an FP32 V(2,2) cycle of cell-centred multigrid with constant
// coefficients (the box is the same on every grid: C, C/2, ..., 2 cells) solves A e = r
// approximately: red-black Gauss-Seidel, residual, restriction by the mean of the 8 child
// cells, trilinear cell-centred prolongation (weights 3/4, 1/4 per axis, the outside
// neighbour replaced by the cell itself at the box faces), and the exact solve of the 2^3
// grid in the eigenbasis of its operator; then Z += e in FP64. GB300's FP64 unit runs at
// 1/64 of the FP32 rate: an all-FP64 cycle spends about 80 FP64 operations per cell and is
// bound by that unit, this scheme about 11 (the residual and the update). No coefficient
// arrays: every kernel streams Z and the right-hand side only.
#include <math.h>

#include "common.cuh"
#include "philox.cuh"
#include "prof.cuh"
#include "spde.cuh"
#include "widen.cuh"

namespace mlmc {
namespace {

constexpr int kT = 256;

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

// ln s for normal s > 0: s = m 2^e, m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(t) =
// 2 t (1 + t^2/3 + ... + t^10/11), t = (m - 1)/(m + 1), |t| < 0.172; plus e ln 2 with ln 2
// split into a 16-bit head and a tail (Cody and Waite). Every step rounds once.
__device__ __forceinline__ float log_series(float s) {
  const unsigned b = __float_as_uint(s);
  int e = (int)((b >> 23) & 0xffu) - 127;
  float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
  if (m > 0x1.6a09e6p+0f) {
    m = __fmul_rn(0.5f, m);
    e += 1;
  }
  const float t = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float t2 = __fmul_rn(t, t);
  float p = __fmaf_rn(t2, 0x1.745d18p-4f, 0x1.c71c72p-4f);
  p = __fmaf_rn(t2, p, 0x1.24924ap-3f);
  p = __fmaf_rn(t2, p, 0x1.99999ap-3f);
  p = __fmaf_rn(t2, p, 0x1.555556p-2f);
  p = __fmaf_rn(t2, p, 1.0f);
  const float lm = __fmul_rn(__fmul_rn(2.0f, t), p);
  const float fe = (float)e;
  return __fmaf_rn(fe, 0x1.62e400p-1f, __fmaf_rn(fe, 0x1.7f7d1cp-20f, lm));
}

// A word w gives U = ((w >> 8) - 2^23 + 1/2) 2^-23 in (-1, 1), exactly.
__device__ __forceinline__ float unit_pm(uint32_t w) {
  return __fmul_rn(__fadd_rn((float)((int)(w >> 8) - 8388608), 0.5f), 0x1p-23f);
}

// Standard normal of octant `oct`: attempt a = 0..31 uses the word pair (2(a&1), 2(a&1)+1)
// of Philox with counter (id lo, id hi, oct lo, 0x5D000000 | (a >> 1) << 8 | oct >> 32);
// the first pair with 0 < s = U1^2 + U2^2 < 1 gives U1 sqrt(-2 ln s / s); 0 if none.
__device__ float octant_normal(uint32_t k0, uint32_t k1, uint64_t id, uint64_t oct) {
  for (int call = 0; call < 16; ++call) {
    uint32_t c0 = (uint32_t)id, c1 = (uint32_t)(id >> 32), c2 = (uint32_t)oct,
             c3 = 0x5D000000u | ((uint32_t)call << 8) | (uint32_t)(oct >> 32);
    philox10(c0, c1, c2, c3, k0, k1);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const float u1 = unit_pm(half ? c2 : c0), u2 = unit_pm(half ? c3 : c1);
      const float sq = __fmaf_rn(u1, u1, __fmul_rn(u2, u2));
      if (sq > 0.0f && sq < 1.0f) {
        const float q = __fdiv_rn(__fmul_rn(-2.0f, log_series(sq)), sq);
        return __fmul_rn(u1, __fsqrt_rn(q));
      }
    }
  }
  return 0.0f;
}

// g = W(cell) / h for every cell of B samples: the octants of cell i along an axis are
// 2 r i + 2 - r .. 2 r i + 1 + r (r = h / h_f), of Mo per axis; sums in z, y, x order.
// Grid (cells / blockDim, samples): C = 2^lc cells per axis, x = i mod C, ...
__global__ void k_spde_noise(const uint64_t* __restrict__ ids, int B, int lc, int r, uint64_t Mo, uint32_t k0,
                             uint32_t k1, double scale, double* __restrict__ g) {
  const int C = 1 << lc;
  const size_t C3 = (size_t)1 << (3 * lc);
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C3) return;
  const int x = (int)(i & (C - 1)), y = (int)((i >> lc) & (C - 1)), z = (int)(i >> (2 * lc));
  for (int s = blockIdx.y; s < B; s += gridDim.y) {
    const size_t t = (size_t)s * C3 + i;
    const uint64_t id = ids[s];
    const long az0 = 2L * r * z + 2 - r, ay0 = 2L * r * y + 2 - r, ax0 = 2L * r * x + 2 - r;
    double sum = 0.0;
    for (long az = az0; az < az0 + 2 * r; ++az)
      for (long ay = ay0; ay < ay0 + 2 * r; ++ay)
        for (long ax = ax0; ax < ax0 + 2 * r; ++ax)
          sum += (double)octant_normal(k0, k1, id, ((uint64_t)az * Mo + (uint64_t)ay) * Mo + (uint64_t)ax);
    g[t] = scale * sum;
  }
}

// One colour of red-black Gauss-Seidel (red: x + y + z even):
// Z_p = (g_p + sum of the neighbours inside the box) / (c h^2 + n_p), with the four
// possible reciprocals of the diagonal precomputed.
// Grid (colour cells / blockDim, samples), C = 2^lc >= 4.
template <typename T>
__global__ void k_cc_rbgs(int colour, int lc, int B, T i3, T i4, T i5, T i6, const T* __restrict__ g,
                          T* __restrict__ Z, const int* __restrict__ active) {
  const int C = 1 << lc;
  const size_t C3 = (size_t)1 << (3 * lc), C2 = (size_t)1 << (2 * lc);
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (C3 >> 1)) return;
  const int xi = (int)(q & ((C >> 1) - 1));
  const size_t row = q >> (lc - 1);
  const int y = (int)(row & (C - 1)), z = (int)(row >> lc);
  const int x = 2 * xi + ((y + z + colour) & 1);
  for (int s = blockIdx.y; s < B; s += gridDim.y) {
    if (!active[s]) continue;
    const size_t p = (size_t)s * C3 + ((size_t)z << (2 * lc)) + ((size_t)y << lc) + x;
    T acc = g[p];
    int np = 0;
    if (x > 0) { acc += Z[p - 1]; ++np; }
    if (x < C - 1) { acc += Z[p + 1]; ++np; }
    if (y > 0) { acc += Z[p - C]; ++np; }
    if (y < C - 1) { acc += Z[p + C]; ++np; }
    if (z > 0) { acc += Z[p - C2]; ++np; }
    if (z < C - 1) { acc += Z[p + C2]; ++np; }
    Z[p] = acc * (np == 6 ? i6 : (np == 5 ? i5 : (np == 4 ? i4 : i3)));
  }
}

template <int THREADS>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double part[THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) part[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = lane < THREADS / 32 ? part[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;
}

// z-slabs of the column kernels: a function of C only (a sample's sums never depend on its
// batch), enough (column block, slab) pairs to fill the GPU for one sample, slabs at least
// 8 cells deep so that carrying Z of the planes below and above in registers pays.
int zslabs(int C, int* zslab) {
  long long slabs = (131072LL + (long long)C * C - 1) / ((long long)C * C);
  const int deep = C / 8 > 1 ? C / 8 : 1;
  if (slabs > deep) slabs = deep;
  if (slabs < 1) slabs = 1;
  *zslab = (int)((C + slabs - 1) / slabs);
  return (C + *zslab - 1) / *zslab;
}
int col_blocks(int C) { return (C * C + 127) / 128; }

// r = g - A Z (stored if r != NULL) by column z-marches, and per-(column block, slab)
// partial sums of r^2 (of g^2 when Z == NULL) if partial != NULL. Grid (column blocks,
// slabs, B), 128 threads: thread column x + C y, planes z0 .. z0 + zslab - 1.
template <typename T, typename TR>
__global__ void __launch_bounds__(128) k_cc_residual(int lc, int zslab, T ch2, const T* __restrict__ g,
                                                     const T* __restrict__ Z, TR* __restrict__ r,
                                                     double* __restrict__ partial, const int* __restrict__ active) {
  const int s = blockIdx.z;
  if (!active[s]) return;
  const int C = 1 << lc;
  const size_t C2 = (size_t)1 << (2 * lc), C3 = C2 << lc;
  const int c = blockIdx.x * 128 + threadIdx.x;
  const int z0 = blockIdx.y * zslab, z1 = min(C, z0 + zslab);
  double sq = 0.0;
  if (c < C * C) {
    const int x = c & (C - 1), y = c >> lc;
    const size_t base = (size_t)s * C3 + c;
    if (Z) {
      const int nxy = (x > 0) + (x < C - 1) + (y > 0) + (y < C - 1);
      T zm = z0 > 0 ? Z[base + (size_t)(z0 - 1) * C2] : T(0);
      T zc = Z[base + (size_t)z0 * C2];
      for (int z = z0; z < z1; ++z) {
        const size_t p = base + (size_t)z * C2;
        const T zp = z < C - 1 ? Z[p + C2] : T(0);
        T nb = zm + zp;
        if (x > 0) nb += Z[p - 1];
        if (x < C - 1) nb += Z[p + 1];
        if (y > 0) nb += Z[p - C];
        if (y < C - 1) nb += Z[p + C];
        const int np = nxy + (z > 0) + (z < C - 1);
        const T v = g[p] - ((ch2 + (T)np) * zc - nb);
        if (r) r[p] = (TR)v;
        if (partial) sq = fma((double)v, (double)v, sq);
        zm = zc;
        zc = zp;
      }
    } else {
      for (int z = z0; z < z1; ++z) {
        const double v = (double)g[base + (size_t)z * C2];
        sq = fma(v, v, sq);
      }
    }
  }
  if (partial) {
    const double b = block_sum<128>(sq);
    if (threadIdx.x == 0) partial[((size_t)s * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = b;
  }
}

// The FP64 residual of the refinement, by the column z-march of k_cc_residual: r = g - D Z
// + (sum of the neighbours inside the box) with D = c h^2 + n_p from a table (no
// integer-to-FP64 conversion), stored in FP32 as the next correction cycle's right-hand
// side (narrowed on the integer pipe), and per-(column block, slab) partial sums of its
// square accumulated in FP32 per thread (the convergence test needs a few digits of
// ||r||, not sixteen). Seven FP64 operations per cell: one fma and six adds.
__global__ void __launch_bounds__(128) k_cc_residual64(int lc, int zslab, double d3, double d4, double d5, double d6,
                                                       const double* __restrict__ g, const double* __restrict__ Z,
                                                       float* __restrict__ r, double* __restrict__ partial,
                                                       const int* __restrict__ active) {
  const int s = blockIdx.z;
  if (!active[s]) return;
  const int C = 1 << lc;
  const size_t C2 = (size_t)1 << (2 * lc), C3 = C2 << lc;
  const int c = blockIdx.x * 128 + threadIdx.x;
  const int z0 = blockIdx.y * zslab, z1 = min(C, z0 + zslab);
  float sq = 0.0f;
  if (c < C * C) {
    const int x = c & (C - 1), y = c >> lc;
    const size_t base = (size_t)s * C3 + c;
    const int nxy = (x > 0) + (x < C - 1) + (y > 0) + (y < C - 1);
    double zm = z0 > 0 ? Z[base + (size_t)(z0 - 1) * C2] : 0.0;
    double zc = Z[base + (size_t)z0 * C2];
    for (int z = z0; z < z1; ++z) {
      const size_t p = base + (size_t)z * C2;
      const double zp = z < C - 1 ? Z[p + C2] : 0.0;
      const int np = nxy + (z > 0) + (z < C - 1);
      const double D = np == 6 ? d6 : (np == 5 ? d5 : (np == 4 ? d4 : d3));
      double v = fma(-D, zc, g[p]);
      v += zm;
      v += zp;
      if (x > 0) v += Z[p - 1];
      if (x < C - 1) v += Z[p + 1];
      if (y > 0) v += Z[p - C];
      if (y < C - 1) v += Z[p + C];
      const float vf = narrow(v);
      r[p] = vf;
      sq = fmaf(vf, vf, sq);
      zm = zc;
      zc = zp;
    }
  }
  const double b = block_sum<128>(widen(sq));
  if (threadIdx.x == 0) partial[((size_t)s * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = b;
}

// Coarse right-hand side: the mean of the 8 children's unscaled residuals, rescaled to
// the coarse h: g_c = (2h)^2 (1/8) sum r / h^2 = (1/2) sum of the children's r.
// Grid (coarse cells / blockDim, samples), Cc = 2^lcc.
template <typename T>
__global__ void k_cc_restrict(int lcc, int B, const T* __restrict__ r, T* __restrict__ gc,
                              const int* __restrict__ active) {
  const int Cc = 1 << lcc, Cf = 2 * Cc;
  const size_t Cc3 = (size_t)1 << (3 * lcc), Cf3 = Cc3 << 3;
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Cc3) return;
  const int X = (int)(q & (Cc - 1)), Y = (int)((q >> lcc) & (Cc - 1)), Zc = (int)(q >> (2 * lcc));
  for (int s = blockIdx.y; s < B; s += gridDim.y) {
    if (!active[s]) continue;
    const size_t t = (size_t)s * Cc3 + q;
    const T* rb = r + (size_t)s * Cf3;
    T sum = 0;
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) sum += rb[((size_t)(2 * Zc + c) * Cf + (2 * Y + b)) * Cf + (2 * X + a)];
    gc[t] = T(0.5) * sum;
  }
}

// Z += trilinear cell-centred interpolation of the coarse correction: a fine cell sits a
// quarter coarse cell from its parent's centre, towards one neighbour; weights 3/4 (parent)
// and 1/4 (that neighbour, or the parent again at a box face: zero flux).
// Grid (fine cells / blockDim, samples), Cf = 2^lcf.
template <typename T>
__global__ void k_cc_prolong(int lcf, int B, const T* __restrict__ ec, T* __restrict__ Z,
                             const int* __restrict__ active) {
  const int Cf = 1 << lcf, Cc = Cf / 2;
  const size_t Cf3 = (size_t)1 << (3 * lcf), Cc3 = Cf3 >> 3;
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Cf3) return;
  const int x = (int)(q & (Cf - 1)), y = (int)((q >> lcf) & (Cf - 1)), z = (int)(q >> (2 * lcf));
  for (int s = blockIdx.y; s < B; s += gridDim.y) {
    if (!active[s]) continue;
    const size_t t = (size_t)s * Cf3 + q;
    int ix[2] = {x >> 1, (x & 1) ? (x >> 1) + 1 : (x >> 1) - 1};
    int iy[2] = {y >> 1, (y & 1) ? (y >> 1) + 1 : (y >> 1) - 1};
    int iz[2] = {z >> 1, (z & 1) ? (z >> 1) + 1 : (z >> 1) - 1};
    if (ix[1] < 0 || ix[1] >= Cc) ix[1] = ix[0];
    if (iy[1] < 0 || iy[1] >= Cc) iy[1] = iy[0];
    if (iz[1] < 0 || iz[1] >= Cc) iz[1] = iz[0];
    // separable: the x lerp of four coarse rows, the y lerp of two, the z lerp of one
    const T* eb = ec + (size_t)s * Cc3;
    T vz[2];
    for (int c = 0; c < 2; ++c) {
      T vy[2];
      for (int b = 0; b < 2; ++b) {
        const size_t row = ((size_t)iz[c] * Cc + iy[b]) * Cc;
        vy[b] = T(0.75) * eb[row + ix[0]] + T(0.25) * eb[row + ix[1]];
      }
      vz[c] = T(0.75) * vy[0] + T(0.25) * vy[1];
    }
    Z[t] += T(0.75) * vz[0] + T(0.25) * vz[1];
  }
}

// Exact solve on the 2^3 grid: the operator is c h^2 I + L with L = L1 x I x I + ... and
// L1 = [[1, -1], [-1, 1]] (eigenvalues 0 and 2 on (1, 1) and (1, -1)); in the sign basis
// v_s(p) = (-1)^{popc(s & p)}, A^-1 g = (1/8) sum_s v_s (v_s . g) / (c h^2 + 2 popc(s)).
template <typename T>
__global__ void k_cc_coarse(int B, T ch2, const T* __restrict__ g, T* __restrict__ Z, const int* __restrict__ active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B || !active[s]) return;
  const T* gb = g + (size_t)s * 8;
  T G[8];
  for (int m = 0; m < 8; ++m) {
    T a = 0;
    for (int p = 0; p < 8; ++p) a += (__popc(m & p) & 1) ? -gb[p] : gb[p];
    G[m] = a / (ch2 + T(2) * (T)__popc(m));
  }
  for (int p = 0; p < 8; ++p) {
    T a = 0;
    for (int m = 0; m < 8; ++m) a += (__popc(m & p) & 1) ? -G[m] : G[m];
    Z[(size_t)s * 8 + p] = T(0.125) * a;
  }
}

// Z += e (FP32 correction widened on the integer pipe), active samples only.
__global__ void k_cc_update(int lc, int B, const float* __restrict__ e, double* __restrict__ Z,
                            const int* __restrict__ active) {
  const size_t C3 = (size_t)1 << (3 * lc);
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= C3) return;
  for (int s = blockIdx.y; s < B; s += gridDim.y) {
    if (!active[s]) continue;
    const size_t t = (size_t)s * C3 + q;
    Z[t] += widen(e[t]);
  }
}

// Sum of a sample's NB partials by one warp in a fixed order: lane l adds l, l + 32, ...,
// then a fixed shuffle tree.
__device__ __forceinline__ double warp_partial_sum(const double* __restrict__ part, int NB) {
  const int lane = threadIdx.x & 31;
  double a = 0.0;
  for (int b = lane; b < NB; b += 32) a += part[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  return a;  // valid in lane 0
}

// Per sample (one warp each): the sum of its partials into out[s].
__global__ void k_cc_sum(int B, int NB, const double* __restrict__ partial, double* __restrict__ out,
                         const int* __restrict__ active) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= B || !active[s]) return;
  const double a = warp_partial_sum(partial + (size_t)s * NB, NB);
  if ((threadIdx.x & 31) == 0) out[s] = a;
}

// After c cycles (one warp per sample): ||r|| / ||g|| <= rtol ends a sample; so does the
// cycle cap (flag bit 2). Bit 1 of the flag: some sample still runs.
__global__ void k_cc_check(int B, int NB, int c, const double* __restrict__ partial, const double* __restrict__ g2,
                           double rtol, int max_cycles, int* __restrict__ active, int* __restrict__ cycles,
                           int* __restrict__ flag) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= B || !active[s]) return;
  const double rr = warp_partial_sum(partial + (size_t)s * NB, NB);
  if ((threadIdx.x & 31) != 0) return;
  cycles[s] = c;
  const bool done = g2[s] > 0.0 ? rr <= rtol * rtol * g2[s] : true;
  if (done) {
    active[s] = 0;
  } else if (c >= max_cycles) {
    active[s] = 0;
    atomicOr(flag, 2);
  } else {
    atomicOr(flag, 1);
  }
}

// k at the n^3 nodes of D: node j is cell j + off.
__global__ void k_spde_extract(int n, int C, int off, int B, double a, const double* __restrict__ Z, int dtype,
                               void* __restrict__ kout) {
  const size_t n3 = (size_t)n * n * n, C3 = (size_t)C * C * C, total = (size_t)B * n3;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(t / n3);
    const size_t q = t - (size_t)s * n3;
    const int x = (int)(q % n), y = (int)((q / n) % n), z = (int)(q / ((size_t)n * n));
    const double v = exp(a * Z[(size_t)s * C3 + ((size_t)(z + off) * C + (y + off)) * C + (x + off)]);
    if (dtype == MLMC_F64)
      ((double*)kout)[t] = v;
    else
      ((float*)kout)[t] = (float)v;
  }
}

__global__ void k_set_int(int B, int v, int* __restrict__ a) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < B) a[s] = v;
}

struct SpdeLevels {
  int nl = 0;
  int C[16];
  double *Z64, *g64;                // the FP64 iterate and right-hand side (finest grid)
  float *e[16], *g[16], *r[16];     // the FP32 correction cycle's grids
  double* partial;
  double* g2;
  int *active, *cycles, *flag;
};

size_t carve_levels(int B, int n, char* base, SpdeLevels* L) {
  char* p = base;
  auto take = [&](size_t bytes) {
    char* q = p;
    p += a256(bytes);
    return q;
  };
  const int C = 2 * (n - 1);
  const size_t cells0 = (size_t)B * C * C * C;
  double* Z64 = (double*)take(cells0 * 8);
  double* g64 = (double*)take(cells0 * 8);
  int nl = 0;
  for (int c = C; c >= 2; c /= 2) {
    const size_t cells = (size_t)B * c * c * c;
    float* e = (float*)take(cells * 4);
    float* g = (float*)take(cells * 4);
    float* r = (float*)take(cells * 4);
    if (L) {
      L->C[nl] = c;
      L->e[nl] = e;
      L->g[nl] = g;
      L->r[nl] = r;
    }
    ++nl;
  }
  int zs = 0;
  const int NB = col_blocks(C) * zslabs(C, &zs);
  double* partial = (double*)take((size_t)B * NB * 8);
  double* g2 = (double*)take((size_t)B * 8);
  int* active = (int*)take((size_t)B * 4);
  int* cycles = (int*)take((size_t)B * 4);
  int* flag = (int*)take(4);
  if (L) {
    L->nl = nl;
    L->Z64 = Z64;
    L->g64 = g64;
    L->partial = partial;
    L->g2 = g2;
    L->active = active;
    L->cycles = cycles;
    L->flag = flag;
  }
  return (size_t)(p - base);
}

int log2i(int c) {
  int l = 0;
  while ((1 << l) < c) ++l;
  return l;
}

// Grid of a per-sample cell kernel: enough blocks for `per` items, samples on y.
dim3 cell_grid(size_t per, int B) { return dim3((unsigned)((per + kT - 1) / kT), (unsigned)(B < 65535 ? B : 65535)); }

// FP32 V(2,2) cycle on grid l: e_l ~ A_l^-1 g_l (e_l zero on entry).
int vcycle32(const SpdeLevels& L, int l, int B, double kappa, double h0, cudaStream_t st) {
  const int C = L.C[l], lc = log2i(C);
  const double hl = h0 * (double)(1 << l), ch2d = kappa * kappa * hl * hl;
  const float ch2 = (float)ch2d;
  const size_t cells = (size_t)B * C * C * C;
  if (C == 2) {
    MLMC_LAUNCH("spde_coarse", cells * 8.0, cells * 64.0, st,
                (k_cc_coarse<float><<<(B + 127) / 128, 128, 0, st>>>(B, ch2, L.g[l], L.e[l], L.active)));
    return MLMC_OK;
  }
  const float i3 = (float)(1.0 / (ch2d + 3.0)), i4 = (float)(1.0 / (ch2d + 4.0)), i5 = (float)(1.0 / (ch2d + 5.0)),
              i6 = (float)(1.0 / (ch2d + 6.0));
  auto sweep = [&]() {
    for (int colour = 0; colour < 2; ++colour)
      MLMC_LAUNCH("spde_rbgs", cells * 6.0, cells * 4.0, st,
                  (k_cc_rbgs<float><<<cell_grid(((size_t)C * C * C) / 2, B), kT, 0, st>>>(
                      colour, lc, B, i3, i4, i5, i6, L.g[l], L.e[l], L.active)));
  };
  sweep();
  sweep();
  int zs = 0;
  const int slabs = zslabs(C, &zs);
  MLMC_LAUNCH("spde_residual", cells * 12.0, cells * 9.0, st,
              (k_cc_residual<float, float><<<dim3(col_blocks(C), slabs, B), 128, 0, st>>>(
                  lc, zs, ch2, L.g[l], L.e[l], L.r[l], nullptr, L.active)));
  const int Cc = L.C[l + 1];
  const size_t ccells = (size_t)B * Cc * Cc * Cc;
  MLMC_LAUNCH("spde_restrict", cells * 4.0 + ccells * 4.0, cells * 1.0, st,
              (k_cc_restrict<float><<<cell_grid((size_t)Cc * Cc * Cc, B), kT, 0, st>>>(lc - 1, B, L.r[l], L.g[l + 1],
                                                                                        L.active)));
  MLMC_CUDA_TRY(cudaMemsetAsync(L.e[l + 1], 0, ccells * sizeof(float), st));
  MLMC_TRY(vcycle32(L, l + 1, B, kappa, h0, st));
  MLMC_LAUNCH("spde_prolong", cells * 8.0 + ccells * 4.0, cells * 10.0, st,
              (k_cc_prolong<float><<<cell_grid((size_t)C * C * C, B), kT, 0, st>>>(lc, B, L.e[l + 1], L.e[l],
                                                                                    L.active)));
  sweep();
  sweep();
  return MLMC_OK;
}

}  // namespace

size_t spde_scratch_bytes(int B, int n) { return carve_levels(B, n, nullptr, nullptr); }

int spde_field_dev(const mlmc_field_cfg& cfg, const uint64_t* ids_dev, int B, int n, int n_noise, int dtype,
                   void* k_out, void* scratch, cudaStream_t st) {
  if (!valid_grid(n) || n > 1025 || (n_noise != n && n_noise != 2 * n - 1) || n_noise > 1025 || B < 1) {
    set_error("spde field: n=%d n_noise=%d batch=%d (n_noise = n or 2n - 1, both <= 1025)", n, n_noise, B);
    return MLMC_ERR_INVALID;
  }
  SpdeLevels L;
  carve_levels(B, n, (char*)scratch, &L);
  const int C = 2 * (n - 1), lc = log2i(C), r = (n_noise - 1) / (n - 1);
  const size_t C3 = (size_t)C * C * C, cells = (size_t)B * C3;
  const double h = 1.0 / (double)(n - 1), hf = 1.0 / (double)(n_noise - 1), v = 0.5 * hf;
  const double scale = sqrt(v * v * v) / h;
  const uint64_t Mo = 4 * (uint64_t)(n_noise - 1) + 1;
  const double octants = (double)cells * 8.0 * r * r * r;
  MLMC_LAUNCH("spde_noise", cells * 8.0, octants * 120.0, st,
              (k_spde_noise<<<cell_grid(C3, B), kT, 0, st>>>(ids_dev, B, lc, r, Mo, (uint32_t)cfg.run_seed,
                                                             (uint32_t)(cfg.run_seed >> 32), scale, L.g64)));
  MLMC_LAUNCH("spde_check", B * 8.0, B * 1.0, st, (k_set_int<<<(B + 127) / 128, 128, 0, st>>>(B, 1, L.active)));
  int zs = 0;
  const int slabs = zslabs(C, &zs), NB = col_blocks(C) * slabs;
  const dim3 rgrid(col_blocks(C), slabs, B);
  MLMC_LAUNCH("spde_residual", cells * 8.0, cells * 2.0, st,
              (k_cc_residual<double, float><<<rgrid, 128, 0, st>>>(lc, zs, 0.0, L.g64, nullptr, nullptr, L.partial,
                                                                  L.active)));
  MLMC_LAUNCH("spde_check", B * NB * 8.0, B * NB * 1.0, st,
              (k_cc_sum<<<(B + 3) / 4, 128, 0, st>>>(B, NB, L.partial, L.g2, L.active)));
  MLMC_CUDA_TRY(cudaMemsetAsync(L.Z64, 0, cells * sizeof(double), st));
  const double kappa = 1.0 / cfg.ell;
  const double ch2 = kappa * kappa * h * h;
  int flag = 0;
  for (int c = 0; c <= kSpdeMaxCycles; ++c) {
    // FP64 residual of the iterate after c corrections: the convergence test and, in
    // FP32, the right-hand side of the next correction cycle
    MLMC_LAUNCH("spde_residual64", cells * 20.0, cells * 14.0, st,
                (k_cc_residual64<<<rgrid, 128, 0, st>>>(lc, zs, ch2 + 3.0, ch2 + 4.0, ch2 + 5.0, ch2 + 6.0, L.g64,
                                                        L.Z64, L.g[0], L.partial, L.active)));
    MLMC_CUDA_TRY(cudaMemsetAsync(L.flag, 0, sizeof(int), st));
    MLMC_LAUNCH("spde_check", B * NB * 8.0, B * NB * 1.0, st,
                (k_cc_check<<<(B + 3) / 4, 128, 0, st>>>(B, NB, c, L.partial, L.g2, kSpdeRtol, kSpdeMaxCycles,
                                                        L.active, L.cycles, L.flag)));
    MLMC_CUDA_TRY(cudaMemcpyAsync(&flag, L.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    MLMC_CUDA_TRY(cudaStreamSynchronize(st));
    if (!(flag & 1)) break;
    MLMC_CUDA_TRY(cudaMemsetAsync(L.e[0], 0, cells * sizeof(float), st));
    MLMC_TRY(vcycle32(L, 0, B, kappa, h, st));
    MLMC_LAUNCH("spde_update", cells * 20.0, cells * 1.0, st,
                (k_cc_update<<<cell_grid(C3, B), kT, 0, st>>>(lc, B, L.e[0], L.Z64, L.active)));
  }
  const int off = (n - 1) / 2;
  const double a = sqrt(8.0 * 3.14159265358979323846 * kappa * cfg.sigma2);
  const size_t nodes = (size_t)B * cube(n);
  MLMC_LAUNCH("spde_extract", nodes * 16.0, nodes * 20.0, st,
              (k_spde_extract<<<blocks_for(nodes, kT), kT, 0, st>>>(n, C, off, B, a, L.Z64, dtype, k_out)));
  MLMC_CUDA_TRY(cudaGetLastError());
  if (flag & 2) {
    set_error("spde field: a sample missed the relative residual %g in %d cycles", kSpdeRtol, kSpdeMaxCycles);
    return MLMC_ERR_NOT_CONVERGED;
  }
  return MLMC_OK;
}

}  // namespace mlmc
