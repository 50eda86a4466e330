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
// Solver: V(2,2) cycles of cell-centred multigrid with constant coefficients (the box is
// the same on every grid: C, C/2, ..., 2 cells): red-black Gauss-Seidel, residual,
// restriction by the mean of the 8 child cells, trilinear cell-centred prolongation
// (weights 3/4, 1/4 per axis, the outside neighbour replaced by the cell itself at the box
// faces), and the exact solve of the 2^3 grid in the eigenbasis of its operator. No
// coefficient arrays: every kernel streams Z and the right-hand side only.
#include <math.h>

#include "common.cuh"
#include "philox.cuh"
#include "prof.cuh"
#include "spde.cuh"

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
__global__ void k_spde_noise(const uint64_t* __restrict__ ids, int B, int C, int r, uint64_t Mo, uint32_t k0,
                             uint32_t k1, double scale, double* __restrict__ g) {
  const size_t C3 = (size_t)C * C * C, total = (size_t)B * C3;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(t / C3);
    const size_t p = t - (size_t)s * C3;
    const int x = (int)(p % C), y = (int)((p / C) % C), z = (int)(p / ((size_t)C * C));
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
__global__ void k_cc_rbgs(int colour, int C, int B, double i3, double i4, double i5, double i6,
                          const double* __restrict__ g, double* __restrict__ Z, const int* __restrict__ active) {
  const int half = C >> 1;
  const size_t C3 = (size_t)C * C * C, per = C3 >> 1, total = per * B;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(t / per);
    if (!active[s]) continue;
    const size_t q = t - (size_t)s * per;
    const int xi = (int)(q % half);
    const size_t row = q / half;
    const int y = (int)(row % C), z = (int)(row / C);
    const int x = 2 * xi + ((y + z + colour) & 1);
    const size_t p = (size_t)s * C3 + ((size_t)z * C + y) * C + x;
    const size_t C2 = (size_t)C * C;
    double acc = g[p];
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

// r = g - A Z (stored if r != NULL) and, if partial != NULL, per-block sums of r^2 (or of
// g^2 when Z == NULL). Grid (NB, B): block b of sample s strides over its cells.
__global__ void __launch_bounds__(kT) k_cc_residual(int C, double ch2, const double* __restrict__ g,
                                                    const double* __restrict__ Z, double* __restrict__ r,
                                                    double* __restrict__ partial, const int* __restrict__ active) {
  const int s = blockIdx.y, NB = gridDim.x;
  if (!active[s]) return;
  const size_t C3 = (size_t)C * C * C, C2 = (size_t)C * C, base = (size_t)s * C3;
  double sq = 0.0;
  for (size_t i = (size_t)blockIdx.x * kT + threadIdx.x; i < C3; i += (size_t)NB * kT) {
    const size_t p = base + i;
    double v = g[p];
    if (Z) {
      const int x = (int)(i % C), y = (int)((i / C) % C), z = (int)(i / C2);
      double nb = 0.0;
      int np = 0;
      if (x > 0) { nb += Z[p - 1]; ++np; }
      if (x < C - 1) { nb += Z[p + 1]; ++np; }
      if (y > 0) { nb += Z[p - C]; ++np; }
      if (y < C - 1) { nb += Z[p + C]; ++np; }
      if (z > 0) { nb += Z[p - C2]; ++np; }
      if (z < C - 1) { nb += Z[p + C2]; ++np; }
      v = v - ((ch2 + (double)np) * Z[p] - nb);
      if (r) r[p] = v;
    }
    sq = fma(v, v, sq);
  }
  if (partial) {
    const double b = block_sum<kT>(sq);
    if (threadIdx.x == 0) partial[(size_t)s * NB + blockIdx.x] = b;
  }
}

// Coarse right-hand side: the mean of the 8 children's unscaled residuals, rescaled to
// the coarse h: g_c = (2h)^2 (1/8) sum r / h^2 = (1/2) sum of the children's r.
__global__ void k_cc_restrict(int Cc, int B, const double* __restrict__ r, double* __restrict__ gc,
                              const int* __restrict__ active) {
  const int Cf = 2 * Cc;
  const size_t Cc3 = (size_t)Cc * Cc * Cc, Cf3 = (size_t)Cf * Cf * Cf, total = (size_t)B * Cc3;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(t / Cc3);
    if (!active[s]) continue;
    const size_t q = t - (size_t)s * Cc3;
    const int X = (int)(q % Cc), Y = (int)((q / Cc) % Cc), Zc = (int)(q / ((size_t)Cc * Cc));
    const double* rb = r + (size_t)s * Cf3;
    double sum = 0.0;
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) sum += rb[((size_t)(2 * Zc + c) * Cf + (2 * Y + b)) * Cf + (2 * X + a)];
    gc[t] = 0.5 * sum;
  }
}

// Z += trilinear cell-centred interpolation of the coarse correction: a fine cell sits a
// quarter coarse cell from its parent's centre, towards one neighbour; weights 3/4 (parent)
// and 1/4 (that neighbour, or the parent again at a box face: zero flux).
__global__ void k_cc_prolong(int Cf, int B, const double* __restrict__ ec, double* __restrict__ Z,
                             const int* __restrict__ active) {
  const int Cc = Cf / 2;
  const size_t Cf3 = (size_t)Cf * Cf * Cf, Cc3 = (size_t)Cc * Cc * Cc, total = (size_t)B * Cf3;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int s = (int)(t / Cf3);
    if (!active[s]) continue;
    const size_t q = t - (size_t)s * Cf3;
    const int x = (int)(q % Cf), y = (int)((q / Cf) % Cf), z = (int)(q / ((size_t)Cf * Cf));
    int ix[2] = {x >> 1, (x & 1) ? (x >> 1) + 1 : (x >> 1) - 1};
    int iy[2] = {y >> 1, (y & 1) ? (y >> 1) + 1 : (y >> 1) - 1};
    int iz[2] = {z >> 1, (z & 1) ? (z >> 1) + 1 : (z >> 1) - 1};
    if (ix[1] < 0 || ix[1] >= Cc) ix[1] = ix[0];
    if (iy[1] < 0 || iy[1] >= Cc) iy[1] = iy[0];
    if (iz[1] < 0 || iz[1] >= Cc) iz[1] = iz[0];
    const double w[2] = {0.75, 0.25};
    const double* eb = ec + (size_t)s * Cc3;
    double v = 0.0;
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a)
          v += w[c] * w[b] * w[a] * eb[((size_t)iz[c] * Cc + iy[b]) * Cc + ix[a]];
    Z[t] += v;
  }
}

// Exact solve on the 2^3 grid: the operator is c h^2 I + L with L = L1 x I x I + ... and
// L1 = [[1, -1], [-1, 1]] (eigenvalues 0 and 2 on (1, 1) and (1, -1)); in the sign basis
// v_s(p) = (-1)^{popc(s & p)}, A^-1 g = (1/8) sum_s v_s (v_s . g) / (c h^2 + 2 popc(s)).
__global__ void k_cc_coarse(int B, double ch2, const double* __restrict__ g, double* __restrict__ Z,
                            const int* __restrict__ active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B || !active[s]) return;
  const double* gb = g + (size_t)s * 8;
  double G[8];
  for (int m = 0; m < 8; ++m) {
    double a = 0.0;
    for (int p = 0; p < 8; ++p) a += (__popc(m & p) & 1) ? -gb[p] : gb[p];
    G[m] = a / (ch2 + 2.0 * __popc(m));
  }
  for (int p = 0; p < 8; ++p) {
    double a = 0.0;
    for (int m = 0; m < 8; ++m) a += (__popc(m & p) & 1) ? -G[m] : G[m];
    Z[(size_t)s * 8 + p] = 0.125 * a;
  }
}

// Per sample: the sum of the partials (in block order) into out[s].
__global__ void k_cc_sum(int B, int NB, const double* __restrict__ partial, double* __restrict__ out,
                         const int* __restrict__ active) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B || !active[s]) return;
  double a = 0.0;
  for (int b = 0; b < NB; ++b) a += partial[(size_t)s * NB + b];
  out[s] = a;
}

// After a cycle: ||r|| / ||g|| <= rtol ends a sample; so does the cycle cap (flag bit 2).
// Bit 1 of the flag: some sample still runs.
__global__ void k_cc_check(int B, int NB, const double* __restrict__ partial, const double* __restrict__ g2,
                           double rtol, int max_cycles, int* __restrict__ active, int* __restrict__ cycles,
                           int* __restrict__ flag) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B || !active[s]) return;
  double rr = 0.0;
  for (int b = 0; b < NB; ++b) rr += partial[(size_t)s * NB + b];
  const int c = ++cycles[s];
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

int reduce_blocks_cc(size_t cells) {
  size_t nb = (cells + 4095) / 4096;
  if (nb < 1) nb = 1;
  if (nb > 1024) nb = 1024;
  return (int)nb;
}

struct SpdeLevels {
  int nl = 0;
  int C[16];
  double *Z[16], *g[16], *r[16];
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
  int C = 2 * (n - 1), nl = 0;
  for (int c = C; c >= 2; c /= 2) {
    const size_t cells = (size_t)B * c * c * c;
    if (L) {
      L->C[nl] = c;
      L->Z[nl] = (double*)take(cells * 8);
      L->g[nl] = (double*)take(cells * 8);
      L->r[nl] = (double*)take(cells * 8);
    } else {
      take(cells * 8);
      take(cells * 8);
      take(cells * 8);
    }
    ++nl;
  }
  const int NB = reduce_blocks_cc((size_t)C * C * C);
  double* partial = (double*)take((size_t)B * NB * 8);
  double* g2 = (double*)take((size_t)B * 8);
  int* active = (int*)take((size_t)B * 4);
  int* cycles = (int*)take((size_t)B * 4);
  int* flag = (int*)take(4);
  if (L) {
    L->nl = nl;
    L->partial = partial;
    L->g2 = g2;
    L->active = active;
    L->cycles = cycles;
    L->flag = flag;
  }
  return (size_t)(p - base);
}

int vcycle(const SpdeLevels& L, int l, int B, double kappa, double h0, cudaStream_t st) {
  const int C = L.C[l];
  const double hl = h0 * (double)(1 << l), ch2 = kappa * kappa * hl * hl;
  const size_t cells = (size_t)B * C * C * C;
  if (C == 2) {
    MLMC_LAUNCH("spde_coarse", cells * 16.0, cells * 64.0, st,
                (k_cc_coarse<<<(B + 127) / 128, 128, 0, st>>>(B, ch2, L.g[l], L.Z[l], L.active)));
    return MLMC_OK;
  }
  const double i3 = 1.0 / (ch2 + 3.0), i4 = 1.0 / (ch2 + 4.0), i5 = 1.0 / (ch2 + 5.0), i6 = 1.0 / (ch2 + 6.0);
  auto sweep = [&]() {
    for (int colour = 0; colour < 2; ++colour)
      MLMC_LAUNCH("spde_rbgs", cells * 12.0, cells * 4.0, st,
                  (k_cc_rbgs<<<blocks_for(cells / 2, kT, 152u * 32u), kT, 0, st>>>(colour, C, B, i3, i4, i5, i6,
                                                                                    L.g[l], L.Z[l], L.active)));
  };
  sweep();
  sweep();
  const int NB = reduce_blocks_cc((size_t)C * C * C);
  MLMC_LAUNCH("spde_residual", cells * 24.0, cells * 9.0, st,
              (k_cc_residual<<<dim3(NB, B), kT, 0, st>>>(C, ch2, L.g[l], L.Z[l], L.r[l], nullptr, L.active)));
  const int Cc = L.C[l + 1];
  const size_t ccells = (size_t)B * Cc * Cc * Cc;
  MLMC_LAUNCH("spde_restrict", cells * 8.0 + ccells * 8.0, cells * 1.0, st,
              (k_cc_restrict<<<blocks_for(ccells, kT, 152u * 32u), kT, 0, st>>>(Cc, B, L.r[l], L.g[l + 1],
                                                                                L.active)));
  MLMC_CUDA_TRY(cudaMemsetAsync(L.Z[l + 1], 0, ccells * sizeof(double), st));
  MLMC_TRY(vcycle(L, l + 1, B, kappa, h0, st));
  MLMC_LAUNCH("spde_prolong", cells * 16.0 + ccells * 8.0, cells * 24.0, st,
              (k_cc_prolong<<<blocks_for(cells, kT, 152u * 32u), kT, 0, st>>>(C, B, L.Z[l + 1], L.Z[l],
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
  const int C = 2 * (n - 1), r = (n_noise - 1) / (n - 1);
  const size_t C3 = (size_t)C * C * C, cells = (size_t)B * C3;
  const double h = 1.0 / (double)(n - 1), hf = 1.0 / (double)(n_noise - 1), v = 0.5 * hf;
  const double scale = sqrt(v * v * v) / h;
  const uint64_t Mo = 4 * (uint64_t)(n_noise - 1) + 1;
  const double octants = (double)cells * 8.0 * r * r * r;
  MLMC_LAUNCH("spde_noise", cells * 8.0, octants * 120.0, st,
              (k_spde_noise<<<blocks_for(cells, kT, 152u * 64u), kT, 0, st>>>(
                  ids_dev, B, C, r, Mo, (uint32_t)cfg.run_seed, (uint32_t)(cfg.run_seed >> 32), scale, L.g[0])));
  MLMC_LAUNCH("spde_check", B * 8.0, B * 1.0, st,
              (k_set_int<<<(B + 127) / 128, 128, 0, st>>>(B, 1, L.active)));
  MLMC_LAUNCH("spde_check", B * 8.0, B * 1.0, st,
              (k_set_int<<<(B + 127) / 128, 128, 0, st>>>(B, 0, L.cycles)));
  const int NB = reduce_blocks_cc(C3);
  MLMC_LAUNCH("spde_residual", cells * 8.0, cells * 2.0, st,
              (k_cc_residual<<<dim3(NB, B), kT, 0, st>>>(C, 0.0, L.g[0], nullptr, nullptr, L.partial, L.active)));
  MLMC_LAUNCH("spde_check", B * NB * 8.0, B * NB * 1.0, st,
              (k_cc_sum<<<(B + 127) / 128, 128, 0, st>>>(B, NB, L.partial, L.g2, L.active)));
  MLMC_CUDA_TRY(cudaMemsetAsync(L.Z[0], 0, cells * sizeof(double), st));
  const double kappa = 1.0 / cfg.ell;
  const double ch2 = kappa * kappa * h * h;
  int flag = 0;
  for (int c = 0; c < kSpdeMaxCycles; ++c) {
    MLMC_TRY(vcycle(L, 0, B, kappa, h, st));
    MLMC_LAUNCH("spde_residual", cells * 16.0, cells * 9.0, st,
                (k_cc_residual<<<dim3(NB, B), kT, 0, st>>>(C, ch2, L.g[0], L.Z[0], nullptr, L.partial, L.active)));
    MLMC_CUDA_TRY(cudaMemsetAsync(L.flag, 0, sizeof(int), st));
    MLMC_LAUNCH("spde_check", B * NB * 8.0, B * NB * 1.0, st,
                (k_cc_check<<<(B + 127) / 128, 128, 0, st>>>(B, NB, L.partial, L.g2, kSpdeRtol, kSpdeMaxCycles,
                                                            L.active, L.cycles, L.flag)));
    MLMC_CUDA_TRY(cudaMemcpyAsync(&flag, L.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    MLMC_CUDA_TRY(cudaStreamSynchronize(st));
    if (!(flag & 1)) break;
  }
  const int off = (n - 1) / 2;
  const double a = sqrt(8.0 * 3.14159265358979323846 * kappa * cfg.sigma2);
  const size_t nodes = (size_t)B * cube(n);
  MLMC_LAUNCH("spde_extract", nodes * 16.0, nodes * 20.0, st,
              (k_spde_extract<<<blocks_for(nodes, kT), kT, 0, st>>>(n, C, off, B, a, L.Z[0], dtype, k_out)));
  MLMC_CUDA_TRY(cudaGetLastError());
  if (flag & 2) {
    set_error("spde field: a sample missed the relative residual %g in %d cycles", kSpdeRtol, kSpdeMaxCycles);
    return MLMC_ERR_NOT_CONVERGED;
  }
  return MLMC_OK;
}

}  // namespace mlmc
