// Batched geometric multigrid: V(nu1, nu2) cycles with red-black Gauss-Seidel, full
// weighting, trilinear prolongation, rediscretised coarse operators and an exact 5^3
// solve (the deterministic solver inside every sample of Algorithm 1, for the model problem
// of Sec. 3, Eq. 16; the cycle family of Sec. 7.1).
//
// Scaled form. With faces K_pq = 2 k_p k_q / (k_p + k_q) and D_p = sum_q K_pq, every
// grid stores the h^2-scaled operator (A~ u)_p = D_p u_p - sum_q K_pq u_q and the
// scaled right-hand side g = h^2 f, so
//   smoothing     u_p <- (g_p + sum_q K_pq u_q) * (1 / D_p)      (6 FMA + 1 MUL)
//   residual      r~_p = g_p - D_p u_p + sum_q K_pq u_q = h^2 r_p  (7 FMA)
//   restriction   g_c = h_c^2 FW(r) = 4 FW(r~)
//   norms         ||r|| / ||f|| = ||r~|| / ||g||.
// No division runs inside a cycle; faces, D and 1/D are computed once per solve.
//
// Precision MLMC_PREC_MIXED: the V-cycle's faces are the FP32 harmonic means of the
// FP32-rounded nodal k and the V-cycle runs entirely in FP32 as a correction solve; the
// outer residual g - A~ u, on FP64 faces of the FP64 nodal k of the finest grid, and the
// update u += e run in FP64 (iterative refinement, or flexible CG with the FP32 cycle as
// preconditioner): the fixed point is the FP64 solution of the FP64 operator, the one
// an all-FP64 solve reaches.
//
// Every kernel skips samples whose `active` flag is 0, so each sample stops at its own
// cycle count; every per-sample sum is a fixed tree that depends only on n. A sample's
// result therefore does not depend on the batch it is solved in.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <vector>

#include "common.cuh"
#include "mg.cuh"
#include "prof.cuh"
#include "smooth.cuh"
#include "tune.cuh"
#include "widen.cuh"

namespace mlmc {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxLevels = 12;
constexpr int kPlaneThreads = 128;

// Plane launches: blockIdx.x (with threadIdx.x) enumerates the work items of one z-plane,
// blockIdx.y strides over the (sample, z) planes, so every in-sample index is 32-bit
// (n^3 < 2^31 for every valid n) and no thread divides a 64-bit index.
inline dim3 plane_grid(int per_plane, long long planes) {
  return dim3((unsigned)((per_plane + kPlaneThreads - 1) / kPlaneThreads),
              (unsigned)(planes < 65535 ? (planes > 0 ? planes : 1) : 65535));
}

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

// Colour-split storage (see the colour-split kernels below).
__host__ __device__ __forceinline__ int split_pitch(int n) { return (((n + 1) >> 1) + 3) & ~3; }
// elements of one sample in colour-split storage
__host__ __device__ __forceinline__ size_t split_elems(int n) { return (size_t)2 * n * n * (size_t)split_pitch(n); }
__device__ __forceinline__ unsigned split_index(int n, int x, int y, int z) {
  const int P = split_pitch(n);
  return (unsigned)((x + y + z) & 1) * (unsigned)(n * n * P) + (unsigned)((z * n + y) * P + (x >> 1));
}

// Index of node (x, y, z) of sample s of an n^3 grid in the plain or (SPLIT) the
// colour-split storage.
template <bool SPLIT>
__device__ __forceinline__ size_t node_at(int n, int s, int x, int y, int z) {
  return SPLIT ? (size_t)s * split_elems(n) + split_index(n, x, y, z)
               : (((size_t)s * n + z) * n + y) * n + x;
}

// Carves 256-byte aligned pieces; with base == nullptr it only measures.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base((char*)b) {}
  template <typename T>
  T* take(size_t count) {
    T* p = base ? (T*)(base + off) : nullptr;
    off += a256(count * sizeof(T)) + 256;  // slack: 16-byte-rounded bulk copies may read past the end
    return p;
  }
};

// x in the arithmetic type TD (FP32 to FP64 through widen)
template <typename TD, typename T>
__device__ __forceinline__ TD to_t(T x) {
  return (TD)x;
}
template <>
__device__ __forceinline__ double to_t<double, float>(float x) {
  return widen(x);
}

__device__ __forceinline__ double harm(double a, double b, double) {
  return __ddiv_rn(__dmul_rn(2.0 * a, b), __dadd_rn(a, b));
}
__device__ __forceinline__ float harm(double a, double b, float) {
  const float a32 = __double2float_rn(a), b32 = __double2float_rn(b);
  return __fdiv_rn(__fmul_rn(2.0f * a32, b32), __fadd_rn(a32, b32));
}

// ---------------------------------------------------------------------------------
// Operator set-up
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void k_faces(const double* __restrict__ k0, int n0, int st0, int n, int B, T* __restrict__ Kx,
                        T* __restrict__ Ky, T* __restrict__ Kz) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // node of the plane
  if (q >= n * n) return;
  const int y = q / n, x = q - y * n;
  const size_t n3 = (size_t)n * n * n, n03 = (size_t)n0 * n0 * n0;
  for (int zz = blockIdx.y; zz < B * n; zz += gridDim.y) {
    const int s = zz / n, z = zz - s * n;
    const double* kb = k0 + (size_t)s * n03;
    const size_t p0 = ((size_t)(st0 * z) * n0 + (size_t)(st0 * y)) * n0 + (size_t)(st0 * x);
    const size_t t = (size_t)s * n3 + (size_t)(z * n * n + q);
    const double a = kb[p0];
    Kx[t] = x < n - 1 ? harm(a, kb[p0 + st0], T()) : T(0);
    Ky[t] = y < n - 1 ? harm(a, kb[p0 + (size_t)st0 * n0], T()) : T(0);
    Kz[t] = z < n - 1 ? harm(a, kb[p0 + (size_t)st0 * n0 * n0], T()) : T(0);
  }
}

// D = sum of the six faces at interior nodes (fixed order), Dinv = 1 / D; 0 on the boundary.
template <typename T, typename TD>
__global__ void k_diag(int n, int B, const T* __restrict__ Kx, const T* __restrict__ Ky, const T* __restrict__ Kz,
                       TD* __restrict__ D, TD* __restrict__ Dinv) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // node of the plane
  if (q >= n * n) return;
  const int y = q / n, x = q - y * n;
  const size_t n3 = (size_t)n * n * n, n2 = (size_t)n * n;
  for (int zz = blockIdx.y; zz < B * n; zz += gridDim.y) {
    const int s = zz / n, z = zz - s * n;
    const size_t t = (size_t)s * n3 + (size_t)(z * n * n + q);
    const bool in = x > 0 && y > 0 && z > 0 && x < n - 1 && y < n - 1 && z < n - 1;
    TD d = 0;
    if (in) {
      d = to_t<TD>(Kx[t - 1]);
      d += to_t<TD>(Kx[t]);
      d += to_t<TD>(Ky[t - n]);
      d += to_t<TD>(Ky[t]);
      d += to_t<TD>(Kz[t - n2]);
      d += to_t<TD>(Kz[t]);
    }
    if (D) D[t] = d;
    if (Dinv) Dinv[t] = in ? (TD)1 / d : (TD)0;
  }
}

// Dense 27x27 scaled operator of the 5^3 grid, its Cholesky factor, and the inverse,
// one warp per sample (lane i < 27 owns row i of the working matrix in global scratch;
// the factorisation and the 27 triangular solves run column by column across the warp).
template <typename T>
__global__ void k_coarse_setup(int B, const T* __restrict__ Kx, const T* __restrict__ Ky, const T* __restrict__ Kz,
                               double* __restrict__ Lws, double* __restrict__ Ainv) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= B) return;
  const int s = warp, n = 5, N = 27;
  const size_t base = (size_t)s * 125;
  double* A = Lws + (size_t)s * N * N;
  double* X = Ainv + (size_t)s * N * N;
  const int i = lane;
  if (i < N) {
    for (int c = 0; c < N; ++c) A[i * N + c] = 0.0;
    const int x = 1 + i % 3, y = 1 + (i / 3) % 3, z = 1 + i / 9;
    const size_t p = base + (size_t)(z * n + y) * n + x;
    const double f[6] = {(double)Kx[p - 1], (double)Kx[p], (double)Ky[p - n], (double)Ky[p], (double)Kz[p - 25],
                         (double)Kz[p]};
    const int nb[6] = {x > 1 ? i - 1 : -1, x < 3 ? i + 1 : -1, y > 1 ? i - 3 : -1,
                       y < 3 ? i + 3 : -1, z > 1 ? i - 9 : -1, z < 3 ? i + 9 : -1};
    double d = 0.0;
    for (int q = 0; q < 6; ++q) {
      d += f[q];
      if (nb[q] >= 0) A[i * N + nb[q]] = -f[q];
    }
    A[i * N + i] = d;
  }
  __syncwarp();
  // Cholesky A = L L^T (lower triangle in place): column j is finished by the warp
  for (int j = 0; j < N; ++j) {
    double ljj = 0.0;
    if (lane == 0) {
      double d = A[j * N + j];
      for (int q = 0; q < j; ++q) d -= A[j * N + q] * A[j * N + q];
      ljj = sqrt(d);
      A[j * N + j] = ljj;
    }
    ljj = __shfl_sync(0xffffffffu, ljj, 0);
    __syncwarp();
    if (i > j && i < N) {
      double v = A[i * N + j];
      for (int q = 0; q < j; ++q) v -= A[i * N + q] * A[j * N + q];
      A[i * N + j] = v / ljj;
    }
    __syncwarp();
  }
  // column c of the inverse solves L L^T x = e_c; lane c < 27 solves column c
  if (i < N) {
    double y[27];
    for (int r = 0; r < N; ++r) {
      double v = (r == i) ? 1.0 : 0.0;
      for (int q = 0; q < r; ++q) v -= A[r * N + q] * y[q];
      y[r] = v / A[r * N + r];
    }
    for (int r = N - 1; r >= 0; --r) {
      double v = y[r];
      for (int q = r + 1; q < N; ++q) v -= A[q * N + r] * y[q];
      y[r] = v / A[r * N + r];
    }
    for (int r = 0; r < N; ++r) X[r * N + i] = y[r];
  }
}

// u = A~^-1 g on the 5^3 grid (interior nodes; boundary untouched); SPLIT: g and u in
// colour-split storage.
template <typename T, bool SPLIT = false>
__global__ void k_coarse_apply(int B, const double* __restrict__ Ainv, const T* __restrict__ g, T* __restrict__ u,
                               const int* __restrict__ active) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * 27) return;
  const int s = t / 27, i = t - s * 27;
  if (active && !active[s]) return;
  const double* X = Ainv + (size_t)s * 729 + (size_t)i * 27;
  const size_t base = (size_t)s * (SPLIT ? split_elems(5) : (size_t)125);
  auto at = [&](int x, int y, int z) -> size_t {
    return base + (SPLIT ? (size_t)split_index(5, x, y, z) : (size_t)((z * 5 + y) * 5 + x));
  };
  double v = 0.0;
  for (int j = 0; j < 27; ++j) {
    const int x = 1 + j % 3, y = 1 + (j / 3) % 3, z = 1 + j / 9;
    v = fma(X[j], (double)g[at(x, y, z)], v);
  }
  const int x = 1 + i % 3, y = 1 + (i / 3) % 3, z = 1 + i / 9;
  u[at(x, y, z)] = (T)v;
}

// ---------------------------------------------------------------------------------
// Cycle kernels
// ---------------------------------------------------------------------------------

// One colour of a red-black sweep: threads enumerate only the nodes of that colour.
template <typename T>
__global__ void k_rbgs(int colour, int n, int B, const T* __restrict__ Kx, const T* __restrict__ Ky,
                       const T* __restrict__ Kz, const T* __restrict__ Dinv, const T* __restrict__ g, T* __restrict__ u,
                       const int* __restrict__ active) {
  // n = 2^p + 1: a row holds half = 2^(p-1) nodes of each colour
  const int m = n - 2, half = (n - 1) / 2, lh = 31 - __clz(half);
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // colour node of an interior plane
  if (q >= m * half) return;
  const int xi = q & (half - 1), y = 1 + (q >> lh);
  const size_t n3 = (size_t)n * n * n, n2 = (size_t)n * n;
  for (int zz = blockIdx.y; zz < B * m; zz += gridDim.y) {
    const int s = zz / m, z = 1 + (zz - s * m);
    if (active && !active[s]) continue;
    const int x = (((1 + y + z) & 1) == colour ? 1 : 2) + 2 * xi;
    if (x > n - 2) continue;
    const size_t p = (size_t)s * n3 + (size_t)(z * n * n + y * n + x);
    T acc = g[p];
    acc = fma(Kx[p - 1], u[p - 1], acc);
    acc = fma(Kx[p], u[p + 1], acc);
    acc = fma(Ky[p - n], u[p - n], acc);
    acc = fma(Ky[p], u[p + n], acc);
    acc = fma(Kz[p - n2], u[p - n2], acc);
    acc = fma(Kz[p], u[p + n2], acc);
    u[p] = acc * Dinv[p];
  }
}

// Reciprocal nodal coefficient rho = 1/k of an MG grid in the grid's precision (injection
// from the finest k): the input of the nodal-coefficient sweep, whose harmonic faces are
// 2ab/(a+b) = 2/(rho_a + rho_b).
template <typename T>
__global__ void k_nodal_k(const double* __restrict__ k0, int n0, int st0, int n, int B, T* __restrict__ kn) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // node of the plane
  if (q >= n * n) return;
  const int y = q / n, x = q - y * n;
  const size_t n3 = (size_t)n * n * n, n03 = (size_t)n0 * n0 * n0;
  for (int zz = blockIdx.y; zz < B * n; zz += gridDim.y) {
    const int s = zz / n, z = zz - s * n;
    const size_t p0 = ((size_t)(st0 * z) * n0 + (size_t)(st0 * y)) * n0 + (size_t)(st0 * x);
    kn[(size_t)s * n3 + (size_t)(z * n * n + q)] = (T)(1.0 / k0[(size_t)s * n03 + p0]);
  }
}

// Harmonic face of the nodal-coefficient kernels from the reciprocal coefficients:
// 2ab / (a + b) = 2 / (rho_a + rho_b), with the fast reciprocal (__fdividef, within 2
// ulp). Symmetric in the two nodes, so both see the same value; the faces differ from the
// stored IEEE ones by a few ulps.
__device__ __forceinline__ float nodal_face(float ra, float rb) { return __fdividef(2.0f, __fadd_rn(ra, rb)); }

// One colour of a red-black sweep that reads the (reciprocal) nodal coefficient (FP32) instead of
// stored faces: the six harmonic faces, their sum D and 1/D of the updated node are
// recomputed per update with fast reciprocals, so a sweep reads 4 words per node (u read
// and written, g, k) instead of 7. It is the Gauss-Seidel sweep of an operator within a
// few ulps of the stored FP32 one: used only inside the FP32 correction cycle, whose
// result the FP64 outer residual (stored faces) corrects, so the converged solution is
// that of the stored operator.
__global__ void k_rbgs_nodal(int colour, int n, int B, const float* __restrict__ kn, const float* __restrict__ g,
                             float* __restrict__ u, const int* __restrict__ active) {
  const int m = n - 2, half = (n - 1) / 2, lh = 31 - __clz(half);
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // colour node of an interior plane
  if (q >= m * half) return;
  const int xi = q & (half - 1), y = 1 + (q >> lh);
  const size_t n3 = (size_t)n * n * n, n2 = (size_t)n * n;
  for (int zz = blockIdx.y; zz < B * m; zz += gridDim.y) {
    const int s = zz / m, z = 1 + (zz - s * m);
    if (active && !active[s]) continue;
    const int x = (((1 + y + z) & 1) == colour ? 1 : 2) + 2 * xi;
    if (x > n - 2) continue;
    const size_t p = (size_t)s * n3 + (size_t)(z * n * n + y * n + x);
    const float kc = kn[p];
    const float kxm = nodal_face(kn[p - 1], kc), kxp = nodal_face(kc, kn[p + 1]);
    const float kym = nodal_face(kn[p - n], kc), kyp = nodal_face(kc, kn[p + n]);
    const float kzm = nodal_face(kn[p - n2], kc), kzp = nodal_face(kc, kn[p + n2]);
    float d = kxm;
    d += kxp;
    d += kym;
    d += kyp;
    d += kzm;
    d += kzp;
    const float dinv = __fdividef(1.0f, d);
    float acc = g[p];
    acc = fmaf(kxm, u[p - 1], acc);
    acc = fmaf(kxp, u[p + 1], acc);
    acc = fmaf(kym, u[p - n], acc);
    acc = fmaf(kyp, u[p + n], acc);
    acc = fmaf(kzm, u[p - n2], acc);
    acc = fmaf(kzp, u[p + n2], acc);
    u[p] = acc * dinv;
  }
}

// r~ = g - D u + sum K u_q of an FP32 grid from the nodal coefficient (faces and D
// recomputed as in k_rbgs_nodal, then k_residual_z's operation order): the residual of the
// operator the nodal sweep smooths; r~ on interior nodes, 0 on the boundary; 4 words per
// node instead of 7.
__global__ void k_residual_nodal(int n, int B, const float* __restrict__ kn, const float* __restrict__ g,
                                 const float* __restrict__ u, float* __restrict__ r, const int* __restrict__ active) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // node of the plane
  if (q >= n * n) return;
  const int y = q / n, x = q - y * n;
  const size_t n3 = (size_t)n * n * n, n2 = (size_t)n * n;
  for (int zz = blockIdx.y; zz < B * n; zz += gridDim.y) {
    const int s = zz / n, z = zz - s * n;
    if (active && !active[s]) continue;
    const size_t p = (size_t)s * n3 + (size_t)(z * n * n + q);
    float rr = 0.0f;
    if (x > 0 && y > 0 && z > 0 && x < n - 1 && y < n - 1 && z < n - 1) {
      const float kc = kn[p];
      const float kxm = nodal_face(kn[p - 1], kc), kxp = nodal_face(kc, kn[p + 1]);
      const float kym = nodal_face(kn[p - n], kc), kyp = nodal_face(kc, kn[p + n]);
      const float kzm = nodal_face(kn[p - n2], kc), kzp = nodal_face(kc, kn[p + n2]);
      float d = kxm;
      d += kxp;
      d += kym;
      d += kyp;
      d += kzm;
      d += kzp;
      rr = fmaf(-d, u[p], g[p]);
      rr = fmaf(kxm, u[p - 1], rr);
      rr = fmaf(kxp, u[p + 1], rr);
      rr = fmaf(kym, u[p - n], rr);
      rr = fmaf(kyp, u[p + n], rr);
      rr = fmaf(kzm, u[p - n2], rr);
      rr = fmaf(kzp, u[p + n2], rr);
    }
    r[p] = rr;
  }
}

// ---------------------------------------------------------------------------------
// Colour-split storage of the FP32 correction hierarchy (MLMC_SMOOTH_SPLIT): per sample
// the nodes of colour c = (x + y + z) & 1 form one block of n x n rows of P slots, node
// (x, y, z) at slot x >> 1 of row (z, y) of its colour's block; P = (n + 1) / 2 rounded up
// to a multiple of 4, so that every row starts on a 16-byte boundary (four slots per
// vector access). A colour pass
// of the red-black sweep then streams the lines of the colour it updates plus those of
// the other colour it reads (2.5 instead of 4 words per node and pass at line
// granularity). Neighbours of node x = 2 xi + q (q = x parity) in the other colour: x - 1
// at slot xi - 1 + q, x + 1 at slot xi + q, y +- 1 and z +- 1 at slot xi. The slot x = n
// of odd-parity rows and the padding slots do not exist in the grid: a kernel may load
// them along with a vector of slots but never uses their values.
// ---------------------------------------------------------------------------------
// Reciprocal nodal coefficient 1/k of an FP32 grid (every node) into colour-split storage.
__global__ void k_nodal_k_split(const double* __restrict__ k0, int n0, int st0, int n, int B, float* __restrict__ kn) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // node of the plane
  if (q >= n * n) return;
  const int y = q / n, x = q - y * n;
  const size_t ns = split_elems(n), n03 = (size_t)n0 * n0 * n0;
  for (int zz = blockIdx.y; zz < B * n; zz += gridDim.y) {
    const int s = zz / n, z = zz - s * n;
    const size_t p0 = ((size_t)(st0 * z) * n0 + (size_t)(st0 * y)) * n0 + (size_t)(st0 * x);
    kn[(size_t)s * ns + split_index(n, x, y, z)] = (float)(1.0 / k0[(size_t)s * n03 + p0]);
  }
}

// Compile-time geometry of a colour-split grid of n = 2^LG + 1 nodes per axis: with n a
// constant, the row / slot split of a thread index and every neighbour offset are
// shifts, multiplications by constants and immediate load offsets (the runtime-n form of
// these kernels spent about 280 instructions per updated node and was issue-bound).
template <int LG>
struct SplitGeo {
  static constexpr int n = (1 << LG) + 1, m = n - 2, P = (((n + 1) / 2) + 3) & ~3, NP = n * P, BLK = n * n * P;
  static constexpr int Q4 = P / 4;               // four-slot groups per row
  static constexpr size_t NS = (size_t)2 * BLK;  // elements per sample
};

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float comp(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

// The nodal-coefficient update of one node from its own k^-1 and right-hand side and the
// six neighbours' k^-1 and iterate, in k_rbgs_nodal's order of operations.
__device__ __forceinline__ float nodal_update(float kc, float gp, float kl, float ul, float kr, float ur, float kym,
                                              float uym, float kyp, float uyp, float kzm, float uzm, float kzp,
                                              float uzp) {
  const float fxm = nodal_face(kl, kc), fxp = nodal_face(kc, kr);
  const float fym = nodal_face(kym, kc), fyp = nodal_face(kc, kyp);
  const float fzm = nodal_face(kzm, kc), fzp = nodal_face(kc, kzp);
  float d = fxm;
  d += fxp;
  d += fym;
  d += fyp;
  d += fzm;
  d += fzp;
  const float dinv = __fdividef(1.0f, d);
  float acc = gp;
  acc = fmaf(fxm, ul, acc);
  acc = fmaf(fxp, ur, acc);
  acc = fmaf(fym, uym, acc);
  acc = fmaf(fyp, uyp, acc);
  acc = fmaf(fzm, uzm, acc);
  acc = fmaf(fzp, uzp, acc);
  return acc * dinv;
}

// The residual of one node in k_residual_nodal's order of operations.
__device__ __forceinline__ float nodal_residual(float kc, float gp, float up, float kl, float ul, float kr, float ur,
                                                float kym, float uym, float kyp, float uyp, float kzm, float uzm,
                                                float kzp, float uzp) {
  const float fxm = nodal_face(kl, kc), fxp = nodal_face(kc, kr);
  const float fym = nodal_face(kym, kc), fyp = nodal_face(kc, kyp);
  const float fzm = nodal_face(kzm, kc), fzp = nodal_face(kc, kzp);
  float d = fxm;
  d += fxp;
  d += fym;
  d += fyp;
  d += fzm;
  d += fzp;
  float rr = fmaf(-d, up, gp);
  rr = fmaf(fxm, ul, rr);
  rr = fmaf(fxp, ur, rr);
  rr = fmaf(fym, uym, rr);
  rr = fmaf(fyp, uyp, rr);
  rr = fmaf(fzm, uzm, rr);
  rr = fmaf(fzp, uzp, rr);
  return rr;
}

// One colour of the nodal-coefficient red-black sweep on colour-split storage: the same
// operations in the same order as k_rbgs_nodal (bit for bit the same iterate). A thread
// updates the four nodes of one four-slot group of an interior row with 16-byte loads:
// its own k^-1 and g, the other colour's k^-1 and u in the same slots of its row (x - 1
// or x + 1 of the group's nodes) and of the rows y +- 1, z +- 1, plus one scalar slot
// outside the group. Grid (groups of the interior rows of a plane, interior planes,
// samples).
template <int LG>
__global__ void __launch_bounds__(128) k_rbgs_split(int colour, const float* __restrict__ kn,
                                                    const float* __restrict__ g, float* __restrict__ u,
                                                    const int* __restrict__ active) {
  using G = SplitGeo<LG>;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // group of an interior row
  if (q >= G::m * G::Q4) return;
  const int s = blockIdx.z;
  if (active && !active[s]) return;
  const int yi = q / G::Q4, qi = q - yi * G::Q4, y = 1 + yi, z = 1 + (int)blockIdx.y;
  const int par = (colour + y + z) & 1, xi0 = 4 * qi, x0 = 2 * xi0 + par;  // node i: x = x0 + 2 i
  if (x0 > G::n - 2) return;  // boundary and padding slots only
  const int o = (z * G::n + y) * G::P + xi0;
  const size_t cb = (size_t)s * G::NS + (size_t)colour * G::BLK, ob = (size_t)s * G::NS + (size_t)(1 - colour) * G::BLK;
  const float* ko = kn + ob;
  const float* uo = u + ob;
  const float4 kc4 = ld4(kn + cb + o), g4 = ld4(g + cb + o);
  const float4 km4 = ld4(ko + o), kym4 = ld4(ko + o - G::P), kyp4 = ld4(ko + o + G::P);
  const float4 kzm4 = ld4(ko + o - G::NP), kzp4 = ld4(ko + o + G::NP);
  const float4 um4 = ld4(uo + o), uym4 = ld4(uo + o - G::P), uyp4 = ld4(uo + o + G::P);
  const float4 uzm4 = ld4(uo + o - G::NP), uzp4 = ld4(uo + o + G::NP);
  // the other-colour slot beside the group: left of node 0 (x parity 0) or right of node 3
  float kext = 0.0f, uext = 0.0f;
  if (par) {
    kext = ko[o + 4];
    uext = uo[o + 4];
  } else if (x0 > 0) {
    kext = ko[o - 1];
    uext = uo[o - 1];
  }
  float out[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float kl = par ? comp(km4, i) : (i == 0 ? kext : comp(km4, i - 1));
    const float ul = par ? comp(um4, i) : (i == 0 ? uext : comp(um4, i - 1));
    const float kr = par ? (i == 3 ? kext : comp(km4, i + 1)) : comp(km4, i);
    const float ur = par ? (i == 3 ? uext : comp(um4, i + 1)) : comp(um4, i);
    out[i] = nodal_update(comp(kc4, i), comp(g4, i), kl, ul, kr, ur, comp(kym4, i), comp(uym4, i), comp(kyp4, i),
                          comp(uyp4, i), comp(kzm4, i), comp(uzm4, i), comp(kzp4, i), comp(uzp4, i));
  }
  float* uc = u + cb + o;
  if (x0 >= 1 && x0 + 6 <= G::n - 2) {
    *reinterpret_cast<float4*>(uc) = make_float4(out[0], out[1], out[2], out[3]);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (x0 + 2 * i >= 1 && x0 + 2 * i <= G::n - 2) uc[i] = out[i];
  }
}

// r~ = g - D u + sum K u_q (k_residual_nodal's operations and order) at the interior
// nodes of one colour, four slots per thread as in k_rbgs_split, into r in colour-split
// storage (the restriction reads only interior fine nodes; boundary and padding slots of
// r are not written). Grid (groups of the interior rows of a plane, 2 x interior planes,
// samples): colour = blockIdx.y & 1, so the two colours of a plane run back to back and
// the 1/k and u rows each reads as the other colour's are still in L2.
template <int LG>
__global__ void __launch_bounds__(128, 8) k_residual_split(const float* __restrict__ kn, const float* __restrict__ g,
                                                        const float* __restrict__ u, float* __restrict__ r,
                                                        const int* __restrict__ active) {
  using G = SplitGeo<LG>;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= G::m * G::Q4) return;
  const int s = blockIdx.z, colour = blockIdx.y & 1;
  if (active && !active[s]) return;
  const int yi = q / G::Q4, qi = q - yi * G::Q4, y = 1 + yi, z = 1 + (int)(blockIdx.y >> 1);
  const int par = (colour + y + z) & 1, xi0 = 4 * qi, x0 = 2 * xi0 + par;
  if (x0 > G::n - 2) return;
  const int o = (z * G::n + y) * G::P + xi0;
  const size_t cb = (size_t)s * G::NS + (size_t)colour * G::BLK, ob = (size_t)s * G::NS + (size_t)(1 - colour) * G::BLK;
  const float* ko = kn + ob;
  const float* uo = u + ob;
  const float4 kc4 = ld4(kn + cb + o), g4 = ld4(g + cb + o), up4 = ld4(u + cb + o);
  const float4 km4 = ld4(ko + o), kym4 = ld4(ko + o - G::P), kyp4 = ld4(ko + o + G::P);
  const float4 kzm4 = ld4(ko + o - G::NP), kzp4 = ld4(ko + o + G::NP);
  const float4 um4 = ld4(uo + o), uym4 = ld4(uo + o - G::P), uyp4 = ld4(uo + o + G::P);
  const float4 uzm4 = ld4(uo + o - G::NP), uzp4 = ld4(uo + o + G::NP);
  float kext = 0.0f, uext = 0.0f;
  if (par) {
    kext = ko[o + 4];
    uext = uo[o + 4];
  } else if (x0 > 0) {
    kext = ko[o - 1];
    uext = uo[o - 1];
  }
  float out[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float kl = par ? comp(km4, i) : (i == 0 ? kext : comp(km4, i - 1));
    const float ul = par ? comp(um4, i) : (i == 0 ? uext : comp(um4, i - 1));
    const float kr = par ? (i == 3 ? kext : comp(km4, i + 1)) : comp(km4, i);
    const float ur = par ? (i == 3 ? uext : comp(um4, i + 1)) : comp(um4, i);
    out[i] = nodal_residual(comp(kc4, i), comp(g4, i), comp(up4, i), kl, ul, kr, ur, comp(kym4, i), comp(uym4, i),
                            comp(kyp4, i), comp(uyp4, i), comp(kzm4, i), comp(uzm4, i), comp(kzp4, i),
                            comp(uzp4, i));
  }
  float* rc = r + cb + o;
  if (x0 >= 1 && x0 + 6 <= G::n - 2) {
    *reinterpret_cast<float4*>(rc) = make_float4(out[0], out[1], out[2], out[3]);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (x0 + 2 * i >= 1 && x0 + 2 * i <= G::n - 2) rc[i] = out[i];
  }
}

// g_c = 4 FW(r~) (k_restrict's weights and order) from r~ in colour-split storage into the
// coarse grid's colour-split g, at interior coarse nodes. LG: the fine grid's. Grid
// (interior coarse nodes of a plane, interior coarse planes, samples).
template <int LG, typename T = float>
__global__ void __launch_bounds__(128) k_restrict_split(const T* __restrict__ r, T* __restrict__ gc,
                                                        const int* __restrict__ active) {
  using F = SplitGeo<LG>;
  using C = SplitGeo<LG - 1>;
  constexpr int mc = C::n - 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= mc * mc) return;
  const int s = blockIdx.z;
  if (active && !active[s]) return;
  const int Y = 1 + q / mc, X = 1 + q - (Y - 1) * mc, Z = 1 + (int)blockIdx.y;
  const T* rb = r + (size_t)s * F::NS;
  T v = 0;
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const T wgt = (T)((2 - abs(dx)) * (2 - abs(dy)) * (2 - abs(dz))) * (T)(1.0 / 16.0);
        const int fx = 2 * X + dx, fy = 2 * Y + dy, fz = 2 * Z + dz;  // colour (dx + dy + dz) & 1
        v = fma(wgt, rb[(size_t)((dx + dy + dz) & 1) * F::BLK + (size_t)((fz * F::n + fy) * F::P + (fx >> 1))], v);
      }
  gc[(size_t)s * C::NS + (size_t)((X + Y + Z) & 1) * C::BLK + (size_t)((Z * C::n + Y) * C::P + (X >> 1))] = v;
}

// u_f += trilinear interpolation of e_c on colour-split storage of both grids: the
// coarse terms of k_prolong in its order (rows (Z, Y), (Z, Y+1), (Z+1, Y), (Z+1, Y+1),
// each X then X+1) and its weights, so the result is bit for bit that of k_prolong. A
// thread corrects the four fine nodes of one four-slot group of one colour (x = x0 + 2 i,
// coarse X = xi0 + i, one x parity, hence one weight pattern) with a 16-byte update of u;
// each coarse row it needs is gathered once for the group (X = xi0 .. xi0 + 4). LG: the
// fine grid's. Grid (groups of the interior rows of a plane, interior planes,
// 2 x samples: colour = blockIdx.z & 1).
template <int LG>
__global__ void __launch_bounds__(128) k_prolong_split(const float* __restrict__ ec, float* __restrict__ u,
                                                       const int* __restrict__ active) {
  using F = SplitGeo<LG>;
  using C = SplitGeo<LG - 1>;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= F::m * F::Q4) return;
  const int s = blockIdx.z >> 1, colour = blockIdx.z & 1;
  if (active && !active[s]) return;
  const int yi = q / F::Q4, qi = q - yi * F::Q4, y = 1 + yi, z = 1 + (int)blockIdx.y;
  const int xo = (colour + y + z) & 1, xi0 = 4 * qi, x0 = 2 * xi0 + xo;
  if (x0 > F::n - 2) return;
  const int yo = y & 1, zo = z & 1, Y = y >> 1, Z = z >> 1;
  const float* e = ec + (size_t)s * C::NS;
  // coarse row (Y + b, Z + c) at X = xi0 + t, t = 0 .. 4 (xi0 even: colour (t + Y + b + Z + c) & 1,
  // slot xi0 / 2 + t / 2)
  auto row = [&](int b, int c, float* cv) {
    const int cy = Y + b, cz = Z + c, base = (cz * C::n + cy) * C::P + (xi0 >> 1);
#pragma unroll
    for (int t = 0; t < 5; ++t)
      if (t < 4 || xo) cv[t] = e[(size_t)((t + cy + cz) & 1) * C::BLK + (size_t)(base + (t >> 1))];
  };
  float r00[5], r10[5], r01[5], r11[5];  // rows (Y, Z), (Y+1, Z), (Y, Z+1), (Y+1, Z+1)
  row(0, 0, r00);
  if (yo) row(1, 0, r10);
  if (zo) {
    row(0, 1, r01);
    if (yo) row(1, 1, r11);
  }
  const float w = xo + yo + zo == 0 ? 1.0f : xo + yo + zo == 1 ? 0.5f : xo + yo + zo == 2 ? 0.25f : 0.125f;
  float* uc = u + (size_t)s * F::NS + (size_t)colour * F::BLK + (size_t)((z * F::n + y) * F::P + xi0);
  const float4 u4 = ld4(uc);
  float out[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float v = 0.0f;
    v += r00[i];
    if (xo) v += r00[i + 1];
    if (yo) {
      v += r10[i];
      if (xo) v += r10[i + 1];
    }
    if (zo) {
      v += r01[i];
      if (xo) v += r01[i + 1];
      if (yo) {
        v += r11[i];
        if (xo) v += r11[i + 1];
      }
    }
    out[i] = comp(u4, i) + w * v;
  }
  if (x0 >= 1 && x0 + 6 <= F::n - 2) {
    *reinterpret_cast<float4*>(uc) = make_float4(out[0], out[1], out[2], out[3]);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (x0 + 2 * i >= 1 && x0 + 2 * i <= F::n - 2) uc[i] = out[i];
  }
}

// ---------------------------------------------------------------------------------
// Colour-split storage of FP64 stored-face grids (MLMC_SMOOTH_SPLIT in an FP64 solve):
// u, g, r, the faces Kx, Ky, Kz (each at its lower node), D and 1/D of every grid but the
// coarsest in the split storage. A colour pass then reads its own colour's faces, 1/D and
// g, the other colour's three lower faces and u, and writes its own u: 5 words per node and
// pass at line granularity against the plain layout's ~7. Every kernel performs the
// two-pass kernels' operations in their order, so the iterates are those of
// MLMC_SMOOTH_TWO_PASS bit for bit.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double2 ld2(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ double comp2(const double2& v, int i) { return i == 0 ? v.x : v.y; }

// harmonic faces of the (injected) FP64 nodal k into colour-split storage (k_faces).
__global__ void k_faces_split(const double* __restrict__ k0, int n0, int st0, int n, int B, double* __restrict__ Kx,
                              double* __restrict__ Ky, double* __restrict__ Kz) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // node of the plane
  if (q >= n * n) return;
  const int y = q / n, x = q - y * n;
  const size_t ns = split_elems(n), n03 = (size_t)n0 * n0 * n0;
  for (int zz = blockIdx.y; zz < B * n; zz += gridDim.y) {
    const int s = zz / n, z = zz - s * n;
    const double* kb = k0 + (size_t)s * n03;
    const size_t p0 = ((size_t)(st0 * z) * n0 + (size_t)(st0 * y)) * n0 + (size_t)(st0 * x);
    const size_t t = (size_t)s * ns + split_index(n, x, y, z);
    const double a = kb[p0];
    Kx[t] = x < n - 1 ? harm(a, kb[p0 + st0], double()) : 0.0;
    Ky[t] = y < n - 1 ? harm(a, kb[p0 + (size_t)st0 * n0], double()) : 0.0;
    Kz[t] = z < n - 1 ? harm(a, kb[p0 + (size_t)st0 * n0 * n0], double()) : 0.0;
  }
}

// D = sum of the six faces (k_diag's order) and 1/D at interior nodes, 0 on the boundary,
// all in colour-split storage.
__global__ void k_diag_split(int n, int B, const double* __restrict__ Kx, const double* __restrict__ Ky,
                             const double* __restrict__ Kz, double* __restrict__ D, double* __restrict__ Dinv) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  const int y = q / n, x = q - y * n;
  const size_t ns = split_elems(n);
  for (int zz = blockIdx.y; zz < B * n; zz += gridDim.y) {
    const int s = zz / n, z = zz - s * n;
    const size_t b = (size_t)s * ns, t = b + split_index(n, x, y, z);
    const bool in = x > 0 && y > 0 && z > 0 && x < n - 1 && y < n - 1 && z < n - 1;
    double d = 0.0;
    if (in) {
      d = Kx[b + split_index(n, x - 1, y, z)];
      d += Kx[t];
      d += Ky[b + split_index(n, x, y - 1, z)];
      d += Ky[t];
      d += Kz[b + split_index(n, x, y, z - 1)];
      d += Kz[t];
    }
    D[t] = d;
    Dinv[t] = in ? 1.0 / d : 0.0;
  }
}

// plain <-> colour-split copies of B samples of an n^3 grid (every node)
template <typename T, bool TO_SPLIT>
__global__ void k_split_copy(int n, int B, const T* __restrict__ a, T* __restrict__ b) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n * n) return;
  const int y = q / n, x = q - y * n;
  const size_t n3 = (size_t)n * n * n, ns = split_elems(n);
  for (int zz = blockIdx.y; zz < B * n; zz += gridDim.y) {
    const int s = zz / n, z = zz - s * n;
    const size_t tp = (size_t)s * n3 + (size_t)(z * n * n + q), ts = (size_t)s * ns + split_index(n, x, y, z);
    if (TO_SPLIT)
      b[ts] = a[tp];
    else
      b[tp] = a[ts];
  }
}

// One colour of the stored-face sweep on colour-split FP64 storage (k_rbgs's operations
// and order), two nodes per thread on 16-byte loads: its own Kx, Ky, Kz, 1/D and g, the
// other colour's lower faces (x - 1, y - 1, z - 1 nodes) and u of the six neighbours.
// Grid (two-slot groups of the interior rows of a plane, interior planes, samples).
template <int LG>
__global__ void __launch_bounds__(128) k_rbgs_split64(int colour, const double* __restrict__ Kx,
                                                      const double* __restrict__ Ky, const double* __restrict__ Kz,
                                                      const double* __restrict__ Dinv, const double* __restrict__ g,
                                                      double* __restrict__ u, const int* __restrict__ active) {
  using G = SplitGeo<LG>;
  constexpr int Q2 = G::P / 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= G::m * Q2) return;
  const int s = blockIdx.z;
  if (active && !active[s]) return;
  const int yi = q / Q2, qi = q - yi * Q2, y = 1 + yi, z = 1 + (int)blockIdx.y;
  const int par = (colour + y + z) & 1, xi0 = 2 * qi, x0 = 2 * xi0 + par;  // node i: x = x0 + 2 i
  if (x0 > G::n - 2) return;
  const int o = (z * G::n + y) * G::P + xi0;
  const size_t cb = (size_t)s * G::NS + (size_t)colour * G::BLK, ob = (size_t)s * G::NS + (size_t)(1 - colour) * G::BLK;
  const double2 kx2 = ld2(Kx + cb + o), ky2 = ld2(Ky + cb + o), kz2 = ld2(Kz + cb + o);
  const double2 di2 = ld2(Dinv + cb + o), g2 = ld2(g + cb + o);
  const double* kxo = Kx + ob;
  const double* uo = u + ob;
  const double2 kxm2 = ld2(kxo + o), kym2 = ld2(Ky + ob + o - G::P), kzm2 = ld2(Kz + ob + o - G::NP);
  const double2 um2 = ld2(uo + o), uym2 = ld2(uo + o - G::P), uyp2 = ld2(uo + o + G::P);
  const double2 uzm2 = ld2(uo + o - G::NP), uzp2 = ld2(uo + o + G::NP);
  // the other-colour slot beside the pair: left of node 0 (x parity 0) or right of node 1
  double kext = 0.0, uext = 0.0;
  if (par) {
    uext = uo[o + 2];
  } else if (x0 > 0) {
    kext = kxo[o - 1];
    uext = uo[o - 1];
  }
  double out[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    // lower x face at the x - 1 node: slot xi0 + i - 1 + par of the other colour
    const double kl = par ? comp2(kxm2, i) : (i == 0 ? kext : comp2(kxm2, i - 1));
    const double ul = par ? comp2(um2, i) : (i == 0 ? uext : comp2(um2, i - 1));
    const double ur = par ? (i == 1 ? uext : comp2(um2, i + 1)) : comp2(um2, i);
    double acc = comp2(g2, i);
    acc = fma(kl, ul, acc);
    acc = fma(comp2(kx2, i), ur, acc);
    acc = fma(comp2(kym2, i), comp2(uym2, i), acc);
    acc = fma(comp2(ky2, i), comp2(uyp2, i), acc);
    acc = fma(comp2(kzm2, i), comp2(uzm2, i), acc);
    acc = fma(comp2(kz2, i), comp2(uzp2, i), acc);
    out[i] = acc * comp2(di2, i);
  }
  double* uc = u + cb + o;
  if (x0 >= 1 && x0 + 2 <= G::n - 2) {
    *reinterpret_cast<double2*>(uc) = make_double2(out[0], out[1]);
  } else {
#pragma unroll
    for (int i = 0; i < 2; ++i)
      if (x0 + 2 * i >= 1 && x0 + 2 * i <= G::n - 2) uc[i] = out[i];
  }
}

// r~ = g - D u + sum K u_q (k_residual_z's operations and order) at the interior nodes of
// one colour, two per thread, into r in colour-split storage (interior nodes only).
// Grid (two-slot groups of the interior rows of a plane, 2 x interior planes, samples):
// colour = blockIdx.y & 1 (the two colours of a plane back to back).
template <int LG>
__global__ void __launch_bounds__(128) k_residual_split64(const double* __restrict__ Kx, const double* __restrict__ Ky,
                                                          const double* __restrict__ Kz, const double* __restrict__ D,
                                                          const double* __restrict__ g, const double* __restrict__ u,
                                                          double* __restrict__ r, const int* __restrict__ active) {
  using G = SplitGeo<LG>;
  constexpr int Q2 = G::P / 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= G::m * Q2) return;
  const int s = blockIdx.z, colour = blockIdx.y & 1;
  if (active && !active[s]) return;
  const int yi = q / Q2, qi = q - yi * Q2, y = 1 + yi, z = 1 + (int)(blockIdx.y >> 1);
  const int par = (colour + y + z) & 1, xi0 = 2 * qi, x0 = 2 * xi0 + par;
  if (x0 > G::n - 2) return;
  const int o = (z * G::n + y) * G::P + xi0;
  const size_t cb = (size_t)s * G::NS + (size_t)colour * G::BLK, ob = (size_t)s * G::NS + (size_t)(1 - colour) * G::BLK;
  const double2 kx2 = ld2(Kx + cb + o), ky2 = ld2(Ky + cb + o), kz2 = ld2(Kz + cb + o);
  const double2 d2 = ld2(D + cb + o), g2 = ld2(g + cb + o), up2 = ld2(u + cb + o);
  const double* kxo = Kx + ob;
  const double* uo = u + ob;
  const double2 kxm2 = ld2(kxo + o), kym2 = ld2(Ky + ob + o - G::P), kzm2 = ld2(Kz + ob + o - G::NP);
  const double2 um2 = ld2(uo + o), uym2 = ld2(uo + o - G::P), uyp2 = ld2(uo + o + G::P);
  const double2 uzm2 = ld2(uo + o - G::NP), uzp2 = ld2(uo + o + G::NP);
  double kext = 0.0, uext = 0.0;
  if (par) {
    uext = uo[o + 2];
  } else if (x0 > 0) {
    kext = kxo[o - 1];
    uext = uo[o - 1];
  }
  double out[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double kl = par ? comp2(kxm2, i) : (i == 0 ? kext : comp2(kxm2, i - 1));
    const double ul = par ? comp2(um2, i) : (i == 0 ? uext : comp2(um2, i - 1));
    const double ur = par ? (i == 1 ? uext : comp2(um2, i + 1)) : comp2(um2, i);
    double rr = fma(-comp2(d2, i), comp2(up2, i), comp2(g2, i));
    rr = fma(kl, ul, rr);
    rr = fma(comp2(kx2, i), ur, rr);
    rr = fma(comp2(kym2, i), comp2(uym2, i), rr);
    rr = fma(comp2(ky2, i), comp2(uyp2, i), rr);
    rr = fma(comp2(kzm2, i), comp2(uzm2, i), rr);
    rr = fma(comp2(kz2, i), comp2(uzp2, i), rr);
    out[i] = rr;
  }
  double* rc = r + cb + o;
  if (x0 >= 1 && x0 + 2 <= G::n - 2) {
    *reinterpret_cast<double2*>(rc) = make_double2(out[0], out[1]);
  } else {
#pragma unroll
    for (int i = 0; i < 2; ++i)
      if (x0 + 2 * i >= 1 && x0 + 2 * i <= G::n - 2) rc[i] = out[i];
  }
}

// Dispatch of a colour-split kernel template on n = 2^LG + 1 (5 .. 1025).
#define MLMC_SPLIT_DISPATCH(n, CALL)         \
  switch (n) {                               \
    case 5: { constexpr int LG = 2; CALL; } break;   \
    case 9: { constexpr int LG = 3; CALL; } break;   \
    case 17: { constexpr int LG = 4; CALL; } break;  \
    case 33: { constexpr int LG = 5; CALL; } break;  \
    case 65: { constexpr int LG = 6; CALL; } break;  \
    case 129: { constexpr int LG = 7; CALL; } break; \
    case 257: { constexpr int LG = 8; CALL; } break; \
    case 513: { constexpr int LG = 9; CALL; } break; \
    default: { constexpr int LG = 10; CALL; } break; \
  }

template <int THREADS>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double warp_part[THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) warp_part[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = lane < THREADS / 32 ? warp_part[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

// Blocks per sample of the deterministic reductions: a function of the grid size only
// (never of the batch), so that a sample's sums do not depend on its batch; up to 1024
// blocks so that one or two large samples still fill the GPU.
inline int reduce_blocks(size_t work) {
  size_t nb = (work + 4095) / 4096;
  if (nb < 1) nb = 1;
  if (nb > 1024) nb = 1024;
  return (int)nb;
}

// Sum of squares over interior nodes of an FP64 array (initial ||g||). Grid (NB, B).
__global__ void __launch_bounds__(kThreads) k_sumsq(int n, const double* __restrict__ v, double* __restrict__ partial) {
  const int s = blockIdx.y;
  const unsigned n3 = (unsigned)n * n * n, n2 = (unsigned)n * n, un = (unsigned)n;
  const unsigned chunk = (n3 + gridDim.x - 1) / gridDim.x;
  const unsigned lo = blockIdx.x * chunk, hi = lo + chunk < n3 ? lo + chunk : n3;
  double sq = 0.0;
  for (unsigned i = lo + threadIdx.x; i < hi; i += kThreads) {
    const unsigned zq = i / n2, rem = i - zq * n2, yq = rem / un;
    const int z = (int)zq, y = (int)yq, x = (int)(rem - yq * un);
    if (x > 0 && y > 0 && z > 0 && x < n - 1 && y < n - 1 && z < n - 1) {
      const double a = v[(size_t)s * n3 + i];
      sq += a * a;
    }
  }
  const double b = block_sum<kThreads>(sq);
  if (threadIdx.x == 0) partial[(size_t)s * gridDim.x + blockIdx.x] = b;
}

// Sum of a sample's NB block partials by one warp: lane l adds partials l, l+32, ...
// in order, then a fixed shuffle tree; the result depends only on NB (not on the batch).
__device__ __forceinline__ double warp_sum_partials(const double* __restrict__ p, int NB) {
  const int lane = threadIdx.x & 31;
  double t = 0.0;
  for (int b = lane; b < NB; b += 32) t += p[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// Per sample: total of the NB partials (fixed order). mode 0: store ||g||^2.
// mode 1: relative residual, cycle count and active flag after `inc` cycles.
__global__ void k_norm_update(int B, int NB, const double* __restrict__ partial, double* __restrict__ g2,
                              double* __restrict__ relres, int* __restrict__ cycles, int* __restrict__ active,
                              int mode, int inc, double rtol, int max_cycles, int* __restrict__ n_active) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // one warp per sample
  if (s >= B) return;
  if (mode == 1 && !active[s]) return;
  const double t = warp_sum_partials(partial + (size_t)s * NB, NB);
  if ((threadIdx.x & 31) != 0) return;
  if (mode == 0) {
    g2[s] = t;
    return;
  }
  const double rel = g2[s] > 0.0 ? sqrt(t / g2[s]) : 0.0;
  relres[s] = rel;
  cycles[s] += inc;
  const int c = cycles[s];
  const int still = (rtol > 0.0) ? (rel > rtol && c < max_cycles) : (c < max_cycles);
  active[s] = still;
  if (still) atomicAdd(n_active, 1);
}

// g_c = 4 FW(r~) at interior coarse nodes (the coarse boundary of g_c is zeroed once per
// solve and never written).
template <typename T, bool SPLIT_OUT = false>
__global__ void k_restrict(int nf, int B, const T* __restrict__ r, T* __restrict__ gc, const int* __restrict__ active) {
  // nc - 1 = 2^(p-1) = hc: an interior coarse row is X = 1 .. hc - 1
  const int nc = (nf + 1) / 2, hc = nc - 1, lc = 31 - __clz(hc);
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // interior coarse node of a plane
  if (q >= (nc - 2) * hc) return;
  const int X = 1 + (q & (hc - 1)), Y = 1 + (q >> lc);
  if (X > nc - 2) return;
  const size_t nc3 = (size_t)nc * nc * nc, nf3 = (size_t)nf * nf * nf;
  const int nf2 = nf * nf;
  for (int zz = blockIdx.y; zz < B * (nc - 2); zz += gridDim.y) {
    const int s = zz / (nc - 2), Z = 1 + (zz - s * (nc - 2));
    if (active && !active[s]) continue;
    const T* rb = r + (size_t)s * nf3 + (size_t)(2 * Z * nf2 + 2 * Y * nf + 2 * X);
    T v = 0;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const T wgt = (T)((2 - abs(dx)) * (2 - abs(dy)) * (2 - abs(dz))) * (T)(1.0 / 16.0);
          v = fma(wgt, rb[dz * nf2 + dy * nf + dx], v);
        }
    if (SPLIT_OUT)
      gc[(size_t)s * split_elems(nc) + split_index(nc, X, Y, Z)] = v;
    else
      gc[(size_t)s * nc3 + (size_t)((Z * nc + Y) * nc + X)] = v;
  }
}

// u_f += trilinear interpolation of e_c at interior fine nodes: a fine node with k odd
// coordinates is the mean of its 2^k coarse neighbours (k = 0: the coincident coarse
// node). Threads of a row take the odd x first and the even x after them, so that a warp
// shares one parity pattern and sums only the distinct neighbours (4.3 instead of 8
// terms per node on average).
template <typename T>
__global__ void k_prolong(int nf, int B, const T* __restrict__ ec, T* __restrict__ u, const int* __restrict__ active) {
  // nf - 1 = 2^p = P: interior x of a row, odd ones (r < P/2: x = 2r + 1) then even ones
  const int nc = (nf + 1) / 2, P = nf - 1, lp = 31 - __clz(P), hp = P >> 1;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (nf - 2) * P) return;
  const int rr = q & (P - 1), y = 1 + (q >> lp);
  const int x = rr < hp ? 2 * rr + 1 : 2 * (rr - hp) + 2;
  if (x > nf - 2) return;
  const size_t nc3 = (size_t)nc * nc * nc, nf3 = (size_t)nf * nf * nf;
  const int xo = x & 1, yo = y & 1, X = x >> 1, Y = y >> 1;
  for (int zz = blockIdx.y; zz < B * (nf - 2); zz += gridDim.y) {
    const int s = zz / (nf - 2), z = 1 + (zz - s * (nf - 2));
    if (active && !active[s]) continue;
    const int zo = z & 1, Z = z >> 1;
    // the distinct coarse neighbours in the order (Z, Y), (Z, Y+1), (Z+1, Y), (Z+1, Y+1),
    // each row X then X+1, as straight-line code (parities decide which exist)
    const T* r0 = ec + (size_t)s * nc3 + (size_t)((Z * nc + Y) * nc + X);
    T v = 0;
    v += r0[0];
    if (xo) v += r0[1];
    if (yo) {
      v += r0[nc];
      if (xo) v += r0[nc + 1];
    }
    if (zo) {
      const T* r2 = r0 + nc * nc;
      v += r2[0];
      if (xo) v += r2[1];
      if (yo) {
        v += r2[nc];
        if (xo) v += r2[nc + 1];
      }
    }
    const T w = xo + yo + zo == 0 ? T(1) : xo + yo + zo == 1 ? T(0.5) : xo + yo + zo == 2 ? T(0.25) : T(0.125);
    const size_t p = (size_t)s * nf3 + (size_t)((z * nf + y) * nf + x);
    u[p] += w * v;
  }
}

// The sums of k_prolong for the eight fine nodes (2X + dx, 2Y + dy, 2Z + dz) of one coarse
// cell, c = e_c at (X, Y, Z), (X+1, Y, Z), (X, Y+1, Z), (X+1, Y+1, Z), then the same at Z+1:
// every node's sum takes its terms in k_prolong's order, and the nodes whose term
// sequences share a prefix share its partial sum (14 additions for the block instead of 27).
// v[dx + 2 dy + 4 dz].
template <typename T>
__device__ __forceinline__ void prolong_block_sums(const T (&c)[8], T (&v)[8]) {
  T sa = 0;
  sa += c[0];
  const T sab = sa + c[1], sac = sa + c[2];
  const T sabcd = (sab + c[2]) + c[3];
  v[0] = sa;
  v[1] = sab;
  v[2] = sac;
  v[3] = sabcd;
  v[4] = sa + c[4];
  v[5] = (sab + c[4]) + c[5];
  v[6] = (sac + c[4]) + c[6];
  v[7] = (((sabcd + c[4]) + c[5]) + c[6]) + c[7];
}

// k_prolong's result (bit for bit) with one thread per coarse cell: the eight fine nodes
// (2X + dx, 2Y + dy, 2Z + dz) of the cell, their sums from prolong_block_sums, u += w v at
// the interior ones. Every thread runs the same operations (no parity divergence) and the
// block shares partial sums: 2.75 instead of 4.4 FP64 operations per fine node. Grid: coarse
// cells of a plane, (sample, cell plane) planes.
template <typename T>
__global__ void __launch_bounds__(128) k_prolong_blk(int nf, int B, const T* __restrict__ ec, T* __restrict__ u,
                                                     const int* __restrict__ active) {
  const int nc = (nf + 1) / 2, mc = nc - 1;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= mc * mc) return;
  const int Y = q / mc, X = q - Y * mc;
  const size_t nc3 = (size_t)nc * nc * nc, nf3 = (size_t)nf * nf * nf, nc2 = (size_t)nc * nc;
  for (int zz = blockIdx.y; zz < B * mc; zz += gridDim.y) {
    const int s = zz / mc, Z = zz - s * mc;
    if (active && !active[s]) continue;
    const T* e = ec + (size_t)s * nc3 + (size_t)((Z * nc + Y) * nc + X);
    const T c[8] = {e[0], e[1], e[nc], e[nc + 1], e[nc2], e[nc2 + 1], e[nc2 + nc], e[nc2 + nc + 1]};
    T v[8];
    prolong_block_sums(c, v);
    T* ub = u + (size_t)s * nf3;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
      const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
      if (x < 1 || y < 1 || z < 1 || x > nf - 2 || y > nf - 2 || z > nf - 2) continue;
      const T w = dx + dy + dz == 0 ? T(1) : dx + dy + dz == 1 ? T(0.5) : dx + dy + dz == 2 ? T(0.25) : T(0.125);
      ub[(size_t)((z * nf + y) * nf + x)] += w * v[k];
    }
  }
}

// k_prolong_blk on colour-split storage of both grids (LG: the fine grid's). Fine node
// (2X + dx, ...) is colour (dx + dy + dz) & 1, slot X; coarse (X', Y', Z') colour
// (X' + Y' + Z') & 1, slot X' / 2. Grid (coarse cells of a plane, cell planes, samples).
template <int LG, typename T>
__global__ void __launch_bounds__(128) k_prolong_blk_split(const T* __restrict__ ec, T* __restrict__ u,
                                                           const int* __restrict__ active) {
  using F = SplitGeo<LG>;
  using C = SplitGeo<LG - 1>;
  constexpr int mc = C::n - 1;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= mc * mc) return;
  const int s = blockIdx.z;
  if (active && !active[s]) return;
  const int Y = q / mc, X = q - Y * mc, Z = (int)blockIdx.y;
  const T* e = ec + (size_t)s * C::NS;
  auto at = [&](int i, int j, int k) -> T {
    const int xx = X + i, yy = Y + j, zz = Z + k;
    return e[(size_t)((xx + yy + zz) & 1) * C::BLK + (size_t)((zz * C::n + yy) * C::P + (xx >> 1))];
  };
  const T c[8] = {at(0, 0, 0), at(1, 0, 0), at(0, 1, 0), at(1, 1, 0), at(0, 0, 1), at(1, 0, 1), at(0, 1, 1), at(1, 1, 1)};
  T v[8];
  prolong_block_sums(c, v);
  T* ub = u + (size_t)s * F::NS;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
    const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
    if (x < 1 || y < 1 || z < 1 || x > F::n - 2 || y > F::n - 2 || z > F::n - 2) continue;
    const T w = dx + dy + dz == 0 ? T(1) : dx + dy + dz == 1 ? T(0.5) : dx + dy + dz == 2 ? T(0.25) : T(0.125);
    ub[(size_t)((dx + dy + dz) & 1) * F::BLK + (size_t)((z * F::n + y) * F::P + X)] += w * v[k];
  }
}

// g = h^2 f (f == NULL: h^2) on interior nodes, 0 on the boundary; u boundary := 0.
template <bool SPLIT = false>
__global__ void k_prepare(int n, int B, double h2, const double* __restrict__ f, double* __restrict__ g,
                          double* __restrict__ u) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // node of the plane
  if (q >= n * n) return;
  const int y = q / n, x = q - y * n;
  const size_t n3 = (size_t)n * n * n;
  for (int zz = blockIdx.y; zz < B * n; zz += gridDim.y) {
    const int s = zz / n, z = zz - s * n;
    const size_t tp = (size_t)s * n3 + (size_t)(z * n * n + q), t = SPLIT ? node_at<true>(n, s, x, y, z) : tp;
    const bool in = x > 0 && y > 0 && z > 0 && x < n - 1 && y < n - 1 && z < n - 1;
    g[t] = in ? h2 * (f ? f[tp] : 1.0) : 0.0;
    if (!in) u[t] = 0.0;
  }
}

// Mixed refinement update u64 += e32 at interior nodes of active samples (SPLIT: e in
// colour-split storage).
template <bool SPLIT>
__global__ void k_update_mixed(int n, int B, const float* __restrict__ e, double* __restrict__ u,
                               const int* __restrict__ active) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // node of the plane
  if (q >= n * n) return;
  const int y = q / n, x = q - y * n;
  const size_t n3 = (size_t)n * n * n;
  for (int zz = blockIdx.y; zz < B * n; zz += gridDim.y) {
    const int s = zz / n, z = zz - s * n;
    if (!active[s]) continue;
    const size_t t = (size_t)s * n3 + (size_t)(z * n * n + q);
    const float ev = SPLIT ? e[(size_t)s * split_elems(n) + split_index(n, x, y, z)] : e[t];
    u[t] += widen(ev);  // e is zero on the boundary
  }
}

// QoI partial sums (trapezoid weights, Kahan in each thread). Grid (NB, B).
__global__ void __launch_bounds__(kThreads) k_qoi(int n, const double* __restrict__ u, double* __restrict__ partial) {
  const int s = blockIdx.y;
  const int lo = (n - 1) / 4, S = (n - 1) / 2 + 1;
  const unsigned S3 = (unsigned)S * S * S, S2 = (unsigned)S * S, uS = (unsigned)S;
  const size_t n3 = (size_t)n * n * n;
  const unsigned chunk = (S3 + gridDim.x - 1) / gridDim.x;
  const unsigned a = blockIdx.x * chunk, b = a + chunk < S3 ? a + chunk : S3;
  double sum = 0.0, comp = 0.0;
  for (unsigned i = a + threadIdx.x; i < b; i += kThreads) {
    const unsigned czq = i / S2, rem = i - czq * S2, cyq = rem / uS;
    const int cz = (int)czq, cy = (int)cyq, cx = (int)(rem - cyq * uS);
    const double w = (cx == 0 || cx == S - 1 ? 0.5 : 1.0) * (cy == 0 || cy == S - 1 ? 0.5 : 1.0) *
                     (cz == 0 || cz == S - 1 ? 0.5 : 1.0);
    const double v = w * u[(size_t)s * n3 + ((size_t)(lo + cz) * n + (lo + cy)) * n + (lo + cx)];
    const double yk = v - comp;
    const double tk = sum + yk;
    comp = (tk - sum) - yk;
    sum = tk;
  }
  const double tot = block_sum<kThreads>(sum);
  if (threadIdx.x == 0) partial[(size_t)s * gridDim.x + blockIdx.x] = tot;
}

__global__ void k_qoi_final(int B, int NB, double scale, const double* __restrict__ partial, double* __restrict__ Q) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  double t = 0.0;
  for (int b = 0; b < NB; ++b) t += partial[(size_t)s * NB + b];
  Q[s] = scale * t;
}

// ---------------------------------------------------------------------------------
// P1 finite elements on the tetrahedral mesh (Sec. 3.1): every grid cube is cut into the
// six tetrahedra {O, O + e_a, O + e_a + e_b, O + (1,1,1)}; the stiffness with the four-vertex
// quadrature of k couples only the axis edges of each element's vertex path (the
// barycentric gradients of the path's non-adjacent vertices are orthogonal), so the
// operator keeps the seven-point form with, per axis edge, the mean over the six elements
// that share it of their vertex-mean coefficient kbar:
//   K_a(P) = (k_P + k_{P+a}) / 4 + (k_{P+a+b} + k_{P+a+c} + k_{P+a+b+c} + k_{P-b} + k_{P-c}
//            + k_{P-b-c}) / 12      ({a, b, c} = {x, y, z}),
// in the h^2-scaled form (FE matrix / h); the load of f = 1 is h^3 per interior node, the
// g = h^2 f of the scaled form.
// ---------------------------------------------------------------------------------
template <typename T>
__global__ void k_faces_fe(const double* __restrict__ k0, int n0, int st0, int n, int B, T* __restrict__ Kx,
                           T* __restrict__ Ky, T* __restrict__ Kz) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // node of the plane
  if (q >= n * n) return;
  const int y = q / n, x = q - y * n;
  const size_t n3 = (size_t)n * n * n, n03 = (size_t)n0 * n0 * n0;
  for (int zz = blockIdx.y; zz < B * n; zz += gridDim.y) {
    const int s = zz / n, z = zz - s * n;
    const double* kb = k0 + (size_t)s * n03;
    auto K = [&](int dx, int dy, int dz) {
      return kb[((size_t)(st0 * (z + dz)) * n0 + (size_t)(st0 * (y + dy))) * n0 + (size_t)(st0 * (x + dx))];
    };
    const bool ix = x >= 1 && x <= n - 2, iy = y >= 1 && y <= n - 2, iz = z >= 1 && z <= n - 2;
    const size_t t = (size_t)s * n3 + (size_t)(z * n * n + q);
    double fx = 0.0, fy = 0.0, fz = 0.0;
    if (x <= n - 2 && iy && iz)
      fx = (K(0, 0, 0) + K(1, 0, 0)) * 0.25 +
           (K(1, 1, 0) + K(1, 0, 1) + K(1, 1, 1) + K(0, -1, 0) + K(0, 0, -1) + K(0, -1, -1)) * (1.0 / 12.0);
    if (y <= n - 2 && ix && iz)
      fy = (K(0, 0, 0) + K(0, 1, 0)) * 0.25 +
           (K(0, 1, 1) + K(1, 1, 0) + K(1, 1, 1) + K(0, 0, -1) + K(-1, 0, 0) + K(-1, 0, -1)) * (1.0 / 12.0);
    if (z <= n - 2 && ix && iy)
      fz = (K(0, 0, 0) + K(0, 0, 1)) * 0.25 +
           (K(1, 0, 1) + K(0, 1, 1) + K(1, 1, 1) + K(-1, 0, 0) + K(0, -1, 0) + K(-1, -1, 0)) * (1.0 / 12.0);
    Kx[t] = (T)fx;
    Ky[t] = (T)fy;
    Kz[t] = (T)fz;
  }
}

// P1 interpolation between nested tetrahedral meshes, added on interior fine nodes: a
// fine node with odd coordinates d (a 0/1 vector) is the midpoint of the coarse edge from
// c0 = (f - d) / 2 to c0 + d (a mesh edge: every direction e_a, e_a + e_b, (1,1,1) is
// one), so it takes the mean of the two; a node with d = 0 is a coarse node.
template <typename T, bool SPLIT = false>
__global__ void k_prolong_p1(int nf, int B, const T* __restrict__ ec, T* __restrict__ u,
                             const int* __restrict__ active) {
  const int m = nf - 2, nc = (nf + 1) / 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // interior node of the plane
  if (q >= m * m) return;
  const int y = 1 + q / m, x = 1 + q - (y - 1) * m;
  for (int zz = blockIdx.y; zz < B * m; zz += gridDim.y) {
    const int s = zz / m, z = 1 + zz - s * m;
    if (active && !active[s]) continue;
    const int dx = x & 1, dy = y & 1, dz = z & 1;
    const int X0 = (x - dx) >> 1, Y0 = (y - dy) >> 1, Z0 = (z - dz) >> 1;
    T v = ec[node_at<SPLIT>(nc, s, X0, Y0, Z0)];
    if (dx | dy | dz) v = T(0.5) * (v + ec[node_at<SPLIT>(nc, s, X0 + dx, Y0 + dy, Z0 + dz)]);
    u[node_at<SPLIT>(nf, s, x, y, z)] += v;
  }
}

// Its transpose on interior coarse nodes, scaled for the coarse h^2-scaled system:
// g_c = (h / h_c) P^T r = (1/2) (r(2c) + (1/2) sum over the 14 mesh-edge directions d of
// r(2c + d)) (the fine residual r is zero on the boundary).
template <typename T, bool SPLIT = false>
__global__ void k_restrict_p1(int nf, int B, const T* __restrict__ r, T* __restrict__ gc,
                              const int* __restrict__ active) {
  const int nc = (nf + 1) / 2, mc = nc - 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // interior coarse node of the plane
  if (q >= mc * mc) return;
  const int Y = 1 + q / mc, X = 1 + q - (Y - 1) * mc;
  for (int zz = blockIdx.y; zz < B * mc; zz += gridDim.y) {
    const int s = zz / mc, Z = 1 + zz - s * mc;
    if (active && !active[s]) continue;
    auto R = [&](int dx, int dy, int dz) { return r[node_at<SPLIT>(nf, s, 2 * X + dx, 2 * Y + dy, 2 * Z + dz)]; };
    T acc = R(-1, 0, 0) + R(1, 0, 0);
    acc += R(0, -1, 0) + R(0, 1, 0);
    acc += R(0, 0, -1) + R(0, 0, 1);
    acc += R(-1, -1, 0) + R(1, 1, 0);
    acc += R(0, -1, -1) + R(0, 1, 1);
    acc += R(-1, 0, -1) + R(1, 0, 1);
    acc += R(-1, -1, -1) + R(1, 1, 1);
    gc[node_at<SPLIT>(nc, s, X, Y, Z)] = T(0.5) * R(0, 0, 0) + T(0.25) * acc;
  }
}

// Q[s] = u(1/4, 1/4, 1/4) (a node: (n - 1) / 4 in every coordinate).
__global__ void k_qoi_point(int n, int B, const double* __restrict__ u, double* __restrict__ Q) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  const int c = (n - 1) / 4;
  Q[s] = u[(size_t)s * n * n * n + ((size_t)c * n + c) * n + c];
}

// Flux of k du/dx_2 across x_2 = 1/4 as the mean over the layer of elements between
// x_2 = 1/4 - h and 1/4: per cube of the layer (origin y = (n-1)/4 - 1) and each of its
// six elements (path a, b, c), kbar times the difference of u along the path's y step;
// per-block partial sums (grid (NB, B)), scaled by h/6 in k_qoi_final. k from the FP64
// field k0 (stride st0).
__global__ void __launch_bounds__(kThreads) k_qoi_flux(int n, const double* __restrict__ u,
                                                       const double* __restrict__ k0, int n0, int st0,
                                                       double* __restrict__ partial) {
  const int s = blockIdx.y, NB = gridDim.x;
  const int m = n - 1, j0 = (n - 1) / 4 - 1;
  const size_t n3 = (size_t)n * n * n, n03 = (size_t)n0 * n0 * n0;
  const double* ub = u + (size_t)s * n3;
  const double* kb = k0 + (size_t)s * n03;
  double acc = 0.0;
  for (int c = blockIdx.x * kThreads + threadIdx.x; c < m * m; c += NB * kThreads) {
    const int zc = c / m, xc = c - zc * m;
    double uv[8], kv[8];  // cube corners, bit 0 = x, bit 1 = y, bit 2 = z
    for (int v = 0; v < 8; ++v) {
      const int X = xc + (v & 1), Y = j0 + ((v >> 1) & 1), Z = zc + (v >> 2);
      uv[v] = ub[((size_t)Z * n + Y) * n + X];
      kv[v] = kb[((size_t)(st0 * Z) * n0 + (size_t)(st0 * Y)) * n0 + (size_t)(st0 * X)];
    }
    const int ax[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int e = 0; e < 6; ++e) {
      int v = 0, vs[4];
      vs[0] = 0;
      double dy = 0.0;
      for (int i = 0; i < 3; ++i) {
        const int w = v | (1 << ax[e][i]);
        if (ax[e][i] == 1) dy = uv[w] - uv[v];
        v = w;
        vs[i + 1] = v;
      }
      const double kbar = 0.25 * (kv[vs[0]] + kv[vs[1]] + kv[vs[2]] + kv[vs[3]]);
      acc = fma(kbar, dy, acc);
    }
  }
  const double b = block_sum<kThreads>(acc);
  if (threadIdx.x == 0) partial[(size_t)s * NB + blockIdx.x] = b;
}

// ---------------------------------------------------------------------------------
// Flexible preconditioned conjugate gradients (FP64 recurrences; the V-cycle is the
// preconditioner). All vectors are FP64 on the finest grid; per-sample scalars.
// ---------------------------------------------------------------------------------

// q = A~ p on interior nodes (0 on the boundary): v = D p, then the six faces in the order
// -x, +x, -y, +y, -z, +z, and partials of p.q, by column z-marches: a thread owns one
// (x, y) column of a z-slab and carries p and Kz of the planes below and above in
// registers (11 loads per node), FP32 faces widened on the integer pipe. Grid (column blocks, z-slabs, B), 128 threads; one partial of p.q per
// (column block, slab), a partition fixed by n (apply_slabs).
template <typename TK, typename TD>
__global__ void __launch_bounds__(128)
    k_apply_dot_z(int n, int zslab, const TK* __restrict__ Kx, const TK* __restrict__ Ky, const TK* __restrict__ Kz,
                  const TD* __restrict__ D, const double* __restrict__ p, double* __restrict__ q,
                  double* __restrict__ partial, const int* __restrict__ active) {
  const int s = blockIdx.z;
  if (!active[s]) return;
  const int nb = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
  const int c = blockIdx.x * 128 + threadIdx.x;  // column y n + x
  const int zlo = 1 + blockIdx.y * zslab, zhi = min(n - 2, zlo + zslab - 1);
  const size_t n2 = (size_t)n * n;
  double acc = 0.0;
  if (c < n * n) {
    const int y = c / n, x = c - y * n;
    const size_t col = (size_t)s * n2 * n + c;
    if (x > 0 && y > 0 && x < n - 1 && y < n - 1) {
      double pm = p[col + (size_t)(zlo - 1) * n2], pc = p[col + (size_t)zlo * n2];
      double kzm = widen(Kz[col + (size_t)(zlo - 1) * n2]);
      for (int z = zlo; z <= zhi; ++z) {
        const size_t t = col + (size_t)z * n2;
        const double pp = p[t + n2];
        const double kzp = widen(Kz[t]);
        double v = widen(D[t]) * pc;
        v = fma(-widen(Kx[t - 1]), p[t - 1], v);
        v = fma(-widen(Kx[t]), p[t + 1], v);
        v = fma(-widen(Ky[t - n]), p[t - n], v);
        v = fma(-widen(Ky[t]), p[t + n], v);
        v = fma(-kzm, pm, v);
        v = fma(-kzp, pp, v);
        acc = fma(pc, v, acc);
        q[t] = v;
        pm = pc;
        pc = pp;
        kzm = kzp;
      }
    } else {
      for (int z = zlo; z <= zhi; ++z) q[col + (size_t)z * n2] = 0.0;
    }
    if (blockIdx.y == 0) q[col] = 0.0;                                    // plane z = 0
    if (blockIdx.y == gridDim.y - 1) q[col + (size_t)(n - 1) * n2] = 0.0;  // plane z = n-1
  }
  const double bs = block_sum<128>(acc);
  if (threadIdx.x == 0) partial[(size_t)s * nb + b] = bs;
}

// z-slabs of the column z-march kernels: a function of n only (so a sample's sums do not
// depend on the batch): enough (column, slab) threads to fill the GPU for one sample, but
// slabs of at least 8 planes, so that carrying the planes below and above in registers
// saves loads (one-plane slabs would load more than the flat kernels).
inline int apply_slabs(int n, int* zslab) {
  int slabs = (int)((131072LL + (long long)n * n - 1) / ((long long)n * n));
  const int deep = (n - 2) / 8 > 1 ? (n - 2) / 8 : 1;
  if (slabs > deep) slabs = deep;
  if (slabs < 1) slabs = 1;
  *zslab = (n - 2 + slabs - 1) / slabs;
  return (n - 2 + *zslab - 1) / *zslab;
}
inline int apply_blocks(int n) {
  int zs = 0;
  return ((n * n + 127) / 128) * apply_slabs(n, &zs);
}

// r~ = g - D u + sum K u_q on interior nodes (0 on the boundary) by column z-marches (the
// launch shape and partition of k_apply_dot_z): rr = g - D u, then the faces in the order
// -x, +x, -y, +y, -z, +z; optional store of r~ (type TR) and per-(column block, slab)
// partials of r~^2 (FP64).
template <typename T, typename TD, typename TU, typename TR, bool SPLIT_OUT = false>
__global__ void __launch_bounds__(128)
    k_residual_z(int n, int zslab, const T* __restrict__ Kx, const T* __restrict__ Ky, const T* __restrict__ Kz,
                 const TD* __restrict__ D, const TD* __restrict__ g, const TU* __restrict__ u, TR* __restrict__ r,
                 double* __restrict__ partial, const int* __restrict__ active) {
  const int s = blockIdx.z;
  if (active && !active[s]) return;
  const int nb = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
  const int c = blockIdx.x * 128 + threadIdx.x;  // column y n + x
  const int zlo = 1 + blockIdx.y * zslab, zhi = min(n - 2, zlo + zslab - 1);
  const size_t n2 = (size_t)n * n;
  double sq = 0.0;
  // store index of r~ at plane z of this column
  const int cy = c < n * n ? c / n : 0, cx = c - cy * n;
  auto rix = [&](size_t t, int z) -> size_t {
    return SPLIT_OUT ? (size_t)s * split_elems(n) + split_index(n, cx, cy, z) : t;
  };
  if (c < n * n) {
    const int y = cy, x = cx;
    const size_t col = (size_t)s * n2 * n + c;
    if (x > 0 && y > 0 && x < n - 1 && y < n - 1) {
      TD um = to_t<TD>(u[col + (size_t)(zlo - 1) * n2]), uc = to_t<TD>(u[col + (size_t)zlo * n2]);
      TD kzm = to_t<TD>(Kz[col + (size_t)(zlo - 1) * n2]);
      for (int z = zlo; z <= zhi; ++z) {
        const size_t t = col + (size_t)z * n2;
        const TD up = to_t<TD>(u[t + n2]);
        const TD kzp = to_t<TD>(Kz[t]);
        TD rr = fma(-D[t], uc, g[t]);
        rr = fma(to_t<TD>(Kx[t - 1]), to_t<TD>(u[t - 1]), rr);
        rr = fma(to_t<TD>(Kx[t]), to_t<TD>(u[t + 1]), rr);
        rr = fma(to_t<TD>(Ky[t - n]), to_t<TD>(u[t - n]), rr);
        rr = fma(to_t<TD>(Ky[t]), to_t<TD>(u[t + n]), rr);
        rr = fma(kzm, um, rr);
        rr = fma(kzp, up, rr);
        if (r) r[rix(t, z)] = (TR)rr;
        sq += (double)rr * (double)rr;
        um = uc;
        uc = up;
        kzm = kzp;
      }
    } else if (r) {
      for (int z = zlo; z <= zhi; ++z) r[rix(col + (size_t)z * n2, z)] = TR(0);
    }
    if (r && blockIdx.y == 0) r[rix(col, 0)] = TR(0);                                          // plane z = 0
    if (r && blockIdx.y == gridDim.y - 1) r[rix(col + (size_t)(n - 1) * n2, n - 1)] = TR(0);  // plane z = n-1
  }
  if (partial) {
    const double bs = block_sum<128>(sq);
    if (threadIdx.x == 0) partial[(size_t)s * nb + b] = bs;
  }
}

// The convergence residual of an FP64 colour-split grid: k_residual_z's column z-march,
// launch shape and partition (partials of r~^2 per (column block, slab)), reading the
// split storage; nothing stored. Grid (column blocks, z-slabs, samples), 128 threads.
__global__ void __launch_bounds__(128)
    k_residual_norm_split(int n, int zslab, const double* __restrict__ Kx, const double* __restrict__ Ky,
                          const double* __restrict__ Kz, const double* __restrict__ D, const double* __restrict__ g,
                          const double* __restrict__ u, double* __restrict__ partial, const int* __restrict__ active) {
  const int s = blockIdx.z;
  if (active && !active[s]) return;
  const int nb = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
  const int c = blockIdx.x * 128 + threadIdx.x;
  const int zlo = 1 + blockIdx.y * zslab, zhi = min(n - 2, zlo + zslab - 1);
  const size_t base = (size_t)s * split_elems(n);
  double sq = 0.0;
  if (c < n * n) {
    const int y = c / n, x = c - y * n;
    if (x > 0 && y > 0 && x < n - 1 && y < n - 1) {
      auto at = [&](int xx, int yy, int zz) -> size_t { return base + split_index(n, xx, yy, zz); };
      double um = u[at(x, y, zlo - 1)], uc = u[at(x, y, zlo)];
      double kzm = Kz[at(x, y, zlo - 1)];
      for (int z = zlo; z <= zhi; ++z) {
        const size_t t = at(x, y, z);
        const double up = u[at(x, y, z + 1)];
        const double kzp = Kz[t];
        double rr = fma(-D[t], uc, g[t]);
        rr = fma(Kx[at(x - 1, y, z)], u[at(x - 1, y, z)], rr);
        rr = fma(Kx[t], u[at(x + 1, y, z)], rr);
        rr = fma(Ky[at(x, y - 1, z)], u[at(x, y - 1, z)], rr);
        rr = fma(Ky[t], u[at(x, y + 1, z)], rr);
        rr = fma(kzm, um, rr);
        rr = fma(kzp, up, rr);
        sq += (double)rr * (double)rr;
        um = uc;
        uc = up;
        kzm = kzp;
      }
    }
  }
  const double bs = block_sum<128>(sq);
  if (threadIdx.x == 0) partial[(size_t)s * nb + b] = bs;
}

inline dim3 zmarch_grid(int n, int B, int* zslab) {
  const int slabs = apply_slabs(n, zslab);
  return dim3((unsigned)((n * n + 127) / 128), (unsigned)slabs, (unsigned)B);
}

// x += alpha p, r -= alpha q; partials of r.r and r.z (z: the previous preconditioned
// residual); optionally r32 = (float) r for an FP32 preconditioner (SPLIT: in colour-split
// storage). Grid (NB, B).
template <bool SPLIT>
__global__ void __launch_bounds__(kThreads)
    k_cg_update(int n, const double* __restrict__ alpha, const double* __restrict__ p,
                const double* __restrict__ q, double* __restrict__ x, double* __restrict__ r,
                const double* __restrict__ z, float* __restrict__ r32, double* __restrict__ part_rr,
                double* __restrict__ part_rz, const int* __restrict__ active) {
  const int s = blockIdx.y;
  if (!active[s]) return;
  const unsigned n3 = (unsigned)n * n * n;
  const unsigned chunk = (n3 + gridDim.x - 1) / gridDim.x;
  const unsigned lo = blockIdx.x * chunk, hi = lo + chunk < n3 ? lo + chunk : n3;
  const double a = alpha[s];
  double rr = 0.0, rz = 0.0;
  for (unsigned i = lo + threadIdx.x; i < hi; i += kThreads) {
    const size_t t = (size_t)s * n3 + i;
    x[t] = fma(a, p[t], x[t]);
    const double rn = fma(-a, q[t], r[t]);  // q and p vanish on the boundary
    r[t] = rn;
    if (r32) {
      if (SPLIT) {
        const unsigned zq = i / (unsigned)(n * n), rem = i - zq * (unsigned)(n * n), yq = rem / (unsigned)n;
        r32[(size_t)s * split_elems(n) + split_index(n, (int)(rem - yq * (unsigned)n), (int)yq, (int)zq)] = (float)rn;
      } else {
        r32[t] = (float)rn;
      }
    }
    rr = fma(rn, rn, rr);
    rz = fma(rn, z[t], rz);
  }
  const double b1 = block_sum<kThreads>(rr);
  if (threadIdx.x == 0) part_rr[(size_t)s * gridDim.x + blockIdx.x] = b1;
  const double b2 = block_sum<kThreads>(rz);
  if (threadIdx.x == 0) part_rz[(size_t)s * gridDim.x + blockIdx.x] = b2;
}

// z = (double) e (when e32 is given; SPLIT: in colour-split storage) and partial sums of
// r.z. Grid (NB, B).
template <bool SPLIT>
__global__ void __launch_bounds__(kThreads)
    k_precond_dot(int n, const float* __restrict__ e32, double* __restrict__ z, const double* __restrict__ r,
                  double* __restrict__ partial, const int* __restrict__ active) {
  const int s = blockIdx.y;
  if (!active[s]) return;
  const unsigned n3 = (unsigned)n * n * n;
  const unsigned chunk = (n3 + gridDim.x - 1) / gridDim.x;
  const unsigned lo = blockIdx.x * chunk, hi = lo + chunk < n3 ? lo + chunk : n3;
  double acc = 0.0;
  for (unsigned i = lo + threadIdx.x; i < hi; i += kThreads) {
    const size_t t = (size_t)s * n3 + i;
    double zv;
    if (e32) {
      if (SPLIT) {
        const unsigned zq = i / (unsigned)(n * n), rem = i - zq * (unsigned)(n * n), yq = rem / (unsigned)n;
        zv = widen(e32[(size_t)s * split_elems(n) + split_index(n, (int)(rem - yq * (unsigned)n), (int)yq, (int)zq)]);
      } else {
        zv = widen(e32[t]);
      }
      z[t] = zv;
    } else {
      zv = z[t];
    }
    acc = fma(r[t], zv, acc);
  }
  const double b = block_sum<kThreads>(acc);
  if (threadIdx.x == 0) partial[(size_t)s * gridDim.x + blockIdx.x] = b;
}

// p = z + beta p (beta = 0: p = z).
__global__ void k_p_update(int n, int B, const double* __restrict__ beta, const double* __restrict__ z,
                           double* __restrict__ p, const int* __restrict__ active) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // node of the plane
  if (q >= n * n) return;
  const size_t n3 = (size_t)n * n * n;
  for (int zz = blockIdx.y; zz < B * n; zz += gridDim.y) {
    const int s = zz / n, zp = zz - s * n;
    if (!active[s]) continue;
    const size_t t = (size_t)s * n3 + (size_t)(zp * n * n + q);
    p[t] = beta ? fma(beta[s], p[t], z[t]) : z[t];
  }
}

__global__ void k_to_f32(size_t total, const double* __restrict__ a, float* __restrict__ b) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x)
    b[t] = (float)a[t];
}

// b = (float) a, a in the plain layout, b in colour-split storage (plane launch).
__global__ void k_to_f32_split(int n, int B, const double* __restrict__ a, float* __restrict__ b) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // node of the plane
  if (q >= n * n) return;
  const int y = q / n, x = q - y * n;
  const size_t n3 = (size_t)n * n * n, ns = split_elems(n);
  for (int zz = blockIdx.y; zz < B * n; zz += gridDim.y) {
    const int s = zz / n, z = zz - s * n;
    b[(size_t)s * ns + split_index(n, x, y, z)] = (float)a[(size_t)s * n3 + (size_t)(z * n * n + q)];
  }
}

// Per-sample CG scalars from block partials (fixed order).
//   mode 0: rz = sum(part)                         (after the first preconditioning)
//   mode 1: alpha = rz / sum(part)                 (part = p.q)
//   mode 2: beta = (sum(part) - rzo) / rz, rz = sum (part = r.z_new; flexible beta)
//   mode 3: rzo = sum(part)                        (part = r_new.z_old)
__global__ void k_cg_scalar(int B, int NB, int mode, const double* __restrict__ part, double* __restrict__ rz,
                            double* __restrict__ rzo, double* __restrict__ alpha, double* __restrict__ beta,
                            const int* __restrict__ active) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // one warp per sample
  if (s >= B || !active[s]) return;
  const double t = warp_sum_partials(part + (size_t)s * NB, NB);
  if ((threadIdx.x & 31) != 0) return;
  if (mode == 0) {
    rz[s] = t;
  } else if (mode == 1) {
    alpha[s] = t != 0.0 ? rz[s] / t : 0.0;
  } else if (mode == 2) {
    beta[s] = rz[s] != 0.0 ? (t - rzo[s]) / rz[s] : 0.0;
    rz[s] = t;
  } else {
    rzo[s] = t;
  }
}

// ---------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------
template <typename T>
struct Level {
  int n = 0;
  size_t n3 = 0;
  T *Kx = nullptr, *Ky = nullptr, *Kz = nullptr, *D = nullptr, *Dinv = nullptr;
  T *u = nullptr, *g = nullptr, *r = nullptr;
  T* u2 = nullptr;  // spare iterate for the fused (double-buffered) sweep
  T* kn = nullptr;  // reciprocal nodal coefficient 1/k (FP32 grids: input of the nodal sweep)
};

template <typename T>
struct Hier {
  int L = 0, B = 0;
  Level<T> lv[kMaxLevels];
  double* Ainv = nullptr;
  double* Lws = nullptr;
  // level-0 FP64 state
  double* g64 = nullptr;   // h^2 f
  double* D64 = nullptr;   // mixed: FP64 diagonal of the FP64 faces
  double *K64x = nullptr, *K64y = nullptr, *K64z = nullptr;  // mixed: FP64 faces of the finest grid
  int n_act = 0;           // host copy of the number of active samples (launch accounting)
  double* partial = nullptr;
  double* g2 = nullptr;
  double* relres = nullptr;
  int* cycles = nullptr;
  int* active = nullptr;
  int* n_active = nullptr;
  int* err = nullptr;  // device error word of bounded waits
  int NB = 1;   // partials per sample of the flat-chunk reductions (reduce_blocks)
  int NBz = 1;  // partials per sample of the column z-march kernels (apply_blocks)
  // flexible PCG (FP64 vectors on the finest grid) and per-sample scalars
  double *R = nullptr, *P = nullptr, *Q = nullptr, *Z = nullptr;
  double *part2 = nullptr, *rz = nullptr, *rzo = nullptr, *alpha = nullptr, *beta = nullptr;
  double* part_apply = nullptr;  // partials of p.q (k_apply_dot_z's partition)
  int tile[kMaxLevels] = {};      // fused-sweep tile shape per level
  bool fused[kMaxLevels] = {};    // fused (one pass) or two-pass smoother per level
  bool nodal[kMaxLevels] = {};    // two-pass sweep on the nodal coefficient (FP32)
  bool p1 = false;                // P1 finite elements: P1 transfers instead of FW / trilinear
  bool split = false;             // FP32 hierarchy in colour-split storage (MLMC_SMOOTH_SPLIT)
};

// Lays out the workspace. Level-0 u of FP64 solves is the caller's array (not carved).
template <typename T>
void layout(Hier<T>& H, Carver& c, int B, int n, bool mixed, bool cg) {
  H.B = B;
  H.L = hierarchy_depth(n);
  int nl = n;
  for (int j = 0; j < H.L; ++j) {
    Level<T>& v = H.lv[j];
    v.n = nl;
    v.n3 = cube(nl);
    const size_t e = (size_t)B * v.n3;
    // room for the colour-split storage (2 n^2 P instead of n^3 elements per sample, P =
    // (n + 1) / 2 rounded up to a multiple of 4) where a solve may take it: u, g, r and 1/k
    // of FP32 correction cycles; every array of FP64 stationary cycles (not of CG)
    const bool split64 = !mixed && !cg;
    const size_t es = (size_t)B * split_elems(nl);
    const size_t ef = split64 ? es : e, eu = (mixed || split64) ? es : e;
    v.Kx = c.template take<T>(ef);
    v.Ky = c.template take<T>(ef);
    v.Kz = c.template take<T>(ef);
    v.D = c.template take<T>(ef);
    v.Dinv = c.template take<T>(ef);
    // level 0 of an FP64 solve iterates in a copy of the caller's u (so that every array
    // the smoothers stage is carved here, with slack behind it); its g is g64 (or R for CG),
    // or the colour-split copy of g64 (MLMC_SMOOTH_SPLIT)
    v.u = c.template take<T>(eu);
    if (j > 0 || mixed || split64) v.g = c.template take<T>(eu);
    if (j < H.L - 1) v.u2 = c.template take<T>(e);
    if (j < H.L - 1) v.r = c.template take<T>(eu);
    if (mixed && j < H.L - 1) v.kn = c.template take<T>(es);
    nl = (nl + 1) / 2;
  }
  const size_t e0 = (size_t)B * cube(n);
  H.g64 = c.template take<double>(e0);
  if (mixed) {
    H.D64 = c.template take<double>(e0);
    H.K64x = c.template take<double>(e0);
    H.K64y = c.template take<double>(e0);
    H.K64z = c.template take<double>(e0);
  }
  H.Ainv = c.template take<double>((size_t)B * 729);
  H.Lws = c.template take<double>((size_t)B * 729);
  H.NB = reduce_blocks(cube(n));
  H.NBz = apply_blocks(n);
  H.partial = c.template take<double>((size_t)B * (H.NB > H.NBz ? H.NB : H.NBz));
  H.g2 = c.template take<double>(B);
  H.relres = c.template take<double>(B);
  H.cycles = c.template take<int>(B);
  H.active = c.template take<int>(B);
  H.n_active = c.template take<int>(1);
  H.err = c.template take<int>(1);
  if (cg) {
    H.R = c.template take<double>(e0);
    H.P = c.template take<double>(e0);
    H.Q = c.template take<double>(e0);
    if (mixed) H.Z = c.template take<double>(e0);
    H.part2 = c.template take<double>((size_t)B * H.NB);
    H.part_apply = c.template take<double>((size_t)B * apply_blocks(n));
    H.rz = c.template take<double>(B);
    H.rzo = c.template take<double>(B);
    H.alpha = c.template take<double>(B);
    H.beta = c.template take<double>(B);
  }
}

template <typename T>
struct Names;
template <>
struct Names<double> {
  static constexpr const char* rbgs = "rbgs_f64";
  static constexpr const char* residual = "residual_f64";
  static constexpr const char* restrict_ = "restrict_f64";
  static constexpr const char* prolong = "prolong_f64";
  static constexpr const char* faces = "faces_f64";
  static constexpr const char* diag = "diag_f64";
  static constexpr const char* coarse = "coarse_apply_f64";
};
template <>
struct Names<float> {
  static constexpr const char* rbgs = "rbgs_f32";
  static constexpr const char* residual = "residual_f32";
  static constexpr const char* restrict_ = "restrict_f32";
  static constexpr const char* prolong = "prolong_f32";
  static constexpr const char* faces = "faces_f32";
  static constexpr const char* diag = "diag_f32";
  static constexpr const char* coarse = "coarse_apply_f32";
};

inline double interior(int n) { return (double)(n - 2) * (n - 2) * (n - 2); }

template <typename T>
void vcycle(Hier<T>& H, int j, int nu1, int nu2, cudaStream_t st);

// One level of the V-cycle on colour-split FP32 storage: nodal-coefficient colour passes,
// the residual into the plain r, full weighting into the coarse grid's split g, the
// coarser levels, the trilinear correction on split storage, post-smoothing.
template <typename T>
void vcycle_split(Hier<T>& H, int j, int nu1, int nu2, cudaStream_t st) {
  Level<T>& v = H.lv[j];
  Level<T>& w = H.lv[j + 1];
  const int* act = H.active;
  const int B = H.B, m = v.n - 2;
  const double Ba = (double)H.n_act, W = 4.0;
  float* u = (float*)(void*)v.u;
  const float* g = (const float*)(const void*)v.g;
  const float* kn = (const float*)(const void*)v.kn;
  const dim3 gs((unsigned)((m * (split_pitch(v.n) / 4) + 127) / 128), (unsigned)m, (unsigned)B);
  auto smooth = [&](int sweeps) {
    for (int s = 0; s < sweeps; ++s)
      for (int c = 0; c < 2; ++c)
        MLMC_LAUNCH(prof::sized("rbgs_split_f32", v.n), Ba * interior(v.n) * 2.0 * W, Ba * interior(v.n) * 0.5 * 37.0,
                    st, MLMC_SPLIT_DISPATCH(v.n, (k_rbgs_split<LG><<<gs, 128, 0, st>>>(c, kn, g, u, act))));
  };
  smooth(nu1);
  const unsigned groups = (unsigned)((m * (split_pitch(v.n) / 4) + 127) / 128);
  float* r = (float*)(void*)v.r;  // colour-split r~ (room for n^2 (n+1) elements: carved as n^3 + slack)
  MLMC_LAUNCH(prof::sized("residual_split_f32", v.n), Ba * interior(v.n) * 4.0 * W, Ba * interior(v.n) * 37.0, st,
              MLMC_SPLIT_DISPATCH(v.n, (k_residual_split<LG><<<dim3(groups, (unsigned)(2 * m), (unsigned)B), 128, 0,
                                                                st>>>(kn, g, u, r, act))));
  MLMC_LAUNCH(Names<T>::restrict_, Ba * ((double)v.n3 + (double)w.n3) * W, Ba * interior(w.n) * 54.0, st,
              MLMC_SPLIT_DISPATCH(v.n, (k_restrict_split<LG><<<dim3((unsigned)(((w.n - 2) * (w.n - 2) + 127) / 128),
                                                                    (unsigned)(w.n - 2), (unsigned)B), 128, 0, st>>>(
                                                r, (float*)(void*)w.g, act))));
  cudaMemsetAsync(w.u, 0, (size_t)B * split_elems(w.n) * sizeof(T), st);
  vcycle(H, j + 1, nu1, nu2, st);
  MLMC_LAUNCH(prof::sized("prolong_split_f32", v.n), Ba * (2.0 * (double)v.n3 + (double)w.n3) * W,
              Ba * interior(v.n) * 4.375, st,
              MLMC_SPLIT_DISPATCH(v.n, (k_prolong_split<LG><<<dim3(groups, (unsigned)m, (unsigned)(2 * B)), 128, 0,
                                                               st>>>((const float*)(const void*)w.u, u, act))));
  smooth(nu2);
}

// One level of the V-cycle on colour-split FP64 storage (stored faces): two-pass colour
// sweeps, the residual into split r, full weighting into the coarse split g, the coarser
// levels, the trilinear correction on split storage, post-smoothing.
template <typename T>
void vcycle_split64(Hier<T>& H, int j, int nu1, int nu2, cudaStream_t st) {
  Level<T>& v = H.lv[j];
  Level<T>& w = H.lv[j + 1];
  const int* act = H.active;
  const int B = H.B, m = v.n - 2;
  const double Ba = (double)H.n_act, W = 8.0;
  const double* Kx = (const double*)(const void*)v.Kx;
  const double* Ky = (const double*)(const void*)v.Ky;
  const double* Kz = (const double*)(const void*)v.Kz;
  const double* D = (const double*)(const void*)v.D;
  const double* Dinv = (const double*)(const void*)v.Dinv;
  const double* g = (const double*)(const void*)v.g;
  double* u = (double*)(void*)v.u;
  double* r = (double*)(void*)v.r;
  const unsigned pairs = (unsigned)((m * (split_pitch(v.n) / 2) + 127) / 128);
  auto smooth = [&](int sweeps) {
    for (int s = 0; s < sweeps; ++s)
      for (int c = 0; c < 2; ++c)
        MLMC_LAUNCH(prof::sized("rbgs_split_f64", v.n), Ba * interior(v.n) * 3.5 * W, Ba * interior(v.n) * 0.5 * 13.0,
                    st, MLMC_SPLIT_DISPATCH(v.n, (k_rbgs_split64<LG><<<dim3(pairs, (unsigned)m, (unsigned)B), 128, 0,
                                                                         st>>>(c, Kx, Ky, Kz, Dinv, g, u, act))));
  };
  smooth(nu1);
  MLMC_LAUNCH(prof::sized("residual_split_f64", v.n), Ba * interior(v.n) * 7.0 * W, Ba * interior(v.n) * 14.0, st,
              MLMC_SPLIT_DISPATCH(v.n, (k_residual_split64<LG><<<dim3(pairs, (unsigned)(2 * m), (unsigned)B), 128, 0,
                                                                  st>>>(Kx, Ky, Kz, D, g, u, r, act))));
  if (H.p1)
    MLMC_LAUNCH("restrict_p1", Ba * ((double)v.n3 + (double)w.n3) * W, Ba * interior(w.n) * 16.0, st,
                (k_restrict_p1<double, true><<<plane_grid((w.n - 2) * (w.n - 2), (long long)B * (w.n - 2)),
                                               kPlaneThreads, 0, st>>>(v.n, B, r, (double*)(void*)w.g, act)));
  else
    MLMC_LAUNCH(Names<T>::restrict_, Ba * ((double)v.n3 + (double)w.n3) * W, Ba * interior(w.n) * 54.0, st,
                MLMC_SPLIT_DISPATCH(v.n, (k_restrict_split<LG, double><<<dim3((unsigned)(((w.n - 2) * (w.n - 2) +
                                                                                       127) / 128),
                                                                              (unsigned)(w.n - 2), (unsigned)B),
                                                                         128, 0, st>>>(r, (double*)(void*)w.g,
                                                                                       act))));
  cudaMemsetAsync(w.u, 0, (size_t)B * split_elems(w.n) * sizeof(T), st);
  vcycle(H, j + 1, nu1, nu2, st);
  if (H.p1) {
    MLMC_LAUNCH("prolong_p1", Ba * (2.0 * (double)v.n3 + (double)w.n3) * W, Ba * interior(v.n) * 1.5, st,
                (k_prolong_p1<double, true><<<plane_grid(m * m, (long long)B * m), kPlaneThreads, 0, st>>>(
                    v.n, B, (const double*)(const void*)w.u, u, act)));
    smooth(nu2);
    return;
  }
  MLMC_LAUNCH(prof::sized("prolong_split_f64", v.n), Ba * (2.0 * (double)v.n3 + (double)w.n3) * W,
              Ba * interior(v.n) * 4.375, st,
              MLMC_SPLIT_DISPATCH(v.n, (k_prolong_blk_split<LG, double><<<dim3((unsigned)(((w.n - 1) * (w.n - 1) +
                                                                                          127) / 128),
                                                                                (unsigned)(w.n - 1), (unsigned)B),
                                                                           128, 0, st>>>(
                                           (const double*)(const void*)w.u, u, act))));
  smooth(nu2);
}

template <typename T>
void vcycle(Hier<T>& H, int j, int nu1, int nu2, cudaStream_t st) {
  Level<T>& v = H.lv[j];
  const int* act = H.active;
  const int B = H.B;
  // launches cover all B samples; masked (finished) samples do no work, so the
  // algorithmic bytes and flops count the active ones only
  const double Ba = (double)H.n_act;
  const double W = (double)sizeof(T);
  if (j == H.L - 1) {
    if (H.split)
      MLMC_LAUNCH(Names<T>::coarse, Ba * (729.0 * 8 + 54 * W), Ba * 27 * 54.0, st,
                  (k_coarse_apply<T, true><<<(B * 27 + 127) / 128, 128, 0, st>>>(B, H.Ainv, v.g, v.u, act)));
    else
      MLMC_LAUNCH(Names<T>::coarse, Ba * (729.0 * 8 + 54 * W), Ba * 27 * 54.0, st,
                  (k_coarse_apply<T><<<(B * 27 + 127) / 128, 128, 0, st>>>(B, H.Ainv, v.g, v.u, act)));
    return;
  }
  if (H.split) {
    if constexpr (sizeof(T) == 4)
      vcycle_split(H, j, nu1, nu2, st);
    else
      vcycle_split64(H, j, nu1, nu2, st);
    return;
  }
  const int m = v.n - 2;
  const dim3 gs = plane_grid(m * ((v.n - 1) / 2), (long long)B * m);
  // one colour: half of the 7 words per node of a full sweep; 13 flops per updated node
  const double sweep_bytes = Ba * interior(v.n) * 3.5 * W, sweep_flops = Ba * interior(v.n) * 0.5 * 13.0;
  auto smooth = [&](int sweeps) {
    for (int s = 0; s < sweeps; ++s) {
      if constexpr (sizeof(T) == 4) {
        if (H.nodal[j]) {
          for (int c = 0; c < 2; ++c)
            MLMC_LAUNCH(prof::sized("rbgs_nodal_f32", v.n), Ba * interior(v.n) * 2.0 * W, Ba * interior(v.n) * 0.5 * 37.0, st,
                        (k_rbgs_nodal<<<gs, kPlaneThreads, 0, st>>>(c, v.n, B, (const float*)v.kn,
                                                                   (const float*)v.g, (float*)v.u, act)));
          continue;
        }
      }
      if (H.fused[j]) {
        rbgs_fused_sweep<T>(H.tile[j], v.n, B, v.Kx, v.Ky, v.Kz, v.Dinv, v.g, v.u, v.u2, act, H.err, st, Ba);
        T* t = v.u;
        v.u = v.u2;
        v.u2 = t;
      } else {
        for (int c = 0; c < 2; ++c)
          MLMC_LAUNCH(prof::sized(Names<T>::rbgs, v.n), sweep_bytes, sweep_flops, st,
                      (k_rbgs<T><<<gs, kPlaneThreads, 0, st>>>(c, v.n, B, v.Kx, v.Ky, v.Kz, v.Dinv, v.g, v.u, act)));
      }
    }
  };
  smooth(nu1);
  bool nodal_res = false;
  if constexpr (sizeof(T) == 4) {
    if (H.nodal[j]) {
      MLMC_LAUNCH(prof::sized("residual_nodal_f32", v.n), Ba * interior(v.n) * 4.0 * W, Ba * interior(v.n) * 37.0, st,
                  (k_residual_nodal<<<plane_grid(v.n * v.n, (long long)B * v.n), kPlaneThreads, 0, st>>>(
                      v.n, B, (const float*)v.kn, (const float*)v.g, (const float*)v.u, (float*)v.r, act)));
      nodal_res = true;
    }
  }
  if (!nodal_res) {
    int zs = 0;
    const dim3 rz = zmarch_grid(v.n, B, &zs);
    MLMC_LAUNCH(prof::sized(Names<T>::residual, v.n), Ba * interior(v.n) * 7.0 * W, Ba * interior(v.n) * 14.0, st,
                (k_residual_z<T, T, T, T><<<rz, 128, 0, st>>>(v.n, zs, v.Kx, v.Ky, v.Kz, v.D, v.g, v.u, v.r, nullptr,
                                                              act)));
  }
  Level<T>& w = H.lv[j + 1];
  if (H.p1)
    MLMC_LAUNCH("restrict_p1", Ba * ((double)v.n3 + (double)w.n3) * W, Ba * interior(w.n) * 16.0, st,
                (k_restrict_p1<T><<<plane_grid((w.n - 2) * (w.n - 2), (long long)B * (w.n - 2)), kPlaneThreads, 0,
                                    st>>>(v.n, B, v.r, w.g, act)));
  else
    MLMC_LAUNCH(Names<T>::restrict_, Ba * ((double)v.n3 + (double)w.n3) * W, Ba * interior(w.n) * 54.0, st,
                (k_restrict<T><<<plane_grid((w.n - 2) * (w.n - 1), (long long)B * (w.n - 2)), kPlaneThreads, 0,
                                 st>>>(v.n, B, v.r, w.g, act)));
  cudaMemsetAsync(w.u, 0, (size_t)B * w.n3 * sizeof(T), st);
  vcycle(H, j + 1, nu1, nu2, st);
  if (H.p1)
    MLMC_LAUNCH("prolong_p1", Ba * (2.0 * (double)v.n3 + (double)w.n3) * W, Ba * interior(v.n) * 1.5, st,
                (k_prolong_p1<T><<<plane_grid(m * m, (long long)B * m), kPlaneThreads, 0, st>>>(v.n, B, w.u, v.u,
                                                                                               act)));
  else
    MLMC_LAUNCH(Names<T>::prolong, Ba * (2.0 * (double)v.n3 + (double)w.n3) * W, Ba * interior(v.n) * 4.375, st,
                (k_prolong_blk<T><<<plane_grid((w.n - 1) * (w.n - 1), (long long)B * (w.n - 1)), 128, 0, st>>>(
                    v.n, B, w.u, v.u, act)));
  smooth(nu2);
}

// Runs one V-cycle, as a CUDA graph when enabled: the first call captures the cycle's
// launches (counted by the launch tape on every replay), later calls replay it.
inline bool graphs_allowed() {
  static const bool off = [] {
    const char* e = getenv("MLMC_NO_GRAPHS");
    return e && e[0] == '1';
  }();
  return !off;
}

inline bool fmg_graphs() {
  static const bool on = [] {
    const char* e = getenv("MLMC_FMG_GRAPHS");
    return e && e[0] == '1';
  }();
  return on;
}

template <typename T>
struct GraphRunner {
  bool enabled = false;
  cudaGraphExec_t exec = nullptr;
  prof::Tape tape;
  int cap_act = 1;  // active samples when the cycle was captured (its tape's accounting)
  ~GraphRunner() {
    if (exec) cudaGraphExecDestroy(exec);
  }
  // one V-cycle from grid j0 (the same j0 on every call of one runner)
  int run(Hier<T>& H, int nu1, int nu2, cudaStream_t st, int j0 = 0) {
    if (!enabled) {
      vcycle<T>(H, j0, nu1, nu2, st);
      return MLMC_OK;
    }
    if (!exec) {
      MLMC_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      prof::tape_begin();
      vcycle<T>(H, j0, nu1, nu2, st);
      tape = prof::tape_end();
      cap_act = H.n_act > 0 ? H.n_act : 1;
      cudaGraph_t graph = nullptr;
      MLMC_CUDA_TRY(cudaStreamEndCapture(st, &graph));
      const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        exec = nullptr;
        set_error("cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
        return MLMC_ERR_CUDA;
      }
    }
    prof::tape_replay(tape, (double)H.n_act / (double)cap_act);
    MLMC_CUDA_TRY(cudaGraphLaunch(exec, st));
    return MLMC_OK;
  }
};

template <typename T>
int pcg_loop(Hier<T>& H, const MGSolveArgs& a, int nu1, int nu2, double rtol, int maxc, cudaStream_t st,
             GraphRunner<T>& gr) {
  const bool mixed = a.cfg.precision == MLMC_PREC_MIXED;
  const int B = H.B, n = a.n;
  Level<T>& l0 = H.lv[0];
  // algorithmic work of the active samples (H.n_act, updated after every convergence test)
  double nodes = H.n_act * interior(n), all = (double)H.n_act * l0.n3;
  auto set_active = [&](int na) {
    H.n_act = na;
    nodes = na * interior(n);
    all = (double)na * l0.n3;
  };
  dim3 rg(H.NB, B);
  const unsigned sb = (B + 3) / 4;  // 128-thread blocks, one warp per sample
  const unsigned g0 = blocks_for((size_t)B * l0.n3, kThreads);
  const dim3 pg = plane_grid(n * n, (long long)B * n);
  int azslab = 0;
  const int aslabs = apply_slabs(n, &azslab), NBa = apply_blocks(n);
  const dim3 ag((unsigned)((n * n + 127) / 128), (unsigned)aslabs, (unsigned)B);
  // the outer operator is FP64 in both precisions: the FP64 faces of the finest grid
  const double* D = mixed ? H.D64 : (const double*)(const void*)l0.D;
  const double* Fx = mixed ? H.K64x : (const double*)(const void*)l0.Kx;
  const double* Fy = mixed ? H.K64y : (const double*)(const void*)l0.Ky;
  const double* Fz = mixed ? H.K64z : (const double*)(const void*)l0.Kz;
  auto sync_count = [&](int* out) -> int {
    MLMC_CUDA_TRY(cudaMemcpyAsync(out, H.n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
    MLMC_CUDA_TRY(cudaStreamSynchronize(st));
    return MLMC_OK;
  };
  // z = M r: one V-cycle from zero on the (FP32 copy of the) residual; partials of r.z
  const size_t u0_elems = H.split ? split_elems(n) : l0.n3;
  auto precondition = [&]() {
    MLMC_CUDA_TRY(cudaMemsetAsync(H.lv[0].u, 0, (size_t)B * u0_elems * sizeof(T), st));
    MLMC_TRY(gr.run(H, nu1, nu2, st));
    double* z = mixed ? H.Z : (double*)(void*)H.lv[0].u;
    const float* e32 = mixed ? (const float*)(const void*)H.lv[0].u : nullptr;
    if (H.split)
      MLMC_LAUNCH("cg_precond_dot", all * 20.0, nodes * 2.0, st,
                  (k_precond_dot<true><<<rg, kThreads, 0, st>>>(n, e32, z, H.R, H.partial, H.active)));
    else
      MLMC_LAUNCH("cg_precond_dot", all * (mixed ? 20.0 : 16.0), nodes * 2.0, st,
                  (k_precond_dot<false><<<rg, kThreads, 0, st>>>(n, e32, z, H.R, H.partial, H.active)));
    return MLMC_OK;
  };
  auto zcur = [&]() -> double* { return mixed ? H.Z : (double*)(void*)H.lv[0].u; };
  // r = g - A x, ||r||
  MLMC_CUDA_TRY(cudaMemsetAsync(H.n_active, 0, sizeof(int), st));
  MLMC_LAUNCH("cg_residual", nodes * (3 * 8.0 + 32), nodes * 16.0, st,
              (k_residual_z<double, double, double, double><<<ag, 128, 0, st>>>(n, azslab, Fx, Fy, Fz, D, H.g64,
                                                                               a.u, H.R, H.partial, H.active)));
  MLMC_LAUNCH("norm_update", B * NBa * 8.0, B * NBa * 1.0, st,
              (k_norm_update<<<sb, 128, 0, st>>>(B, NBa, H.partial, H.g2, H.relres, H.cycles, H.active, 1, 0, rtol,
                                                 maxc, H.n_active)));
  int na = 0;
  MLMC_TRY(sync_count(&na));
  set_active(na);
  if (na == 0) return MLMC_OK;
  if (mixed && H.split)
    MLMC_LAUNCH("to_f32", all * 12.0, 0.0, st,
                (k_to_f32_split<<<pg, kPlaneThreads, 0, st>>>(n, B, H.R, (float*)(void*)l0.g)));
  else if (mixed)
    MLMC_LAUNCH("to_f32", all * 12.0, 0.0, st,
                (k_to_f32<<<g0, kThreads, 0, st>>>((size_t)B * l0.n3, H.R, (float*)(void*)l0.g)));
  MLMC_TRY(precondition());
  MLMC_LAUNCH("cg_scalar", B * H.NB * 8.0, 0.0, st,
              (k_cg_scalar<<<sb, 128, 0, st>>>(B, H.NB, 0, H.partial, H.rz, H.rzo, H.alpha, H.beta, H.active)));
  MLMC_LAUNCH("cg_p_update", all * 16.0, 0.0, st,
              (k_p_update<<<pg, kPlaneThreads, 0, st>>>(n, B, nullptr, zcur(), H.P, H.active)));
  while (true) {
    MLMC_LAUNCH("cg_apply_dot", nodes * (3 * 8.0 + 8 + 16), nodes * 16.0, st,
                (k_apply_dot_z<double, double><<<ag, 128, 0, st>>>(n, azslab, Fx, Fy, Fz, D, H.P, H.Q,
                                                                    H.part_apply, H.active)));
    MLMC_LAUNCH("cg_scalar", B * NBa * 8.0, 0.0, st,
                (k_cg_scalar<<<sb, 128, 0, st>>>(B, NBa, 1, H.part_apply, H.rz, H.rzo, H.alpha, H.beta, H.active)));
    if (H.split)
      MLMC_LAUNCH("cg_update", all * 60.0, nodes * 8.0, st,
                  (k_cg_update<true><<<rg, kThreads, 0, st>>>(n, H.alpha, H.P, H.Q, a.u, H.R, zcur(),
                                                              (float*)(void*)l0.g, H.partial, H.part2, H.active)));
    else
      MLMC_LAUNCH("cg_update", all * (mixed ? 60.0 : 56.0), nodes * 8.0, st,
                  (k_cg_update<false><<<rg, kThreads, 0, st>>>(n, H.alpha, H.P, H.Q, a.u, H.R, zcur(),
                                                               mixed ? (float*)(void*)l0.g : nullptr, H.partial,
                                                               H.part2, H.active)));
    MLMC_LAUNCH("cg_scalar", B * H.NB * 8.0, 0.0, st,
                (k_cg_scalar<<<sb, 128, 0, st>>>(B, H.NB, 3, H.part2, H.rz, H.rzo, H.alpha, H.beta, H.active)));
    MLMC_CUDA_TRY(cudaMemsetAsync(H.n_active, 0, sizeof(int), st));
    MLMC_LAUNCH("norm_update", B * H.NB * 8.0, B * H.NB * 1.0, st,
                (k_norm_update<<<sb, 128, 0, st>>>(B, H.NB, H.partial, H.g2, H.relres, H.cycles, H.active, 1, 1,
                                                   rtol, maxc, H.n_active)));
    MLMC_TRY(sync_count(&na));
    set_active(na);
    if (na == 0) break;
    MLMC_TRY(precondition());
    MLMC_LAUNCH("cg_scalar", B * H.NB * 8.0, 0.0, st,
                (k_cg_scalar<<<sb, 128, 0, st>>>(B, H.NB, 2, H.partial, H.rz, H.rzo, H.alpha, H.beta, H.active)));
    MLMC_LAUNCH("cg_p_update", all * 24.0, nodes * 2.0, st,
                (k_p_update<<<pg, kPlaneThreads, 0, st>>>(n, B, H.beta, zcur(), H.P, H.active)));
  }
  return MLMC_OK;
}

// ---------------------------------------------------------------------------------
// Small-grid engine (MLMC_ENGINE_CTA): one persistent launch runs the whole solve of a
// batch on grids up to 33^3. Each CTA takes the next sample from a device counter and
// runs that sample's cycles to convergence -- V-cycles, convergence tests, and the CG
// recurrences -- with block barriers between the phases instead of kernel launches and
// without host round trips. Every node update uses the operations of the batched
// kernels in their order, and every per-sample sum uses the batched kernels' partition
// (column z-march blocks of 128 threads, flat chunks of 256 threads) and reduction trees,
// so a sample's iterates, cycle count and residuals are bit for bit those of the batched
// path.
// ---------------------------------------------------------------------------------
constexpr int kCtaThreads = 256;
constexpr int kCtaMaxN = 33;

// MLMC_ENGINE_CTA where it applies (finite volumes, stationary cycles, refinement or CG,
// grids up to 33^3); MLMC_ENGINE_AUTO takes it for grids up to 17^3 (measured 1.15-1.4x
// faster than the batched engine at every batch size from 1 to 4096 samples, with 16-20x
// fewer launches); a 33^3 sample is too much work for one CTA (0.45-0.97x).
inline bool cta_engine_chosen(const mg_cfg& c, int n, int B) {
  const bool ok = c.disc == MLMC_DISC_FV && c.accel != MLMC_ACCEL_FMG && n <= kCtaMaxN;
  if (!ok || c.engine == MLMC_ENGINE_BATCHED) return false;
  if (c.engine == MLMC_ENGINE_CTA) return true;
  static const int env = [] {
    const char* e = getenv("MLMC_ENGINE");
    return e ? atoi(e) : 0;
  }();
  if (env == MLMC_ENGINE_BATCHED) return false;
  if (env == MLMC_ENGINE_CTA) return true;
  // measured: 17^3 1.15-1.4x the batched kernels at 1..4096 samples; 33^3 about even at
  // 1024 samples (FP64 stationary: 73.6 against 74.8 ms, 34 against 757 launches) and
  // slower below (256 samples of mixed CG: 31.0 against 24.8 ms; one CTA per sample leaves
  // SMs idle while fewer samples than resident CTAs remain)
  return n <= 17 || (n <= 33 && B >= 1024);
}
constexpr int kCtaMaxPartials = 64;

template <typename T>
struct CtaLevel {
  int n = 0;
  const T *Kx = nullptr, *Ky = nullptr, *Kz = nullptr, *D = nullptr, *Dinv = nullptr;
  const T* kn = nullptr;  // reciprocal nodal coefficient (FP32 nodal sweep), else nullptr
  T *u = nullptr, *g = nullptr, *r = nullptr;
};

enum { kCtaStationary = 0, kCtaRefinement = 1, kCtaCG = 2 };

template <typename T>
struct CtaArgs {
  int L = 0, B = 0, nu1 = 2, nu2 = 2, maxc = 1, mode = 0;
  double rtol = 0.0;
  CtaLevel<T> lv[4];
  const double* Ainv = nullptr;
  // outer FP64 operator (FP64 faces and diagonal of the finest grid), right-hand side, iterate
  const double *Fx = nullptr, *Fy = nullptr, *Fz = nullptr, *D = nullptr, *g64 = nullptr;
  double* x = nullptr;
  double *R = nullptr, *P = nullptr, *Q = nullptr, *Z = nullptr;  // CG vectors (Z: mixed only)
  const double* g2 = nullptr;
  double* relres = nullptr;
  int *cycles = nullptr, *active = nullptr, *work = nullptr;
  int NB = 1, zslab = 1, slabs = 1;  // flat-chunk partials per sample; column z-march geometry
};

// block_sum<128> of one half of a 256-thread CTA (threads 128 h .. 128 h + 127): the same
// shuffle tree; valid in thread 128 h. Both halves must call it together.
__device__ __forceinline__ double half_block_sum128(double v, double* warp_part8) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, h = threadIdx.x >> 7;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) warp_part8[wid] = v;
  __syncthreads();
  double r = 0.0;
  if ((wid & 3) == 0) {
    r = lane < 4 ? warp_part8[4 * h + lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;
}

template <typename T>
__device__ void cta_smooth(const CtaLevel<T>& v, int s, int colour) {
  const int n = v.n, m = n - 2, half = (n - 1) / 2, lh = 31 - __clz(half), per = m * half;
  const size_t n3 = (size_t)n * n * n, n2 = (size_t)n * n;
  for (int it = threadIdx.x; it < per * m; it += blockDim.x) {
    const int zi = it / per, q = it - zi * per;
    const int xi = q & (half - 1), y = 1 + (q >> lh), z = 1 + zi;
    const int x = (((1 + y + z) & 1) == colour ? 1 : 2) + 2 * xi;
    if (x > n - 2) continue;
    const size_t p = (size_t)s * n3 + (size_t)(z * n * n + y * n + x);
    if constexpr (sizeof(T) == 4) {
      if (v.kn) {
        const float* kn = (const float*)v.kn;
        float* u = (float*)v.u;
        const float kc = kn[p];
        const float kxm = nodal_face(kn[p - 1], kc), kxp = nodal_face(kc, kn[p + 1]);
        const float kym = nodal_face(kn[p - n], kc), kyp = nodal_face(kc, kn[p + n]);
        const float kzm = nodal_face(kn[p - n2], kc), kzp = nodal_face(kc, kn[p + n2]);
        float d = kxm;
        d += kxp;
        d += kym;
        d += kyp;
        d += kzm;
        d += kzp;
        const float dinv = __fdividef(1.0f, d);
        float acc = ((const float*)v.g)[p];
        acc = fmaf(kxm, u[p - 1], acc);
        acc = fmaf(kxp, u[p + 1], acc);
        acc = fmaf(kym, u[p - n], acc);
        acc = fmaf(kyp, u[p + n], acc);
        acc = fmaf(kzm, u[p - n2], acc);
        acc = fmaf(kzp, u[p + n2], acc);
        u[p] = acc * dinv;
        continue;
      }
    }
    T* u = v.u;
    T acc = v.g[p];
    acc = fma(v.Kx[p - 1], u[p - 1], acc);
    acc = fma(v.Kx[p], u[p + 1], acc);
    acc = fma(v.Ky[p - n], u[p - n], acc);
    acc = fma(v.Ky[p], u[p + n], acc);
    acc = fma(v.Kz[p - n2], u[p - n2], acc);
    acc = fma(v.Kz[p], u[p + n2], acc);
    u[p] = acc * v.Dinv[p];
  }
}

// in-cycle residual r~ (k_residual_z / k_residual_nodal operations), 0 on the boundary
template <typename T>
__device__ void cta_residual(const CtaLevel<T>& v, int s) {
  const int n = v.n;
  const size_t n3 = (size_t)n * n * n, n2 = (size_t)n * n;
  for (int i = threadIdx.x; i < (int)n3; i += blockDim.x) {
    const int z = i / (n * n), rem = i - z * n * n, y = rem / n, x = rem - y * n;
    const size_t p = (size_t)s * n3 + (size_t)i;
    T rr = T(0);
    if (x > 0 && y > 0 && z > 0 && x < n - 1 && y < n - 1 && z < n - 1) {
      bool done = false;
      if constexpr (sizeof(T) == 4) {
        if (v.kn) {
          const float* kn = (const float*)v.kn;
          const float* u = (const float*)v.u;
          const float kc = kn[p];
          const float kxm = nodal_face(kn[p - 1], kc), kxp = nodal_face(kc, kn[p + 1]);
          const float kym = nodal_face(kn[p - n], kc), kyp = nodal_face(kc, kn[p + n]);
          const float kzm = nodal_face(kn[p - n2], kc), kzp = nodal_face(kc, kn[p + n2]);
          float d = kxm;
          d += kxp;
          d += kym;
          d += kyp;
          d += kzm;
          d += kzp;
          float q = fmaf(-d, u[p], ((const float*)v.g)[p]);
          q = fmaf(kxm, u[p - 1], q);
          q = fmaf(kxp, u[p + 1], q);
          q = fmaf(kym, u[p - n], q);
          q = fmaf(kyp, u[p + n], q);
          q = fmaf(kzm, u[p - n2], q);
          q = fmaf(kzp, u[p + n2], q);
          rr = (T)q;
          done = true;
        }
      }
      if (!done) {
        const T* u = v.u;
        rr = fma(-v.D[p], u[p], v.g[p]);
        rr = fma(v.Kx[p - 1], u[p - 1], rr);
        rr = fma(v.Kx[p], u[p + 1], rr);
        rr = fma(v.Ky[p - n], u[p - n], rr);
        rr = fma(v.Ky[p], u[p + n], rr);
        rr = fma(v.Kz[p - n2], u[p - n2], rr);
        rr = fma(v.Kz[p], u[p + n2], rr);
      }
    }
    v.r[p] = rr;
  }
}

// g_c = 4 FW(r~) at interior coarse nodes and u_c = 0 (k_restrict's operations)
template <typename T>
__device__ void cta_restrict(const CtaLevel<T>& v, const CtaLevel<T>& w, int s) {
  const int nf = v.n, nc = w.n, mc = nc - 2;
  const size_t nf3 = (size_t)nf * nf * nf, nc3 = (size_t)nc * nc * nc;
  const int nf2 = nf * nf;
  for (int i = threadIdx.x; i < (int)nc3; i += blockDim.x) w.u[(size_t)s * nc3 + i] = T(0);
  for (int i = threadIdx.x; i < mc * mc * mc; i += blockDim.x) {
    const int Z = 1 + i / (mc * mc), rem = i - (Z - 1) * mc * mc, Y = 1 + rem / mc, X = 1 + rem - (Y - 1) * mc;
    const T* rb = v.r + (size_t)s * nf3 + (size_t)(2 * Z * nf2 + 2 * Y * nf + 2 * X);
    T acc = 0;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const T wgt = (T)((2 - abs(dx)) * (2 - abs(dy)) * (2 - abs(dz))) * (T)(1.0 / 16.0);
          acc = fma(wgt, rb[dz * nf2 + dy * nf + dx], acc);
        }
    w.g[(size_t)s * nc3 + (size_t)((Z * nc + Y) * nc + X)] = acc;
  }
}

// u_f += trilinear interpolation of e_c (k_prolong's operations)
template <typename T>
__device__ void cta_prolong(const CtaLevel<T>& w, const CtaLevel<T>& v, int s) {
  // one coarse cell per thread (k_prolong_blk's sums, bit for bit k_prolong's)
  const int nf = v.n, nc = w.n, mc = nc - 1;
  const size_t nf3 = (size_t)nf * nf * nf, nc3 = (size_t)nc * nc * nc, nc2 = (size_t)nc * nc;
  for (int i = threadIdx.x; i < mc * mc * mc; i += blockDim.x) {
    const int Z = i / (mc * mc), rem = i - Z * mc * mc, Y = rem / mc, X = rem - Y * mc;
    const T* e = w.u + (size_t)s * nc3 + (size_t)((Z * nc + Y) * nc + X);
    const T c[8] = {e[0], e[1], e[nc], e[nc + 1], e[nc2], e[nc2 + 1], e[nc2 + nc], e[nc2 + nc + 1]};
    T val[8];
    prolong_block_sums(c, val);
    T* ub = v.u + (size_t)s * nf3;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int dx = k & 1, dy = (k >> 1) & 1, dz = k >> 2;
      const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
      if (x < 1 || y < 1 || z < 1 || x > nf - 2 || y > nf - 2 || z > nf - 2) continue;
      const T wgt = dx + dy + dz == 0 ? T(1) : dx + dy + dz == 1 ? T(0.5) : dx + dy + dz == 2 ? T(0.25) : T(0.125);
      ub[(size_t)((z * nf + y) * nf + x)] += wgt * val[k];
    }
  }
}

template <typename T>
__device__ void cta_vcycle(const CtaArgs<T>& A, int s) {
  // down: smoothing, residual, restriction
  for (int j = 0; j < A.L - 1; ++j) {
    for (int k = 0; k < A.nu1; ++k)
      for (int c = 0; c < 2; ++c) {
        cta_smooth(A.lv[j], s, c);
        __syncthreads();
      }
    cta_residual(A.lv[j], s);
    __syncthreads();
    cta_restrict(A.lv[j], A.lv[j + 1], s);
    __syncthreads();
  }
  // exact solve on the 5^3 grid (k_coarse_apply)
  {
    const CtaLevel<T>& v = A.lv[A.L - 1];
    const int i = threadIdx.x;
    if (i < 27) {
      const double* X = A.Ainv + (size_t)s * 729 + (size_t)i * 27;
      const size_t base = (size_t)s * 125;
      double val = 0.0;
      for (int q = 0; q < 27; ++q) {
        const int x = 1 + q % 3, y = 1 + (q / 3) % 3, z = 1 + q / 9;
        val = fma(X[q], (double)v.g[base + (z * 5 + y) * 5 + x], val);
      }
      const int x = 1 + i % 3, y = 1 + (i / 3) % 3, z = 1 + i / 9;
      v.u[base + (z * 5 + y) * 5 + x] = (T)val;
    }
    __syncthreads();
  }
  // up: correction, smoothing
  for (int j = A.L - 2; j >= 0; --j) {
    cta_prolong(A.lv[j + 1], A.lv[j], s);
    __syncthreads();
    for (int k = 0; k < A.nu2; ++k)
      for (int c = 0; c < 2; ++c) {
        cta_smooth(A.lv[j], s, c);
        __syncthreads();
      }
  }
}

// Column z-march partials (k_residual_z / k_apply_dot_z partition, 128-thread blocks, two
// per pass of the CTA): APPLY = false: r~ = g - D x + sum K x_q (stored as TR into r when
// r != nullptr) and partials of r~^2; APPLY = true: q = D p - sum K p_q and partials of
// p.q. Returns the total of the partials (k_norm_update / k_cg_scalar's warp tree).
template <bool APPLY, typename TR>
__device__ double cta_zmarch(const double* __restrict__ Fx, const double* __restrict__ Fy,
                             const double* __restrict__ Fz, const double* __restrict__ D,
                             const double* __restrict__ g, const double* __restrict__ x, TR* __restrict__ r, int n,
                             int zslab, int slabs, int s, double* part, double* warp_part8, double* bcast) {
  const int CB = (n * n + 127) / 128, nb = CB * slabs, h = threadIdx.x >> 7, t = threadIdx.x & 127;
  const size_t n2 = (size_t)n * n;
  for (int vb0 = 0; vb0 < nb; vb0 += 2) {
    const int vb = vb0 + h;
    double acc = 0.0;
    if (vb < nb) {
      const int cb = vb % CB, slab = vb / CB;
      const int c = cb * 128 + t;
      const int zlo = 1 + slab * zslab, zhi = min(n - 2, zlo + zslab - 1);
      if (c < n * n) {
        const int y = c / n, xx = c - y * n;
        const size_t col = (size_t)s * n2 * n + c;
        if (xx > 0 && y > 0 && xx < n - 1 && y < n - 1) {
          double pm = x[col + (size_t)(zlo - 1) * n2], pc = x[col + (size_t)zlo * n2];
          double kzm = Fz[col + (size_t)(zlo - 1) * n2];
          for (int z = zlo; z <= zhi; ++z) {
            const size_t p = col + (size_t)z * n2;
            const double pp = x[p + n2];
            const double kzp = Fz[p];
            if (APPLY) {
              double v = D[p] * pc;
              v = fma(-Fx[p - 1], x[p - 1], v);
              v = fma(-Fx[p], x[p + 1], v);
              v = fma(-Fy[p - n], x[p - n], v);
              v = fma(-Fy[p], x[p + n], v);
              v = fma(-kzm, pm, v);
              v = fma(-kzp, pp, v);
              acc = fma(pc, v, acc);
              r[p] = (TR)v;
            } else {
              double rr = fma(-D[p], pc, g[p]);
              rr = fma(Fx[p - 1], x[p - 1], rr);
              rr = fma(Fx[p], x[p + 1], rr);
              rr = fma(Fy[p - n], x[p - n], rr);
              rr = fma(Fy[p], x[p + n], rr);
              rr = fma(kzm, pm, rr);
              rr = fma(kzp, pp, rr);
              if (r) r[p] = (TR)rr;
              acc += rr * rr;
            }
            pm = pc;
            pc = pp;
            kzm = kzp;
          }
        } else if (r) {
          for (int z = zlo; z <= zhi; ++z) r[col + (size_t)z * n2] = TR(0);
        }
        if (r && slab == 0) r[col] = TR(0);
        if (r && slab == slabs - 1) r[col + (size_t)(n - 1) * n2] = TR(0);
      }
    }
    const double bs = half_block_sum128(acc, warp_part8);
    if (t == 0 && vb < nb) part[vb] = bs;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const double tot = warp_sum_partials(part, nb);
    if (threadIdx.x == 0) *bcast = tot;
  }
  __syncthreads();
  return *bcast;
}

// convergence bookkeeping of one sample (k_norm_update, mode 1); returns the active flag
__device__ __forceinline__ int cta_norm_update(double t, double g2, double rtol, int maxc, int inc, double* rel,
                                               int* cyc) {
  *rel = g2 > 0.0 ? sqrt(t / g2) : 0.0;
  *cyc += inc;
  return (rtol > 0.0) ? (*rel > rtol && *cyc < maxc) : (*cyc < maxc);
}

template <typename T>
__global__ void __launch_bounds__(kCtaThreads) k_solve_cta(CtaArgs<T> A) {
  __shared__ double part[kCtaMaxPartials], part2[kCtaMaxPartials], warp_part8[8], bcast[1];
  __shared__ int s_next;
  const int n = A.lv[0].n;
  const size_t n3 = (size_t)n * n * n;
  const unsigned chunk = ((unsigned)n3 + A.NB - 1) / A.NB;
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(A.work, 1);
    __syncthreads();
    const int s = s_next;
    __syncthreads();
    if (s >= A.B) return;
    const double g2 = A.g2[s];
    double rel = 0.0;
    int cyc = 0, act = 0;
    if (A.mode == kCtaStationary) {
      // FP64 V-cycles on the level-0 iterate until the residual test passes
      for (int inc = 0;; inc = 1) {
        const double t = cta_zmarch<false, double>(A.Fx, A.Fy, A.Fz, A.D, A.g64, A.x, (double*)nullptr, n, A.zslab,
                                                   A.slabs, s, part, warp_part8, bcast);
        act = cta_norm_update(t, g2, A.rtol, A.maxc, inc, &rel, &cyc);
        if (!act) break;
        cta_vcycle(A, s);
      }
    } else if (A.mode == kCtaRefinement) {
      // FP32 V-cycles on FP64 residuals: r32 = g - A x, e = V(r32), x += e
      CtaLevel<T>& l0 = A.lv[0];
      for (int inc = 0;; inc = 1) {
        const double t = cta_zmarch<false, T>(A.Fx, A.Fy, A.Fz, A.D, A.g64, A.x, l0.g, n, A.zslab, A.slabs, s, part,
                                              warp_part8, bcast);
        act = cta_norm_update(t, g2, A.rtol, A.maxc, inc, &rel, &cyc);
        if (!act) break;
        for (size_t i = threadIdx.x; i < n3; i += blockDim.x) l0.u[(size_t)s * n3 + i] = T(0);
        __syncthreads();
        cta_vcycle(A, s);
        for (size_t i = threadIdx.x; i < n3; i += blockDim.x) A.x[(size_t)s * n3 + i] += widen(l0.u[(size_t)s * n3 + i]);
        __syncthreads();
      }
    } else {
      // flexible preconditioned CG (pcg_loop's recurrences)
      CtaLevel<T>& l0 = A.lv[0];
      const bool mixed = sizeof(T) == 4;
      double* zv = mixed ? A.Z : (double*)(void*)l0.u;
      const size_t b0 = (size_t)s * n3;
      double rz = 0.0, rzo = 0.0, alpha = 0.0, beta = 0.0;
      // z = M r and the partials of r.z (flat chunks): the preconditioner
      auto precondition = [&]() -> double {
        for (size_t i = threadIdx.x; i < n3; i += blockDim.x) l0.u[b0 + i] = T(0);
        __syncthreads();
        cta_vcycle(A, s);
        for (int b = 0; b < A.NB; ++b) {
          const unsigned lo = b * chunk, hi = lo + chunk < (unsigned)n3 ? lo + chunk : (unsigned)n3;
          double acc = 0.0;
          for (unsigned i = lo + threadIdx.x; i < hi; i += kCtaThreads) {
            const size_t t = b0 + i;
            double z;
            if (mixed) {
              z = widen(((const float*)(const void*)l0.u)[t]);
              zv[t] = z;
            } else {
              z = zv[t];
            }
            acc = fma(A.R[t], z, acc);
          }
          const double bsum = block_sum<kCtaThreads>(acc);
          if (threadIdx.x == 0) part[b] = bsum;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
          const double tot = warp_sum_partials(part, A.NB);
          if (threadIdx.x == 0) *bcast = tot;
        }
        __syncthreads();
        return *bcast;
      };
      const double t0 = cta_zmarch<false, double>(A.Fx, A.Fy, A.Fz, A.D, A.g64, A.x, A.R, n, A.zslab, A.slabs, s,
                                                  part, warp_part8, bcast);
      act = cta_norm_update(t0, g2, A.rtol, A.maxc, 0, &rel, &cyc);
      if (act) {
        if (mixed)
          for (size_t i = threadIdx.x; i < n3; i += blockDim.x) ((float*)(void*)l0.g)[b0 + i] = (float)A.R[b0 + i];
        __syncthreads();
        rz = precondition();
        for (size_t i = threadIdx.x; i < n3; i += blockDim.x) A.P[b0 + i] = zv[b0 + i];
        __syncthreads();
        for (;;) {
          const double pq = cta_zmarch<true, double>(A.Fx, A.Fy, A.Fz, A.D, nullptr, A.P, A.Q, n, A.zslab, A.slabs, s,
                                                     part, warp_part8, bcast);
          alpha = pq != 0.0 ? rz / pq : 0.0;
          // x += alpha p, r -= alpha q; partials of r.r and r.z_old (flat chunks)
          for (int b = 0; b < A.NB; ++b) {
            const unsigned lo = b * chunk, hi = lo + chunk < (unsigned)n3 ? lo + chunk : (unsigned)n3;
            double rr = 0.0, rzp = 0.0;
            for (unsigned i = lo + threadIdx.x; i < hi; i += kCtaThreads) {
              const size_t t = b0 + i;
              A.x[t] = fma(alpha, A.P[t], A.x[t]);
              const double rn = fma(-alpha, A.Q[t], A.R[t]);
              A.R[t] = rn;
              if (mixed) ((float*)(void*)l0.g)[t] = (float)rn;
              rr = fma(rn, rn, rr);
              rzp = fma(rn, zv[t], rzp);
            }
            const double b1 = block_sum<kCtaThreads>(rr);
            if (threadIdx.x == 0) part[b] = b1;
            const double b2 = block_sum<kCtaThreads>(rzp);
            if (threadIdx.x == 0) part2[b] = b2;
          }
          __syncthreads();
          if (threadIdx.x < 32) {
            const double a1 = warp_sum_partials(part2, A.NB);
            const double a2 = warp_sum_partials(part, A.NB);
            if (threadIdx.x == 0) {
              bcast[0] = a1;
              warp_part8[0] = a2;
            }
          }
          __syncthreads();
          rzo = bcast[0];
          const double trr = warp_part8[0];
          __syncthreads();
          act = cta_norm_update(trr, g2, A.rtol, A.maxc, 1, &rel, &cyc);
          if (!act) break;
          const double rzn = precondition();
          beta = rz != 0.0 ? (rzn - rzo) / rz : 0.0;
          rz = rzn;
          for (size_t i = threadIdx.x; i < n3; i += blockDim.x) A.P[b0 + i] = fma(beta, A.P[b0 + i], zv[b0 + i]);
          __syncthreads();
        }
      }
    }
    if (threadIdx.x == 0) {
      A.relres[s] = rel;
      A.cycles[s] = cyc;
      A.active[s] = act;
    }
    __syncthreads();
  }
}

template <typename T>
int solve_impl(const MGSolveArgs& a, void* ws, cudaStream_t st, int* cycles_host, double* relres_host,
               int* n_unconv, int* cycles_dev, double* relres_dev) {
  const bool mixed = a.cfg.precision == MLMC_PREC_MIXED;
  const bool cg = a.cfg.accel == MLMC_ACCEL_CG;
  const bool fmg = a.cfg.accel == MLMC_ACCEL_FMG;
  Hier<T> H;
  Carver c(ws);
  layout<T>(H, c, a.B, a.n, mixed, cg);
  H.p1 = a.cfg.disc == MLMC_DISC_FE;
  const int B = a.B;
  const double W = (double)sizeof(T);
  // the sweep count of the cycle (tuned for the finest grid, or as given) and whether the
  // FP32 hierarchy runs on colour-split storage (the finest grid's smoother decides for
  // every grid)
  int nu1 = a.cfg.nu1, nu2 = a.cfg.nu2;
  // the small-grid engine: one persistent launch for the whole solve (grids up to 33^3)
  const bool use_cta = cta_engine_chosen(a.cfg, a.n, a.B);
  {
    int sm0 = a.cfg.smoother;
    resolve_tuning(a.n, a.cfg.precision, &sm0, &nu1, &nu2);
    // FP32 correction cycles on finite volumes (mixed), or FP64 stationary and FMG cycles
    // on finite volumes or P1 elements (the split kernels are instantiated for n = 5 .. 1025)
    H.split = !use_cta && sm0 == MLMC_SMOOTH_SPLIT && a.n <= 1025 &&
              (mixed ? a.cfg.disc == MLMC_DISC_FV : !cg);
  }
  // operators of every level (k injected from k0); colour-split grids need no faces
  // except on the coarsest grid (its dense solve)
  int stride = a.st0;
  for (int j = 0; j < H.L; ++j) {
    Level<T>& v = H.lv[j];
    const dim3 gb = plane_grid(v.n * v.n, (long long)B * v.n);
    if (H.split) {
      if (j > 0) MLMC_CUDA_TRY(cudaMemsetAsync(v.g, 0, (size_t)B * split_elems(v.n) * sizeof(T), st));
      if (j < H.L - 1) {
        if constexpr (sizeof(T) == 8) {
          // FP64: stored faces, D and 1/D in the split storage (the coarsest grid keeps the
          // plain faces its dense factorisation reads); P1 faces are assembled in the plain
          // layout into the level's spare arrays and copied over
          if (a.cfg.disc == MLMC_DISC_FE) {
            double* t[3] = {(double*)(void*)v.u2, (double*)(void*)v.r, (double*)(void*)v.u};
            MLMC_LAUNCH("faces_fe", B * (double)v.n3 * (8.0 + 3 * W), B * (double)v.n3 * 36.0, st,
                        (k_faces_fe<double><<<gb, kPlaneThreads, 0, st>>>(a.k0, a.n_k0, stride, v.n, B, t[0], t[1],
                                                                          t[2])));
            double* K[3] = {(double*)(void*)v.Kx, (double*)(void*)v.Ky, (double*)(void*)v.Kz};
            for (int d = 0; d < 3; ++d)
              MLMC_LAUNCH("split_copy", B * (double)v.n3 * 16.0, 0.0, st,
                          (k_split_copy<double, true><<<gb, kPlaneThreads, 0, st>>>(v.n, B, t[d], K[d])));
          } else {
            MLMC_LAUNCH(Names<T>::faces, B * (double)v.n3 * (8.0 + 3 * W), B * (double)v.n3 * 12.0, st,
                        (k_faces_split<<<gb, kPlaneThreads, 0, st>>>(a.k0, a.n_k0, stride, v.n, B, (double*)v.Kx,
                                                                      (double*)v.Ky, (double*)v.Kz)));
          }
          MLMC_LAUNCH(Names<T>::diag, B * (double)v.n3 * 5 * W, B * (double)v.n3 * 6.0, st,
                      (k_diag_split<<<gb, kPlaneThreads, 0, st>>>(v.n, B, (const double*)v.Kx, (const double*)v.Ky,
                                                                   (const double*)v.Kz, (double*)v.D,
                                                                   (double*)v.Dinv)));
        }
        stride *= 2;
        continue;
      }
    }
    if (a.cfg.disc == MLMC_DISC_FE)
      MLMC_LAUNCH("faces_fe", B * (double)v.n3 * (8.0 + 3 * W), B * (double)v.n3 * 36.0, st,
                  (k_faces_fe<T><<<gb, kPlaneThreads, 0, st>>>(a.k0, a.n_k0, stride, v.n, B, v.Kx, v.Ky, v.Kz)));
    else
      MLMC_LAUNCH(Names<T>::faces, B * (double)v.n3 * (8.0 + 3 * W), B * (double)v.n3 * 12.0, st,
                  (k_faces<T><<<gb, kPlaneThreads, 0, st>>>(a.k0, a.n_k0, stride, v.n, B, v.Kx, v.Ky, v.Kz)));
    MLMC_LAUNCH(Names<T>::diag, B * (double)v.n3 * 5 * W, B * (double)v.n3 * 6.0, st,
                (k_diag<T, T><<<gb, kPlaneThreads, 0, st>>>(v.n, B, v.Kx, v.Ky, v.Kz, v.D, v.Dinv)));
    // restriction writes only interior coarse nodes: the boundary of g stays zero
    if (j > 0 && !H.split) MLMC_CUDA_TRY(cudaMemsetAsync(v.g, 0, (size_t)B * v.n3 * sizeof(T), st));
    stride *= 2;
  }
  // smoother per level (explicit choice, or the tuned / default one for that grid)
  for (int j = 0; j < H.L; ++j) {
    Level<T>& v = H.lv[j];
    if (H.split) {
      H.nodal[j] = H.fused[j] = false;
      if (mixed && j < H.L - 1)
        MLMC_LAUNCH("nodal_k", B * (double)v.n3 * (8.0 + W), 0.0, st,
                    (k_nodal_k_split<<<plane_grid(v.n * v.n, (long long)B * v.n), kPlaneThreads, 0, st>>>(
                        a.k0, a.n_k0, a.st0 << j, v.n, B, (float*)(void*)v.kn)));
      continue;
    }
    int sm = a.cfg.smoother, d1 = 1, d2 = 1;
    resolve_tuning(v.n, a.cfg.precision, &sm, &d1, &d2);
    if (sm == MLMC_SMOOTH_SPLIT) sm = MLMC_SMOOTH_NODAL;  // split storage only for the whole hierarchy
    // the small-grid engine runs the two-pass arithmetic (bit for bit that of the fused and
    // bulk sweeps) or the nodal one
    if (use_cta && sm != MLMC_SMOOTH_NODAL) sm = MLMC_SMOOTH_TWO_PASS;
    // the nodal-coefficient sweep exists for FP32 grids (an FP64 solve takes the two-pass)
    H.nodal[j] = v.kn != nullptr && sm == MLMC_SMOOTH_NODAL;
    H.fused[j] = v.u2 != nullptr && sm != MLMC_SMOOTH_TWO_PASS && sm != MLMC_SMOOTH_NODAL;
    if (H.nodal[j]) {
      MLMC_LAUNCH("nodal_k", B * (double)v.n3 * (8.0 + W), 0.0, st,
                  (k_nodal_k<T><<<plane_grid(v.n * v.n, (long long)B * v.n), kPlaneThreads, 0, st>>>(
                      a.k0, a.n_k0, a.st0 << j, v.n, B, v.kn)));
    }
    switch (sm) {
      case MLMC_SMOOTH_FUSED_32x16: H.tile[j] = kTile32x16; break;
      case MLMC_SMOOTH_FUSED_64x8: H.tile[j] = kTile64x8; break;
      case MLMC_SMOOTH_BULK_32x8: H.tile[j] = kBulk32x8; break;
      case MLMC_SMOOTH_BULK_32x16: H.tile[j] = kBulk32x16; break;
      case MLMC_SMOOTH_BULK_64x8: H.tile[j] = kBulk64x8; break;
      default: H.tile[j] = kTile32x8;
    }
    if (v.u2) MLMC_CUDA_TRY(cudaMemsetAsync(v.u2, 0, (size_t)B * v.n3 * sizeof(T), st));
    if (H.fused[j]) MLMC_TRY(rbgs_fused_configure<T>(H.tile[j]));
  }
  // The V-cycle as a CUDA graph: captured on the first cycle, replayed on the others.
  // Only when no per-launch events are recorded, the stream can be captured (not the
  // legacy default stream), and every level's double buffer returns to its starting
  // pointer after a cycle (nu1 + nu2 even).
  GraphRunner<T> gr;
  gr.enabled = !prof::timing_enabled() && st != nullptr && ((nu1 + nu2) % 2 == 0) && graphs_allowed();
  Level<T>& l0 = H.lv[0];
  const unsigned g0 = blocks_for((size_t)B * l0.n3, kThreads);
  H.n_act = B;
  if (mixed) {
    // the outer FP64 operator: faces of the FP64 nodal k (not of its FP32 rounding), so
    // that the refinement converges to the FP64 solution
    const dim3 gb0 = plane_grid(l0.n * l0.n, (long long)B * l0.n);
    MLMC_LAUNCH("faces64_mixed", B * (double)l0.n3 * (8.0 + 3 * 8.0), B * (double)l0.n3 * 12.0, st,
                (k_faces<double><<<gb0, kPlaneThreads, 0, st>>>(a.k0, a.n_k0, a.st0, l0.n, B, H.K64x, H.K64y,
                                                               H.K64z)));
    MLMC_LAUNCH("diag64_mixed", B * (double)l0.n3 * (3 * 8.0 + 8), B * (double)l0.n3 * 5.0, st,
                (k_diag<double, double><<<gb0, kPlaneThreads, 0, st>>>(l0.n, B, H.K64x, H.K64y, H.K64z, H.D64,
                                                                      nullptr)));
  }
  Level<T>& lc = H.lv[H.L - 1];
  MLMC_LAUNCH("coarse_setup", B * 2 * 729.0 * 8, B * 40000.0, st,
              (k_coarse_setup<T><<<(B + 3) / 4, 128, 0, st>>>(B, lc.Kx, lc.Ky, lc.Kz, H.Lws, H.Ainv)));
  const double h = 1.0 / (double)(a.n - 1);
  MLMC_LAUNCH("prepare", B * (double)l0.n3 * (a.f ? 16.0 : 8.0), B * (double)l0.n3, st,
              (k_prepare<<<plane_grid(a.n * a.n, (long long)B * a.n), kPlaneThreads, 0, st>>>(a.n, B, h * h, a.f,
                                                                                             H.g64, a.u)));
  if (!mixed && !cg && H.split) {
    // colour-split copies of g = h^2 f and of the initial guess; copied back at the end
    const dim3 pg0 = plane_grid(a.n * a.n, (long long)B * a.n);
    MLMC_LAUNCH("split_copy", B * (double)l0.n3 * 16.0, 0.0, st,
                (k_split_copy<double, true><<<pg0, kPlaneThreads, 0, st>>>(a.n, B, H.g64, (double*)(void*)l0.g)));
    MLMC_LAUNCH("split_copy", B * (double)l0.n3 * 16.0, 0.0, st,
                (k_split_copy<double, true><<<pg0, kPlaneThreads, 0, st>>>(a.n, B, a.u, (double*)(void*)l0.u)));
  } else if (!mixed && !cg) {
    l0.g = (T*)H.g64;
    // iterate in the workspace copy; copied back after the last cycle
    MLMC_CUDA_TRY(cudaMemcpyAsync(l0.u, a.u, (size_t)B * l0.n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  if (!mixed && cg) l0.g = (T*)H.R;  // FP64 CG: the cycle maps R to z (level-0 u)
  dim3 rg(H.NB, B);
  const unsigned sb = (B + 3) / 4;  // 128-thread blocks, one warp per sample
  MLMC_LAUNCH("norm", B * (double)l0.n3 * 8, B * (double)l0.n3 * 2, st,
              (k_sumsq<<<rg, kThreads, 0, st>>>(a.n, H.g64, H.partial)));
  MLMC_LAUNCH("norm_update", B * H.NB * 8.0, B * H.NB * 1.0, st,
              (k_norm_update<<<sb, 128, 0, st>>>(B, H.NB, H.partial, H.g2, nullptr, nullptr, nullptr, 0, 0, 0.0, 0,
                                                 nullptr)));
  MLMC_CUDA_TRY(cudaMemsetAsync(H.cycles, 0, B * sizeof(int), st));
  MLMC_CUDA_TRY(cudaMemsetAsync(H.err, 0, sizeof(int), st));
  {
    // every sample starts active; the first residual decides
    std::vector<int> ones(B, 1);
    MLMC_CUDA_TRY(cudaMemcpyAsync(H.active, ones.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
    MLMC_CUDA_TRY(cudaStreamSynchronize(st));
  }
  const double rtol = a.cfg.rtol;
  const int maxc = a.cfg.max_cycles;
  auto residual_check = [&](int inc) -> int {
    MLMC_CUDA_TRY(cudaMemsetAsync(H.n_active, 0, sizeof(int), st));
    int zs = 0;
    const dim3 rz = zmarch_grid(a.n, B, &zs);
    const double Ba = (double)H.n_act;
    if (mixed && H.split) {
      MLMC_LAUNCH("residual_mixed", Ba * interior(a.n) * (3 * 8.0 + 8 * 3 + W), Ba * interior(a.n) * 16.0, st,
                  (k_residual_z<double, double, double, T, true><<<rz, 128, 0, st>>>(
                      a.n, zs, H.K64x, H.K64y, H.K64z, H.D64, H.g64, a.u, l0.g, H.partial, H.active)));
    } else if (mixed) {
      MLMC_LAUNCH("residual_mixed", Ba * interior(a.n) * (3 * 8.0 + 8 * 3 + W), Ba * interior(a.n) * 16.0, st,
                  (k_residual_z<double, double, double, T><<<rz, 128, 0, st>>>(a.n, zs, H.K64x, H.K64y, H.K64z, H.D64,
                                                                               H.g64, a.u, l0.g, H.partial,
                                                                               H.active)));
    } else if (H.split) {
      MLMC_LAUNCH("residual_norm_f64", Ba * interior(a.n) * 6.0 * 8, Ba * interior(a.n) * 16.0, st,
                  (k_residual_norm_split<<<rz, 128, 0, st>>>(a.n, zs, (const double*)l0.Kx, (const double*)l0.Ky,
                                                             (const double*)l0.Kz, (const double*)l0.D,
                                                             (const double*)l0.g, (const double*)l0.u, H.partial,
                                                             H.active)));
    } else {
      MLMC_LAUNCH("residual_norm_f64", Ba * interior(a.n) * 6.0 * 8, Ba * interior(a.n) * 16.0, st,
                  (k_residual_z<T, T, T, T><<<rz, 128, 0, st>>>(a.n, zs, l0.Kx, l0.Ky, l0.Kz, l0.D, l0.g, l0.u,
                                                                nullptr, H.partial, H.active)));
    }
    MLMC_LAUNCH("norm_update", B * H.NBz * 8.0, B * H.NBz * 1.0, st,
                (k_norm_update<<<sb, 128, 0, st>>>(B, H.NBz, H.partial, H.g2, H.relres, H.cycles, H.active, 1, inc,
                                                   rtol, maxc, H.n_active)));
    int na = 0;
    MLMC_CUDA_TRY(cudaMemcpyAsync(&na, H.n_active, sizeof(int), cudaMemcpyDeviceToHost, st));
    MLMC_CUDA_TRY(cudaStreamSynchronize(st));
    H.n_act = na;
    return na;
  };
  if (use_cta) {
    CtaArgs<T> A;
    A.L = H.L;
    A.B = B;
    A.nu1 = nu1;
    A.nu2 = nu2;
    A.maxc = maxc;
    A.rtol = rtol;
    A.mode = cg ? kCtaCG : (mixed ? kCtaRefinement : kCtaStationary);
    for (int j = 0; j < H.L; ++j) {
      Level<T>& v = H.lv[j];
      A.lv[j].n = v.n;
      A.lv[j].Kx = v.Kx;
      A.lv[j].Ky = v.Ky;
      A.lv[j].Kz = v.Kz;
      A.lv[j].D = v.D;
      A.lv[j].Dinv = v.Dinv;
      A.lv[j].kn = H.nodal[j] ? v.kn : nullptr;
      A.lv[j].u = v.u;
      A.lv[j].g = v.g;
      A.lv[j].r = v.r;
    }
    A.Ainv = H.Ainv;
    A.Fx = mixed ? H.K64x : (const double*)(const void*)l0.Kx;
    A.Fy = mixed ? H.K64y : (const double*)(const void*)l0.Ky;
    A.Fz = mixed ? H.K64z : (const double*)(const void*)l0.Kz;
    A.D = mixed ? H.D64 : (const double*)(const void*)l0.D;
    A.g64 = H.g64;
    A.x = (!mixed && !cg) ? (double*)(void*)l0.u : a.u;
    A.R = H.R;
    A.P = H.P;
    A.Q = H.Q;
    A.Z = H.Z;
    A.g2 = H.g2;
    A.relres = H.relres;
    A.cycles = H.cycles;
    A.active = H.active;
    A.work = H.n_active;
    A.NB = H.NB;
    A.slabs = apply_slabs(a.n, &A.zslab);
    int dev = 0, sms = 0, per_sm = 0;
    MLMC_CUDA_TRY(cudaGetDevice(&dev));
    MLMC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MLMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_cta<T>, kCtaThreads, 0));
    const int grid = B < sms * (per_sm > 0 ? per_sm : 1) ? B : sms * (per_sm > 0 ? per_sm : 1);
    MLMC_CUDA_TRY(cudaMemsetAsync(H.n_active, 0, sizeof(int), st));
    MLMC_LAUNCH(prof::sized(sizeof(T) == 4 ? "solve_cta_mixed" : "solve_cta_f64", a.n), 0.0, 0.0, st,
                (k_solve_cta<T><<<grid, kCtaThreads, 0, st>>>(A)));
    MLMC_CUDA_TRY(cudaGetLastError());
  }
  if (cg && !use_cta) {
    const int st_pcg = pcg_loop<T>(H, a, nu1, nu2, rtol, maxc, st, gr);
    if (st_pcg < 0) return st_pcg;
  }
  if (fmg) {
    // One FMG cycle (nested iteration, Sec. 7): every grid's own right-hand side h_j^2 f
    // (f = 1), the exact solve on the coarsest grid, then per finer grid the P1 (or
    // trilinear) interpolation of the coarser solution and max_cycles V(nu1, nu2) cycles.
    for (int j = 1; j < H.L; ++j) {
      Level<T>& v = H.lv[j];
      const double hj = 1.0 / (double)(v.n - 1);
      if (H.split)
        MLMC_LAUNCH("prepare", B * (double)v.n3 * 8.0, B * (double)v.n3, st,
                    (k_prepare<true><<<plane_grid(v.n * v.n, (long long)B * v.n), kPlaneThreads, 0, st>>>(
                        v.n, B, hj * hj, nullptr, (double*)v.g, (double*)v.u)));
      else
        MLMC_LAUNCH("prepare", B * (double)v.n3 * 8.0, B * (double)v.n3, st,
                    (k_prepare<<<plane_grid(v.n * v.n, (long long)B * v.n), kPlaneThreads, 0, st>>>(
                        v.n, B, hj * hj, nullptr, (double*)v.g, (double*)v.u)));
    }
    vcycle(H, H.L - 1, nu1, nu2, st);
    for (int j = H.L - 2; j >= 0; --j) {
      Level<T>& v = H.lv[j];
      Level<T>& w = H.lv[j + 1];
      const int m = v.n - 2;
      MLMC_CUDA_TRY(cudaMemsetAsync(v.u, 0, (size_t)B * (H.split ? split_elems(v.n) : v.n3) * sizeof(T), st));
      if (H.p1 && H.split)
        MLMC_LAUNCH("prolong_p1", B * (2.0 * (double)v.n3 + (double)w.n3) * W, B * interior(v.n) * 1.5, st,
                    (k_prolong_p1<T, true><<<plane_grid(m * m, (long long)B * m), kPlaneThreads, 0, st>>>(
                        v.n, B, w.u, v.u, H.active)));
      else if (H.p1)
        MLMC_LAUNCH("prolong_p1", B * (2.0 * (double)v.n3 + (double)w.n3) * W, B * interior(v.n) * 1.5, st,
                    (k_prolong_p1<T><<<plane_grid(m * m, (long long)B * m), kPlaneThreads, 0, st>>>(
                        v.n, B, w.u, v.u, H.active)));
      else if (H.split) {
        if constexpr (sizeof(T) == 8)
          MLMC_LAUNCH(Names<T>::prolong, B * (2.0 * (double)v.n3 + (double)w.n3) * W, B * interior(v.n) * 4.375, st,
                      MLMC_SPLIT_DISPATCH(v.n, (k_prolong_blk_split<LG, double><<<
                                                   dim3((unsigned)(((w.n - 1) * (w.n - 1) + 127) / 128),
                                                        (unsigned)(w.n - 1), (unsigned)B),
                                                   128, 0, st>>>((const double*)(const void*)w.u,
                                                                 (double*)(void*)v.u, H.active))));
      } else
        MLMC_LAUNCH(Names<T>::prolong, B * (2.0 * (double)v.n3 + (double)w.n3) * W, B * interior(v.n) * 4.375, st,
                    (k_prolong_blk<T><<<plane_grid((w.n - 1) * (w.n - 1), (long long)B * (w.n - 1)), 128, 0, st>>>(
                        v.n, B, w.u, v.u, H.active)));
      // with MLMC_FMG_GRAPHS=1 the cycles of grid j replay one graph captured for them (on
      // created streams): a level alone runs 4-6% faster, but the capture and instantiation
      // of every grid's graph in every solve cost more than they save while other level
      // streams keep the GPU busy, so direct launches are the default
      GraphRunner<T> fr;
      fr.enabled = gr.enabled && fmg_graphs();
      for (int cyc = 0; cyc < maxc; ++cyc) MLMC_TRY(fr.run(H, nu1, nu2, st, j));
    }
    std::vector<int> cyc(B, maxc);
    MLMC_CUDA_TRY(cudaMemcpyAsync(H.cycles, cyc.data(), B * sizeof(int), cudaMemcpyHostToDevice, st));
    // the final relative residual, for the statistics only (the cycle's work is fixed)
    MLMC_CUDA_TRY(cudaMemsetAsync(H.n_active, 0, sizeof(int), st));
    int zs = 0;
    const dim3 rz = zmarch_grid(a.n, B, &zs);
    if (H.split)
      MLMC_LAUNCH("residual_norm_f64", B * interior(a.n) * 6.0 * 8, B * interior(a.n) * 16.0, st,
                  (k_residual_norm_split<<<rz, 128, 0, st>>>(a.n, zs, (const double*)l0.Kx, (const double*)l0.Ky,
                                                             (const double*)l0.Kz, (const double*)l0.D,
                                                             (const double*)l0.g, (const double*)l0.u, H.partial,
                                                             H.active)));
    else
      MLMC_LAUNCH("residual_norm_f64", B * interior(a.n) * 6.0 * 8, B * interior(a.n) * 16.0, st,
                  (k_residual_z<T, T, T, T><<<rz, 128, 0, st>>>(a.n, zs, l0.Kx, l0.Ky, l0.Kz, l0.D, l0.g, l0.u,
                                                                nullptr, H.partial, H.active)));
    MLMC_LAUNCH("norm_update", B * H.NBz * 8.0, B * H.NBz * 1.0, st,
                (k_norm_update<<<sb, 128, 0, st>>>(B, H.NBz, H.partial, H.g2, H.relres, H.cycles, H.active, 1, 0,
                                                   0.0, maxc, H.n_active)));
  }
  int na = (cg || fmg || use_cta) ? 0 : residual_check(0);
  if (na < 0) return na;
  while (na > 0) {
    if (mixed) {
      MLMC_CUDA_TRY(
          cudaMemsetAsync(H.lv[0].u, 0, (size_t)B * (H.split ? split_elems(a.n) : l0.n3) * sizeof(T), st));
      MLMC_TRY(gr.run(H, nu1, nu2, st));
      const dim3 ug = plane_grid(a.n * a.n, (long long)B * a.n);
      if (H.split)
        MLMC_LAUNCH("update_mixed", H.n_act * (double)l0.n3 * (W + 16), H.n_act * (double)l0.n3, st,
                    (k_update_mixed<true><<<ug, kPlaneThreads, 0, st>>>(a.n, B, (const float*)H.lv[0].u, a.u,
                                                                          H.active)));
      else
        MLMC_LAUNCH("update_mixed", H.n_act * (double)l0.n3 * (W + 16), H.n_act * (double)l0.n3, st,
                    (k_update_mixed<false><<<ug, kPlaneThreads, 0, st>>>(a.n, B, (const float*)H.lv[0].u, a.u,
                                                                           H.active)));
    } else {
      MLMC_TRY(gr.run(H, nu1, nu2, st));
    }
    na = residual_check(1);
    if (na < 0) return na;
  }
  // FP64 solves iterate in place on the caller's u; the fused smoother may leave the
  // latest iterate in the spare buffer
  if (!mixed && !cg && H.split)
    MLMC_LAUNCH("split_copy", B * (double)l0.n3 * 16.0, 0.0, st,
                (k_split_copy<double, false><<<plane_grid(a.n * a.n, (long long)B * a.n), kPlaneThreads, 0, st>>>(
                    a.n, B, (const double*)(const void*)H.lv[0].u, a.u)));
  else if (!mixed && !cg)
    MLMC_CUDA_TRY(cudaMemcpyAsync(a.u, H.lv[0].u, (size_t)B * l0.n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  MLMC_CUDA_TRY(cudaGetLastError());
  if (cycles_dev)
    MLMC_CUDA_TRY(cudaMemcpyAsync(cycles_dev, H.cycles, B * sizeof(int), cudaMemcpyDeviceToDevice, st));
  if (relres_dev)
    MLMC_CUDA_TRY(cudaMemcpyAsync(relres_dev, H.relres, B * sizeof(double), cudaMemcpyDeviceToDevice, st));
  std::vector<int> cyc(B);
  std::vector<double> rel(B);
  int errw = 0;
  MLMC_CUDA_TRY(cudaMemcpyAsync(&errw, H.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  MLMC_CUDA_TRY(cudaMemcpyAsync(cyc.data(), H.cycles, B * sizeof(int), cudaMemcpyDeviceToHost, st));
  MLMC_CUDA_TRY(cudaMemcpyAsync(rel.data(), H.relres, B * sizeof(double), cudaMemcpyDeviceToHost, st));
  MLMC_CUDA_TRY(cudaStreamSynchronize(st));
  if (errw == 1) {
    set_error("a staging wait of the fused smoother ran out of its time budget");
    return MLMC_ERR_TIMEOUT;
  }
  if (errw) {
    set_error("the fused smoother's bounds check failed (code %d)", errw);
    return MLMC_ERR_CUDA;
  }
  int bad = 0;
  for (int s = 0; s < B; ++s) {
    if (cycles_host) cycles_host[s] = cyc[s];
    if (relres_host) relres_host[s] = rel[s];
    if (!fmg && rtol > 0.0 && !(rel[s] <= rtol)) ++bad;
  }
  if (n_unconv) *n_unconv = bad;
  return MLMC_OK;
}

}  // namespace

size_t mg_workspace_bytes(int B, int n, int precision, int accel) {
  Carver c(nullptr);
  if (precision == MLMC_PREC_MIXED) {
    Hier<float> H;
    layout<float>(H, c, B, n, true, accel == MLMC_ACCEL_CG);
  } else {
    Hier<double> H;
    layout<double>(H, c, B, n, false, accel == MLMC_ACCEL_CG);
  }
  return c.off;
}

int mg_solve_dev(const MGSolveArgs& a, void* ws, cudaStream_t st, int* cycles_host, double* relres_host,
                 int* n_unconv, int* cycles_dev, double* relres_dev) {
  if (a.cfg.precision == MLMC_PREC_MIXED)
    return solve_impl<float>(a, ws, st, cycles_host, relres_host, n_unconv, cycles_dev, relres_dev);
  return solve_impl<double>(a, ws, st, cycles_host, relres_host, n_unconv, cycles_dev, relres_dev);
}

int interpolate_dev(const double* uc, int nf, int B, double* uf, cudaStream_t st) {
  MLMC_CUDA_TRY(cudaMemsetAsync(uf, 0, (size_t)B * cube(nf) * sizeof(double), st));
  const int mc = (nf + 1) / 2 - 1;
  MLMC_LAUNCH("interpolate_f64", B * (2.0 * (double)cube(nf) + (double)cube((nf + 1) / 2)) * 8.0,
              B * interior(nf) * 4.375, st,
              (k_prolong_blk<double><<<plane_grid(mc * mc, (long long)B * mc), 128, 0, st>>>(nf, B, uc, uf,
                                                                                             nullptr)));
  return MLMC_OK;
}

size_t qoi_scratch_bytes(int B, int n) {
  const int S = (n - 1) / 2 + 1;
  const size_t a = (size_t)B * reduce_blocks(cube(S)) * sizeof(double);
  const size_t b = (size_t)B * reduce_blocks((size_t)(n - 1) * (n - 1)) * sizeof(double);
  return a256(a > b ? a : b);
}

int qoi_dev(const double* u, int n, int B, double* Q, void* scratch, cudaStream_t st) {
  const int S = (n - 1) / 2 + 1;
  const int NB = reduce_blocks(cube(S));
  double* partial = (double*)scratch;
  MLMC_LAUNCH("qoi", B * (double)cube(S) * 8, B * (double)cube(S) * 6, st,
              (k_qoi<<<dim3(NB, B), kThreads, 0, st>>>(n, u, partial)));
  const double h = 1.0 / (double)(n - 1);
  MLMC_LAUNCH("qoi_final", B * NB * 8.0, B * NB * 1.0, st,
              (k_qoi_final<<<(B + 127) / 128, 128, 0, st>>>(B, NB, 8.0 * h * h * h, partial, Q)));
  MLMC_CUDA_TRY(cudaGetLastError());
  return MLMC_OK;
}

int qoi_any(int qoi, const double* u, int n, int B, double* Q, void* scratch, const double* k0, int n_k0, int st0,
            cudaStream_t st) {
  if (qoi == MLMC_QOI_MEAN) return qoi_dev(u, n, B, Q, scratch, st);
  if (qoi == MLMC_QOI_POINT) {
    MLMC_LAUNCH("qoi", B * 8.0, 0.0, st, (k_qoi_point<<<(B + 127) / 128, 128, 0, st>>>(n, B, u, Q)));
    return MLMC_OK;
  }
  const int NB = reduce_blocks((size_t)(n - 1) * (n - 1));
  double* partial = (double*)scratch;
  MLMC_LAUNCH("qoi", B * (double)(n - 1) * (n - 1) * 8 * 16, B * (double)(n - 1) * (n - 1) * 6 * 8, st,
              (k_qoi_flux<<<dim3(NB, B), kThreads, 0, st>>>(n, u, k0, n_k0, st0, partial)));
  const double h = 1.0 / (double)(n - 1);
  MLMC_LAUNCH("qoi_final", B * NB * 8.0, B * NB * 1.0, st,
              (k_qoi_final<<<(B + 127) / 128, 128, 0, st>>>(B, NB, h / 6.0, partial, Q)));
  MLMC_CUDA_TRY(cudaGetLastError());
  return MLMC_OK;
}

}  // namespace mlmc
