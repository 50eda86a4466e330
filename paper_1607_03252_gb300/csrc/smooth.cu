// Fused red-black Gauss-Seidel sweep: both colours in ONE pass over the grid.
//
// A red-black sweep (red nodes (i+j+k) even first, then black) updates
//   u_p <- (g_p + sum_q K_pq u_q) * (1 / D_p)
// where every red update reads only black (old) values and every black update reads
// only red (new) values. Marching in z, the red update of plane z and the black update
// of plane z-1 can therefore run in the same step: after red(z), all red neighbours of
// black(z-1) are final.
//
// Each CTA owns one (x, y) tile of one sample and marches z. Its in-plane neighbours
// belong to other CTAs that progress independently, so the kernel never reads values
// another CTA writes during the sweep: it reads the old iterate from `uin`, writes the
// new one to `uout` (double buffer), and recomputes the red colour on a one-cell ring
// around its tile (which needs old values on a two-cell ring). The result equals the
// sequential red-then-black sweep exactly: same operations on the same operands.
//
// Plane data (u, Kx, Ky, Kz, Dinv, g on the tile plus a two-cell ring) is staged in
// shared memory with cp.async, two planes ahead of the plane being updated, in a ring
// of five plane slots; one thread per staged column keeps the work per barrier even.
// z is split into independent slabs (each recomputes the red plane just outside its
// ends) so that a launch has enough CTAs. HBM traffic per sweep is one read of each
// array and one write of u (7 words per node), against 12+ words for two separate
// colour passes.
#include "common.cuh"
#include "prof.cuh"
#include "smooth.cuh"

namespace mlmc {
namespace {

__device__ __forceinline__ void cp_async(float* dst, const float* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(double* dst, const double* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

constexpr int kSlots = 5;    // plane ring of the staged arrays (z-1 .. z+2 live, z+3 in flight)
constexpr int kArrays = 6;   // u, Kx, Ky, Kz, Dinv, g

template <typename T, int BX, int BY>
struct FusedLayout {
  static constexpr int W2 = BX + 4, H2 = BY + 4;  // tile + 2-ring: one thread per column
  static constexpr int W1 = BX + 2, H1 = BY + 2;  // tile + 1-ring
  static constexpr int P2 = W2 * H2, P1 = W1 * H1;
  static constexpr int threads = P2;
  static constexpr size_t bytes = sizeof(T) * ((size_t)kArrays * kSlots * P2 + 3 * (size_t)P1);
};

// One thread per column of the tile + 2-ring: every thread stages its own column of the
// six arrays; ring-1 and tile threads compute the red update of their column; tile
// threads compute the black update (one plane behind) and write the output.
template <typename T, int BX, int BY>
__global__ void __launch_bounds__(FusedLayout<T, BX, BY>::threads)
    k_rbgs_fused(int n, int ntx, int ntiles, int zslab, const T* __restrict__ Kx, const T* __restrict__ Ky,
                 const T* __restrict__ Kz, const T* __restrict__ Dinv, const T* __restrict__ g,
                 const T* __restrict__ uin, T* __restrict__ uout, const int* __restrict__ active) {
  using Lay = FusedLayout<T, BX, BY>;
  constexpr int W2 = Lay::W2, H2 = Lay::H2, P2 = Lay::P2, W1 = Lay::W1, P1 = Lay::P1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* stage = (T*)smem_raw;                          // [array][slot][P2]
  T* red = stage + (size_t)kArrays * kSlots * P2;   // [3][P1]: plane after its red phase
  const int s = blockIdx.y;
  const int tid = threadIdx.x;
  const int tile = blockIdx.x % ntiles, slab = blockIdx.x / ntiles;
  const int x0 = (tile % ntx) * BX + 1, y0 = (tile / ntx) * BY + 1;  // first owned node
  const int zlo = 1 + slab * zslab, zhi = min(n - 2, zlo + zslab - 1);
  const size_t n2 = (size_t)n * n, base = (size_t)s * n2 * n;
  // this thread's column
  const int ci = tid % W2, cj = tid / W2;
  const int gx = x0 - 2 + ci, gy = y0 - 2 + cj;
  const bool in_grid = gx >= 0 && gx < n && gy >= 0 && gy < n;
  const bool ring1 = ci >= 1 && ci <= W2 - 2 && cj >= 1 && cj <= H2 - 2;
  const bool owned = ci >= 2 && ci <= W2 - 3 && cj >= 2 && cj <= H2 - 3;
  const bool interior_col = gx >= 1 && gx <= n - 2 && gy >= 1 && gy <= n - 2;
  const int c = tid;                                   // position in the 2-ring plane
  const int c1 = (cj - 1) * W1 + (ci - 1);             // position in the 1-ring plane (ring1 only)
  if (active && !active[s]) {
    // a finished sample keeps its iterate: carry the owned block over to uout
    if (owned && interior_col)
      for (int z = zlo; z <= zhi; ++z) {
        const size_t p = base + (size_t)z * n2 + (size_t)gy * n + gx;
        uout[p] = uin[p];
      }
    return;
  }
  const T* src[kArrays] = {uin, Kx, Ky, Kz, Dinv, g};
  auto sm = [&](int a, int slot, int i) -> T& { return stage[((size_t)a * kSlots + slot) * P2 + i]; };
  const size_t col = base + (size_t)gy * n + gx;
  auto issue = [&](int z) {
    if (z < 0 || z >= n) return;
    const int slot = z % kSlots;
    if (in_grid) {
      const size_t off = col + (size_t)z * n2;
#pragma unroll
      for (int a = 0; a < kArrays; ++a) cp_async(&sm(a, slot, c), src[a] + off);
    } else {
#pragma unroll
      for (int a = 0; a < kArrays; ++a) sm(a, slot, c) = T(0);
    }
  };
  T kz_m2 = T(0);  // Kz(z-2) of this column

  // steps z = zlo-1 .. zhi+1: red phase on plane z, black phase on plane z-1
  const int zs = zlo - 1, ze = zhi + 1;
  issue(zs - 1);
  cp_async_commit();
  issue(zs);
  cp_async_commit();
  issue(zs + 1);
  cp_async_commit();
  for (int z = zs; z <= ze; ++z) {
    // slot of plane z+2 held plane z-3, last read before the previous step's barriers
    issue(z + 2);
    cp_async_commit();
    cp_async_wait1();  // planes <= z+1 of this thread's column have landed
    __syncthreads();   // ... and of every column
    const int sz = z % kSlots, szm = (z + kSlots - 1) % kSlots, szp = (z + 1) % kSlots;
    T* rz = red + (size_t)(z % 3) * P1;
    if (ring1) {
      T v = sm(0, sz, c);
      if (z >= 1 && z <= n - 2 && interior_col && ((gx + gy + z) & 1) == 0) {
        T acc = sm(5, sz, c);
        acc = fma(sm(1, sz, c - 1), sm(0, sz, c - 1), acc);
        acc = fma(sm(1, sz, c), sm(0, sz, c + 1), acc);
        acc = fma(sm(2, sz, c - W2), sm(0, sz, c - W2), acc);
        acc = fma(sm(2, sz, c), sm(0, sz, c + W2), acc);
        acc = fma(sm(3, szm, c), sm(0, szm, c), acc);
        acc = fma(sm(3, sz, c), sm(0, szp, c), acc);
        v = acc * sm(4, sz, c);
      }
      rz[c1] = v;
    }
    __syncthreads();
    if (z > zs) {
      const int zb = z - 1, sb = szm;
      const T kz_m1 = sm(3, sb, c);  // Kz(z-1) of this column
      if (owned && interior_col && zb >= zlo && zb <= zhi) {
        const T* rb = red + (size_t)(zb % 3) * P1;
        T v = rb[c1];
        if (((gx + gy + zb) & 1) == 1) {
          const T* rbm = red + (size_t)((zb + 2) % 3) * P1;  // plane z-2
          T acc = sm(5, sb, c);
          acc = fma(sm(1, sb, c - 1), rb[c1 - 1], acc);
          acc = fma(sm(1, sb, c), rb[c1 + 1], acc);
          acc = fma(sm(2, sb, c - W2), rb[c1 - W1], acc);
          acc = fma(sm(2, sb, c), rb[c1 + W1], acc);
          acc = fma(kz_m2, rbm[c1], acc);
          acc = fma(kz_m1, rz[c1], acc);
          v = acc * sm(4, sb, c);
        }
        uout[col + (size_t)zb * n2] = v;
      }
      kz_m2 = kz_m1;
    } else {
      kz_m2 = sm(3, szm, c);  // Kz(zs-1): only used when zs-1 is a staged plane
    }
  }
}

template <typename T, int BX, int BY>
int launch_shape(int n, int B, const T* Kx, const T* Ky, const T* Kz, const T* Dinv, const T* g, const T* uin,
                 T* uout, const int* active, cudaStream_t st) {
  using Lay = FusedLayout<T, BX, BY>;
  static bool configured = false;  // per template instance; attribute set once per process
  if (!configured) {
    MLMC_CUDA_TRY(cudaFuncSetAttribute(k_rbgs_fused<T, BX, BY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Lay::bytes));
    configured = true;
  }
  const int m = n - 2;
  const int ntx = (m + BX - 1) / BX, nty = (m + BY - 1) / BY, ntiles = ntx * nty;
  // split z into independent slabs until the launch has ~12 CTAs per SM (the result is
  // the same for any split); slabs of at least 8 planes
  int slabs = (int)((152LL * 12 + (long long)ntiles * B - 1) / ((long long)ntiles * B));
  if (slabs > m / 8) slabs = m / 8;
  if (slabs < 1) slabs = 1;
  const int zslab = (m + slabs - 1) / slabs;
  slabs = (m + zslab - 1) / zslab;
  dim3 grid((unsigned)(ntiles * slabs), (unsigned)B);
  k_rbgs_fused<T, BX, BY><<<grid, Lay::threads, Lay::bytes, st>>>(n, ntx, ntiles, zslab, Kx, Ky, Kz, Dinv, g, uin,
                                                                  uout, active);
  return MLMC_OK;
}

}  // namespace

const char* tile_name(int shape) {
  switch (shape) {
    case kTile32x8: return "32x8";
    case kTile32x16: return "32x16";
    case kTile64x8: return "64x8";
  }
  return "?";
}

template <typename T>
int rbgs_fused_sweep(int shape, int n, int B, const T* Kx, const T* Ky, const T* Kz, const T* Dinv, const T* g,
                     const T* uin, T* uout, const int* active, cudaStream_t st) {
  const double interior = (double)(n - 2) * (n - 2) * (n - 2);
  const char* cls = sizeof(T) == 4 ? "rbgs_fused_f32" : "rbgs_fused_f64";
  // one full sweep: 7 words per interior node (u read + write, Kx, Ky, Kz, Dinv, g), 13 flops
  prof::Scope scope(cls, B * interior * 7.0 * sizeof(T), B * interior * 13.0, st);
  switch (shape) {
    case kTile32x16:
      return launch_shape<T, 32, 16>(n, B, Kx, Ky, Kz, Dinv, g, uin, uout, active, st);
    case kTile64x8:
      return launch_shape<T, 64, 8>(n, B, Kx, Ky, Kz, Dinv, g, uin, uout, active, st);
    default:
      return launch_shape<T, 32, 8>(n, B, Kx, Ky, Kz, Dinv, g, uin, uout, active, st);
  }
}

template int rbgs_fused_sweep<float>(int, int, int, const float*, const float*, const float*, const float*,
                                     const float*, const float*, float*, const int*, cudaStream_t);
template int rbgs_fused_sweep<double>(int, int, int, const double*, const double*, const double*, const double*,
                                      const double*, const double*, double*, const int*, cudaStream_t);

}  // namespace mlmc
