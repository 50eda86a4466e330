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
  static constexpr int kStaged = 3;               // u, Kx, Ky: read by in-plane neighbours
  static constexpr int W2 = BX + 4, H2 = BY + 4;  // tile + 2-ring: one thread per column
  static constexpr int W1 = BX + 2, H1 = BY + 2;  // tile + 1-ring
  static constexpr int P2 = W2 * H2, P1 = W1 * H1;
  static constexpr int threads = P2;
  static constexpr size_t bytes = sizeof(T) * ((size_t)kStaged * kSlots * P2 + 3 * (size_t)P1);
};

// One thread per column of the tile + 2-ring. u, Kx and Ky (which in-plane neighbours
// read) are staged in shared memory with cp.async; Kz, 1/D and g are read only by the
// column's own updates and travel in a five-plane register window, loaded two planes
// ahead. Ring-1 and tile threads compute the red update of their column; tile threads
// compute the black update (one plane behind) and write the output.
template <typename T, int BX, int BY>
__global__ void __launch_bounds__(FusedLayout<T, BX, BY>::threads)
    k_rbgs_fused(int n, int ntx, int ntiles, int zslab, const T* __restrict__ Kx, const T* __restrict__ Ky,
                 const T* __restrict__ Kz, const T* __restrict__ Dinv, const T* __restrict__ g,
                 const T* __restrict__ uin, T* __restrict__ uout, const int* __restrict__ active) {
  using Lay = FusedLayout<T, BX, BY>;
  constexpr int W2 = Lay::W2, H2 = Lay::H2, P2 = Lay::P2, W1 = Lay::W1, P1 = Lay::P1, NS = Lay::kStaged;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* stage = (T*)smem_raw;                      // [array][slot][P2]
  T* red = stage + (size_t)NS * kSlots * P2;    // [3][P1]: plane after its red phase
  const int s = blockIdx.y;
  const int tid = threadIdx.x;
  const int tile = blockIdx.x % ntiles, slab = blockIdx.x / ntiles;
  const int x0 = (tile % ntx) * BX + 1, y0 = (tile / ntx) * BY + 1;  // first owned node
  const int zlo = 1 + slab * zslab, zhi = min(n - 2, zlo + zslab - 1);
  const size_t n2 = (size_t)n * n, base = (size_t)s * n2 * n;
  const int ci = tid % W2, cj = tid / W2;
  const int gx = x0 - 2 + ci, gy = y0 - 2 + cj;
  const bool in_grid = gx >= 0 && gx < n && gy >= 0 && gy < n;
  const bool ring1 = ci >= 1 && ci <= W2 - 2 && cj >= 1 && cj <= H2 - 2;
  const bool owned = ci >= 2 && ci <= W2 - 3 && cj >= 2 && cj <= H2 - 3;
  const bool interior_col = gx >= 1 && gx <= n - 2 && gy >= 1 && gy <= n - 2;
  const int c = tid;
  const int c1 = (cj - 1) * W1 + (ci - 1);
  if (active && !active[s]) {
    if (owned && interior_col)
      for (int z = zlo; z <= zhi; ++z) {
        const size_t p = base + (size_t)z * n2 + (size_t)gy * n + gx;
        uout[p] = uin[p];
      }
    return;
  }
  const T* src[NS] = {uin, Kx, Ky};
  auto sm = [&](int a, int slot, int i) -> T& { return stage[((size_t)a * kSlots + slot) * P2 + i]; };
  const size_t col = base + (size_t)gy * n + gx;
  auto issue = [&](int z) {
    if (z < 0 || z >= n) return;
    const int slot = z % kSlots;
    if (in_grid) {
      const size_t off = col + (size_t)z * n2;
#pragma unroll
      for (int a = 0; a < NS; ++a) cp_async(&sm(a, slot, c), src[a] + off);
    } else {
#pragma unroll
      for (int a = 0; a < NS; ++a) sm(a, slot, c) = T(0);
    }
  };
  // this column's Kz, 1/D, g on planes z-2 .. z+2 (m2, m1, c0, p1, p2)
  const bool need_regs = ring1 && in_grid;
  auto ld = [&](const T* a, int z) -> T { return (need_regs && z >= 0 && z < n) ? a[col + (size_t)z * n2] : T(0); };
  const int zs = zlo - 1, ze = zhi + 1;
  T kz_m2 = ld(Kz, zs - 2), kz_m1 = ld(Kz, zs - 1), kz_0 = ld(Kz, zs), kz_p1 = ld(Kz, zs + 1), kz_p2;
  T di_m1 = ld(Dinv, zs - 1), di_0 = ld(Dinv, zs), di_p1 = ld(Dinv, zs + 1), di_p2;
  T g_m1 = ld(g, zs - 1), g_0 = ld(g, zs), g_p1 = ld(g, zs + 1), g_p2;

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
    kz_p2 = ld(Kz, z + 2);
    di_p2 = ld(Dinv, z + 2);
    g_p2 = ld(g, z + 2);
    cp_async_wait1();  // planes <= z+1 of this thread's column have landed
    __syncthreads();   // ... and of every column
    const int sz = z % kSlots, szm = (z + kSlots - 1) % kSlots, szp = (z + 1) % kSlots;
    T* rz = red + (size_t)(z % 3) * P1;
    if (ring1) {
      T v = sm(0, sz, c);
      if (z >= 1 && z <= n - 2 && interior_col && ((gx + gy + z) & 1) == 0) {
        T acc = g_0;
        acc = fma(sm(1, sz, c - 1), sm(0, sz, c - 1), acc);
        acc = fma(sm(1, sz, c), sm(0, sz, c + 1), acc);
        acc = fma(sm(2, sz, c - W2), sm(0, sz, c - W2), acc);
        acc = fma(sm(2, sz, c), sm(0, sz, c + W2), acc);
        acc = fma(kz_m1, sm(0, szm, c), acc);
        acc = fma(kz_0, sm(0, szp, c), acc);
        v = acc * di_0;
      }
      rz[c1] = v;
    }
    __syncthreads();
    if (z > zs) {
      const int zb = z - 1, sb = szm;
      if (owned && interior_col && zb >= zlo && zb <= zhi) {
        const T* rb = red + (size_t)(zb % 3) * P1;
        T v = rb[c1];
        if (((gx + gy + zb) & 1) == 1) {
          const T* rbm = red + (size_t)((zb + 2) % 3) * P1;  // plane z-2
          T acc = g_m1;
          acc = fma(sm(1, sb, c - 1), rb[c1 - 1], acc);
          acc = fma(sm(1, sb, c), rb[c1 + 1], acc);
          acc = fma(sm(2, sb, c - W2), rb[c1 - W1], acc);
          acc = fma(sm(2, sb, c), rb[c1 + W1], acc);
          acc = fma(kz_m2, rbm[c1], acc);
          acc = fma(kz_m1, rz[c1], acc);
          v = acc * di_m1;
        }
        uout[col + (size_t)zb * n2] = v;
      }
    }
    // advance the register window by one plane
    kz_m2 = kz_m1;
    kz_m1 = kz_0;
    kz_0 = kz_p1;
    kz_p1 = kz_p2;
    di_m1 = di_0;
    di_0 = di_p1;
    di_p1 = di_p2;
    g_m1 = g_0;
    g_0 = g_p1;
    g_p1 = g_p2;
  }
}

// ---------------------------------------------------------------------------------
// The same sweep with the plane rows staged by the TMA unit: one cp.async.bulk per row
// of the tile + 2-ring per array (instead of one 4-byte cp.async per element), issued
// by warp 0 and completing on one mbarrier per plane slot. A bulk copy needs 16-byte
// aligned source, destination and size, so each row copy starts at the aligned address
// at or below the row's first staged element and every staged row records its offset.
// Elements that the copy brings in from beyond the row's ends (x < 0, x >= n) are
// never read by an update. Rows outside the grid (y < 0, y >= n) are zero-filled once.
// Every mbarrier wait is bounded by a clock budget; on expiry the CTA records an error
// word and leaves at the next barrier.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return done != 0;
}
// bounded wait: about one second of SM clock
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(b, parity))
    if (clock64() - t0 > 2000000000LL) return false;
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(b))
      : "memory");
}

template <typename T, int BX, int BY>
struct BulkLayout {
  static constexpr int W2 = BX + 4, H2 = BY + 4;
  static constexpr int W1 = BX + 2, H1 = BY + 2;
  static constexpr int P1 = W1 * H1;
  static constexpr int EPV = 16 / (int)sizeof(T);  // elements per 16 bytes
  static constexpr int RP = ((W2 + 2 * EPV + EPV - 1) / EPV) * EPV;  // staged row pitch
  static constexpr int PLANE = H2 * RP;
  static constexpr int threads = W2 * H2;
  static constexpr size_t stage_bytes = sizeof(T) * (size_t)kArrays * kSlots * PLANE;
  static constexpr size_t red_off = stage_bytes;
  static constexpr size_t offs_off = red_off + sizeof(T) * 3 * (size_t)P1;
  static constexpr size_t mbar_off = (offs_off + sizeof(int) * kSlots * H2 + 7) & ~(size_t)7;
  static constexpr size_t flag_off = mbar_off + 8 * kSlots;
  static constexpr size_t bytes = flag_off + 16;
};

template <typename T, int BX, int BY>
__global__ void __launch_bounds__(BulkLayout<T, BX, BY>::threads)
    k_rbgs_bulk(int n, int ntx, int ntiles, int zslab, const T* __restrict__ Kx, const T* __restrict__ Ky,
                const T* __restrict__ Kz, const T* __restrict__ Dinv, const T* __restrict__ g,
                const T* __restrict__ uin, T* __restrict__ uout, const int* __restrict__ active,
                int* __restrict__ err) {
  using Lay = BulkLayout<T, BX, BY>;
  constexpr int W2 = Lay::W2, H2 = Lay::H2, W1 = Lay::W1, P1 = Lay::P1, RP = Lay::RP, PLANE = Lay::PLANE;
  constexpr int EPV = Lay::EPV;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* stage = (T*)smem_raw;
  T* red = (T*)(smem_raw + Lay::red_off);
  int* offs = (int*)(smem_raw + Lay::offs_off);  // [slot][row]
  uint64_t* mbar = (uint64_t*)(smem_raw + Lay::mbar_off);
  volatile int* abort_flag = (volatile int*)(smem_raw + Lay::flag_off);
  const int s = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tile = blockIdx.x % ntiles, slab = blockIdx.x / ntiles;
  const int x0 = (tile % ntx) * BX + 1, y0 = (tile / ntx) * BY + 1;
  const int zlo = 1 + slab * zslab, zhi = min(n - 2, zlo + zslab - 1);
  const size_t n2 = (size_t)n * n, base = (size_t)s * n2 * n;
  const int ci = tid % W2, cj = tid / W2;
  const int gx = x0 - 2 + ci, gy = y0 - 2 + cj;
  const bool ring1 = ci >= 1 && ci <= W2 - 2 && cj >= 1 && cj <= H2 - 2;
  const bool owned = ci >= 2 && ci <= W2 - 3 && cj >= 2 && cj <= H2 - 3;
  const bool interior_col = gx >= 1 && gx <= n - 2 && gy >= 1 && gy <= n - 2;
  const int c1 = (cj - 1) * W1 + (ci - 1);
  if (active && !active[s]) {
    if (owned && interior_col)
      for (int z = zlo; z <= zhi; ++z) {
        const size_t p = base + (size_t)z * n2 + (size_t)gy * n + gx;
        uout[p] = uin[p];
      }
    return;
  }
  const T* src[kArrays] = {uin, Kx, Ky, Kz, Dinv, g};
  if (tid == 0) {
    for (int k = 0; k < kSlots; ++k) mbar_init(&mbar[k], 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  // row offsets of every slot start at 0 (a slot is read before its first staging only
  // where the value is unused, but its index must stay inside the staging buffer)
  for (int t = tid; t < kSlots * H2; t += Lay::threads) offs[t] = 0;
  // rows outside the grid: zeros in every slot, never copied
  for (int t = tid; t < kArrays * kSlots * H2; t += Lay::threads) {
    const int j = t % H2;
    const int yy = y0 - 2 + j;
    if (yy < 0 || yy >= n)
      for (int e = 0; e < RP; ++e) stage[(size_t)(t / H2) * PLANE + (size_t)j * RP + e] = T(0);
  }
  __syncthreads();
  const int zs = zlo - 1, ze = zhi + 1;
  // warp 0 stages plane z (rows of all six arrays) into slot z % kSlots
  auto issue = [&](int z) {
    if (warp != 0 || z < 0 || z >= n) return;
    const int slot = z % kSlots;
    unsigned bytes = 0;
    for (int it = lane; it < kArrays * H2; it += 32) {
      const int a = it / H2, j = it % H2;
      const int yy = y0 - 2 + j;
      if (yy < 0 || yy >= n) {
        if (a == 0) offs[slot * H2 + j] = 0;
        continue;
      }
      const size_t row = base + (size_t)z * n2 + (size_t)yy * n;
      const size_t lo = row + (size_t)max(x0 - 2, 0), hi = row + (size_t)min(x0 + BX + 2, n);
      const size_t A = lo & ~(size_t)(EPV - 1), E = (hi + EPV - 1) & ~(size_t)(EPV - 1);
      bytes += (unsigned)((E - A) * sizeof(T));
      if (a == 0) offs[slot * H2 + j] = (int)((long long)row + (x0 - 2) - (long long)A);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive_expect_tx(&mbar[slot], bytes);
    __syncwarp();
    for (int it = lane; it < kArrays * H2; it += 32) {
      const int a = it / H2, j = it % H2;
      const int yy = y0 - 2 + j;
      if (yy < 0 || yy >= n) continue;
      const size_t row = base + (size_t)z * n2 + (size_t)yy * n;
      const size_t lo = row + (size_t)max(x0 - 2, 0), hi = row + (size_t)min(x0 + BX + 2, n);
      const size_t A = lo & ~(size_t)(EPV - 1), E = (hi + EPV - 1) & ~(size_t)(EPV - 1);
      T* dst = stage + ((size_t)(a * kSlots + slot) * H2 + j) * RP;
      bulk_g2s(dst, src[a] + A, (unsigned)((E - A) * sizeof(T)), &mbar[slot]);
    }
  };
  // the k-th plane staged into a slot completes that slot's barrier phase k: the
  // parity counts uses of the slot from the first staged plane of this CTA
  const int pstart = max(zs - 1, 0);
  auto parity = [&](int z) { return (unsigned)(((z - pstart) / kSlots) & 1); };
  auto wait_plane = [&](int z) {
    if (z < 0 || z >= n) return;
    if (!mbar_wait_bounded(&mbar[z % kSlots], parity(z))) {
      *abort_flag = 1;
      atomicExch(err, 1);
    }
  };
  // element (array a, plane slot sl, staged row j, column i of the tile + 2-ring)
  // (bounds-checked: an index outside the staging buffer records error 2 and reads 0)
  auto at = [&](int a, int sl, int j, int i) -> T {
    const long long k = ((long long)(a * kSlots + sl) * H2 + j) * RP + offs[sl * H2 + j] + i;
    if ((unsigned long long)k >= (unsigned long long)kArrays * kSlots * PLANE) {
      atomicExch(err, 2);
      return T(0);
    }
    return stage[k];
  };
  T kz_m2 = T(0);
  issue(zs - 1);
  issue(zs);
  issue(zs + 1);
  wait_plane(zs - 1);
  wait_plane(zs);
  for (int z = zs; z <= ze; ++z) {
    if (z + 2 <= ze + 1) issue(z + 2);
    wait_plane(z + 1);
    const int sz = z % kSlots, szm = (z + kSlots - 1) % kSlots, szp = (z + 1) % kSlots;
    T* rz = red + (size_t)(z % 3) * P1;
    if (ring1) {
      T v = at(0, sz, cj, ci);
      if (z >= 1 && z <= n - 2 && interior_col && ((gx + gy + z) & 1) == 0) {
        T acc = at(5, sz, cj, ci);
        acc = fma(at(1, sz, cj, ci - 1), at(0, sz, cj, ci - 1), acc);
        acc = fma(at(1, sz, cj, ci), at(0, sz, cj, ci + 1), acc);
        acc = fma(at(2, sz, cj - 1, ci), at(0, sz, cj - 1, ci), acc);
        acc = fma(at(2, sz, cj, ci), at(0, sz, cj + 1, ci), acc);
        acc = fma(at(3, szm, cj, ci), at(0, szm, cj, ci), acc);
        acc = fma(at(3, sz, cj, ci), at(0, szp, cj, ci), acc);
        v = acc * at(4, sz, cj, ci);
      }
      rz[c1] = v;
    }
    __syncthreads();
    if (*abort_flag) {
      // a wait ran out: drain the copies still in flight (bounded), then every thread leaves
      for (int p = z + 1; p <= min(z + 2, min(ze + 1, n - 1)); ++p) mbar_wait_bounded(&mbar[p % kSlots], parity(p));
      return;
    }
    if (z > zs) {
      const int zb = z - 1, sb = szm;
      const T kz_m1 = owned ? at(3, sb, cj, ci) : T(0);  // only owned columns use Kz
      if (owned && interior_col && zb >= zlo && zb <= zhi) {
        const T* rb = red + (size_t)(zb % 3) * P1;
        T v = rb[c1];
        if (((gx + gy + zb) & 1) == 1) {
          const T* rbm = red + (size_t)((zb + 2) % 3) * P1;
          T acc = at(5, sb, cj, ci);
          acc = fma(at(1, sb, cj, ci - 1), rb[c1 - 1], acc);
          acc = fma(at(1, sb, cj, ci), rb[c1 + 1], acc);
          acc = fma(at(2, sb, cj - 1, ci), rb[c1 - W1], acc);
          acc = fma(at(2, sb, cj, ci), rb[c1 + W1], acc);
          acc = fma(kz_m2, rbm[c1], acc);
          acc = fma(kz_m1, rz[c1], acc);
          v = acc * at(4, sb, cj, ci);
        }
        uout[base + (size_t)zb * n2 + (size_t)gy * n + gx] = v;
      }
      kz_m2 = kz_m1;
    } else if (owned && zs >= 1) {
      kz_m2 = at(3, szm, cj, ci);  // Kz(zs-1): plane zs-1 was staged
    }
    __syncthreads();  // slot (z+3) % kSlots = plane z-2 is reused by the next issue
  }
}

template <typename T, int BX, int BY>
int launch_bulk(int n, int B, const T* Kx, const T* Ky, const T* Kz, const T* Dinv, const T* g, const T* uin,
                T* uout, const int* active, int* err, cudaStream_t st) {
  using Lay = BulkLayout<T, BX, BY>;
  static bool configured = false;
  if (!configured) {
    MLMC_CUDA_TRY(cudaFuncSetAttribute(k_rbgs_bulk<T, BX, BY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)Lay::bytes));
    configured = true;
  }
  const int m = n - 2;
  const int ntx = (m + BX - 1) / BX, nty = (m + BY - 1) / BY, ntiles = ntx * nty;
  int slabs = (int)((152LL * 12 + (long long)ntiles * B - 1) / ((long long)ntiles * B));
  if (slabs > m / 8) slabs = m / 8;
  if (slabs < 1) slabs = 1;
  const int zslab = (m + slabs - 1) / slabs;
  slabs = (m + zslab - 1) / zslab;
  dim3 grid((unsigned)(ntiles * slabs), (unsigned)B);
  k_rbgs_bulk<T, BX, BY><<<grid, Lay::threads, Lay::bytes, st>>>(n, ntx, ntiles, zslab, Kx, Ky, Kz, Dinv, g, uin,
                                                                 uout, active, err);
  return MLMC_OK;
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
    case kBulk32x8: return "bulk 32x8";
    case kBulk32x16: return "bulk 32x16";
    case kBulk64x8: return "bulk 64x8";
  }
  return "?";
}

template <typename T>
int rbgs_fused_sweep(int shape, int n, int B, const T* Kx, const T* Ky, const T* Kz, const T* Dinv, const T* g,
                     const T* uin, T* uout, const int* active, int* err, cudaStream_t st) {
  const double interior = (double)(n - 2) * (n - 2) * (n - 2);
  const bool bulk = shape == kBulk32x8 || shape == kBulk32x16 || shape == kBulk64x8;
  const char* cls = bulk ? (sizeof(T) == 4 ? "rbgs_bulk_f32" : "rbgs_bulk_f64")
                         : (sizeof(T) == 4 ? "rbgs_fused_f32" : "rbgs_fused_f64");
  // one full sweep: 7 words per interior node (u read + write, Kx, Ky, Kz, Dinv, g), 13 flops
  prof::Scope scope(cls, B * interior * 7.0 * sizeof(T), B * interior * 13.0, st);
  switch (shape) {
    case kTile32x16:
      return launch_shape<T, 32, 16>(n, B, Kx, Ky, Kz, Dinv, g, uin, uout, active, st);
    case kTile64x8:
      return launch_shape<T, 64, 8>(n, B, Kx, Ky, Kz, Dinv, g, uin, uout, active, st);
    case kBulk32x8:
      return launch_bulk<T, 32, 8>(n, B, Kx, Ky, Kz, Dinv, g, uin, uout, active, err, st);
    case kBulk32x16:
      return launch_bulk<T, 32, 16>(n, B, Kx, Ky, Kz, Dinv, g, uin, uout, active, err, st);
    case kBulk64x8:
      return launch_bulk<T, 64, 8>(n, B, Kx, Ky, Kz, Dinv, g, uin, uout, active, err, st);
    default:
      return launch_shape<T, 32, 8>(n, B, Kx, Ky, Kz, Dinv, g, uin, uout, active, st);
  }
}

template int rbgs_fused_sweep<float>(int, int, int, const float*, const float*, const float*, const float*,
                                     const float*, const float*, float*, const int*, int*, cudaStream_t);
template int rbgs_fused_sweep<double>(int, int, int, const double*, const double*, const double*, const double*,
                                      const double*, const double*, double*, const int*, int*, cudaStream_t);

}  // namespace mlmc
