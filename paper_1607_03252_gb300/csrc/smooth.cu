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
// Staging: u, Kx and Ky of the tile + 2-ring (the arrays that in-plane neighbours read)
// are copied into shared memory by 16-byte cp.async copies, u two planes ahead and Kx,
// Ky one plane ahead, each in a ring of four plane slots. Grid rows have odd length, so
// a row starts at any element offset modulo 16 bytes: each staged row is copied from the
// 16-byte boundary at or below its first element (in the frame of the array's element
// index), and reads add that row's offset, computed from the element index. Kz, 1/D and
// g, which only a column's own updates read, travel in per-column register windows.
// Each thread owns four consecutive rows of one column of the staged tile: at every
// (x, z) two of them are red and two black, so a thread does two independent red
// updates of plane z and two black updates of plane z-1 per step. In-sample index
// arithmetic is 32-bit (n^3 < 2^31). z is split into independent slabs (each recomputes
// the red plane just outside its ends) so that a launch has enough CTAs. HBM traffic
// per sweep is one read of each array and one write of u (7 words per node), against
// 12+ words for two separate colour passes.
#include "common.cuh"
#include "prof.cuh"
#include "smooth.cuh"
#include "bulk.cuh"

namespace mlmc {
namespace {

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Ring depth of the fused sweep. At step z the red phase reads u on planes z-1..z+1 and
// Kx, Ky on plane z, the black phase Kx, Ky on plane z-1 and the red planes z-2..z; u of
// plane z+2 and Kx, Ky of plane z+1 are in flight. A thread that has passed step z's
// second barrier may start step z+1 (and overwrite the slot four planes back) while
// others still run step z's black phase, which reads nothing that old: four slots
// suffice for every ring.
constexpr int kSlots = 4;
constexpr int kBulkSlots = 5;  // plane ring of the bulk-copy variant
constexpr int kArrays = 6;     // u, Kx, Ky, Kz, Dinv, g (bulk-copy variant)

template <int K>
struct StepK {
  static constexpr int value = K;
};

template <typename T, int BX, int BY>
struct FusedLayout {
  static_assert(BY % 4 == 0, "the tile height must be a multiple of 4 (column quads)");
  static constexpr int kStaged = 3;                 // u, Kx, Ky
  static constexpr int E = 16 / (int)sizeof(T);     // elements per 16-byte copy
  static constexpr int W2 = BX + 4, H2 = BY + 4;    // tile + 2-ring
  static constexpr int W1 = BX + 2, H1 = BY + 2;    // tile + 1-ring
  static constexpr int NCH = (W2 + 2 * E - 2) / E;  // 16-byte copies per staged row, any alignment
  static constexpr int RW = NCH * E;                // staged row pitch (elements)
  // staged plane: rows -1 .. H2 (rows -1 and H2 are padding, never staged, read only
  // where the value is unused), row r at (r + 1) RW
  static constexpr int PLANE = (H2 + 2) * RW;
  static constexpr int ASTRIDE = kSlots * PLANE;    // one staged array, all slots
  static constexpr int RP = W1 + (W1 & 1);          // red-plane row pitch (even)
  // red plane: the plane after its red phase on staged rows -1 .. H2 (only rows 1 ..
  // H2-2, the 1-ring, are written; the others are padding read only where the value is
  // unused), staged row r at (r + 1) RP
  static constexpr int RPLANE = (H2 + 2) * RP;
  static constexpr int threads = W2 * (H2 / 4);     // one thread per column quad
  static constexpr int pairs = H2 * NCH;            // (row, copy) pairs of a staged plane
  static constexpr int per_thread = (pairs + threads - 1) / threads;
  static constexpr size_t bytes = sizeof(T) * ((size_t)kStaged * ASTRIDE + (size_t)kSlots * RPLANE);
};

template <typename T, int BX, int BY>
__global__ void __launch_bounds__(FusedLayout<T, BX, BY>::threads, sizeof(T) == 4 ? 3 : 2)
    k_rbgs_fused(int n, int ntx, int ntiles, int zslab, const T* __restrict__ Kx, const T* __restrict__ Ky,
                 const T* __restrict__ Kz, const T* __restrict__ Dinv, const T* __restrict__ g,
                 const T* __restrict__ uin, T* __restrict__ uout, const int* __restrict__ active) {
  using Lay = FusedLayout<T, BX, BY>;
  constexpr int E = Lay::E, W2 = Lay::W2, H2 = Lay::H2, RW = Lay::RW, PLANE = Lay::PLANE, RP = Lay::RP,
                RPLANE = Lay::RPLANE, NT = Lay::threads, NCH = Lay::NCH, PT = Lay::per_thread,
                AS = Lay::ASTRIDE;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* stage = (T*)smem_raw;                     // [array][slot][H2 + 2][RW]: u, Kx, Ky
  T* red = stage + (size_t)Lay::kStaged * AS;  // [slot][H2 + 2][RP]: plane after its red phase
  const T* U = stage;
  const T* SKX = stage + AS;
  const T* SKY = stage + 2 * AS;
  const int s = blockIdx.y, tid = threadIdx.x;
  const int tile = blockIdx.x % ntiles, slab = blockIdx.x / ntiles;
  const int x0 = (tile % ntx) * BX + 1, y0 = (tile / ntx) * BY + 1;  // first owned node
  const int zlo = 1 + slab * zslab, zhi = min(n - 2, zlo + zslab - 1);
  const int n2 = n * n, n3 = n2 * n;
  const size_t base = (size_t)s * (size_t)n3;
  const int ci = tid % W2, r0 = 4 * (tid / W2);  // staged column, first of the four rows
  const int gx = x0 - 2 + ci, gy0 = y0 - 2 + r0;
  const bool xin = gx >= 1 && gx <= n - 2;
  // per-row bits (row r0 + j): red updates (1-ring, interior), outputs (owned, interior)
  int redmask = 0, outmask = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = r0 + j, gy = gy0 + j;
    const bool yin = gy >= 1 && gy <= n - 2;
    if (xin && yin && ci >= 1 && ci <= W2 - 2 && r >= 1 && r <= H2 - 2) redmask |= 1 << j;
    if (xin && yin && ci >= 2 && ci <= W2 - 3 && r >= 2 && r <= H2 - 3) outmask |= 1 << j;
  }
  const int colrow = gy0 * n + gx;  // in-sample offset of (gx, gy0, z = 0)
  if (active && !active[s]) {
    for (int z = zlo; z <= zhi; ++z)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (outmask >> j & 1) uout[base + (size_t)(z * n2 + colrow + j * n)] = uin[base + (size_t)(z * n2 + colrow + j * n)];
    return;
  }
  // 16-byte alignment is a property of the array's element index: sample s starts sb
  // elements past a 16-byte boundary, so in-sample offsets are aligned in the frame
  // shifted by sb
  const int sb = (int)(base & (size_t)(E - 1));
  // this thread's (row, copy) pairs: shifted in-sample offset of the copy's row start
  // (plus k E) and the destination within a staged plane; -1: nothing to copy
  int pr_row[PT], pr_dst[PT];
#pragma unroll
  for (int i = 0; i < PT; ++i) {
    const int q = tid + i * NT;
    const int j = q / NCH, k = q - j * NCH;
    const int gy = y0 - 2 + j;
    const bool on = q < Lay::pairs && gy >= 0 && gy < n;  // rows outside the grid are never read
    pr_row[i] = sb + gy * n + (x0 - 2) + k * E;
    pr_dst[i] = on ? (j + 1) * RW + k * E : -1;
  }
  const T* const ub = uin + base;
  const T* const kxb = Kx + base;
  const T* const kyb = Ky + base;
  // copies of plane z of u (into slot su) and, when zk >= 0, of plane zk of Kx, Ky (slot sk)
  auto issue = [&](int z, int su, int zk, int sk) {
    const bool zu = z >= 0 && z < n, zkk = zk >= 0 && zk < n;
#pragma unroll
    for (int i = 0; i < PT; ++i) {
      if (pr_dst[i] < 0) continue;
      if (zu) {
        const int c = ((z * n2 + pr_row[i]) & ~(E - 1)) - sb;  // in-sample start of the copy
        T* dst = stage + pr_dst[i] + su * PLANE;
        if (c >= 0 && c + E <= n3)
          cp_async16(dst, ub + c);
        else
          *(int4*)dst = make_int4(0, 0, 0, 0);  // outside the sample: never read by an update
      }
      if (zkk) {
        const int c = ((zk * n2 + pr_row[i]) & ~(E - 1)) - sb;
        T* dx = stage + AS + pr_dst[i] + sk * PLANE;
        T* dy = stage + 2 * AS + pr_dst[i] + sk * PLANE;
        if (c >= 0 && c + E <= n3) {
          cp_async16(dx, kxb + c);
          cp_async16(dy, kyb + c);
        } else {
          *(int4*)dx = make_int4(0, 0, 0, 0);
          *(int4*)dy = make_int4(0, 0, 0, 0);
        }
      }
    }
  };
  // register windows of the four rows: entry (p - zs + 1) mod 4 holds plane p
  const T* kzs = Kz + base + colrow;
  const T* dis = Dinv + base + colrow;
  const T* gs = g + base + colrow;
  T kz[4][kSlots], di[4][kSlots], gg[4][kSlots];
  auto load_window = [&](int z, int w) {
    const bool zin = z >= 0 && z < n;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool on = zin && (redmask >> j & 1);
      const int o = z * n2 + j * n;
      kz[j][w] = on ? kzs[o] : T(0);
      di[j][w] = on ? dis[o] : T(0);
      gg[j][w] = on ? gs[o] : T(0);
    }
  };
  // staged index of row r0 - 1 + i (i = 0..5) of a plane whose in-sample offset is zo
  const int cbase = r0 * RW + ci;
  const int rlo = sb + (gy0 - 1) * n + (x0 - 2);
  auto rows_at = [&](int zo, int* I) {
    const int t = zo + rlo;
#pragma unroll
    for (int i = 0; i < 6; ++i) I[i] = cbase + i * RW + ((t + i * n) & (E - 1));
  };
  const int rpb = r0 * RP + (ci - 1);  // red-plane index of staged row r0 - 1 (+ i RP: row r0 - 1 + i)
  const bool cr = ci >= 1 && ci <= W2 - 2;  // a 1-ring column: its rows r0..r0+3 go to the red plane
  const int storemask = cr ? ((r0 >= 1 ? 1 : 0) | 6 | (r0 + 3 <= H2 - 2 ? 8 : 0)) : 0;
  const int zs = zlo - 1, ze = zhi + 1;
  const int par0 = (gx + gy0 + zs) & 1;
  int Ia[kSlots][6];  // staged row indices of planes z-1 .. z+1 (same slot map)

  auto step = [&](auto KC, int z) {
    constexpr int K = decltype(KC)::value;
    constexpr int Im2 = (K + 3) % kSlots, Im1 = K % kSlots, I0 = (K + 1) % kSlots, Ip1 = (K + 2) % kSlots,
                  Ip2 = (K + 3) % kSlots;
    constexpr int S0 = Im1 * PLANE, S1 = I0 * PLANE, S2 = Ip1 * PLANE;
    issue(z + 2 <= ze + 1 ? z + 2 : -1, Ip2, z + 1 <= ze ? z + 1 : -1, Ip1);
    cp_async_commit();
    load_window(z + 1, Ip1);
    rows_at((z + 1) * n2, Ia[Ip1]);
    cp_async_wait1();  // this thread's copies issued before this step have landed
    __syncthreads();   // ... and every thread's
    const int par = par0 ^ ((z - zs) & 1);  // rows r0 + par, r0 + par + 2 are red at z
    const int* Iz = Ia[I0];
    const int* Im = Ia[Im1];
    const int* Ip = Ia[Ip1];
    // rows a = r0 + par, b = a + 2 (staged row indices 1 + par, 3 + par) and neighbours
    const int ia = par ? Iz[2] : Iz[1], ib = par ? Iz[4] : Iz[3];
    const int iam = par ? Iz[1] : Iz[0], iab = par ? Iz[3] : Iz[2], ibp = par ? Iz[5] : Iz[4];
    T* rz = red + I0 * RPLANE;
    const bool zr = z >= 1 && z <= n - 2;
    {
      const T ua_m = U[S1 + iam], u_ab = U[S1 + iab], ub_p = U[S1 + ibp];
      T va = U[S1 + ia], vb = U[S1 + ib];
      if (zr && (redmask >> par & 1)) {
        T acc = par ? gg[1][I0] : gg[0][I0];
        acc = fma(SKX[S1 + ia - 1], U[S1 + ia - 1], acc);
        acc = fma(SKX[S1 + ia], U[S1 + ia + 1], acc);
        acc = fma(SKY[S1 + iam], ua_m, acc);
        acc = fma(SKY[S1 + ia], u_ab, acc);
        acc = fma(par ? kz[1][Im1] : kz[0][Im1], U[S0 + (par ? Im[2] : Im[1])], acc);
        acc = fma(par ? kz[1][I0] : kz[0][I0], U[S2 + (par ? Ip[2] : Ip[1])], acc);
        va = acc * (par ? di[1][I0] : di[0][I0]);
      }
      if (zr && (redmask >> (par + 2) & 1)) {
        T acc = par ? gg[3][I0] : gg[2][I0];
        acc = fma(SKX[S1 + ib - 1], U[S1 + ib - 1], acc);
        acc = fma(SKX[S1 + ib], U[S1 + ib + 1], acc);
        acc = fma(SKY[S1 + iab], u_ab, acc);
        acc = fma(SKY[S1 + ib], ub_p, acc);
        acc = fma(par ? kz[3][Im1] : kz[2][Im1], U[S0 + (par ? Im[4] : Im[3])], acc);
        acc = fma(par ? kz[3][I0] : kz[2][I0], U[S2 + (par ? Ip[4] : Ip[3])], acc);
        vb = acc * (par ? di[3][I0] : di[2][I0]);
      }
      // rows r0 .. r0+3 after the red phase: red rows take va / vb, black rows keep u
      const T w0 = par ? ua_m : va, w1 = par ? va : u_ab, w2 = par ? u_ab : vb, w3 = par ? vb : ub_p;
      if (storemask & 1) rz[rpb + RP] = w0;
      if (storemask & 2) rz[rpb + 2 * RP] = w1;
      if (storemask & 4) rz[rpb + 3 * RP] = w2;
      if (storemask & 8) rz[rpb + 4 * RP] = w3;
    }
    __syncthreads();
    const int zb = z - 1;
    if (outmask && zb >= zlo && zb <= zhi) {
      const T* Rb = red + Im1 * RPLANE;  // plane z-1 after red
      const T* Rm = red + Im2 * RPLANE;  // plane z-2 after red
      // black rows of plane z-1 are a and b (the red rows of plane z)
      const int ja = par ? Im[2] : Im[1], jb = par ? Im[4] : Im[3];
      const int jam = par ? Im[1] : Im[0], jab = par ? Im[3] : Im[2];
      const int ra = rpb + (1 + par) * RP, rbb = ra + 2 * RP;
      const T ya = Rb[ra - RP], yab = Rb[ra + RP], yb = Rb[rbb + RP];
      T va = T(0), vb = T(0);
      if (outmask >> par & 1) {
        T acc = par ? gg[1][Im1] : gg[0][Im1];
        acc = fma(SKX[S0 + ja - 1], Rb[ra - 1], acc);
        acc = fma(SKX[S0 + ja], Rb[ra + 1], acc);
        acc = fma(SKY[S0 + jam], ya, acc);
        acc = fma(SKY[S0 + ja], yab, acc);
        acc = fma(par ? kz[1][Im2] : kz[0][Im2], Rm[ra], acc);
        acc = fma(par ? kz[1][Im1] : kz[0][Im1], rz[ra], acc);
        va = acc * (par ? di[1][Im1] : di[0][Im1]);
      }
      if (outmask >> (par + 2) & 1) {
        T acc = par ? gg[3][Im1] : gg[2][Im1];
        acc = fma(SKX[S0 + jb - 1], Rb[rbb - 1], acc);
        acc = fma(SKX[S0 + jb], Rb[rbb + 1], acc);
        acc = fma(SKY[S0 + jab], yab, acc);
        acc = fma(SKY[S0 + jb], yb, acc);
        acc = fma(par ? kz[3][Im2] : kz[2][Im2], Rm[rbb], acc);
        acc = fma(par ? kz[3][Im1] : kz[2][Im1], rz[rbb], acc);
        vb = acc * (par ? di[3][Im1] : di[2][Im1]);
      }
      // rows r0 .. r0+3 of plane z-1: black results and the red rows' values
      const T o0 = par ? ya : va, o1 = par ? va : yab, o2 = par ? yab : vb, o3 = par ? vb : yb;
      T* out = uout + base + (size_t)(zb * n2 + colrow);
      if (outmask & 1) out[0] = o0;
      if (outmask >> 1 & 1) out[n] = o1;
      if (outmask >> 2 & 1) out[2 * n] = o2;
      if (outmask >> 3 & 1) out[3 * n] = o3;
    }
  };

  // prologue: u of planes zs-1, zs, zs+1 and Kx, Ky of plane zs; windows of zs-2 .. zs
  load_window(zs - 2, kSlots - 1);
  load_window(zs - 1, 0);
  load_window(zs, 1);
  rows_at((zs - 1) * n2, Ia[0]);
  rows_at(zs * n2, Ia[1]);
  issue(zs - 1, 0, -1, 0);
  issue(zs, 1, zs, 1);
  cp_async_commit();
  issue(zs + 1, 2, -1, 0);
  cp_async_commit();
  for (int z = zs; z <= ze; z += kSlots) {
    step(StepK<0>{}, z);
    if (z + 1 > ze) break;
    step(StepK<1>{}, z + 1);
    if (z + 2 > ze) break;
    step(StepK<2>{}, z + 2);
    if (z + 3 > ze) break;
    step(StepK<3>{}, z + 3);
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
template <typename T, int BX, int BY>
struct BulkLayout {
  static constexpr int W2 = BX + 4, H2 = BY + 4;
  static constexpr int W1 = BX + 2, H1 = BY + 2;
  static constexpr int P1 = W1 * H1;
  static constexpr int EPV = 16 / (int)sizeof(T);  // elements per 16 bytes
  static constexpr int RP = ((W2 + 2 * EPV + EPV - 1) / EPV) * EPV;  // staged row pitch
  static constexpr int PLANE = H2 * RP;
  static constexpr int threads = W2 * H2;
  static constexpr size_t stage_bytes = sizeof(T) * (size_t)kArrays * kBulkSlots * PLANE;
  static constexpr size_t red_off = stage_bytes;
  static constexpr size_t offs_off = red_off + sizeof(T) * 3 * (size_t)P1;
  static constexpr size_t mbar_off = (offs_off + sizeof(int) * kBulkSlots * H2 + 7) & ~(size_t)7;
  static constexpr size_t flag_off = mbar_off + 8 * kBulkSlots;
  static constexpr size_t bytes = flag_off + 16;
};

template <typename T, int BX, int BY>
__global__ void __launch_bounds__(BulkLayout<T, BX, BY>::threads)
    k_rbgs_bulk(int n, int ntx, int ntiles, int zslab, const T* __restrict__ Kx, const T* __restrict__ Ky,
                const T* __restrict__ Kz, const T* __restrict__ Dinv, const T* __restrict__ g,
                const T* __restrict__ uin, T* __restrict__ uout, const int* __restrict__ active,
                int* __restrict__ err, long long budget) {
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
    for (int k = 0; k < kBulkSlots; ++k) mbar_init(&mbar[k], 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  // row offsets of every slot start at 0 (a slot is read before its first staging only
  // where the value is unused, but its index must stay inside the staging buffer)
  for (int t = tid; t < kBulkSlots * H2; t += Lay::threads) offs[t] = 0;
  // rows outside the grid: zeros in every slot, never copied
  for (int t = tid; t < kArrays * kBulkSlots * H2; t += Lay::threads) {
    const int j = t % H2;
    const int yy = y0 - 2 + j;
    if (yy < 0 || yy >= n)
      for (int e = 0; e < RP; ++e) stage[(size_t)(t / H2) * PLANE + (size_t)j * RP + e] = T(0);
  }
  __syncthreads();
  const int zs = zlo - 1, ze = zhi + 1;
  // warp 0 stages plane z (rows of all six arrays) into slot z % kBulkSlots
  auto issue = [&](int z) {
    if (warp != 0 || z < 0 || z >= n) return;
    const int slot = z % kBulkSlots;
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
    fence_proxy_async();
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
      T* dst = stage + ((size_t)(a * kBulkSlots + slot) * H2 + j) * RP;
      bulk_g2s(dst, src[a] + A, (unsigned)((E - A) * sizeof(T)), &mbar[slot]);
    }
  };
  // the k-th plane staged into a slot completes that slot's barrier phase k: the
  // parity counts uses of the slot from the first staged plane of this CTA
  const int pstart = max(zs - 1, 0);
  auto parity = [&](int z) { return (unsigned)(((z - pstart) / kBulkSlots) & 1); };
  auto wait_plane = [&](int z) {
    if (z < 0 || z >= n) return;
    if (!mbar_wait_bounded(&mbar[z % kBulkSlots], parity(z), budget)) {
      *abort_flag = 1;
      atomicExch(err, 1);
    }
  };
  // element (array a, plane slot sl, staged row j, column i of the tile + 2-ring)
  // (bounds-checked: an index outside the staging buffer records error 2 and reads 0)
  auto at = [&](int a, int sl, int j, int i) -> T {
    const long long k = ((long long)(a * kBulkSlots + sl) * H2 + j) * RP + offs[sl * H2 + j] + i;
    if ((unsigned long long)k >= (unsigned long long)kArrays * kBulkSlots * PLANE) {
      atomicExch(err, 2);
      return T(0);
    }
    return stage[k];
  };
  T kz_m2 = T(0);
  int last_issued = min(zs + 1, n - 1);  // highest plane whose copies were issued
  issue(zs - 1);
  issue(zs);
  issue(zs + 1);
  wait_plane(zs - 1);
  wait_plane(zs);
  for (int z = zs; z <= ze; ++z) {
    if (z + 2 <= ze + 1) {
      issue(z + 2);
      last_issued = min(z + 2, n - 1);
    }
    wait_plane(z + 1);
    const int sz = z % kBulkSlots, szm = (z + kBulkSlots - 1) % kBulkSlots, szp = (z + 1) % kBulkSlots;
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
      // a wait ran out: drain the copies of the last kBulkSlots issued planes (any of them
      // may still be in flight, the early waits included; a completed phase returns at
      // once), each bounded by kDrainBudget, then every thread leaves
      for (int p = max(pstart, last_issued - (kBulkSlots - 1)); p <= last_issued; ++p)
        mbar_wait_bounded(&mbar[p % kBulkSlots], parity(p), kDrainBudget);
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
    __syncthreads();  // slot (z+3) % kBulkSlots = plane z-2 is reused by the next issue
  }
}

template <typename T, int BX, int BY>
int launch_bulk(int n, int B, const T* Kx, const T* Ky, const T* Kz, const T* Dinv, const T* g, const T* uin,
                T* uout, const int* active, int* err, cudaStream_t st, long long budget) {
  using Lay = BulkLayout<T, BX, BY>;
  const int m = n - 2;
  const int ntx = (m + BX - 1) / BX, nty = (m + BY - 1) / BY, ntiles = ntx * nty;
  int slabs = (int)((152LL * 12 + (long long)ntiles * B - 1) / ((long long)ntiles * B));
  if (slabs > m / 8) slabs = m / 8;
  if (slabs < 1) slabs = 1;
  const int zslab = (m + slabs - 1) / slabs;
  slabs = (m + zslab - 1) / zslab;
  dim3 grid((unsigned)(ntiles * slabs), (unsigned)B);
  k_rbgs_bulk<T, BX, BY><<<grid, Lay::threads, Lay::bytes, st>>>(n, ntx, ntiles, zslab, Kx, Ky, Kz, Dinv, g, uin,
                                                                 uout, active, err, budget);
  return MLMC_OK;
}

// z-slab count of a fused sweep: each slab re-stages four planes of u, Kx, Ky and six
// of Kz, 1/D, g around its ends, and the CTAs of a launch spread over 152 SMs, so the
// count minimises (CTAs per SM, rounded up) x (planes a CTA streams); slabs of at least
// 8 planes. The result of the sweep does not depend on the split.
inline int fused_slabs(int m, long long ctas_per_slab) {
  int best = 1;
  long long best_cost = -1;
  for (int sl = 1; sl <= (m / 8 > 1 ? m / 8 : 1); ++sl) {
    const int zslab = (m + sl - 1) / sl, used = (m + zslab - 1) / zslab;
    const long long per_sm = (ctas_per_slab * used + 151) / 152;
    const long long cost = per_sm * (zslab + 6);
    if (best_cost < 0 || cost < best_cost) best_cost = cost, best = used;
  }
  return best;
}

template <typename T, int BX, int BY>
int launch_shape(int n, int B, const T* Kx, const T* Ky, const T* Kz, const T* Dinv, const T* g, const T* uin,
                 T* uout, const int* active, cudaStream_t st) {
  using Lay = FusedLayout<T, BX, BY>;
  const int m = n - 2;
  const int ntx = (m + BX - 1) / BX, nty = (m + BY - 1) / BY, ntiles = ntx * nty;
  int slabs = fused_slabs(m, (long long)ntiles * B);
  const int zslab = (m + slabs - 1) / slabs;
  slabs = (m + zslab - 1) / zslab;
  dim3 grid((unsigned)(ntiles * slabs), (unsigned)B);
  k_rbgs_fused<T, BX, BY><<<grid, Lay::threads, Lay::bytes, st>>>(n, ntx, ntiles, zslab, Kx, Ky, Kz, Dinv, g, uin,
                                                                  uout, active);
  return MLMC_OK;
}

}  // namespace

// The dynamic shared-memory opt-in of each kernel instance, set once per process (the
// library drives one device per process). Function-local statics make the first call
// thread-safe; it happens before any stream capture because solve setup configures
// every fused level first.
template <typename T, int BX, int BY>
int configure_shape() {
  using Lay = FusedLayout<T, BX, BY>;
  static const cudaError_t e = cudaFuncSetAttribute(k_rbgs_fused<T, BX, BY>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes);
  MLMC_CUDA_TRY(e);
  return MLMC_OK;
}

template <typename T, int BX, int BY>
int configure_bulk() {
  using Lay = BulkLayout<T, BX, BY>;
  static const cudaError_t e = cudaFuncSetAttribute(k_rbgs_bulk<T, BX, BY>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes);
  MLMC_CUDA_TRY(e);
  return MLMC_OK;
}

template <typename T>
int rbgs_fused_configure(int shape) {
  switch (shape) {
    case kTile32x16: return configure_shape<T, 32, 16>();
    case kTile64x8: return configure_shape<T, 64, 8>();
    case kBulk32x8: return configure_bulk<T, 32, 8>();
    case kBulk32x16: return configure_bulk<T, 32, 16>();
    case kBulk64x8: return configure_bulk<T, 64, 8>();
    default: return configure_shape<T, 32, 8>();
  }
}
template int rbgs_fused_configure<float>(int);
template int rbgs_fused_configure<double>(int);

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
                     const T* uin, T* uout, const int* active, int* err, cudaStream_t st, double active_samples) {
  const double interior = (double)(n - 2) * (n - 2) * (n - 2);
  const bool bulk = shape == kBulk32x8 || shape == kBulk32x16 || shape == kBulk64x8;
  const char* cls = bulk ? (sizeof(T) == 4 ? "rbgs_bulk_f32" : "rbgs_bulk_f64")
                         : (sizeof(T) == 4 ? "rbgs_fused_f32" : "rbgs_fused_f64");
  // one full sweep: 7 words per interior node (u read + write, Kx, Ky, Kz, Dinv, g), 13 flops
  MLMC_TRY(rbgs_fused_configure<T>(shape));
  // (masked samples are copied, not smoothed: the work counts the active ones)
  prof::Scope scope(prof::sized(cls, n), active_samples * interior * 7.0 * sizeof(T), active_samples * interior * 13.0,
                    st);
  const long long budget = wait_budget_clocks();
  switch (shape) {
    case kTile32x16:
      return launch_shape<T, 32, 16>(n, B, Kx, Ky, Kz, Dinv, g, uin, uout, active, st);
    case kTile64x8:
      return launch_shape<T, 64, 8>(n, B, Kx, Ky, Kz, Dinv, g, uin, uout, active, st);
    case kBulk32x8:
      return launch_bulk<T, 32, 8>(n, B, Kx, Ky, Kz, Dinv, g, uin, uout, active, err, st, budget);
    case kBulk32x16:
      return launch_bulk<T, 32, 16>(n, B, Kx, Ky, Kz, Dinv, g, uin, uout, active, err, st, budget);
    case kBulk64x8:
      return launch_bulk<T, 64, 8>(n, B, Kx, Ky, Kz, Dinv, g, uin, uout, active, err, st, budget);
    default:
      return launch_shape<T, 32, 8>(n, B, Kx, Ky, Kz, Dinv, g, uin, uout, active, st);
  }
}

template int rbgs_fused_sweep<float>(int, int, int, const float*, const float*, const float*, const float*,
                                     const float*, const float*, float*, const int*, int*, cudaStream_t, double);
template int rbgs_fused_sweep<double>(int, int, int, const double*, const double*, const double*, const double*,
                                      const double*, const double*, double*, const int*, int*, cudaStream_t,
                                      double);

}  // namespace mlmc
