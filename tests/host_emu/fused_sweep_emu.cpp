// Host emulation of the fused red-black sweep kernel (k_rbgs_fused): the kernel body,
// extracted from the CUDA source, runs with one std::thread per CUDA thread, a
// std::barrier for __syncthreads, cp.async as an immediate 16-byte copy that asserts
// 16-byte alignment of both addresses, and shared memory / grids in exact-size heap
// buffers (built with -fsanitize=address, every out-of-bounds access aborts). Shared
// memory starts filled with NaN patterns, so a read of a slot that was never staged
// shows up as a wrong result. Each case compares the emulated sweep bitwise with a
// sequential red-then-black sweep written out in plain loops (same FMA order).
#include <algorithm>
#include <barrier>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <thread>
#include <vector>

struct dim3 {
  unsigned x = 1, y = 1, z = 1;
  dim3() {}
  dim3(unsigned a, unsigned b = 1, unsigned c = 1) : x(a), y(b), z(c) {}
};
thread_local dim3 threadIdx, blockIdx;
static dim3 gridDim, blockDim;
static std::barrier<>* g_bar = nullptr;
static inline void __syncthreads() { g_bar->arrive_and_wait(); }
static unsigned char* g_smem = nullptr;
using std::fma;
using std::max;
using std::min;
static inline void cp_async16(void* dst, const void* src) {
  if (((uintptr_t)dst & 15) || ((uintptr_t)src & 15)) {
    fprintf(stderr, "misaligned 16-byte copy: dst=%p src=%p\n", dst, src);
    abort();
  }
  std::memcpy(dst, src, 16);
}
static inline void emu_zero16(void* dst) {
  if ((uintptr_t)dst & 15) {
    fprintf(stderr, "misaligned 16-byte store %p\n", dst);
    abort();
  }
  std::memset(dst, 0, 16);
}
static inline void cp_async_commit() {}
static inline void cp_async_wait1() {}
typedef void* cudaStream_t;
#define MLMC_OK 0
template <typename T, int BX, int BY, typename... A>
void emu_launch(dim3 grid, A... args);
#define emu_smem g_smem
#include "fused_sweep.inc"
#undef emu_smem

template <typename T, int BX, int BY, typename... A>
void emu_launch(dim3 grid, A... args) {
  using Lay = FusedLayout<T, BX, BY>;
  gridDim = grid;
  blockDim = dim3(Lay::threads);
  for (unsigned by = 0; by < grid.y; ++by)
    for (unsigned bx = 0; bx < grid.x; ++bx) {
      unsigned char* sm = (unsigned char*)aligned_alloc(128, (Lay::bytes + 127) / 128 * 128);
      std::memset(sm, 0xFF, Lay::bytes);
      g_smem = sm;
      std::barrier<> bar(Lay::threads);
      g_bar = &bar;
      std::vector<std::thread> th;
      for (int t = 0; t < Lay::threads; ++t)
        th.emplace_back([&, t] {
          threadIdx = dim3(t);
          blockIdx = dim3(bx, by);
          k_rbgs_fused<T, BX, BY>(args...);
        });
      for (auto& x : th) x.join();
      free(sm);
    }
}

template <typename T>
void ref_sweep(int n, int B, const T* Kx, const T* Ky, const T* Kz, const T* Di, const T* g, T* u) {
  const size_t n2 = (size_t)n * n, n3 = n2 * n;
  for (int c = 0; c < 2; ++c)
    for (int s = 0; s < B; ++s)
      for (int z = 1; z < n - 1; ++z)
        for (int y = 1; y < n - 1; ++y)
          for (int x = 1; x < n - 1; ++x) {
            if (((x + y + z) & 1) != c) continue;
            const size_t p = s * n3 + z * n2 + (size_t)y * n + x;
            T acc = g[p];
            acc = fma(Kx[p - 1], u[p - 1], acc);
            acc = fma(Kx[p], u[p + 1], acc);
            acc = fma(Ky[p - n], u[p - n], acc);
            acc = fma(Ky[p], u[p + n], acc);
            acc = fma(Kz[p - n2], u[p - n2], acc);
            acc = fma(Kz[p], u[p + n2], acc);
            u[p] = acc * Di[p];
          }
}

template <typename T, int BX, int BY>
int run(int n, int B, int inactive) {
  const size_t n3 = (size_t)n * n * n, N = B * n3;
  std::mt19937_64 rng(n * 131 + B);
  std::uniform_real_distribution<double> U(0.1, 1.0);
  auto boundary = [&](size_t i) {
    const size_t r = i % n3;
    const int z = (int)(r / (n * n)), y = (int)((r / n) % n), x = (int)(r % n);
    return x == 0 || y == 0 || z == 0 || x == n - 1 || y == n - 1 || z == n - 1;
  };
  auto mk = [&](bool bnd0) {
    T* a = (T*)malloc(N * sizeof(T));
    for (size_t i = 0; i < N; ++i) a[i] = (bnd0 && boundary(i)) ? T(0) : (T)U(rng);
    return a;
  };
  T *Kx = mk(false), *Ky = mk(false), *Kz = mk(false), *Di = mk(false), *g = mk(true), *u = mk(true);
  T* out = (T*)calloc(N, sizeof(T));
  int* act = (int*)malloc(B * sizeof(int));
  for (int s = 0; s < B; ++s) act[s] = (s == inactive) ? 0 : 1;
  std::vector<T> want(u, u + N);
  ref_sweep<T>(n, B, Kx, Ky, Kz, Di, g, want.data());
  for (int s = 0; s < B; ++s)
    if (!act[s]) std::copy(u + s * n3, u + (s + 1) * n3, want.begin() + s * n3);
  launch_shape<T, BX, BY>(n, B, Kx, Ky, Kz, Di, g, u, out, act, nullptr);
  size_t bad = 0;
  for (size_t i = 0; i < N; ++i)
    if (std::memcmp(&out[i], &want[i], sizeof(T)) != 0) ++bad;
  printf("%s %dx%d n=%d B=%d inactive=%d: %s (%zu differing nodes)\n", sizeof(T) == 4 ? "f32" : "f64", BX, BY, n,
         B, inactive, bad ? "FAIL" : "ok", bad);
  free(Kx); free(Ky); free(Kz); free(Di); free(g); free(u); free(out); free(act);
  return bad ? 1 : 0;
}

int main(int argc, char** argv) {
  int fails = 0;
  const int ns[] = {5, 9, 17, 33};
  for (int n : ns) {
    fails += run<float, 32, 8>(n, 2, -1);
    fails += run<float, 32, 16>(n, 4, 1);
    fails += run<float, 64, 8>(n, 1, -1);
    fails += run<double, 32, 8>(n, 2, 0);
    fails += run<double, 32, 16>(n, 1, -1);
    fails += run<double, 64, 8>(n, 3, -1);
  }
  if (argc > 1) {  // several x tiles, partial tiles, z slabs
    fails += run<float, 32, 16>(65, 2, -1);
    fails += run<double, 64, 8>(65, 1, -1);
    fails += run<float, 64, 8>(129, 1, -1);
  }
  printf(fails ? "FAILURES %d\n" : "all ok\n", fails);
  return fails != 0;
}
