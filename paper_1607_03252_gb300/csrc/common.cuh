// Common definitions of the CUDA library: status handling, device arena, small helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <string>

#include "mlmc.h"

namespace mlmc {

// Thread-local last-error text (mlmc_last_error_string).
void set_error(const char* fmt, ...);
const char* last_error();

// Budget, in SM clocks, of every bounded wait inside a kernel (mlmc_set_wait_budget;
// about one second by default).
long long wait_budget_clocks();

#define MLMC_CUDA_TRY(expr)                                                                 \
  do {                                                                                      \
    cudaError_t _e = (expr);                                                                \
    if (_e != cudaSuccess) {                                                                \
      ::mlmc::set_error("%s failed at %s:%d: %s", #expr, __FILE__, __LINE__,                 \
                        cudaGetErrorString(_e));                                            \
      return _e == cudaErrorMemoryAllocation ? MLMC_ERR_OOM : MLMC_ERR_CUDA;                 \
    }                                                                                       \
  } while (0)

#define MLMC_TRY(expr)          \
  do {                          \
    int _s = (expr);            \
    if (_s < 0) return _s;      \
  } while (0)

// A grid size n is valid when n = 2^p + 1 with p >= 2 (5, 9, 17, ...).
inline bool valid_grid(int n) {
  if (n < 5 || n > 4097) return false;
  int m = n - 1;
  return (m & (m - 1)) == 0;
}

// Number of grids of the multigrid hierarchy n -> (n+1)/2 -> ... -> 5.
inline int hierarchy_depth(int n) {
  int d = 1;
  while (n > 5) {
    n = (n + 1) / 2;
    ++d;
  }
  return d;
}

inline size_t cube(int n) { return (size_t)n * (size_t)n * (size_t)n; }

// Stream-ordered device allocation owned by one call: cudaMallocAsync on construction,
// cudaFreeAsync on the same stream when it goes out of scope.
class DevBuf {
 public:
  DevBuf() = default;
  ~DevBuf() { release(); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  int alloc(size_t bytes, cudaStream_t st);
  void release();
  void* get() const { return p_; }
  template <typename T>
  T* as() const { return (T*)p_; }

 private:
  void* p_ = nullptr;
  cudaStream_t st_ = nullptr;
};

// Grid-stride geometry helper.
inline unsigned int blocks_for(size_t work, int threads, size_t cap = 152u * 64u) {
  size_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned int)b;
}

}  // namespace mlmc
