// Fused (both colours, one pass) red-black Gauss-Seidel sweep (internal interface).
#pragma once
#include <cuda_runtime.h>

namespace mlmc {

// x-y tile shapes of the fused sweep (the autotuner chooses among them per grid size).
// kTile*: cp.async element staging; kBulk*: TMA bulk row copies on mbarriers.
enum { kTile32x8 = 0, kTile32x16 = 1, kTile64x8 = 2, kBulk32x8 = 3, kBulk32x16 = 4, kBulk64x8 = 5 };
const char* tile_name(int shape);

// One full red-black sweep over B samples of an n^3 grid: reads uin, writes uout
// (distinct buffers; uout's boundary nodes must already be zero). Samples whose
// active flag is 0 are copied from uin to uout unchanged. The bulk-copy variants set
// *err (device) to 1 if a staging wait runs out of its time budget (wait_budget_clocks()
// SM clocks, read at launch).
// Sets the shared-memory attribute of a fused-sweep variant (once per process); must run
// before the variant's first launch, and outside stream capture.
template <typename T>
int rbgs_fused_configure(int shape);

// active_samples: the number of samples whose flag is 1 (launch accounting only).
template <typename T>
int rbgs_fused_sweep(int shape, int n, int B, const T* Kx, const T* Ky, const T* Kz, const T* Dinv, const T* g,
                     const T* uin, T* uout, const int* active, int* err, cudaStream_t st, double active_samples);

}  // namespace mlmc
