// Fused (both colours, one pass) red-black Gauss-Seidel sweep (internal interface).
#pragma once
#include <cuda_runtime.h>

namespace mlmc {

// x-y tile shapes of the fused sweep (the autotuner chooses among them per grid size).
enum { kTile32x8 = 0, kTile32x16 = 1, kTile64x8 = 2, kTileShapes = 3 };
const char* tile_name(int shape);

// One full red-black sweep over B samples of an n^3 grid: reads uin, writes uout
// (distinct buffers; uout's boundary nodes must already be zero). Samples whose
// active flag is 0 are copied from uin to uout unchanged.
template <typename T>
int rbgs_fused_sweep(int shape, int n, int B, const T* Kx, const T* Ky, const T* Kz, const T* Dinv, const T* g,
                     const T* uin, T* uout, const int* active, cudaStream_t st);

}  // namespace mlmc
