// SPDE field sampler on the device (Sec. 3.2): white noise, cell-centred multigrid for
// (kappa^2 - Laplace) Z = W on a zero-flux box, k = exp(sqrt(8 pi kappa sigma^2) Z).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlmc.h"

namespace mlmc {

// Solve tolerance and cycle cap of the SPDE solves (relative residual in the 2-norm).
constexpr double kSpdeRtol = 1e-12;
constexpr int kSpdeMaxCycles = 60;

// Bytes of device scratch spde_field_dev needs for B samples of level grid n.
size_t spde_scratch_bytes(int B, int n);

// k_out[s][z][y][x] = exp(log k) at the n^3 nodes of D for the B ids in ids_dev (device),
// with the white noise on the octants of grid n_noise (n itself, or 2n - 1 when grid n is
// the coarse grid of a pair). dtype MLMC_F64 or MLMC_F32. scratch: spde_scratch_bytes(B, n)
// bytes, 256-aligned. Synchronises `st` once per cycle (the convergence test); returns
// MLMC_ERR_NOT_CONVERGED if some sample misses kSpdeRtol in kSpdeMaxCycles cycles.
int spde_field_dev(const mlmc_field_cfg& cfg, const uint64_t* ids_dev, int B, int n, int n_noise, int dtype,
                   void* k_out, void* scratch, cudaStream_t st);

}  // namespace mlmc
