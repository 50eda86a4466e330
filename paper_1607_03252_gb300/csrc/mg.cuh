// Batched geometric multigrid on structured (2^p+1)^3 grids (internal interface).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlmc.h"

namespace mlmc {

// Arguments of one batched solve A u = f on the grid with n nodes per axis.
// The nodal coefficient of the solve grid is the injection k0[s][st0 z][st0 y][st0 x]
// of an FP64 grid with n_k0 = (n - 1) st0 + 1 nodes per axis (st0 = 1: k0 is the
// solve grid itself; st0 = 2: the coarse solve of an MLMC pair reads the fine field).
struct MGSolveArgs {
  const double* k0 = nullptr;
  int n_k0 = 0;
  int st0 = 1;
  const double* f = nullptr;  // B x n^3 FP64, NULL = 1
  double* u = nullptr;        // B x n^3 FP64, initial guess in, solution out
  int n = 0;
  int B = 0;
  mg_cfg cfg{};
};

// Device workspace of a solve (bytes, 256-aligned pieces).
size_t mg_workspace_bytes(int B, int n, int precision, int accel);

// Enqueues the solve on `st` and synchronises it once per cycle to test convergence.
// cycles_host / relres_host: B entries each (may be NULL); cycles_dev / relres_dev:
// optional device copies. *n_unconverged receives the number of samples that missed rtol.
int mg_solve_dev(const MGSolveArgs& a, void* workspace, cudaStream_t st, int* cycles_host, double* relres_host,
                 int* n_unconverged, int* cycles_dev = nullptr, double* relres_dev = nullptr);

// Q[s] = mean of u over [0.25,0.75]^3 (trapezoid) for B samples of an n^3 grid.
size_t qoi_scratch_bytes(int B, int n);
int qoi_dev(const double* u, int n, int B, double* Q_dev, void* scratch, cudaStream_t st);

// Q[s] for the quantity of interest `qoi` (MLMC_QOI_*) of the B solutions u on grid n; the
// flux reads the FP64 field k0 (n_k0 nodes per axis, stride st0 to grid n). scratch:
// qoi_scratch_bytes(B, n).
int qoi_any(int qoi, const double* u, int n, int B, double* Q_dev, void* scratch, const double* k0, int n_k0,
            int st0, cudaStream_t st);

// uf = trilinear interpolation of uc ((nf+1)/2)^3 onto the nf^3 grid (0 on the boundary):
// the initial guess of a fine solve from the coarse solution of the same realisation.
int interpolate_dev(const double* uc, int nf, int B, double* uf, cudaStream_t st);

}  // namespace mlmc
