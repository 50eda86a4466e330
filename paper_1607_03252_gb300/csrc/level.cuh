// The batched MLMC level pipeline, for the service (internal interface).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlmc.h"

namespace mlmc {

// Device bytes one batch of b samples of a level (fine grid nf, coarse grid nc, 0 for
// level 0) holds while it runs.
size_t level_batch_bytes(int b, int nf, int nc, const mlmc_field_cfg& fc, int precision, int accel);

// Runs b samples (host ids) through field, fine and coarse solves and QoI on `st`,
// allocating and releasing the batch's device memory; host outputs of b entries.
// *n_unconv counts solves that missed rtol. Blocking.
int run_level_batch_host(const mlmc_field_cfg& fc, const mg_cfg& mc, int nf, int nc, const uint64_t* ids_host,
                         int b, double* Qf, double* Qc, int* cyc_f, int* cyc_c, int* n_unconv, cudaStream_t st);

// Checks field and solver parameters (MLMC_OK or MLMC_ERR_INVALID with the error text set).
int validate_level_cfg(const mlmc_field_cfg& fc, const mg_cfg& mc);

}  // namespace mlmc
