// Random-field evaluation on the device (feature draw + separable phasor sum).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlmc.h"

namespace mlmc {

// Bytes of device scratch field_eval_dev needs for B samples, M features, n nodes per axis.
size_t field_scratch_bytes(int B, int M, int n);

// Arithmetic of the log k sum: double-float on the FP32 pipe with one (y, z) line per
// thread (the default), FP64, or double-float with flattened outputs.
enum { kFieldDF32Line = 0, kFieldFP64 = 1, kFieldDF32 = 2 };

// The arithmetic field_eval_dev uses by default: kFieldDF32Line, or the value of the
// environment variable MLMC_FIELD_ARITH (0..2) read once.
int field_arith_default();

// k_out[s][z][y][x] = exp(log k) at the n^3 nodes for the B ids in ids_dev (device).
// dtype MLMC_F64 or MLMC_F32. scratch: field_scratch_bytes(B, M, n) bytes, 256-aligned.
int field_eval_dev(const mlmc_field_cfg& cfg, const uint64_t* ids_dev, int B, int n, int dtype, void* k_out,
                   void* scratch, cudaStream_t st, int arith = -1);

}  // namespace mlmc
