// Random-field evaluation on the device (feature draw + separable phasor sum).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlmc.h"

namespace mlmc {

// Bytes of device scratch field_eval_dev needs for B samples, M features, n nodes per axis.
size_t field_scratch_bytes(int B, int M, int n);

// Arithmetic of the log k sum: double-float on the FP32 pipe with one (y, z) line per
// thread, FP64, double-float with flattened outputs, or bf16 slices on the tensor cores with
// exact FP32 group sums (on grids with (n - 1) a multiple of 16 from n = 17, other grids take
// the double-float line form): kFieldTC (the default) runs the volume on tcgen05 from n = 65
// and on the warp-level mma.sync below, kFieldTCWarp on mma.sync everywhere.
enum { kFieldDF32Line = 0, kFieldFP64 = 1, kFieldDF32 = 2, kFieldTC = 3, kFieldTCWarp = 4 };

// The arithmetic field_eval_dev uses by default: kFieldTC, or the value of the environment
// variable MLMC_FIELD_ARITH (0..4) read once.
int field_arith_default();

// 1 if a bounded wait of a tensor-core field block has run out since the last call (the
// block's nodes hold NaN); clears the flag. Reads it on stream st and synchronises st.
int field_wait_error_take(cudaStream_t st);

// The next `launches` launches of the tcgen05 field kernel also wait on an mbarrier that
// nothing arrives on (host-side fault injection, mlmc_inject_wait_failure).
void field_inject_wait_failure(int launches);

// k_out[s][z][y][x] = exp(log k) at the n^3 nodes for the B ids in ids_dev (device).
// dtype MLMC_F64 or MLMC_F32. scratch: field_scratch_bytes(B, M, n) bytes, 256-aligned.
int field_eval_dev(const mlmc_field_cfg& cfg, const uint64_t* ids_dev, int B, int n, int dtype, void* k_out,
                   void* scratch, cudaStream_t st, int arith = -1);

}  // namespace mlmc
