// Process-wide tuning table: for a grid size and precision, the smoother
// implementation and the sweep count nu (V(nu, nu)) chosen by mlmc_autotune.
#pragma once

namespace mlmc {

// Stores the choice for (n, precision).
void tune_store(int n, int precision, int smoother, int nu);
// Looks up (n, precision); returns false if untuned.
bool tune_lookup(int n, int precision, int* smoother, int* nu);
void tune_clear();

// Resolves MLMC_SMOOTH_AUTO and nu1 = nu2 = 0 for a solve on grid n: the tuned values
// if present, else the defaults (two-pass FP64 smoother, fused FP32 smoother with
// 32x8 tiles up to 33^3 and 32x16 above, nu = 2).
void resolve_tuning(int n, int precision, int* smoother, int* nu1, int* nu2);

}  // namespace mlmc
