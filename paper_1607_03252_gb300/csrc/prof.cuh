// In-library launch accounting: every kernel launch of the library is counted per
// kernel class together with its algorithmic bytes and flops; when timing is enabled,
// CUDA events are recorded around each launch on the launching stream so that the
// device time per class can be read back (mlmc_profile_* in include/mlmc.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mlmc {
namespace prof {

bool timing_enabled();
// Records the start of one launch of `cls`; returns a token for end().
int begin(const char* cls, double bytes, double flops, cudaStream_t st);
void end(int token, cudaStream_t st);

// RAII scope around one kernel launch.
struct Scope {
  int tok;
  cudaStream_t st;
  Scope(const char* cls, double bytes, double flops, cudaStream_t s) : tok(begin(cls, bytes, flops, s)), st(s) {}
  ~Scope() { end(tok, st); }
};

}  // namespace prof
}  // namespace mlmc

// Launch `launch_expr` (a kernel<<<...>>>(...) expression) accounted under `cls`.
#define MLMC_LAUNCH(cls, bytes, flops, st, launch_expr)                        \
  do {                                                                          \
    ::mlmc::prof::Scope _mlmc_scope((cls), (double)(bytes), (double)(flops), (st)); \
    launch_expr;                                                                \
  } while (0)
