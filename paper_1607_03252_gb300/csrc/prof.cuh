// In-library launch accounting: every kernel launch of the library is counted per
// kernel class together with its algorithmic bytes and flops; when timing is enabled,
// CUDA events are recorded around each launch on the launching stream so that the
// device time per class can be read back (mlmc_profile_* in include/mlmc.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace mlmc {
namespace prof {

bool timing_enabled();

// Launch tape for CUDA-graph capture: between tape_begin() and tape_end() launches are
// recorded (class, bytes, flops) instead of counted; tape_replay() counts them once per
// replay of the captured graph. Per calling thread.
struct Tape {
  std::vector<std::string> cls;
  std::vector<double> bytes, flops;
};
void tape_begin();
Tape tape_end();
// `scale` multiplies the recorded bytes and flops (the active share of the batch at this
// replay over that at capture).
void tape_replay(const Tape& t, double scale = 1.0);
// Records the start of one launch of `cls`; returns a token for end().
int begin(const char* cls, double bytes, double flops, cudaStream_t st);
void end(int token, cudaStream_t st);

// "base@n": a launch class per grid size (the name is copied when the launch is counted).
const char* sized(const char* base, int n);

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
