// Tuning table (see tune.cuh).
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "tune.cuh"

namespace mlmc {
namespace {
std::mutex g_mu;
std::map<std::pair<int, int>, std::pair<int, int>> g_table;
}  // namespace

void tune_store(int n, int precision, int smoother, int nu) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table[{n, precision}] = {smoother, nu};
}

bool tune_lookup(int n, int precision, int* smoother, int* nu) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find({n, precision});
  if (it == g_table.end()) return false;
  *smoother = it->second.first;
  *nu = it->second.second;
  return true;
}

void tune_clear() {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table.clear();
}

void resolve_tuning(int n, int precision, int* smoother, int* nu1, int* nu2) {
  int ts = 0, tnu = 0;
  const bool tuned = tune_lookup(n, precision, &ts, &tnu);
  if (*smoother == MLMC_SMOOTH_AUTO) {
    // untuned grids: the two-pass colour sweep, measured fastest on GB300 at every grid
    // size in both precisions (the fused sweeps stay available to the autotuner)
    *smoother = tuned ? ts : MLMC_SMOOTH_TWO_PASS;
  }
  if (*nu1 == 0 && *nu2 == 0) {
    const int nu = tuned ? tnu : 2;
    *nu1 = nu;
    *nu2 = nu;
  }
}

}  // namespace mlmc
