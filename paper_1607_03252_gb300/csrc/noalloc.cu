// mg_solve_batch_noalloc: the batched multigrid solve of mg_solve_batch for callers
// that cannot allocate device memory -- for example code running inside another
// framework whose memory pool or allocator hooks own every device allocation, or an
// embedded runtime with a fixed device-memory budget set at start-up. Its workspace is
// a fixed array in this library's device image instead of a cudaMallocAsync block; the
// caller still owns k, f and u.
#include <mutex>
#include <vector>

#include "common.cuh"
#include "mg.cuh"

namespace mlmc {
namespace {

// 32 MiB: enough for a batch of about 75 samples at 17^3, 11 at 33^3 or 1 at 65^3 in
// FP64. Every GPU that loads the library keeps this array until the process exits.
constexpr size_t kNoAllocBytes = (size_t)32 << 20;
__device__ __align__(256) unsigned char g_noalloc_workspace[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per device and
// kept for the life of the process (the first call on a device does the look-up). The
// cached address is not refreshed after cudaDeviceReset: a process that resets a device
// must not call this entry point on it again.
int workspace_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error("no usable CUDA device: %s", cudaGetErrorString(e));
    return MLMC_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device index %d beyond %d", dev, kMaxDevices);
    return MLMC_ERR_INVALID;
  }
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_workspace);
    if (e != cudaSuccess || !p) {
      set_error("cudaGetSymbolAddress of the no-allocation workspace failed: %s", cudaGetErrorString(e));
      return MLMC_ERR_CUDA;
    }
    g_dev_ptr[dev] = p;
  }
  *out = g_dev_ptr[dev];
  return MLMC_OK;
}

}  // namespace
}  // namespace mlmc

using namespace mlmc;

extern "C" int mg_solve_batch_noalloc(const mg_cfg* cfg, int batch, int n, const double* k, const double* f,
                                      double* u, mg_stats* stats_host, void* stream) {
  if (!cfg || !k || !u) {
    set_error("mg_solve_batch_noalloc: cfg, k and u must not be NULL");
    return MLMC_ERR_INVALID;
  }
  if (cfg->nu1 < 0 || cfg->nu1 > 8 || cfg->nu2 < 0 || cfg->nu2 > 8 || cfg->max_cycles < 1 ||
      cfg->max_cycles > 1000 || !(cfg->rtol < 1.0) ||
      (cfg->precision != MLMC_PREC_F64 && cfg->precision != MLMC_PREC_MIXED) ||
      cfg->smoother < MLMC_SMOOTH_AUTO || cfg->smoother > MLMC_SMOOTH_SPLIT ||
      (cfg->accel != MLMC_ACCEL_NONE && cfg->accel != MLMC_ACCEL_CG) ||
      (cfg->disc != MLMC_DISC_FV && cfg->disc != MLMC_DISC_FE) ||
      (cfg->disc == MLMC_DISC_FE && cfg->precision != MLMC_PREC_F64) || cfg->engine < MLMC_ENGINE_AUTO ||
      cfg->engine > MLMC_ENGINE_CTA) {
    set_error("mg_solve_batch_noalloc: invalid mg_cfg (FMG is not offered here; P1 elements need FP64)");
    return MLMC_ERR_INVALID;
  }
  if (!valid_grid(n) || batch < 1 || batch > 65535) {
    set_error("mg_solve_batch_noalloc: n=%d (need 2^p+1, 5..1025) or batch=%d invalid", n, batch);
    return MLMC_ERR_INVALID;
  }
  const size_t need = mg_workspace_bytes(batch, n, cfg->precision, cfg->accel);
  if (need > kNoAllocBytes) {
    set_error("mg_solve_batch_noalloc: batch=%d at n=%d needs %zu bytes of workspace; the fixed no-allocation "
              "workspace holds %zu bytes (use a smaller batch or mg_solve_batch)",
              batch, n, need, kNoAllocBytes);
    return MLMC_ERR_INVALID;
  }
  // one call at a time per process: every call uses the same array
  std::lock_guard<std::mutex> lk(g_mu);
  void* ws = nullptr;
  MLMC_TRY(workspace_address(&ws));
  cudaStream_t st = (cudaStream_t)stream;
  MGSolveArgs a;
  a.k0 = k;
  a.n_k0 = n;
  a.st0 = 1;
  a.f = f;
  a.u = u;
  a.n = n;
  a.B = batch;
  a.cfg = *cfg;
  std::vector<int> cyc(batch);
  std::vector<double> rel(batch);
  int bad = 0;
  // drain the stream on every path before the lock is released, so that no kernel of a
  // failed call still writes the array while the next call uses it
  const int rc = mg_solve_dev(a, ws, st, cyc.data(), rel.data(), &bad);
  const cudaError_t se = cudaStreamSynchronize(st);
  if (rc < 0) return rc;
  if (se != cudaSuccess) {
    set_error("cudaStreamSynchronize failed: %s", cudaGetErrorString(se));
    return MLMC_ERR_CUDA;
  }
  if (stats_host)
    for (int s = 0; s < batch; ++s) {
      stats_host[s].cycles = cyc[s];
      stats_host[s].rel_res = rel[s];
    }
  if (bad) {
    set_error("%d of %d samples did not reach rtol=%g in %d cycles", bad, batch, cfg->rtol, cfg->max_cycles);
    return MLMC_ERR_NOT_CONVERGED;
  }
  return MLMC_OK;
}
