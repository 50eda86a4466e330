// extern "C" entry points of include/mlmc.h, the batched MLMC level pipeline, and
// error reporting.
#include <math.h>
#include <stddef.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <utility>
#include <vector>

#include "common.cuh"
#include "field.cuh"
#include "mg.cuh"
#include "level.cuh"
#include "spde.cuh"
#include "prof.cuh"
#include "tune.cuh"

namespace mlmc {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

const char* last_error() { return g_err; }

// Budget of the kernels' bounded waits (mlmc_set_wait_budget).
static std::atomic<long long> g_wait_budget{2000000000LL};
long long wait_budget_clocks() { return g_wait_budget.load(); }

// Host-side allocation-failure injection (mlmc_inject_alloc_failure): -1 = off, else the
// number of further allocations that still succeed before every later one fails.
static std::atomic<long long> g_alloc_budget{-1};

int DevBuf::alloc(size_t bytes, cudaStream_t st) {
  release();
  st_ = st;
  if (bytes == 0) bytes = 256;
  for (long long b = g_alloc_budget.load(); b >= 0;) {
    if (b == 0) {
      set_error("cudaMallocAsync(%zu bytes) not attempted: allocation failure injected", bytes);
      return MLMC_ERR_OOM;
    }
    if (g_alloc_budget.compare_exchange_weak(b, b - 1)) break;
  }
  cudaError_t e = cudaMallocAsync(&p_, bytes, st);
  if (e != cudaSuccess) {
    p_ = nullptr;
    set_error("cudaMallocAsync(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? MLMC_ERR_OOM : MLMC_ERR_CUDA;
  }
  return MLMC_OK;
}

void DevBuf::release() {
  if (p_) cudaFreeAsync(p_, st_);
  p_ = nullptr;
}

static int check_mg(const mg_cfg* c) {
  if (!c) {
    set_error("mg_cfg is NULL");
    return MLMC_ERR_INVALID;
  }
  if (c->nu1 < 0 || c->nu1 > 8 || c->nu2 < 0 || c->nu2 > 8) {
    set_error("nu1=%d nu2=%d out of range 0..8 (both 0: tuned count)", c->nu1, c->nu2);
    return MLMC_ERR_INVALID;
  }
  if (c->smoother < MLMC_SMOOTH_AUTO || c->smoother > MLMC_SMOOTH_SPLIT) {
    set_error("unknown smoother %d", c->smoother);
    return MLMC_ERR_INVALID;
  }
  if (c->max_cycles < 1 || c->max_cycles > 1000) {
    set_error("max_cycles=%d out of range 1..1000", c->max_cycles);
    return MLMC_ERR_INVALID;
  }
  if (!(c->rtol < 1.0) || isnan(c->rtol)) {
    set_error("rtol=%g must be < 1", c->rtol);
    return MLMC_ERR_INVALID;
  }
  if (c->precision != MLMC_PREC_F64 && c->precision != MLMC_PREC_MIXED) {
    set_error("unknown precision %d", c->precision);
    return MLMC_ERR_INVALID;
  }
  if (c->accel != MLMC_ACCEL_NONE && c->accel != MLMC_ACCEL_CG && c->accel != MLMC_ACCEL_FMG) {
    set_error("unknown accel %d", c->accel);
    return MLMC_ERR_INVALID;
  }
  if (c->disc != MLMC_DISC_FV && c->disc != MLMC_DISC_FE) {
    set_error("unknown disc %d", c->disc);
    return MLMC_ERR_INVALID;
  }
  if (c->engine != MLMC_ENGINE_AUTO && c->engine != MLMC_ENGINE_BATCHED && c->engine != MLMC_ENGINE_CTA) {
    set_error("unknown engine %d", c->engine);
    return MLMC_ERR_INVALID;
  }
  if ((c->disc == MLMC_DISC_FE || c->accel == MLMC_ACCEL_FMG) && c->precision != MLMC_PREC_F64) {
    set_error("the P1 finite elements and the FMG cycle run in FP64 (precision %d)", c->precision);
    return MLMC_ERR_INVALID;
  }
  return MLMC_OK;
}

// `cov` sits in what was the struct's tail padding: the size and every other offset are
// those of the four-field layout, so zero-initialised callers get the Gaussian covariance.
static_assert(sizeof(mlmc_field_cfg) == 32 && offsetof(mlmc_field_cfg, cov) == 28, "mlmc_field_cfg layout");
static_assert(sizeof(mg_cfg) == 40 && offsetof(mg_cfg, disc) == 32 && offsetof(mg_cfg, engine) == 36,
              "mg_cfg layout");
static_assert(sizeof(mlmc_cfg) == 96 && offsetof(mlmc_cfg, qoi) == 88, "mlmc_cfg layout");

static int check_field(const mlmc_field_cfg* c) {
  if (!c) {
    set_error("mlmc_field_cfg is NULL");
    return MLMC_ERR_INVALID;
  }
  if (c->M < 1 || c->M > 65536 || !(c->ell > 0.0) || !(c->sigma2 >= 0.0) || isinf(c->sigma2) || isinf(c->ell) ||
      (c->cov != MLMC_COV_GAUSS && c->cov != MLMC_COV_EXP && c->cov != MLMC_COV_SPDE)) {
    set_error("field cfg invalid: M=%d ell=%g sigma2=%g cov=%d", c->M, c->ell, c->sigma2, c->cov);
    return MLMC_ERR_INVALID;
  }
  return MLMC_OK;
}

static int check_grid(int n, int batch) {
  if (!valid_grid(n)) {
    set_error("n=%d is not 2^p+1 with 5 <= n <= 4097", n);
    return MLMC_ERR_INVALID;
  }
  if (batch < 1 || batch > 65535) {
    set_error("batch=%d out of range 1..65535", batch);
    return MLMC_ERR_INVALID;
  }
  return MLMC_OK;
}

static int device_ready() {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error("no usable CUDA device: %s", cudaGetErrorString(e));
    return MLMC_ERR_CUDA;
  }
  return MLMC_OK;
}

// Running statistics of one MLMC level in device memory (the level mean and variance of Algorithm 1):
// Kahan-compensated sum and Welford mean / M2 of Y, accumulated sequentially in
// sample-id order, so the record does not depend on how the samples were batched.
struct LevelRecord {
  double N, sum, comp, mean, M2, cyc_f, cyc_c, max_cyc;
};

// Y = Qf - Qc (Qc NULL: level 0) for b samples, folded into *rec in order. One warp: the
// lanes load (and store Y for) 32 samples at a time, lane 0 folds them in order, so that
// the loads of a chunk overlap instead of sitting on the fold's dependency chain.
__global__ void k_level_stats(const double* __restrict__ Qf, const double* __restrict__ Qc,
                              const int* __restrict__ cf, const int* __restrict__ cc, int b, double* __restrict__ Y,
                              LevelRecord* __restrict__ rec) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  __shared__ double ys[32];
  __shared__ int cfs[32], ccs[32];
  const int lane = threadIdx.x;
  LevelRecord r{};
  if (lane == 0) r = *rec;
  for (int i0 = 0; i0 < b; i0 += 32) {
    const int i = i0 + lane;
    if (i < b) {
      const double y = Qc ? Qf[i] - Qc[i] : Qf[i];
      if (Y) Y[i] = y;
      ys[lane] = y;
      cfs[lane] = cf[i];
      ccs[lane] = cc ? cc[i] : 0;
    }
    __syncwarp();
    if (lane == 0) {
      const int cnt = b - i0 < 32 ? b - i0 : 32;
      // cycle counts summed and maximised as integers (exact, the same values as adding
      // them to the FP64 fields one by one), off the FP64 pipe that the fold waits on
      long long sf = 0, sc = 0;
      int mx = 0;
      for (int j = 0; j < cnt; ++j) {
        const double y = ys[j];
        const double yk = y - r.comp;
        const double tk = r.sum + yk;
        r.comp = (tk - r.sum) - yk;
        r.sum = tk;
        r.N += 1.0;
        const double d = y - r.mean;
        r.mean += d / r.N;
        r.M2 += d * (y - r.mean);
        sf += cfs[j];
        mx = cfs[j] > mx ? cfs[j] : mx;
        if (cc) {
          sc += ccs[j];
          mx = ccs[j] > mx ? ccs[j] : mx;
        }
      }
      r.cyc_f += (double)sf;
      if (cc) r.cyc_c += (double)sc;
      r.max_cyc = fmax(r.max_cyc, (double)mx);
    }
    __syncwarp();
  }
  if (lane == 0) *rec = r;
}

// One batch of an MLMC level: field on the fine grid, fine solve, coarse solve on the
// same realisation, QoI of both. Fourier-feature fields: the coarse coefficient is the fine
// one injected (the coarse grid's nodes are every other fine node). SPDE fields: each grid
// solves its own discretisation of the SPDE with the white noise of the fine grid.
struct LevelBatch {
  int nf = 0, nc = 0, B = 0, M = 0, prec = 0, cov = 0;
  DevBuf ids, k0, kc, uf, uc, Q, cyc, rec, scratch;
  size_t scratch_bytes = 0;

  static size_t scratch_for(int B, int nf, int nc, const mlmc_field_cfg& fc, int prec, int accel) {
    size_t s = fc.cov == MLMC_COV_SPDE ? spde_scratch_bytes(B, nf) : field_scratch_bytes(B, fc.M, nf);
    size_t m = mg_workspace_bytes(B, nf, prec, accel);
    if (m > s) s = m;
    if (nc) {
      m = mg_workspace_bytes(B, nc, prec, accel);
      if (m > s) s = m;
    }
    m = qoi_scratch_bytes(B, nf);
    if (m > s) s = m;
    return s;
  }

  static size_t bytes_for(int B, int nf, int nc, const mlmc_field_cfg& fc, int prec, int accel) {
    const size_t kc_bytes = (fc.cov == MLMC_COV_SPDE && nc) ? cube(nc) * 8 : 0;
    return scratch_for(B, nf, nc, fc, prec, accel) + (size_t)B * (cube(nf) * 16 + (nc ? cube(nc) * 8 : 0) +
                                                                   kc_bytes + 64);
  }

  int init(int B_, int nf_, int nc_, const mlmc_field_cfg& fc, int prec_, int accel, cudaStream_t st) {
    B = B_;
    nf = nf_;
    nc = nc_;
    M = fc.M;
    cov = fc.cov;
    prec = prec_;
    scratch_bytes = scratch_for(B, nf, nc, fc, prec, accel);
    MLMC_TRY(ids.alloc((size_t)B * sizeof(uint64_t), st));
    MLMC_TRY(k0.alloc((size_t)B * cube(nf) * sizeof(double), st));
    if (cov == MLMC_COV_SPDE && nc) MLMC_TRY(kc.alloc((size_t)B * cube(nc) * sizeof(double), st));
    MLMC_TRY(uf.alloc((size_t)B * cube(nf) * sizeof(double), st));
    if (nc) MLMC_TRY(uc.alloc((size_t)B * cube(nc) * sizeof(double), st));
    MLMC_TRY(Q.alloc((size_t)3 * B * sizeof(double), st));
    MLMC_TRY(cyc.alloc((size_t)2 * B * sizeof(int), st));
    MLMC_TRY(rec.alloc(sizeof(LevelRecord), st));
    MLMC_CUDA_TRY(cudaMemsetAsync(rec.get(), 0, sizeof(LevelRecord), st));
    MLMC_TRY(scratch.alloc(scratch_bytes, st));
    return MLMC_OK;
  }

  // b <= B samples with device ids; Qf/Qc/Y: device outputs of b entries (Qc, Y may be
  // NULL). Folds the batch into the level record.
  int run(const mlmc_field_cfg& fc, const mg_cfg& mc, const uint64_t* ids_dev, int b, double* Qf, double* Qc,
          double* Y, int* n_unconv, cudaStream_t st, int qoi = MLMC_QOI_MEAN) {
    const bool spde = fc.cov == MLMC_COV_SPDE;
    if (spde) {
      MLMC_TRY(spde_field_dev(fc, ids_dev, b, nf, nf, MLMC_F64, k0.get(), scratch.get(), st));
      if (nc) MLMC_TRY(spde_field_dev(fc, ids_dev, b, nc, nf, MLMC_F64, kc.get(), scratch.get(), st));
    } else {
      MLMC_TRY(field_eval_dev(fc, ids_dev, b, nf, MLMC_F64, k0.get(), scratch.get(), st));
    }
    MGSolveArgs a;
    a.k0 = k0.as<double>();
    a.n_k0 = nf;
    a.f = nullptr;
    a.B = b;
    a.cfg = mc;
    int bad = 0;
    int* cf = cyc.as<int>();
    int* cc = cyc.as<int>() + B;
    double* qc = Qc ? Qc : Q.as<double>() + B;
    if (nc) {
      // coarse solve first (its coefficient is the fine one injected); its solution,
      // interpolated, starts the fine solve (nested iteration, the first step of FMG)
      MLMC_CUDA_TRY(cudaMemsetAsync(uc.get(), 0, (size_t)b * cube(nc) * sizeof(double), st));
      if (spde) {
        a.k0 = kc.as<double>();
        a.n_k0 = nc;
        a.st0 = 1;
      } else {
        a.st0 = 2;
      }
      a.u = uc.as<double>();
      a.n = nc;
      MLMC_TRY(mg_solve_dev(a, scratch.get(), st, nullptr, nullptr, &bad, cc, nullptr));
      *n_unconv += bad;
      MLMC_TRY(qoi_any(qoi, uc.as<double>(), nc, b, qc, scratch.get(), spde ? kc.as<double>() : k0.as<double>(),
                       spde ? nc : nf, spde ? 1 : 2, st));
      MLMC_TRY(interpolate_dev(uc.as<double>(), nf, b, uf.as<double>(), st));
    } else {
      MLMC_CUDA_TRY(cudaMemsetAsync(uf.get(), 0, (size_t)b * cube(nf) * sizeof(double), st));
    }
    a.k0 = k0.as<double>();
    a.n_k0 = nf;
    a.st0 = 1;
    a.u = uf.as<double>();
    a.n = nf;
    bad = 0;
    MLMC_TRY(mg_solve_dev(a, scratch.get(), st, nullptr, nullptr, &bad, cf, nullptr));
    *n_unconv += bad;
    MLMC_TRY(qoi_any(qoi, uf.as<double>(), nf, b, Qf, scratch.get(), k0.as<double>(), nf, 1, st));
    if (nc) {
      MLMC_LAUNCH("level_stats", b * 24.0, b * 10.0, st,
                  (k_level_stats<<<1, 32, 0, st>>>(Qf, qc, cf, cc, b, Y, rec.as<LevelRecord>())));
    } else {
      if (Qc) MLMC_CUDA_TRY(cudaMemsetAsync(Qc, 0, (size_t)b * sizeof(double), st));
      MLMC_LAUNCH("level_stats", b * 16.0, b * 10.0, st,
                  (k_level_stats<<<1, 32, 0, st>>>(Qf, nullptr, cf, nullptr, b, Y, rec.as<LevelRecord>())));
    }
    MLMC_CUDA_TRY(cudaGetLastError());
    return MLMC_OK;
  }

  int read_record(LevelRecord* r, cudaStream_t st) {
    MLMC_CUDA_TRY(cudaMemcpyAsync(r, rec.get(), sizeof(LevelRecord), cudaMemcpyDeviceToHost, st));
    MLMC_CUDA_TRY(cudaStreamSynchronize(st));
    if (field_wait_error_take(st)) {
      set_error("level batch: a bounded wait of the tensor-core field ran out (budget %lld SM clocks)",
                wait_budget_clocks());
      return MLMC_ERR_TIMEOUT;
    }
    return MLMC_OK;
  }
};

int validate_level_cfg(const mlmc_field_cfg& fc, const mg_cfg& mc) {
  MLMC_TRY(check_field(&fc));
  MLMC_TRY(check_mg(&mc));
  return MLMC_OK;
}

size_t level_batch_bytes(int b, int nf, int nc, const mlmc_field_cfg& fc, int precision, int accel) {
  return LevelBatch::bytes_for(b, nf, nc, fc, precision, accel);
}

int run_level_batch_host(const mlmc_field_cfg& fc, const mg_cfg& mc, int nf, int nc, const uint64_t* ids_host,
                         int b, double* Qf, double* Qc, int* cyc_f, int* cyc_c, int* n_unconv, cudaStream_t st) {
  LevelBatch lb;
  MLMC_TRY(lb.init(b, nf, nc, fc, mc.precision, mc.accel, st));
  MLMC_CUDA_TRY(cudaMemcpyAsync(lb.ids.get(), ids_host, (size_t)b * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  double* qf = lb.Q.as<double>();
  double* qc = nc ? lb.Q.as<double>() + b : nullptr;
  MLMC_TRY(lb.run(fc, mc, lb.ids.as<uint64_t>(), b, qf, qc, nullptr, n_unconv, st));
  MLMC_CUDA_TRY(cudaMemcpyAsync(Qf, qf, (size_t)b * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (qc) MLMC_CUDA_TRY(cudaMemcpyAsync(Qc, qc, (size_t)b * sizeof(double), cudaMemcpyDeviceToHost, st));
  MLMC_CUDA_TRY(cudaMemcpyAsync(cyc_f, lb.cyc.as<int>(), (size_t)b * sizeof(int), cudaMemcpyDeviceToHost, st));
  if (nc) MLMC_CUDA_TRY(cudaMemcpyAsync(cyc_c, lb.cyc.as<int>() + b, (size_t)b * sizeof(int), cudaMemcpyDeviceToHost, st));
  MLMC_CUDA_TRY(cudaStreamSynchronize(st));
  if (!nc)
    for (int i = 0; i < b; ++i) {
      Qc[i] = 0.0;
      cyc_c[i] = 0;
    }
  return MLMC_OK;
}

static void fill_stats(const LevelRecord& r, double secs, mlmc_level_stats* out) {
  if (!out) return;
  const double N = r.N > 0 ? r.N : 1.0;
  out->N = (int64_t)r.N;
  out->mean = r.mean;
  out->var_biased = r.M2 / N;
  out->var_unbiased = r.N > 1 ? r.M2 / (r.N - 1.0) : 0.0;
  out->sum = r.sum;
  out->sum_comp = r.comp;
  out->M2 = r.M2;
  out->mean_cycles_fine = r.cyc_f / N;
  out->mean_cycles_coarse = r.cyc_c / N;
  out->max_cycles_seen = (int)r.max_cyc;
  out->seconds = secs;
  out->cost_per_sample = secs / N;
}

static int check_level(const mlmc_cfg* cfg, int level, int N, int* nf, int* nc) {
  if (!cfg) {
    set_error("mlmc_cfg is NULL");
    return MLMC_ERR_INVALID;
  }
  MLMC_TRY(check_field(&cfg->field));
  MLMC_TRY(check_mg(&cfg->mg));
  if (cfg->qoi != MLMC_QOI_MEAN && cfg->qoi != MLMC_QOI_POINT && cfg->qoi != MLMC_QOI_FLUX) {
    set_error("unknown qoi %d", cfg->qoi);
    return MLMC_ERR_INVALID;
  }
  if (level < 0 || level > 8 || N < 1 || !valid_grid(cfg->n0) || cfg->max_batch < 0) {
    set_error("level=%d N=%d n0=%d max_batch=%d invalid", level, N, cfg->n0, cfg->max_batch);
    return MLMC_ERR_INVALID;
  }
  const long long nfl = (long long)(cfg->n0 - 1) * (1LL << level) + 1;
  if (nfl > 1025 || !valid_grid((int)nfl)) {
    set_error("level %d gives n=%lld beyond 1025", level, nfl);
    return MLMC_ERR_INVALID;
  }
  *nf = (int)nfl;
  *nc = level > 0 ? (cfg->n0 - 1) * (1 << (level - 1)) + 1 : 0;
  return MLMC_OK;
}

static int choose_batch(const mlmc_cfg* cfg, int N, int nf, int nc, int* B) {
  int b = cfg->max_batch;
  if (b == 0) {
    size_t fr = 0, tot = 0;
    MLMC_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    const size_t per = LevelBatch::bytes_for(1, nf, nc, cfg->field, cfg->mg.precision, cfg->mg.accel);
    size_t fit = (size_t)(0.6 * (double)fr) / (per + 1);
    if (fit < 1) fit = 1;
    b = (int)(fit < (size_t)N ? fit : (size_t)N);
  }
  if (b > N) b = N;
  if (b > 65535) b = 65535;
  *B = b;
  return MLMC_OK;
}

}  // namespace mlmc

using namespace mlmc;

extern "C" {

const char* mlmc_last_error_string(void) { return last_error(); }

const char* mlmc_version(void) { return "mlmc-gb300 0.2 (sm_103a)"; }

int mlmc_set_wait_budget(int64_t clocks, int64_t* previous) {
  if (clocks < 0) {
    set_error("mlmc_set_wait_budget: clocks=%lld must be >= 0", (long long)clocks);
    return MLMC_ERR_INVALID;
  }
  const long long old = g_wait_budget.exchange((long long)clocks);
  if (previous) *previous = (int64_t)old;
  return MLMC_OK;
}

int mlmc_inject_alloc_failure(int64_t after) {
  if (after < -1) {
    set_error("mlmc_inject_alloc_failure: after=%lld must be >= -1", (long long)after);
    return MLMC_ERR_INVALID;
  }
  g_alloc_budget.store((long long)after);
  return MLMC_OK;
}

int mlmc_inject_wait_failure(int launches) {
  if (launches < 0) {
    set_error("mlmc_inject_wait_failure: launches=%d must be >= 0", launches);
    return MLMC_ERR_INVALID;
  }
  field_inject_wait_failure(launches);
  return MLMC_OK;
}

static int field_eval_impl(const mlmc_field_cfg* cfg, const uint64_t* sample_ids_host, int batch, int n,
                           int n_fine, int dtype, void* k_out, void* stream) {
  MLMC_TRY(check_field(cfg));
  MLMC_TRY(check_grid(n, batch));
  if (!sample_ids_host || !k_out || (dtype != MLMC_F64 && dtype != MLMC_F32)) {
    set_error("mlmc_field_eval: NULL pointer or unknown dtype %d", dtype);
    return MLMC_ERR_INVALID;
  }
  if (n_fine != n && n_fine != 2 * n - 1) {
    set_error("mlmc_field_eval_pair: n_fine=%d is neither n=%d nor 2n-1", n_fine, n);
    return MLMC_ERR_INVALID;
  }
  const bool spde = cfg->cov == MLMC_COV_SPDE;
  if (spde && n_fine > 1025) {
    set_error("SPDE field: grids up to 1025 nodes per axis (n_fine=%d)", n_fine);
    return MLMC_ERR_INVALID;
  }
  MLMC_TRY(device_ready());
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf ids, scratch;
  MLMC_TRY(ids.alloc((size_t)batch * sizeof(uint64_t), st));
  MLMC_TRY(scratch.alloc(spde ? spde_scratch_bytes(batch, n) : field_scratch_bytes(batch, cfg->M, n), st));
  MLMC_CUDA_TRY(
      cudaMemcpyAsync(ids.get(), sample_ids_host, (size_t)batch * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
  if (spde)
    MLMC_TRY(spde_field_dev(*cfg, ids.as<uint64_t>(), batch, n, n_fine, dtype, k_out, scratch.get(), st));
  else
    MLMC_TRY(field_eval_dev(*cfg, ids.as<uint64_t>(), batch, n, dtype, k_out, scratch.get(), st));
  // the host ids may be reused by the caller as soon as this returns
  MLMC_CUDA_TRY(cudaStreamSynchronize(st));
  if (!spde && field_wait_error_take(st)) {
    set_error("mlmc_field_eval: a bounded wait of the tensor-core field ran out (budget %lld SM clocks); the "
              "nodes of the blocks concerned hold NaN",
              wait_budget_clocks());
    return MLMC_ERR_TIMEOUT;
  }
  return MLMC_OK;
}

int mlmc_field_eval(const mlmc_field_cfg* cfg, const uint64_t* sample_ids_host, int batch, int n, int dtype,
                    void* k_out, void* stream) {
  return field_eval_impl(cfg, sample_ids_host, batch, n, n, dtype, k_out, stream);
}

int mlmc_field_eval_pair(const mlmc_field_cfg* cfg, const uint64_t* sample_ids_host, int batch, int n, int n_fine,
                         int dtype, void* k_out, void* stream) {
  return field_eval_impl(cfg, sample_ids_host, batch, n, n_fine, dtype, k_out, stream);
}

int mg_solve_batch(const mg_cfg* cfg, int batch, int n, const double* k, const double* f, double* u,
                   mg_stats* stats_host, void* stream) {
  MLMC_TRY(check_mg(cfg));
  MLMC_TRY(check_grid(n, batch));
  if (!k || !u) {
    set_error("mg_solve_batch: k and u must be device pointers");
    return MLMC_ERR_INVALID;
  }
  if (cfg->accel == MLMC_ACCEL_FMG && f) {
    set_error("mg_solve_batch: the FMG cycle solves f = 1 (pass f = NULL)");
    return MLMC_ERR_INVALID;
  }
  MLMC_TRY(device_ready());
  cudaStream_t st = (cudaStream_t)stream;
  DevBuf ws;
  MLMC_TRY(ws.alloc(mg_workspace_bytes(batch, n, cfg->precision, cfg->accel), st));
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
  MLMC_TRY(mg_solve_dev(a, ws.get(), st, cyc.data(), rel.data(), &bad));
  if (stats_host)
    for (int s = 0; s < batch; ++s) {
      stats_host[s].cycles = cyc[s];
      stats_host[s].rel_res = rel[s];
    }
  ws.release();
  MLMC_CUDA_TRY(cudaStreamSynchronize(st));
  if (bad) {
    set_error("%d of %d samples did not reach rtol=%g in %d cycles", bad, batch, cfg->rtol, cfg->max_cycles);
    return MLMC_ERR_NOT_CONVERGED;
  }
  return MLMC_OK;
}

int mlmc_level_estimate(const mlmc_cfg* cfg, int level, uint64_t first_id, int N, double* Y_host, double* Qf_host,
                        double* Qc_host, mlmc_level_stats* out) {
  int nf = 0, nc = 0;
  MLMC_TRY(check_level(cfg, level, N, &nf, &nc));
  MLMC_TRY(device_ready());
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = (cudaStream_t)cfg->stream;
  int B = 0;
  MLMC_TRY(choose_batch(cfg, N, nf, nc, &B));
  LevelBatch lb;
  MLMC_TRY(lb.init(B, nf, nc, cfg->field, cfg->mg.precision, cfg->mg.accel, st));
  std::vector<uint64_t> ids(B);
  int unconv = 0;
  double* Qf = lb.Q.as<double>();
  double* Qc = nc ? lb.Q.as<double>() + B : nullptr;
  double* Y = lb.Q.as<double>() + 2 * B;
  for (int s0 = 0; s0 < N; s0 += B) {
    const int b = (N - s0) < B ? (N - s0) : B;
    for (int i = 0; i < b; ++i) ids[i] = first_id + (uint64_t)(s0 + i);
    MLMC_CUDA_TRY(cudaMemcpyAsync(lb.ids.get(), ids.data(), (size_t)b * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    MLMC_TRY(lb.run(cfg->field, cfg->mg, lb.ids.as<uint64_t>(), b, Qf, Qc, Y, &unconv, st, cfg->qoi));
    if (Y_host) MLMC_CUDA_TRY(cudaMemcpyAsync(Y_host + s0, Y, b * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (Qf_host) MLMC_CUDA_TRY(cudaMemcpyAsync(Qf_host + s0, Qf, b * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (Qc_host) {
      if (Qc)
        MLMC_CUDA_TRY(cudaMemcpyAsync(Qc_host + s0, Qc, b * sizeof(double), cudaMemcpyDeviceToHost, st));
      else
        memset(Qc_host + s0, 0, b * sizeof(double));
    }
    MLMC_CUDA_TRY(cudaStreamSynchronize(st));
  }
  LevelRecord r;
  MLMC_TRY(lb.read_record(&r, st));
  fill_stats(r, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(), out);
  if (unconv) {
    set_error("%d solves of level %d did not reach rtol=%g", unconv, level, cfg->mg.rtol);
    return MLMC_ERR_NOT_CONVERGED;
  }
  return MLMC_OK;
}

int mlmc_level_run(const mlmc_cfg* cfg, int level, const uint64_t* ids_dev, int N, double* Y_dev, double* Qf_dev,
                   double* Qc_dev, mlmc_level_stats* out) {
  int nf = 0, nc = 0;
  MLMC_TRY(check_level(cfg, level, N, &nf, &nc));
  if (!ids_dev) {
    set_error("mlmc_level_run: ids_dev is NULL");
    return MLMC_ERR_INVALID;
  }
  MLMC_TRY(device_ready());
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = (cudaStream_t)cfg->stream;
  int B = 0;
  MLMC_TRY(choose_batch(cfg, N, nf, nc, &B));
  LevelBatch lb;
  MLMC_TRY(lb.init(B, nf, nc, cfg->field, cfg->mg.precision, cfg->mg.accel, st));
  int unconv = 0;
  for (int s0 = 0; s0 < N; s0 += B) {
    const int b = (N - s0) < B ? (N - s0) : B;
    double* Qf = Qf_dev ? Qf_dev + s0 : lb.Q.as<double>();
    double* Qc = Qc_dev ? Qc_dev + s0 : nullptr;
    double* Y = Y_dev ? Y_dev + s0 : nullptr;
    MLMC_TRY(lb.run(cfg->field, cfg->mg, ids_dev + s0, b, Qf, Qc, Y, &unconv, st, cfg->qoi));
  }
  if (out) {
    LevelRecord r;
    MLMC_TRY(lb.read_record(&r, st));
    fill_stats(r, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(), out);
  }
  if (unconv) {
    set_error("%d solves of level %d did not reach rtol=%g", unconv, level, cfg->mg.rtol);
    return MLMC_ERR_NOT_CONVERGED;
  }
  return MLMC_OK;
}

int mlmc_autotune(const mlmc_cfg* cfg, int level, uint64_t first_id, int samples, mlmc_tune_entry* table,
                  int table_len, int* n_entries, int* best_smoother, int* best_nu) {
  int nf = 0, nc = 0;
  MLMC_TRY(check_level(cfg, level, samples, &nf, &nc));
  if (table_len < 0 || (table_len > 0 && !table)) {
    set_error("mlmc_autotune: bad table");
    return MLMC_ERR_INVALID;
  }
  MLMC_TRY(device_ready());
  cudaStream_t st = (cudaStream_t)cfg->stream;
  int B = 0;
  MLMC_TRY(choose_batch(cfg, samples, nf, nc, &B));
  const int smoothers[9] = {MLMC_SMOOTH_TWO_PASS,  MLMC_SMOOTH_FUSED_32x8, MLMC_SMOOTH_FUSED_32x16,
                            MLMC_SMOOTH_FUSED_64x8, MLMC_SMOOTH_BULK_32x8, MLMC_SMOOTH_BULK_32x16,
                            MLMC_SMOOTH_BULK_64x8,  MLMC_SMOOTH_NODAL,     MLMC_SMOOTH_SPLIT};
  std::vector<uint64_t> ids(samples);
  for (int i = 0; i < samples; ++i) ids[i] = first_id + (uint64_t)i;
  int count = 0, bs = MLMC_SMOOTH_TWO_PASS, bnu = 2;
  // an explicit V(nu, nu) in cfg is kept: only the smoother implementation is tuned
  const bool fixed_nu = cfg->mg.nu1 > 0 && cfg->mg.nu1 == cfg->mg.nu2;
  const int nu_lo = fixed_nu ? cfg->mg.nu1 : 1, nu_hi = fixed_nu ? cfg->mg.nu1 : 4;
  // the nodal-coefficient sweeps exist only in FP32 correction cycles on finite volumes;
  // the colour-split storage there and in FP64 stationary and FMG cycles
  const bool fv = cfg->mg.disc == MLMC_DISC_FV, mixed = cfg->mg.precision == MLMC_PREC_MIXED;
  int cand[9], n_sm = 0;
  for (int si = 0; si < 9; ++si) {
    if (smoothers[si] == MLMC_SMOOTH_NODAL && !(fv && mixed)) continue;
    if (smoothers[si] == MLMC_SMOOTH_SPLIT && !(mixed ? fv : cfg->mg.accel != MLMC_ACCEL_CG)) continue;
    cand[n_sm++] = smoothers[si];
  }
  // one timed pass of a candidate over the tuning samples (batches as the level runs them)
  auto time_once = [&](const mg_cfg& mc, LevelRecord& r, double& secs) -> int {
    LevelBatch lb;
    MLMC_TRY(lb.init(B, nf, nc, cfg->field, mc.precision, mc.accel, st));
    MLMC_CUDA_TRY(cudaStreamSynchronize(st));
    const auto t0 = std::chrono::steady_clock::now();
    int unconv = 0;
    for (int s0 = 0; s0 < samples; s0 += B) {
      const int b = (samples - s0) < B ? (samples - s0) : B;
      MLMC_CUDA_TRY(cudaMemcpyAsync(lb.ids.get(), ids.data() + s0, (size_t)b * sizeof(uint64_t),
                                    cudaMemcpyHostToDevice, st));
      MLMC_TRY(lb.run(cfg->field, mc, lb.ids.as<uint64_t>(), b, lb.Q.as<double>(), nc ? lb.Q.as<double>() + B : nullptr,
                      nullptr, &unconv, st));
    }
    MLMC_TRY(lb.read_record(&r, st));
    secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (unconv) secs = 1e300;  // a candidate that misses rtol never wins
    return MLMC_OK;
  };
  auto cand_cfg = [&](int smoother, int nu) {
    mg_cfg mc = cfg->mg;
    mc.smoother = smoother;
    mc.nu1 = nu;
    mc.nu2 = nu;
    // the batched engine: the stored choice also serves this grid size as a level inside
    // the batched V-cycles of larger grids (the small-grid engine runs every smoother of
    // one arithmetic family in the same time, so it could not tell them apart)
    mc.engine = MLMC_ENGINE_BATCHED;
    return mc;
  };
  // every candidate: the best of three passes (the first also pays first-launch costs)
  std::vector<double> per_cand;
  std::vector<int> cand_sm, cand_nu;
  for (int nu = nu_lo; nu <= nu_hi; ++nu)
    for (int si = 0; si < n_sm; ++si) {
      const mg_cfg mc = cand_cfg(cand[si], nu);
      double secs = 1e300;
      LevelRecord r{};
      for (int rep = 0; rep < 3; ++rep) {
        double t = 0.0;
        MLMC_TRY(time_once(mc, r, t));
        if (t < secs) secs = t;
      }
      const double per = secs / samples;
      if (count < table_len) {
        table[count].smoother = cand[si];
        table[count].nu = nu;
        table[count].seconds_per_sample = per;
        table[count].mean_cycles = r.N > 0 ? r.cyc_f / r.N : 0.0;
      }
      per_cand.push_back(per);
      cand_sm.push_back(cand[si]);
      cand_nu.push_back(nu);
      ++count;
    }
  // run-off of the two fastest, interleaved, so that a slow drift of the clocks during the
  // sweep cannot decide between close candidates
  int i1 = -1, i2 = -1;
  for (int i = 0; i < (int)per_cand.size(); ++i) {
    if (i1 < 0 || per_cand[i] < per_cand[i1]) {
      i2 = i1;
      i1 = i;
    } else if (i2 < 0 || per_cand[i] < per_cand[i2]) {
      i2 = i;
    }
  }
  if (i2 >= 0 && per_cand[i2] < 1e299) {
    for (int rep = 0; rep < 2; ++rep)
      for (int i : {i1, i2}) {
        LevelRecord r{};
        double t = 0.0;
        MLMC_TRY(time_once(cand_cfg(cand_sm[i], cand_nu[i]), r, t));
        if (t / samples < per_cand[i]) per_cand[i] = t / samples;
      }
    if (per_cand[i2] < per_cand[i1]) std::swap(i1, i2);
    for (int i : {i1, i2})
      if (i < table_len) table[i].seconds_per_sample = per_cand[i];
  }
  if (i1 >= 0) {
    bs = cand_sm[i1];
    bnu = cand_nu[i1];
  }
  tune_store(nf, cfg->mg.precision, bs, bnu);
  if (n_entries) *n_entries = count;
  if (best_smoother) *best_smoother = bs;
  if (best_nu) *best_nu = bnu;
  return MLMC_OK;
}

int mlmc_tune_set(int n, int precision, int smoother, int nu) {
  if (!valid_grid(n) || (precision != MLMC_PREC_F64 && precision != MLMC_PREC_MIXED) ||
      smoother < MLMC_SMOOTH_TWO_PASS || smoother > MLMC_SMOOTH_SPLIT || nu < 1 || nu > 8) {
    set_error("mlmc_tune_set: invalid arguments (n=%d precision=%d smoother=%d nu=%d)", n, precision, smoother, nu);
    return MLMC_ERR_INVALID;
  }
  tune_store(n, precision, smoother, nu);
  return MLMC_OK;
}

}  // extern "C"
