// Adaptive multilevel Monte Carlo (Algorithm 2 of Sec. 2.4) behind the C ABI.
//
// A round computes the missing samples of every level (through the level pipeline of
// mlmc_level_estimate, or a caller's sampler), folds each level's (N, mean, M2) record
// into the running record by Chan's pairwise merge (the sample mean Y-hat_l and s_l^2 of
// Sec. 2.3), takes the cost per sample C_l (measured wall time, or the node count of the
// level's two grids), and sizes N_l by Eq. 15 for eps_s^2 = theta eps^2 (Eq. 6). With
// level growth enabled, the bias estimate of Eq. 14, |Y-hat_L| / (8^alpha - 1), is
// compared with eps_b; while it is larger and L < max_level the next level joins with its
// pilot count. The run stops when a round changes neither N_l nor L. alpha is given or
// fitted online (minus the least-squares slope of log_8 |Y-hat_l| over the levels l >= 1
// with samples, M_l ~ 8^l); beta and gamma (Eq. 12) are fitted the same way from s_l^2
// and C_l and reported.
//
// Sample i of level l has the realisation id (l << 48) | i, in order, so a run resumed
// from its state continues with the ids an uninterrupted run would use. The levels of a
// round may run concurrently on `lanes` streams (one host thread each, levels placed
// longest first by node count); a level's record does not depend on that.
//
// Host arithmetic here is compiled without floating-point contraction (build flags), so
// the decisions are the same on every host architecture.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

struct mlmc_adaptive {
  mlmc_adaptive_cfg cfg;
  mlmc_level_sampler sampler = nullptr;
  void* user = nullptr;
  int L = 0;
  int rounds = 0;
  int64_t have[MLMC_MAX_LEVELS] = {};
  int64_t target[MLMC_MAX_LEVELS] = {};
  double N[MLMC_MAX_LEVELS] = {}, mean[MLMC_MAX_LEVELS] = {}, M2[MLMC_MAX_LEVELS] = {};
  double seconds[MLMC_MAX_LEVELS] = {};
  std::vector<mlmc_adaptive_round> log;
};

namespace mlmc {
namespace {

constexpr uint32_t kStateMagic = 0x4D4C4D43u;  // "MLMC"
constexpr uint32_t kStateVersion = 1;

// Chan et al.'s merge of a record of nb samples (mean mb, M2 m2b) into (n, mean, m2).
void chan_merge(double* n, double* mean, double* m2, double nb, double mb, double m2b) {
  if (nb == 0.0) return;
  const double tot = *n + nb;
  const double d = mb - *mean;
  *mean = *mean + d * nb / tot;
  *m2 = *m2 + m2b + d * d * *n * nb / tot;
  *n = tot;
}

// Neumaier's compensated sum (order-independent to within an ulp of the exact sum).
double compensated_sum(const double* v, int n) {
  double s = 0.0, c = 0.0;
  for (int i = 0; i < n; ++i) {
    const double t = s + v[i];
    c += fabs(s) >= fabs(v[i]) ? (s - t) + v[i] : (v[i] - t) + s;
    s = t;
  }
  return s + c;
}

int level_n(int n0, int l) { return (n0 - 1) * (1 << l) + 1; }

double node_cost(int n0, int l) {
  const double nf = (double)level_n(n0, l);
  const double nc = l > 0 ? (double)level_n(n0, l - 1) : 0.0;
  return nf * nf * nf + nc * nc * nc;
}

// a in |v_l| ~ c 8^(-a l): minus the least-squares slope of log_8 |v| against l (normal
// equations of the line fit, compensated sums). false with fewer than two levels or a
// zero value.
bool fit_rate(const int* ls, const double* v, int m, double* rate) {
  if (m < 2) return false;
  std::vector<double> x(m), y(m), xx(m), xy(m);
  for (int i = 0; i < m; ++i) {
    if (v[i] == 0.0) return false;
    x[i] = (double)ls[i];
    y[i] = log(fabs(v[i])) / log(8.0);
    xx[i] = x[i] * x[i];
    xy[i] = x[i] * y[i];
  }
  const double n = (double)m, sx = compensated_sum(x.data(), m), sy = compensated_sum(y.data(), m);
  const double sxx = compensated_sum(xx.data(), m), sxy = compensated_sum(xy.data(), m);
  const double den = n * sxx - sx * sx;
  if (den == 0.0) return false;
  *rate = -(n * sxy - sx * sy) / den;
  return true;
}

double variance(const mlmc_adaptive* A, int l) { return A->N[l] > 1.0 ? A->M2[l] / (A->N[l] - 1.0) : 0.0; }

double cost(const mlmc_adaptive* A, int l) {
  if (A->cfg.cost_model == MLMC_COST_NODES) return node_cost(A->cfg.level.n0, l);
  return A->have[l] > 0 ? A->seconds[l] / (double)A->have[l] : 0.0;
}

// (alpha as the bias test uses it, beta, gamma; NAN where no fit exists)
void rates(const mlmc_adaptive* A, double* alpha, double* beta, double* gamma) {
  int ls[MLMC_MAX_LEVELS], m = 0;
  double mv[MLMC_MAX_LEVELS], vv[MLMC_MAX_LEVELS], cv[MLMC_MAX_LEVELS];
  bool all_have = true;
  for (int l = 0; l <= A->L; ++l) all_have = all_have && A->have[l] > 0;
  for (int l = 1; l <= A->L; ++l)
    if (A->have[l] > 0) {
      ls[m] = l;
      mv[m] = A->mean[l];
      vv[m] = variance(A, l);
      cv[m] = cost(A, l);
      ++m;
    }
  double fa = 0.0;
  const bool have_fa = fit_rate(ls, mv, m, &fa);
  if (A->cfg.alpha > 0.0)
    *alpha = A->cfg.alpha;
  else
    *alpha = std::max(have_fa ? fa : A->cfg.alpha0, A->cfg.alpha_floor);
  bool vpos = true, cpos = all_have;
  for (int i = 0; i < m; ++i) {
    vpos = vpos && vv[i] > 0.0;
    cpos = cpos && cv[i] > 0.0;
  }
  double b = 0.0, g = 0.0;
  *beta = (vpos && fit_rate(ls, vv, m, &b)) ? b : NAN;
  *gamma = (cpos && fit_rate(ls, cv, m, &g)) ? -g : NAN;
}

double bias_estimate(const mlmc_adaptive* A, double alpha) { return fabs(A->mean[A->L]) / (pow(8.0, alpha) - 1.0); }

void eps_split(const mlmc_adaptive_cfg& c, double* eps_s, double* eps_b) {
  *eps_s = sqrt(c.theta) * c.eps;
  *eps_b = sqrt(1.0 - c.theta) * c.eps;
}

// N_l = ceil(eps_s^-2 (sum_k sqrt(V_k C_k)) sqrt(V_l / C_l)), at least 2 (Eq. 11 / 15).
void sample_sizes(const double* V, const double* C, int nl, double eps_s, int64_t* out) {
  double total = 0.0;
  for (int l = 0; l < nl; ++l) total += sqrt(V[l] * C[l]);
  for (int l = 0; l < nl; ++l) {
    const double x = ceil(total * sqrt(V[l] / C[l]) / (eps_s * eps_s));
    out[l] = x < 2.0 ? 2 : (x > 9.0e18 ? (int64_t)9e18 : (int64_t)x);
  }
}

int64_t pilot(const mlmc_adaptive_cfg& c, int l) {
  for (int k = l; k >= 0; --k)
    if (c.N_init[k] > 0) return c.N_init[k];
  return 2;
}

// Samples have[l] .. have[l] + count - 1 of level l on `stream`, folded into the record.
int add_samples(mlmc_adaptive* A, int l, int64_t count, void* stream) {
  if (count <= 0) return MLMC_OK;
  double nb = 0.0, mb = 0.0, m2b = 0.0;
  const auto t0 = std::chrono::steady_clock::now();
  if (A->sampler) {
    const int st = A->sampler(A->user, l, (uint64_t)A->have[l], count, &nb, &mb, &m2b);
    if (st < 0) {
      set_error("mlmc_adaptive: the sampler of level %d returned %d", l, st);
      return st;
    }
    if (nb != (double)count) {
      set_error("mlmc_adaptive: the sampler of level %d returned N=%g for %lld samples", l, nb, (long long)count);
      return MLMC_ERR_INVALID;
    }
  } else {
    if (count > 0x7fffffff) {
      set_error("mlmc_adaptive: %lld samples of level %d in one round exceed one level call", (long long)count, l);
      return MLMC_ERR_INVALID;
    }
    mlmc_cfg c = A->cfg.level;
    c.stream = stream;
    mlmc_level_stats out;
    const uint64_t first = ((uint64_t)l << 48) | (uint64_t)A->have[l];
    const int st = mlmc_level_estimate(&c, l, first, (int)count, nullptr, nullptr, nullptr, &out);
    if (st < 0) return st;
    nb = (double)out.N;
    mb = out.mean;
    m2b = out.M2;
  }
  A->seconds[l] += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  chan_merge(&A->N[l], &A->mean[l], &A->M2[l], nb, mb, m2b);
  A->have[l] += count;
  return MLMC_OK;
}

// The missing samples of every level, on the configured lanes.
int add_round(mlmc_adaptive* A) {
  std::vector<std::pair<int, int64_t>> todo;
  for (int l = 0; l <= A->L; ++l)
    if (A->target[l] > A->have[l]) todo.push_back({l, A->target[l] - A->have[l]});
  const int lanes = A->cfg.lanes > 1 ? A->cfg.lanes : 1;
  auto stream_of = [&](int k) -> void* {
    if (k == 0) return A->cfg.lane_streams[0] ? A->cfg.lane_streams[0] : A->cfg.level.stream;
    return A->cfg.lane_streams[k];
  };
  if (lanes <= 1 || todo.size() <= 1) {
    for (auto& t : todo) MLMC_TRY(add_samples(A, t.first, t.second, stream_of(0)));
    return MLMC_OK;
  }
  // longest first (count x node cost, ties in level order) onto the least-loaded lane
  std::stable_sort(todo.begin(), todo.end(), [&](const std::pair<int, int64_t>& a, const std::pair<int, int64_t>& b) {
    return (double)a.second * node_cost(A->cfg.level.n0, a.first) >
           (double)b.second * node_cost(A->cfg.level.n0, b.first);
  });
  std::vector<std::vector<std::pair<int, int64_t>>> plan(lanes);
  std::vector<double> load(lanes, 0.0);
  for (auto& t : todo) {
    int k = 0;
    for (int j = 1; j < lanes; ++j)
      if (load[j] < load[k]) k = j;
    plan[k].push_back(t);
    load[k] += (double)t.second * node_cost(A->cfg.level.n0, t.first);
  }
  std::vector<int> status(lanes, MLMC_OK);
  std::vector<std::string> errs(lanes);
  int dev = 0;
  cudaGetDevice(&dev);
  auto run_lane = [&](int k) {
    if (k > 0) cudaSetDevice(dev);
    for (auto& t : plan[k]) {
      const int st = add_samples(A, t.first, t.second, stream_of(k));
      if (st < 0) {
        status[k] = st;
        errs[k] = last_error();
        return;
      }
    }
  };
  std::vector<std::thread> threads;
  for (int k = 1; k < lanes; ++k)
    if (!plan[k].empty()) threads.emplace_back(run_lane, k);
  run_lane(0);
  for (auto& t : threads) t.join();
  for (int k = 0; k < lanes; ++k)
    if (status[k] < 0) {
      set_error("%s", errs[k].c_str());
      return status[k];
    }
  return MLMC_OK;
}

int check_cfg(const mlmc_adaptive_cfg* c) {
  if (!c) {
    set_error("mlmc_adaptive_cfg is NULL");
    return MLMC_ERR_INVALID;
  }
  if (c->L0 < 0 || c->L0 > MLMC_MAX_LEVELS - 1 || c->max_level < c->L0 || c->max_level > MLMC_MAX_LEVELS - 1) {
    set_error("mlmc_adaptive: need 0 <= L0 <= max_level <= %d (L0=%d max_level=%d)", MLMC_MAX_LEVELS - 1, c->L0,
              c->max_level);
    return MLMC_ERR_INVALID;
  }
  if (c->max_level > c->L0 && c->L0 < 1) {
    set_error("mlmc_adaptive: level growth starts from levels 0..L0 with L0 >= 1");
    return MLMC_ERR_INVALID;
  }
  if (!(c->eps > 0.0) || !(c->theta > 0.0 && c->theta < 1.0) ||
      (c->cost_model != MLMC_COST_MEASURED && c->cost_model != MLMC_COST_NODES) || !(c->alpha_floor >= 0.0) ||
      (c->alpha <= 0.0 && !(c->alpha0 > 0.0)) || c->lanes < 0 || c->lanes > 8 || isnan(c->alpha)) {
    set_error("mlmc_adaptive: invalid eps=%g theta=%g cost_model=%d alpha=%g alpha0=%g alpha_floor=%g lanes=%d", c->eps,
              c->theta, c->cost_model, c->alpha, c->alpha0, c->alpha_floor, c->lanes);
    return MLMC_ERR_INVALID;
  }
  for (int l = 0; l <= c->L0; ++l)
    if (c->N_init[l] < 1) {
      set_error("mlmc_adaptive: N_init[%d]=%lld must be >= 1 for the starting levels", l, (long long)c->N_init[l]);
      return MLMC_ERR_INVALID;
    }
  for (int k = 1; k < (c->lanes > 1 ? c->lanes : 1); ++k)
    if (!c->lane_streams[k]) {
      set_error("mlmc_adaptive: lane %d has no stream (lanes 1.. need created streams)", k);
      return MLMC_ERR_INVALID;
    }
  const long long nf = (long long)(c->level.n0 - 1) * (1LL << c->max_level) + 1;
  if (!valid_grid(c->level.n0) || nf > 1025) {
    set_error("mlmc_adaptive: n0=%d with max_level %d gives grids beyond 1025", c->level.n0, c->max_level);
    return MLMC_ERR_INVALID;
  }
  return MLMC_OK;
}

}  // namespace
}  // namespace mlmc

using namespace mlmc;

extern "C" {

int mlmc_sample_sizes(const double* var, const double* cost, int levels, double eps, double theta, int64_t* N_out) {
  if (!var || !cost || !N_out || levels < 1 || levels > 64 || !(eps > 0.0) || !(theta > 0.0 && theta < 1.0)) {
    set_error("mlmc_sample_sizes: invalid arguments (levels=%d eps=%g theta=%g)", levels, eps, theta);
    return MLMC_ERR_INVALID;
  }
  for (int l = 0; l < levels; ++l)
    if (!(var[l] > 0.0) || !(cost[l] > 0.0) || isinf(var[l]) || isinf(cost[l])) {
      set_error("mlmc_sample_sizes: level %d has variance %g and cost %g (both must be positive)", l, var[l],
                cost[l]);
      return MLMC_ERR_INVALID;
    }
  mlmc_adaptive_cfg c;
  memset(&c, 0, sizeof(c));
  c.eps = eps;
  c.theta = theta;
  double eps_s = 0.0, eps_b = 0.0;
  eps_split(c, &eps_s, &eps_b);
  sample_sizes(var, cost, levels, eps_s, N_out);
  return MLMC_OK;
}

int mlmc_merge_records(const double* records, int count, double* out) {
  if ((!records && count > 0) || !out || count < 0) {
    set_error("mlmc_merge_records: NULL argument or count %d < 0", count);
    return MLMC_ERR_INVALID;
  }
  double n = 0.0, mean = 0.0, m2 = 0.0;
  for (int i = 0; i < count; ++i) chan_merge(&n, &mean, &m2, records[3 * i], records[3 * i + 1], records[3 * i + 2]);
  out[0] = n;
  out[1] = mean;
  out[2] = m2;
  return MLMC_OK;
}

mlmc_adaptive* mlmc_adaptive_create(const mlmc_adaptive_cfg* cfg) {
  if (check_cfg(cfg) != MLMC_OK) return nullptr;
  mlmc_adaptive* A = new mlmc_adaptive();
  A->cfg = *cfg;
  A->L = cfg->L0;
  for (int l = 0; l <= A->L; ++l) A->target[l] = cfg->N_init[l];
  return A;
}

void mlmc_adaptive_destroy(mlmc_adaptive* A) { delete A; }

int mlmc_adaptive_set_sampler(mlmc_adaptive* A, mlmc_level_sampler fn, void* user) {
  if (!A) {
    set_error("mlmc_adaptive_set_sampler: NULL handle");
    return MLMC_ERR_INVALID;
  }
  A->sampler = fn;
  A->user = user;
  return MLMC_OK;
}

int mlmc_adaptive_step(mlmc_adaptive* A, int* finished) {
  if (!A || !finished) {
    set_error("mlmc_adaptive_step: NULL argument");
    return MLMC_ERR_INVALID;
  }
  A->rounds += 1;
  MLMC_TRY(add_round(A));
  const int nl = A->L + 1;
  double V[MLMC_MAX_LEVELS], C[MLMC_MAX_LEVELS];
  for (int l = 0; l < nl; ++l) {
    V[l] = std::max(variance(A, l), 1e-30);
    C[l] = cost(A, l);
    if (!(C[l] > 0.0)) {
      set_error("mlmc_adaptive: cost of level %d is %g", l, C[l]);
      return MLMC_ERR_INVALID;
    }
  }
  double eps_s = 0.0, eps_b = 0.0;
  eps_split(A->cfg, &eps_s, &eps_b);
  int64_t need[MLMC_MAX_LEVELS];
  sample_sizes(V, C, nl, eps_s, need);
  double alpha, beta, gamma;
  rates(A, &alpha, &beta, &gamma);
  const double bias = bias_estimate(A, alpha);
  const bool grow = A->cfg.max_level > A->cfg.L0 && bias > eps_b && A->L < A->cfg.max_level;
  mlmc_adaptive_round e;
  memset(&e, 0, sizeof(e));
  e.round = A->rounds;
  e.L = A->L;
  for (int l = 0; l < nl; ++l) {
    e.have[l] = A->have[l];
    e.N_next[l] = need[l];
  }
  e.alpha = alpha;
  e.bias = bias;
  e.grow = grow ? 1 : 0;
  A->log.push_back(e);
  bool enough = true;
  for (int l = 0; l < nl; ++l) enough = enough && need[l] <= A->have[l];
  if (!grow && enough) {
    *finished = 1;
    return MLMC_OK;
  }
  for (int l = 0; l < nl; ++l) A->target[l] = std::max(A->target[l], need[l]);
  if (grow) {
    A->L += 1;
    A->have[A->L] = 0;
    A->N[A->L] = A->mean[A->L] = A->M2[A->L] = A->seconds[A->L] = 0.0;
    A->target[A->L] = pilot(A->cfg, A->L);
  }
  *finished = 0;
  return MLMC_OK;
}

int mlmc_adaptive_run(mlmc_adaptive* A, int max_rounds, int* finished) {
  if (!A || max_rounds < 1) {
    set_error("mlmc_adaptive_run: NULL handle or max_rounds < 1");
    return MLMC_ERR_INVALID;
  }
  int fin = 0;
  for (int r = 0; r < max_rounds && !fin; ++r) MLMC_TRY(mlmc_adaptive_step(A, &fin));
  if (finished) *finished = fin;
  return MLMC_OK;
}

int mlmc_adaptive_result(const mlmc_adaptive* A, mlmc_adaptive_summary* out) {
  if (!A || !out) {
    set_error("mlmc_adaptive_result: NULL argument");
    return MLMC_ERR_INVALID;
  }
  memset(out, 0, sizeof(*out));
  const int nl = A->L + 1;
  double sv[MLMC_MAX_LEVELS];
  for (int l = 0; l < nl; ++l) {
    out->N[l] = A->have[l];
    out->mean[l] = A->mean[l];
    out->var[l] = variance(A, l);
    out->M2[l] = A->M2[l];
    out->seconds[l] = A->seconds[l];
    out->cost[l] = cost(A, l);
    sv[l] = A->have[l] > 0 ? out->var[l] / (double)A->have[l] : 0.0;
  }
  out->L = A->L;
  out->rounds = A->rounds;
  out->Q_hat = compensated_sum(A->mean, nl);
  out->sampling_var = compensated_sum(sv, nl);
  double eps_s = 0.0, eps_b = 0.0;
  eps_split(A->cfg, &eps_s, &eps_b);
  out->eps_s2 = eps_s * eps_s;
  rates(A, &out->alpha, &out->beta, &out->gamma);
  out->bias = bias_estimate(A, out->alpha);
  out->bias_ok = out->bias <= eps_b ? 1 : 0;
  return MLMC_OK;
}

int mlmc_adaptive_log_count(const mlmc_adaptive* A) { return A ? (int)A->log.size() : 0; }

int mlmc_adaptive_log_get(const mlmc_adaptive* A, int index, mlmc_adaptive_round* out) {
  if (!A || !out || index < 0 || index >= (int)A->log.size()) {
    set_error("mlmc_adaptive_log_get: bad handle, output or index %d", index);
    return MLMC_ERR_INVALID;
  }
  *out = A->log[index];
  return MLMC_OK;
}

int mlmc_adaptive_get_state(const mlmc_adaptive* A, mlmc_adaptive_state* st) {
  if (!A || !st) {
    set_error("mlmc_adaptive_get_state: NULL argument");
    return MLMC_ERR_INVALID;
  }
  memset(st, 0, sizeof(*st));
  st->magic = kStateMagic;
  st->version = kStateVersion;
  st->L = A->L;
  st->rounds = A->rounds;
  for (int l = 0; l < MLMC_MAX_LEVELS; ++l) {
    st->have[l] = A->have[l];
    st->target[l] = A->target[l];
    st->N[l] = A->N[l];
    st->mean[l] = A->mean[l];
    st->M2[l] = A->M2[l];
    st->seconds[l] = A->seconds[l];
  }
  return MLMC_OK;
}

int mlmc_adaptive_set_state(mlmc_adaptive* A, const mlmc_adaptive_state* st) {
  if (!A || !st) {
    set_error("mlmc_adaptive_set_state: NULL argument");
    return MLMC_ERR_INVALID;
  }
  if (st->magic != kStateMagic || st->version != kStateVersion || st->L < A->cfg.L0 || st->L > A->cfg.max_level ||
      st->rounds < 0) {
    set_error("mlmc_adaptive_set_state: not a state of this configuration (magic %08x version %u L %d)", st->magic,
              st->version, st->L);
    return MLMC_ERR_INVALID;
  }
  for (int l = 0; l < MLMC_MAX_LEVELS; ++l)
    if (st->have[l] < 0 || st->target[l] < 0 || st->N[l] != (double)st->have[l] || (l > st->L && st->have[l] != 0)) {
      set_error("mlmc_adaptive_set_state: inconsistent counts at level %d", l);
      return MLMC_ERR_INVALID;
    }
  A->L = st->L;
  A->rounds = st->rounds;
  for (int l = 0; l < MLMC_MAX_LEVELS; ++l) {
    A->have[l] = st->have[l];
    A->target[l] = st->target[l];
    A->N[l] = st->N[l];
    A->mean[l] = st->mean[l];
    A->M2[l] = st->M2[l];
    A->seconds[l] = st->seconds[l];
  }
  A->log.clear();
  return MLMC_OK;
}

}  // extern "C"
