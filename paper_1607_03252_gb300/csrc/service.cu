// Device-resident MLMC solve service with continuous batching.
//
// The paper assigns samples to process groups with static or dynamic schedules (Secs.
// 4-5; the dynamic variants take the next sample from a shared counter). On one GPU the
// same job -- keep the machine busy with samples of several levels whose cost differs
// by 8x per level -- is done by a request loop: requests (level, realisation id) are
// queued per level; worker threads, each with its own CUDA stream, repeatedly take the
// level whose oldest request has waited longest, batch up to max_batch requests of that
// level (or fewer once the oldest has waited batch_wait_ms), admit the batch only while
// the device bytes of all batches in flight stay within hbm_budget_bytes, and run the
// level pipeline (field, fine and coarse solves on the shared realisation, QoI) for it.
// Requests that arrive while batches run are admitted into the next batches as slots
// and memory free up; batches of different levels overlap on the device.
//
// A sample's result does not depend on the batch it ran in (every kernel masks per
// sample and every per-sample sum has a fixed shape), so a request gives the same Y
// alone and in the mix.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "level.cuh"

namespace mlmc {
namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

struct Req {
  uint64_t ticket;
  int level;
  uint64_t id;
  double t_submit;
};

}  // namespace
}  // namespace mlmc

struct mlmc_service {
  mlmc_service_cfg cfg;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<std::deque<mlmc::Req>> queues;
  std::map<uint64_t, mlmc_result> results;  // done or pending (status MLMC_PENDING)
  std::vector<std::thread> workers;
  bool stopping = false;
  uint64_t next_ticket = 1;
  size_t bytes_in_use = 0;
  int inflight = 0;
  int64_t submitted = 0, completed = 0, rejected = 0, cancelled = 0;
  int64_t queued = 0;
  double t_first = 0.0, t_last = 0.0;
  std::vector<std::vector<double>> latencies;  // per level, seconds
};

namespace mlmc {
namespace {

int level_grid(const mlmc_service_cfg& c, int level, int* nf, int* nc) {
  const long long f = (long long)(c.n0 - 1) * (1LL << level) + 1;
  if (level < 0 || level > 8 || f > 1025 || !valid_grid((int)f)) return MLMC_ERR_INVALID;
  *nf = (int)f;
  *nc = level > 0 ? (c.n0 - 1) * (1 << (level - 1)) + 1 : 0;
  return MLMC_OK;
}

void worker_loop(mlmc_service* S) {
  cudaSetDevice(S->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  std::vector<Req> batch;
  std::vector<uint64_t> ids;
  std::vector<double> qf, qc;
  std::vector<int> cf, cc;
  for (;;) {
    int level = -1, nf = 0, nc = 0;
    size_t need = 0;
    batch.clear();
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stopping) {
          lk.unlock();
          cudaStreamDestroy(st);
          return;
        }
        // the level whose oldest request has waited longest
        level = -1;
        double oldest = 1e300;
        for (int l = 0; l < (int)S->queues.size(); ++l)
          if (!S->queues[l].empty() && S->queues[l].front().t_submit < oldest) {
            oldest = S->queues[l].front().t_submit;
            level = l;
          }
        if (level >= 0) {
          auto& q = S->queues[level];
          const double waited_ms = 1e3 * (now_s() - q.front().t_submit);
          const bool full = (int)q.size() >= S->cfg.max_batch;
          if (full || waited_ms >= S->cfg.batch_wait_ms) {
            level_grid(S->cfg, level, &nf, &nc);
            int b = std::min((int)q.size(), S->cfg.max_batch);
            // admission by device bytes: shrink the batch to what fits the budget
            while (b > 0) {
              need = level_batch_bytes(b, nf, nc, S->cfg.field, S->cfg.mg.precision, S->cfg.mg.accel);
              if (S->bytes_in_use + need <= S->cfg.hbm_budget_bytes) break;
              b /= 2;
            }
            if (b == 0 && S->inflight == 0) {
              // a single request larger than the whole budget runs alone
              b = 1;
              need = level_batch_bytes(1, nf, nc, S->cfg.field, S->cfg.mg.precision, S->cfg.mg.accel);
            }
            if (b > 0) {
              for (int i = 0; i < b; ++i) {
                batch.push_back(q.front());
                q.pop_front();
              }
              S->queued -= b;
              S->bytes_in_use += need;
              S->inflight += 1;
              const double t = now_s();
              for (auto& r : batch) S->results[r.ticket].t_start = t;
              break;
            }
          }
        }
        // nothing admissible yet: wait for a submission, a completion or the batch timer
        S->cv_work.wait_for(lk, std::chrono::microseconds(level >= 0 ? 200 : 20000));
      }
    }
    // run the batch on this worker's stream
    const int b = (int)batch.size();
    ids.resize(b);
    qf.assign(b, 0.0);
    qc.assign(b, 0.0);
    cf.assign(b, 0);
    cc.assign(b, 0);
    for (int i = 0; i < b; ++i) ids[i] = batch[i].id;
    int unconv = 0;
    int status = run_level_batch_host(S->cfg.field, S->cfg.mg, nf, nc, ids.data(), b, qf.data(), qc.data(),
                                      cf.data(), cc.data(), &unconv, st);
    const double t = now_s();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (int i = 0; i < b; ++i) {
        mlmc_result& r = S->results[batch[i].ticket];
        r.Qf = qf[i];
        r.Qc = qc[i];
        r.Y = qf[i] - qc[i];
        r.cycles_fine = cf[i];
        r.cycles_coarse = cc[i];
        r.t_done = t;
        if (status < 0)
          r.status = status;
        else if (S->cfg.mg.rtol > 0.0 && unconv > 0 && (cf[i] >= S->cfg.mg.max_cycles || cc[i] >= S->cfg.mg.max_cycles))
          r.status = MLMC_ERR_NOT_CONVERGED;
        else
          r.status = MLMC_OK;
        S->latencies[level].push_back(t - r.t_submit);
      }
      S->completed += b;
      S->t_last = t;
      S->bytes_in_use -= need;
      S->inflight -= 1;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = p * (double)(v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - (double)i;
  return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace
}  // namespace mlmc

using namespace mlmc;

extern "C" {

mlmc_service* mlmc_service_create(const mlmc_service_cfg* cfg) {
  if (!cfg || cfg->max_batch < 1 || cfg->max_batch > 65535 || cfg->workers < 1 || cfg->workers > 16 ||
      cfg->queue_capacity < 1 || cfg->hbm_budget_bytes == 0 || !valid_grid(cfg->n0) || cfg->max_level < 0 ||
      cfg->max_level > 8 || cfg->batch_wait_ms < 0.0) {
    set_error("mlmc_service_create: invalid configuration");
    return nullptr;
  }
  if (validate_level_cfg(cfg->field, cfg->mg) != MLMC_OK) return nullptr;
  int nf = 0, nc = 0;
  if (level_grid(*cfg, cfg->max_level, &nf, &nc) != MLMC_OK) {
    set_error("mlmc_service_create: max_level %d gives a grid beyond 1025", cfg->max_level);
    return nullptr;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_error("mlmc_service_create: no usable CUDA device");
    return nullptr;
  }
  mlmc_service* S = new mlmc_service();
  S->cfg = *cfg;
  S->device = dev;
  S->queues.resize(cfg->max_level + 1);
  S->latencies.resize(cfg->max_level + 1);
  for (int i = 0; i < cfg->workers; ++i) S->workers.emplace_back(worker_loop, S);
  return S;
}

void mlmc_service_destroy(mlmc_service* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  delete S;
}

int mlmc_submit(mlmc_service* S, const mlmc_request* req, uint64_t* ticket) {
  if (!S || !req || !ticket) {
    set_error("mlmc_submit: NULL argument");
    return MLMC_ERR_INVALID;
  }
  if (req->level < 0 || req->level > S->cfg.max_level) {
    set_error("mlmc_submit: level %d outside 0..%d", req->level, S->cfg.max_level);
    return MLMC_ERR_INVALID;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->queued >= S->cfg.queue_capacity) {
      ++S->rejected;
      set_error("mlmc_submit: queue full (%d pending)", S->cfg.queue_capacity);
      return MLMC_ERR_BUSY;
    }
    const double t = now_s();
    const uint64_t tk = S->next_ticket++;
    S->queues[req->level].push_back(Req{tk, req->level, req->sample_id, t});
    mlmc_result r;
    memset(&r, 0, sizeof(r));
    r.status = MLMC_PENDING;
    r.level = req->level;
    r.sample_id = req->sample_id;
    r.t_submit = t;
    S->results[tk] = r;
    ++S->queued;
    ++S->submitted;
    if (S->submitted == 1) S->t_first = t;
    *ticket = tk;
  }
  S->cv_work.notify_one();
  return MLMC_OK;
}

int mlmc_poll(mlmc_service* S, uint64_t ticket, mlmc_result* res) {
  if (!S || !res) {
    set_error("mlmc_poll: NULL argument");
    return MLMC_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->results.find(ticket);
  if (it == S->results.end()) {
    set_error("mlmc_poll: unknown ticket %llu", (unsigned long long)ticket);
    return MLMC_ERR_NOT_FOUND;
  }
  *res = it->second;
  if (it->second.status == MLMC_PENDING) return MLMC_PENDING;
  S->results.erase(it);  // a finished result is delivered once
  return MLMC_OK;
}

int mlmc_cancel(mlmc_service* S, uint64_t ticket) {
  if (!S) {
    set_error("mlmc_cancel: NULL service");
    return MLMC_ERR_INVALID;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) {
      set_error("mlmc_cancel: unknown ticket %llu", (unsigned long long)ticket);
      return MLMC_ERR_NOT_FOUND;
    }
    auto& q = S->queues[it->second.level];
    auto qi = std::find_if(q.begin(), q.end(), [&](const Req& r) { return r.ticket == ticket; });
    if (qi == q.end()) {
      set_error("mlmc_cancel: ticket %llu is already running or finished", (unsigned long long)ticket);
      return MLMC_ERR_BUSY;
    }
    q.erase(qi);
    --S->queued;
    ++S->cancelled;
    it->second.status = MLMC_ERR_CANCELLED;
    it->second.t_done = now_s();
  }
  S->cv_done.notify_all();
  return MLMC_OK;
}

int mlmc_wait(mlmc_service* S, uint64_t ticket, double timeout_ms, mlmc_result* res) {
  if (!S || !res) {
    set_error("mlmc_wait: NULL argument");
    return MLMC_ERR_INVALID;
  }
  const auto deadline = Clock::now() + std::chrono::microseconds((long long)(timeout_ms * 1e3));
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    auto it = S->results.find(ticket);
    if (it == S->results.end()) {
      set_error("mlmc_wait: unknown ticket %llu", (unsigned long long)ticket);
      return MLMC_ERR_NOT_FOUND;
    }
    if (it->second.status != MLMC_PENDING) {
      *res = it->second;
      S->results.erase(it);
      return MLMC_OK;
    }
    if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      *res = it->second;
      set_error("mlmc_wait: ticket %llu still pending after %.1f ms", (unsigned long long)ticket, timeout_ms);
      return MLMC_ERR_TIMEOUT;
    }
  }
}

int mlmc_service_stats(mlmc_service* S, mlmc_service_report* out) {
  if (!S || !out) {
    set_error("mlmc_service_stats: NULL argument");
    return MLMC_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->rejected = S->rejected;
  out->cancelled = S->cancelled;
  out->pending = S->queued;
  out->inflight_batches = S->inflight;
  out->bytes_in_use = S->bytes_in_use;
  const double span = S->t_last - S->t_first;
  out->samples_per_s = span > 0.0 ? (double)S->completed / span : 0.0;
  for (int l = 0; l < (int)S->latencies.size() && l < 9; ++l) {
    out->count[l] = (int64_t)S->latencies[l].size();
    out->p50_ms[l] = 1e3 * percentile(S->latencies[l], 0.50);
    out->p99_ms[l] = 1e3 * percentile(S->latencies[l], 0.99);
  }
  return MLMC_OK;
}

}  // extern "C"
