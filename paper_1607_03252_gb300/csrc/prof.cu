// Launch accounting and optional per-launch CUDA-event timing (see prof.cuh).
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "prof.cuh"

namespace mlmc {
namespace prof {

namespace {

struct Entry {
  int64_t launches = 0;
  double bytes = 0.0, flops = 0.0;
  double ms = 0.0;      // resolved event time
  int64_t timed = 0;    // launches with resolved events
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};

struct Registry {
  std::mutex mu;
  std::map<std::string, Entry> entries;
  std::vector<std::pair<std::string, cudaEvent_t>> open;  // token -> (class, start event)
  std::atomic<bool> timing{false};
  std::atomic<int64_t> total_launches{0};
};

Registry& reg() {
  static Registry* r = new Registry();  // never destroyed: events may outlive static teardown
  return *r;
}

cudaEvent_t make_event() {
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void resolve(Entry& e) {
  for (auto& pr : e.pending) {
    float ms = 0.f;
    if (pr.first && pr.second && cudaEventSynchronize(pr.second) == cudaSuccess &&
        cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
      e.ms += ms;
      ++e.timed;
    }
    if (pr.first) cudaEventDestroy(pr.first);
    if (pr.second) cudaEventDestroy(pr.second);
  }
  e.pending.clear();
}

}  // namespace

bool timing_enabled() { return reg().timing.load(); }

const char* sized(const char* base, int n) {
  static thread_local char buf[96];
  snprintf(buf, sizeof(buf), "%s@%d", base, n);
  return buf;
}

static thread_local Tape* t_tape = nullptr;
static thread_local Tape t_tape_store;

void tape_begin() {
  t_tape_store = Tape();
  t_tape = &t_tape_store;
}

Tape tape_end() {
  t_tape = nullptr;
  return t_tape_store;
}

void tape_replay(const Tape& t, double scale) {
  Registry& r = reg();
  r.total_launches.fetch_add((int64_t)t.cls.size());
  std::lock_guard<std::mutex> lk(r.mu);
  for (size_t i = 0; i < t.cls.size(); ++i) {
    Entry& e = r.entries[t.cls[i]];
    ++e.launches;
    e.bytes += scale * t.bytes[i];
    e.flops += scale * t.flops[i];
  }
}

int begin(const char* cls, double bytes, double flops, cudaStream_t st) {
  if (t_tape) {  // being captured into a graph: counted when the graph is replayed
    t_tape->cls.emplace_back(cls);
    t_tape->bytes.push_back(bytes);
    t_tape->flops.push_back(flops);
    return -1;
  }
  Registry& r = reg();
  r.total_launches.fetch_add(1);
  std::lock_guard<std::mutex> lk(r.mu);
  Entry& e = r.entries[cls];
  ++e.launches;
  e.bytes += bytes;
  e.flops += flops;
  if (!r.timing.load()) return -1;
  cudaEvent_t a = make_event();
  if (a) cudaEventRecord(a, st);
  r.open.emplace_back(std::string(cls), a);
  return (int)r.open.size() - 1;
}

void end(int token, cudaStream_t st) {
  if (token < 0) return;
  Registry& r = reg();
  std::lock_guard<std::mutex> lk(r.mu);
  if (token >= (int)r.open.size()) return;
  cudaEvent_t b = make_event();
  if (b) cudaEventRecord(b, st);
  auto& o = r.open[token];
  r.entries[o.first].pending.emplace_back(o.second, b);
  o.second = nullptr;
  // tokens are consumed in LIFO order by the RAII scopes
  while (!r.open.empty() && r.open.back().second == nullptr) r.open.pop_back();
}

}  // namespace prof
}  // namespace mlmc

namespace mlmc {
namespace {
// FMA throughput probe: every thread runs 8 independent dependency chains of `iters` FMAs
// (x = x * a + b); the inputs come from arguments so nothing folds, and the sum of the
// chains is stored only when it equals a value it never takes (out[0] stays untouched).
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T a, T b, T never, T* out) {
  T x0 = (T)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, b);
    x1 = fma(x1, a, b);
    x2 = fma(x2, a, b);
    x3 = fma(x3, a, b);
    x4 = fma(x4, a, b);
    x5 = fma(x5, a, b);
    x6 = fma(x6, a, b);
    x7 = fma(x7, a, b);
  }
  const T t = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (t == never) out[0] = t;
}

template <typename T>
int fma_probe(double* tflops) {
  int dev = 0, sms = 0;
  MLMC_CUDA_TRY(cudaGetDevice(&dev));
  MLMC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DevBuf out;
  MLMC_TRY(out.alloc(sizeof(T), nullptr));
  const int iters = 1 << 14, threads = 256, blocks = sms * 8;
  cudaEvent_t e0, e1;
  MLMC_CUDA_TRY(cudaEventCreate(&e0));
  MLMC_CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {  // the first launch warms up; the best of the rest counts
    cudaEventRecord(e0, nullptr);
    k_fma_probe<T><<<blocks, threads>>>(iters, (T)0.999999, (T)1e-7, (T)-12345.0, out.as<T>());
    cudaEventRecord(e1, nullptr);
    MLMC_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    MLMC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  MLMC_CUDA_TRY(cudaGetLastError());
  *tflops = 2.0 * 8.0 * (double)iters * threads * blocks / (best * 1e-3) / 1e12;
  return MLMC_OK;
}
}  // namespace
}  // namespace mlmc

using namespace mlmc;

extern "C" {

int mlmc_profile_fma_peak(int precision, double* tflops) {
  if (!tflops || (precision != MLMC_PREC_F64 && precision != MLMC_PREC_MIXED)) {
    set_error("mlmc_profile_fma_peak: precision must be MLMC_PREC_F64 or MLMC_PREC_MIXED (FP32) and tflops non-NULL");
    return MLMC_ERR_INVALID;
  }
  return precision == MLMC_PREC_F64 ? fma_probe<double>(tflops) : fma_probe<float>(tflops);
}

int mlmc_profile_enable(int on) {
  prof::reg().timing.store(on != 0);
  return MLMC_OK;
}

int mlmc_profile_reset(void) {
  auto& r = prof::reg();
  std::lock_guard<std::mutex> lk(r.mu);
  for (auto& kv : r.entries) {
    for (auto& pr : kv.second.pending) {
      if (pr.first) cudaEventDestroy(pr.first);
      if (pr.second) cudaEventDestroy(pr.second);
    }
  }
  r.entries.clear();
  r.total_launches.store(0);
  return MLMC_OK;
}

int64_t mlmc_profile_total_launches(void) { return prof::reg().total_launches.load(); }

int mlmc_profile_count(void) {
  auto& r = prof::reg();
  std::lock_guard<std::mutex> lk(r.mu);
  return (int)r.entries.size();
}

int mlmc_profile_get(int index, char* name, int name_len, int64_t* launches, int64_t* timed_launches, double* ms,
                     double* bytes, double* flops) {
  auto& r = prof::reg();
  std::lock_guard<std::mutex> lk(r.mu);
  if (index < 0 || index >= (int)r.entries.size() || !name || name_len < 1) {
    set_error("mlmc_profile_get: index %d out of range or bad buffer", index);
    return MLMC_ERR_INVALID;
  }
  auto it = r.entries.begin();
  std::advance(it, index);
  prof::resolve(it->second);
  strncpy(name, it->first.c_str(), (size_t)name_len - 1);
  name[name_len - 1] = 0;
  if (launches) *launches = it->second.launches;
  if (timed_launches) *timed_launches = it->second.timed;
  if (ms) *ms = it->second.ms;
  if (bytes) *bytes = it->second.bytes;
  if (flops) *flops = it->second.flops;
  return MLMC_OK;
}

}  // extern "C"
