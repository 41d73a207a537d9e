// Measurement counters: kernel launches and CUDA-event timing of sampler launches.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace hsaw {

static std::atomic<unsigned long long> g_launches{0};
static std::atomic<int> g_enabled{0};
static std::mutex g_mu;
struct Timed {
  cudaEvent_t a, b;
  uint64_t attempts;
};
static std::vector<Timed> g_timed;
struct PhaseTimed {
  cudaEvent_t a, b;
  int phase;
};
static std::vector<PhaseTimed> g_phase;
static uint64_t g_steps = 0, g_sampler_launches = 0, g_attempts = 0;
// Timing events are recycled: creating two per phase in every worker thread of a server
// costs more host time than the phases themselves.
static std::vector<cudaEvent_t> g_free_events;

static bool take_events(cudaEvent_t* a, cudaEvent_t* b) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_free_events.size() >= 2) {
      *a = g_free_events.back();
      g_free_events.pop_back();
      *b = g_free_events.back();
      g_free_events.pop_back();
      return true;
    }
  }
  if (cudaEventCreate(a) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (cudaEventCreate(b) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(*a);
    return false;
  }
  return true;
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void* profile_begin(cudaStream_t s) {
  if (!g_enabled.load()) return nullptr;
  Timed* t = new Timed();
  if (!take_events(&t->a, &t->b)) {
    delete t;
    return nullptr;
  }
  cudaEventRecord(t->a, s);
  return t;
}

void profile_end(void* token, cudaStream_t s, uint64_t attempts) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_sampler_launches++;
  g_attempts += attempts;
  if (!token) return;
  Timed* t = static_cast<Timed*>(token);
  cudaEventRecord(t->b, s);
  t->attempts = attempts;
  g_timed.push_back(*t);
  delete t;
}

void* phase_begin(cudaStream_t s) {
  if (!g_enabled.load()) return nullptr;
  PhaseTimed* t = new PhaseTimed();
  if (!take_events(&t->a, &t->b)) {
    delete t;
    return nullptr;
  }
  cudaEventRecord(t->a, s);
  return t;
}

void phase_end(void* token, cudaStream_t s, int phase) {
  if (!token) return;
  PhaseTimed* t = static_cast<PhaseTimed*>(token);
  cudaEventRecord(t->b, s);
  t->phase = phase;
  std::lock_guard<std::mutex> lk(g_mu);
  g_phase.push_back(*t);
  delete t;
}

void profile_add_steps(uint64_t steps) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_steps += steps;
}

}  // namespace hsaw

using namespace hsaw;

extern "C" {

hsaw_status hsaw_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& t : g_timed) {
    g_free_events.push_back(t.a);
    g_free_events.push_back(t.b);
  }
  g_timed.clear();
  for (auto& t : g_phase) {
    g_free_events.push_back(t.a);
    g_free_events.push_back(t.b);
  }
  g_phase.clear();
  g_steps = g_sampler_launches = g_attempts = 0;
  g_launches.store(0);
  g_enabled.store(on ? 1 : 0);
  return HSAW_OK;
}

hsaw_status hsaw_profile_read(hsaw_profile* out) {
  if (!out) return fail(HSAW_E_INVALID, "profile: NULL out");
  HSAW_CK(cudaDeviceSynchronize());
  std::lock_guard<std::mutex> lk(g_mu);
  double ms = 0.0;
  for (auto& t : g_timed) {
    float x = 0.f;
    if (cudaEventElapsedTime(&x, t.a, t.b) == cudaSuccess) ms += x;
    else cudaGetLastError();
  }
  for (int i = 0; i < 8; ++i) out->phase_ms[i] = 0.0;
  for (auto& t : g_phase) {
    float x = 0.f;
    if (t.phase >= 0 && t.phase < 8 && cudaEventElapsedTime(&x, t.a, t.b) == cudaSuccess) out->phase_ms[t.phase] += x;
    else cudaGetLastError();
  }
  out->kernel_launches = g_launches.load();
  out->sampler_launches = g_sampler_launches;
  out->sampler_ms = ms;
  out->sampler_steps = g_steps;
  out->sampler_attempts = g_attempts;
  return HSAW_OK;
}

}  // extern "C"
