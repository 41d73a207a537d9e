// Measurement counters: kernel launches and CUDA-event timing of sampler launches.
#include <cuda_runtime.h>

#include <algorithm>
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

// ------------------------------------------------------------------ random-gather probe
// The ceiling the sampler's memory pattern runs into: every lane follows a chain of
// dependent reads of random 32-byte records (the size of a walk record), one record per
// step, the next index taken from the record just read - the same one-dependent-read-per-
// draw pattern as a walk, with no Philox or walk logic around it.  `chains` independent
// chains per lane show whether more requests in flight would raise the rate.
namespace hsaw {

__device__ __forceinline__ uint32_t probe_mix(uint32_t x) {  // 32-bit integer finaliser (Murmur3 fmix32)
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

__global__ void k_probe_fill(uint4* __restrict__ t, uint64_t n_records, uint32_t salt) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_records;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t h = probe_mix((uint32_t)i ^ probe_mix((uint32_t)(i >> 32) + salt));
    t[2 * i] = make_uint4(h, h ^ 0x9E3779B9u, (uint32_t)i, 0u);
    t[2 * i + 1] = make_uint4(~h, 0u, 0u, 0u);
  }
}

template <int CHAINS>
__global__ void __launch_bounds__(256, 6) k_probe_gather(const uint4* __restrict__ t, uint64_t n_records,
                                                         uint32_t steps, unsigned long long* __restrict__ sink) {
  const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t idx[CHAINS];
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) idx[c] = (uint32_t)(((uint64_t)probe_mix(gid * CHAINS + c + 1) * n_records) >> 32);
  for (uint32_t s = 0; s < steps; ++s) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
      const uint4 a = __ldg(&t[2 * (size_t)idx[c]]);
      const uint4 b = __ldg(&t[2 * (size_t)idx[c] + 1]);
      acc += a.w + b.y;
      idx[c] = (uint32_t)(((uint64_t)probe_mix(a.x ^ (s * 0x27D4EB2Fu) ^ gid) * n_records) >> 32);
    }
  }
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) acc += idx[c];
  if (acc == 0x12345678u) atomicAdd(sink, 1ull);  // keeps the loads live; practically never taken
}

}  // namespace hsaw

extern "C" hsaw_status hsaw_probe_gather(uint64_t table_bytes, int32_t chains, uint32_t steps, int32_t blocks_per_sm,
                                         double* reads_per_s, double* ms, void* stream) {
  using namespace hsaw;
  if (!reads_per_s || table_bytes < 64 || (chains != 1 && chains != 2 && chains != 4) || steps < 1)
    return fail(HSAW_E_INVALID, "probe: need table_bytes >= 64, chains in {1, 2, 4}, steps >= 1");
  const uint64_t n_records = std::min<uint64_t>(table_bytes / 32, 1ull << 32);
  cudaStream_t s = (cudaStream_t)stream;
  void* t = nullptr;
  HSAW_TRY(dmalloc(&t, n_records * 32 + 64, s));
  unsigned long long* sink = reinterpret_cast<unsigned long long*>((char*)t + n_records * 32);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hsaw_status st = HSAW_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = fail(HSAW_E_DEVICE, "probe: events");
  int bps = 0;
  if (st == HSAW_OK) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_probe_gather<1>, 256, 0);
    count_launch();
    k_probe_fill<<<sm_count() * 8, 256, 0, s>>>((uint4*)t, n_records, 0x5EEDu);
    cudaMemsetAsync(sink, 0, 8, s);
    if (blocks_per_sm > 0) bps = std::min(bps, (int)blocks_per_sm);
    const unsigned grid = (unsigned)(sm_count() * std::max(bps, 1));
    for (int rep = 0; rep < 2 && st == HSAW_OK; ++rep) {  // the first pass warms up, the second is timed
      cudaEventRecord(e0, s);
      count_launch();
      if (chains == 1) k_probe_gather<1><<<grid, 256, 0, s>>>((const uint4*)t, n_records, steps, sink);
      else if (chains == 2) k_probe_gather<2><<<grid, 256, 0, s>>>((const uint4*)t, n_records, steps, sink);
      else k_probe_gather<4><<<grid, 256, 0, s>>>((const uint4*)t, n_records, steps, sink);
      cudaEventRecord(e1, s);
      if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
        st = fail(HSAW_E_DEVICE, "probe: launch failed");
    }
    float t_ms = 0.f;
    if (st == HSAW_OK) {
      cudaEventElapsedTime(&t_ms, e0, e1);
      *reads_per_s = (double)grid * 256.0 * chains * steps / (t_ms * 1e-3);
      if (ms) *ms = t_ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dfree(t, s);
  cudaStreamSynchronize(s);
  return st;
}
