// HSAW sampling (Sec. 4, Alg. 1-3) on sm_103a.
//
// Attempt a is one live-edge world: node v's live in-edge and source coin come from
// Philox(seed; a, v), so a walk is a trajectory of a functional graph and O(1)-space cycle
// detection (the idea of Sec. 4.2.2) is exact: any revisit proves the cycle.  A persistent warp claims
// chunks of consecutive attempts; lanes that finish take the next attempt of the warp's
// chunk cursor at once (no lane waits for the warp's longest walk).  Hits are recorded
// per chunk as (attempt offset, length); the compaction kernel orders each chunk's hits
// by attempt id and places them by an exclusive scan over chunks, so the stream is
// ordered by attempt id regardless of which warp ran what.  Hit walks are then
// re-derived from their attempt id (the paper's <Seed_h, Len_h> path encoding) straight
// into the flat walk buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "solver.cuh"

namespace hsaw {

enum : uint32_t { ST_OVERFLOW = 1u, ST_STEP_CAP = 2u };

struct SampleParams {
  const uint4* __restrict__ node;
  const uint2* __restrict__ edge;
  const uint4* __restrict__ erec;
  const uint4* __restrict__ grec;
  const uint32_t* __restrict__ s_bits;
  const uint32_t* __restrict__ p32;
  const uint8_t* __restrict__ edge_removed;
  const uint8_t* __restrict__ node_removed;
  uint32_t n;
  uint32_t k0, k1;
  uint64_t a0;           // first attempt of this launch
  uint32_t n_attempts;   // attempts in this launch
  uint32_t chunk;        // attempts per chunk
  uint32_t n_chunks;
  uint32_t cap;          // hit records per chunk
  uint32_t step_cap;
  uint32_t* chunk_ctr;   // [0] work counter, [1] status bits
  uint32_t* chunk_hits;  // n_chunks
  uint2* recs;           // n_chunks * cap
  unsigned long long* steps;
  PhiloxKeys keys;       // round keys of (k0, k1)
};

template <bool HAS_P, bool HAS_REM>
__global__ void __launch_bounds__(256, 6) k_sample(const __grid_constant__ SampleParams P) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t cur = 0, cur_end = 0;  // warp's attempt cursor within the launch
  bool more = true;
  bool active = false;
  uint32_t off = 0, v = 0, len = 0;
  uint4 rec = make_uint4(0, 0, 0, 0);  // node record of v: first in-edge, in-degree, equal weight, in-sum
  Ckpt ck;
  ck.reset(0);
  unsigned long long my_steps = 0;
  for (;;) {
    unsigned need = __ballot_sync(FULL, !active);
    while (need) {
      if (cur >= cur_end) {
        if (!more) break;
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(P.chunk_ctr, 1u);
        c = __shfl_sync(FULL, c, 0);
        if (c >= P.n_chunks) { more = false; break; }
        cur = c * P.chunk;
        cur_end = min(cur + P.chunk, P.n_attempts);
      }
      const uint32_t avail = cur_end - cur;
      const uint32_t rank = __popc(need & lt);
      if (!active && rank < avail) {
        off = cur + rank;
        {
          const uint64_t a = P.a0 + off;
          v = __umulhi(philox4x32_10_rk(make_uint4((uint32_t)a, (uint32_t)(a >> 32), 0u, 1u), P.keys).x, P.n);
        }
        rec = __ldg(&P.node[v]);
        ck.reset(v);
        len = 1;
        active = true;
      }
      cur += min((uint32_t)__popc(need), avail);
      need = __ballot_sync(FULL, !active);
    }
    if (!__any_sync(FULL, active)) break;
    if (active) {
      // one live-edge draw at node v (Alg. 1 lines 5-13); the tail's record comes with it
      const uint64_t a = P.a0 + off;
      int outcome = -1;  // -1 continue, 0 miss, 1 hit
      if (HAS_REM && len == 1 && P.node_removed && P.node_removed[v]) outcome = 0;
      if (outcome < 0) {
        const uint32_t sw = __ldg(&P.s_bits[v >> 5]);
        const uint4 x = philox4x32_10_rk(make_uint4((uint32_t)a, (uint32_t)(a >> 32), v, 0u), P.keys);
        const bool live = x.x < rec.w;
        uint4 ra = make_uint4(0, 0, 0, 0), rb = make_uint4(0, 0, 0, 0);
        uint32_t e = 0;
        if (live) {
          if (rec.z) {  // equal weights: j = r / w
            e = rec.x + x.x / rec.z;
            ra = __ldg(&P.erec[2 * (size_t)e]);
            rb = __ldg(&P.erec[2 * (size_t)e + 1]);
          } else {  // the bucket's candidate record, then step through the walk records
            const size_t gp = 2 * ((size_t)rec.x + guide_bucket(x.x, rec.y, rec.w));
            ra = __ldg(&P.grec[gp]);
            rb = __ldg(&P.grec[gp + 1]);
            e = rec.x + rb.z;
            if (x.x >= rb.y) {
              do {
                ++e;
                rb = __ldg(&P.erec[2 * (size_t)e + 1]);
              } while (x.x >= rb.y);
              ra = __ldg(&P.erec[2 * (size_t)e]);
            }
          }
        }
        const bool suspect = (sw >> (v & 31)) & 1u;
        if (suspect && (!HAS_P || source_coin(x.y, __ldg(&P.p32[v])))) {
          outcome = 1;
        } else {
          ++my_steps;
          if (!live) {
            outcome = 0;  // no live in-edge
          } else {
            const uint32_t u = ra.x;
            if (HAS_REM && ((P.edge_removed && P.edge_removed[e]) || (P.node_removed && P.node_removed[u]))) {
              outcome = 0;
            } else if (ck.seen(u)) {
              outcome = 0;  // the walk closed a cycle
            } else {
              ck.keep(u, len);
              v = u;
              rec = make_uint4(ra.y, ra.z, ra.w, rb.x);
              if (++len > P.step_cap) {
                atomicOr(P.chunk_ctr + 1, ST_STEP_CAP);
                outcome = 0;
              }
            }
          }
        }
      }
      if (outcome >= 0) {
        active = false;
        if (outcome == 1) {
          const uint32_t ck_i = off / P.chunk;
          const uint32_t slot = atomicAdd(&P.chunk_hits[ck_i], 1u);
          if (slot < P.cap) P.recs[(size_t)ck_i * P.cap + slot] = make_uint2(off, len);
          else atomicOr(P.chunk_ctr + 1, ST_OVERFLOW);
        }
      }
    }
  }
  // steps of this warp
#pragma unroll
  for (int o = 16; o; o >>= 1) my_steps += __shfl_down_sync(FULL, my_steps, o);
  if (lane == 0 && my_steps) atomicAdd(P.steps, my_steps);
}

// Order each chunk's hits by attempt id and write them at the chunk's scanned offset.
// One warp per chunk; rank = number of the chunk's records with a smaller offset.
__global__ void k_compact(const uint32_t* __restrict__ chunk_hits, const uint32_t* __restrict__ chunk_off,
                          const uint2* __restrict__ recs, uint32_t cap, uint32_t n_chunks, uint64_t a0,
                          uint64_t* __restrict__ out_aid, uint32_t* __restrict__ out_len) {
  const int lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t ck = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; ck < n_chunks; ck += warps) {
    const uint32_t c = min(chunk_hits[ck], cap);
    if (c == 0) continue;
    const uint2* r = recs + (size_t)ck * cap;
    const uint32_t base = chunk_off[ck];
    for (uint32_t i = lane; i < c; i += 32) {
      const uint2 me = r[i];
      uint32_t rank = 0;
      for (uint32_t j = 0; j < c; ++j) rank += (r[j].x < me.x) ? 1u : 0u;
      out_aid[base + rank] = a0 + me.x;
      out_len[base + rank] = me.y;
    }
  }
}

__global__ void k_clamp(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, uint32_t n, uint32_t cap) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = min(in[i], cap);
}

__global__ void k_len_to_u64(const uint32_t* __restrict__ len, int64_t n, uint64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = len[i];
}

__global__ void k_offsets(const uint64_t* __restrict__ excl, int64_t n, int64_t base, int64_t* __restrict__ node_off,
                          const uint64_t* __restrict__ total) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
    node_off[i] = base + (int64_t)(i < n ? excl[i] : *total);
}

// Re-derive hit walks from their attempt ids (path encoding) into the flat buffers.
__global__ void k_rewalk(const uint4* __restrict__ node, const uint4* __restrict__ erec, const uint4* __restrict__ grec,
                         uint32_t n, uint32_t k0, uint32_t k1, const uint64_t* __restrict__ aid,
                         const uint32_t* __restrict__ len, const int64_t* __restrict__ node_off, int64_t h0, int64_t h1,
                         int32_t* __restrict__ nodes, int32_t* __restrict__ edges) {
  for (int64_t h = h0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < h1; h += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = aid[h];
    const uint32_t l = len[h];
    const int64_t nb = node_off[h], eb = nb - h;
    uint32_t v = start_node(a, n, k0, k1);
    nodes[nb] = (int32_t)v;
    uint4 rec = l > 1 ? __ldg(&node[v]) : make_uint4(0, 0, 0, 0);
    for (uint32_t i = 1; i < l; ++i) {
      const uint4 x = node_draw(a, v, k0, k1);
      if (x.x >= rec.w) break;  // a hit's walk has a live in-edge at each of its first l - 1 nodes
      uint4 ra, rb;
      const uint32_t e = record_step(erec, grec, rec, x.x, ra, rb);
      nodes[nb + i] = (int32_t)ra.x;
      edges[eb + i - 1] = (int32_t)e;
      v = ra.x;
      rec = make_uint4(ra.y, ra.z, ra.w, rb.x);
    }
  }
}

// Per-attempt outcome (0 no edge, 1 hit, 2 cycle, 3 removed) and nodes walked.
template <bool HAS_P, bool HAS_REM>
__global__ void k_classify(SampleParams P, uint64_t first, int64_t count, int8_t* __restrict__ outcome,
                           int32_t* __restrict__ length) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = first + (uint64_t)i;
    uint32_t v = start_node(a, P.n, P.k0, P.k1), len = 1;
    Ckpt ck;
    ck.reset(v);
    int out = -1;
    if (HAS_REM && P.node_removed && P.node_removed[v]) out = 3;
    while (out < 0) {
      const bool suspect = (__ldg(&P.s_bits[v >> 5]) >> (v & 31)) & 1u;
      const uint4 x = node_draw(a, v, P.k0, P.k1);
      if (suspect && (!HAS_P || source_coin(x.y, __ldg(&P.p32[v])))) { out = 1; break; }
      const uint4 nd = __ldg(&P.node[v]);
      if (x.x >= nd.w) { out = 0; break; }
      const uint32_t e = nd.x + pick_in_edge(P.edge, nd, x.x);
      const uint32_t u = __ldg(&P.edge[e].x);
      if (HAS_REM && ((P.edge_removed && P.edge_removed[e]) || (P.node_removed && P.node_removed[u]))) { out = 3; break; }
      if (ck.seen(u)) { out = 2; break; }
      ck.keep(u, len);
      v = u;
      if (++len > P.step_cap) { atomicOr(P.chunk_ctr + 1, ST_STEP_CAP); out = 0; break; }
    }
    outcome[i] = (int8_t)out;
    length[i] = (int32_t)len;
  }
}

// ------------------------------------------------------------------ host
__global__ void k_set_bits(const int32_t* __restrict__ src, const uint32_t* __restrict__ p, int32_t cnt,
                           uint32_t* __restrict__ bits, uint32_t* __restrict__ p32) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    const uint32_t v = (uint32_t)src[i];
    atomicOr(&bits[v >> 5], 1u << (v & 31));
    if (p32) p32[v] = p[i];
  }
}

hsaw_status query_upload(const Graph& g, const hsaw_query* q, QueryDev& qd, cudaStream_t s) {
  if (!q) return fail(HSAW_E_INVALID, "query: NULL");
  if (q->n_sources < 1 || !q->sources) return fail(HSAW_E_INVALID, "query: need at least one source");
  std::vector<uint8_t> seen((size_t)g.n, 0);
  for (int32_t i = 0; i < q->n_sources; ++i) {
    int32_t v = q->sources[i];
    if (v < 0 || v >= g.n) return fail(HSAW_E_RANGE, "query: source outside [0, n)");
    if (seen[v]) return fail(HSAW_E_INVALID, "query: duplicate source");
    seen[v] = 1;
  }
  const size_t words = (size_t)(g.n + 31) / 32;
  HSAW_TRY(dmalloc((void**)&qd.s_bits, words * 4, s));
  HSAW_CK(cudaMemsetAsync(qd.s_bits, 0, words * 4, s));
  if (q->p_fixed) {
    HSAW_TRY(dmalloc((void**)&qd.p32, (size_t)g.n * 4, s));
    HSAW_CK(cudaMemsetAsync(qd.p32, 0, (size_t)g.n * 4, s));
  }
  // the source list stays with the query (walk-pool queries read their sources' lists);
  // on failure the caller's query_release frees what was allocated
  HSAW_TRY(dmalloc((void**)&qd.s_list, (size_t)q->n_sources * 4, s));
  qd.n_src = q->n_sources;
  HSAW_CK(cudaMemcpyAsync(qd.s_list, q->sources, (size_t)q->n_sources * 4, cudaMemcpyHostToDevice, s));
  uint32_t* d_p = nullptr;
  if (q->p_fixed) {
    HSAW_TRY(dmalloc((void**)&d_p, (size_t)q->n_sources * 4, s));
    if (cudaMemcpyAsync(d_p, q->p_fixed, (size_t)q->n_sources * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      dfree(d_p, s);
      return fail(HSAW_E_DEVICE, "query: probability upload failed");
    }
  }
  count_launch();
  k_set_bits<<<grid_for(q->n_sources, 256, 1024), 256, 0, s>>>(qd.s_list, d_p, q->n_sources, qd.s_bits, qd.p32);
  const cudaError_t le = cudaGetLastError();
  dfree(d_p, s);
  if (le != cudaSuccess) return fail(HSAW_E_DEVICE, "query: suspect bits launch failed");
  qd.seed = q->seed;
  return HSAW_OK;
}

void query_release(QueryDev& qd, cudaStream_t s) {
  dfree(qd.s_bits, s);
  dfree(qd.s_list, s);
  dfree(qd.p32, s);
  if (qd.owns_removed) {
    dfree(qd.edge_removed, s);
    dfree(qd.node_removed, s);
  }
  qd = QueryDev();
}

void Stream::release(cudaStream_t s) {
  aid.release(s); len.release(s); node_off.release(s); nodes.release(s); edges.release(s);
  chunk_hits.release(s); chunk_off.release(s); ctrs.release(s); recs.release(s); tmp64.release(s);
  pbits.release(s); pcnt.release(s);
}

hsaw_status stream_init(Stream& st, uint64_t first_attempt, uint64_t max_attempts, cudaStream_t s) {
  st.count = 0;
  st.total_nodes = 0;
  st.first_attempt = first_attempt;
  st.next_attempt = first_attempt;
  st.steps = 0;
  st.max_attempts = max_attempts ? max_attempts : (1ull << 62);
  HSAW_TRY(st.node_off.ensure(1024, s));
  HSAW_CK(cudaMemsetAsync(st.node_off.p, 0, sizeof(int64_t), s));
  HSAW_TRY(st.ctrs.ensure(8, s));
  return HSAW_OK;
}

static SampleParams make_params(const Graph& g, const QueryDev& qd) {
  SampleParams P{};
  P.node = g.node;
  P.edge = g.edge;
  P.erec = g.erec;
  P.grec = g.grec;
  P.s_bits = qd.s_bits;
  P.p32 = qd.p32;
  P.edge_removed = qd.edge_removed;
  P.node_removed = qd.node_removed;
  P.n = (uint32_t)g.n;
  P.k0 = (uint32_t)qd.seed;
  P.k1 = (uint32_t)(qd.seed >> 32);
  P.keys = philox_round_keys(P.k0, P.k1);
  P.step_cap = (uint32_t)std::min<uint64_t>(4ull * (uint64_t)g.n + 64ull, 0xFFFFFFF0ull);
  return P;
}

static int sample_blocks_per_sm() {
  static const int cached = [] {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_sample<false, false>, 256, 0);
    return b > 0 ? b : 1;
  }();
  return cached;
}

// Sampler occupancy autotuner.  A walk makes one dependent record read per draw; with the
// records in DRAM the random-read rate of this GPU peaks at 1-2 blocks of 256 per SM and
// falls a little as more requests queue, while graphs whose records sit in L2 are bound by
// issue and want every warp.  So each graph's first two sampler launches of at least 2^23
// attempts run with 6 and 3 blocks per SM (draws per ms by CUDA events on the launching
// stream), and its later launches use 3 if it was faster by more than 3%, else 6.  (Trials
// at 4 and 2 blocks per SM gained nothing on the billion-edge graph and cost up to 47% of a
// launch on L2-resident ones.)  The grid does not change any result: hits are ordered by
// attempt id.  HSAW_SAMPLE_BLOCKS=b in the environment forces b blocks per SM (measurement).
namespace {
constexpr int kTuneN = 2;
constexpr int kTuneCands[kTuneN] = {6, 3};
struct SampleTune {
  int next_trial = 0, done = 0, best = 0;
  float rate[kTuneN] = {0.f, 0.f};
};
std::mutex g_stune_mu;
std::unordered_map<const void*, SampleTune> g_stune;  // keyed by the graph's node array
}  // namespace

void sample_tune_forget(const Graph& g) {
  std::lock_guard<std::mutex> lk(g_stune_mu);
  g_stune.erase(g.node);
}

// Blocks per SM for the next launch over `batch` attempts; *trial >= 0 when it is a timed trial.
static int sample_blocks_for(const Graph& g, uint64_t batch, int* trial) {
  *trial = -1;
  const int full = sample_blocks_per_sm();
  if (const char* f = getenv("HSAW_SAMPLE_BLOCKS")) {
    const int b = atoi(f);
    return std::max(1, std::min(full, b > 0 ? b : full));
  }
  std::lock_guard<std::mutex> lk(g_stune_mu);
  SampleTune& t = g_stune[g.node];
  if (t.best) return std::min(full, t.best);
  if (batch < (1ull << 23) || t.next_trial >= kTuneN) return full;
  *trial = t.next_trial++;
  return std::min(full, kTuneCands[*trial]);
}

static void sample_tune_record(const Graph& g, int trial, double draws, float ms) {
  if (trial < 0 || !(ms > 0.f)) return;
  std::lock_guard<std::mutex> lk(g_stune_mu);
  SampleTune& t = g_stune[g.node];
  t.rate[trial] = (float)(draws / ms);
  if (++t.done < kTuneN) return;
  int best = 0;
  for (int i = 1; i < kTuneN; ++i)
    if (t.rate[i] > t.rate[best] * 1.03f) best = i;
  t.best = kTuneCands[best];
  if (getenv("HSAW_LOG_LAUNCHES"))
    fprintf(stderr, "hsaw: k_sample tuned blocks_per_sm=%d (G draws/s: 6 %.1f, 3 %.1f)\n", t.best, t.rate[0] / 1e6,
            t.rate[1] / 1e6);
}

static void launch_sample(const SampleParams& P, unsigned grid, cudaStream_t s) {
  const bool hp = P.p32 != nullptr, hr = (P.edge_removed || P.node_removed);
  if (hp && hr) { count_launch(); k_sample<true, true><<<grid, 256, 0, s>>>(P); }
  else if (hp) { count_launch(); k_sample<true, false><<<grid, 256, 0, s>>>(P); }
  else if (hr) { count_launch(); k_sample<false, true><<<grid, 256, 0, s>>>(P); }
  else { count_launch(); k_sample<false, false><<<grid, 256, 0, s>>>(P); }
}

// One sampler launch over attempts [st.next_attempt, + batch): hits are recorded per chunk
// and compacted in attempt order into aid/len at st.count; *new_hits receives their number.
static hsaw_status sample_window(const Graph& g, const QueryDev& qd, Stream& st, uint64_t batch, uint32_t* new_hits,
                                 cudaStream_t s) {
  SampleParams P = make_params(g, qd);
  const uint32_t CHUNK = 256;
  const uint32_t n_chunks = (uint32_t)((batch + CHUNK - 1) / CHUNK);
  // records per chunk: a few standard deviations above the expected hits, else all
  double exp_hits = std::max(st.hit_rate, 0.0) * CHUNK;
  uint32_t cap = (uint32_t)std::min<double>(CHUNK, std::ceil(exp_hits + 6.0 * std::sqrt(exp_hits + 1.0) + 8.0));
  if (st.hit_rate == 0.0) cap = CHUNK;
  for (;;) {
    HSAW_TRY(st.tmp64.ensure(1, s));
    HSAW_TRY(st.chunk_hits.ensure(n_chunks, s));
    HSAW_TRY(st.chunk_off.ensure(n_chunks, s));
    HSAW_TRY(st.recs.ensure((size_t)n_chunks * cap, s));
    HSAW_CK(cudaMemsetAsync(st.chunk_hits.p, 0, (size_t)n_chunks * 4, s));
    HSAW_CK(cudaMemsetAsync(st.ctrs.p, 0, 8 * 4, s));
    unsigned long long* d_steps = reinterpret_cast<unsigned long long*>(st.tmp64.p);
    HSAW_CK(cudaMemsetAsync(d_steps, 0, 8, s));
    P.a0 = st.next_attempt;
    P.n_attempts = (uint32_t)batch;
    P.chunk = CHUNK;
    P.n_chunks = n_chunks;
    P.cap = cap;
    P.chunk_ctr = st.ctrs.p;
    P.chunk_hits = st.chunk_hits.p;
    P.recs = st.recs.p;
    P.steps = d_steps;
    int trial = -1;
    const int bps = sample_blocks_for(g, batch, &trial);
    const unsigned grid = (unsigned)std::max(1, std::min<int>(sm_count() * bps, (int)((n_chunks + 7) / 8)));
    cudaEvent_t tev[2] = {nullptr, nullptr};
    if (trial >= 0 && (cudaEventCreate(&tev[0]) != cudaSuccess || cudaEventCreate(&tev[1]) != cudaSuccess)) {
      cudaGetLastError();
      trial = -1;
    }
    if (trial >= 0) cudaEventRecord(tev[0], s);
    void* prof = profile_begin(s);
    launch_sample(P, grid, s);
    profile_end(prof, s, batch);
    if (trial >= 0) cudaEventRecord(tev[1], s);
    HSAW_CK(cudaGetLastError());
    count_launch();
    k_clamp<<<grid_for(n_chunks, 256, 4096), 256, 0, s>>>(st.chunk_hits.p, st.chunk_off.p, n_chunks, cap);
    HSAW_CK(cudaGetLastError());
    HSAW_TRY(exclusive_scan_u32(st.chunk_off.p, n_chunks, st.ctrs.p + 2, s));
    uint32_t h[4];
    unsigned long long hs = 0;
    HSAW_CK(cudaMemcpyAsync(h, st.ctrs.p, 16, cudaMemcpyDeviceToHost, s));
    HSAW_CK(cudaMemcpyAsync(&hs, d_steps, 8, cudaMemcpyDeviceToHost, s));
    HSAW_CK(cudaStreamSynchronize(s));
    if (trial >= 0) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, tev[0], tev[1]) == cudaSuccess) sample_tune_record(g, trial, (double)hs, ms);
      cudaEventDestroy(tev[0]);
      cudaEventDestroy(tev[1]);
    }
    if (h[1] & ST_STEP_CAP) return fail(HSAW_E_STEP_CAP, "sampling: a walk exceeded its step guard");
    if ((h[1] & ST_OVERFLOW) && cap < CHUNK) {
      cap = CHUNK;  // rare: rerun this launch with room for every attempt to hit
      continue;
    }
    st.steps += hs;
    profile_add_steps(hs);
    if (getenv("HSAW_LOG_LAUNCHES"))  // measurement aid: attempts and live-edge draws of each sampler launch
      fprintf(stderr, "hsaw: k_sample launch attempts=%llu draws=%llu blocks_per_sm=%d\n", (unsigned long long)batch,
              hs, bps);
    *new_hits = h[2];
    if (h[2]) {
      HSAW_TRY(st.aid.ensure((size_t)st.count + h[2], s, true));
      HSAW_TRY(st.len.ensure((size_t)st.count + h[2], s, true));
      count_launch();
      k_compact<<<grid_for((size_t)n_chunks * 32, 256, 8192), 256, 0, s>>>(
          st.chunk_hits.p, st.chunk_off.p, st.recs.p, cap, n_chunks, st.next_attempt, st.aid.p + st.count,
          st.len.p + st.count);
      HSAW_CK(cudaGetLastError());
    }
    return HSAW_OK;
  }
}

hsaw_status stream_extend(const Graph& g, const QueryDev& qd, Stream& st, int64_t want, cudaStream_t s) {
  st.elem_range[0] = g.n;
  st.elem_range[1] = g.m;
  const uint32_t CHUNK = 256;
  // the walk pool serves this query's attempts below pool.attempts when the walk seed
  // matches and the graph is not a residual one
  const bool pool_ok = g.pool.ent && g.pool.seed == qd.seed && qd.s_list && !qd.edge_removed && !qd.node_removed;
  while (st.count < want) {
    if (cancel_requested()) return fail(HSAW_E_CANCELLED, "sampling: query cancelled");
    const uint64_t used = st.next_attempt - st.first_attempt;
    if (used >= st.max_attempts) return fail(HSAW_E_TIMEOUT, "sampling: attempt budget exhausted before enough hits");
    // window size from the hit rate so far (2^20 .. 2^28 attempts; doubling while no hit),
    // with a margin of 4 standard deviations of the rate estimate (st.count hits seen) and
    // of the window's own hit count (need): attempts past the last hit a solve uses are
    // wasted, and a window that falls short only costs one more launch
    const double need = (double)(want - st.count);
    st.hit_rate = used ? (double)st.count / (double)used : 0.0;
    const double margin = std::min(1.25, 1.0 + 4.0 / std::sqrt(std::max(1.0, (double)st.count)) + 4.0 / std::sqrt(need));
    double target = st.hit_rate > 0 ? need / st.hit_rate * margin + 4096.0 : std::max(1048576.0, 2.0 * (double)used);
    target = std::max(target, 1048576.0);
    target = std::min(target, 268435456.0);
    uint64_t batch = (uint64_t)target;
    batch = std::min<uint64_t>(batch, st.max_attempts - used);
    uint32_t new_hits = 0;
    if (pool_ok && st.next_attempt < g.pool.attempts) {
      // whole blocks of the index where the pool and the budget allow
      const uint64_t B = 1ull << g.pool.shift;
      uint64_t a1 = std::min<uint64_t>(g.pool.attempts, (st.next_attempt + batch + B - 1) / B * B);
      a1 = std::min<uint64_t>(a1, st.next_attempt + (st.max_attempts - used));
      batch = a1 - st.next_attempt;
      HSAW_TRY(pool_hits(g, qd, st, st.next_attempt, a1, &new_hits, s));
    } else {
      batch = (batch + CHUNK - 1) / CHUNK * CHUNK;
      HSAW_TRY(sample_window(g, qd, st, batch, &new_hits, s));
    }
    HSAW_TRY(stream_take_hits(g, qd, st, new_hits, s));
    st.next_attempt += batch;
  }
  return HSAW_OK;
}

hsaw_status stream_take_hits(const Graph& g, const QueryDev& qd, Stream& st, uint32_t new_hits, cudaStream_t s) {
  if (!new_hits) return HSAW_OK;
  const uint32_t k0 = (uint32_t)qd.seed, k1 = (uint32_t)(qd.seed >> 32);
  // walk offsets, then the hits' nodes and edges re-drawn from their attempt ids
  HSAW_TRY(st.node_off.ensure((size_t)st.count + new_hits + 1, s, true));
  HSAW_TRY(st.tmp64.ensure((size_t)new_hits + 1, s));
  count_launch();
  k_len_to_u64<<<grid_for(new_hits, 256, 4096), 256, 0, s>>>(st.len.p + st.count, new_hits, st.tmp64.p);
  HSAW_CK(cudaGetLastError());
  HSAW_TRY(exclusive_scan_u64(st.tmp64.p, new_hits, st.tmp64.p + new_hits, s));
  count_launch();
  k_offsets<<<grid_for((size_t)new_hits + 1, 256, 4096), 256, 0, s>>>(
      st.tmp64.p, new_hits, st.total_nodes, st.node_off.p + st.count, st.tmp64.p + new_hits);
  HSAW_CK(cudaGetLastError());
  uint64_t added = 0;
  HSAW_CK(cudaMemcpyAsync(&added, st.tmp64.p + new_hits, 8, cudaMemcpyDeviceToHost, s));
  HSAW_CK(cudaStreamSynchronize(s));
  const int64_t tot = st.total_nodes + (int64_t)added;
  HSAW_TRY(st.nodes.ensure((size_t)tot, s, true));
  HSAW_TRY(st.edges.ensure((size_t)tot, s, true));
  count_launch();
  k_rewalk<<<grid_for(new_hits, 128, 1u << 16), 128, 0, s>>>(g.node, g.erec, g.grec, (uint32_t)g.n, k0, k1, st.aid.p,
                                                               st.len.p,
                                                               st.node_off.p, st.count, st.count + new_hits,
                                                               st.nodes.p, st.edges.p);
  HSAW_CK(cudaGetLastError());
  st.total_nodes = tot;
  st.count += new_hits;
  return HSAW_OK;
}

hsaw_status classify_attempts(const Graph& g, const QueryDev& qd, uint64_t first, int64_t count, int8_t* outcome,
                              int32_t* length, cudaStream_t s) {
  SampleParams P = make_params(g, qd);
  uint32_t* d_ctr = nullptr;
  HSAW_TRY(dmalloc((void**)&d_ctr, 16, s));
  HSAW_CK(cudaMemsetAsync(d_ctr, 0, 16, s));
  P.chunk_ctr = d_ctr;
  const unsigned grid = grid_for(count, 128, 1u << 16);
  const bool hp = P.p32 != nullptr, hr = (P.edge_removed || P.node_removed);
  if (hp && hr) { count_launch(); k_classify<true, true><<<grid, 128, 0, s>>>(P, first, count, outcome, length); }
  else if (hp) { count_launch(); k_classify<true, false><<<grid, 128, 0, s>>>(P, first, count, outcome, length); }
  else if (hr) { count_launch(); k_classify<false, true><<<grid, 128, 0, s>>>(P, first, count, outcome, length); }
  else { count_launch(); k_classify<false, false><<<grid, 128, 0, s>>>(P, first, count, outcome, length); }
  HSAW_CK(cudaGetLastError());
  uint32_t h[2] = {0, 0};
  HSAW_CK(cudaMemcpyAsync(h, d_ctr, 8, cudaMemcpyDeviceToHost, s));
  HSAW_CK(cudaStreamSynchronize(s));
  dfree(d_ctr, s);
  if (h[1] & ST_STEP_CAP) return fail(HSAW_E_STEP_CAP, "classify: a walk exceeded its step guard");
  return HSAW_OK;
}

}  // namespace hsaw

// ------------------------------------------------------------------ allocation-free variant
// Scratch of hsaw_sample_hits_static: file-scope device arrays sized for at most
// HSAW_STATIC_MAX_ATTEMPTS attempts per call (about 2 MiB in total).  Every GPU that loads
// this library holds them until the process exits.  Host code cannot pass these names to
// a kernel (in host code they are stand-ins, not device addresses); their device
// addresses are looked up once per device with cudaGetSymbolAddress.
namespace hsaw {

constexpr uint32_t STATIC_CHUNK = 256;
constexpr uint32_t STATIC_CHUNKS = HSAW_STATIC_MAX_ATTEMPTS / STATIC_CHUNK;

static __device__ __align__(256) uint32_t g_static_ctrs[8];                 // work counter, status, total
static __device__ __align__(256) unsigned long long g_static_steps[1];
static __device__ __align__(256) uint32_t g_static_chunk_hits[STATIC_CHUNKS];
static __device__ __align__(256) uint32_t g_static_chunk_off[STATIC_CHUNKS];
static __device__ __align__(256) uint2 g_static_recs[STATIC_CHUNKS * STATIC_CHUNK];

struct StaticScratch {
  uint32_t* ctrs = nullptr;
  unsigned long long* steps = nullptr;
  uint32_t* chunk_hits = nullptr;
  uint32_t* chunk_off = nullptr;
  uint2* recs = nullptr;
  bool ready = false;
};
static StaticScratch g_static_dev[64];
static std::mutex g_static_mu;

// Device addresses of the static scratch on the current device (set-up on first use).
static hsaw_status static_scratch(StaticScratch** out) {
  int dev = 0;
  HSAW_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(HSAW_E_DEVICE, "static sampler: device index out of range");
  std::lock_guard<std::mutex> lk(g_static_mu);
  StaticScratch& s = g_static_dev[dev];
  if (!s.ready) {
    HSAW_CK(cudaGetSymbolAddress((void**)&s.ctrs, g_static_ctrs));
    HSAW_CK(cudaGetSymbolAddress((void**)&s.steps, g_static_steps));
    HSAW_CK(cudaGetSymbolAddress((void**)&s.chunk_hits, g_static_chunk_hits));
    HSAW_CK(cudaGetSymbolAddress((void**)&s.chunk_off, g_static_chunk_off));
    HSAW_CK(cudaGetSymbolAddress((void**)&s.recs, g_static_recs));
    s.ready = true;
  }
  *out = &s;
  return HSAW_OK;
}

// Single-block exclusive scan of at most STATIC_CHUNKS counts (clamped to cap); writes the
// total to *total.  One block of 1024 threads, no temporary memory.
__global__ void __launch_bounds__(1024) k_static_scan(const uint32_t* __restrict__ in, uint32_t n, uint32_t cap,
                                                      uint32_t* __restrict__ out, uint32_t* __restrict__ total) {
  __shared__ uint32_t warp_sum[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (uint32_t base = 0; base < n; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < n ? min(in[i], cap) : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[w] = x;
    __syncthreads();
    uint32_t before = carry;
    for (int k = 0; k < w; ++k) before += warp_sum[k];
    if (i < n) out[i] = before + x - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

}  // namespace hsaw

extern "C" hsaw_status hsaw_sample_hits_static(hsaw_graph g, const uint32_t* suspect_bits, uint64_t seed,
                                               uint64_t first_attempt, int64_t n_attempts, uint64_t* aid_out,
                                               uint32_t* len_out, int64_t out_cap, int64_t* n_hits, void* stream) {
  using namespace hsaw;
  if (!g || !suspect_bits || !n_hits || (out_cap > 0 && (!aid_out || !len_out)))
    return fail(HSAW_E_INVALID, "static sampler: NULL argument");
  *n_hits = 0;
  if (n_attempts < 0 || n_attempts > (int64_t)HSAW_STATIC_MAX_ATTEMPTS)
    return fail(HSAW_E_INVALID, "static sampler: n_attempts must be in [0, HSAW_STATIC_MAX_ATTEMPTS]");
  if (n_attempts == 0) return HSAW_OK;
  const Graph& G = g->g;
  int cur_dev = -1;
  HSAW_CK(cudaGetDevice(&cur_dev));
  if (cur_dev != G.device) return fail(HSAW_E_DEVICE, "static sampler: the current device is not the graph's device");
  StaticScratch* sc = nullptr;
  HSAW_TRY(static_scratch(&sc));
  cudaStream_t s = (cudaStream_t)stream;
  SampleParams P{};
  P.node = G.node;
  P.edge = G.edge;
  P.erec = G.erec;
  P.grec = G.grec;
  P.s_bits = suspect_bits;
  P.n = (uint32_t)G.n;
  P.k0 = (uint32_t)seed;
  P.k1 = (uint32_t)(seed >> 32);
  P.keys = philox_round_keys(P.k0, P.k1);
  P.step_cap = (uint32_t)std::min<uint64_t>(4ull * (uint64_t)G.n + 64ull, 0xFFFFFFF0ull);
  const uint32_t n_chunks = (uint32_t)((n_attempts + STATIC_CHUNK - 1) / STATIC_CHUNK);
  P.a0 = first_attempt;
  P.n_attempts = (uint32_t)n_attempts;
  P.chunk = STATIC_CHUNK;
  P.n_chunks = n_chunks;
  P.cap = STATIC_CHUNK;  // room for every attempt of a chunk to hit: no overflow
  P.chunk_ctr = sc->ctrs;
  P.chunk_hits = sc->chunk_hits;
  P.recs = sc->recs;
  P.steps = sc->steps;
  // the shared scratch keeps the previous call's contents: clear what must start at zero
  HSAW_CK(cudaMemsetAsync(sc->ctrs, 0, sizeof(g_static_ctrs), s));
  HSAW_CK(cudaMemsetAsync(sc->steps, 0, sizeof(g_static_steps), s));
  HSAW_CK(cudaMemsetAsync(sc->chunk_hits, 0, (size_t)n_chunks * sizeof(uint32_t), s));
  const unsigned grid = (unsigned)std::max(1, std::min<int>(sm_count() * sample_blocks_per_sm(),
                                                             (int)((n_chunks + 7) / 8)));
  count_launch();
  k_sample<false, false><<<grid, 256, 0, s>>>(P);
  HSAW_CK(cudaGetLastError());
  count_launch();
  k_static_scan<<<1, 1024, 0, s>>>(sc->chunk_hits, n_chunks, STATIC_CHUNK, sc->chunk_off, sc->ctrs + 2);
  HSAW_CK(cudaGetLastError());
  uint32_t h[4] = {0, 0, 0, 0};
  HSAW_CK(cudaMemcpyAsync(h, sc->ctrs, sizeof(h), cudaMemcpyDeviceToHost, s));
  HSAW_CK(cudaStreamSynchronize(s));
  if (h[1] & ST_STEP_CAP) return fail(HSAW_E_STEP_CAP, "static sampler: a walk exceeded its step guard");
  *n_hits = h[2];
  if ((int64_t)h[2] > out_cap) return fail(HSAW_E_INVALID, "static sampler: more hits than out_cap");
  if (h[2]) {
    count_launch();
    k_compact<<<grid_for((size_t)n_chunks * 32, 256, 8192), 256, 0, s>>>(
        sc->chunk_hits, sc->chunk_off, sc->recs, STATIC_CHUNK, n_chunks, first_attempt, aid_out, len_out);
    HSAW_CK(cudaGetLastError());
  }
  HSAW_CK(cudaStreamSynchronize(s));
  return HSAW_OK;
}
