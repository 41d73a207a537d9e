// Occurrence counting, inverted index, greedy max-coverage and out-of-sample coverage
// over the ordered HSAW stream (Alg. 4 / 7 "Greedy", Alg. 5 line 2 "Cov_{R'_t}").
//
// The walk elements of a range of walks are sorted by element id with their entry
// positions (stable radix sort): the runs give the touched elements in increasing id
// with their occurrence counts, and the run contents are the inverted index element ->
// walks.  Greedy runs k rounds in ONE cooperative launch: a grid-wide argmax of
// (count, -index) packed in 64 bits (ties to the smallest id), then the picked
// element's uncovered walks are marked and every element of those walks is decremented.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "solver.cuh"

namespace hsaw {

enum : uint32_t { GS_BARRIER_TIMEOUT = 1u };

void Cover::release(cudaStream_t s) {
  keys.release(s); vals.release(s); keys2.release(s); vals2.release(s); run_flag.release(s);
  uid.release(s); cnt.release(s); inv_off.release(s); inv_walk.release(s); entry_uidx.release(s);
  walk_eoff.release(s); cnt_work.release(s); covered.release(s); dirty.release(s); partial.release(s);
  inv_ent.release(s); g_idx.release(s); g_list.release(s); g_cnt.release(s); g_entry.release(s); g_rng.release(s);
}

// entry offsets of walks [first, first + count) relative to the first walk's first entry
__global__ void k_walk_eoff(const int64_t* __restrict__ node_off, int64_t first, int64_t count, int edge_mode,
                            uint32_t* __restrict__ eoff) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= count; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = first + i;
    const int64_t b0 = node_off[first] - (edge_mode ? first : 0);
    eoff[i] = (uint32_t)(node_off[j] - (edge_mode ? j : 0) - b0);
  }
}

__global__ void k_keys_iota(const int32_t* __restrict__ el, uint32_t E, uint32_t* __restrict__ keys,
                            uint32_t* __restrict__ vals) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < E; p += gridDim.x * blockDim.x) {
    keys[p] = (uint32_t)el[p];
    vals[p] = p;
  }
}

__global__ void k_walk_of_entry(const uint32_t* __restrict__ eoff, uint32_t count, uint32_t* __restrict__ wof) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    for (uint32_t p = eoff[i]; p < eoff[i + 1]; ++p) wof[p] = i;
}

__global__ void k_run_flags(const uint32_t* __restrict__ skeys, uint32_t E, uint32_t* __restrict__ flag) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < E; q += gridDim.x * blockDim.x)
    flag[q] = (q == 0 || skeys[q] != skeys[q - 1]) ? 1u : 0u;
}

// excl = exclusive scan of the run flags
__global__ void k_runs(const uint32_t* __restrict__ skeys, const uint32_t* __restrict__ svals,
                       const uint32_t* __restrict__ excl, const uint32_t* __restrict__ wof, uint32_t E,
                       int32_t* __restrict__ uid, uint32_t* __restrict__ inv_off, uint32_t* __restrict__ inv_walk,
                       uint32_t* __restrict__ entry_uidx) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < E; q += gridDim.x * blockDim.x) {
    const bool start = (q == 0 || skeys[q] != skeys[q - 1]);
    const uint32_t r = excl[q] + (start ? 1u : 0u) - 1u;
    if (start) {
      uid[r] = (int32_t)skeys[q];
      inv_off[r] = q;
    }
    const uint32_t p = svals[q];
    inv_walk[q] = wof[p];
    entry_uidx[p] = r;
  }
}

__global__ void k_counts(const uint32_t* __restrict__ inv_off, uint32_t U, uint32_t* __restrict__ cnt) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < U; r += gridDim.x * blockDim.x)
    cnt[r] = inv_off[r + 1] - inv_off[r];
}

// ------------------------------------------------------------------ dense strategy
// Counts by atomics into a dense array over the element range [0, M), touched elements by
// an exclusive scan of the nonzero flags (so uid stays increasing), the inverted index by
// a counting fill (walks within one element's list in arrival order: the greedy treats a
// list as a set, so results do not depend on that order).
__global__ void k_dense_count(const int32_t* __restrict__ el, uint32_t E, uint32_t* __restrict__ dcnt) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < E; p += gridDim.x * blockDim.x)
    atomicAdd(&dcnt[el[p]], 1u);
}

__global__ void k_dense_flags(const uint32_t* __restrict__ dcnt, int64_t M, uint32_t* __restrict__ didx) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < M; x += (int64_t)gridDim.x * blockDim.x)
    didx[x] = dcnt[x] ? 1u : 0u;
}

// didx = exclusive scan of the flags: the unique index of each touched element
__global__ void k_dense_unique(const uint32_t* __restrict__ dcnt, const uint32_t* __restrict__ didx, int64_t M,
                               int32_t* __restrict__ uid, uint32_t* __restrict__ cnt) {
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < M; x += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = dcnt[x];
    if (c) {
      uid[didx[x]] = (int32_t)x;
      cnt[didx[x]] = c;
    }
  }
}

// entry -> unique index, and the inverted index (cursor = dcnt, cleared beforehand)
__global__ void k_dense_fill(const int32_t* __restrict__ el, uint32_t E, const uint32_t* __restrict__ wof,
                             const uint32_t* __restrict__ didx, const uint32_t* __restrict__ inv_off,
                             uint32_t* __restrict__ cursor, uint32_t* __restrict__ inv_walk,
                             uint32_t* __restrict__ entry_uidx) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < E; p += gridDim.x * blockDim.x) {
    const uint32_t r = didx[el[p]];
    entry_uidx[p] = r;
    inv_walk[inv_off[r] + atomicAdd(&cursor[r], 1u)] = wof[p];
  }
}

static hsaw_status cover_build_dense(const int32_t* el, uint32_t E, int64_t M, int64_t count, Cover& cv,
                                     cudaStream_t s) {
  HSAW_TRY(cv.keys.ensure((size_t)M, s));   // dense counts, then the fill cursors
  HSAW_TRY(cv.vals.ensure((size_t)M + 1, s));  // flags -> unique indices
  HSAW_TRY(cv.keys2.ensure(E, s));          // walk of each entry
  HSAW_TRY(cv.inv_walk.ensure(E, s));
  HSAW_TRY(cv.entry_uidx.ensure(E, s));
  uint32_t* dcnt = cv.keys.p;
  uint32_t* didx = cv.vals.p;
  uint32_t* wof = cv.keys2.p;
  HSAW_CK(cudaMemsetAsync(dcnt, 0, (size_t)M * 4, s));
  count_launch();
  k_dense_count<<<grid_for(E, 256, 8192), 256, 0, s>>>(el, E, dcnt);
  count_launch();
  k_walk_of_entry<<<grid_for(count, 128, 8192), 128, 0, s>>>(cv.walk_eoff.p, (uint32_t)count, wof);
  count_launch();
  k_dense_flags<<<grid_for(M, 256, 8192), 256, 0, s>>>(dcnt, M, didx);
  HSAW_CK(cudaGetLastError());
  HSAW_TRY(exclusive_scan_u32(didx, (size_t)M, didx + M, s));
  uint32_t U = 0;
  HSAW_CK(cudaMemcpyAsync(&U, didx + M, 4, cudaMemcpyDeviceToHost, s));
  HSAW_CK(cudaStreamSynchronize(s));
  cv.unique = U;
  HSAW_TRY(cv.uid.ensure(U, s));
  HSAW_TRY(cv.cnt.ensure(U, s));
  HSAW_TRY(cv.inv_off.ensure((size_t)U + 1, s));
  count_launch();
  k_dense_unique<<<grid_for(M, 256, 8192), 256, 0, s>>>(dcnt, didx, M, cv.uid.p, cv.cnt.p);
  HSAW_CK(cudaGetLastError());
  HSAW_CK(cudaMemcpyAsync(cv.inv_off.p, cv.cnt.p, (size_t)U * 4, cudaMemcpyDeviceToDevice, s));
  HSAW_TRY(exclusive_scan_u32(cv.inv_off.p, U, cv.inv_off.p + U, s));
  HSAW_CK(cudaMemsetAsync(dcnt, 0, (size_t)U * 4, s));
  count_launch();
  k_dense_fill<<<grid_for(E, 256, 8192), 256, 0, s>>>(el, E, wof, didx, cv.inv_off.p, dcnt, cv.inv_walk.p,
                                                      cv.entry_uidx.p);
  HSAW_CK(cudaGetLastError());
  return HSAW_OK;
}

// ------------------------------------------------------------------ autotuner
// Strategy per (element range M, log2 of the entry count): the first call with both
// strategies eligible times both (CUDA events) and keeps the faster for later calls.
// HSAW_HIST=sort|dense in the environment forces one.
enum HistStrategy { HIST_UNKNOWN = 0, HIST_SORT = 1, HIST_DENSE = 2 };
static std::mutex g_tune_mu;
static std::map<std::pair<int64_t, int>, int> g_tune;

static int forced_strategy() {
  const char* f = getenv("HSAW_HIST");
  if (!f) return HIST_UNKNOWN;
  return f[0] == 'd' ? HIST_DENSE : (f[0] == 's' ? HIST_SORT : HIST_UNKNOWN);
}

static hsaw_status cover_build_sort(const int32_t* el, uint32_t E, int64_t M, int64_t count, Cover& cv,
                                    cudaStream_t s);

hsaw_status cover_build(const Stream& st, hsaw_mode mode, int64_t first, int64_t count, Cover& cv, cudaStream_t s) {
  cv.walks = count;
  cv.entries = 0;
  cv.unique = 0;
  if (count <= 0) return HSAW_OK;
  if (first < 0 || first + count > st.count) return fail(HSAW_E_INVALID, "cover: walk range outside the stream");
  const bool em = (mode == HSAW_EDGE);
  int64_t nb[2];
  HSAW_CK(cudaMemcpyAsync(&nb[0], st.node_off.p + first, 8, cudaMemcpyDeviceToHost, s));
  HSAW_CK(cudaMemcpyAsync(&nb[1], st.node_off.p + first + count, 8, cudaMemcpyDeviceToHost, s));
  HSAW_CK(cudaStreamSynchronize(s));
  const int64_t E64 = em ? (nb[1] - (first + count)) - (nb[0] - first) : nb[1] - nb[0];
  if (E64 >= 0xFFFFFFFFll || count >= 0xFFFFFFFFll) return fail(HSAW_E_INVALID, "cover: too many walk elements");
  const uint32_t E = (uint32_t)E64;
  cv.entries = E;
  HSAW_TRY(cv.walk_eoff.ensure((size_t)count + 1, s));
  count_launch();
  k_walk_eoff<<<grid_for((size_t)count + 1, 256, 8192), 256, 0, s>>>(st.node_off.p, first, count, em ? 1 : 0,
                                                                      cv.walk_eoff.p);
  HSAW_CK(cudaGetLastError());
  if (E == 0) return HSAW_OK;
  const int32_t* el = em ? st.edges.p + (nb[0] - first) : st.nodes.p + nb[0];
  const int64_t M = st.elem_range[em ? 1 : 0];
  const bool dense_ok = M > 0 && M <= (1ll << 28) && M <= 64ll * (int64_t)E + (1 << 20);
  int strat = forced_strategy();
  if (strat == HIST_DENSE && !dense_ok) strat = HIST_SORT;
  if (strat == HIST_UNKNOWN) {
    if (!dense_ok) {
      strat = HIST_SORT;
    } else {
      const std::pair<int64_t, int> key(M, bit_width(E));
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) strat = it->second;
      }
      if (strat == HIST_UNKNOWN) {  // time both once, keep the faster
        cudaEvent_t ev[3];
        for (auto& e : ev) HSAW_CK(cudaEventCreate(&e));
        HSAW_CK(cudaEventRecord(ev[0], s));
        hsaw_status a = cover_build_sort(el, E, M, count, cv, s);
        HSAW_CK(cudaEventRecord(ev[1], s));
        if (a == HSAW_OK) a = cover_build_dense(el, E, M, count, cv, s);
        HSAW_CK(cudaEventRecord(ev[2], s));
        HSAW_CK(cudaEventSynchronize(ev[2]));
        float t_sort = 0.f, t_dense = 0.f;
        cudaEventElapsedTime(&t_sort, ev[0], ev[1]);
        cudaEventElapsedTime(&t_dense, ev[1], ev[2]);
        for (auto& e : ev) cudaEventDestroy(e);
        HSAW_TRY(a);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = t_dense < t_sort ? HIST_DENSE : HIST_SORT;
        return HSAW_OK;
      }
    }
  }
  if (strat == HIST_DENSE) return cover_build_dense(el, E, M, count, cv, s);
  return cover_build_sort(el, E, M, count, cv, s);
}

static hsaw_status cover_build_sort(const int32_t* el, uint32_t E, int64_t M, int64_t count, Cover& cv,
                                    cudaStream_t s) {
  HSAW_TRY(cv.keys.ensure(E, s));
  HSAW_TRY(cv.vals.ensure(E, s));
  HSAW_TRY(cv.keys2.ensure(E, s));
  HSAW_TRY(cv.vals2.ensure(E, s));
  HSAW_TRY(cv.run_flag.ensure((size_t)E + 1, s));
  HSAW_TRY(cv.inv_walk.ensure(E, s));
  HSAW_TRY(cv.entry_uidx.ensure(E, s));
  count_launch();
  k_keys_iota<<<grid_for(E, 256, 8192), 256, 0, s>>>(el, E, cv.keys.p, cv.vals.p);
  HSAW_CK(cudaGetLastError());
  // the largest element id bounds the sort width
  bool alt = false;
  HSAW_TRY(radix_sort_pairs(cv.keys.p, cv.vals.p, cv.keys2.p, cv.vals2.p, E, M > 0 ? bit_width((uint64_t)(M - 1)) : 31,
                            s, &alt));
  uint32_t* sk = alt ? cv.keys2.p : cv.keys.p;
  uint32_t* sv = alt ? cv.vals2.p : cv.vals.p;
  uint32_t* wof = alt ? cv.keys.p : cv.keys2.p;  // the free pair member
  count_launch();
  k_walk_of_entry<<<grid_for(count, 128, 8192), 128, 0, s>>>(cv.walk_eoff.p, (uint32_t)count, wof);
  HSAW_CK(cudaGetLastError());
  count_launch();
  k_run_flags<<<grid_for(E, 256, 8192), 256, 0, s>>>(sk, E, cv.run_flag.p);
  HSAW_CK(cudaGetLastError());
  HSAW_TRY(exclusive_scan_u32(cv.run_flag.p, E, cv.run_flag.p + E, s));
  uint32_t U = 0;
  HSAW_CK(cudaMemcpyAsync(&U, cv.run_flag.p + E, 4, cudaMemcpyDeviceToHost, s));
  HSAW_CK(cudaStreamSynchronize(s));
  cv.unique = U;
  HSAW_TRY(cv.uid.ensure(U, s));
  HSAW_TRY(cv.inv_off.ensure((size_t)U + 1, s));
  HSAW_TRY(cv.cnt.ensure(U, s));
  count_launch();
  k_runs<<<grid_for(E, 256, 8192), 256, 0, s>>>(sk, sv, cv.run_flag.p, wof, E, cv.uid.p, cv.inv_off.p, cv.inv_walk.p,
                                                  cv.entry_uidx.p);
  HSAW_CK(cudaGetLastError());
  HSAW_CK(cudaMemcpyAsync(cv.inv_off.p + U, &E, 4, cudaMemcpyHostToDevice, s));
  count_launch();
  k_counts<<<grid_for(U, 256, 8192), 256, 0, s>>>(cv.inv_off.p, U, cv.cnt.p);
  HSAW_CK(cudaGetLastError());
  HSAW_CK(cudaStreamSynchronize(s));  // E lives on the host stack
  return HSAW_OK;
}

// ------------------------------------------------------------------ greedy
// Running counts carry an exclusion flag in bit 31 (not a candidate, or already picked).
// The argmax key of element u is (count << 32) | (2^32 - 1 - u): the largest count wins and
// ties go to the smallest index, i.e. the smallest id (ids increase with u).  Elements are
// grouped by 256; each group caches its largest key and is refreshed only when one of its
// counts changed (dirty flag), and each CTA owns a fixed range of groups.
constexpr uint32_t GREEDY_GROUP = 256;
constexpr uint32_t EXCLUDED = 0x80000000u;

struct GreedyParams {
  uint32_t U, NG;
  int32_t k;
  uint32_t* cnt;  // running marginal counts | EXCLUDED
  const uint32_t* inv_off;
  const uint32_t* inv_walk;
  const uint32_t* walk_eoff;
  const uint32_t* entry_uidx;
  uint32_t* covered;         // per walk: nonzero once covered
  unsigned long long* gkey;  // NG: cached largest key of each group
  uint8_t* dirty;            // NG
  unsigned long long* partial;  // gridDim.x
  uint32_t* out_u;
  uint32_t* out_gain;
  uint32_t* ctl;  // [0] barrier count, [1] barrier generation, [2] status, [3] rounds done
};

__device__ __forceinline__ void grid_barrier(uint32_t* ctl, unsigned nblocks) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t* vstatus = ctl + 2;
    if (!(*vstatus & GS_BARRIER_TIMEOUT)) {
      volatile uint32_t* vgen = ctl + 1;
      const uint32_t g = *vgen;
      __threadfence();
      const uint32_t arrived = atomicAdd(ctl, 1u);
      if (arrived == nblocks - 1) {
        atomicExch(ctl, 0u);
        __threadfence();
        atomicAdd(ctl + 1, 1u);
      } else {
        uint32_t spins = 0;
        while (*vgen == g) {
          __nanosleep(32);
          if (++spins > (1u << 26)) {  // a few seconds: record and stop waiting
            atomicOr(ctl + 2, GS_BARRIER_TIMEOUT);
            break;
          }
          if (*vstatus & GS_BARRIER_TIMEOUT) break;
        }
      }
      __threadfence();
    }
  }
  __syncthreads();
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    unsigned long long y = __shfl_xor_sync(0xffffffffu, v, o);
    v = y > v ? y : v;
  }
  return v;
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_max_u64(v);
  __syncthreads();
  if (lane == 0) sm[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sm[lane] : 0ull;
    v = warp_max_u64(v);
    if (lane == 0) sm[32] = v;
  }
  __syncthreads();
  return sm[32];
}

__device__ __forceinline__ unsigned long long elem_key(uint32_t c, uint32_t u) {
  return ((c & EXCLUDED) || c == 0) ? 0ull : (((unsigned long long)c << 32) | (0xFFFFFFFFu - u));
}

__global__ void __launch_bounds__(512) k_greedy(GreedyParams P) {
  __shared__ unsigned long long sm[33];
  const unsigned G = gridDim.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t gsz = (size_t)G * blockDim.x;
  const uint32_t g0 = (uint32_t)((uint64_t)P.NG * blockIdx.x / G);
  const uint32_t g1 = (uint32_t)((uint64_t)P.NG * (blockIdx.x + 1) / G);
  int32_t r = 0;
  for (; r < P.k; ++r) {
    // refresh this CTA's dirty groups (one warp per group)
    for (uint32_t g = g0 + w; g < g1; g += nw) {
      if (__ldcg(&P.dirty[g])) {
        unsigned long long best = 0;
        const uint32_t base = g * GREEDY_GROUP;
        for (uint32_t i = lane; i < GREEDY_GROUP; i += 32) {
          const uint32_t u = base + i;
          if (u < P.U) {
            const unsigned long long key = elem_key(__ldcg(&P.cnt[u]), u);
            best = key > best ? key : best;
          }
        }
        best = warp_max_u64(best);
        if (lane == 0) {
          P.gkey[g] = best;
          P.dirty[g] = 0;
        }
      }
    }
    __syncthreads();
    unsigned long long best = 0;
    for (uint32_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
      const unsigned long long x = P.gkey[g];
      best = x > best ? x : best;
    }
    best = block_max_u64(best, sm);
    if (threadIdx.x == 0) P.partial[blockIdx.x] = best;
    grid_barrier(P.ctl, G);
    best = 0;
    for (unsigned b = threadIdx.x; b < G; b += blockDim.x) {
      const unsigned long long x = __ldcg(&P.partial[b]);
      best = x > best ? x : best;
    }
    best = block_max_u64(best, sm);
    const uint32_t gain = (uint32_t)(best >> 32);
    if (gain == 0) break;  // every remaining gain is zero (same decision in every block)
    const uint32_t u = 0xFFFFFFFFu - (uint32_t)best;
    if (gtid == 0) {
      P.out_u[r] = u;
      P.out_gain[r] = gain;
      atomicOr(&P.cnt[u], EXCLUDED);
      P.dirty[u / GREEDY_GROUP] = 1;
    }
    // mark the picked element's uncovered walks and take their elements' counts down
    const uint32_t q0 = P.inv_off[u], q1 = P.inv_off[u + 1];
    for (size_t q = q0 + gtid; q < q1; q += gsz) {
      const uint32_t j = P.inv_walk[q];
      if (!__ldcg(&P.covered[j])) {
        P.covered[j] = 1;
        for (uint32_t p = P.walk_eoff[j]; p < P.walk_eoff[j + 1]; ++p) {
          const uint32_t x = P.entry_uidx[p];
          atomicSub(&P.cnt[x], 1u);
          P.dirty[x / GREEDY_GROUP] = 1;
        }
      }
    }
    grid_barrier(P.ctl, G);
  }
  if (gtid == 0) P.ctl[3] = (uint32_t)r;
}

// ------------------------------------------------------------------ greedy on one cluster
// The same greedy on one thread-block cluster.  CTA r owns the elements
// [r * epc, (r + 1) * epc), in groups of 2^gshift: the largest key of each owned group lives
// in its shared memory, and so do the owned counts and walk-list ranges when they fit there
// (the on-chip version; otherwise the counts stay in global memory).  Counts only fall, so
// a group's largest key changes only when the count of that key's own element changes: a
// decrement of x marks x's group stale only if x is the element of its largest key, and
// the next pick rescans just the stale groups.
//
// A pick costs one cluster barrier: after it every CTA knows the winner and its walk-list
// range (pushed with the winning key), reads all of the winner's walks that no earlier pick
// covered, and takes down the counts of the elements it owns; then it rescans its stale
// groups and pushes its largest key into every CTA's slot for the next pick (two slot
// sets, by the pick's parity, so a CTA that runs ahead never overwrites keys a slower CTA
// still reads).  Walks carry a stamp, 0 or 1 + the pick that covered them, so every CTA
// takes the same walks as new (stamp 0 or this pick's).  A pick whose walks hold many
// entries is instead covered once across the cluster: each walk by one CTA, decrements
// sent to the owner (shared-memory atomics on chip, global atomics otherwise) together with
// a read of the owner's group key, and a second barrier before the rescans.
namespace cg = cooperative_groups;

// Entries of walk elements that the greedy does not track carry this index.
constexpr uint32_t UNTRACKED = 0xFFFFFFFFu;

struct ClusterGreedyParams {
  uint32_t U;
  uint32_t epc;          // elements per CTA (a multiple of the group size)
  uint32_t gshift;       // groups of 2^gshift elements
  uint32_t ng;           // groups per CTA (epc >> gshift)
  uint32_t short_walks;  // 1: walks average few elements, one thread per walk when covering across the cluster
  uint32_t min_gain;     // stop before a pick whose gain is below this (>= 1)
  uint32_t owned_max;    // cover by ownership while (walks of the pick) x avg_entries is at most this
  uint32_t avg_entries;  // walk entries per walk, rounded up
  uint32_t tag0;         // picks of earlier runs over the same stamps
  int32_t k;
  uint32_t* cnt;         // counts | EXCLUDED: the running counts, or the initial ones for the on-chip version
  const uint2* rng;      // per element: its entries [x, y) of inv_ent
  const uint4* inv_ent;  // {walk, first entry, end entry, 0} per inverted-index entry
  const uint32_t* entry_uidx;  // per walk entry: element index, or UNTRACKED
  uint32_t* stamp;       // per walk: 0, or tag0 + 1 + the pick that covered it
  uint32_t* out_u;
  uint32_t* out_gain;
  uint32_t* ctl;  // [3] rounds done, [4] picks covered across the cluster
};

// Exclusive prefix sum of one value per thread of the block; *total gets the block's sum.
// wsum holds 33 words.
__device__ __forceinline__ uint32_t block_exsum(uint32_t v, uint32_t* wsum, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    const uint32_t s = lane < nw ? wsum[lane] : 0u;
    uint32_t si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += y;
    }
    if (lane < nw) wsum[lane] = si - s;
    if (lane == 31) wsum[32] = si;
  }
  __syncthreads();
  *total = wsum[32];
  return wsum[w] + inc - v;
}

template <bool ONCHIP>
struct ClusterGreedyState {
  const ClusterGreedyParams& P;
  cg::cluster_group& cluster;
  unsigned long long* gkey;  // ng: largest key of each owned group
  unsigned long long* wmax;  // (ng + 31) / 32: largest key of each 32 groups
  uint2* rng_s;              // on chip: epc walk-list ranges
  uint32_t* cnt_s;           // on chip: epc counts
  uint32_t* sbits;           // stale bits of the owned groups
  uint32_t lo;               // first owned element

  __device__ __forceinline__ uint32_t count(uint32_t lx) const {
    return ONCHIP ? cnt_s[lx] : __ldcg(&P.cnt[lo + lx]);
  }
  __device__ __forceinline__ void mark(uint32_t* bits, uint32_t gl) const { atomicOr(&bits[gl >> 5], 1u << (gl & 31)); }
  // one decrement of an owned element x (lx = x - lo)
  __device__ __forceinline__ void dec_owned(uint32_t x, uint32_t lx) const {
    if (ONCHIP)
      atomicSub(&cnt_s[lx], 1u);
    else
      atomicSub(&P.cnt[x], 1u);
    const uint32_t gl = lx >> P.gshift;
    const unsigned long long top = gkey[gl];
    if (top != 0 && 0xFFFFFFFFu - (uint32_t)top == x) mark(sbits, gl);
  }
  // one decrement of any element x, at its owner
  __device__ __forceinline__ void dec_remote(uint32_t x) const {
    if (x == UNTRACKED) return;
    const uint32_t owner = x / P.epc, lx = x - owner * P.epc, gl = lx >> P.gshift;
    if (ONCHIP)
      atomicSub(cluster.map_shared_rank(&cnt_s[lx], owner), 1u);
    else
      atomicSub(&P.cnt[x], 1u);
    const unsigned long long top = *cluster.map_shared_rank(&gkey[gl], owner);
    if (top != 0 && 0xFFFFFFFFu - (uint32_t)top == x) mark(cluster.map_shared_rank(sbits, owner), gl);
  }
};

template <bool ONCHIP>
__device__ __forceinline__ void greedy_cluster_body(const ClusterGreedyParams& P) {
  extern __shared__ unsigned long long smem_u64[];
  __shared__ unsigned long long red[32];
  __shared__ ulonglong2 slot[2][16];  // by pick parity, per CTA: {largest key, its walk range q0 << 32 | q1}
  __shared__ uint32_t wy[1024];       // cover by ownership: first entry of each new walk of the pass
  __shared__ uint32_t woff[1025];     // and the new walks' entry offsets (woff[n] = all entries)
  __shared__ uint32_t wsum[33];
  cg::cluster_group cluster = cg::this_cluster();
  const uint32_t rank = cluster.block_rank();
  const uint32_t C = cluster.num_blocks();
  const uint32_t ng = P.ng, words = (ng + 31) / 32, epc = P.epc;
  const uint32_t lo = rank * epc;
  const uint32_t own = P.U > lo ? min(epc, P.U - lo) : 0u;
  ClusterGreedyState<ONCHIP> S{P, cluster, smem_u64, smem_u64 + ng, nullptr, nullptr, nullptr, lo};
  S.rng_s = reinterpret_cast<uint2*>(S.wmax + words);
  S.cnt_s = reinterpret_cast<uint32_t*>(S.rng_s + (ONCHIP ? epc : 0u));
  S.sbits = S.cnt_s + (ONCHIP ? epc : 0u);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (ONCHIP) {
    for (uint32_t i = threadIdx.x; i < epc; i += blockDim.x) S.cnt_s[i] = i < own ? P.cnt[lo + i] : EXCLUDED;
    for (uint32_t i = threadIdx.x; i < own; i += blockDim.x) S.rng_s[i] = P.rng[lo + i];
  }
  for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) S.sbits[i] = 0xFFFFFFFFu;
  for (uint32_t i = threadIdx.x; i < ng; i += blockDim.x) S.gkey[i] = 0ull;
  cluster.sync();
  const uint32_t gsz = 1u << P.gshift;
  // with more than two groups per thread, keep the largest key of every 32 groups too, so
  // the per-pick scan reads those and only rescanned words are refreshed
  const bool word_max = ng > 2 * blockDim.x;
  uint32_t q0 = 0, q1 = 0;  // the previous pick's walk-list range
  bool owned = true;
  uint32_t spread = 0;  // picks covered across the cluster
  int32_t r = 0;
  for (; r < P.k; ++r) {
    // 1. cover the previous pick's walks
    if (r > 0) {
      const uint32_t tag = P.tag0 + (uint32_t)r;
      if (owned) {
        for (uint32_t b0 = q0; b0 < q1; b0 += blockDim.x) {
          const uint32_t n = min((uint32_t)blockDim.x, q1 - b0);
          uint32_t y = 0, len = 0;
          if (threadIdx.x < n) {
            const uint4 ent = __ldg(&P.inv_ent[b0 + threadIdx.x]);
            const uint32_t s = __ldcg(&P.stamp[ent.x]);
            if (s == 0u || s == tag) {
              y = ent.y;
              len = ent.z - ent.y;
              if (s == 0u && rank == 0) P.stamp[ent.x] = tag;
            }
          }
          uint32_t total = 0;
          const uint32_t off = block_exsum(len, wsum, &total);
          if (threadIdx.x < n) {
            wy[threadIdx.x] = y;
            woff[threadIdx.x] = off;
          }
          if (threadIdx.x == 0) woff[n] = total;
          __syncthreads();
          // thread t takes the entry positions [t c, (t + 1) c) of the new walks, in order
          const uint32_t c = (total + blockDim.x - 1) / blockDim.x;
          const uint64_t f64 = (uint64_t)threadIdx.x * c;
          uint32_t f = (uint32_t)(f64 < total ? f64 : (uint64_t)total);
          const uint32_t fend = (uint32_t)(f64 + c < total ? f64 + c : (uint64_t)total);
          if (f < fend) {
            uint32_t a = 0, b = n;  // the walk holding position f: the last i < n with woff[i] <= f
            while (b - a > 1) {
              const uint32_t m = (a + b) >> 1;
              if (woff[m] <= f) a = m; else b = m;
            }
            uint32_t i = a, nxt = woff[a + 1], at = wy[a] - woff[a];  // position f is entry at + f
            while (f < fend) {
              uint32_t xs[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                xs[j] = UNTRACKED;
                if (f < fend) {
                  while (f >= nxt) {
                    ++i;
                    nxt = woff[i + 1];
                    at = wy[i] - woff[i];
                  }
                  xs[j] = __ldg(&P.entry_uidx[at + f]);
                  ++f;
                }
              }
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const uint32_t lx = xs[j] - lo;
                if (xs[j] != UNTRACKED && lx < epc) S.dec_owned(xs[j], lx);
              }
            }
          }
          __syncthreads();  // wy, woff and wsum are reused by the next pass
        }
      } else {
        ++spread;
        if (P.short_walks) {
          for (uint32_t q = q0 + rank * blockDim.x + threadIdx.x; q < q1; q += C * blockDim.x) {
            const uint4 ent = __ldg(&P.inv_ent[q]);
            const uint32_t x0 = ent.y < ent.z ? __ldg(&P.entry_uidx[ent.y]) : 0u;  // in flight with the stamp
            if (__ldcg(&P.stamp[ent.x])) continue;
            P.stamp[ent.x] = tag;
            if (ent.y < ent.z) S.dec_remote(x0);
            for (uint32_t p = ent.y + 1; p < ent.z; ++p) S.dec_remote(__ldg(&P.entry_uidx[p]));
          }
        } else {
          for (uint32_t q = q0 + rank * nw + w; q < q1; q += C * nw) {
            const uint4 ent = __ldg(&P.inv_ent[q]);
            const uint32_t p = ent.y + lane;
            const uint32_t x = p < ent.z ? __ldg(&P.entry_uidx[p]) : 0u;  // in flight with the stamp
            uint32_t fresh = 0;
            if (lane == 0) fresh = __ldcg(&P.stamp[ent.x]) ? 0u : 1u;
            fresh = __shfl_sync(0xffffffffu, fresh, 0);
            if (!fresh) continue;
            if (lane == 0) P.stamp[ent.x] = tag;
            if (p < ent.z) S.dec_remote(x);
            for (uint32_t pp = p + 32; pp < ent.z; pp += 32) S.dec_remote(__ldg(&P.entry_uidx[pp]));
          }
        }
        cluster.sync();  // every decrement and stale mark is in place before the rescans
      }
    }
    __syncthreads();
    // 2. rescan the owned groups marked stale, one warp per group
    for (uint32_t wi = w; wi < words; wi += nw) {
      uint32_t todo = S.sbits[wi];
      __syncwarp();
      if (!todo) continue;
      if (lane == 0) S.sbits[wi] = 0;
      while (todo) {
        const uint32_t gl = wi * 32 + __ffs(todo) - 1;
        todo &= todo - 1;
        if (gl >= ng) continue;
        const uint32_t e0 = gl << P.gshift;
        const uint32_t e1 = min(own, e0 + gsz);
        unsigned long long best = 0;
        for (uint32_t lx = e0 + lane; lx < e1; lx += 32) {
          const unsigned long long key = elem_key(S.count(lx), lo + lx);
          best = key > best ? key : best;
        }
        best = warp_max_u64(best);
        if (lane == 0) S.gkey[gl] = best;
      }
      if (word_max) {
        __syncwarp();
        const uint32_t gl = wi * 32 + lane;
        const unsigned long long m = warp_max_u64(gl < ng ? S.gkey[gl] : 0ull);
        if (lane == 0) S.wmax[wi] = m;
      }
    }
    __syncthreads();
    // 3. this CTA's largest key with its walk-list range, pushed into every CTA's slot
    unsigned long long key = 0;
    if (word_max)
      for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) key = S.wmax[i] > key ? S.wmax[i] : key;
    else
      for (uint32_t gl = threadIdx.x; gl < ng; gl += blockDim.x) key = S.gkey[gl] > key ? S.gkey[gl] : key;
    key = warp_max_u64(key);
    if (lane == 0) red[w] = key;
    __syncthreads();
    const int par = r & 1;
    if (w == 0) {
      key = lane < nw ? red[lane] : 0ull;
      key = warp_max_u64(key);
      unsigned long long qr = 0;
      if (key) {
        const uint32_t u = 0xFFFFFFFFu - (uint32_t)key;
        const uint2 g = ONCHIP ? S.rng_s[u - lo] : __ldg(&P.rng[u]);
        qr = ((unsigned long long)g.x << 32) | g.y;
      }
      if (lane < (int)C) *cluster.map_shared_rank(&slot[par][rank], lane) = make_ulonglong2(key, qr);
    }
    cluster.sync();
    // 4. the cluster's largest key: the pick (the same in every CTA)
    const unsigned long long mine = lane < (int)C ? slot[par][lane].x : 0ull;
    const unsigned long long best = warp_max_u64(mine);
    const uint32_t gain = (uint32_t)(best >> 32);
    if (gain < P.min_gain) break;  // the same decision in every CTA (gain 0: every remaining gain is zero)
    const uint32_t u = 0xFFFFFFFFu - (uint32_t)best;
    const int src = __ffs(__ballot_sync(0xffffffffu, lane < (int)C && mine == best)) - 1;
    const unsigned long long qr = slot[par][src].y;
    q0 = (uint32_t)(qr >> 32);
    q1 = (uint32_t)qr;
    owned = (unsigned long long)(q1 - q0) * P.avg_entries <= P.owned_max;
    if (rank == 0 && threadIdx.x == 0) {
      P.out_u[r] = u;
      P.out_gain[r] = gain;
    }
    if (u - lo < epc && threadIdx.x == 0) {  // the owner takes the pick out of the candidates
      if (ONCHIP)
        atomicOr(&S.cnt_s[u - lo], EXCLUDED);
      else
        atomicOr(&P.cnt[u], EXCLUDED);
      S.mark(S.sbits, (u - lo) >> P.gshift);
    }
  }
  cluster.sync();  // no CTA leaves while a peer may still read its shared memory
  if (rank == 0 && threadIdx.x == 0) {
    P.ctl[3] = (uint32_t)r;
    P.ctl[4] = spread;
  }
}

__global__ void __launch_bounds__(1024, 1) k_greedy_cluster(ClusterGreedyParams P) { greedy_cluster_body<false>(P); }

// The on-chip version: when the counts and walk-list ranges of all elements fit in the
// cluster's shared memory (about 17 K elements per CTA), decrements and rescans stay on chip
// and a CTA's candidate travels with its range, so covering starts without a global lookup.
constexpr uint32_t ONCHIP_GROUP = 32;

__global__ void __launch_bounds__(1024, 1) k_greedy_onchip(ClusterGreedyParams P) { greedy_cluster_body<true>(P); }

// Inverted-index entries with their walk's entry range: {j, walk_eoff[j], walk_eoff[j + 1], 0}.
__global__ void k_inv_ranges(const uint32_t* __restrict__ inv_walk, const uint32_t* __restrict__ walk_eoff, uint32_t E,
                             uint4* __restrict__ inv_ent) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < E; q += gridDim.x * blockDim.x) {
    const uint32_t j = inv_walk[q];
    inv_ent[q] = make_uint4(j, walk_eoff[j], walk_eoff[j + 1], 0u);
  }
}

__global__ void k_greedy_init(const int32_t* __restrict__ uid, const uint32_t* __restrict__ cnt, uint32_t U,
                              const uint8_t* __restrict__ cand, uint32_t* __restrict__ cnt_work) {
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < U; u += gridDim.x * blockDim.x)
    cnt_work[u] = cnt[u] | ((cand && !cand[uid[u]]) ? EXCLUDED : 0u);
}

__global__ void k_pick_ids(const uint32_t* __restrict__ out_u, const int32_t* __restrict__ uid, int32_t r,
                           int64_t* __restrict__ ids) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < r; i += gridDim.x * blockDim.x) ids[i] = uid[out_u[i]];
}

__global__ void k_mark_bits(const int64_t* __restrict__ ids, int32_t r, uint32_t* __restrict__ bits) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < r; i += gridDim.x * blockDim.x)
    atomicOr(&bits[ids[i] >> 5], 1u << (ids[i] & 31));
}

// Zero-gain picks: the smallest ids of C not picked yet, in increasing order (one block).
__global__ void __launch_bounds__(1024) k_zero_fill(int64_t M, const uint8_t* __restrict__ cand,
                                                    const uint32_t* __restrict__ picked_bits, int32_t r0, int32_t k,
                                                    int64_t* __restrict__ ids, uint32_t* __restrict__ gains) {
  __shared__ int32_t warp_cnt[32];
  __shared__ int32_t filled;
  if (threadIdx.x == 0) filled = r0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t base = 0; base < M; base += blockDim.x) {
    if (filled >= k) break;
    const int64_t x = base + threadIdx.x;
    const bool ok = x < M && (!cand || cand[x]) && !((picked_bits[x >> 5] >> (x & 31)) & 1u);
    const unsigned b = __ballot_sync(0xffffffffu, ok);
    if (lane == 0) warp_cnt[w] = __popc(b);
    __syncthreads();
    int32_t before = 0;
    for (int i = 0; i < w; ++i) before += warp_cnt[i];
    const int32_t pos = filled + before + __popc(b & ((1u << lane) - 1u));
    if (ok && pos < k) {
      ids[pos] = x;
      gains[pos] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t tot = 0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += warp_cnt[i];
      filled += tot;
    }
    __syncthreads();
  }
}

static int greedy_grid() {
  static const int cached = [] {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_greedy, 512, 0);
    return std::max(1, std::min(b, 2)) * sm_count();
  }();
  return cached;
}

// The largest cluster (16 CTAs, else 8) that a 1024-thread greedy kernel with the full
// opt-in shared memory can run on, and that memory less room for its static arrays.
struct ClusterCfg {
  int size = 0;
  size_t smem_cap = 0;
};

template <class Kernel>
static ClusterCfg cluster_cfg_for(Kernel kernel) {
  ClusterCfg c;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  c.smem_cap = optin > 16384 ? (size_t)optin - 12288 : 0;  // keep room for the static shared arrays
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem_cap) != cudaSuccess) {
    cudaGetLastError();
    return c;
  }
  const int want[2] = {16, 8};
  for (int i = 0; i < 2 && !c.size; ++i) {
    if (want[i] > 8 && cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = want[i];
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(want[i]);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = c.smem_cap;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg) == cudaSuccess && nclusters > 0)
      c.size = want[i];
    else
      cudaGetLastError();
  }
  return c;
}

// The elements a cluster greedy works on: U of them with running counts (| EXCLUDED), each
// element's entries [x, y) of cv.inv_ent, and per walk entry the element's index (or
// UNTRACKED).  The caller sets up the counts and clears the walk stamps (or, for a second
// run over walks the first one partly covered, gives the first run's picks as tag0).
struct GreedyView {
  uint32_t U = 0;
  uint32_t tag0 = 0;  // picks already made over the same walk stamps
  uint32_t* cnt = nullptr;
  const uint2* rng = nullptr;
  const uint32_t* eidx = nullptr;
};

static void log_greedy(const char* kind, const Cover& cv, const GreedyView& V, uint32_t csize, const char* what,
                       uint32_t size, int32_t k, const uint32_t* h, cudaEvent_t ev0, cudaEvent_t ev1) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  fprintf(stderr, "hsaw: %s walks=%lld entries=%lld unique=%u cluster=%u %s=%u k=%d picks=%u spread=%u ms=%.3f\n",
          kind, (long long)cv.walks, (long long)cv.entries, V.U, csize, what, size, k, h[3], h[4], ms);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
}

// The launch parameters both cluster versions share; the caller sets the ownership (epc,
// gshift, ng).  HSAW_GREEDY_OWNED_MAX overrides the largest pick, in walk entries, that
// every CTA covers by ownership (a measurement aid).
static ClusterGreedyParams greedy_params(const Cover& cv, const GreedyView& V, int32_t k, uint32_t min_gain,
                                         bool short_walks, uint32_t* out_u, uint32_t* out_gain, uint32_t* ctl) {
  const char* e = getenv("HSAW_GREEDY_OWNED_MAX");
  const uint32_t owned_max = e ? (uint32_t)strtoul(e, nullptr, 10) : 16384u;
  ClusterGreedyParams P = {};
  P.U = V.U;
  P.short_walks = short_walks ? 1u : 0u;
  P.min_gain = min_gain;
  P.owned_max = owned_max;
  P.avg_entries = cv.walks > 0 ? (uint32_t)std::max<int64_t>(1, (cv.entries + cv.walks - 1) / cv.walks) : 1u;
  P.tag0 = V.tag0;
  P.k = k;
  P.cnt = V.cnt;
  P.rng = V.rng;
  P.inv_ent = cv.inv_ent.p;
  P.entry_uidx = V.eidx;
  P.stamp = cv.covered.p;
  P.out_u = out_u;
  P.out_gain = out_gain;
  P.ctl = ctl;
  return P;
}

// The greedy with on-chip counts when one cluster's shared memory holds every element's
// count and walk-list range; *done = false leaves the other versions to run.
static hsaw_status onchip_greedy(Cover& cv, const GreedyView& V, int32_t k, uint32_t min_gain, uint32_t* out_u,
                                 uint32_t* out_gain, uint32_t* ctl, uint32_t csize, bool short_walks, int32_t* rounds,
                                 bool* done, cudaStream_t s) {
  static const ClusterCfg cfg1 = cluster_cfg_for(k_greedy_onchip);
  if (!cfg1.size) return HSAW_OK;
  const uint32_t U = V.U;
  auto need = [](uint32_t per) {
    const size_t ng = (per + ONCHIP_GROUP - 1) / ONCHIP_GROUP;
    return ng * 8 + (ng + 31) / 32 * 12 + (size_t)per * 8 + (size_t)per * 4 + 64;
  };
  auto per_for = [U](uint32_t c) { return (uint32_t)(((uint64_t)U + c - 1) / c + 31) / 32 * 32; };
  csize = std::min<uint32_t>(std::max<uint32_t>(csize, 1), (uint32_t)cfg1.size);
  while (need(per_for(csize)) > cfg1.smem_cap && (int)csize < cfg1.size) csize *= 2;
  const uint32_t per = per_for(csize);
  if (need(per) > cfg1.smem_cap) return HSAW_OK;
  ClusterGreedyParams P = greedy_params(cv, V, k, min_gain, short_walks, out_u, out_gain, ctl);
  P.epc = per;
  P.gshift = 5;
  P.ng = per / ONCHIP_GROUP;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(csize);
  cfg.blockDim = dim3(1024);
  cfg.dynamicSmemBytes = need(per);
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const bool log = getenv("HSAW_LOG_LAUNCHES") != nullptr;  // measurement aid
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (log) {
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, s);
  }
  count_launch();
  HSAW_CK(cudaLaunchKernelEx(&cfg, k_greedy_onchip, P));
  uint32_t h[8];
  HSAW_CK(cudaMemcpyAsync(h, ctl, sizeof(h), cudaMemcpyDeviceToHost, s));
  if (log) cudaEventRecord(ev1, s);
  HSAW_CK(cudaStreamSynchronize(s));
  if (log) log_greedy("k_greedy_onchip", cv, V, csize, "per", per, k, h, ev0, ev1);
  *rounds = (int32_t)h[3];
  *done = true;
  return HSAW_OK;
}

// The cluster greedies (on-chip counts when they fit, else counts in global memory with the
// group maxima in shared memory); *done = false when no cluster can run it.  HSAW_GREEDY=grid
// selects the grid-wide version, HSAW_GREEDY=cluster the version with counts in global memory
// (tests).
static hsaw_status cluster_greedy(Cover& cv, const GreedyView& V, int32_t k, uint32_t min_gain, uint32_t* out_u,
                                  uint32_t* out_gain, uint32_t* ctl, int32_t* rounds, bool* done, cudaStream_t s) {
  *done = false;
  const char* force = getenv("HSAW_GREEDY");
  if (force && force[0] == 'g') return HSAW_OK;
  static const ClusterCfg cfg0 = cluster_cfg_for(k_greedy_cluster);
  const int cluster_size = cfg0.size;
  const size_t smem_cap = cfg0.smem_cap;
  if (!cluster_size) return HSAW_OK;
  const uint32_t U = V.U;
  // a cluster whose shared memory holds the keys of 256-element groups; beyond the largest
  // cluster, larger groups
  auto need = [](uint32_t per) { return (size_t)per * 8 + ((size_t)per + 31) / 32 * 12 + 64; };
  uint32_t gshift = 8, csize = 1;
  uint32_t NG = (uint32_t)(((uint64_t)U + 255) >> 8), per = NG;
  // more CTAs (more warps to cover walks and refresh the groups they touch) for larger
  // samples: one CTA per 2^14 walk entries
  const uint64_t walks = (uint64_t)cv.walks;
  const bool short_walks = walks > 0 && (uint64_t)cv.entries < 8ull * walks;
  while ((int)csize < cluster_size && ((uint64_t)csize << 14) < (uint64_t)cv.entries) csize *= 2;
  if (!(force && strcmp(force, "cluster") == 0)) {
    HSAW_TRY(onchip_greedy(cv, V, k, min_gain, out_u, out_gain, ctl, csize, short_walks, rounds, done, s));
    if (*done) return HSAW_OK;
  }
  per = (NG + csize - 1) / csize;
  while (need(per) > smem_cap && (int)csize < cluster_size) {
    csize *= 2;
    per = (NG + csize - 1) / csize;
  }
  while (need(per) > smem_cap) {
    if (++gshift > 20) return HSAW_OK;
    NG = (uint32_t)(((uint64_t)U + (1ull << gshift) - 1) >> gshift);
    per = (NG + csize - 1) / csize;
  }
  // smaller groups make a stale group's rescan cheaper (2^gshift / 32 reads per lane) while
  // the per-pick scan of a CTA's group keys grows: shrink them down to 32 elements while a
  // CTA owns at most 2,048 groups (two keys per thread)
  while (gshift > 5) {
    const uint32_t ng2 = (uint32_t)(((uint64_t)U + (1ull << (gshift - 1)) - 1) >> (gshift - 1));
    const uint32_t per2 = (ng2 + csize - 1) / csize;
    if (per2 > 2048 || need(per2) > smem_cap) break;
    --gshift;
    NG = ng2;
    per = per2;
  }
  ClusterGreedyParams P = greedy_params(cv, V, k, min_gain, short_walks, out_u, out_gain, ctl);
  P.epc = per << gshift;
  P.gshift = gshift;
  P.ng = per;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(csize);
  cfg.blockDim = dim3(1024);
  cfg.dynamicSmemBytes = need(per);
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const bool log = getenv("HSAW_LOG_LAUNCHES") != nullptr;  // measurement aid
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (log) {
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, s);
  }
  count_launch();
  HSAW_CK(cudaLaunchKernelEx(&cfg, k_greedy_cluster, P));
  uint32_t h[8];
  HSAW_CK(cudaMemcpyAsync(h, ctl, sizeof(h), cudaMemcpyDeviceToHost, s));
  if (log) cudaEventRecord(ev1, s);
  HSAW_CK(cudaStreamSynchronize(s));
  if (log) log_greedy("k_greedy_cluster", cv, V, csize, "gshift", gshift, k, h, ev0, ev1);
  *rounds = (int32_t)h[3];
  *done = true;
  return HSAW_OK;
}

// ------------------------------------------------------------------ heavy elements first
// An element that occurs in one walk only can gain at most 1, so while some candidate
// still gains 2 or more the argmax is among the candidates that occurred at least twice
// (on R-MAT walks most touched edges occur once).  The greedy first runs on those alone,
// a smaller set whose counts stay in L2 or shared memory, and stops before a pick of gain
// below 2; the remaining picks then run on every element, with counts recounted over the
// walks not covered yet.  The picks are those of the greedy on every element.
__global__ void k_heavy_flags(const int32_t* __restrict__ uid, const uint32_t* __restrict__ cnt, uint32_t U,
                              const uint8_t* __restrict__ cand, uint32_t* __restrict__ flag) {
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < U; u += gridDim.x * blockDim.x)
    flag[u] = (cnt[u] >= 2u && (!cand || cand[uid[u]])) ? 1u : 0u;
}

// hidx = exclusive scan of the flags: heavy element u gets index hidx[u]
__global__ void k_heavy_view(const uint32_t* __restrict__ cnt, const uint32_t* __restrict__ inv_off,
                             const uint32_t* __restrict__ hidx, uint32_t U, uint32_t* __restrict__ hlist,
                             uint32_t* __restrict__ cnt_h, uint2* __restrict__ rng_h) {
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < U; u += gridDim.x * blockDim.x) {
    const uint32_t h = hidx[u];
    if (hidx[u + 1] != h) {
      hlist[h] = u;
      cnt_h[h] = cnt[u];
      rng_h[h] = make_uint2(inv_off[u], inv_off[u + 1]);
    }
  }
}

__global__ void k_heavy_entries(const uint32_t* __restrict__ entry_uidx, const uint32_t* __restrict__ hidx, uint32_t E,
                                uint32_t* __restrict__ entry_h) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < E; p += gridDim.x * blockDim.x) {
    const uint32_t u = entry_uidx[p];
    entry_h[p] = hidx[u + 1] != hidx[u] ? hidx[u] : UNTRACKED;
  }
}

__global__ void k_ranges(const uint32_t* __restrict__ inv_off, uint32_t U, uint2* __restrict__ rng) {
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < U; u += gridDim.x * blockDim.x)
    rng[u] = make_uint2(inv_off[u], inv_off[u + 1]);
}

// picks of the heavy phase: heavy index -> unique index
__global__ void k_map_picks(uint32_t* __restrict__ out_u, int32_t r, const uint32_t* __restrict__ hlist) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < r; i += gridDim.x * blockDim.x) out_u[i] = hlist[out_u[i]];
}

// counts over the walks not covered yet (| EXCLUDED for non-candidates and picked elements)
__global__ void k_recount(const int32_t* __restrict__ uid, const uint32_t* __restrict__ inv_off,
                          const uint32_t* __restrict__ inv_walk, const uint32_t* __restrict__ covered, uint32_t U,
                          const uint8_t* __restrict__ cand, uint32_t* __restrict__ cnt_work) {
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < U; u += gridDim.x * blockDim.x) {
    uint32_t c = 0;
    for (uint32_t q = inv_off[u]; q < inv_off[u + 1]; ++q) c += covered[inv_walk[q]] ? 0u : 1u;
    cnt_work[u] = c | ((cand && !cand[uid[u]]) ? EXCLUDED : 0u);
  }
}

__global__ void k_exclude_picks(const uint32_t* __restrict__ out_u, int32_t r, uint32_t* __restrict__ cnt_work) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < r; i += gridDim.x * blockDim.x)
    atomicOr(&cnt_work[out_u[i]], EXCLUDED);
}

hsaw_status cover_greedy(Cover& cv, const uint8_t* cand_dev, int64_t M, int32_t k, int64_t* ids_host,
                         uint32_t* gains_host, cudaStream_t s) {
  if (k < 1) return fail(HSAW_E_INVALID, "greedy: k < 1");
  const uint32_t U = (uint32_t)cv.unique;
  DBuf<int64_t> ids;
  DBuf<uint32_t> outs;  // out_u[k], out_gain[k]
  HSAW_TRY(ids.ensure(k, s));
  HSAW_TRY(outs.ensure((size_t)2 * k + 8, s));
  uint32_t* ctl = outs.p + 2 * (size_t)k;
  HSAW_CK(cudaMemsetAsync(ctl, 0, 8 * sizeof(uint32_t), s));
  int32_t rounds = 0;
  hsaw_status st = HSAW_OK;
  bool done = false;
  if (U > 0 && cv.walks > 0) {
    HSAW_TRY(cv.cnt_work.ensure(U, s));
    HSAW_TRY(cv.covered.ensure((size_t)cv.walks, s));
    HSAW_TRY(cv.inv_ent.ensure((size_t)cv.entries, s));
    HSAW_TRY(cv.g_rng.ensure(U, s));
    HSAW_CK(cudaMemsetAsync(cv.covered.p, 0, (size_t)cv.walks * sizeof(uint32_t), s));
    count_launch();
    k_inv_ranges<<<grid_for((size_t)cv.entries, 256, 8192), 256, 0, s>>>(cv.inv_walk.p, cv.walk_eoff.p,
                                                                        (uint32_t)cv.entries, cv.inv_ent.p);
    HSAW_CK(cudaGetLastError());
    // the heavy elements first, when they are clearly fewer than all
    const char* heavy_env = getenv("HSAW_GREEDY_HEAVY");
    const char* force = getenv("HSAW_GREEDY");
    bool heavy_done = false;
    if (!(heavy_env && heavy_env[0] == '0') && !(force && force[0] == 'g') && U >= 4096) {
      HSAW_TRY(cv.g_idx.ensure((size_t)U + 1, s));
      count_launch();
      k_heavy_flags<<<grid_for(U, 256, 8192), 256, 0, s>>>(cv.uid.p, cv.cnt.p, U, cand_dev, cv.g_idx.p);
      HSAW_CK(cudaGetLastError());
      HSAW_TRY(exclusive_scan_u32(cv.g_idx.p, U, cv.g_idx.p + U, s));
      uint32_t H = 0;
      HSAW_CK(cudaMemcpyAsync(&H, cv.g_idx.p + U, 4, cudaMemcpyDeviceToHost, s));
      HSAW_CK(cudaStreamSynchronize(s));
      if (H > 0 && (uint64_t)H * 4 <= (uint64_t)U * 3) {
        HSAW_TRY(cv.g_list.ensure(H, s));
        HSAW_TRY(cv.g_cnt.ensure(H, s));
        HSAW_TRY(cv.g_entry.ensure((size_t)cv.entries, s));
        count_launch();
        k_heavy_view<<<grid_for(U, 256, 8192), 256, 0, s>>>(cv.cnt.p, cv.inv_off.p, cv.g_idx.p, U, cv.g_list.p,
                                                            cv.g_cnt.p, cv.g_rng.p);
        count_launch();
        k_heavy_entries<<<grid_for((size_t)cv.entries, 256, 8192), 256, 0, s>>>(cv.entry_uidx.p, cv.g_idx.p,
                                                                               (uint32_t)cv.entries, cv.g_entry.p);
        HSAW_CK(cudaGetLastError());
        GreedyView Vh;
        Vh.U = H;
        Vh.cnt = cv.g_cnt.p;
        Vh.rng = cv.g_rng.p;
        Vh.eidx = cv.g_entry.p;
        st = cluster_greedy(cv, Vh, k, 2u, outs.p, outs.p + k, ctl, &rounds, &heavy_done, s);
        if (st == HSAW_OK && heavy_done && rounds > 0) {
          count_launch();
          k_map_picks<<<grid_for(rounds, 256, 1024), 256, 0, s>>>(outs.p, rounds, cv.g_list.p);
          if (cudaGetLastError() != cudaSuccess) st = fail(HSAW_E_DEVICE, "greedy: pick map launch failed");
        }
        if (st == HSAW_OK && heavy_done) {
          done = true;
          if (rounds < k) {  // every remaining gain is below 2: all elements, counts over the uncovered walks
            count_launch();
            k_recount<<<grid_for(U, 256, 8192), 256, 0, s>>>(cv.uid.p, cv.inv_off.p, cv.inv_walk.p, cv.covered.p, U,
                                                             cand_dev, cv.cnt_work.p);
            if (rounds > 0) {
              count_launch();
              k_exclude_picks<<<grid_for(rounds, 256, 1024), 256, 0, s>>>(outs.p, rounds, cv.cnt_work.p);
            }
            count_launch();
            k_ranges<<<grid_for(U, 256, 8192), 256, 0, s>>>(cv.inv_off.p, U, cv.g_rng.p);
            HSAW_CK(cudaGetLastError());
            GreedyView V;
            V.U = U;
            V.cnt = cv.cnt_work.p;
            V.rng = cv.g_rng.p;
            V.eidx = cv.entry_uidx.p;
            V.tag0 = (uint32_t)rounds;
            int32_t more = 0;
            bool d2 = false;
            HSAW_CK(cudaMemsetAsync(ctl, 0, 8 * sizeof(uint32_t), s));
            st = cluster_greedy(cv, V, k - rounds, 1u, outs.p + rounds, outs.p + k + rounds, ctl, &more, &d2, s);
            if (st == HSAW_OK && !d2) st = fail(HSAW_E_DEVICE, "greedy: cluster unavailable after the heavy phase");
            rounds += more;
          }
          if (st == HSAW_OK && rounds > 0) {
            count_launch();
            k_pick_ids<<<grid_for(rounds, 256, 1024), 256, 0, s>>>(outs.p, cv.uid.p, rounds, ids.p);
            if (cudaGetLastError() != cudaSuccess) st = fail(HSAW_E_DEVICE, "greedy: id launch failed");
          }
        }
      }
    }
    if (st == HSAW_OK && !done) {
      count_launch();
      k_greedy_init<<<grid_for(U, 256, 8192), 256, 0, s>>>(cv.uid.p, cv.cnt.p, U, cand_dev, cv.cnt_work.p);
      count_launch();
      k_ranges<<<grid_for(U, 256, 8192), 256, 0, s>>>(cv.inv_off.p, U, cv.g_rng.p);
      HSAW_CK(cudaGetLastError());
      GreedyView V;
      V.U = U;
      V.cnt = cv.cnt_work.p;
      V.rng = cv.g_rng.p;
      V.eidx = cv.entry_uidx.p;
      st = cluster_greedy(cv, V, k, 1u, outs.p, outs.p + k, ctl, &rounds, &done, s);
      if (st == HSAW_OK && done && rounds > 0) {
        count_launch();
        k_pick_ids<<<grid_for(rounds, 256, 1024), 256, 0, s>>>(outs.p, cv.uid.p, rounds, ids.p);
        if (cudaGetLastError() != cudaSuccess) st = fail(HSAW_E_DEVICE, "greedy: id launch failed");
      }
    }
  }
  if (st == HSAW_OK && !done && U > 0 && cv.walks > 0) {
    const int G = greedy_grid();
    const uint32_t NG = (U + GREEDY_GROUP - 1) / GREEDY_GROUP;
    HSAW_TRY(cv.cnt_work.ensure(U, s));
    HSAW_TRY(cv.dirty.ensure(NG, s));
    HSAW_TRY(cv.covered.ensure((size_t)cv.walks, s));
    HSAW_TRY(cv.partial.ensure((size_t)G + NG, s));
    HSAW_CK(cudaMemsetAsync(cv.covered.p, 0, (size_t)cv.walks * sizeof(uint32_t), s));
    HSAW_CK(cudaMemsetAsync(cv.dirty.p, 1, NG, s));
    count_launch();
    k_greedy_init<<<grid_for(U, 256, 8192), 256, 0, s>>>(cv.uid.p, cv.cnt.p, U, cand_dev, cv.cnt_work.p);
    HSAW_CK(cudaGetLastError());
    GreedyParams P;
    P.U = U;
    P.NG = NG;
    P.k = k;
    P.cnt = cv.cnt_work.p;
    P.inv_off = cv.inv_off.p;
    P.inv_walk = cv.inv_walk.p;
    P.walk_eoff = cv.walk_eoff.p;
    P.entry_uidx = cv.entry_uidx.p;
    P.covered = cv.covered.p;
    P.dirty = cv.dirty.p;
    P.partial = cv.partial.p;
    P.gkey = cv.partial.p + G;
    P.out_u = outs.p;
    P.out_gain = outs.p + k;
    P.ctl = ctl;
    void* args[] = {&P};
    count_launch();
    HSAW_CK(cudaLaunchCooperativeKernel((const void*)k_greedy, dim3(G), dim3(512), args, 0, s));
    uint32_t h[4];
    HSAW_CK(cudaMemcpyAsync(h, ctl, 16, cudaMemcpyDeviceToHost, s));
    HSAW_CK(cudaStreamSynchronize(s));
    if (h[2] & GS_BARRIER_TIMEOUT) st = fail(HSAW_E_DEVICE, "greedy: grid barrier timed out");
    rounds = (int32_t)h[3];
    if (st == HSAW_OK && rounds > 0) {
      count_launch();
      k_pick_ids<<<grid_for(rounds, 256, 1024), 256, 0, s>>>(outs.p, cv.uid.p, rounds, ids.p);
      if (cudaGetLastError() != cudaSuccess) st = fail(HSAW_E_DEVICE, "greedy: id launch failed");
    }
  }
  if (st == HSAW_OK && rounds < k) {
    uint32_t* bits = nullptr;
    const size_t words = (size_t)(M + 31) / 32;
    st = dmalloc((void**)&bits, words * 4, s);
    if (st == HSAW_OK) {
      cudaMemsetAsync(bits, 0, words * 4, s);
      if (rounds > 0) { count_launch(); k_mark_bits<<<grid_for(rounds, 256, 1024), 256, 0, s>>>(ids.p, rounds, bits); }
      count_launch();
      k_zero_fill<<<1, 1024, 0, s>>>(M, cand_dev, bits, rounds, k, ids.p, outs.p + k);
      if (cudaGetLastError() != cudaSuccess) st = fail(HSAW_E_DEVICE, "greedy: zero-fill launch failed");
      dfree(bits, s);
    }
  }
  if (st == HSAW_OK) {
    if (ids_host) cudaMemcpyAsync(ids_host, ids.p, (size_t)k * 8, cudaMemcpyDeviceToHost, s);
    if (gains_host) cudaMemcpyAsync(gains_host, outs.p + k, (size_t)k * 4, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) st = fail(HSAW_E_DEVICE, "greedy: result copy failed");
  }
  ids.release(s);
  outs.release(s);
  return st;
}

// ------------------------------------------------------------------ coverage on R'_t
__global__ void k_cover_count(const int64_t* __restrict__ node_off, const int32_t* __restrict__ nodes,
                              const int32_t* __restrict__ edges, int edge_mode, int64_t first, int64_t count,
                              const uint32_t* __restrict__ T_sorted, int32_t k, unsigned long long* __restrict__ cov) {
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = first + i;
    const int64_t b = node_off[j] - (edge_mode ? j : 0), e = node_off[j + 1] - (edge_mode ? j + 1 : 0);
    const int32_t* el = edge_mode ? edges : nodes;
    for (int64_t p = b; p < e; ++p) {
      const uint32_t x = (uint32_t)el[p];
      int32_t lo = 0, hi = k;
      while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (T_sorted[mid] < x) lo = mid + 1; else hi = mid;
      }
      if (lo < k && T_sorted[lo] == x) { ++c; break; }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(cov, c);
}

hsaw_status cover_count(const Stream& st, hsaw_mode mode, int64_t first, int64_t count, const int64_t* T, int32_t k,
                        uint64_t* cov, cudaStream_t s) {
  *cov = 0;
  if (count <= 0 || k <= 0) return HSAW_OK;
  if (first < 0 || first + count > st.count) return fail(HSAW_E_INVALID, "coverage: walk range outside the stream");
  // T is a host array of k ids: sort it here (k is at most a few thousand) and search it on the device
  std::vector<uint32_t> sorted(T, T + k);
  std::sort(sorted.begin(), sorted.end());
  uint32_t* buf = nullptr;
  HSAW_TRY(dmalloc((void**)&buf, (size_t)k * 4 + 64, s));
  unsigned long long* dcov = (unsigned long long*)(((uintptr_t)(buf + k) + 15) & ~(uintptr_t)7);
  hsaw_status stt = HSAW_OK;
  unsigned long long h = 0;
  if (cudaMemcpyAsync(buf, sorted.data(), (size_t)k * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(dcov, 0, 8, s) != cudaSuccess) {
    stt = fail(HSAW_E_DEVICE, "coverage: upload failed");
  } else {
    count_launch();
    k_cover_count<<<grid_for(count, 256, 8192), 256, 0, s>>>(st.node_off.p, st.nodes.p, st.edges.p,
                                                             mode == HSAW_EDGE ? 1 : 0, first, count, buf, k, dcov);
    cudaMemcpyAsync(&h, dcov, 8, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      stt = fail(HSAW_E_DEVICE, "coverage kernel failed");
  }
  *cov = h;
  dfree(buf, s);
  return stt;
}

}  // namespace hsaw
