// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/hsaw.h"

namespace hsaw {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
hsaw_status fail(hsaw_status st, const std::string& msg);
hsaw_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define HSAW_CK(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) return ::hsaw::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define HSAW_TRY(expr)                 \
  do {                                 \
    hsaw_status s_ = (expr);           \
    if (s_ != HSAW_OK) return s_;      \
  } while (0)

// ------------------------------------------------------------------ device memory
// Stream-ordered allocations from the device's default memory pool; freed blocks stay
// cached in the pool (release threshold raised at first use), so per-call temporaries
// cost no driver round trip after warm-up.
hsaw_status dmalloc(void** p, size_t bytes, cudaStream_t s);
void dfree(void* p, cudaStream_t s);

template <typename T>
struct DBuf {  // grow-only device buffer
  T* p = nullptr;
  size_t cap = 0;  // elements
  hsaw_status ensure(size_t n, cudaStream_t s, bool keep = false) {
    if (n <= cap) return HSAW_OK;
    size_t nc = cap ? cap : 1024;
    while (nc < n) nc *= 2;
    void* np = nullptr;
    HSAW_TRY(dmalloc(&np, nc * sizeof(T), s));
    if (keep && p && cap) HSAW_CK(cudaMemcpyAsync(np, p, cap * sizeof(T), cudaMemcpyDeviceToDevice, s));
    dfree(p, s);
    p = static_cast<T*>(np);
    cap = nc;
    return HSAW_OK;
  }
  void release(cudaStream_t s) {
    dfree(p, s);
    p = nullptr;
    cap = 0;
  }
};

// ------------------------------------------------------------------ graph
// Device in-adjacency (Sec. 2.1).  node[v] = {first in-edge, in-degree, uniform weight
// (0 if the in-weights differ), in-sum}; edge[e] = {tail node u of (u, v), running sum of
// v's in-weights through e}.  In-edge j of v is live for a draw r iff
// thr[j-1] <= r < thr[j]; none is live when r >= in-sum.
// erec[2e], erec[2e+1] = the 32-byte walk record of edge e = (u, v): {u, node[u].x,
// node[u].y, node[u].z}, {node[u].w, thr[e], 0, 0}.  One sector read gives both the tail
// node and everything the next draw at u needs, so a walk makes one dependent DRAM access
// per live-edge draw at equal-weight nodes (the tail's record is replicated per in-edge:
// 32 B per edge of HBM for half the dependent latency and DRAM sectors per draw).
// Guide tables (only when some node has unequal in-weights): for node v and bucket
// b = floor(r * deg / in-sum) in [0, deg), the guide entry is the live in-edge index j0 of
// the smallest draw of the bucket, ceil(b * in-sum / deg); the answer for any r of the
// bucket is at or after it (Chen & Asau's guide table), usually within a step or two.
// grec[2p], grec[2p+1] (p = first(v) + b) hold the walk record of in-edge j0 with j0 in
// the second half's third word, so a draw reads its candidate record directly (one
// dependent access, like equal weights) and steps through erec only past it.
// Walk pool (query-independent traces, kept as an inverted index): for walk seed `seed`,
// trace a (a < attempts) is attempt a's walk ignoring sources - its nodes until no live
// in-edge or a detected cycle.  A query's HSAW of attempt a is the trace's prefix up to its
// first real source (the source test is per node, with the same node-keyed coin), so
// attempt a hits exactly when its trace holds a real source.  Attempts are grouped in
// blocks of 2^shift; for block b and node v, ent[boff[b] + noff[b (n + 1) + v] ..
// boff[b] + noff[b (n + 1) + v + 1]) lists (in no particular order, possibly twice) the
// attempts a - (b << shift) of the block whose trace passes through v.
struct WalkPool {
  uint64_t seed = 0;
  uint64_t attempts = 0;
  uint32_t shift = 0;
  uint32_t blocks = 0;
  uint64_t entries = 0;
  uint64_t* boff = nullptr;  // blocks + 1
  uint32_t* noff = nullptr;  // blocks * (n + 1)
  uint32_t* ent = nullptr;   // entries
};

struct Graph {
  int64_t n = 0, m = 0;
  WalkPool pool;
  uint4* node = nullptr;
  uint2* edge = nullptr;
  uint4* erec = nullptr;
  uint4* grec = nullptr;
  int64_t* input_index = nullptr;  // CSR position -> input edge index (NULL = identity)
  int device = 0;
};

// Sampler occupancy autotuner state of a graph (sample.cu): forget it when the graph goes.
void sample_tune_forget(const Graph& g);

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: 10 rounds of two 32x32->64 multiplies with the
// published multipliers, key bumped by the published Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The same generator with its ten round keys (key + i * the Weyl constants, i = 0..9)
// computed once per launch: a kernel that keeps them in its parameters (constant bank)
// saves the two key additions of every round.
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};
inline PhiloxKeys philox_round_keys(uint32_t k0, uint32_t k1) {
  PhiloxKeys K;
  for (int i = 0; i < 10; ++i) {
    K.k0[i] = k0 + (uint32_t)i * 0x9E3779B9u;
    K.k1[i] = k1 + (uint32_t)i * 0xBB67AE85u;
  }
  return K;
}
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const PhiloxKeys& K) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ K.k0[i], lo1, hi0 ^ c.w ^ K.k1[i], lo0);
  }
  return c;
}

// Draw of node v in attempt a (one live-edge world per attempt).
__device__ __forceinline__ uint4 node_draw(uint64_t a, uint32_t v, uint32_t k0, uint32_t k1) {
  return philox4x32_10(make_uint4((uint32_t)a, (uint32_t)(a >> 32), v, 0u), k0, k1);
}
// Start node of attempt a: floor(x0 * n / 2^32).
__device__ __forceinline__ uint32_t start_node(uint64_t a, uint32_t n, uint32_t k0, uint32_t k1) {
  const uint4 x = philox4x32_10(make_uint4((uint32_t)a, (uint32_t)(a >> 32), 0u, 1u), k0, k1);
  return __umulhi(x.x, n);
}
__device__ __forceinline__ bool source_coin(uint32_t x1, uint32_t p32) {
  return p32 == 0xFFFFFFFFu || x1 < p32;
}
// Live in-edge index j in [0, deg) of a node with record nd for draw r < nd.w (in-sum):
// the first j with r < thr[j] (equal weights: j = r / w; otherwise binary search).
__device__ __forceinline__ uint32_t pick_in_edge(const uint2* __restrict__ edge, uint4 nd, uint32_t r) {
  if (nd.z) return r / nd.z;  // equal weights: thr[j] = (j+1) w
  uint32_t lo = 0, hi = nd.y;  // first j with r < thr[j]
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    const uint32_t t = __ldg(&edge[nd.x + mid].y);
    if (r < t) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// Guide-table bucket of draw r at a node with in-degree deg and in-sum insum (r < insum).
__device__ __forceinline__ uint32_t guide_bucket(uint32_t r, uint32_t deg, uint32_t insum) {
  return (uint32_t)(((uint64_t)r * deg) / insum);
}

// Exact cycle detection in registers: the walk keeps the nodes it saw at positions
// 0, 1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 15, 18, ... (each 1.25x the last) in a ring of 8
// registers.  A tail node equal to a kept node is a revisit, so the world's backward chain
// is a cycle (miss); a cycle entered at position mu is seen within about 0.25 mu + lambda
// draws, against mu + lambda for a whole-walk check and about 2 (mu + lambda) for Brent.
struct Ckpt {
  uint32_t c0, c1, c2, c3, c4, c5, c6, c7;
  uint32_t count, next;
  __device__ __forceinline__ void reset(uint32_t v) {
    c0 = c1 = c2 = c3 = c4 = c5 = c6 = c7 = v;
    count = 1;
    next = 1;
  }
  __device__ __forceinline__ bool seen(uint32_t u) const {
    return (u == c0) | (u == c1) | (u == c2) | (u == c3) | (u == c4) | (u == c5) | (u == c6) | (u == c7);
  }
  // u is the node at walk position pos (>= 1)
  __device__ __forceinline__ void keep(uint32_t u, uint32_t pos) {
    if (pos < next) return;
    const uint32_t slot = count & 7u;
    c0 = slot == 0 ? u : c0; c1 = slot == 1 ? u : c1; c2 = slot == 2 ? u : c2; c3 = slot == 3 ? u : c3;
    c4 = slot == 4 ? u : c4; c5 = slot == 5 ? u : c5; c6 = slot == 6 ? u : c6; c7 = slot == 7 ? u : c7;
    ++count;
    next = next + max(1u, next >> 2);
  }
};

// ------------------------------------------------------------------ primitives (primitives.cu)
// Exclusive prefix sum in place; *total (device, may be NULL) receives the sum.
hsaw_status exclusive_scan_u32(uint32_t* d, size_t n, uint32_t* total, cudaStream_t s);
hsaw_status exclusive_scan_u64(uint64_t* d, size_t n, uint64_t* total, cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the key.  The
// result ends in (keys, vals) or (keys_alt, vals_alt); *in_alt tells which.
hsaw_status radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, size_t n,
                             int bits, cudaStream_t s, bool* in_alt);
int bit_width(uint64_t x);  // bits needed for values in [0, x]

// ------------------------------------------------------------------ launch helpers
inline unsigned grid_for(size_t n, unsigned block, unsigned cap = 1u << 30) {
  size_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}
int sm_count();

// Launch accounting (profiling): every kernel launch of the library calls count_launch();
// sampler launches are bracketed by profile_begin / profile_end.
void count_launch();
void* profile_begin(cudaStream_t s);
void profile_end(void* token, cudaStream_t s, uint64_t attempts);
void profile_add_steps(uint64_t steps);
// Phase timing (profiling only): 0 sampling, 1 counting + index, 2 greedy, 3 coverage.
enum { PH_SAMPLE = 0, PH_COUNT = 1, PH_GREEDY = 2, PH_COVERAGE = 3 };
void* phase_begin(cudaStream_t s);
void phase_end(void* token, cudaStream_t s, int phase);

// ------------------------------------------------------------------ walk-record steps
// The live in-edge e of a node with record rec = {first in-edge, in-degree, equal weight or
// 0, in-sum} for a draw r < rec.w, read through the walk records (the same choice as
// pick_in_edge: j = r / w at equal weights, otherwise the first j with r < thr[j], found
// from the guide bucket's candidate onward).  ra, rb receive e's walk record: the tail is
// ra.x and its node record is {ra.y, ra.z, ra.w, rb.x}.
__device__ __forceinline__ uint32_t record_step(const uint4* __restrict__ erec, const uint4* __restrict__ grec,
                                                uint4 rec, uint32_t r, uint4& ra, uint4& rb) {
  uint32_t e;
  if (rec.z) {
    e = rec.x + r / rec.z;
    ra = __ldg(&erec[2 * (size_t)e]);
    rb = __ldg(&erec[2 * (size_t)e + 1]);
  } else {
    const size_t gp = 2 * ((size_t)rec.x + guide_bucket(r, rec.y, rec.w));
    ra = __ldg(&grec[gp]);
    rb = __ldg(&grec[gp + 1]);
    e = rec.x + rb.z;
    if (r >= rb.y) {
      do {
        ++e;
        rb = __ldg(&erec[2 * (size_t)e + 1]);
      } while (r >= rb.y);
      ra = __ldg(&erec[2 * (size_t)e]);
    }
  }
  return e;
}

}  // namespace hsaw

// Opaque handle types of the ABI.
struct hsaw_graph_s {
  hsaw::Graph g;
};
