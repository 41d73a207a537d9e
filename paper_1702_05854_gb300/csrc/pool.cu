// Walk pool: query-independent traces of attempts [0, A) for one walk seed, and the scan
// that turns them into a query's ordered hits (see WalkPool in common.cuh).
//
// Build: pass 1 walks every attempt ignoring sources and stores its node count; an
// exclusive scan gives the offsets; pass 2 walks again and writes nodes and edges.  The
// walk stops at no live in-edge or at a detected cycle (register checkpoints), so a trace
// may end with a few repeated nodes; a source can only be met before the first repeat.
// Scan: for each attempt of a launch range, the first node of its trace that is a real
// source for the query (suspect bit, and the node-keyed coin when p < 1) gives a hit of
// that length; hits are recorded per chunk exactly like the sampler's, so the ordered
// compaction is shared, and hit walks are copied out of the pool instead of re-walked.
#include <cuda_runtime.h>

#include <algorithm>

#include "solver.cuh"

namespace hsaw {

template <bool WRITE>
__global__ void k_trace(const uint4* __restrict__ node, const uint2* __restrict__ edge, uint32_t n, uint32_t k0,
                        uint32_t k1, uint64_t a0, uint64_t count, uint32_t step_cap, uint64_t* __restrict__ lens,
                        const uint64_t* __restrict__ off, int32_t* __restrict__ nodes, int32_t* __restrict__ edges,
                        uint32_t* __restrict__ status) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t a = a0 + i;
    uint32_t v = start_node(a, n, k0, k1), len = 1;
    uint64_t nb = 0, eb = 0;
    if (WRITE) {
      nb = off[a];
      eb = nb - a;
      nodes[nb] = (int32_t)v;
    }
    Ckpt ck;
    ck.reset(v);
    for (;;) {
      const uint4 x = node_draw(a, v, k0, k1);
      const uint4 nd = __ldg(&node[v]);
      if (x.x >= nd.w) break;  // no live in-edge
      const uint32_t e = nd.x + pick_in_edge(edge, nd, x.x);
      const uint32_t u = __ldg(&edge[e].x);
      if (WRITE) {
        nodes[nb + len] = (int32_t)u;
        edges[eb + len - 1] = (int32_t)e;
      }
      ++len;
      if (ck.seen(u)) break;  // cycle: u repeats an earlier node
      ck.keep(u, len - 1);
      v = u;
      if (len > step_cap) {
        atomicOr(status, 1u);
        break;
      }
    }
    if (!WRITE) lens[i] = len;
  }
}

// First real source on each trace of attempts [a0, a0 + n_attempts) (launch offsets).
// One warp per 32 consecutive attempts: their traces are contiguous in the pool, so the
// lanes stride over the concatenated nodes with coalesced loads; a source at position q
// belongs to the trace whose offset range holds q (binary search over the trace starts,
// one per lane), and the first such position of each trace is kept in shared memory.
template <bool HAS_P>
__global__ void __launch_bounds__(256) k_pool_scan(const uint64_t* __restrict__ off, const int32_t* __restrict__ nodes,
                                                   const uint32_t* __restrict__ s_bits,
                                                   const uint32_t* __restrict__ p32, uint32_t k0, uint32_t k1,
                                                   uint64_t a0, uint32_t n_attempts, uint32_t chunk, uint32_t cap,
                                                   uint32_t* __restrict__ chunk_hits, uint2* __restrict__ recs,
                                                   uint32_t* __restrict__ status) {
  __shared__ uint32_t first_hit[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t groups = (n_attempts + 31) / 32;
  for (uint32_t gi = blockIdx.x * 8 + w; gi < groups; gi += gridDim.x * 8) {
    const uint32_t i0 = gi * 32;
    const uint32_t cnt = min(32u, n_attempts - i0);
    const uint64_t my_off = off[a0 + i0 + min((uint32_t)lane, cnt)];  // lane t holds the start of trace t
    const uint64_t b = __shfl_sync(0xffffffffu, my_off, 0);
    const uint64_t e = off[a0 + i0 + cnt];  // end of the group's last trace (the 33rd offset)
    first_hit[w][lane] = 0xFFFFFFFFu;
    __syncwarp();
    for (uint64_t q0 = b; q0 < e; q0 += 32) {
      const uint64_t q = q0 + lane;
      bool src = false;
      uint32_t u = 0;
      if (q < e) {
        u = (uint32_t)__ldg(&nodes[q]);
        src = (__ldg(&s_bits[u >> 5]) >> (u & 31)) & 1u;
      }
      const unsigned m = __ballot_sync(0xffffffffu, src);
      if (!m) continue;
      // trace of position q: largest t with off[t] <= q (search over the lanes' offsets)
      uint32_t lo = 0, hi = cnt - 1;
      for (int it = 0; it < 6; ++it) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        const uint64_t om = __shfl_sync(0xffffffffu, my_off, mid);
        if (lo < hi) {
          if (om <= q) lo = mid; else hi = mid - 1;
        }
      }
      const uint64_t trace_start = __shfl_sync(0xffffffffu, my_off, lo);  // every lane takes part
      if (src) {
        const uint32_t t = lo;
        bool real = true;
        if (HAS_P) real = source_coin(node_draw(a0 + i0 + t, u, k0, k1).y, __ldg(&p32[u]));
        if (real) atomicMin(&first_hit[w][t], (uint32_t)(q - trace_start));
      }
    }
    __syncwarp();
    if ((uint32_t)lane < cnt && first_hit[w][lane] != 0xFFFFFFFFu) {
      const uint32_t i = i0 + lane;
      const uint32_t ck = i / chunk;
      const uint32_t slot = atomicAdd(&chunk_hits[ck], 1u);
      if (slot < cap) recs[(size_t)ck * cap + slot] = make_uint2(i, first_hit[w][lane] + 1);
      else atomicOr(status, 1u);
    }
    __syncwarp();
  }
}

// Copy hit walks out of the pool: one warp per hit.
__global__ void k_pool_copy(const uint64_t* __restrict__ off, const int32_t* __restrict__ pnodes,
                            const int32_t* __restrict__ pedges, const uint64_t* __restrict__ aid,
                            const uint32_t* __restrict__ len, const int64_t* __restrict__ node_off, int64_t h0,
                            int64_t h1, int32_t* __restrict__ nodes, int32_t* __restrict__ edges) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t h = h0 + ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); h < h1; h += warps) {
    const uint64_t a = aid[h];
    const uint32_t l = len[h];
    const uint64_t src = off[a];
    const int64_t dst = node_off[h];
    for (uint32_t i = lane; i < l; i += 32) nodes[dst + i] = pnodes[src + i];
    for (uint32_t i = lane; i + 1 < l; i += 32) edges[dst - h + i] = pedges[src - a + i];
  }
}

void pool_release(WalkPool& p) {
  if (p.off) cudaFree(p.off);
  if (p.nodes) cudaFree(p.nodes);
  if (p.edges) cudaFree(p.edges);
  p = WalkPool();
}

hsaw_status pool_build(Graph& g, uint64_t seed, uint64_t attempts, cudaStream_t s) {
  pool_release(g.pool);
  if (attempts == 0) return HSAW_OK;
  if (attempts > (1ull << 32)) return fail(HSAW_E_INVALID, "walk pool: at most 2^32 attempts");
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const uint32_t cap = (uint32_t)std::min<uint64_t>(4ull * (uint64_t)g.n + 64ull, 0xFFFFFFF0ull);
  WalkPool p;
  p.seed = seed;
  p.attempts = attempts;
  HSAW_CK(cudaMalloc((void**)&p.off, (attempts + 1) * sizeof(uint64_t)));
  uint32_t* status = nullptr;
  hsaw_status st = dmalloc((void**)&status, 16, s);
  if (st != HSAW_OK) {
    pool_release(p);
    return st;
  }
  cudaMemsetAsync(status, 0, 16, s);
  const unsigned grid = (unsigned)(sm_count() * 16);
  count_launch();
  k_trace<false><<<grid, 128, 0, s>>>(g.node, g.edge, (uint32_t)g.n, k0, k1, 0, attempts, cap, p.off, nullptr,
                                       nullptr, nullptr, status);
  uint64_t* total = nullptr;
  st = dmalloc((void**)&total, 8, s);
  if (st == HSAW_OK) st = exclusive_scan_u64(p.off, attempts, total, s);
  uint64_t tot = 0;
  uint32_t hs = 0;
  if (st == HSAW_OK) {
    cudaMemcpyAsync(p.off + attempts, total, 8, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(&tot, total, 8, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&hs, status, 4, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) st = fail(HSAW_E_DEVICE, "walk pool: trace lengths failed");
  }
  if (st == HSAW_OK && hs) st = fail(HSAW_E_STEP_CAP, "walk pool: a walk exceeded its step guard");
  if (st == HSAW_OK) {
    if (cudaMalloc((void**)&p.nodes, std::max<uint64_t>(tot, 1) * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc((void**)&p.edges, std::max<uint64_t>(tot, 1) * sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      st = fail(HSAW_E_NOMEM, "walk pool: the traces do not fit in device memory");
    }
  }
  if (st == HSAW_OK) {
    count_launch();
    k_trace<true><<<grid, 128, 0, s>>>(g.node, g.edge, (uint32_t)g.n, k0, k1, 0, attempts, cap, nullptr, p.off,
                                        p.nodes, p.edges, status);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
      st = fail(HSAW_E_DEVICE, "walk pool: trace write failed");
  }
  dfree(status, s);
  dfree(total, s);
  if (st != HSAW_OK) {
    cudaStreamSynchronize(s);
    pool_release(p);
    return st;
  }
  g.pool = p;
  return HSAW_OK;
}

void pool_scan_launch(const Graph& g, const QueryDev& qd, uint64_t a0, uint32_t n_attempts, uint32_t chunk,
                      uint32_t cap, uint32_t* chunk_hits, uint2* recs, uint32_t* status, cudaStream_t s) {
  const uint32_t k0 = (uint32_t)qd.seed, k1 = (uint32_t)(qd.seed >> 32);
  const unsigned grid = grid_for((n_attempts + 31) / 32, 8, (unsigned)sm_count() * 8);
  count_launch();
  if (qd.p32)
    k_pool_scan<true><<<grid, 256, 0, s>>>(g.pool.off, g.pool.nodes, qd.s_bits, qd.p32, k0, k1, a0, n_attempts, chunk,
                                           cap, chunk_hits, recs, status);
  else
    k_pool_scan<false><<<grid, 256, 0, s>>>(g.pool.off, g.pool.nodes, qd.s_bits, nullptr, k0, k1, a0, n_attempts,
                                            chunk, cap, chunk_hits, recs, status);
}

void pool_copy_launch(const Graph& g, const Stream& st, int64_t h0, int64_t h1, cudaStream_t s) {
  count_launch();
  k_pool_copy<<<grid_for((size_t)(h1 - h0) * 32, 256, 1u << 16), 256, 0, s>>>(
      g.pool.off, g.pool.nodes, g.pool.edges, st.aid.p, st.len.p, st.node_off.p, h0, h1, st.nodes.p, st.edges.p);
}

}  // namespace hsaw

using namespace hsaw;

extern "C" {

hsaw_status hsaw_graph_build_walk_pool(hsaw_graph g, uint64_t seed, uint64_t attempts, void* stream) {
  if (!g) return fail(HSAW_E_INVALID, "walk pool: NULL graph");
  return pool_build(g->g, seed, attempts, (cudaStream_t)stream);
}

hsaw_status hsaw_graph_drop_walk_pool(hsaw_graph g) {
  if (!g) return fail(HSAW_E_INVALID, "walk pool: NULL graph");
  cudaDeviceSynchronize();
  pool_release(g->g.pool);
  return HSAW_OK;
}

}  // extern "C"
