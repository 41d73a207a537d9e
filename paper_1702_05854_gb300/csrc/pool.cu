// Walk pool: query-independent traces of attempts [0, A) for one walk seed, kept as an
// inverted index from nodes to the attempts whose trace passes through them, and the
// query-side pass that turns the index into a query's ordered hits (see WalkPool in
// common.cuh).
//
// Build: attempts are grouped in blocks of 2^22.  Pass 1 walks every attempt ignoring
// sources and counts, per block and node, the trace's nodes (warp-aggregated atomics); an
// exclusive scan per block turns the counts into node offsets; pass 2 walks again and
// writes each attempt into the lists of its trace's nodes.  A walk stops at no live
// in-edge or at a detected cycle (register checkpoints), so a trace may hold a few nodes
// after its first repeat; those are cycle nodes listed for the attempt already, and a
// trace's first real source always comes before its first repeat.
// Query: over the blocks of a window, the lists of the query's sources set one bit per
// attempt (after the node-keyed coin when p < 1); the set bits, in order, are the hits.
// Each hit's length comes from walking it again up to its first real source, and its
// nodes and edges are re-drawn like the sampler's hits.

#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "solver.cuh"

namespace hsaw {

constexpr uint32_t POOL_SHIFT = 22;

// Calls f(v) for every node of attempt a's trace (the detected repeat that ends it is not
// passed); false when the step guard trips.
template <class F>
__device__ __forceinline__ bool for_trace(const uint4* __restrict__ node, const uint2* __restrict__ edge, uint32_t n,
                                          uint32_t k0, uint32_t k1, uint64_t a, uint32_t step_cap, uint32_t* len,
                                          F&& f) {
  uint32_t v = start_node(a, n, k0, k1), l = 1;
  f(v);
  Ckpt ck;
  ck.reset(v);
  for (;;) {
    const uint4 x = node_draw(a, v, k0, k1);
    const uint4 nd = __ldg(&node[v]);
    if (x.x >= nd.w) break;  // no live in-edge
    const uint32_t u = __ldg(&edge[nd.x + pick_in_edge(edge, nd, x.x)].x);
    if (ck.seen(u)) break;  // cycle: u repeats an earlier node
    ++l;
    f(u);
    ck.keep(u, l - 1);
    v = u;
    if (l > step_cap) {
      *len = l;
      return false;
    }
  }
  *len = l;
  return true;
}

// Pass 1: cnt[b (n + 1) + v] += trace nodes of block b's attempts at v; btot[b] += their sum.
__global__ void k_pool_count(const uint4* __restrict__ node, const uint2* __restrict__ edge, uint32_t n, uint32_t k0,
                             uint32_t k1, uint64_t attempts, uint32_t step_cap, uint32_t* __restrict__ cnt,
                             unsigned long long* __restrict__ btot, uint32_t* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  uint64_t cur = ~0ull;  // block whose trace nodes acc holds (flushed when it changes)
  unsigned long long acc = 0;
  for (uint64_t a = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; a < attempts;
       a += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = a >> POOL_SHIFT;
    if (b != cur) {
      if (acc) atomicAdd(&btot[cur], acc);
      cur = b;
      acc = 0;
    }
    const uint64_t base = b * ((uint64_t)n + 1);
    uint32_t len = 0;
    const bool ok = for_trace(node, edge, n, k0, k1, a, step_cap, &len, [&](uint32_t v) {
      const unsigned long long key = base + v;
      const unsigned grp = __match_any_sync(__activemask(), key);
      if (lane == __ffs(grp) - 1) atomicAdd(&cnt[key], (uint32_t)__popc(grp));
    });
    if (!ok) atomicOr(status, 1u);
    acc += len;
  }
  if (acc) atomicAdd(&btot[cur], acc);
}

// Pass 2: each trace node v of attempt a takes the next slot of its list (cursor starts
// as the node offsets) and receives a's id within its block.
__global__ void k_pool_fill(const uint4* __restrict__ node, const uint2* __restrict__ edge, uint32_t n, uint32_t k0,
                            uint32_t k1, uint64_t attempts, uint32_t step_cap, uint32_t* __restrict__ cursor,
                            const uint64_t* __restrict__ boff, uint32_t* __restrict__ ent) {
  const int lane = threadIdx.x & 31;
  for (uint64_t a = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; a < attempts;
       a += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = a >> POOL_SHIFT;
    const uint64_t base = b * ((uint64_t)n + 1);
    uint32_t* out = ent + boff[b];
    const uint32_t local = (uint32_t)(a - (b << POOL_SHIFT));
    uint32_t len = 0;
    for_trace(node, edge, n, k0, k1, a, step_cap, &len, [&](uint32_t v) {
      const unsigned long long key = base + v;
      const unsigned grp = __match_any_sync(__activemask(), key);
      const int leader = __ffs(grp) - 1;
      uint32_t first = 0;
      if (lane == leader) first = atomicAdd(&cursor[key], (uint32_t)__popc(grp));
      first = __shfl_sync(grp, first, leader);
      out[first + __popc(grp & ((1u << lane) - 1u))] = local;
    });
  }
}

// Query side.  Pair p = i * nb + j stands for source s_list[i] in block b0 + j.
__global__ void k_pool_pairs(const uint32_t* __restrict__ noff, uint32_t n, const int32_t* __restrict__ s_list,
                             uint32_t n_src, uint64_t b0, uint32_t nb, uint64_t* __restrict__ cnt) {
  const uint64_t P = (uint64_t)n_src * nb;
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < P; p += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t idx = (b0 + p % nb) * ((uint64_t)n + 1) + (uint32_t)s_list[p / nb];
    cnt[p] = noff[idx + 1] - noff[idx];
  }
}

// Every listed entry of the pairs (pre = exclusive prefix of the pair sizes, pre[P] = all)
// whose attempt lies in [a0, a1) and whose source passes its coin sets the attempt's bit.
// Each warp takes 32 x 8 consecutive entries, lanes interleaved (coalesced list reads).
template <bool HAS_P>
__global__ void __launch_bounds__(256) k_pool_mark(const uint64_t* __restrict__ boff, const uint32_t* __restrict__ noff,
                                                   const uint32_t* __restrict__ ent, uint32_t n,
                                                   const int32_t* __restrict__ s_list, const uint32_t* __restrict__ p32,
                                                   uint32_t k0, uint32_t k1, uint64_t b0, uint32_t nb,
                                                   const uint64_t* __restrict__ pre, uint64_t P, uint64_t a0,
                                                   uint64_t a1, uint32_t* __restrict__ bits) {
  const uint64_t E = pre[P];
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t w0 = warp * 256; w0 < E; w0 += warps * 256) {
    uint64_t i = w0 + lane;
    if (i >= E) continue;
    uint64_t lo = 0, hi = P - 1;  // last pair with pre[p] <= i
    while (lo < hi) {
      const uint64_t mid = (lo + hi + 1) >> 1;
      if (pre[mid] <= i) lo = mid; else hi = mid - 1;
    }
    uint64_t p = lo;
    for (int t = 0; t < 8 && i < E; ++t, i += 32) {
      while (pre[p + 1] <= i) ++p;
      const uint64_t b = b0 + p % nb;
      const uint32_t v = (uint32_t)s_list[p / nb];
      const uint32_t e = ent[boff[b] + noff[b * ((uint64_t)n + 1) + v] + (i - pre[p])];
      const uint64_t a = (b << POOL_SHIFT) + e;
      if (a < a0 || a >= a1) continue;
      if (HAS_P && !source_coin(node_draw(a, v, k0, k1).y, __ldg(&p32[v]))) continue;
      const uint64_t r = a - a0;
      atomicOr(&bits[r >> 5], 1u << (r & 31));
    }
  }
}

__global__ void k_bits_popc(const uint32_t* __restrict__ bits, uint32_t words, uint32_t* __restrict__ cnt) {
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < words; w += gridDim.x * blockDim.x)
    cnt[w] = __popc(bits[w]);
}

// The set bits in order: the hits of word w start at off[w]; bit t is attempt a0 + 32 w + t.
__global__ void k_bits_emit(const uint32_t* __restrict__ bits, const uint32_t* __restrict__ off, uint32_t words,
                            uint64_t a0, uint64_t* __restrict__ aid) {
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < words; w += gridDim.x * blockDim.x) {
    uint32_t b = bits[w], o = off[w];
    while (b) {
      const uint32_t t = __ffs(b) - 1;
      b &= b - 1;
      aid[o++] = a0 + 32ull * w + t;
    }
  }
}

// Length of each pooled hit: nodes walked up to and including its first real source.  A
// walk that meets no source first (impossible for an attempt the index lists) sets bit 2.
template <bool HAS_P>
__global__ void k_hit_len(const uint4* __restrict__ node, const uint4* __restrict__ erec, const uint4* __restrict__ grec,
                          uint32_t n, uint32_t k0, uint32_t k1, const uint32_t* __restrict__ s_bits,
                          const uint32_t* __restrict__ p32, const uint64_t* __restrict__ aid, uint32_t count,
                          uint32_t step_cap, uint32_t* __restrict__ len, uint32_t* __restrict__ status) {
  for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < count; h += gridDim.x * blockDim.x) {
    const uint64_t a = aid[h];
    uint32_t v = start_node(a, n, k0, k1), l = 1;
    uint4 rec = __ldg(&node[v]);
    for (;;) {
      const uint4 x = node_draw(a, v, k0, k1);
      if (((__ldg(&s_bits[v >> 5]) >> (v & 31)) & 1u) && (!HAS_P || source_coin(x.y, __ldg(&p32[v])))) break;
      if (x.x >= rec.w || l >= step_cap) {
        atomicOr(status, 2u);
        break;
      }
      uint4 ra, rb;
      record_step(erec, grec, rec, x.x, ra, rb);
      v = ra.x;
      rec = make_uint4(ra.y, ra.z, ra.w, rb.x);
      ++l;
    }
    len[h] = l;
  }
}

void pool_release(WalkPool& p) {
  if (p.boff) cudaFree(p.boff);
  if (p.noff) cudaFree(p.noff);
  if (p.ent) cudaFree(p.ent);
  p = WalkPool();
}

static uint32_t pool_step_cap(const Graph& g) {
  return (uint32_t)std::min<uint64_t>(4ull * (uint64_t)g.n + 64ull, 0xFFFFFFF0ull);
}

hsaw_status pool_build(Graph& g, uint64_t seed, uint64_t attempts, cudaStream_t s) {
  pool_release(g.pool);
  if (attempts == 0) return HSAW_OK;
  if (attempts > (1ull << 32)) return fail(HSAW_E_INVALID, "walk pool: at most 2^32 attempts");
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const uint32_t cap = pool_step_cap(g);
  const uint32_t blocks = (uint32_t)((attempts + (1ull << POOL_SHIFT) - 1) >> POOL_SHIFT);
  const size_t noff_n = (size_t)blocks * ((size_t)g.n + 1);
  WalkPool p;
  p.seed = seed;
  p.attempts = attempts;
  p.shift = POOL_SHIFT;
  p.blocks = blocks;
  uint32_t* status = nullptr;
  unsigned long long* btot = nullptr;
  uint32_t* cursor = nullptr;
  auto finish = [&](hsaw_status st) {
    cudaStreamSynchronize(s);
    dfree(status, s);
    dfree(btot, s);
    dfree(cursor, s);
    if (st != HSAW_OK) pool_release(p);
    return st;
  };
  if (cudaMalloc((void**)&p.noff, noff_n * 4) != cudaSuccess ||
      cudaMalloc((void**)&p.boff, ((size_t)blocks + 1) * 8) != cudaSuccess) {
    cudaGetLastError();
    return finish(fail(HSAW_E_NOMEM, "walk pool: node offsets do not fit in device memory"));
  }
  hsaw_status st = dmalloc((void**)&status, 16, s);
  if (st == HSAW_OK) st = dmalloc((void**)&btot, (size_t)blocks * 8, s);
  if (st != HSAW_OK) return finish(st);
  if (cudaMemsetAsync(status, 0, 16, s) != cudaSuccess || cudaMemsetAsync(btot, 0, (size_t)blocks * 8, s) != cudaSuccess ||
      cudaMemsetAsync(p.noff, 0, noff_n * 4, s) != cudaSuccess)
    return finish(fail(HSAW_E_DEVICE, "walk pool: clearing the counts failed"));
  const unsigned grid = (unsigned)(sm_count() * 16);
  count_launch();
  k_pool_count<<<grid, 128, 0, s>>>(g.node, g.edge, (uint32_t)g.n, k0, k1, attempts, cap, p.noff, btot, status);
  std::vector<unsigned long long> tot(blocks);
  uint32_t hs = 0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(tot.data(), btot, (size_t)blocks * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&hs, status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return finish(fail(HSAW_E_DEVICE, "walk pool: trace counts failed"));
  if (hs) return finish(fail(HSAW_E_STEP_CAP, "walk pool: a walk exceeded its step guard"));
  std::vector<uint64_t> boff((size_t)blocks + 1, 0);
  for (uint32_t b = 0; b < blocks; ++b) {
    if (tot[b] > 0xFFFFFFFFull) return finish(fail(HSAW_E_INVALID, "walk pool: a block's traces exceed 2^32 nodes"));
    boff[b + 1] = boff[b] + tot[b];
  }
  p.entries = boff[blocks];
  // node offsets within each block (the count slot at v = n is 0, so it receives the total)
  for (uint32_t b = 0; b < blocks && st == HSAW_OK; ++b)
    st = exclusive_scan_u32(p.noff + (size_t)b * ((size_t)g.n + 1), (size_t)g.n + 1, status + 1, s);
  if (st != HSAW_OK) return finish(st);
  if (cudaMemcpyAsync(p.boff, boff.data(), ((size_t)blocks + 1) * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return finish(fail(HSAW_E_DEVICE, "walk pool: block offsets upload failed"));
  if (cudaMalloc((void**)&p.ent, std::max<uint64_t>(p.entries, 1) * 4) != cudaSuccess) {
    cudaGetLastError();
    return finish(fail(HSAW_E_NOMEM, "walk pool: the index does not fit in device memory"));
  }
  st = dmalloc((void**)&cursor, noff_n * 4, s);
  if (st != HSAW_OK) return finish(st);
  if (cudaMemcpyAsync(cursor, p.noff, noff_n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return finish(fail(HSAW_E_DEVICE, "walk pool: cursor copy failed"));
  count_launch();
  k_pool_fill<<<grid, 128, 0, s>>>(g.node, g.edge, (uint32_t)g.n, k0, k1, attempts, cap, cursor, p.boff, p.ent);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
    return finish(fail(HSAW_E_DEVICE, "walk pool: index fill failed"));
  st = finish(HSAW_OK);
  g.pool = p;
  return st;
}

hsaw_status pool_hits(const Graph& g, const QueryDev& qd, Stream& st, uint64_t a0, uint64_t a1, uint32_t* new_hits,
                      cudaStream_t s) {
  const WalkPool& pl = g.pool;
  *new_hits = 0;
  if (a1 <= a0) return HSAW_OK;
  const uint32_t k0 = (uint32_t)qd.seed, k1 = (uint32_t)(qd.seed >> 32);
  const uint64_t b0 = a0 >> pl.shift, b1 = (a1 - 1) >> pl.shift;
  const uint32_t nb = (uint32_t)(b1 - b0 + 1);
  const uint64_t P = (uint64_t)qd.n_src * nb;
  const uint32_t words = (uint32_t)((a1 - a0 + 31) / 32);
  HSAW_TRY(st.pcnt.ensure(P + 1, s));
  HSAW_TRY(st.pbits.ensure(words, s));
  HSAW_TRY(st.chunk_off.ensure(words, s));
  HSAW_CK(cudaMemsetAsync(st.pbits.p, 0, (size_t)words * 4, s));
  HSAW_CK(cudaMemsetAsync(st.ctrs.p, 0, 8 * 4, s));
  count_launch();
  k_pool_pairs<<<grid_for(P, 256, 4096), 256, 0, s>>>(pl.noff, (uint32_t)g.n, qd.s_list, (uint32_t)qd.n_src, b0, nb,
                                                     st.pcnt.p);
  HSAW_CK(cudaGetLastError());
  HSAW_TRY(exclusive_scan_u64(st.pcnt.p, P, st.pcnt.p + P, s));
  const unsigned mgrid = (unsigned)sm_count() * 8;
  count_launch();
  if (qd.p32)
    k_pool_mark<true><<<mgrid, 256, 0, s>>>(pl.boff, pl.noff, pl.ent, (uint32_t)g.n, qd.s_list, qd.p32, k0, k1, b0, nb,
                                            st.pcnt.p, P, a0, a1, st.pbits.p);
  else
    k_pool_mark<false><<<mgrid, 256, 0, s>>>(pl.boff, pl.noff, pl.ent, (uint32_t)g.n, qd.s_list, nullptr, k0, k1, b0,
                                             nb, st.pcnt.p, P, a0, a1, st.pbits.p);
  HSAW_CK(cudaGetLastError());
  count_launch();
  k_bits_popc<<<grid_for(words, 256, 8192), 256, 0, s>>>(st.pbits.p, words, st.chunk_off.p);
  HSAW_CK(cudaGetLastError());
  HSAW_TRY(exclusive_scan_u32(st.chunk_off.p, words, st.ctrs.p + 2, s));
  uint32_t h = 0;
  HSAW_CK(cudaMemcpyAsync(&h, st.ctrs.p + 2, 4, cudaMemcpyDeviceToHost, s));
  HSAW_CK(cudaStreamSynchronize(s));
  if (!h) return HSAW_OK;
  HSAW_TRY(st.aid.ensure((size_t)st.count + h, s, true));
  HSAW_TRY(st.len.ensure((size_t)st.count + h, s, true));
  count_launch();
  k_bits_emit<<<grid_for(words, 256, 8192), 256, 0, s>>>(st.pbits.p, st.chunk_off.p, words, a0, st.aid.p + st.count);
  HSAW_CK(cudaGetLastError());
  const unsigned hgrid = grid_for(h, 128, 1u << 16);
  count_launch();
  if (qd.p32)
    k_hit_len<true><<<hgrid, 128, 0, s>>>(g.node, g.erec, g.grec, (uint32_t)g.n, k0, k1, qd.s_bits, qd.p32,
                                          st.aid.p + st.count, h, pool_step_cap(g), st.len.p + st.count,
                                          st.ctrs.p + 3);
  else
    k_hit_len<false><<<hgrid, 128, 0, s>>>(g.node, g.erec, g.grec, (uint32_t)g.n, k0, k1, qd.s_bits, nullptr,
                                           st.aid.p + st.count, h, pool_step_cap(g), st.len.p + st.count,
                                           st.ctrs.p + 3);
  HSAW_CK(cudaGetLastError());
  uint32_t bad = 0;
  HSAW_CK(cudaMemcpyAsync(&bad, st.ctrs.p + 3, 4, cudaMemcpyDeviceToHost, s));
  HSAW_CK(cudaStreamSynchronize(s));
  if (bad) return fail(HSAW_E_DEVICE, "walk pool: a listed attempt did not reach a source");
  *new_hits = h;
  return HSAW_OK;
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
