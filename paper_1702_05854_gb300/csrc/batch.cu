// Multi-instance sampling for batches of fixed-N solves: one persistent sampler launch per
// round serves a window of attempts of every instance that still needs hits (each with its
// own graph, suspects and walk seed), then one scan and one compaction order every
// instance's hits by attempt id and append them to its stream as attempt ids and lengths;
// the caller then draws each instance's walks from their attempt ids (in parallel).  A warp takes chunks of one instance until that instance's window is
// exhausted and its lanes are idle, then moves to the next instance, so the lanes of a warp
// always walk the same graph; all warps take the instances in the same order.  The walks, draws and hit records are those of the one-
// instance sampler (Alg. 1-3 with node-keyed Philox draws), so every stream, and with it
// every result, equals the instance solved alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "solver.cuh"

namespace hsaw {

constexpr uint32_t BCHUNK = 256;                       // attempts per chunk
constexpr uint64_t BATCH_ROUND_ATTEMPTS = 1ull << 32;  // attempts of all instances in one launch

struct BatchInst {
  const uint4* node;
  const uint4* erec;
  const uint4* grec;
  const uint32_t* s_bits;
  const uint32_t* p32;  // NULL: p == 1
  uint64_t a0;          // first attempt of this instance's window
  uint32_t n, k0, k1, step_cap;
  uint32_t n_attempts;  // window size
  uint32_t n_chunks;
  uint32_t chunk0;      // first global chunk of the window
  uint32_t cap;         // hit records per chunk (a few standard deviations above the expected hits)
  uint64_t rec0;        // first record of the window
};

struct BatchParams {
  const BatchInst* inst;
  uint32_t K;
  uint32_t* inst_ctr;      // K chunk counters
  uint32_t* chunk_hits;    // all chunks
  uint2* recs;             // the windows' records
  unsigned long long* steps;  // K
  uint32_t* overflow;      // K: a chunk of the window had more hits than its records
  uint32_t* status;
};

enum : uint32_t { BST_STEP_CAP = 2u };

__global__ void __launch_bounds__(256, 4) k_sample_batch(BatchParams B) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  // every warp takes the instances in the same order, so the GPU works through one
  // instance's window at a time (its graph's hot records stay in L2) and moves on as the
  // window runs out; warps that finish early start the next instance
  for (uint32_t i = 0; i < B.K; ++i) {
    const BatchInst I = B.inst[i];
    uint32_t cur = 0, cur_end = 0;
    bool more = true, active = false;
    uint32_t off = 0, v = 0, len = 0;
    uint4 rec = make_uint4(0, 0, 0, 0);
    Ckpt ck;
    ck.reset(0);
    unsigned long long my_steps = 0;
    for (;;) {
      unsigned need = __ballot_sync(FULL, !active);
      while (need) {
        if (cur >= cur_end) {
          if (!more) break;
          uint32_t c = 0;
          if (lane == 0) c = atomicAdd(&B.inst_ctr[i], 1u);
          c = __shfl_sync(FULL, c, 0);
          if (c >= I.n_chunks) { more = false; break; }
          cur = c * BCHUNK;
          cur_end = min(cur + BCHUNK, I.n_attempts);
        }
        const uint32_t avail = cur_end - cur;
        const uint32_t rank = __popc(need & lt);
        if (!active && rank < avail) {
          off = cur + rank;
          v = start_node(I.a0 + off, I.n, I.k0, I.k1);
          rec = __ldg(&I.node[v]);
          ck.reset(v);
          len = 1;
          active = true;
        }
        cur += min((uint32_t)__popc(need), avail);
        need = __ballot_sync(FULL, !active);
      }
      if (!__any_sync(FULL, active)) break;
      if (active) {
        const uint64_t a = I.a0 + off;
        int outcome = -1;
        const uint32_t sw = __ldg(&I.s_bits[v >> 5]);
        const uint4 x = node_draw(a, v, I.k0, I.k1);
        const bool live = x.x < rec.w;
        uint4 ra = make_uint4(0, 0, 0, 0), rb = make_uint4(0, 0, 0, 0);
        if (live) {
          if (rec.z) {
            const uint32_t e = rec.x + x.x / rec.z;
            ra = __ldg(&I.erec[2 * (size_t)e]);
            rb = __ldg(&I.erec[2 * (size_t)e + 1]);
          } else {
            const size_t gp = 2 * ((size_t)rec.x + guide_bucket(x.x, rec.y, rec.w));
            ra = __ldg(&I.grec[gp]);
            rb = __ldg(&I.grec[gp + 1]);
            uint32_t e = rec.x + rb.z;
            if (x.x >= rb.y) {
              do {
                ++e;
                rb = __ldg(&I.erec[2 * (size_t)e + 1]);
              } while (x.x >= rb.y);
              ra = __ldg(&I.erec[2 * (size_t)e]);
            }
          }
        }
        const bool suspect = (sw >> (v & 31)) & 1u;
        if (suspect && (!I.p32 || source_coin(x.y, __ldg(&I.p32[v])))) {
          outcome = 1;
        } else {
          ++my_steps;
          if (!live) {
            outcome = 0;
          } else {
            const uint32_t u = ra.x;
            if (ck.seen(u)) {
              outcome = 0;
            } else {
              ck.keep(u, len);
              v = u;
              rec = make_uint4(ra.y, ra.z, ra.w, rb.x);
              if (++len > I.step_cap) {
                atomicOr(B.status, BST_STEP_CAP);
                outcome = 0;
              }
            }
          }
        }
        if (outcome >= 0) {
          active = false;
          if (outcome == 1) {
            const uint32_t lc = off / BCHUNK;
            const uint32_t slot = atomicAdd(&B.chunk_hits[I.chunk0 + lc], 1u);
            if (slot < I.cap) B.recs[I.rec0 + (size_t)lc * I.cap + slot] = make_uint2(off, len);
            else B.overflow[i] = 1u;
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) my_steps += __shfl_down_sync(FULL, my_steps, o);
    if (lane == 0 && my_steps) atomicAdd(&B.steps[i], my_steps);
  }
}

// The instance whose window holds chunk gc: the last one with chunk0 <= gc.
__device__ __forceinline__ uint32_t batch_owner(const BatchInst* __restrict__ inst, uint32_t K, uint32_t gc) {
  uint32_t lo = 0, hi = K;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (inst[mid].chunk0 <= gc) lo = mid; else hi = mid;
  }
  return lo;
}

// Records kept per chunk (its hits, at most its instance's cap), to be scanned.
__global__ void k_clamp_batch(const BatchInst* __restrict__ inst, uint32_t K, const uint32_t* __restrict__ chunk_hits,
                              uint32_t n_chunks, uint32_t* __restrict__ kept) {
  for (uint32_t gc = blockIdx.x * blockDim.x + threadIdx.x; gc < n_chunks; gc += gridDim.x * blockDim.x)
    kept[gc] = min(chunk_hits[gc], inst[batch_owner(inst, K, gc)].cap);
}

// Order each chunk's hits by attempt id and write them at the chunk's global offset, as
// attempt ids of its instance's window.
__global__ void k_compact_batch(const BatchInst* __restrict__ inst, uint32_t K, const uint32_t* __restrict__ chunk_hits,
                                const uint32_t* __restrict__ chunk_off, const uint2* __restrict__ recs,
                                uint32_t n_chunks, uint64_t* __restrict__ out_aid, uint32_t* __restrict__ out_len) {
  const int lane = threadIdx.x & 31;
  const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t gc = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; gc < n_chunks; gc += warps) {
    if (chunk_hits[gc] == 0) continue;
    const uint32_t lo = batch_owner(inst, K, gc);
    const BatchInst& I = inst[lo];
    const uint32_t c = min(chunk_hits[gc], I.cap);
    const uint64_t a0 = I.a0;
    const uint2* r = recs + I.rec0 + (size_t)(gc - I.chunk0) * I.cap;
    const uint32_t base = chunk_off[gc];
    for (uint32_t q = lane; q < c; q += 32) {
      const uint2 me = r[q];
      uint32_t rank = 0;
      for (uint32_t j = 0; j < c; ++j) rank += (r[j].x < me.x) ? 1u : 0u;
      out_aid[base + rank] = a0 + me.x;
      out_len[base + rank] = me.y;
    }
  }
}

// Hits of each instance: [bound[i], bound[i + 1]) of the compacted arrays.
__global__ void k_batch_bounds(const BatchInst* __restrict__ inst, uint32_t K, const uint32_t* __restrict__ chunk_off,
                               const uint32_t* __restrict__ total, uint32_t* __restrict__ bound) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= K; i += gridDim.x * blockDim.x)
    bound[i] = i < K ? chunk_off[inst[i].chunk0] : *total;
}

hsaw_status batch_sample(const Graph* const* gs, const QueryDev* const* qds, Stream* const* sts, const int64_t* want,
                         int32_t count, hsaw_status* status, int64_t* staged, cudaStream_t s) {
  std::vector<BatchInst> inst;
  std::vector<int32_t> who;  // instance index of each descriptor
  DBuf<BatchInst> d_inst;
  DBuf<uint32_t> ctr, chunk_hits, chunk_off, bound, ovf;
  std::vector<char> full_cap(count, 0);  // a window overflowed its records: redo it with room for every hit
  DBuf<uint2> recs;
  DBuf<unsigned long long> steps;
  DBuf<uint64_t> out_aid;
  DBuf<uint32_t> out_len;
  auto release = [&]() {
    d_inst.release(s); ctr.release(s); chunk_hits.release(s); chunk_off.release(s); bound.release(s); ovf.release(s);
    recs.release(s); steps.release(s); out_aid.release(s); out_len.release(s);
  };
  hsaw_status rc = HSAW_OK;
  for (int32_t i = 0; i < count; ++i) {
    sts[i]->elem_range[0] = gs[i]->n;
    sts[i]->elem_range[1] = gs[i]->m;
    staged[i] = 0;
  }
  const int grid = sm_count() * 4;
  for (;;) {
    if (cancel_requested()) { rc = fail(HSAW_E_CANCELLED, "batch: cancelled"); break; }
    inst.clear();
    who.clear();
    int32_t active = 0;
    for (int32_t i = 0; i < count; ++i) {
      if (status[i] != HSAW_OK || sts[i]->count + staged[i] >= want[i]) continue;
      if (sts[i]->next_attempt - sts[i]->first_attempt >= sts[i]->max_attempts) {
        status[i] = HSAW_E_TIMEOUT;  // this instance alone: its attempt budget ran out
        continue;
      }
      ++active;
    }
    if (!active) break;
    // windows as the one-instance sampler sizes them, within a per-launch budget
    const double share = std::max(1048576.0, (double)BATCH_ROUND_ATTEMPTS / active);
    uint32_t chunks = 0;
    uint64_t nrecs = 0;
    for (int32_t i = 0; i < count; ++i) {
      Stream& st = *sts[i];
      const int64_t have = st.count + staged[i];
      if (status[i] != HSAW_OK || have >= want[i]) continue;
      const uint64_t used = st.next_attempt - st.first_attempt;
      const double need = (double)(want[i] - have);
      st.hit_rate = used ? (double)have / (double)used : 0.0;
      const double margin = std::min(1.25, 1.0 + 4.0 / std::sqrt(std::max(1.0, (double)have)) + 4.0 / std::sqrt(need));
      double target = st.hit_rate > 0 ? need / st.hit_rate * margin + 4096.0 : std::max(1048576.0, 2.0 * (double)used);
      target = std::min(std::max(target, 1048576.0), std::min(share, 268435456.0));
      uint64_t batch = std::min<uint64_t>((uint64_t)target, st.max_attempts - used);
      batch = (batch + BCHUNK - 1) / BCHUNK * BCHUNK;
      const Graph& g = *gs[i];
      const QueryDev& qd = *qds[i];
      BatchInst b{};
      b.node = g.node;
      b.erec = g.erec;
      b.grec = g.grec;
      b.s_bits = qd.s_bits;
      b.p32 = qd.p32;
      b.a0 = st.next_attempt;
      b.n = (uint32_t)g.n;
      b.k0 = (uint32_t)qd.seed;
      b.k1 = (uint32_t)(qd.seed >> 32);
      b.step_cap = (uint32_t)std::min<uint64_t>(4ull * (uint64_t)g.n + 64ull, 0xFFFFFFF0ull);
      b.n_attempts = (uint32_t)batch;
      b.n_chunks = (uint32_t)(batch / BCHUNK);
      b.chunk0 = chunks;
      const double exp_hits = st.hit_rate * BCHUNK;
      b.cap = (st.hit_rate == 0.0 || full_cap[i])
                  ? BCHUNK
                  : (uint32_t)std::min<double>(BCHUNK, std::ceil(exp_hits + 6.0 * std::sqrt(exp_hits + 1.0) + 8.0));
      b.rec0 = nrecs;
      nrecs += (uint64_t)b.n_chunks * b.cap;
      chunks += b.n_chunks;
      inst.push_back(b);
      who.push_back(i);
    }
    const uint32_t K = (uint32_t)inst.size();
    if ((rc = d_inst.ensure(K, s)) != HSAW_OK || (rc = ctr.ensure((size_t)K + 2, s)) != HSAW_OK ||
        (rc = chunk_hits.ensure(chunks, s)) != HSAW_OK || (rc = chunk_off.ensure((size_t)chunks + 1, s)) != HSAW_OK ||
        (rc = bound.ensure((size_t)K + 1, s)) != HSAW_OK || (rc = recs.ensure((size_t)nrecs, s)) != HSAW_OK ||
        (rc = steps.ensure(K, s)) != HSAW_OK || (rc = ovf.ensure(K, s)) != HSAW_OK)
      break;
    if (cudaMemcpyAsync(d_inst.p, inst.data(), K * sizeof(BatchInst), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(ctr.p, 0, ((size_t)K + 2) * 4, s) != cudaSuccess ||
        cudaMemsetAsync(chunk_hits.p, 0, (size_t)chunks * 4, s) != cudaSuccess ||
        cudaMemsetAsync(steps.p, 0, (size_t)K * 8, s) != cudaSuccess ||
        cudaMemsetAsync(ovf.p, 0, (size_t)K * 4, s) != cudaSuccess) {
      rc = fail(HSAW_E_DEVICE, "batch: set-up copies failed");
      break;
    }
    BatchParams P;
    P.inst = d_inst.p;
    P.K = K;
    P.inst_ctr = ctr.p;
    P.chunk_hits = chunk_hits.p;
    P.recs = recs.p;
    P.steps = steps.p;
    P.overflow = ovf.p;
    P.status = ctr.p + K;
    uint64_t round_attempts = 0;
    for (const BatchInst& b : inst) round_attempts += b.n_attempts;
    void* prof = profile_begin(s);
    count_launch();
    k_sample_batch<<<grid, 256, 0, s>>>(P);
    profile_end(prof, s, round_attempts);
    if (cudaGetLastError() != cudaSuccess) { rc = fail(HSAW_E_DEVICE, "batch: sampler launch failed"); break; }
    count_launch();
    k_clamp_batch<<<grid_for(chunks, 256, 8192), 256, 0, s>>>(d_inst.p, K, chunk_hits.p, chunks, chunk_off.p);
    if (cudaGetLastError() != cudaSuccess) { rc = fail(HSAW_E_DEVICE, "batch: clamp launch failed"); break; }
    if ((rc = exclusive_scan_u32(chunk_off.p, chunks, chunk_off.p + chunks, s)) != HSAW_OK) break;
    count_launch();
    k_batch_bounds<<<grid_for((size_t)K + 1, 256, 64), 256, 0, s>>>(d_inst.p, K, chunk_off.p, chunk_off.p + chunks,
                                                                     bound.p);
    std::vector<uint32_t> hb((size_t)K + 1), hovf(K);
    std::vector<unsigned long long> hsteps(K);
    uint32_t status = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(hb.data(), bound.p, ((size_t)K + 1) * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hovf.data(), ovf.p, (size_t)K * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hsteps.data(), steps.p, (size_t)K * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&status, ctr.p + K, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      rc = fail(HSAW_E_DEVICE, "batch: read-back failed");
      break;
    }
    if (status & BST_STEP_CAP) { rc = fail(HSAW_E_STEP_CAP, "batch: a walk exceeded its step guard"); break; }
    uint64_t draws = 0;
    for (uint32_t j = 0; j < K; ++j) draws += hsteps[j];
    profile_add_steps(draws);
    const uint32_t total = hb[K];
    if (total) {
      if ((rc = out_aid.ensure(total, s)) != HSAW_OK || (rc = out_len.ensure(total, s)) != HSAW_OK) break;
      count_launch();
      k_compact_batch<<<grid_for((size_t)chunks * 32, 256, 8192), 256, 0, s>>>(
          d_inst.p, K, chunk_hits.p, chunk_off.p, recs.p, chunks, out_aid.p, out_len.p);
      if (cudaGetLastError() != cudaSuccess) { rc = fail(HSAW_E_DEVICE, "batch: compaction launch failed"); break; }
    }
    for (uint32_t j = 0; j < K && rc == HSAW_OK; ++j) {
      Stream& st = *sts[who[j]];
      const uint32_t h = hb[j + 1] - hb[j];
      st.steps += hsteps[j];
      if (hovf[j]) {  // rare: this window is drawn again next round with room for every hit
        full_cap[who[j]] = 1;
        continue;
      }
      full_cap[who[j]] = 0;
      if (h) {  // staged after the stream's adopted hits; their walks are drawn by the caller
        const size_t at = (size_t)(st.count + staged[who[j]]);
        if ((rc = st.aid.ensure(at + h, s, true)) != HSAW_OK) break;
        if ((rc = st.len.ensure(at + h, s, true)) != HSAW_OK) break;
        if (cudaMemcpyAsync(st.aid.p + at, out_aid.p + hb[j], (size_t)h * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(st.len.p + at, out_len.p + hb[j], (size_t)h * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
          rc = fail(HSAW_E_DEVICE, "batch: hit copy failed");
          break;
        }
        staged[who[j]] += h;
      }
      st.next_attempt += inst[j].n_attempts;
    }
    if (rc != HSAW_OK) break;
  }
  cudaStreamSynchronize(s);
  release();
  return rc;
}

}  // namespace hsaw
