// Batched and served solves: host worker threads, one non-blocking CUDA stream each,
// running the ordinary solve (so every result equals the instance solved alone).
// The server admits queries in submission order against a device-memory budget and
// starts each as soon as a worker is free (continuous batching).
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "solver.cuh"

namespace hsaw {

static int default_workers(int32_t w) { return w > 0 ? (int)w : 8; }

// ------------------------------------------------------------------ batch
// Worker threads, each on its own stream, solve the instances whole (one sampler launch
// already fills the GPU, and the workers overlap each instance's short kernels and
// synchronisations with the others').  With HSAW_BATCH=joint the fixed-N instances that no
// walk pool serves are sampled together instead: multi-instance sampler launches
// (batch.cu) extend all their streams at once, then the workers run every instance's
// counting and greedy.  Both give each instance's result alone; the joint form measured
// no faster on any mix tried (the 256-instance batch 0.93x against 1.02x of serial; 256
// graphs of at most 10^4 nodes 2.29x against 2.34-2.49x).
static bool batchable(const hsaw_graph g, const hsaw_query& q) {
  if (!g || q.sampling != HSAW_FIXED_N || q.n_hsaw < 1 || q.n_sources < 1 || !q.sources) return false;
  const Graph& G = g->g;
  if (G.pool.ent && G.pool.seed == q.seed) return false;
  const bool ok = validate_query(G, &q) == HSAW_OK;  // an invalid one fails on its own path
  if (!ok) set_error("");
  return ok;
}

static hsaw_status run_batch(const hsaw_graph* gs, const hsaw_query* qs, hsaw_result* rs, hsaw_status* statuses,
                             int32_t count, int32_t concurrency, cudaStream_t caller) {
  HSAW_CK(cudaStreamSynchronize(caller));
  int dev = 0;
  HSAW_CK(cudaGetDevice(&dev));
  const int nw = std::max(1, std::min<int>(default_workers(concurrency), count));
  std::vector<hsaw_status> st(count, HSAW_OK);
  std::vector<std::string> msg(count);
  // the instances sampled together, with their device suspects and streams
  const char* mode = getenv("HSAW_BATCH");
  const bool together = mode && mode[0] == 'j';
  std::vector<int32_t> joint;
  std::vector<char> is_joint(count, 0);
  std::vector<int64_t> staged;           // per joint entry: sampled hits whose walks are still to draw
  std::vector<int32_t> pos_in_joint(count, -1);
  std::vector<QueryDev> qds;
  std::vector<Stream> sts;
  cudaStream_t s0 = nullptr;
  if (together) {
    for (int32_t i = 0; i < count; ++i)
      if (batchable(gs[i], qs[i])) joint.push_back(i);
    if (!joint.empty()) HSAW_CK(cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking));
    qds.resize(joint.size());
    sts.resize(joint.size());
    staged.assign(joint.size(), 0);
    for (size_t j = 0; j < joint.size(); ++j) pos_in_joint[joint[j]] = (int32_t)j;
    std::vector<const Graph*> gp;
    std::vector<const QueryDev*> qp;
    std::vector<Stream*> sp;
    std::vector<int64_t> want;
    std::vector<int32_t> gi;  // instance of each joint entry
    for (size_t j = 0; j < joint.size(); ++j) {
      const int32_t i = joint[j];
      is_joint[i] = 1;
      hsaw_status r = query_upload(gs[i]->g, &qs[i], qds[j], s0);
      if (r == HSAW_OK) r = stream_init(sts[j], 0, qs[i].max_attempts, s0);
      if (r != HSAW_OK) {
        st[i] = r;
        msg[i] = hsaw_last_error();
        continue;
      }
      gp.push_back(&gs[i]->g);
      qp.push_back(&qds[j]);
      sp.push_back(&sts[j]);
      want.push_back(qs[i].n_hsaw);
      gi.push_back(i);
    }
    std::vector<hsaw_status> js(gp.size(), HSAW_OK);
    std::vector<int64_t> stg(gp.size(), 0);
    const hsaw_status r = gp.empty() ? HSAW_OK
                                     : batch_sample(gp.data(), qp.data(), sp.data(), want.data(), (int32_t)gp.size(),
                                                    js.data(), stg.data(), s0);
    for (size_t t = 0; t < gi.size(); ++t) staged[pos_in_joint[gi[t]]] = stg[t];
    const std::string m = r != HSAW_OK ? std::string(hsaw_last_error()) : std::string();
    for (size_t t = 0; t < gi.size(); ++t) {
      if (r != HSAW_OK) {  // the joint launches failed: every instance in them
        st[gi[t]] = r;
        msg[gi[t]] = m;
      } else if (js[t] != HSAW_OK) {
        st[gi[t]] = js[t];
        msg[gi[t]] = "batch: attempt budget exhausted before enough hits";
      }
    }
    if (s0) cudaStreamSynchronize(s0);
  }
  std::vector<int32_t> pos_of(count, -1);
  for (size_t j = 0; j < joint.size(); ++j) pos_of[joint[j]] = (int32_t)j;
  std::atomic<int32_t> next{0};
  auto work = [&]() {
    cudaSetDevice(dev);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
    for (;;) {
      const int32_t i = next.fetch_add(1);
      if (i >= count) break;
      if (is_joint[i]) {
        const int32_t j = pos_of[i];
        if (st[i] == HSAW_OK) st[i] = stream_take_hits(gs[i]->g, qds[j], sts[j], (uint32_t)staged[j], s);
        if (st[i] == HSAW_OK) st[i] = solve_fixed_from_stream(gs[i]->g, &qs[i], sts[j], &rs[i], s);
      } else if (!gs[i]) {
        st[i] = fail(HSAW_E_INVALID, "batch: NULL graph");
      } else {
        st[i] = solve_one(gs[i]->g, &qs[i], &rs[i], s);
      }
      if (st[i] != HSAW_OK && msg[i].empty()) msg[i] = hsaw_last_error();
    }
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nw; ++t) th.emplace_back(work);
  for (auto& t : th) t.join();
  for (size_t j = 0; j < joint.size(); ++j) {
    query_release(qds[j], s0);
    sts[j].release(s0);
  }
  if (s0) {
    cudaStreamSynchronize(s0);
    cudaStreamDestroy(s0);
  }
  hsaw_status first = HSAW_OK;
  for (int32_t i = 0; i < count; ++i) {
    if (statuses) statuses[i] = st[i];
    if (first == HSAW_OK && st[i] != HSAW_OK) {
      first = st[i];
      set_error("batch: instance " + std::to_string(i) + ": " + msg[i]);
    }
  }
  return first;
}

// ------------------------------------------------------------------ server
struct Ticket {
  uint64_t id = 0;
  int32_t graph = 0;
  hsaw_query q{};
  std::vector<int32_t> sources;
  std::vector<uint32_t> p;
  std::vector<uint8_t> cand;
  size_t estimate = 0;
  volatile int cancel = 0;
  bool admitted = false;  // its estimate is counted in the server's in-flight bytes
  bool done = false;
  hsaw_status status = HSAW_OK;
  std::string error;
  hsaw_result r{};
  std::vector<int64_t> ids;
  std::vector<uint32_t> gains;
  std::chrono::steady_clock::time_point t_submit, t_done;
};

struct Server {
  std::vector<hsaw_graph> graphs;
  std::vector<double> hits_avg, len_avg;  // per graph: running averages for the memory estimate
  size_t budget = 0, in_flight = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Ticket>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Ticket>> tickets;
  uint64_t next_id = 1;
  bool stop = false;
  std::vector<std::thread> workers;
};

// Device bytes a query is expected to hold: its walk stream (aid, len, offsets and
// elements per walk) plus the counting workspace (about 32 B per walk entry) and the
// suspect bitmap / masks.
static size_t estimate_bytes(const Server& S, const Ticket& t) {
  const Graph& g = S.graphs[t.graph]->g;
  const double len = S.len_avg[t.graph] > 0 ? S.len_avg[t.graph] : 16.0;
  double hits;
  if (t.q.sampling == HSAW_FIXED_N) {
    hits = (double)t.q.n_hsaw;
  } else {
    const int64_t M = t.q.mode == HSAW_EDGE ? g.m : g.n;
    double c6[6];
    const double delta = t.q.delta > 0 ? t.q.delta : 1.0 / (double)g.n;
    stop_constants(M, t.q.k, (t.q.eps > 0 && t.q.eps < 1) ? t.q.eps : 0.1, delta, c6);
    hits = std::max(2.0 * std::ceil(c6[4]), S.hits_avg[t.graph]);
  }
  const double per_walk = 24.0 + 8.0 * len + 40.0 * len;
  const double masks = (double)g.n / 8.0 + (t.q.p_fixed ? 4.0 * (double)g.n : 0.0) +
                       (t.q.candidate_mask ? (double)(t.q.mode == HSAW_EDGE ? g.m : g.n) : 0.0);
  return (size_t)(hits * 1.1 * per_walk + masks + (64 << 20));
}

static void server_worker(Server* S) {
  cudaSetDevice(S->device);
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
  for (;;) {
    std::shared_ptr<Ticket> t;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop) break;
        if (!S->queue.empty()) {
          auto& head = S->queue.front();
          if (head->cancel || S->in_flight + head->estimate <= S->budget || S->in_flight == 0) {
            t = head;
            S->queue.pop_front();
            break;
          }
        }
        S->cv_work.wait(lk);
      }
      if (!t) break;
      if (!t->cancel) {
        S->in_flight += t->estimate;
        t->admitted = true;
      }
    }
    if (t->cancel) {
      t->status = HSAW_E_CANCELLED;
      t->error = "server: query cancelled before it started";
    } else {
      set_cancel_flag(&t->cancel);
      t->r.ids = t->ids.data();
      t->r.gains = t->gains.data();
      t->status = solve_one(S->graphs[t->graph]->g, &t->q, &t->r, s);
      if (t->status != HSAW_OK) t->error = hsaw_last_error();
      set_cancel_flag(nullptr);
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (t->admitted) S->in_flight -= std::min(S->in_flight, t->estimate);
      if (t->status == HSAW_OK) {  // running averages behind the next estimates
        const double a = 0.2;
        double& h = S->hits_avg[t->graph];
        h = h > 0 ? (1 - a) * h + a * (double)t->r.hits : (double)t->r.hits;
        if (t->r.attempts) {
          const double len = 2.0 * (double)t->r.steps / (double)t->r.attempts + 2.0;
          double& l = S->len_avg[t->graph];
          l = l > 0 ? (1 - a) * l + a * len : len;
        }
      }
      t->done = true;
      t->t_done = std::chrono::steady_clock::now();
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  if (s) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
}

}  // namespace hsaw

struct hsaw_server_s {
  hsaw::Server S;
};

using namespace hsaw;

extern "C" {

hsaw_status hsaw_solve_batch(const hsaw_graph* gs, const hsaw_query* qs, hsaw_result* rs, hsaw_status* statuses,
                             int32_t count, int32_t concurrency, void* stream) {
  if (count < 0 || (count > 0 && (!gs || !qs || !rs))) return fail(HSAW_E_INVALID, "batch: NULL argument");
  if (count == 0) return HSAW_OK;
  return run_batch(gs, qs, rs, statuses, count, concurrency, (cudaStream_t)stream);
}

hsaw_status hsaw_server_create(const hsaw_graph* gs, int32_t n_graphs, size_t mem_budget, int32_t workers,
                               hsaw_server* out) {
  if (!out || !gs || n_graphs < 1) return fail(HSAW_E_INVALID, "server: need at least one graph");
  *out = nullptr;
  for (int32_t i = 0; i < n_graphs; ++i)
    if (!gs[i]) return fail(HSAW_E_INVALID, "server: NULL graph");
  auto* h = new (std::nothrow) hsaw_server_s();
  if (!h) return fail(HSAW_E_NOMEM, "server: host allocation");
  Server& S = h->S;
  S.graphs.assign(gs, gs + n_graphs);
  S.hits_avg.assign(n_graphs, 0.0);
  S.len_avg.assign(n_graphs, 0.0);
  cudaGetDevice(&S.device);
  if (mem_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete h;
      return fail(HSAW_E_DEVICE, "server: cudaMemGetInfo failed");
    }
    mem_budget = fr / 4 * 3;
  }
  S.budget = mem_budget;
  const int nw = default_workers(workers);
  for (int i = 0; i < nw; ++i) S.workers.emplace_back(server_worker, &S);
  *out = h;
  return HSAW_OK;
}

hsaw_status hsaw_server_submit(hsaw_server h, int32_t graph_idx, const hsaw_query* q, uint64_t* ticket) {
  if (!h || !q || !ticket) return fail(HSAW_E_INVALID, "server: NULL argument");
  Server& S = h->S;
  if (graph_idx < 0 || graph_idx >= (int32_t)S.graphs.size()) return fail(HSAW_E_RANGE, "server: graph index");
  const Graph& g = S.graphs[graph_idx]->g;
  auto t = std::make_shared<Ticket>();
  t->graph = graph_idx;
  t->q = *q;
  if (q->n_sources < 1 || !q->sources) return fail(HSAW_E_INVALID, "server: query needs sources");
  t->sources.assign(q->sources, q->sources + q->n_sources);
  t->q.sources = t->sources.data();
  if (q->p_fixed) {
    t->p.assign(q->p_fixed, q->p_fixed + q->n_sources);
    t->q.p_fixed = t->p.data();
  }
  if (q->candidate_mask) {
    const int64_t M = q->mode == HSAW_EDGE ? g.m : g.n;
    t->cand.assign(q->candidate_mask, q->candidate_mask + M);
    t->q.candidate_mask = t->cand.data();
  }
  if (q->k < 1) return fail(HSAW_E_INVALID, "server: k < 1");
  t->ids.assign(q->k, 0);
  t->gains.assign(q->k, 0);
  t->t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(S.mu);
    t->estimate = estimate_bytes(S, *t);
    if (t->estimate > S.budget) return fail(HSAW_E_REJECTED, "server: query's memory estimate exceeds the budget");
    t->id = S.next_id++;
    S.tickets[t->id] = t;
    S.queue.push_back(t);
  }
  S.cv_work.notify_one();
  *ticket = t->id;
  return HSAW_OK;
}

hsaw_status hsaw_server_poll(hsaw_server h, uint64_t ticket, hsaw_result* r, int32_t timeout_ms, double* latency_ms) {
  if (!h || !r) return fail(HSAW_E_INVALID, "server: NULL argument");
  Server& S = h->S;
  std::unique_lock<std::mutex> lk(S.mu);
  auto it = S.tickets.find(ticket);
  if (it == S.tickets.end()) return fail(HSAW_E_INVALID, "server: unknown ticket");
  std::shared_ptr<Ticket> t = it->second;
  auto ready = [&] { return t->done; };
  if (timeout_ms < 0) {
    S.cv_done.wait(lk, ready);
  } else if (!S.cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return fail(HSAW_E_PENDING, "server: query still running");
  }
  S.tickets.erase(it);
  lk.unlock();
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(t->t_done - t->t_submit).count();
  if (t->status != HSAW_OK) return fail(t->status, t->error);
  int64_t* ids = r->ids;
  uint32_t* gains = r->gains;
  *r = t->r;
  r->ids = ids;
  r->gains = gains;
  if (ids) memcpy(ids, t->ids.data(), t->ids.size() * sizeof(int64_t));
  if (gains) memcpy(gains, t->gains.data(), t->gains.size() * sizeof(uint32_t));
  return HSAW_OK;
}

hsaw_status hsaw_server_cancel(hsaw_server h, uint64_t ticket) {
  if (!h) return fail(HSAW_E_INVALID, "server: NULL handle");
  Server& S = h->S;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.tickets.find(ticket);
    if (it == S.tickets.end()) return fail(HSAW_E_INVALID, "server: unknown ticket");
    it->second->cancel = 1;
  }
  S.cv_work.notify_all();
  return HSAW_OK;
}

hsaw_status hsaw_server_destroy(hsaw_server h) {
  if (!h) return HSAW_OK;
  Server& S = h->S;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    S.stop = true;
    for (auto& kv : S.tickets) kv.second->cancel = 1;
  }
  S.cv_work.notify_all();
  for (auto& t : S.workers) t.join();
  delete h;
  return HSAW_OK;
}

}  // extern "C"
