// C-ABI entry points: solve (Alg. 6 / 9 or fixed N), the HSAW stream (Alg. 3),
// counting / greedy / coverage on a stream, and the stopping-rule constants (Sec. 5.1).
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <vector>

#include "solver.cuh"

namespace hsaw {

// ------------------------------------------------------------------ stopping rule (Sec. 5.1)
// N_max (Eq. "guard" with M = m, Eq. "nguard" with M = n); the printed t_max has
// ln(delta/3) < 0, so t_max follows Lemma "tmax": ceil(log2(2 N_max / Upsilon)) with
// Upsilon = (2 + 2eps/3) ln(3/delta) / eps^2; Lambda (Eq. "lambda"), Lambda_1 (Eq. "lambda_1").
void stop_constants(int64_t M, int32_t k, double eps, double delta, double out6[6]) {
  const double lnC = std::lgamma((double)M + 1.0) - std::lgamma((double)k + 1.0) - std::lgamma((double)(M - k) + 1.0);
  const double a = 2.0 + 2.0 * eps / 3.0;
  const double b = 2.0 - 1.0 / M_E;
  const double n_max = b * b * a * (double)M * (std::log(6.0 / delta) + lnC) / ((double)k * eps * eps);
  const double ups = a * std::log(3.0 / delta) / (eps * eps);
  double t_max = std::ceil(std::log2(2.0 * n_max / ups));
  if (t_max < 1.0) t_max = 1.0;
  const double lam = a * std::log(3.0 * t_max / delta) / (eps * eps);
  out6[0] = lnC;
  out6[1] = n_max;
  out6[2] = ups;
  out6[3] = t_max;
  out6[4] = lam;
  out6[5] = 1.0 + (1.0 + eps) * lam;
}

// Check (Alg. 5 / Alg. 8).
int check_bound(double c, double cp, double size_rp, int32_t t, double eps, double lambda1, double* eps_t) {
  *eps_t = NAN;
  if (!(cp >= lambda1)) return 0;
  const double scale = std::ldexp(1.0, t - 1);
  const double gap = 1.0 - 1.0 / M_E - eps;
  const double e1 = c / cp - 1.0;
  const double e2 = eps * std::sqrt(size_rp * (1.0 + eps) / (scale * cp));
  const double e3 = eps * std::sqrt(size_rp * (1.0 + eps) * gap / ((1.0 + eps / 3.0) * scale * cp));
  const double et = (e1 + e2 + e1 * e2) * gap + (1.0 - 1.0 / M_E) * e3;
  *eps_t = et;
  return et <= eps ? 1 : 0;
}

// ------------------------------------------------------------------ helpers
static hsaw_status upload_mask(const uint8_t* mask, size_t len, bool on_device, cudaStream_t s, uint8_t** out) {
  *out = nullptr;
  if (!mask) return HSAW_OK;
  HSAW_TRY(dmalloc((void**)out, len, s));
  HSAW_CK(cudaMemcpyAsync(*out, mask, len, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  return HSAW_OK;
}

static hsaw_status validate_common(const Graph& g, const hsaw_query* q, int64_t* n_cand) {
  if (q->mode != HSAW_EDGE && q->mode != HSAW_NODE) return fail(HSAW_E_INVALID, "query: unknown mode");
  const int64_t M = q->mode == HSAW_EDGE ? g.m : g.n;
  int64_t c = M;
  if (q->candidate_mask) {
    c = 0;
    for (int64_t x = 0; x < M; ++x) c += q->candidate_mask[x] ? 1 : 0;
  }
  if (q->k < 1 || q->k > c) return fail(HSAW_E_INVALID, "query: need 1 <= k <= |C|");
  *n_cand = c;
  return HSAW_OK;
}

struct SolveScratch {
  QueryDev qd;
  Stream st;
  Cover cv;
  uint8_t* cand = nullptr;
  cudaStream_t s;
  explicit SolveScratch(cudaStream_t st_) : s(st_) {}
  ~SolveScratch() {
    cudaStreamSynchronize(s);
    query_release(qd, s);
    st.release(s);
    cv.release(s);
    dfree(cand, s);
  }
};

static hsaw_status aid_at(const Stream& st, int64_t j, uint64_t* out, cudaStream_t s) {
  HSAW_CK(cudaMemcpyAsync(out, st.aid.p + j, 8, cudaMemcpyDeviceToHost, s));
  HSAW_CK(cudaStreamSynchronize(s));
  return HSAW_OK;
}

static thread_local const volatile int* t_cancel = nullptr;
void set_cancel_flag(const volatile int* flag) { t_cancel = flag; }
bool cancel_requested() { return t_cancel && *t_cancel; }

// Counting, greedy and the result of a fixed-N solve over the first q->n_hsaw hits of st.
static hsaw_status fixed_tail(const Graph& g, const hsaw_query* q, Stream& st, Cover& cv, const uint8_t* cand,
                              hsaw_result* r, cudaStream_t s) {
  const int64_t M = q->mode == HSAW_EDGE ? g.m : g.n;
  const int32_t k = q->k;
  void* ph = phase_begin(s);
  HSAW_TRY(cover_build(st, q->mode, 0, q->n_hsaw, cv, s));
  phase_end(ph, s, PH_COUNT);
  ph = phase_begin(s);
  HSAW_TRY(cover_greedy(cv, cand, M, k, r->ids, r->gains, s));
  phase_end(ph, s, PH_GREEDY);
  uint64_t last = 0;
  HSAW_TRY(aid_at(st, q->n_hsaw - 1, &last, s));
  uint64_t cov = 0;
  for (int32_t i = 0; i < k; ++i) cov += r->gains[i];
  const double n = (double)g.n;
  r->n_selected = k;
  r->rounds_t = 0;
  r->cov_Rprime = r->hits_Rprime = r->attempts_Rprime = 0;
  r->eps_t = NAN;
  r->hits = (uint64_t)q->n_hsaw;
  r->attempts = last + 1;
  r->cov_R = cov;
  r->spread_base_est = n * (double)r->hits / (double)r->attempts;
  r->spread_reduction_est = n * (double)cov / (double)r->attempts;
  r->steps = st.steps;
  return HSAW_OK;
}

hsaw_status validate_query(const Graph& g, const hsaw_query* q) {
  int64_t n_cand = 0;
  return validate_common(g, q, &n_cand);
}

hsaw_status solve_fixed_from_stream(const Graph& g, const hsaw_query* q, Stream& st, hsaw_result* r, cudaStream_t s) {
  if (!q || !r || !r->ids || !r->gains) return fail(HSAW_E_INVALID, "solve: NULL argument");
  int64_t n_cand = 0;
  HSAW_TRY(validate_common(g, q, &n_cand));
  if (q->n_hsaw < 1 || st.count < q->n_hsaw) return fail(HSAW_E_INVALID, "solve: stream shorter than n_hsaw");
  const int64_t M = q->mode == HSAW_EDGE ? g.m : g.n;
  Cover cv;
  uint8_t* cand = nullptr;
  hsaw_status rc = upload_mask(q->candidate_mask, (size_t)M, false, s, &cand);
  if (rc == HSAW_OK) rc = fixed_tail(g, q, st, cv, cand, r, s);
  cudaStreamSynchronize(s);
  cv.release(s);
  dfree(cand, s);
  return rc;
}

static hsaw_status solve(const Graph& g, const hsaw_query* q, hsaw_result* r, cudaStream_t s) {
  if (!q || !r || !r->ids || !r->gains) return fail(HSAW_E_INVALID, "solve: NULL argument");
  int64_t n_cand = 0;
  HSAW_TRY(validate_common(g, q, &n_cand));
  const int64_t M = q->mode == HSAW_EDGE ? g.m : g.n;
  const int32_t k = q->k;
  const double n = (double)g.n;
  SolveScratch W(s);
  HSAW_TRY(query_upload(g, q, W.qd, s));
  HSAW_TRY(upload_mask(q->candidate_mask, (size_t)M, false, s, &W.cand));
  HSAW_TRY(stream_init(W.st, 0, q->max_attempts, s));
  r->n_selected = k;
  r->rounds_t = 0;
  r->cov_Rprime = r->hits_Rprime = r->attempts_Rprime = 0;
  r->eps_t = NAN;
  if (q->sampling == HSAW_FIXED_N) {
    if (q->n_hsaw < 1) return fail(HSAW_E_INVALID, "query: n_hsaw < 1");
    void* ph = phase_begin(s);
    HSAW_TRY(stream_extend(g, W.qd, W.st, q->n_hsaw, s));
    phase_end(ph, s, PH_SAMPLE);
    HSAW_TRY(fixed_tail(g, q, W.st, W.cv, W.cand, r, s));
  } else if (q->sampling == HSAW_STOP_RULE) {
    if (!(q->eps > 0.0 && q->eps < 1.0)) return fail(HSAW_E_INVALID, "query: need 0 < eps < 1");
    const double delta = q->delta > 0 ? q->delta : 1.0 / n;
    double c6[6];
    stop_constants(M, k, q->eps, delta, c6);
    const double n_max = c6[1], t_max = c6[3], lam1 = c6[5];
    const int64_t L = (int64_t)std::ceil(c6[4]);
    std::vector<int64_t> ids(k);
    std::vector<uint32_t> gains(k);
    for (int32_t t = 1;; ++t) {
      if (cancel_requested()) return fail(HSAW_E_CANCELLED, "solve: query cancelled");
      if (t > 40 || (L << (t - 1)) > (int64_t)1 << 30) return fail(HSAW_E_NOMEM, "stop rule: sample budget beyond device limits");
      const int64_t half = L << (t - 1);
      // Check stops the rule only when Cov_{R'_t}(T) >= Lambda1, and Cov_{R'_t}(T) <= |R'_t|:
      // a round with |R'_t| < Lambda1 (always t = 1, as L < Lambda1) that is not the last one
      // cannot end the loop, and every result field is rewritten by a later round
      if ((double)half < lam1 && !((double)half >= n_max || (double)t >= t_max)) continue;
      void* ph = phase_begin(s);
      HSAW_TRY(stream_extend(g, W.qd, W.st, 2 * half, s));
      phase_end(ph, s, PH_SAMPLE);
      ph = phase_begin(s);
      HSAW_TRY(cover_build(W.st, q->mode, 0, half, W.cv, s));
      phase_end(ph, s, PH_COUNT);
      ph = phase_begin(s);
      HSAW_TRY(cover_greedy(W.cv, W.cand, M, k, ids.data(), gains.data(), s));
      phase_end(ph, s, PH_GREEDY);
      uint64_t cov = 0;
      for (int32_t i = 0; i < k; ++i) cov += gains[i];
      uint64_t covp = 0;
      ph = phase_begin(s);
      HSAW_TRY(cover_count(W.st, q->mode, half, half, ids.data(), k, &covp, s));
      phase_end(ph, s, PH_COVERAGE);
      double et;
      const int ok = check_bound((double)cov, (double)covp, (double)half, t, q->eps, lam1, &et);
      uint64_t a_half = 0, a_all = 0;
      HSAW_TRY(aid_at(W.st, half - 1, &a_half, s));
      HSAW_TRY(aid_at(W.st, 2 * half - 1, &a_all, s));
      for (int32_t i = 0; i < k; ++i) {
        r->ids[i] = ids[i];
        r->gains[i] = gains[i];
      }
      r->rounds_t = t;
      r->hits = (uint64_t)(2 * half);
      r->attempts = a_all + 1;
      r->cov_R = cov;
      r->cov_Rprime = covp;
      r->hits_Rprime = (uint64_t)half;
      r->attempts_Rprime = a_all - a_half;
      r->spread_base_est = n * (double)r->hits / (double)r->attempts;
      r->spread_reduction_est = n * (double)(cov + covp) / (double)r->attempts;
      if (!std::isnan(et)) r->eps_t = et;
      if (ok) break;
      if ((double)half >= n_max || (double)t >= t_max) break;
    }
  } else {
    return fail(HSAW_E_INVALID, "query: unknown sampling rule");
  }
  r->steps = W.st.steps;
  return HSAW_OK;
}

hsaw_status solve_one(const Graph& g, const hsaw_query* q, hsaw_result* r, cudaStream_t s) {
  return solve(g, q, r, s);
}

}  // namespace hsaw

using namespace hsaw;

extern "C" {

hsaw_status hsaw_solve(hsaw_graph g, const hsaw_query* q, hsaw_result* r, void* stream) {
  if (!g) return fail(HSAW_E_INVALID, "solve: NULL graph");
  return solve(g->g, q, r, (cudaStream_t)stream);
}

hsaw_status hsaw_sample(hsaw_graph g, const hsaw_query* q, uint64_t first_attempt, int64_t n_hits,
                        const uint8_t* edge_removed, const uint8_t* node_removed, uint32_t removed_flags,
                        hsaw_walks* out, void* stream) {
  if (!g || !q || !out) return fail(HSAW_E_INVALID, "sample: NULL argument");
  *out = nullptr;
  if (n_hits < 0) return fail(HSAW_E_INVALID, "sample: n_hits < 0");
  cudaStream_t s = (cudaStream_t)stream;
  auto* w = new (std::nothrow) hsaw_walks_s();
  if (!w) return fail(HSAW_E_NOMEM, "sample: host allocation");
  cudaGetDevice(&w->device);
  hsaw_status st = query_upload(g->g, q, w->qd, s);
  const bool dev = removed_flags & HSAW_INPUT_DEVICE;
  if (st == HSAW_OK) st = upload_mask(edge_removed, (size_t)g->g.m, dev, s, &w->qd.edge_removed);
  if (st == HSAW_OK) st = upload_mask(node_removed, (size_t)g->g.n, dev, s, &w->qd.node_removed);
  w->qd.owns_removed = true;
  if (st == HSAW_OK) st = stream_init(w->st, first_attempt, q->max_attempts, s);
  if (st == HSAW_OK) st = stream_extend(g->g, w->qd, w->st, n_hits, s);
  if (st == HSAW_OK) {
    if (cudaStreamSynchronize(s) != cudaSuccess) st = fail(HSAW_E_DEVICE, "sample: stream sync failed");
  }
  if (st != HSAW_OK) {
    cudaStreamSynchronize(s);
    query_release(w->qd, s);
    w->st.release(s);
    delete w;
    return st;
  }
  *out = w;
  return HSAW_OK;
}

__global__ void k_mark_removed(const int64_t* __restrict__ ids, int32_t cnt, uint8_t* __restrict__ mask) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) mask[ids[i]] = 1;
}

hsaw_status hsaw_estimate_spread(hsaw_graph g, const hsaw_query* q, const int64_t* removed, int32_t n_removed,
                                 double* spread, double* std_err, void* stream) {
  if (!g || !q || !spread || (n_removed > 0 && !removed)) return fail(HSAW_E_INVALID, "estimate: NULL argument");
  if (q->n_hsaw < 1) return fail(HSAW_E_INVALID, "estimate: n_hsaw < 1");
  const Graph& G = g->g;
  const bool edges = q->mode == HSAW_EDGE;
  const int64_t M = edges ? G.m : G.n;
  for (int32_t i = 0; i < n_removed; ++i)
    if (removed[i] < 0 || removed[i] >= M) return fail(HSAW_E_RANGE, "estimate: removed id out of range");
  cudaStream_t s = (cudaStream_t)stream;
  SolveScratch W(s);
  HSAW_TRY(query_upload(G, q, W.qd, s));
  if (n_removed > 0) {
    uint8_t* mask = nullptr;
    int64_t* d_ids = nullptr;
    HSAW_TRY(dmalloc((void**)&mask, (size_t)M, s));
    (edges ? W.qd.edge_removed : W.qd.node_removed) = mask;
    W.qd.owns_removed = true;
    HSAW_CK(cudaMemsetAsync(mask, 0, (size_t)M, s));
    HSAW_TRY(dmalloc((void**)&d_ids, (size_t)n_removed * 8, s));
    HSAW_CK(cudaMemcpyAsync(d_ids, removed, (size_t)n_removed * 8, cudaMemcpyHostToDevice, s));
    count_launch();
    k_mark_removed<<<grid_for(n_removed, 256, 1024), 256, 0, s>>>(d_ids, n_removed, mask);
    HSAW_CK(cudaGetLastError());
    dfree(d_ids, s);
  }
  HSAW_TRY(stream_init(W.st, 0, q->max_attempts, s));
  HSAW_TRY(stream_extend(G, W.qd, W.st, q->n_hsaw, s));
  uint64_t last = 0;
  HSAW_TRY(aid_at(W.st, q->n_hsaw - 1, &last, s));
  const double A = (double)(last + 1), f = (double)q->n_hsaw / A, n = (double)G.n;
  *spread = n * (double)q->n_hsaw / A;
  if (std_err) *std_err = n * std::sqrt(f * (1.0 - f) / A);
  return HSAW_OK;
}

hsaw_status hsaw_walks_info(hsaw_walks w, int64_t* count, int64_t* total_nodes, uint64_t* attempts, uint64_t* steps) {
  if (!w) return fail(HSAW_E_INVALID, "walks: NULL handle");
  if (count) *count = w->st.count;
  if (total_nodes) *total_nodes = w->st.total_nodes;
  if (attempts) *attempts = w->st.next_attempt - w->st.first_attempt;
  if (steps) *steps = w->st.steps;
  return HSAW_OK;
}

hsaw_status hsaw_walks_export(hsaw_walks w, uint64_t* aid, int64_t* node_off, int32_t* nodes, int32_t* edges,
                              void* stream) {
  if (!w) return fail(HSAW_E_INVALID, "walks: NULL handle");
  cudaStream_t s = (cudaStream_t)stream;
  const Stream& st = w->st;
  if (aid && st.count) HSAW_CK(cudaMemcpyAsync(aid, st.aid.p, (size_t)st.count * 8, cudaMemcpyDeviceToHost, s));
  if (node_off) HSAW_CK(cudaMemcpyAsync(node_off, st.node_off.p, (size_t)(st.count + 1) * 8, cudaMemcpyDeviceToHost, s));
  if (nodes && st.total_nodes)
    HSAW_CK(cudaMemcpyAsync(nodes, st.nodes.p, (size_t)st.total_nodes * 4, cudaMemcpyDeviceToHost, s));
  if (edges && st.total_nodes > st.count)
    HSAW_CK(cudaMemcpyAsync(edges, st.edges.p, (size_t)(st.total_nodes - st.count) * 4, cudaMemcpyDeviceToHost, s));
  HSAW_CK(cudaStreamSynchronize(s));
  return HSAW_OK;
}

hsaw_status hsaw_walks_export_device(hsaw_walks w, uint64_t* aid, int64_t* node_off, int32_t* nodes, int32_t* edges,
                                     void* stream) {
  if (!w) return fail(HSAW_E_INVALID, "walks: NULL handle");
  cudaStream_t s = (cudaStream_t)stream;
  const Stream& st = w->st;
  const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
  if (aid && st.count) HSAW_CK(cudaMemcpyAsync(aid, st.aid.p, (size_t)st.count * 8, dd, s));
  if (node_off) HSAW_CK(cudaMemcpyAsync(node_off, st.node_off.p, (size_t)(st.count + 1) * 8, dd, s));
  if (nodes && st.total_nodes) HSAW_CK(cudaMemcpyAsync(nodes, st.nodes.p, (size_t)st.total_nodes * 4, dd, s));
  if (edges && st.total_nodes > st.count)
    HSAW_CK(cudaMemcpyAsync(edges, st.edges.p, (size_t)(st.total_nodes - st.count) * 4, dd, s));
  HSAW_CK(cudaStreamSynchronize(s));
  return HSAW_OK;
}

hsaw_status hsaw_walks_destroy(hsaw_walks w) {
  if (!w) return HSAW_OK;
  cudaDeviceSynchronize();
  query_release(w->qd, nullptr);
  w->st.release(nullptr);
  cudaDeviceSynchronize();
  delete w;
  return HSAW_OK;
}

hsaw_status hsaw_classify(hsaw_graph g, const hsaw_query* q, uint64_t first, int64_t count, int8_t* outcome_dev,
                          int32_t* length_dev, void* stream) {
  if (!g || !q || (count > 0 && (!outcome_dev || !length_dev))) return fail(HSAW_E_INVALID, "classify: NULL argument");
  if (count <= 0) return HSAW_OK;
  cudaStream_t s = (cudaStream_t)stream;
  QueryDev qd;
  hsaw_status st = query_upload(g->g, q, qd, s);
  if (st == HSAW_OK) st = classify_attempts(g->g, qd, first, count, outcome_dev, length_dev, s);
  cudaStreamSynchronize(s);
  query_release(qd, s);
  return st;
}

hsaw_status hsaw_histogram(hsaw_walks w, hsaw_mode mode, int64_t first, int64_t count, int32_t* uid, uint32_t* cnt,
                           int64_t cap, int64_t* n_unique, void* stream) {
  if (!w || !n_unique) return fail(HSAW_E_INVALID, "histogram: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  Cover cv;
  hsaw_status st = cover_build(w->st, mode, first, count, cv, s);
  if (st == HSAW_OK) {
    *n_unique = cv.unique;
    if (cv.unique > cap) {
      st = fail(HSAW_E_INVALID, "histogram: output capacity too small");
    } else if (cv.unique > 0) {
      if (uid) cudaMemcpyAsync(uid, cv.uid.p, (size_t)cv.unique * 4, cudaMemcpyDeviceToHost, s);
      if (cnt) cudaMemcpyAsync(cnt, cv.cnt.p, (size_t)cv.unique * 4, cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) st = fail(HSAW_E_DEVICE, "histogram: copy failed");
    }
  }
  cudaStreamSynchronize(s);
  cv.release(s);
  return st;
}

hsaw_status hsaw_greedy(hsaw_walks w, hsaw_graph g, hsaw_mode mode, int64_t first, int64_t count,
                        const uint8_t* candidate_mask, int32_t k, int64_t* ids, uint32_t* gains, void* stream) {
  if (!w || !g || !ids || !gains) return fail(HSAW_E_INVALID, "greedy: NULL argument");
  const int64_t M = mode == HSAW_EDGE ? g->g.m : g->g.n;
  int64_t c = M;
  if (candidate_mask) {
    c = 0;
    for (int64_t x = 0; x < M; ++x) c += candidate_mask[x] ? 1 : 0;
  }
  if (k < 1 || k > c) return fail(HSAW_E_INVALID, "greedy: need 1 <= k <= |C|");
  cudaStream_t s = (cudaStream_t)stream;
  Cover cv;
  uint8_t* cand = nullptr;
  hsaw_status st = upload_mask(candidate_mask, (size_t)M, false, s, &cand);
  if (st == HSAW_OK) st = cover_build(w->st, mode, first, count, cv, s);
  if (st == HSAW_OK) st = cover_greedy(cv, cand, M, k, ids, gains, s);
  cudaStreamSynchronize(s);
  cv.release(s);
  dfree(cand, s);
  return st;
}

hsaw_status hsaw_coverage(hsaw_walks w, hsaw_mode mode, int64_t first, int64_t count, const int64_t* T, int32_t k,
                          uint64_t* cov, void* stream) {
  if (!w || !cov || (k > 0 && !T)) return fail(HSAW_E_INVALID, "coverage: NULL argument");
  return cover_count(w->st, mode, first, count, T, k, cov, (cudaStream_t)stream);
}

hsaw_status hsaw_stop_constants(int64_t M, int32_t k, double eps, double delta, double* out6) {
  if (!out6 || M < 1 || k < 1 || k > M || !(eps > 0 && eps < 1) || !(delta > 0 && delta < 1))
    return fail(HSAW_E_INVALID, "stop constants: need 1 <= k <= M, 0 < eps, delta < 1");
  stop_constants(M, k, eps, delta, out6);
  return HSAW_OK;
}

int hsaw_check(double c, double cp, double size_rprime, int32_t t, double eps, double lambda1, double* eps_t) {
  double tmp;
  return check_bound(c, cp, size_rprime, t, eps, lambda1, eps_t ? eps_t : &tmp);
}

}  // extern "C"
