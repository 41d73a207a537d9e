// Internal state of a query: device suspect set, the ordered HSAW stream and the
// counting / greedy workspaces (not part of the ABI).
#pragma once
#include "common.cuh"

namespace hsaw {

// Device view of the suspects V_I = (V_I, p) (Sec. 2.2) and of an optional residual graph.
struct QueryDev {
  uint32_t* s_bits = nullptr;     // n bits: v in V_I
  uint32_t* p32 = nullptr;        // n words or NULL (p == 1)
  int32_t* s_list = nullptr;      // n_src node ids of V_I
  int32_t n_src = 0;
  uint8_t* edge_removed = nullptr;  // m bytes or NULL
  uint8_t* node_removed = nullptr;  // n bytes or NULL
  uint64_t seed = 0;
  bool owns_removed = false;
};

hsaw_status query_upload(const Graph& g, const hsaw_query* q, QueryDev& qd, cudaStream_t s);
void query_release(QueryDev& qd, cudaStream_t s);

// The ordered HSAW stream R_1, R_2, ... of Alg. 3: hit j has attempt id aid[j], l_j =
// len[j] nodes nodes[node_off[j] .. node_off[j+1]) and l_j - 1 edges starting at
// edges[node_off[j] - j].
struct Stream {
  int64_t count = 0;
  int64_t total_nodes = 0;
  uint64_t first_attempt = 0;
  uint64_t next_attempt = 0;  // first attempt id not examined yet
  uint64_t steps = 0;         // live-edge draws executed
  uint64_t max_attempts = 0;
  DBuf<uint64_t> aid;
  DBuf<uint32_t> len;
  DBuf<int64_t> node_off;  // count + 1
  DBuf<int32_t> nodes;
  DBuf<int32_t> edges;
  // per-launch workspace
  DBuf<uint32_t> chunk_hits, chunk_off, ctrs;
  DBuf<uint2> recs;
  DBuf<uint64_t> tmp64;
  DBuf<uint32_t> pbits;  // walk pool: one bit per attempt of a window
  DBuf<uint64_t> pcnt;   // walk pool: entries per (source, block), then their prefix
  double hit_rate = 0.0;  // running estimate for launch sizing
  int64_t elem_range[2] = {0, 0};  // [node mode, edge mode]: element ids lie in [0, n) / [0, m)
  void release(cudaStream_t s);
};

hsaw_status stream_init(Stream& st, uint64_t first_attempt, uint64_t max_attempts, cudaStream_t s);
// Extend the stream until it holds at least want hits (Alg. 3 loop).
hsaw_status stream_extend(const Graph& g, const QueryDev& qd, Stream& st, int64_t want, cudaStream_t s);
// Adopt new_hits hits whose attempt ids and lengths are already at aid/len[st.count ..]:
// their walk offsets, nodes and edges (re-drawn from the attempt ids), and the count.
hsaw_status stream_take_hits(const Graph& g, const QueryDev& qd, Stream& st, uint32_t new_hits, cudaStream_t s);
hsaw_status classify_attempts(const Graph& g, const QueryDev& qd, uint64_t first, int64_t count, int8_t* outcome,
                              int32_t* length, cudaStream_t s);

// Occurrence counts and inverted index over walks [first, first + count) (a5, a6).
struct Cover {
  int64_t walks = 0, entries = 0, unique = 0;
  DBuf<uint32_t> keys, vals, keys2, vals2;  // sort workspace
  DBuf<uint32_t> run_flag;                  // entries
  DBuf<int32_t> uid;                        // unique element ids, increasing
  DBuf<uint32_t> cnt;                       // occurrence count per unique element
  DBuf<uint32_t> inv_off;                   // unique + 1
  DBuf<uint32_t> inv_walk;                  // entries: local walk index, grouped by element
  DBuf<uint32_t> entry_uidx;                // entries: unique index of each walk entry
  DBuf<uint32_t> walk_eoff;                 // walks + 1: entry offsets of the walks
  DBuf<uint32_t> cnt_work;                  // greedy's running counts
  DBuf<uint32_t> covered;  // greedy: per walk, 0 or 1 + the pick that covered it
  DBuf<uint8_t> dirty;     // greedy (grid version): group dirty flags
  DBuf<uint4> inv_ent;           // cluster greedy: inverted-index entries with their walk's entry range
  DBuf<uint32_t> g_idx, g_list, g_cnt, g_entry;  // greedy on the heavy elements: index map, list, counts, entries
  DBuf<uint2> g_rng;             // greedy: each element's entries of inv_ent
  DBuf<unsigned long long> partial;
  void release(cudaStream_t s);
};

hsaw_status cover_build(const Stream& st, hsaw_mode mode, int64_t first, int64_t count, Cover& cv, cudaStream_t s);
// Greedy (Alg. 4 / 7) on a built Cover; cand (device, M bytes) may be NULL.
hsaw_status cover_greedy(Cover& cv, const uint8_t* cand_dev, int64_t M, int32_t k, int64_t* ids_host,
                         uint32_t* gains_host, cudaStream_t s);
// #walks in [first, first + count) that contain an element of T (T host, k ids).
hsaw_status cover_count(const Stream& st, hsaw_mode mode, int64_t first, int64_t count, const int64_t* T, int32_t k,
                        uint64_t* cov, cudaStream_t s);

// Walk pool (pool.cu).
void pool_release(WalkPool& p);
hsaw_status pool_build(Graph& g, uint64_t seed, uint64_t attempts, cudaStream_t s);
// Append to st (aid, len at st.count) the hits among attempts [a0, a1) (a1 <= pool.attempts),
// in attempt order; *new_hits receives their number.
hsaw_status pool_hits(const Graph& g, const QueryDev& qd, Stream& st, uint64_t a0, uint64_t a1, uint32_t* new_hits,
                      cudaStream_t s);

// Cancellation of the calling thread's current solve (set by the server's workers):
// checked between sampler launches and between stopping-rule rounds.
void set_cancel_flag(const volatile int* flag);
bool cancel_requested();

// One full solve on `s` (the body of hsaw_solve).
hsaw_status solve_one(const Graph& g, const hsaw_query* q, hsaw_result* r, cudaStream_t s);
// The fixed-N solve from a stream that already holds at least q->n_hsaw hits: counting,
// greedy (Alg. 4 / 7) and the result fields.
hsaw_status solve_fixed_from_stream(const Graph& g, const hsaw_query* q, Stream& st, hsaw_result* r, cudaStream_t s);
// Batched fixed-N sampling (batch.cu): extends every stream i to want[i] hits with
// multi-instance sampler launches.
// status[i] (in: HSAW_OK to take part) becomes HSAW_E_TIMEOUT when instance i's attempt
// budget runs out first; the return value reports failures of the launches themselves.
// staged[i] receives the number of hits appended to stream i's aid/len after its count:
// stream_take_hits(..., staged[i]) draws their walks.
hsaw_status batch_sample(const Graph* const* gs, const QueryDev* const* qds, Stream* const* sts, const int64_t* want,
                         int32_t count, hsaw_status* status, int64_t* staged, cudaStream_t s);
// Query checks shared by every solve: mode, 1 <= k <= |C|.
hsaw_status validate_query(const Graph& g, const hsaw_query* q);

// Stopping-rule constants (Sec. 5.1) and Check (Alg. 5), host FP64.
void stop_constants(int64_t M, int32_t k, double eps, double delta, double out6[6]);
int check_bound(double c, double cp, double size_rp, int32_t t, double eps, double lambda1, double* eps_t);

}  // namespace hsaw

struct hsaw_walks_s {
  hsaw::Stream st;
  hsaw::QueryDev qd;
  int device = 0;
};
