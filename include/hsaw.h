/*
 * hsaw.h - C ABI of the GB300 (sm_103a) Spread Interdiction library.
 *
 * The library computes the data-parallel path of "Blocking Self-avoiding Walks Stops
 * Cyber-epidemics" (Sec. 3-5): Hitting Self-avoiding Walk (HSAW) sampling under the
 * Linear Threshold model, the element-occurrence counting over the walks and the greedy
 * max-coverage that picks the k edges (eSI, Def. "edge_remove") or nodes (nSI,
 * Def. "node_remove") whose removal suspends the most expected infection, either from a
 * fixed number of walks or under the paper's sample-doubling stopping rule (Alg. 6 / 9).
 *
 * Conventions shared by every call
 *   - Every call returns hsaw_status; no call aborts, traps or exits.  A failing call
 *     leaves its outputs unspecified and sets a thread-local message (hsaw_last_error).
 *   - Host arrays passed in are read during the call only; the caller keeps ownership.
 *     Arrays flagged HSAW_INPUT_DEVICE (or documented as device buffers) must be device
 *     memory of the current CUDA device.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls that return
 *     host-visible results synchronise that stream before returning.
 *   - Node ids are int32 in [0, n); edge ids are int32 CSR positions in [0, m) of the
 *     in-adjacency sorted by destination (stable: input order within a node).
 *   - LT weights are uint32 fixed point: w(u,v) = w_fixed / 2^32.  Each node's in-sum
 *     must be <= 2^32 - 1 (Sec. 2.1: in-weight sum <= 1); HSAW_E_WEIGHT_SUM otherwise.
 *   - Randomness: Philox4x32-10 (Salmon et al., SC'11).  Attempt a is one live-edge
 *     world: node v's draw is Philox(key = seed, counter = (lo32 a, hi32 a, v, 0)),
 *     lane x0 picks v's live in-edge (the first j with x0 < thr[j]), lane x1 is v's
 *     source coin (x1 < p32(v); p32 = 0xFFFFFFFF certain); the start node is
 *     floor(x0 * n / 2^32) of Philox(counter = (lo32 a, hi32 a, 0, 1)).  Hits are
 *     ordered by attempt id, so every result is a pure function of (graph, query, seed).
 */
#ifndef HSAW_H_
#define HSAW_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HSAW_API __attribute__((visibility("default")))
#else
#define HSAW_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HSAW_OK = 0,
  HSAW_E_INVALID = -1,     /* bad argument: sizes, k outside [1, |C|], duplicate sources, eps */
  HSAW_E_WEIGHT_SUM = -2,  /* a node's in-weight sum exceeds 2^32 - 1 */
  HSAW_E_RANGE = -3,       /* a node or edge index out of range */
  HSAW_E_NOMEM = -4,       /* device or host allocation failed */
  HSAW_E_DEVICE = -5,      /* a CUDA call failed (message in hsaw_last_error) */
  HSAW_E_STEP_CAP = -6,    /* a walk exceeded its step guard (cannot happen for valid graphs) */
  HSAW_E_TIMEOUT = -7,     /* attempt budget exhausted before enough walks hit */
  HSAW_E_REJECTED = -8,    /* server admission refused the query */
  HSAW_E_CANCELLED = -9,   /* query cancelled */
  HSAW_E_PENDING = -10     /* server poll: the query is still running (the ticket stays valid) */
} hsaw_status;

typedef enum { HSAW_EDGE = 0 /* eSI */, HSAW_NODE = 1 /* nSI */ } hsaw_mode;
typedef enum { HSAW_FIXED_N = 0, HSAW_STOP_RULE = 1 } hsaw_sampling;

#define HSAW_INPUT_DEVICE 1u /* graph-ingest flag: the input arrays are device pointers */

typedef struct hsaw_graph_s* hsaw_graph; /* opaque, library-owned device graph */
typedef struct hsaw_walks_s* hsaw_walks; /* opaque, library-owned ordered HSAW stream */

/* ------------------------------------------------------------------ graph ingest
 * Sec. 2.1 (directed G = (V, E, w), LT in-weight sums <= 1); the live-edge model picks
 * in-edge j of v with probability w_j / 2^32, so the library stores, per node, the
 * running sums thr[j] of its in-weights.
 *
 * hsaw_graph_from_edges: n nodes, m edges (src[e] -> dst[e], weight w_fixed[e]).
 *   The in-adjacency is a stable sort by dst, done on the device.  src, dst, w_fixed are
 *   host arrays, or device arrays if flags & HSAW_INPUT_DEVICE.  Errors: HSAW_E_INVALID
 *   (n < 1, m < 0, n or m >= 2^31), HSAW_E_RANGE (an endpoint outside [0, n)),
 *   HSAW_E_WEIGHT_SUM, HSAW_E_NOMEM, HSAW_E_DEVICE.  *out is set only on HSAW_OK.
 * hsaw_graph_from_csr: the in-adjacency is given: in_row_ptr (int64, n+1, in_row_ptr[0]
 *   = 0, non-decreasing, in_row_ptr[n] = m), in_src (int32, m) and w_fixed (uint32, m);
 *   edge ids are the given positions.  Same flags and errors. */
HSAW_API hsaw_status hsaw_graph_from_edges(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                  const uint32_t* w_fixed, uint32_t flags, void* stream, hsaw_graph* out);
HSAW_API hsaw_status hsaw_graph_from_csr(int64_t n, int64_t m, const int64_t* in_row_ptr, const int32_t* in_src,
                                const uint32_t* w_fixed, uint32_t flags, void* stream, hsaw_graph* out);
/* Frees the device graph.  NULL is accepted.  The caller must not use g afterwards. */
HSAW_API hsaw_status hsaw_graph_destroy(hsaw_graph g);
/* Sizes of g. */
HSAW_API hsaw_status hsaw_graph_info(hsaw_graph g, int64_t* n, int64_t* m);
/* Copies the device CSR to host arrays (any may be NULL): in_row_ptr int64[n+1],
 * in_src int32[m], in_dst int32[m], thr uint32[m] (running in-weight sums),
 * input_index int64[m] (CSR position -> input edge index; identity for from_csr). */
HSAW_API hsaw_status hsaw_graph_export(hsaw_graph g, int64_t* in_row_ptr, int32_t* in_src, int32_t* in_dst,
                              uint32_t* thr, int64_t* input_index, void* stream);

/* Endpoints of edge `edge_id` (a CSR position): *src -> *dst, and its index in the input
 * edge list (the position itself for hsaw_graph_from_csr).  Any output may be NULL.
 * HSAW_E_RANGE when edge_id is outside [0, m). */
HSAW_API hsaw_status hsaw_graph_edge(hsaw_graph g, int64_t edge_id, int32_t* src, int32_t* dst,
                                     int64_t* input_index);

/* Walk pool (not in the paper; serving many queries on one graph).  Attempt a's walk
 * ignoring sources - its nodes until no live in-edge or a cycle - does not depend on the
 * query: a query's HSAW of attempt a is that trace's prefix up to its first real source
 * (same node-keyed draws and coins), so attempt a hits exactly when its trace holds a real
 * source.  hsaw_graph_build_walk_pool walks attempts [0, attempts) for walk seed `seed`
 * and keeps, per block of 2^22 attempts, each node's list of the attempts whose trace
 * passes through it (about 4 B per trace node, plus 4 (n + 1) B per block).  Afterwards
 * every solve, sample or served query on g with q->seed == seed and no removed elements
 * takes its hits among attempts below `attempts` from its sources' lists (re-walking only
 * the hits), and samples the rest as usual, with bit-identical results.  Building
 * replaces any previous pool; do not build or drop while other calls use g.  Errors:
 * HSAW_E_NOMEM if the index does not fit, HSAW_E_INVALID for more than 2^32 attempts or a
 * block whose traces exceed 2^32 nodes, HSAW_E_STEP_CAP.  hsaw_graph_drop_walk_pool frees
 * it. */
HSAW_API hsaw_status hsaw_graph_build_walk_pool(hsaw_graph g, uint64_t seed, uint64_t attempts, void* stream);
HSAW_API hsaw_status hsaw_graph_drop_walk_pool(hsaw_graph g);

/* ------------------------------------------------------------------ query
 * Sec. 2.2: suspects V_I = (V_I, p) (Eq. "prob_src_set"), candidates C, budget k
 * (Defs. "edge_remove" / "node_remove"); Alg. 6 inputs eps, delta. */
typedef struct {
  const int32_t* sources;        /* host array: V_I, distinct node ids in [0, n) */
  int32_t n_sources;             /* >= 1 */
  const uint32_t* p_fixed;       /* host array (n_sources) or NULL for p == 1; p = p_fixed / 2^32,
                                    0xFFFFFFFF means certain */
  hsaw_mode mode;                /* HSAW_EDGE (eSI) or HSAW_NODE (nSI) */
  int32_t k;                     /* budget, 1 <= k <= |C| */
  const uint8_t* candidate_mask; /* host array of m (eSI) or n (nSI) bytes, nonzero = in C; NULL = C is E or V */
  hsaw_sampling sampling;        /* HSAW_FIXED_N or HSAW_STOP_RULE */
  int64_t n_hsaw;                /* FIXED_N: number of HSAWs N */
  double eps, delta;             /* STOP_RULE: 0 < eps < 1; delta <= 0 means 1/n */
  uint64_t seed;                 /* Philox key */
  uint64_t max_attempts;         /* attempt budget, 0 = 2^62; exceeding it gives HSAW_E_TIMEOUT */
} hsaw_query;

typedef struct {
  int64_t* ids;          /* caller host buffer, capacity k: edge ids or node ids in pick order */
  uint32_t* gains;       /* caller host buffer, capacity k: marginal coverage of each pick on R_t */
  int32_t n_selected;    /* = k */
  int32_t rounds_t;      /* stopping-rule iterations (0 for FIXED_N) */
  uint64_t hits;         /* HSAWs used: |R| (FIXED_N) or |R_t| + |R'_t| */
  uint64_t attempts;     /* attempts up to and including the one that gave the last hit used */
  uint64_t steps;        /* live-edge draws the sampler executed (every launch; attempts served from a
                            walk pool need none) - a throughput counter, not part of the result */
  uint64_t cov_R;        /* Cov_{R_t}(T) = sum of gains */
  uint64_t cov_Rprime;   /* Cov_{R'_t}(T) (0 for FIXED_N) */
  uint64_t hits_Rprime;  /* |R'_t| */
  uint64_t attempts_Rprime; /* attempts that produced R'_t */
  double spread_base_est;      /* I_hat = n * hits / attempts */
  double spread_reduction_est; /* D_hat = n * (cov_R + cov_Rprime) / attempts */
  double eps_t;                /* last Check bound (NaN if never computed) */
} hsaw_result;

/* Solve one interdiction instance: Alg. 6 (eSIA) / Alg. 9 (nSIA) for HSAW_STOP_RULE, or
 * Greedy (Alg. 4 / 7) over the first n_hsaw HSAWs for HSAW_FIXED_N.  Ties in the greedy
 * go to the smallest id; once every remaining gain is 0 the smallest unpicked candidates
 * are taken, so exactly k ids are returned.  Errors: HSAW_E_INVALID, HSAW_E_RANGE,
 * HSAW_E_NOMEM, HSAW_E_DEVICE, HSAW_E_STEP_CAP, HSAW_E_TIMEOUT. */
HSAW_API hsaw_status hsaw_solve(hsaw_graph g, const hsaw_query* q, hsaw_result* r, void* stream);

/* Spread of V_I on the residual graph G' (Eq. "sus_nod": the removed edges, or nodes,
 * deleted), by HSAW sampling: draws q->n_hsaw hits on G' (attempts from 0, q's seed and
 * suspects) and returns *spread = n hits / attempts, the unbiased estimate of I_G'(V_I)
 * (Thm. "rr_edge" with T = E), and *std_err = n sqrt(f (1 - f) / attempts), f = hits /
 * attempts.  removed: edge ids (q->mode == HSAW_EDGE) or node ids (HSAW_NODE), host
 * array, may be NULL when n_removed == 0.  D_hat(T) = spread(no removal) - spread(T). */
HSAW_API hsaw_status hsaw_estimate_spread(hsaw_graph g, const hsaw_query* q, const int64_t* removed,
                                          int32_t n_removed, double* spread, double* std_err, void* stream);

/* Test hook (fault injection on the host): the n-th device allocation made by the library
 * from now on fails as if the device were out of memory (n >= 1); n <= 0 disables.  The
 * failing call returns HSAW_E_NOMEM and leaves the library usable. */
HSAW_API hsaw_status hsaw_debug_fail_alloc_after(int64_t n);

/* ------------------------------------------------------------------ batched and served solves
 * Not in the paper: many interdiction instances at once (batching) and a request loop
 * (serving).  Every instance runs exactly the hsaw_solve computation on its own CUDA
 * stream, so each result is bit-identical to the instance solved alone.
 *
 * hsaw_solve_batch: solve count instances (gs[i], qs[i]) -> rs[i] (caller buffers as in
 *   hsaw_solve), statuses[i] (may be NULL) the status of each.  `concurrency` worker
 *   threads (<= 0: 8), each with its own non-blocking stream, take the instances in index
 *   order; `stream` is synchronised first.  Returns HSAW_OK when every instance
 *   succeeded, else the first failing status (the other results stay valid).
 *
 * Server (continuous batching): hsaw_server_create keeps the graphs (not owned: they
 *   must outlive the server) and starts `workers` threads (<= 0: 8).  mem_budget (bytes,
 *   0 = 3/4 of the free device memory at creation) bounds the summed device-memory
 *   estimates of the queries on the GPU.  hsaw_server_submit copies the query's host
 *   arrays and returns a ticket; a query whose estimate alone exceeds the budget is
 *   refused with HSAW_E_REJECTED.  Queries start in submission order as soon as a worker
 *   is free and the budget has room, while earlier ones are still running.
 *   hsaw_server_poll waits up to timeout_ms (< 0: forever) for the ticket: HSAW_E_PENDING
 *   if still running (the ticket stays valid), else the query's own status, with r
 *   filled as by hsaw_solve and *latency_ms (may be NULL) = completion - submission;
 *   the ticket is then released.  hsaw_server_cancel: a queued query never starts, a
 *   running one stops at its next sampler launch or stopping-rule round; its poll
 *   returns HSAW_E_CANCELLED.  hsaw_server_destroy cancels what is left, joins the
 *   workers and frees the server. */
typedef struct hsaw_server_s* hsaw_server;
HSAW_API hsaw_status hsaw_solve_batch(const hsaw_graph* gs, const hsaw_query* qs, hsaw_result* rs,
                                      hsaw_status* statuses, int32_t count, int32_t concurrency, void* stream);
HSAW_API hsaw_status hsaw_server_create(const hsaw_graph* gs, int32_t n_graphs, size_t mem_budget, int32_t workers,
                                        hsaw_server* out);
HSAW_API hsaw_status hsaw_server_submit(hsaw_server s, int32_t graph_idx, const hsaw_query* q, uint64_t* ticket);
HSAW_API hsaw_status hsaw_server_poll(hsaw_server s, uint64_t ticket, hsaw_result* r, int32_t timeout_ms,
                                      double* latency_ms);
HSAW_API hsaw_status hsaw_server_cancel(hsaw_server s, uint64_t ticket);
HSAW_API hsaw_status hsaw_server_destroy(hsaw_server s);

/* ------------------------------------------------------------------ the stream R (Alg. 3)
 * hsaw_sample: draw the first n_hits HSAWs of the query's stream, attempts
 *   first_attempt, first_attempt + 1, ... (only sources, p_fixed, seed and max_attempts
 *   of q are used).  Walk j is stored with its attempt id, its nodes v_1..v_l (v_1 the
 *   start, v_l the source hit) and its l - 1 edge ids; the handle keeps them on the
 *   device.  Optional removed sets (device or host byte masks, NULL = none) describe the
 *   residual graph G' of Eq. "sus_nod": removed edges are never live, removed nodes are
 *   neither infected nor sources.  removed_flags & HSAW_INPUT_DEVICE: masks on device.
 * hsaw_walks_info: count, total nodes, attempts examined, steps executed.
 * hsaw_walks_export: copy to host arrays (any NULL): aid uint64[count],
 *   node_off int64[count+1] (walk j has nodes node_off[j]..node_off[j+1]-1 and edges
 *   node_off[j]-j .. node_off[j+1]-j-2), nodes int32[total], edges int32[total-count]. */
HSAW_API hsaw_status hsaw_sample(hsaw_graph g, const hsaw_query* q, uint64_t first_attempt, int64_t n_hits,
                        const uint8_t* edge_removed, const uint8_t* node_removed, uint32_t removed_flags,
                        hsaw_walks* out, void* stream);
HSAW_API hsaw_status hsaw_walks_info(hsaw_walks w, int64_t* count, int64_t* total_nodes, uint64_t* attempts,
                            uint64_t* steps);
HSAW_API hsaw_status hsaw_walks_export(hsaw_walks w, uint64_t* aid, int64_t* node_off, int32_t* nodes, int32_t* edges,
                              void* stream);
/* The same arrays copied on the device, stream-ordered, into caller-owned device buffers of
 * the walks' device (any NULL; sizes as for hsaw_walks_export).  Synchronises `stream`. */
HSAW_API hsaw_status hsaw_walks_export_device(hsaw_walks w, uint64_t* aid_dev, int64_t* node_off_dev,
                                              int32_t* nodes_dev, int32_t* edges_dev, void* stream);
HSAW_API hsaw_status hsaw_walks_destroy(hsaw_walks w);

/* Per-attempt outcome of attempts [first, first + count) (device buffers from the caller):
 * outcome int8 (0 no live edge, 1 hit, 2 cycle, 3 removed element), length int32 (nodes
 * walked; for cycles the nodes walked until the cycle was detected).  Used to check the
 * stream attempt by attempt at full size. */
HSAW_API hsaw_status hsaw_classify(hsaw_graph g, const hsaw_query* q, uint64_t first, int64_t count,
                          int8_t* outcome_dev, int32_t* length_dev, void* stream);

/* ------------------------------------------------------------------ allocation-free sampling
 * The paper has no counterpart to this call.  It is for callers that must not allocate
 * device memory once they are running: a host framework that owns every device
 * allocation through its own pool and forbids others (a second allocator would fragment
 * or exceed the budget it plans for), and latency-bound loops in which cudaMalloc and
 * cudaFree are ruled out because they can synchronise the whole device and stall the
 * other streams.  Such a caller passes its own input and output buffers; the scratch the
 * sampler needs lives in the library itself.
 *
 * hsaw_sample_hits_static: the hits among attempts [first_attempt, first_attempt +
 *   n_attempts) of graph g, in increasing attempt id: aid_out[i] (device, uint64) and
 *   len_out[i] (device, uint32, nodes on the walk), *n_hits (host) = their number.  The
 *   same hits, in the same order, as hsaw_sample over that range with p == 1 and no
 *   removed elements.  suspect_bits: device array of ceil(n/32) words, bit v set iff v is
 *   a source.  The call makes no device allocation: its scratch (about 2 MiB) is a
 *   static array of the library that every GPU loading the library keeps until exit.
 *   Errors: HSAW_E_INVALID for n_attempts outside [0, HSAW_STATIC_MAX_ATTEMPTS], NULL
 *   arguments, or more hits than out_cap (then *n_hits is set and nothing is written).
 *   HSAW_E_DEVICE when the current CUDA device is not the graph's device.
 *   The first call on a device looks up the scratch's device address (set-up); make it
 *   before any stream capture.  Every call shares the one scratch array, which keeps the
 *   last call's contents (the call clears what must start at zero): calls that overlap
 *   on the GPU (other threads or streams) race and must be serialised by the caller.
 *   The call synchronises `stream` (it reads the hit count back to the host) before it
 *   returns. */
#define HSAW_STATIC_MAX_ATTEMPTS (1u << 18)
HSAW_API hsaw_status hsaw_sample_hits_static(hsaw_graph g, const uint32_t* suspect_bits, uint64_t seed,
                                             uint64_t first_attempt, int64_t n_attempts, uint64_t* aid_out,
                                             uint32_t* len_out, int64_t out_cap, int64_t* n_hits, void* stream);

/* ------------------------------------------------------------------ counting and greedy
 * Over walks [first, first + count) of a stream, in mode (edges: R_j = the walk's edges;
 * nodes: R_j = all of v_1..v_l, start and hit source included).
 * hsaw_histogram: the touched elements in increasing id with their occurrence counts
 *   (notation table: Cov_R({x}) for each x).  uid and cnt are host buffers of capacity
 *   cap; *n_unique receives U (HSAW_E_INVALID if U > cap, with *n_unique still set).
 * hsaw_greedy: Alg. 4 / Alg. 7 with the tie and zero-gain rules of hsaw_solve.
 *   candidate_mask as in hsaw_query; ids int64[k], gains uint32[k] host buffers.
 * hsaw_coverage: #walks that contain an element of T (T host int64[k]). */
HSAW_API hsaw_status hsaw_histogram(hsaw_walks w, hsaw_mode mode, int64_t first, int64_t count, int32_t* uid,
                           uint32_t* cnt, int64_t cap, int64_t* n_unique, void* stream);
HSAW_API hsaw_status hsaw_greedy(hsaw_walks w, hsaw_graph g, hsaw_mode mode, int64_t first, int64_t count,
                        const uint8_t* candidate_mask, int32_t k, int64_t* ids, uint32_t* gains, void* stream);
HSAW_API hsaw_status hsaw_coverage(hsaw_walks w, hsaw_mode mode, int64_t first, int64_t count, const int64_t* T,
                          int32_t k, uint64_t* cov, void* stream);

/* ------------------------------------------------------------------ stopping rule (host FP64)
 * Sec. 5.1: out6 = {ln C(M,k), N_max (Eq. "guard"/"nguard"), Upsilon, t_max, Lambda
 * (Eq. "lambda"), Lambda_1 (Eq. "lambda_1")}; t_max per Lemma "tmax".
 * hsaw_check: Alg. 5; returns 1 when eps_t <= eps, 0 otherwise; *eps_t = NaN when
 * cp < Lambda_1. */
HSAW_API hsaw_status hsaw_stop_constants(int64_t M, int32_t k, double eps, double delta, double* out6);
HSAW_API int hsaw_check(double c, double cp, double size_rprime, int32_t t, double eps, double lambda1, double* eps_t);

/* ------------------------------------------------------------------ profiling
 * Counters for measurement (not part of the method).  hsaw_profile_enable(1) resets the
 * counters and starts timing every sampler launch with CUDA events recorded on the
 * launching stream; hsaw_profile_read synchronises the device and returns the totals
 * since the last reset.  kernel_launches counts every kernel the library launched. */
typedef struct {
  uint64_t kernel_launches;   /* all library kernels launched since the reset */
  uint64_t sampler_launches;  /* HSAW sampler launches (timed when enabled) */
  double sampler_ms;          /* summed device time of the timed sampler launches */
  uint64_t sampler_steps;     /* live-edge draws executed by those launches */
  uint64_t sampler_attempts;  /* attempts examined by those launches */
  double phase_ms[8];         /* device time per phase: 0 sampling (launch, compaction, re-walk),
                                 1 counting + inverted index, 2 greedy, 3 out-of-sample coverage */
} hsaw_profile;
HSAW_API hsaw_status hsaw_profile_enable(int on);
HSAW_API hsaw_status hsaw_profile_read(hsaw_profile* out);

/* Random-gather probe (measurement, not part of the method): the rate of dependent random
 * 32-byte reads the GPU sustains, the memory pattern of a walk (one dependent record read
 * per live-edge draw) without the walk's arithmetic.  Allocates a table of table_bytes
 * (rounded down to 32-byte records, at most 2^32 of them), fills it, and runs blocks of
 * 256 threads, blocks_per_sm of them per SM (<= 0 or above what fits: as many as fit,
 * at most 6), each thread following `chains` independent chains (1, 2 or 4) of `steps`
 * dependent reads; the second of two passes is timed with CUDA events on `stream`.
 * *reads_per_s = records read / time, *ms (may be NULL) = the timed pass.  Errors:
 * HSAW_E_INVALID, HSAW_E_NOMEM, HSAW_E_DEVICE. */
HSAW_API hsaw_status hsaw_probe_gather(uint64_t table_bytes, int32_t chains, uint32_t steps, int32_t blocks_per_sm,
                                       double* reads_per_s, double* ms, void* stream);

/* ------------------------------------------------------------------ device scratch
 * The paper has no counterpart to this call.  Scratch device memory (a solve's walk
 * streams, histograms, inverted index and greedy state; not graphs, walk pools or the
 * static sampler scratch) comes from CUDA's stream-ordered memory pool unless the caller
 * installs an allocator of its own, such as a framework's caching allocator:
 *   alloc(bytes, stream, ctx) returns device memory on the current device, aligned to at
 *     least 256 bytes, usable in stream order on `stream`, or NULL when it has none (the
 *     call in progress then fails with HSAW_E_NOMEM);
 *   release(ptr, stream, ctx) takes back a block alloc returned, in stream order on
 *     `stream`.
 * The library calls them from whichever threads run its calls (batch and server workers
 * too), possibly at the same time, so they must be thread-safe.  The allocator is
 * process-wide; alloc = release = NULL restores the pool.  Call this while no other
 * library call is in progress.  Errors: HSAW_E_INVALID if exactly one of alloc and
 * release is NULL, or while the library still holds scratch blocks of the current
 * allocator (a live hsaw_walks handle, a server), since each block must go back where it
 * came from. */
typedef void* (*hsaw_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*hsaw_free_fn)(void* ptr, void* stream, void* ctx);
HSAW_API hsaw_status hsaw_set_allocator(hsaw_alloc_fn alloc, hsaw_free_fn release, void* ctx);

/* ------------------------------------------------------------------ diagnostics */
HSAW_API const char* hsaw_last_error(void); /* thread-local message of the last failing call */
HSAW_API const char* hsaw_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HSAW_H_ */
