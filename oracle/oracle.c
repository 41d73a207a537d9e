/*
 * CPU ORACLE for HSAW-based Spread Interdiction under the LT model
 * ("Blocking Self-avoiding Walks Stops Cyber-epidemics", Sec. 2-5, Alg. 1, 4-9).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct statement
 * of what the GPU path computes.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product library never calls it.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Every function cites the passage it follows.  The readings taken where the paper is
 * silent or garbled are marked "Reading:" and listed again in the design notes.
 *
 * Pins (what checks this file against something other than itself; see tests/):
 *   philox      - published known-answer vectors of Philox4x32-10.
 *   graph_build - invariants (stable order, exact prefix sums) and brute-force selection
 *                 frequencies on tiny graphs.
 *   walk/stream - brute-force enumeration of live-edge worlds on <=12-node graphs
 *                 (spread with and without a removed set, within 4 standard errors);
 *                 per-walk frequency against Eq. "compute_path_inf"; closed forms
 *                 (chains, single edges, cycles); self-avoidance / hitting invariants.
 *   histogram   - direct recount, sum invariant.
 *   greedy      - brute-force optimal max-coverage on tiny inputs (1-1/e bound),
 *                 exact optimum for k=1, tie and zero-gain rules on hand-built cases.
 *   stop rule   - log-binomial against exact integer binomials; the t_max definition
 *                 as a doubling bound; Check's monotonicity and special cases; the
 *                 epsilon_t expression against hand-evaluated cases (t = 1, 3, 5) and
 *                 against the closed-form coverage at which Check starts to pass.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* =====================================================================================
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC'11).  Replaces the paper's linear-recurrence PRG (Sec. 4.2.1): a draw is
 * a pure function of (key, counter), so a walk is re-derivable from its attempt id -
 * the paper's <Seed_h, Len_h> path encoding with the attempt id as the seed.
 * ===================================================================================== */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The draws of attempt a.  An attempt is one live-edge world (Sec. 2.1): every node v
 * gets ONE draw, keyed by (attempt, node), and keeps it however often a walk looks at it.
 *   node draw  : key = (lo32 seed, hi32 seed), counter = (lo32 a, hi32 a, v, 0);
 *                x0 chooses v's live in-edge, x1 is v's source coin.
 *   start draw : counter = (lo32 a, hi32 a, 0, 1); x0 chooses the start node.
 * Reading: the paper draws from a sequential generator (Sec. 4.2.1, Eq. "rand"); keying
 * the draws by node keeps the path encoding (a walk is re-derived from its attempt id)
 * and makes a revisited node repeat its choice, so a walk that closes a cycle is exactly
 * a world in which the start node's backward chain never meets a source. */
static void draw_node(uint64_t seed, uint64_t a, int32_t v, uint32_t x[4]) {
  uint32_t ctr[4] = {(uint32_t)a, (uint32_t)(a >> 32), (uint32_t)v, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  oracle_philox4x32_10(ctr, key, x);
}
static void draw_start(uint64_t seed, uint64_t a, uint32_t x[4]) {
  uint32_t ctr[4] = {(uint32_t)a, (uint32_t)(a >> 32), 0u, 1u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  oracle_philox4x32_10(ctr, key, x);
}

/* =====================================================================================
 * Graph (Sec. 2.1): directed G = (V, E, w), in-weight sum <= 1 per node.
 * Stored as in-adjacency by destination; edge id = position after a STABLE sort by
 * destination (input order kept within a node).  Weights are uint32 fixed point
 * (w = w_fixed / 2^32) and thr[j] is the running sum of the node's in-weights up to and
 * including in-edge j, so in-edge j of v is live for a draw r (uniform on [0, 2^32))
 * iff thr[j-1] <= r < thr[j]: probability exactly w_fixed[j] / 2^32 (live-edge model,
 * Sec. 2.1).  A node whose in-sum exceeds 2^32 - 1 is rejected.
 * ===================================================================================== */
typedef struct {
  int64_t n, m;
  int64_t* row_ptr;     /* n+1 */
  int32_t* src;         /* m, CSR order */
  int32_t* dst;         /* m, CSR order */
  uint32_t* w;          /* m */
  uint32_t* thr;        /* m */
  int64_t* input_index; /* m: CSR position -> input edge index */
} oracle_graph;

void oracle_graph_free(oracle_graph* g) {
  if (!g) return;
  free(g->row_ptr); free(g->src); free(g->dst); free(g->w); free(g->thr); free(g->input_index);
  free(g);
}

/* returns 0, -1 invalid sizes, -2 weight sum, -3 index out of range, -4 no memory */
int oracle_graph_build(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                       const uint32_t* w, oracle_graph** out) {
  *out = NULL;
  if (n < 1 || m < 0) return -1;
  for (int64_t e = 0; e < m; ++e)
    if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return -3;
  oracle_graph* g = (oracle_graph*)calloc(1, sizeof(oracle_graph));
  if (!g) return -4;
  g->n = n; g->m = m;
  g->row_ptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  g->src = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
  g->dst = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
  g->w = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
  g->thr = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
  g->input_index = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m ? m : 1));
  if (!g->row_ptr || !g->src || !g->dst || !g->w || !g->thr || !g->input_index) {
    oracle_graph_free(g);
    return -4;
  }
  /* counting sort by destination, stable */
  for (int64_t e = 0; e < m; ++e) g->row_ptr[dst[e] + 1]++;
  for (int64_t v = 0; v < n; ++v) g->row_ptr[v + 1] += g->row_ptr[v];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!fill) { oracle_graph_free(g); return -4; }
  for (int64_t v = 0; v < n; ++v) fill[v] = g->row_ptr[v];
  for (int64_t e = 0; e < m; ++e) {
    int64_t pos = fill[dst[e]]++;
    g->src[pos] = src[e];
    g->dst[pos] = dst[e];
    g->w[pos] = w[e];
    g->input_index[pos] = e;
  }
  free(fill);
  /* cumulative thresholds, exact in 64-bit */
  for (int64_t v = 0; v < n; ++v) {
    uint64_t acc = 0;
    for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j) {
      acc += g->w[j];
      if (acc > 0xFFFFFFFFull) { oracle_graph_free(g); return -2; }
      g->thr[j] = (uint32_t)acc;
    }
  }
  *out = g;
  return 0;
}

int64_t oracle_graph_n(const oracle_graph* g) { return g->n; }
int64_t oracle_graph_m(const oracle_graph* g) { return g->m; }
void oracle_graph_export(const oracle_graph* g, int64_t* row_ptr, int32_t* src, int32_t* dst, uint32_t* thr,
                         int64_t* input_index) {
  if (row_ptr) memcpy(row_ptr, g->row_ptr, sizeof(int64_t) * (size_t)(g->n + 1));
  if (src) memcpy(src, g->src, sizeof(int32_t) * (size_t)g->m);
  if (dst) memcpy(dst, g->dst, sizeof(int32_t) * (size_t)g->m);
  if (thr) memcpy(thr, g->thr, sizeof(uint32_t) * (size_t)g->m);
  if (input_index) memcpy(input_index, g->input_index, sizeof(int64_t) * (size_t)g->m);
}

/* =====================================================================================
 * Query context: suspects V_I with p(v) (Sec. 2.2, Eq. "prob_src_set"), optional removed
 * edges / nodes (the residual graph G' of Eq. "sus_nod").
 * Reading: p is uint32 fixed point; a suspect u is a real source for this walk iff the
 * coin x1 < p32(u), except p32 = 0xFFFFFFFF which means certain.
 * ===================================================================================== */
typedef struct {
  const oracle_graph* g;
  uint8_t* is_suspect;        /* n */
  uint32_t* p32;              /* n, or NULL when p == 1 for every suspect */
  const uint8_t* edge_removed; /* m (CSR order) or NULL */
  const uint8_t* node_removed; /* n or NULL */
  uint64_t seed;
} oracle_ctx;

/* Source coin with probability p32 / 2^32: x1 < p32, and p32 = 0xFFFFFFFF is certain. */
int oracle_source_coin(uint32_t x1, uint32_t p32) {
  if (p32 == 0xFFFFFFFFu) return 1;
  return x1 < p32;
}

static int coin_says_source(const oracle_ctx* c, int32_t u, uint32_t x1) {
  if (!c->is_suspect[u]) return 0;
  if (!c->p32) return 1;
  return oracle_source_coin(x1, c->p32[u]);
}

/* Live in-edge of v for the draw r (Sec. 2.1 live-edge model): the first in-edge j with
 * r < thr[j], i.e. in-edge j is chosen for r in [thr[j-1], thr[j]); -1 when r is at or
 * above the node's in-sum (no live in-edge). */
int64_t oracle_select_in_edge(const oracle_graph* g, int32_t v, uint32_t r) {
  for (int64_t j = g->row_ptr[v]; j < g->row_ptr[v + 1]; ++j)
    if (r < g->thr[j]) return j;
  return -1;
}

/* Outcome codes of one attempt. */
#define ORACLE_MISS_NO_EDGE 0
#define ORACLE_HIT 1
#define ORACLE_MISS_CYCLE 2
#define ORACLE_MISS_REMOVED 3
#define ORACLE_STEP_CAP (-6)

/* One SAW attempt = one pass of the inner loop of Alg. 1 (HSAW sampling), with the
 * readings below.  nodes[] receives v_1..v_l, edges[] the CSR ids of the edges
 * (v_{i+1}, v_i) walked, *len = l.  Both buffers need room for n entries.
 *   Start: v_1 = floor(x0 * n / 2^32) of the start draw [uniform start, Alg. 1 line 2].
 *   At each node v of the walk, v's own draw decides:
 *     source test: v is a suspect and its coin x1 < p32(v) (p32 = 0xFFFFFFFF: certain)
 *       -> hit, the walk ends at v [Alg. 1 lines 10-11].
 *       Reading (Def. "self_walk" allows l = 1): this test applies to the start node
 *       too, so an infected start node is a hit of length 1.
 *     live in-edge: the first j with x0 < thr[j]; none -> miss [Alg. 1 lines 6-8].
 *   u = tail of the live edge.  u already on the walk -> miss (cycle) [Alg. 1 line 12,
 *     made exact: the whole walk is compared].  A revisited node cannot be a source
 *     (it was tested on its first visit with the same draw), so the order of the hit
 *     and cycle tests does not matter.
 *   Residual graph: a removed edge or a removed tail node means the chosen edge is not
 *     live; a removed start node cannot be infected.
 *   Guard: more than n steps -> ORACLE_STEP_CAP (unreachable for a self-avoiding walk;
 *     Alg. 2 line 9 "Len_h >= n"). */
int oracle_attempt(const oracle_ctx* c, uint64_t a, int32_t* nodes, int32_t* edges, int64_t* len) {
  const oracle_graph* g = c->g;
  uint32_t x[4];
  draw_start(c->seed, a, x);
  int32_t v = (int32_t)(((uint64_t)x[0] * (uint64_t)g->n) >> 32);
  *len = 0;
  if (c->node_removed && c->node_removed[v]) return ORACLE_MISS_REMOVED;
  nodes[0] = v;
  *len = 1;
  for (int64_t s = 1;; ++s) {
    draw_node(c->seed, a, v, x);
    if (coin_says_source(c, v, x[1])) return ORACLE_HIT;
    if (s > g->n) return ORACLE_STEP_CAP;
    int64_t chosen = oracle_select_in_edge(g, v, x[0]);
    if (chosen < 0) return ORACLE_MISS_NO_EDGE;
    int32_t u = g->src[chosen];
    if (c->edge_removed && c->edge_removed[chosen]) return ORACLE_MISS_REMOVED;
    if (c->node_removed && c->node_removed[u]) return ORACLE_MISS_REMOVED;
    for (int64_t i = 0; i < *len; ++i)
      if (nodes[i] == u) return ORACLE_MISS_CYCLE;
    nodes[*len] = u;
    edges[*len - 1] = (int32_t)chosen;
    *len += 1;
    v = u;
  }
}

/* Context construction (suspects given as a list with optional per-suspect p). */
oracle_ctx* oracle_ctx_new(const oracle_graph* g, const int32_t* sources, int64_t n_sources,
                           const uint32_t* p_fixed, const uint8_t* edge_removed,
                           const uint8_t* node_removed, uint64_t seed) {
  oracle_ctx* c = (oracle_ctx*)calloc(1, sizeof(oracle_ctx));
  if (!c) return NULL;
  c->g = g;
  c->seed = seed;
  c->is_suspect = (uint8_t*)calloc((size_t)g->n, 1);
  if (!c->is_suspect) { free(c); return NULL; }
  if (p_fixed) {
    c->p32 = (uint32_t*)calloc((size_t)g->n, sizeof(uint32_t));
    if (!c->p32) { free(c->is_suspect); free(c); return NULL; }
  }
  for (int64_t i = 0; i < n_sources; ++i) {
    c->is_suspect[sources[i]] = 1;
    if (p_fixed) c->p32[sources[i]] = p_fixed[i];
  }
  c->edge_removed = edge_removed;
  c->node_removed = node_removed;
  return c;
}

void oracle_ctx_free(oracle_ctx* c) {
  if (!c) return;
  free(c->is_suspect); free(c->p32); free(c);
}

/* =====================================================================================
 * The HSAW stream R_1, R_2, ... (Alg. 3): attempts are taken in increasing attempt id
 * a = first, first+1, ...; the hits, in that order, form the stream.  A hitting walk j
 * is stored with its attempt id, its nodes v_1..v_l and its edges.
 * ===================================================================================== */
typedef struct {
  int64_t count, cap;
  uint64_t* aid;
  int64_t* node_off;   /* count+1, into nodes; walk j has node_off[j+1]-node_off[j] nodes */
  int32_t* nodes;
  int32_t* edges;      /* walk j's edges start at node_off[j] - j, length l_j - 1 */
  int64_t node_cap;
  uint64_t attempts;   /* attempts consumed: last attempt examined + 1 - first */
  uint64_t next_aid;   /* first attempt id not yet examined */
  uint64_t steps;      /* live-edge draws made (failing final draws included) */
  int status;
} oracle_walks;

void oracle_walks_free(oracle_walks* w) {
  if (!w) return;
  free(w->aid); free(w->node_off); free(w->nodes); free(w->edges); free(w);
}

static int walks_push(oracle_walks* W, uint64_t a, const int32_t* nodes, const int32_t* edges, int64_t len) {
  if (W->count + 1 > W->cap) {
    int64_t nc = W->cap ? W->cap * 2 : 1024;
    uint64_t* na = (uint64_t*)realloc(W->aid, sizeof(uint64_t) * (size_t)nc);
    if (!na) return -4;
    W->aid = na;
    int64_t* no = (int64_t*)realloc(W->node_off, sizeof(int64_t) * (size_t)(nc + 1));
    if (!no) return -4;
    W->node_off = no;
    W->cap = nc;
  }
  int64_t base = W->node_off[W->count];
  if (base + len > W->node_cap) {
    int64_t nc = W->node_cap ? W->node_cap * 2 : 4096;
    while (nc < base + len) nc *= 2;
    int32_t* nn = (int32_t*)realloc(W->nodes, sizeof(int32_t) * (size_t)nc);
    if (!nn) return -4;
    W->nodes = nn;
    int32_t* ne = (int32_t*)realloc(W->edges, sizeof(int32_t) * (size_t)nc);
    if (!ne) return -4;
    W->edges = ne;
    W->node_cap = nc;
  }
  memcpy(W->nodes + base, nodes, sizeof(int32_t) * (size_t)len);
  if (len > 1) memcpy(W->edges + (base - W->count), edges, sizeof(int32_t) * (size_t)(len - 1));
  W->aid[W->count] = a;
  W->node_off[W->count + 1] = base + len;
  W->count++;
  return 0;
}

oracle_walks* oracle_walks_new(uint64_t first_aid) {
  oracle_walks* W = (oracle_walks*)calloc(1, sizeof(oracle_walks));
  if (!W) return NULL;
  W->node_off = (int64_t*)calloc(1, sizeof(int64_t));
  W->next_aid = first_aid;
  return W;
}

/* Extend the stream until it holds `want_hits` walks or `max_attempts` more attempts
 * were examined.  Returns 0, or a negative status. */
int oracle_stream_extend(const oracle_ctx* c, oracle_walks* W, int64_t want_hits, uint64_t max_attempts) {
  int64_t n = c->g->n;
  int32_t* nodes = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int32_t* edges = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  if (!nodes || !edges) { free(nodes); free(edges); return -4; }
  uint64_t done = 0;
  int rc = 0;
  while (W->count < want_hits && done < max_attempts) {
    uint64_t a = W->next_aid++;
    int64_t len = 0;
    int r = oracle_attempt(c, a, nodes, edges, &len);
    done++;
    W->attempts++;
    W->steps += (len > 0 ? (uint64_t)len : 0);  /* one draw per node left, incl. the final one */
    if (r == ORACLE_HIT) W->steps -= 1;           /* a hit's last node needed no further draw */
    if (r == ORACLE_STEP_CAP) { rc = ORACLE_STEP_CAP; break; }
    if (r == ORACLE_HIT) {
      rc = walks_push(W, a, nodes, edges, len);
      if (rc) break;
    }
  }
  free(nodes); free(edges);
  W->status = rc;
  return rc;
}

/* Append to W the walks of `part`, a stream that starts at W's next attempt id (the same
 * query examined over a later, disjoint attempt range), keeping at most `limit` of them
 * (limit < 0: all).  When `part` holds at least `limit` walks, W ends after the attempt of
 * its limit-th walk, exactly as if W had been extended attempt by attempt to that many walks.  Lets a
 * caller examine consecutive attempt ranges independently (Alg. 3's attempts are
 * independent) and join them in attempt order.  Returns 0, -1 (part does not start at
 * W's next attempt) or -4 (out of memory). */
int oracle_walks_append(oracle_walks* W, const oracle_walks* part, uint64_t part_first, int64_t limit) {
  if (part_first != W->next_aid) return -1;
  const int cut = limit >= 0 && part->count >= limit;
  const int64_t take = cut ? limit : part->count;
  for (int64_t j = 0; j < take; ++j) {
    int64_t b = part->node_off[j], e = part->node_off[j + 1];
    int rc = walks_push(W, part->aid[j], part->nodes + b, part->edges + (b - j), e - b);
    if (rc) return rc;
  }
  uint64_t next = part->next_aid;
  if (cut) next = take > 0 ? part->aid[take - 1] + 1 : part_first;
  else W->steps += part->steps; /* draws are known only for a part appended whole */
  W->attempts += next - W->next_aid;
  W->next_aid = next;
  return 0;
}

/* Classify the attempts [first, first+count) one by one: writes the outcome code of each
 * attempt and the length of each walk (sampled-parity checks at full size). */
void oracle_classify(const oracle_ctx* c, uint64_t first, int64_t count, int8_t* outcome, int32_t* length) {
  int64_t n = c->g->n;
  int32_t* nodes = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int32_t* edges = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  for (int64_t i = 0; i < count; ++i) {
    int64_t len = 0;
    int r = oracle_attempt(c, first + (uint64_t)i, nodes, edges, &len);
    outcome[i] = (int8_t)r;
    length[i] = (int32_t)len;
  }
  free(nodes); free(edges);
}

int64_t oracle_walks_count(const oracle_walks* W) { return W->count; }
int64_t oracle_walks_nodes_total(const oracle_walks* W) { return W->node_off[W->count]; }
uint64_t oracle_walks_attempts(const oracle_walks* W) { return W->attempts; }
uint64_t oracle_walks_steps(const oracle_walks* W) { return W->steps; }
void oracle_walks_export(const oracle_walks* W, uint64_t* aid, int64_t* node_off, int32_t* nodes, int32_t* edges) {
  if (aid) memcpy(aid, W->aid, sizeof(uint64_t) * (size_t)W->count);
  if (node_off) memcpy(node_off, W->node_off, sizeof(int64_t) * (size_t)(W->count + 1));
  int64_t tot = W->node_off[W->count];
  if (nodes) memcpy(nodes, W->nodes, sizeof(int32_t) * (size_t)tot);
  if (edges) memcpy(edges, W->edges, sizeof(int32_t) * (size_t)(tot - W->count));
}

/* Element sets R_j (Alg. 3 line 9 for edges; Alg. 9 line 2 for nodes).
 * Reading: the node sample R_j is every node v_1..v_l of the walk, start and hit source
 * included (removing any of them stops the infection of v_1, Thm. "rr_node"). */
#define MODE_EDGE 0
#define MODE_NODE 1
static const int32_t* walk_elems(const oracle_walks* W, int mode, int64_t j, int64_t* cnt) {
  int64_t b = W->node_off[j], e = W->node_off[j + 1];
  if (mode == MODE_NODE) { *cnt = e - b; return W->nodes + b; }
  *cnt = e - b - 1;
  return W->edges + (b - j);
}

/* =====================================================================================
 * Coverage counts (notation table: Cov_R(T) = #samples intersecting T).
 * Histogram: cnt[x] = #walks j in [first, first+count) with x in R_j.
 * ===================================================================================== */
void oracle_histogram(const oracle_walks* W, int mode, int64_t first, int64_t count, int64_t M, uint32_t* cnt) {
  memset(cnt, 0, sizeof(uint32_t) * (size_t)M);
  for (int64_t j = first; j < first + count; ++j) {
    int64_t l;
    const int32_t* x = walk_elems(W, mode, j, &l);
    for (int64_t i = 0; i < l; ++i) cnt[x[i]]++;
  }
}

/* Cov of the set T (k ids) over walks [first, first+count). */
int64_t oracle_coverage(const oracle_walks* W, int mode, int64_t first, int64_t count, int64_t M,
                        const int64_t* T, int32_t k) {
  uint8_t* inT = (uint8_t*)calloc((size_t)M, 1);
  for (int32_t i = 0; i < k; ++i) inT[T[i]] = 1;
  int64_t cov = 0;
  for (int64_t j = first; j < first + count; ++j) {
    int64_t l;
    const int32_t* x = walk_elems(W, mode, j, &l);
    for (int64_t i = 0; i < l; ++i)
      if (inT[x[i]]) { cov++; break; }
  }
  free(inT);
  return cov;
}

/* =====================================================================================
 * Greedy max-coverage (Alg. 4 for edges, Alg. 7 for nodes).  Round i picks the candidate
 * outside T with the largest marginal coverage over the not-yet-covered walks.
 * Reading: ties go to the smallest id; when every remaining gain is 0 the smallest-id
 * unpicked candidate is still taken, so exactly k ids come back (|T_k| = k in Defs.
 * "edge_remove" / "node_remove").  The gain of each pick is reported.
 * Plain form: marginal gains are recounted from scratch every round.
 * ===================================================================================== */
int oracle_greedy(const oracle_walks* W, int mode, int64_t first, int64_t count, int64_t M,
                  const uint8_t* cand_mask, int32_t k, int64_t* ids, uint32_t* gains) {
  uint8_t* covered = (uint8_t*)calloc((size_t)(count ? count : 1), 1);
  uint8_t* picked = (uint8_t*)calloc((size_t)M, 1);
  uint32_t* gain = (uint32_t*)calloc((size_t)M, sizeof(uint32_t));
  int64_t* touched = (int64_t*)malloc(sizeof(int64_t) * (size_t)(M ? M : 1));
  if (!covered || !picked || !gain || !touched) {
    free(covered); free(picked); free(gain); free(touched);
    return -4;
  }
  int64_t n_cand = 0;
  for (int64_t x = 0; x < M; ++x) n_cand += (!cand_mask || cand_mask[x]) ? 1 : 0;
  if (k < 1 || k > n_cand) { free(covered); free(picked); free(gain); free(touched); return -1; }
  for (int32_t round = 0; round < k; ++round) {
    /* recount marginal gains over uncovered walks */
    int64_t nt = 0;
    for (int64_t j = 0; j < count; ++j) {
      if (covered[j]) continue;
      int64_t l;
      const int32_t* x = walk_elems(W, mode, first + j, &l);
      for (int64_t i = 0; i < l; ++i) {
        if (gain[x[i]] == 0) touched[nt++] = x[i];
        gain[x[i]]++;
      }
    }
    int64_t best = -1;
    uint32_t best_gain = 0;
    for (int64_t t = 0; t < nt; ++t) {
      int64_t x = touched[t];
      if (picked[x] || (cand_mask && !cand_mask[x])) continue;
      if (gain[x] > best_gain || (gain[x] == best_gain && best_gain > 0 && x < best)) {
        best = x; best_gain = gain[x];
      }
    }
    for (int64_t t = 0; t < nt; ++t) gain[touched[t]] = 0;
    if (best < 0) { /* every remaining gain is zero: smallest unpicked candidate */
      for (int64_t x = 0; x < M; ++x)
        if (!picked[x] && (!cand_mask || cand_mask[x])) { best = x; break; }
      best_gain = 0;
    }
    ids[round] = best;
    gains[round] = best_gain;
    picked[best] = 1;
    for (int64_t j = 0; j < count; ++j) {
      if (covered[j]) continue;
      int64_t l;
      const int32_t* x = walk_elems(W, mode, first + j, &l);
      for (int64_t i = 0; i < l; ++i)
        if (x[i] == best) { covered[j] = 1; break; }
    }
  }
  free(covered); free(picked); free(gain); free(touched);
  return 0;
}

/* =====================================================================================
 * The same greedy (Alg. 4 / Alg. 7, same tie and zero-gain rules), with the marginal
 * gains kept instead of recounted: gain[x] = number of not-yet-covered walks that contain
 * x.  It starts as the occurrence count, and when a pick covers walk j, every element of
 * R_j loses that walk, so its gain drops by one.  Each round is a scan of the touched
 * elements in increasing id (strict > keeps the smallest id on ties).  For streams too
 * large for the recounting form; it must return exactly what oracle_greedy returns.
 * ===================================================================================== */
int oracle_greedy_lists(const oracle_walks* W, int mode, int64_t first, int64_t count, int64_t M,
                        const uint8_t* cand_mask, int32_t k, int64_t* ids, uint32_t* gains) {
  int64_t n_cand = 0;
  for (int64_t x = 0; x < M; ++x) n_cand += (!cand_mask || cand_mask[x]) ? 1 : 0;
  if (k < 1 || k > n_cand) return -1;
  /* walks of each element (counting sort by element id) */
  int64_t* off = (int64_t*)calloc((size_t)M + 1, sizeof(int64_t));
  uint8_t* picked = (uint8_t*)calloc((size_t)(M ? M : 1), 1);
  uint8_t* covered = (uint8_t*)calloc((size_t)(count ? count : 1), 1);
  if (!off || !picked || !covered) { free(off); free(picked); free(covered); return -4; }
  int64_t total = 0;
  for (int64_t j = 0; j < count; ++j) {
    int64_t l;
    const int32_t* x = walk_elems(W, mode, first + j, &l);
    for (int64_t i = 0; i < l; ++i) off[x[i] + 1]++;
    total += l;
  }
  /* the touched elements in increasing id: element tid[t] has gain tgain[t] and is still
     available (a candidate, not picked) iff tavail[t]; rank[x] = t */
  int64_t nt = 0;
  for (int64_t x = 0; x < M; ++x) nt += off[x + 1] ? 1 : 0;
  int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(total ? total : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(M ? M : 1));
  int64_t* rank = (int64_t*)malloc(sizeof(int64_t) * (size_t)(M ? M : 1));
  int64_t* tid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nt ? nt : 1));
  uint32_t* tgain = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(nt ? nt : 1));
  uint8_t* tavail = (uint8_t*)malloc((size_t)(nt ? nt : 1));
  if (!list || !fill || !rank || !tid || !tgain || !tavail) {
    free(off); free(picked); free(covered); free(list); free(fill); free(rank); free(tid); free(tgain); free(tavail);
    return -4;
  }
  int64_t t = 0;
  for (int64_t x = 0; x < M; ++x) {
    const int64_t c = off[x + 1];
    if (c) {
      tid[t] = x;
      tgain[t] = (uint32_t)c;
      tavail[t] = (!cand_mask || cand_mask[x]) ? 1 : 0;
      rank[x] = t++;
    }
  }
  for (int64_t x = 0; x < M; ++x) off[x + 1] += off[x];
  for (int64_t x = 0; x < M; ++x) fill[x] = off[x];
  for (int64_t j = 0; j < count; ++j) {
    int64_t l;
    const int32_t* x = walk_elems(W, mode, first + j, &l);
    for (int64_t i = 0; i < l; ++i) list[fill[x[i]]++] = j;
  }
  for (int32_t round = 0; round < k; ++round) {
    int64_t best_t = -1;
    uint32_t best_gain = 0;
    for (int64_t u = 0; u < nt; ++u)
      if (tavail[u] && tgain[u] > best_gain) { best_t = u; best_gain = tgain[u]; }
    int64_t best;
    if (best_t < 0) { /* every remaining gain is zero: smallest unpicked candidate */
      best = -1;
      for (int64_t x = 0; x < M; ++x)
        if (!picked[x] && (!cand_mask || cand_mask[x])) { best = x; break; }
      best_gain = 0;
    } else {
      best = tid[best_t];
    }
    ids[round] = best;
    gains[round] = best_gain;
    picked[best] = 1;
    if (off[best + 1] > off[best]) tavail[rank[best]] = 0;
    for (int64_t q = off[best]; q < off[best + 1]; ++q) {
      int64_t j = list[q];
      if (covered[j]) continue;
      covered[j] = 1;
      int64_t l;
      const int32_t* x = walk_elems(W, mode, first + j, &l);
      for (int64_t i = 0; i < l; ++i) tgain[rank[x[i]]]--;
    }
  }
  free(off); free(picked); free(covered); free(list); free(fill); free(rank); free(tid); free(tgain); free(tavail);
  return 0;
}

/* =====================================================================================
 * Stop-and-Stare constants (Sec. 5.1, Eqs. "guard", "nguard", "lambda", "lambda_1").
 *   M = m (eSI) or n (nSI); lnC(M,k) = log binomial(M, k).
 *   N_max  = (2 - 1/e)^2 (2 + 2eps/3) M (ln(6/delta) + lnC(M,k)) / (k eps^2)
 *   Reading (the printed t_max has ln(delta/3) < 0; Lemma "tmax" derives it):
 *   Upsilon = (2 + 2eps/3) ln(3/delta) / eps^2,  t_max = ceil(log2(2 N_max / Upsilon))
 *   Lambda  = (2 + 2eps/3) ln(3 t_max / delta) / eps^2,  Lambda_1 = 1 + (1+eps) Lambda
 *   Reading: Lambda 2^(t-1) is not an integer; L = ceil(Lambda) samples per unit.
 * ===================================================================================== */
static double log_binomial(double M, double k) {
  return lgamma(M + 1.0) - lgamma(k + 1.0) - lgamma(M - k + 1.0);
}

void oracle_stop_constants(int64_t M, int32_t k, double eps, double delta, double* out6) {
  double lnC = log_binomial((double)M, (double)k);
  double c = 2.0 + 2.0 * eps / 3.0;
  double e1 = 2.0 - exp(-1.0);
  double nmax = e1 * e1 * c * (double)M * (log(6.0 / delta) + lnC) / ((double)k * eps * eps);
  double ups = c * log(3.0 / delta) / (eps * eps);
  double tmax = ceil(log2(2.0 * nmax / ups));
  if (tmax < 1.0) tmax = 1.0;
  double lam = c * log(3.0 * tmax / delta) / (eps * eps);
  double lam1 = 1.0 + (1.0 + eps) * lam;
  out6[0] = lnC; out6[1] = nmax; out6[2] = ups; out6[3] = tmax; out6[4] = lam; out6[5] = lam1;
}

/* Check (Alg. 5 / Alg. 8).  c = Cov_{R_t}(T), cp = Cov_{R'_t}(T), size_rp = |R'_t|.
 * Returns 1 when the candidate meets eps; *eps_t receives the bound, or NaN when the
 * coverage condition cp >= Lambda_1 fails and no bound is computed. */
int oracle_check(double c, double cp, double size_rp, int t, double eps, double lambda1, double* eps_t) {
  *eps_t = NAN;
  if (!(cp >= lambda1)) return 0;
  double scale = ldexp(1.0, t - 1);
  double e1 = c / cp - 1.0;
  double e2 = eps * sqrt(size_rp * (1.0 + eps) / (scale * cp));
  double gap = 1.0 - exp(-1.0) - eps;
  double e3 = eps * sqrt(size_rp * (1.0 + eps) * gap / ((1.0 + eps / 3.0) * scale * cp));
  double et = (e1 + e2 + e1 * e2) * gap + (1.0 - exp(-1.0)) * e3;
  *eps_t = et;
  return et <= eps;
}

/* =====================================================================================
 * Full solve: Alg. 6 (eSIA) / Alg. 9 (nSIA) with the stopping rule, or a fixed number of
 * samples N.  Estimates (Thms. "rr_edge" / "rr_node" with a uniform start node):
 *   I_hat = n * hits / attempts,  D_hat = n * Cov(T) / attempts.
 * Reading: attempts = every attempt up to and including the one that gave the last hit
 *   used; the reported reduction uses all samples drawn (R_t and R'_t).
 * Reading (loop order, Alg. 6 lines 3-9): Check first, then the guard |R_t| >= N_max,
 *   with t = t_max as an extra guard.
 * ===================================================================================== */
typedef struct {
  int32_t n_selected, rounds_t;
  uint64_t hits, attempts, steps, cov_R, cov_Rprime, hits_Rprime, attempts_Rprime;
  double spread_base_est, spread_reduction_est, eps_t;
  int32_t status;
} oracle_result;

int oracle_solve(const oracle_ctx* c, int mode, const uint8_t* cand_mask, int32_t k, int stop_rule,
                 int64_t n_hsaw, double eps, double delta, uint64_t max_attempts,
                 int64_t* ids, uint32_t* gains, oracle_result* res) {
  const oracle_graph* g = c->g;
  int64_t M = (mode == MODE_EDGE) ? g->m : g->n;
  memset(res, 0, sizeof(*res));
  res->eps_t = NAN;
  oracle_walks* W = oracle_walks_new(0);
  if (!W) return -4;
  int rc = 0;
  double n = (double)g->n;
  if (!stop_rule) {
    rc = oracle_stream_extend(c, W, n_hsaw, max_attempts);
    if (rc == 0 && W->count < n_hsaw) rc = -7;
    if (rc == 0) rc = oracle_greedy(W, mode, 0, n_hsaw, M, cand_mask, k, ids, gains);
    if (rc == 0) {
      uint64_t cov = 0;
      for (int32_t i = 0; i < k; ++i) cov += gains[i];
      res->n_selected = k;
      res->rounds_t = 0;
      res->hits = (uint64_t)n_hsaw;
      res->attempts = W->aid[n_hsaw - 1] + 1;
      res->cov_R = cov;
      res->spread_base_est = n * (double)res->hits / (double)res->attempts;
      res->spread_reduction_est = n * (double)cov / (double)res->attempts;
    }
  } else {
    if (delta <= 0) delta = 1.0 / n;
    double k6[6];
    oracle_stop_constants(M, k, eps, delta, k6);
    double nmax = k6[1], tmax = k6[3], lam = k6[4], lam1 = k6[5];
    int64_t L = (int64_t)ceil(lam);
    for (int t = 1;; ++t) {
      int64_t half = L << (t - 1);
      rc = oracle_stream_extend(c, W, 2 * half, max_attempts);
      if (rc == 0 && W->count < 2 * half) rc = -7;
      if (rc) break;
      rc = oracle_greedy(W, mode, 0, half, M, cand_mask, k, ids, gains);
      if (rc) break;
      uint64_t cov = 0;
      for (int32_t i = 0; i < k; ++i) cov += gains[i];
      int64_t covp = oracle_coverage(W, mode, half, half, M, ids, k);
      double et;
      int ok = oracle_check((double)cov, (double)covp, (double)half, t, eps, lam1, &et);
      res->n_selected = k;
      res->rounds_t = t;
      res->hits = (uint64_t)(2 * half);
      res->attempts = W->aid[2 * half - 1] + 1;
      res->cov_R = cov;
      res->cov_Rprime = (uint64_t)covp;
      res->hits_Rprime = (uint64_t)half;
      res->attempts_Rprime = W->aid[2 * half - 1] - W->aid[half - 1];
      res->spread_base_est = n * (double)res->hits / (double)res->attempts;
      res->spread_reduction_est = n * (double)(cov + (uint64_t)covp) / (double)res->attempts;
      if (!isnan(et)) res->eps_t = et;
      if (ok) break;
      if ((double)half >= nmax || (double)t >= tmax) break;
    }
  }
  /* steps up to the last attempt used */
  res->steps = W->steps;
  res->status = rc;
  oracle_walks_free(W);
  return rc;
}

/* =====================================================================================
 * Brute force (Sec. 2.1 live-edge equivalence, Eqs. "compute_inf", "prob_src_set",
 * "def:eis"): the exact expected spread I_G(V_I) by enumerating every live-edge world
 * (each node keeps one in-edge j with probability w_j / 2^32, or none) and every seed
 * set X ~ V_I.  A node is infected in a world iff its unique backward chain of chosen
 * edges meets X before repeating a node.  Removed edges are never live, removed nodes
 * are neither infected nor counted nor seeds.  For graphs with <= ~12 nodes.
 * ===================================================================================== */
double oracle_bruteforce_spread(const oracle_graph* g, const int32_t* sources, int32_t n_sources,
                                const uint32_t* p_fixed, const uint8_t* edge_removed,
                                const uint8_t* node_removed) {
  int64_t n = g->n;
  int32_t* choice = (int32_t*)calloc((size_t)n, sizeof(int32_t)); /* index into in-list, d = none */
  int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  uint8_t* inX = (uint8_t*)calloc((size_t)n, 1);
  uint8_t* seen = (uint8_t*)calloc((size_t)n, 1);
  double total = 0.0;
  for (;;) {
    /* probability of this world */
    double pw = 1.0;
    for (int64_t v = 0; v < n; ++v) {
      int64_t b = g->row_ptr[v], d = g->row_ptr[v + 1] - b;
      if (choice[v] < d) {
        pw *= (double)g->w[b + choice[v]] / 4294967296.0;
        int64_t e = b + choice[v];
        int32_t u = g->src[e];
        int live = !(edge_removed && edge_removed[e]) && !(node_removed && node_removed[u]);
        parent[v] = live ? u : -1;
      } else {
        uint64_t sum = d ? g->thr[b + d - 1] : 0;
        pw *= (double)(4294967296ull - sum) / 4294967296.0;
        parent[v] = -1;
      }
    }
    if (pw > 0.0) {
      for (int64_t xs = 0; xs < ((int64_t)1 << n_sources); ++xs) {
        double px = 1.0;
        memset(inX, 0, (size_t)n);
        for (int32_t i = 0; i < n_sources; ++i) {
          double p = 1.0;
          if (p_fixed && p_fixed[i] != 0xFFFFFFFFu) p = (double)p_fixed[i] / 4294967296.0;
          if (xs & ((int64_t)1 << i)) { px *= p; if (!(node_removed && node_removed[sources[i]])) inX[sources[i]] = 1; }
          else px *= (1.0 - p);
        }
        if (px == 0.0) continue;
        int64_t infected = 0;
        for (int64_t v = 0; v < n; ++v) {
          if (node_removed && node_removed[v]) continue;
          memset(seen, 0, (size_t)n);
          int32_t x = (int32_t)v;
          while (x >= 0 && !seen[x]) {
            if (inX[x]) { infected++; break; }
            seen[x] = 1;
            x = parent[x];
          }
        }
        total += pw * px * (double)infected;
      }
    }
    /* next world (mixed-radix counter) */
    int64_t v = 0;
    for (; v < n; ++v) {
      int64_t d = g->row_ptr[v + 1] - g->row_ptr[v];
      if (choice[v] < d) { choice[v]++; break; }
      choice[v] = 0;
    }
    if (v == n) break;
  }
  free(choice); free(parent); free(inX); free(seen);
  return total;
}
