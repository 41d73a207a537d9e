/*
 * Seeded synthetic inputs for the HSAW spread-interdiction path.
 *
 * This module only MAKES inputs: directed power-law graphs shaped like the social
 * networks of the paper's experiments (Sec. 6, Table "Datasets' Statistics"), their
 * LT in-weights in uint32 fixed point, source sets and suspect probabilities.  It holds
 * none of the method's arithmetic (no CSR build, no thresholds, no walks, no counting),
 * and both the CUDA library's tests and the CPU oracle take their inputs from here.
 *
 * Randomness: a counter-based SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014): draw(seed, stream, i) is the
 * (i+1)-th output of a SplitMix64 sequence whose state starts at mix(seed, stream).
 * Every draw is a pure function of (seed, stream, i), so multithreaded generation is
 * bit-identical to a serial one.
 *
 * Built with -ffp-contract=off so the floating-point parts (Chung-Lu weights) give the
 * same bits whatever the host compiler would otherwise fuse.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN64 0x9E3779B97F4A7C15ULL

static inline uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* i-th draw of the stream (seed, stream). */
static inline uint64_t sm_draw(uint64_t seed, uint64_t stream, uint64_t i) {
  uint64_t base = sm_mix(seed * GOLDEN64 + sm_mix(stream + 0x5851F42D4C957F2DULL));
  return sm_mix(base + (i + 1) * GOLDEN64);
}

uint64_t synth_draw(uint64_t seed, uint64_t stream, uint64_t i) { return sm_draw(seed, stream, i); }

/* uniform double in [0,1) from the top 53 bits */
static inline double sm_unit(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

/* ---------------------------------------------------------------- threading helper */
typedef void (*range_fn)(void* ctx, int64_t lo, int64_t hi);
typedef struct { range_fn fn; void* ctx; int64_t lo, hi; } range_job;
static void* range_tramp(void* p) {
  range_job* j = (range_job*)p;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}
static void parallel_range(range_fn fn, void* ctx, int64_t total, int threads) {
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  if (total < 1 << 16 || threads == 1) { fn(ctx, 0, total); return; }
  pthread_t th[256];
  range_job jobs[256];
  int started = 0;
  for (int t = 0; t < threads; ++t) {
    jobs[t].fn = fn; jobs[t].ctx = ctx;
    jobs[t].lo = total * t / threads; jobs[t].hi = total * (t + 1) / threads;
    if (pthread_create(&th[t], NULL, range_tramp, &jobs[t]) != 0) {
      fn(ctx, jobs[t].lo, jobs[t].hi);   /* run inline if no thread could be made */
      jobs[t].fn = NULL;
    } else {
      started++;
    }
  }
  for (int t = 0; t < threads; ++t)
    if (jobs[t].fn) pthread_join(th[t], NULL);
  (void)started;
}

/* ---------------------------------------------------------------- Chung-Lu */
/* Directed Chung-Lu: each of m edge draws picks src ~ out-weight and dst ~ in-weight,
 * weight of rank i proportional to (i+1)^(-1/(gamma-1)); ranks are assigned to nodes by
 * two independent uniform permutations (one for out, one for in).  Self-loops and
 * parallel edges are kept so that m is exact. */
typedef struct {
  const double* cdf; const int32_t* perm_out; const int32_t* perm_in;
  int64_t n; uint64_t seed; int32_t* src; int32_t* dst;
} cl_ctx;

static int64_t cdf_pick(const double* cdf, int64_t n, double u) {
  /* first i with u < cdf[i]; cdf[n-1] == 1.0 */
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (u < cdf[mid]) hi = mid; else lo = mid + 1;
  }
  return lo;
}

static void cl_edges(void* p, int64_t lo, int64_t hi) {
  cl_ctx* c = (cl_ctx*)p;
  for (int64_t e = lo; e < hi; ++e) {
    double u1 = sm_unit(sm_draw(c->seed, 11, (uint64_t)e));
    double u2 = sm_unit(sm_draw(c->seed, 12, (uint64_t)e));
    c->src[e] = c->perm_out[cdf_pick(c->cdf, c->n, u1)];
    c->dst[e] = c->perm_in[cdf_pick(c->cdf, c->n, u2)];
  }
}

static void shuffle_perm(int32_t* perm, int64_t n, uint64_t seed, uint64_t stream) {
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; --i) {
    uint64_t r = sm_draw(seed, stream, (uint64_t)i);
    int64_t j = (int64_t)(((unsigned __int128)r * (uint64_t)(i + 1)) >> 64);
    int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
}

int synth_chung_lu(int64_t n, int64_t m, double gamma, uint64_t seed, int threads,
                   int32_t* src, int32_t* dst) {
  if (n < 1 || m < 0 || !(gamma > 1.0)) return -1;
  double* cdf = (double*)malloc(sizeof(double) * (size_t)n);
  int32_t* po = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* pi = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!cdf || !po || !pi) { free(cdf); free(po); free(pi); return -4; }
  double ex = -1.0 / (gamma - 1.0), acc = 0.0;
  for (int64_t i = 0; i < n; ++i) { acc += pow((double)(i + 1), ex); cdf[i] = acc; }
  for (int64_t i = 0; i < n; ++i) cdf[i] /= acc;
  cdf[n - 1] = 1.0;
  shuffle_perm(po, n, seed, 13);
  shuffle_perm(pi, n, seed, 14);
  cl_ctx c = {cdf, po, pi, n, seed, src, dst};
  parallel_range(cl_edges, &c, m, threads);
  free(cdf); free(po); free(pi);
  return 0;
}

/* ---------------------------------------------------------------- R-MAT */
/* R-MAT (Chakrabarti, Zhan, Faloutsos, SDM 2004): each edge descends `scale` levels of
 * the adjacency matrix; at each level a quadrant is chosen with probabilities
 * (a, b, c, d) = (top-left, top-right, bottom-left, bottom-right), row = src bit,
 * column = dst bit, most significant bit first.  No noise, no permutation; edges are
 * kept as generated (self-loops and duplicates included). */
typedef struct {
  int scale; uint32_t ta, tab, tabc; uint64_t seed; int32_t* src; int32_t* dst;
} rmat_ctx;

static void rmat_edges(void* p, int64_t lo, int64_t hi) {
  rmat_ctx* c = (rmat_ctx*)p;
  int words = (c->scale + 1) / 2;
  for (int64_t e = lo; e < hi; ++e) {
    uint32_t s = 0, d = 0;
    for (int l = 0; l < c->scale; ++l) {
      uint64_t x = sm_draw(c->seed, 21, (uint64_t)e * (uint64_t)words + (uint64_t)(l >> 1));
      uint32_t u = (l & 1) ? (uint32_t)(x >> 32) : (uint32_t)x;
      uint32_t sb, db;
      if (u < c->ta) { sb = 0; db = 0; }
      else if (u < c->tab) { sb = 0; db = 1; }
      else if (u < c->tabc) { sb = 1; db = 0; }
      else { sb = 1; db = 1; }
      s = (s << 1) | sb;
      d = (d << 1) | db;
    }
    c->src[e] = (int32_t)s;
    c->dst[e] = (int32_t)d;
  }
}

int synth_rmat(int scale, int64_t m, double a, double b, double c, uint64_t seed, int threads,
               int32_t* src, int32_t* dst) {
  if (scale < 1 || scale > 30 || m < 0) return -1;
  if (!(a >= 0 && b >= 0 && c >= 0 && a + b + c <= 1.0)) return -1;
  const double two32 = 4294967296.0;
  rmat_ctx x;
  x.scale = scale;
  x.ta = (uint32_t)fmin(a * two32, 4294967295.0);
  x.tab = (uint32_t)fmin((a + b) * two32, 4294967295.0);
  x.tabc = (uint32_t)fmin((a + b + c) * two32, 4294967295.0);
  x.seed = seed; x.src = src; x.dst = dst;
  parallel_range(rmat_edges, &x, m, threads);
  return 0;
}

/* ---------------------------------------------------------------- LT weights */
/* Weighted cascade (Sec. 6 "Parameter Settings": w(u,v) = 1/d_in(v)), in uint32 fixed
 * point: w_fixed = floor((2^32 - 1) / d_in(v)), so a node's in-sum never exceeds
 * 2^32 - 1 (the largest value a cumulative uint32 threshold can hold). */
int synth_wc_weights(int64_t n, int64_t m, const int32_t* dst, uint32_t* w) {
  uint32_t* deg = (uint32_t*)calloc((size_t)n, sizeof(uint32_t));
  if (!deg) return -4;
  for (int64_t e = 0; e < m; ++e) {
    if (dst[e] < 0 || dst[e] >= n) { free(deg); return -3; }
    deg[dst[e]]++;
  }
  for (int64_t e = 0; e < m; ++e) w[e] = (uint32_t)(0xFFFFFFFFu / deg[dst[e]]);
  free(deg);
  return 0;
}

/* Random LT weights: x_e ~ U(0,1) per in-edge, scaled so that node v's in-sum is
 * s_v ~ U(0.5, 1).  In integers: x_e in [1, 2^32), s_v in [2^31, 2^32),
 * w_e = floor(x_e * s_v / sum_{e' into v} x_e'), exact in 64-bit arithmetic. */
int synth_random_lt_weights(int64_t n, int64_t m, const int32_t* dst, uint64_t seed, uint32_t* w) {
  uint64_t* sum = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));
  if (!sum) return -4;
  for (int64_t e = 0; e < m; ++e) {
    if (dst[e] < 0 || dst[e] >= n) { free(sum); return -3; }
    uint64_t x = (sm_draw(seed, 31, (uint64_t)e) >> 32) | 1u;
    sum[dst[e]] += x;
  }
  for (int64_t e = 0; e < m; ++e) {
    int32_t v = dst[e];
    uint64_t x = (sm_draw(seed, 31, (uint64_t)e) >> 32) | 1u;
    uint64_t s = 0x80000000ULL + ((sm_draw(seed, 32, (uint64_t)v) >> 32) >> 1);
    w[e] = (uint32_t)((unsigned __int128)x * s / sum[v]);
  }
  free(sum);
  return 0;
}

/* ---------------------------------------------------------------- sources */
/* `count` distinct nodes drawn uniformly from [0, n), returned in ascending order. */
int synth_sources(int64_t n, int64_t count, uint64_t seed, int32_t* out) {
  if (count < 0 || count > n) return -1;
  uint8_t* seen = (uint8_t*)calloc((size_t)((n + 7) / 8), 1);
  if (!seen) return -4;
  int64_t got = 0;
  for (uint64_t i = 0; got < count; ++i) {
    uint64_t r = sm_draw(seed, 41, i);
    int64_t v = (int64_t)(((unsigned __int128)r * (uint64_t)n) >> 64);
    if (!(seen[v >> 3] & (1u << (v & 7)))) { seen[v >> 3] |= (uint8_t)(1u << (v & 7)); got++; }
  }
  int64_t k = 0;
  for (int64_t v = 0; v < n && k < count; ++v)
    if (seen[v >> 3] & (1u << (v & 7))) out[k++] = (int32_t)v;
  free(seen);
  return 0;
}

/* Suspect probabilities p(v) in uint32 fixed point, uniform over [0, 2^32). */
int synth_probabilities(int64_t count, uint64_t seed, uint32_t* out) {
  for (int64_t i = 0; i < count; ++i) out[i] = (uint32_t)(sm_draw(seed, 51, (uint64_t)i) >> 32);
  return 0;
}
