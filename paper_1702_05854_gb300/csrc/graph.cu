// Graph ingest (Sec. 2.1): edge list or CSR -> device in-adjacency with running uint32
// in-weight sums, per-node records and validation of the LT in-weight condition.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace hsaw {

// ------------------------------------------------------------------ errors / memory
static thread_local std::string t_err;
void set_error(const std::string& msg) { t_err = msg; }
const char* last_error() { return t_err.c_str(); }
hsaw_status fail(hsaw_status st, const std::string& msg) {
  t_err = msg;
  return st;
}
hsaw_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  t_err = buf;
  return (e == cudaErrorMemoryAllocation) ? HSAW_E_NOMEM : HSAW_E_DEVICE;
}

static std::once_flag g_pool_once;
static std::atomic<long long> g_fail_countdown{0};  // test hook: > 0 counts down to a failing allocation

// Scratch allocator: CUDA's stream-ordered pool, or the caller's (hsaw_set_allocator).  The
// allocator changes only while no scratch block is held and no other call runs, so every
// block goes back to the allocator it came from; allocations read it without a lock.
struct ScratchAllocator {
  hsaw_alloc_fn alloc;
  hsaw_free_fn release;
  void* ctx;
};
static std::mutex g_alloc_set_mu;                          // serialises changes
static std::vector<std::unique_ptr<ScratchAllocator>> g_alloc_all;  // every one installed, kept to exit
static std::atomic<const ScratchAllocator*> g_alloc{nullptr};
static std::atomic<long long> g_held{0};                   // scratch blocks handed out, not yet released

hsaw_status dmalloc(void** p, size_t bytes, cudaStream_t s) {
  if (g_fail_countdown.load(std::memory_order_relaxed) > 0 && g_fail_countdown.fetch_sub(1) == 1) {
    *p = nullptr;
    t_err = "device allocation failed (injected by hsaw_debug_fail_alloc_after)";
    return HSAW_E_NOMEM;
  }
  if (bytes == 0) bytes = 16;
  if (const ScratchAllocator* a = g_alloc.load(std::memory_order_acquire)) {
    *p = a->alloc(bytes, (void*)s, a->ctx);
    if (!*p) {
      char buf[128];
      snprintf(buf, sizeof(buf), "device allocation of %zu bytes failed (caller's allocator)", bytes);
      t_err = buf;
      return HSAW_E_NOMEM;
    }
    g_held.fetch_add(1);
    return HSAW_OK;
  }
  std::call_once(g_pool_once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  });
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    char buf[128];
    snprintf(buf, sizeof(buf), "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    t_err = buf;
    return HSAW_E_NOMEM;
  }
  g_held.fetch_add(1);
  return HSAW_OK;
}
void dfree(void* p, cudaStream_t s) {
  if (!p) return;
  if (const ScratchAllocator* a = g_alloc.load(std::memory_order_acquire))
    a->release(p, (void*)s, a->ctx);
  else
    cudaFreeAsync(p, s);
  g_held.fetch_sub(1);
}

// ------------------------------------------------------------------ kernels
enum : uint32_t { ERR_RANGE = 1u, ERR_WEIGHT = 2u, ERR_ROWPTR = 4u };

__global__ void k_validate_nodes(const int32_t* __restrict__ a, int64_t m, int64_t n, uint32_t* __restrict__ err) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    if (a[e] < 0 || a[e] >= n) atomicOr(err, ERR_RANGE);
}

__global__ void k_iota_dst(const int32_t* __restrict__ dst, int64_t m, uint32_t* __restrict__ keys,
                           uint32_t* __restrict__ vals) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    keys[e] = (uint32_t)dst[e];
    vals[e] = (uint32_t)e;
  }
}

// row_start[v] = first CSR position of v (lower bound of v in the sorted destinations).
__global__ void k_row_from_sorted(const uint32_t* __restrict__ sorted_dst, int64_t m, int64_t n,
                                  uint32_t* __restrict__ row_start) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = 0, hi = m;
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if ((int64_t)sorted_dst[mid] < v) lo = mid + 1; else hi = mid;
    }
    row_start[v] = (uint32_t)lo;
  }
}

__global__ void k_gather_edges(const uint32_t* __restrict__ perm, const int32_t* __restrict__ src,
                               const uint32_t* __restrict__ w, int64_t m, uint2* __restrict__ edge,
                               int64_t* __restrict__ input_index) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
    uint32_t e = perm[q];
    edge[q] = make_uint2((uint32_t)src[e], w[e]);
    if (input_index) input_index[q] = e;
  }
}

__global__ void k_csr_rows(const int64_t* __restrict__ rp, int64_t n, int64_t m, uint32_t* __restrict__ row_start,
                           uint32_t* __restrict__ err) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x) {
    int64_t a = rp[v];
    if (a < 0 || a > m || (v < n && rp[v + 1] < a) || (v == 0 && a != 0) || (v == n && a != m))
      atomicOr(err, ERR_ROWPTR);
    row_start[v] = (uint32_t)(a < 0 ? 0 : (a > m ? m : a));
  }
}

__global__ void k_copy_edges(const int32_t* __restrict__ src, const uint32_t* __restrict__ w, int64_t m, int64_t n,
                             uint2* __restrict__ edge, uint32_t* __restrict__ err) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
    int32_t a = src[q];
    if (a < 0 || a >= n) atomicOr(err, ERR_RANGE);
    edge[q] = make_uint2((uint32_t)a, w[q]);
  }
}

// One warp per node: running in-weight sums (exact, 64-bit carry), the in-sum check
// (<= 2^32 - 1), equal-weight detection and the node record.
__global__ void k_thresholds(const uint32_t* __restrict__ row_start, int64_t n, uint2* __restrict__ edge,
                             uint4* __restrict__ node, uint32_t* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const uint32_t b = row_start[v], e = row_start[v + 1];
    const uint32_t deg = e - b;
    uint64_t carry = 0;
    uint32_t w0 = deg ? edge[b].y : 0u;
    bool uniform = true;
    for (uint32_t base = b; base < e; base += 32) {
      uint32_t q = base + lane;
      uint64_t w = q < e ? edge[q].y : 0u;
      if (q < e && (uint32_t)w != w0) uniform = false;
      uint64_t x = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      uint64_t run = carry + x;
      if (q < e) {
        if (run > 0xFFFFFFFFull) atomicOr(err, ERR_WEIGHT);
        edge[q].y = (uint32_t)(run > 0xFFFFFFFFull ? 0xFFFFFFFFull : run);
      }
      carry += __shfl_sync(0xffffffffu, x, 31);
    }
    uniform = __all_sync(0xffffffffu, uniform);
    if (lane == 0) {
      uint32_t insum = (uint32_t)(carry > 0xFFFFFFFFull ? 0xFFFFFFFFull : carry);
      node[v] = make_uint4(b, deg, (uniform && deg) ? w0 : 0u, insum);
    }
  }
}

// 32-byte walk records (see Graph::erec).
__global__ void k_walk_records(const uint2* __restrict__ edge, const uint4* __restrict__ node, int64_t m,
                               uint4* __restrict__ erec) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const uint2 ed = edge[e];
    const uint4 nu = node[ed.x];
    erec[2 * e] = make_uint4(ed.x, nu.x, nu.y, nu.z);
    erec[2 * e + 1] = make_uint4(nu.w, ed.y, 0u, 0u);
  }
}

// Guide tables of the nodes with unequal in-weights (see Graph::guide); one warp per node.
__global__ void k_guide(const uint4* __restrict__ node, const uint2* __restrict__ edge, int64_t n,
                        uint32_t* __restrict__ guide, uint32_t* __restrict__ n_unequal) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t cnt = 0;
  for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const uint4 nd = node[v];
    if (nd.y == 0 || nd.z != 0 || nd.w == 0) continue;  // no in-edge, equal weights, or zero in-sum
    cnt += lane == 0 ? 1u : 0u;
    for (uint32_t b = lane; b < nd.y; b += 32) {
      const uint32_t lb = (uint32_t)(((uint64_t)b * nd.w + nd.y - 1) / nd.y);  // ceil(b * insum / deg)
      uint32_t lo = 0, hi = nd.y;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (lb < edge[nd.x + mid].y) hi = mid; else lo = mid + 1;
      }
      guide[nd.x + b] = lo;
    }
  }
  if (cnt) atomicAdd(n_unequal, cnt);
}

// Bucket records of the nodes with unequal in-weights (see Graph::grec); one warp per node.
__global__ void k_guide_records(const uint4* __restrict__ node, const uint32_t* __restrict__ guide, int64_t n,
                                const uint4* __restrict__ erec, uint4* __restrict__ grec) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const uint4 nd = node[v];
    if (nd.y == 0 || nd.z != 0 || nd.w == 0) continue;
    for (uint32_t b = lane; b < nd.y; b += 32) {
      const size_t p = (size_t)nd.x + b;
      const uint32_t j0 = guide[p];
      const size_t e0 = (size_t)nd.x + j0;
      grec[2 * p] = erec[2 * e0];
      uint4 hi = erec[2 * e0 + 1];
      hi.z = j0;
      grec[2 * p + 1] = hi;
    }
  }
}

// ------------------------------------------------------------------ host
static hsaw_status check_err(uint32_t* d_err, cudaStream_t s) {
  uint32_t h = 0;
  HSAW_CK(cudaMemcpyAsync(&h, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  HSAW_CK(cudaStreamSynchronize(s));
  if (h & ERR_RANGE) return fail(HSAW_E_RANGE, "graph: a node index is outside [0, n)");
  if (h & ERR_ROWPTR) return fail(HSAW_E_INVALID, "graph: in_row_ptr is not a valid CSR offset array");
  if (h & ERR_WEIGHT) return fail(HSAW_E_WEIGHT_SUM, "graph: a node's in-weight sum exceeds 2^32 - 1");
  return HSAW_OK;
}

// True for page-locked (pinned or registered) host memory, whose copies run asynchronously.
static bool host_pinned(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

template <typename T>
static hsaw_status stage(const T* p, size_t count, bool on_device, cudaStream_t s, T** dev, bool* owned) {
  *owned = false;
  if (on_device || count == 0) {
    *dev = const_cast<T*>(p);
    return HSAW_OK;
  }
  HSAW_TRY(dmalloc((void**)dev, count * sizeof(T), s));
  *owned = true;
  const cudaError_t e = cudaMemcpyAsync(*dev, p, count * sizeof(T), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    dfree(*dev, s);
    *dev = nullptr;
    *owned = false;
    return cuda_fail(e, "cudaMemcpyAsync(graph input)", __FILE__, __LINE__);
  }
  return HSAW_OK;
}

void pool_release(WalkPool& p);

static void destroy_graph(Graph& g) {
  pool_release(g.pool);
  if (g.node) cudaFree(g.node);
  if (g.edge) cudaFree(g.edge);
  if (g.input_index) cudaFree(g.input_index);
  if (g.erec) cudaFree(g.erec);
  if (g.grec) cudaFree(g.grec);
  g.erec = nullptr;
  g.grec = nullptr;
  g.node = nullptr;
  g.edge = nullptr;
  g.input_index = nullptr;
}

static hsaw_status alloc_graph(Graph& g, int64_t n, int64_t m, bool with_index) {
  g.n = n;
  g.m = m;
  cudaGetDevice(&g.device);
  HSAW_CK(cudaMalloc((void**)&g.node, (size_t)n * sizeof(uint4)));
  HSAW_CK(cudaMalloc((void**)&g.edge, (size_t)(m ? m : 1) * sizeof(uint2)));
  HSAW_CK(cudaMalloc((void**)&g.erec, (size_t)(m ? m : 1) * 2 * sizeof(uint4)));
  if (with_index) HSAW_CK(cudaMalloc((void**)&g.input_index, (size_t)(m ? m : 1) * sizeof(int64_t)));
  return HSAW_OK;
}

// A second stream (with one event) for copies that overlap work on the call's stream; it is
// drained and destroyed when the call returns, before its temporaries are freed.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  hsaw_status create() {
    HSAW_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    HSAW_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    return HSAW_OK;
  }
  ~SideStream() {
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
    if (ev) cudaEventDestroy(ev);
  }
};

struct Temps {
  std::vector<void*> ptrs;
  cudaStream_t s;
  explicit Temps(cudaStream_t st) : s(st) {}
  template <typename T>
  hsaw_status get(T** p, size_t count) {
    HSAW_TRY(dmalloc((void**)p, (count ? count : 1) * sizeof(T), s));
    ptrs.push_back(*p);
    return HSAW_OK;
  }
  void keep(void* p) { ptrs.push_back(p); }
  ~Temps() {
    for (void* p : ptrs) dfree(p, s);
  }
};

static hsaw_status finish_graph(Graph& g, uint32_t* row_start, uint32_t* d_err, cudaStream_t s) {
  const int64_t n = g.n;
  count_launch();
  k_thresholds<<<grid_for((size_t)n * 32, 256, 1u << 20), 256, 0, s>>>(row_start, n, g.edge, g.node, d_err);
  HSAW_CK(cudaGetLastError());
  HSAW_TRY(check_err(d_err, s));
  if (g.m) {
    count_launch();
    k_walk_records<<<grid_for(g.m, 256, 1u << 16), 256, 0, s>>>(g.edge, g.node, g.m, g.erec);
    HSAW_CK(cudaGetLastError());
    // guide tables and their bucket records, kept only when some node has unequal
    // in-weights (the guide itself is a temporary)
    uint32_t* guide = nullptr;
    HSAW_TRY(dmalloc((void**)&guide, (size_t)g.m * sizeof(uint32_t), s));
    HSAW_CK(cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s));
    count_launch();
    k_guide<<<grid_for((size_t)n * 32, 256, 1u << 20), 256, 0, s>>>(g.node, g.edge, n, guide, d_err);
    uint32_t unequal = 0;
    hsaw_status st = HSAW_OK;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&unequal, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = fail(HSAW_E_DEVICE, "graph: guide tables failed");
    if (st == HSAW_OK && unequal) {
      if (cudaMalloc((void**)&g.grec, (size_t)g.m * 2 * sizeof(uint4)) != cudaSuccess) {
        cudaGetLastError();
        g.grec = nullptr;
        st = fail(HSAW_E_NOMEM, "graph: guide records do not fit in device memory");
      } else {
        count_launch();
        k_guide_records<<<grid_for((size_t)n * 32, 256, 1u << 20), 256, 0, s>>>(g.node, guide, n, g.erec, g.grec);
        if (cudaGetLastError() != cudaSuccess) st = fail(HSAW_E_DEVICE, "graph: guide records failed");
      }
    }
    dfree(guide, s);
    HSAW_TRY(st);
  }
  return HSAW_OK;
}

static hsaw_status from_edges(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const uint32_t* w,
                              uint32_t flags, cudaStream_t s, Graph& g) {
  if (n < 1 || m < 0 || n >= (1ll << 31) || m >= (1ll << 31)) return fail(HSAW_E_INVALID, "graph: need 1 <= n < 2^31, 0 <= m < 2^31");
  if (m > 0 && (!src || !dst || !w)) return fail(HSAW_E_INVALID, "graph: NULL edge array");
  const bool dev = flags & HSAW_INPUT_DEVICE;
  Temps T(s);
  // pinned host input: the destinations are copied first and sorted on s while the
  // sources and weights are copied on a side stream (drained before T frees); pageable
  // input is copied first, all of it, on s (its copies do not overlap kernels)
  SideStream side;
  const bool overlap = !dev && m > 0 && host_pinned(src) && host_pinned(w);
  int32_t *d_src = nullptr, *d_dst = nullptr;
  uint32_t* d_w = nullptr;
  bool o1 = false, o2 = false, o3 = false;
  if (!overlap) {
    HSAW_TRY(stage(src, (size_t)m, dev, s, &d_src, &o1));
    if (o1) T.keep(d_src);
    HSAW_TRY(stage(w, (size_t)m, dev, s, &d_w, &o3));
    if (o3) T.keep(d_w);
  }
  HSAW_TRY(stage(dst, (size_t)m, dev, s, &d_dst, &o2));
  if (o2) T.keep(d_dst);
  uint32_t* d_err = nullptr;
  HSAW_TRY(T.get(&d_err, 1));
  HSAW_CK(cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s));
  if (m) {
    count_launch();
    k_validate_nodes<<<grid_for(m, 256, 8192), 256, 0, s>>>(d_dst, m, n, d_err);
    if (!overlap) {
      count_launch();
      k_validate_nodes<<<grid_for(m, 256, 8192), 256, 0, s>>>(d_src, m, n, d_err);
    }
    HSAW_CK(cudaGetLastError());
    HSAW_TRY(check_err(d_err, s));
  }
  uint32_t *keys, *vals, *keys2, *vals2, *row_start;
  HSAW_TRY(T.get(&keys, m));
  HSAW_TRY(T.get(&vals, m));
  HSAW_TRY(T.get(&keys2, m));
  HSAW_TRY(T.get(&vals2, m));
  HSAW_TRY(T.get(&row_start, n + 1));
  if (m) {
    count_launch();
    k_iota_dst<<<grid_for(m, 256, 8192), 256, 0, s>>>(d_dst, m, keys, vals);
    HSAW_CK(cudaGetLastError());
  }
  bool alt = false;
  HSAW_TRY(radix_sort_pairs(keys, vals, keys2, vals2, (size_t)m, bit_width((uint64_t)(n - 1)), s, &alt));
  uint32_t* sk = alt ? keys2 : keys;
  uint32_t* sv = alt ? vals2 : vals;
  count_launch();
  k_row_from_sorted<<<grid_for(n + 1, 256, 8192), 256, 0, s>>>(sk, m, n, row_start);
  HSAW_CK(cudaGetLastError());
  if (overlap) {  // the destinations' copy finished at the validation's synchronisation
    HSAW_TRY(side.create());
    HSAW_TRY(stage(src, (size_t)m, dev, side.s, &d_src, &o1));
    if (o1) T.keep(d_src);
    HSAW_TRY(stage(w, (size_t)m, dev, side.s, &d_w, &o3));
    if (o3) T.keep(d_w);
    HSAW_CK(cudaEventRecord(side.ev, side.s));
    HSAW_CK(cudaStreamWaitEvent(s, side.ev, 0));
    count_launch();
    k_validate_nodes<<<grid_for(m, 256, 8192), 256, 0, s>>>(d_src, m, n, d_err);
    HSAW_CK(cudaGetLastError());
    HSAW_TRY(check_err(d_err, s));
  }
  HSAW_TRY(alloc_graph(g, n, m, true));
  if (m) {
    count_launch();
    k_gather_edges<<<grid_for(m, 256, 8192), 256, 0, s>>>(sv, d_src, d_w, m, g.edge, g.input_index);
    HSAW_CK(cudaGetLastError());
  }
  return finish_graph(g, row_start, d_err, s);
}

static hsaw_status from_csr(int64_t n, int64_t m, const int64_t* rp, const int32_t* src, const uint32_t* w,
                            uint32_t flags, cudaStream_t s, Graph& g) {
  if (n < 1 || m < 0 || n >= (1ll << 31) || m >= (1ll << 31)) return fail(HSAW_E_INVALID, "graph: need 1 <= n < 2^31, 0 <= m < 2^31");
  if (!rp || (m > 0 && (!src || !w))) return fail(HSAW_E_INVALID, "graph: NULL CSR array");
  const bool dev = flags & HSAW_INPUT_DEVICE;
  Temps T(s);
  int64_t* d_rp;
  int32_t* d_src;
  uint32_t* d_w;
  bool o1, o2, o3;
  HSAW_TRY(stage(rp, (size_t)n + 1, dev, s, &d_rp, &o1));
  if (o1) T.keep(d_rp);
  HSAW_TRY(stage(src, (size_t)m, dev, s, &d_src, &o2));
  if (o2) T.keep(d_src);
  HSAW_TRY(stage(w, (size_t)m, dev, s, &d_w, &o3));
  if (o3) T.keep(d_w);
  uint32_t *d_err, *row_start;
  HSAW_TRY(T.get(&d_err, 1));
  HSAW_TRY(T.get(&row_start, n + 1));
  HSAW_CK(cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s));
  count_launch();
  k_csr_rows<<<grid_for(n + 1, 256, 8192), 256, 0, s>>>(d_rp, n, m, row_start, d_err);
  HSAW_CK(cudaGetLastError());
  HSAW_TRY(check_err(d_err, s));
  HSAW_TRY(alloc_graph(g, n, m, false));
  if (m) {
    count_launch();
    k_copy_edges<<<grid_for(m, 256, 8192), 256, 0, s>>>(d_src, d_w, m, n, g.edge, d_err);
    HSAW_CK(cudaGetLastError());
    HSAW_TRY(check_err(d_err, s));
  }
  return finish_graph(g, row_start, d_err, s);
}

// node record -> host CSR export
static hsaw_status export_graph(const Graph& g, int64_t* rp, int32_t* src, int32_t* dst, uint32_t* thr, int64_t* ii,
                                cudaStream_t s) {
  std::vector<uint4> node((size_t)g.n);
  HSAW_CK(cudaMemcpyAsync(node.data(), g.node, (size_t)g.n * sizeof(uint4), cudaMemcpyDeviceToHost, s));
  std::vector<uint2> edge;
  if (src || thr) {
    edge.resize((size_t)g.m);
    if (g.m) HSAW_CK(cudaMemcpyAsync(edge.data(), g.edge, (size_t)g.m * sizeof(uint2), cudaMemcpyDeviceToHost, s));
  }
  if (ii && g.m) {
    if (g.input_index)
      HSAW_CK(cudaMemcpyAsync(ii, g.input_index, (size_t)g.m * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  }
  HSAW_CK(cudaStreamSynchronize(s));
  if (ii && !g.input_index)
    for (int64_t e = 0; e < g.m; ++e) ii[e] = e;
  if (rp) {
    for (int64_t v = 0; v < g.n; ++v) rp[v] = node[v].x;
    rp[g.n] = g.m;
  }
  if (dst)
    for (int64_t v = 0; v < g.n; ++v)
      for (uint32_t q = node[v].x; q < node[v].x + node[v].y; ++q) dst[q] = (int32_t)v;
  for (int64_t q = 0; q < g.m; ++q) {
    if (src) src[q] = (int32_t)edge[q].x;
    if (thr) thr[q] = edge[q].y;
  }
  return HSAW_OK;
}

}  // namespace hsaw

using namespace hsaw;

extern "C" {

const char* hsaw_last_error(void) { return hsaw::last_error(); }
const char* hsaw_version(void) { return "hsaw-gb300 0.1 (sm_103a)"; }

hsaw_status hsaw_graph_from_edges(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const uint32_t* w_fixed,
                                  uint32_t flags, void* stream, hsaw_graph* out) {
  if (!out) return fail(HSAW_E_INVALID, "graph: NULL out");
  *out = nullptr;
  auto* h = new (std::nothrow) hsaw_graph_s();
  if (!h) return fail(HSAW_E_NOMEM, "graph: host allocation");
  hsaw_status st = from_edges(n, m, src, dst, w_fixed, flags, (cudaStream_t)stream, h->g);
  if (st != HSAW_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    destroy_graph(h->g);
    delete h;
    return st;
  }
  *out = h;
  return HSAW_OK;
}

hsaw_status hsaw_graph_from_csr(int64_t n, int64_t m, const int64_t* in_row_ptr, const int32_t* in_src,
                                const uint32_t* w_fixed, uint32_t flags, void* stream, hsaw_graph* out) {
  if (!out) return fail(HSAW_E_INVALID, "graph: NULL out");
  *out = nullptr;
  auto* h = new (std::nothrow) hsaw_graph_s();
  if (!h) return fail(HSAW_E_NOMEM, "graph: host allocation");
  hsaw_status st = from_csr(n, m, in_row_ptr, in_src, w_fixed, flags, (cudaStream_t)stream, h->g);
  if (st != HSAW_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    destroy_graph(h->g);
    delete h;
    return st;
  }
  *out = h;
  return HSAW_OK;
}

hsaw_status hsaw_graph_destroy(hsaw_graph g) {
  if (!g) return HSAW_OK;
  cudaDeviceSynchronize();
  sample_tune_forget(g->g);
  destroy_graph(g->g);
  delete g;
  return HSAW_OK;
}

hsaw_status hsaw_set_allocator(hsaw_alloc_fn alloc, hsaw_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr))
    return fail(HSAW_E_INVALID, "allocator: give both alloc and release, or neither");
  std::lock_guard<std::mutex> lk(g_alloc_set_mu);
  const long long held = g_held.load();
  if (held != 0) {
    char buf[160];
    snprintf(buf, sizeof(buf), "allocator: %lld scratch blocks of the current allocator are still held", held);
    t_err = buf;
    return HSAW_E_INVALID;
  }
  const ScratchAllocator* next = nullptr;
  if (alloc) {
    g_alloc_all.emplace_back(new ScratchAllocator{alloc, release, ctx});
    next = g_alloc_all.back().get();
  }
  g_alloc.store(next, std::memory_order_release);
  return HSAW_OK;
}

hsaw_status hsaw_debug_fail_alloc_after(int64_t n) {
  g_fail_countdown.store(n > 0 ? n : 0);
  return HSAW_OK;
}

hsaw_status hsaw_graph_edge(hsaw_graph g, int64_t edge_id, int32_t* src, int32_t* dst, int64_t* input_index) {
  if (!g) return fail(HSAW_E_INVALID, "graph: NULL handle");
  if (edge_id < 0 || edge_id >= g->g.m) return fail(HSAW_E_RANGE, "graph: edge id outside [0, m)");
  uint2 ed;
  HSAW_CK(cudaMemcpy(&ed, g->g.edge + edge_id, sizeof(uint2), cudaMemcpyDeviceToHost));
  if (src) *src = (int32_t)ed.x;
  if (dst) {  // the node whose in-range holds edge_id: binary search over the node records
    int64_t lo = 0, hi = g->g.n - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) / 2;
      uint4 nd;
      HSAW_CK(cudaMemcpy(&nd, g->g.node + mid, sizeof(uint4), cudaMemcpyDeviceToHost));
      if ((int64_t)nd.x <= edge_id) lo = mid; else hi = mid - 1;
    }
    // nodes without in-edges share their first position with the next node: take the
    // last node starting at or before edge_id whose range is non-empty
    uint4 nd;
    HSAW_CK(cudaMemcpy(&nd, g->g.node + lo, sizeof(uint4), cudaMemcpyDeviceToHost));
    while (lo > 0 && (int64_t)nd.x + nd.y <= edge_id) {
      --lo;
      HSAW_CK(cudaMemcpy(&nd, g->g.node + lo, sizeof(uint4), cudaMemcpyDeviceToHost));
    }
    *dst = (int32_t)lo;
  }
  if (input_index) {
    if (g->g.input_index) {
      HSAW_CK(cudaMemcpy(input_index, g->g.input_index + edge_id, sizeof(int64_t), cudaMemcpyDeviceToHost));
    } else {
      *input_index = edge_id;
    }
  }
  return HSAW_OK;
}

hsaw_status hsaw_graph_info(hsaw_graph g, int64_t* n, int64_t* m) {
  if (!g) return fail(HSAW_E_INVALID, "graph: NULL handle");
  if (n) *n = g->g.n;
  if (m) *m = g->g.m;
  return HSAW_OK;
}

hsaw_status hsaw_graph_export(hsaw_graph g, int64_t* in_row_ptr, int32_t* in_src, int32_t* in_dst, uint32_t* thr,
                              int64_t* input_index, void* stream) {
  if (!g) return fail(HSAW_E_INVALID, "graph: NULL handle");
  return export_graph(g->g, in_row_ptr, in_src, in_dst, thr, input_index, (cudaStream_t)stream);
}

}  // extern "C"
