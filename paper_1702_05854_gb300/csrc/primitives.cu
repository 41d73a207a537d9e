// Device primitives: prefix sums and a stable LSD radix sort of (key, value) pairs.
// Used by graph ingest (stable sort of edges by destination) and by the occurrence
// histogram / inverted index (sort of walk elements by id).
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"

namespace hsaw {

int sm_count() {
  static const int cached = [] {  // thread-safe one-time initialisation
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return cached;
}

int bit_width(uint64_t x) {
  int b = 0;
  while (x) { ++b; x >>= 1; }
  return b;
}

// ------------------------------------------------------------------ scan
// Three-phase scan: per-block sums, recursive scan of the sums, per-block scan + offset.
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T block_exclusive_sum(T v, T* smem_warp, T* block_total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T w = lane < (int)(blockDim.x >> 5) ? smem_warp[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < (int)(blockDim.x >> 5)) smem_warp[lane] = w;
  }
  __syncthreads();
  T warp_prefix = wid ? smem_warp[wid - 1] : T(0);
  if (block_total) *block_total = smem_warp[(blockDim.x >> 5) - 1];
  return warp_prefix + x - v;
}

template <typename T>
__global__ void k_scan_reduce(const T* __restrict__ d, size_t n, T* __restrict__ part) {
  __shared__ T sw[32];
  const size_t base = (size_t)blockIdx.x * SCAN_TILE;
  T s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    size_t idx = base + (size_t)i * SCAN_THREADS + threadIdx.x;
    if (idx < n) s += d[idx];
  }
  T tot;
  block_exclusive_sum<T>(s, sw, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_scan_apply(T* __restrict__ d, size_t n, const T* __restrict__ part, T* __restrict__ total) {
  __shared__ T sw[32];
  const size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_ITEMS;  // blocked layout
  T v[SCAN_ITEMS];
  T s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    size_t idx = base + i;
    v[i] = idx < n ? d[idx] : T(0);
    s += v[i];
  }
  T tot;
  T run = block_exclusive_sum<T>(s, sw, &tot) + (part ? part[blockIdx.x] : T(0));
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    size_t idx = base + i;
    if (idx < n) d[idx] = run;
    run += v[i];
  }
  if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == SCAN_THREADS - 1) *total = run;
}

template <typename T>
static hsaw_status exclusive_scan_t(T* d, size_t n, T* total, cudaStream_t s) {
  if (n == 0) {
    if (total) HSAW_CK(cudaMemsetAsync(total, 0, sizeof(T), s));
    return HSAW_OK;
  }
  const size_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb == 1) {
    count_launch();
    k_scan_apply<T><<<1, SCAN_THREADS, 0, s>>>(d, n, nullptr, total);
    HSAW_CK(cudaGetLastError());
    return HSAW_OK;
  }
  T* part = nullptr;
  HSAW_TRY(dmalloc((void**)&part, nb * sizeof(T), s));
  count_launch();
  k_scan_reduce<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(d, n, part);
  hsaw_status st = HSAW_OK;
  if (cudaGetLastError() != cudaSuccess) st = fail(HSAW_E_DEVICE, "scan reduce launch failed");
  if (st == HSAW_OK) st = exclusive_scan_t<T>(part, nb, nullptr, s);
  if (st == HSAW_OK) {
    count_launch();
    k_scan_apply<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(d, n, part, total);
    if (cudaGetLastError() != cudaSuccess) st = fail(HSAW_E_DEVICE, "scan apply launch failed");
  }
  dfree(part, s);
  return st;
}

hsaw_status exclusive_scan_u32(uint32_t* d, size_t n, uint32_t* total, cudaStream_t s) {
  return exclusive_scan_t<uint32_t>(d, n, total, s);
}
hsaw_status exclusive_scan_u64(uint64_t* d, size_t n, uint64_t* total, cudaStream_t s) {
  return exclusive_scan_t<uint64_t>(d, n, total, s);
}

// ------------------------------------------------------------------ radix sort
// Tile = 8 warps x 16 batches x 32 lanes.  Warp w owns the contiguous sub-tile
// [w*512, (w+1)*512) of its tile and walks it batch by batch, so ranks follow input
// order (stable).  Digit offsets are laid out digit-major over tiles: offset[d*T + t].
constexpr int RS_WARPS = 8;
constexpr int RS_BATCH = 16;
constexpr int RS_SUB = RS_BATCH * 32;
constexpr int RS_TILE = RS_WARPS * RS_SUB;

__global__ void __launch_bounds__(256) k_rs_hist(const uint32_t* __restrict__ keys, size_t n, int shift,
                                                 uint32_t* __restrict__ counts, uint32_t tiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const size_t base = (size_t)blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += 256) {
    size_t idx = base + i;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(size_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// One stable scatter pass.  The tile is first ordered by digit in shared memory (ranks
// follow input order: warp sub-tiles in order, batches in order, lanes in order), then
// written out in that order, so each digit's items leave as one contiguous run (about 16
// items per digit and tile) instead of one scattered word per item.
__global__ void __launch_bounds__(256) k_rs_scatter(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                                                    size_t n, int shift, const uint32_t* __restrict__ offsets,
                                                    uint32_t tiles, uint32_t* __restrict__ keys_out,
                                                    uint32_t* __restrict__ vals_out) {
  __shared__ uint32_t wc[RS_WARPS][256];
  __shared__ uint32_t dstart[256];  // first tile position of each digit
  __shared__ uint32_t sw[32];
  __shared__ uint32_t ks[RS_TILE], vs[RS_TILE];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * 256; i += 256) (&wc[0][0])[i] = 0;
  __syncthreads();
  const size_t tile0 = (size_t)blockIdx.x * RS_TILE;
  const size_t sub = tile0 + (size_t)w * RS_SUB;
  uint32_t k[RS_BATCH], v[RS_BATCH];
#pragma unroll
  for (int b = 0; b < RS_BATCH; ++b) {
    size_t idx = sub + (size_t)b * 32 + lane;
    bool ok = idx < n;
    k[b] = ok ? keys[idx] : 0u;
    v[b] = ok ? vals[idx] : 0u;
    unsigned act = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      uint32_t d = (k[b] >> shift) & 255u;
      unsigned same = __match_any_sync(act, d);
      if (lane == __ffs(same) - 1) wc[w][d] += __popc(same);
    }
    __syncwarp();
  }
  __syncthreads();
  {
    // tile position of digit d's first item from warp ww: digits in order, then warps
    const int d = threadIdx.x;
    uint32_t tot = 0;
    for (int ww = 0; ww < RS_WARPS; ++ww) tot += wc[ww][d];
    uint32_t run = block_exclusive_sum<uint32_t>(tot, sw, nullptr);
    dstart[d] = run;
    for (int ww = 0; ww < RS_WARPS; ++ww) {
      uint32_t c = wc[ww][d];
      wc[ww][d] = run;
      run += c;
    }
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int b = 0; b < RS_BATCH; ++b) {
    size_t idx = sub + (size_t)b * 32 + lane;
    bool ok = idx < n;
    unsigned act = __ballot_sync(0xffffffffu, ok);
    uint32_t d = (k[b] >> shift) & 255u;
    unsigned same = ok ? __match_any_sync(act, d) : 0u;
    uint32_t base = ok ? wc[w][d] : 0u;
    __syncwarp();
    if (ok) {
      uint32_t pos = base + __popc(same & lt);
      ks[pos] = k[b];
      vs[pos] = v[b];
      if (lane == __ffs(same) - 1) wc[w][d] = base + __popc(same);
    }
    __syncwarp();
  }
  __syncthreads();
  const uint32_t items = (uint32_t)min((size_t)RS_TILE, n - tile0);
  for (uint32_t i = threadIdx.x; i < items; i += 256) {
    const uint32_t key = ks[i];
    const uint32_t d = (key >> shift) & 255u;
    const uint32_t pos = offsets[(size_t)d * tiles + blockIdx.x] + (i - dstart[d]);
    keys_out[pos] = key;
    vals_out[pos] = vs[i];
  }
}

hsaw_status radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, size_t n,
                             int bits, cudaStream_t s, bool* in_alt) {
  *in_alt = false;
  if (n <= 1 || bits <= 0) return HSAW_OK;
  if (n > 0xFFFFFFFFull) return fail(HSAW_E_INVALID, "radix sort: too many items");
  const uint32_t tiles = (uint32_t)((n + RS_TILE - 1) / RS_TILE);
  uint32_t* counts = nullptr;
  HSAW_TRY(dmalloc((void**)&counts, (size_t)tiles * 256 * sizeof(uint32_t), s));
  hsaw_status st = HSAW_OK;
  uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  for (int shift = 0; shift < bits && st == HSAW_OK; shift += 8) {
    count_launch();
    k_rs_hist<<<tiles, 256, 0, s>>>(ki, n, shift, counts, tiles);
    if (cudaGetLastError() != cudaSuccess) { st = fail(HSAW_E_DEVICE, "radix hist launch failed"); break; }
    st = exclusive_scan_u32(counts, (size_t)tiles * 256, nullptr, s);
    if (st != HSAW_OK) break;
    count_launch();
    k_rs_scatter<<<tiles, 256, 0, s>>>(ki, vi, n, shift, counts, tiles, ko, vo);
    if (cudaGetLastError() != cudaSuccess) { st = fail(HSAW_E_DEVICE, "radix scatter launch failed"); break; }
    uint32_t* t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
    *in_alt = !*in_alt;
  }
  dfree(counts, s);
  return st;
}

}  // namespace hsaw
