// mpm_sort.cu -- step a1 of the path: binning particles by cell.
//
// Paper (arXiv 1909.13380), ISOPARAMETRIC MESH: locating material points in
// the mesh is one of the critical costs of MPM; CODE OVERVIEW: every
// particle points to the cell that holds it and the cell gives its nodes.
// On the GPU the particles are binned every step by a stable LSD radix sort
// of (tile-major cell key, storage index), 8-bit digits, and the tile
// boundaries are read off the sorted keys.  Stability makes the order a
// pure function of the keys and the previous order, so every reduction
// that follows it is deterministic.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mpm_internal.h"

namespace mpm {
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 4096 keys per block
constexpr int RADIX = 256;
constexpr int RS_WARPS = RS_THREADS / 32;

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Per-block digit histograms, digit-major: hist[d * nblocks + block].
__global__ void __launch_bounds__(RS_THREADS) rs_upsweep(const uint32_t *__restrict__ keys, int64_t n,
                                                         int shift, uint32_t *__restrict__ hist,
                                                         int nblocks) {
  __shared__ uint32_t cnt[RADIX];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int64_t i = base + r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & (RADIX - 1)], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Block-wide exclusive scan of 16 consecutive items per thread.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_tot, uint32_t &total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < RS_WARPS ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < RS_WARPS) warp_tot[lane] = t;  // inclusive warp prefix
  }
  __syncthreads();
  total = warp_tot[RS_WARPS - 1];
  const uint32_t wbase = w ? warp_tot[w - 1] : 0u;
  __syncthreads();
  return wbase + x - v;
}

// Chunk sums of 4096 items.
__global__ void __launch_bounds__(RS_THREADS) scan_chunk_sums(const uint32_t *__restrict__ in, int64_t n,
                                                              uint32_t *__restrict__ sums) {
  __shared__ uint32_t wt[RS_WARPS];
  const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)threadIdx.x * RS_ITEMS;
  uint32_t s = 0;
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r)
    if (base + r < n) s += in[base + r];
  uint32_t tot;
  block_exclusive_scan(s, wt, tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Exclusive scan of the chunk sums by one block (any length).
__global__ void __launch_bounds__(RS_THREADS) scan_sums_single(uint32_t *__restrict__ sums, int64_t m) {
  __shared__ uint32_t wt[RS_WARPS];
  uint32_t carry = 0;
  for (int64_t c0 = 0; c0 < m; c0 += RS_TILE) {
    const int64_t base = c0 + (int64_t)threadIdx.x * RS_ITEMS;
    uint32_t loc[RS_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
      loc[r] = (base + r < m) ? sums[base + r] : 0u;
      s += loc[r];
    }
    uint32_t tot;
    uint32_t pre = block_exclusive_scan(s, wt, tot) + carry;
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
      if (base + r < m) sums[base + r] = pre;
      pre += loc[r];
    }
    carry += tot;
  }
}

// out[i] = exclusive prefix of in[] (uses the scanned chunk sums).  May run
// in place (out == in): each thread reads its items into registers before it
// writes the same items, so in and out are not declared __restrict__.
__global__ void __launch_bounds__(RS_THREADS) scan_apply(const uint32_t *in, int64_t n,
                                                         const uint32_t *__restrict__ sums, uint32_t *out) {
  __shared__ uint32_t wt[RS_WARPS];
  const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)threadIdx.x * RS_ITEMS;
  uint32_t loc[RS_ITEMS];
  uint32_t s = 0;
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    loc[r] = (base + r < n) ? in[base + r] : 0u;
    s += loc[r];
  }
  uint32_t tot;
  uint32_t pre = block_exclusive_scan(s, wt, tot) + sums[blockIdx.x];
#pragma unroll
  for (int r = 0; r < RS_ITEMS; ++r) {
    if (base + r < n) out[base + r] = pre;
    pre += loc[r];
  }
}

// Stable scatter of one digit pass.  Items are ranked in index order: within
// a warp by __match_any_sync peers, across the warps of a round by per-warp
// digit counts, across rounds by running per-digit counters.
__global__ void __launch_bounds__(RS_THREADS) rs_downsweep(const uint32_t *__restrict__ kin,
                                                           const int32_t *__restrict__ vin,
                                                           uint32_t *__restrict__ kout,
                                                           int32_t *__restrict__ vout, int64_t n,
                                                           int shift, const uint32_t *__restrict__ offs,
                                                           int nblocks) {
  __shared__ uint32_t running[RADIX];
  __shared__ uint16_t wcnt[RS_WARPS][RADIX + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  running[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  for (int k = 0; k < RS_WARPS; ++k) wcnt[k][threadIdx.x] = 0;
  if (threadIdx.x < RS_WARPS) wcnt[threadIdx.x][RADIX] = 0;
  __syncthreads();
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ITEMS; ++r) {
    const int64_t i = base + r * RS_THREADS + threadIdx.x;
    const bool valid = i < n;
    uint32_t key = 0;
    int32_t val = 0;
    int d = RADIX;  // invalid items get a digit of their own
    if (valid) {
      key = kin[i];
      val = vin ? vin[i] : (int32_t)i;
      d = (key >> shift) & (RADIX - 1);
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt_mask);
    if (rank == 0) wcnt[w][d] = (uint16_t)__popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t pos = running[d] + rank;
      for (int k = 0; k < w; ++k) pos += wcnt[k][d];
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    {
      const int dd = threadIdx.x;
      uint32_t add = 0;
#pragma unroll
      for (int k = 0; k < RS_WARPS; ++k) {
        add += wcnt[k][dd];
        wcnt[k][dd] = 0;
      }
      running[dd] += add;
    }
    __syncthreads();
  }
}

// tile_start[u] = lower bound of u * 64 in the sorted keys.
__global__ void k_tile_bounds(const uint32_t *__restrict__ keys, int64_t n, int ntiles,
                              int32_t *__restrict__ tile_start) {
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u <= ntiles + 1; u += gridDim.x * blockDim.x) {
    if (u == ntiles + 1) {
      tile_start[u] = (int32_t)n;
      continue;
    }
    const uint32_t target = (uint32_t)u << LOCAL_BITS;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (keys[mid] < target) lo = mid + 1; else hi = mid;
    }
    tile_start[u] = (int32_t)lo;
  }
}

}  // namespace

size_t sort_scratch_bytes(int64_t n) {
  const int64_t nb = cdiv(n > 0 ? n : 1, RS_TILE);
  const int64_t hn = (int64_t)RADIX * nb;
  const int64_t nsum = cdiv(hn, RS_TILE);
  return align256(sizeof(uint32_t) * n) * 2 + align256(sizeof(int32_t) * n) * 2 +
         align256(sizeof(uint32_t) * hn) + align256(sizeof(uint32_t) * nsum) + 1024;
}

cudaError_t sort_pairs(const uint32_t *keys_in, const int32_t *vals_in, uint32_t *keys_out,
                       int32_t *perm_out, int64_t n, int key_bits, void *scratch, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int nb = (int)cdiv(n, RS_TILE);
  const int64_t hn = (int64_t)RADIX * nb;
  const int nsum = (int)cdiv(hn, RS_TILE);
  char *p = (char *)scratch;
  uint32_t *k0 = (uint32_t *)p; p += align256(sizeof(uint32_t) * n);
  uint32_t *k1 = (uint32_t *)p; p += align256(sizeof(uint32_t) * n);
  int32_t *v0 = (int32_t *)p; p += align256(sizeof(int32_t) * n);
  int32_t *v1 = (int32_t *)p; p += align256(sizeof(int32_t) * n);
  uint32_t *hist = (uint32_t *)p; p += align256(sizeof(uint32_t) * hn);
  uint32_t *sums = (uint32_t *)p;
  const int passes = key_bits <= 0 ? 1 : (key_bits + 7) / 8;
  const uint32_t *kin = keys_in;
  const int32_t *vin = vals_in;
  for (int ps = 0; ps < passes; ++ps) {
    const bool last = ps == passes - 1;
    uint32_t *ko = last ? keys_out : (ps & 1 ? k1 : k0);
    int32_t *vo = last ? perm_out : (ps & 1 ? v1 : v0);
    const int shift = 8 * ps;
    rs_upsweep<<<nb, RS_THREADS, 0, st>>>(kin, n, shift, hist, nb);
    scan_chunk_sums<<<nsum, RS_THREADS, 0, st>>>(hist, hn, sums);
    scan_sums_single<<<1, RS_THREADS, 0, st>>>(sums, nsum);
    scan_apply<<<nsum, RS_THREADS, 0, st>>>(hist, hn, sums, hist);
    rs_downsweep<<<nb, RS_THREADS, 0, st>>>(kin, vin, ko, vo, n, shift, hist, nb);
    kin = ko;
    vin = vo;
  }
  return cudaGetLastError();
}

cudaError_t tile_bounds(const uint32_t *keys_sorted, int64_t n, int ntiles, int32_t *tile_start,
                        cudaStream_t st) {
  k_tile_bounds<<<(ntiles + 2 + 255) / 256, 256, 0, st>>>(keys_sorted, n, ntiles, tile_start);
  return cudaGetLastError();
}

}  // namespace mpm
