// mpm_bin.cu -- step a1 of the path: binning the particles by cell, every step.
//
// Paper (arXiv 1909.13380), ISOPARAMETRIC MESH: locating the material points
// in the mesh is one of the critical costs of MPM, and a search that starts
// from each point's current cell (neighbourhood search) is far cheaper than a
// brute-force one; CODE OVERVIEW: a particle points to its cell, the cell to
// its nodes.
//
// GPU form of the neighbourhood idea.  The particle state is stored in the
// previous step's binning order and a particle moves at most one cell per
// step, so the new binning is the old one plus a few movers:
//   bin_movers  compares each stored particle's new key with the key it was
//               binned under last step and lists the particles that changed
//               tile (counts per tile in and out);
//   bin_scan_*  two passes over the tiles: new tile ranges = old ranges -
//               leavers + arrivals
//               (exclusive scan over tiles), arrival bucket offsets, the
//               active tile list, counter resets;
//   bin_bucket  groups the arrivals by destination tile;
//   bin_tiles   one CTA per tile: the tile's particles are the stayers of its
//               old range plus its arrivals; a stable counting sort by local
//               cell, in storage order, writes the permutation and the keys
//               in binning order.
// The result is exactly the stable sort of the new keys by storage position
// (arrivals from lower tiles precede the stayers, arrivals from higher tiles
// follow them), i.e. the same permutation a full stable radix sort gives, at
// the cost of reading each key twice instead of several sort passes.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mpm_internal.h"

namespace mpm {
namespace {

constexpr int BT = 256;          // bin_tiles threads
constexpr int BT_WARPS = BT / 32;
constexpr int BUCKET_SMEM = 1024;
constexpr int SCAN_T = 256;
constexpr int SCAN_ITEMS = 4;

__global__ void bin_movers(const uint32_t *__restrict__ knew, const uint32_t *__restrict__ kold, int64_t n,
                           int ntiles, int32_t *__restrict__ in_cnt, int32_t *__restrict__ out_cnt,
                           int32_t *__restrict__ movers, int32_t *__restrict__ ctr) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int tn = min((int)(knew[i] >> LOCAL_BITS), ntiles);
    const int to = min((int)(kold[i] >> LOCAL_BITS), ntiles);
    if (tn != to) {
      atomicAdd(&in_cnt[tn], 1);
      atomicAdd(&out_cnt[to], 1);
      movers[atomicAdd(&ctr[C_MOVERS], 1)] = (int32_t)i;
    }
  }
}

// Inclusive warp scan.
__device__ __forceinline__ int warp_incl(int x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive scan across the CTA of one value per thread; returns the prefix
// and writes the total.
__device__ __forceinline__ int cta_excl(int v, int *wsum, int &total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int inc = warp_incl(v);
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    int s = lane < nw ? wsum[lane] : 0;
    s = warp_incl(s);
    if (lane < nw) wsum[lane] = s;
  }
  __syncthreads();
  total = wsum[nw - 1];
  const int base = w ? wsum[w - 1] : 0;
  __syncthreads();
  return base + inc - v;
}

// Per tile e (tiles plus the dead range): new count = old count - leavers +
// arrivals; arrivals; active flag.
__device__ __forceinline__ void tile_counts(int e, int ntiles, const int32_t *old_start, const int32_t *in_cnt,
                                            const int32_t *out_cnt, int &cn, int &cb, int &ca) {
  const int in = in_cnt[e], out = out_cnt[e];
  cn = (old_start[e + 1] - old_start[e]) - out + in;
  cb = in;
  ca = (e < ntiles && cn > 0) ? 1 : 0;
}

// Scan over tiles, pass 1: block totals of (count, arrivals, active).
__global__ void __launch_bounds__(SCAN_T) bin_scan_totals(int ntiles, const int32_t *__restrict__ old_start,
                                                          const int32_t *__restrict__ in_cnt,
                                                          const int32_t *__restrict__ out_cnt,
                                                          int32_t *__restrict__ tot) {
  __shared__ int wsum[32];
  const int m = ntiles + 1;
  const int e0 = blockIdx.x * SCAN_T * SCAN_ITEMS + threadIdx.x * SCAN_ITEMS;
  int sn = 0, sb = 0, sa = 0;
#pragma unroll
  for (int r = 0; r < SCAN_ITEMS; ++r) {
    const int e = e0 + r;
    if (e < m) {
      int cn, cb, ca;
      tile_counts(e, ntiles, old_start, in_cnt, out_cnt, cn, cb, ca);
      sn += cn;
      sb += cb;
      sa += ca;
    }
  }
  int tn, tb, ta;
  cta_excl(sn, wsum, tn);
  cta_excl(sb, wsum, tb);
  cta_excl(sa, wsum, ta);
  if (threadIdx.x == 0) {
    tot[3 * blockIdx.x + 0] = tn;
    tot[3 * blockIdx.x + 1] = tb;
    tot[3 * blockIdx.x + 2] = ta;
  }
}

// Scan over tiles, pass 2: each block adds the totals of the blocks before
// it, scans its own tiles, writes new ranges, arrival offsets and the active
// list, and clears the per-tile counters for the next step.
__global__ void __launch_bounds__(SCAN_T) bin_scan_apply(int64_t n, int ntiles, const int32_t *__restrict__ old_start,
                                                         int32_t *__restrict__ new_start, int32_t *__restrict__ in_cnt,
                                                         int32_t *__restrict__ out_cnt, int32_t *__restrict__ bstart,
                                                         int32_t *__restrict__ bfill, int32_t *__restrict__ active,
                                                         const int32_t *__restrict__ tot, int32_t *__restrict__ ctr) {
  __shared__ int wsum[32];
  const int m = ntiles + 1;
  int on = 0, ob = 0, oa = 0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += SCAN_T) {
    on += tot[3 * b];
    ob += tot[3 * b + 1];
    oa += tot[3 * b + 2];
  }
  int t0, t1, t2;
  cta_excl(on, wsum, t0);
  cta_excl(ob, wsum, t1);
  cta_excl(oa, wsum, t2);
  on = t0;
  ob = t1;
  oa = t2;
  const int e0 = blockIdx.x * SCAN_T * SCAN_ITEMS + threadIdx.x * SCAN_ITEMS;
  int cn[SCAN_ITEMS], cb[SCAN_ITEMS], ca[SCAN_ITEMS];
  int sn = 0, sb = 0, sa = 0;
#pragma unroll
  for (int r = 0; r < SCAN_ITEMS; ++r) {
    const int e = e0 + r;
    cn[r] = cb[r] = ca[r] = 0;
    if (e < m) tile_counts(e, ntiles, old_start, in_cnt, out_cnt, cn[r], cb[r], ca[r]);
    sn += cn[r];
    sb += cb[r];
    sa += ca[r];
  }
  int tn, tb, ta;
  int pn = cta_excl(sn, wsum, tn) + on;
  int pb = cta_excl(sb, wsum, tb) + ob;
  int pa = cta_excl(sa, wsum, ta) + oa;
#pragma unroll
  for (int r = 0; r < SCAN_ITEMS; ++r) {
    const int e = e0 + r;
    if (e < m) {
      new_start[e] = pn;
      bstart[e] = pb;
      if (ca[r]) active[pa] = e;
      in_cnt[e] = 0;
      out_cnt[e] = 0;
      bfill[e] = 0;
    }
    pn += cn[r];
    pb += cb[r];
    pa += ca[r];
  }
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctr[C_MOVERS_SNAP] = ctr[C_MOVERS];
    ctr[C_MOVERS] = 0;
    ctr[C_WORK_BIN] = ctr[C_WORK_P2G] = ctr[C_WORK_NODE] = ctr[C_WORK_P2G2] = ctr[C_WORK_NODE2] = 0;
  }
  if (blockIdx.x == gridDim.x - 1) {
    __syncthreads();  // new_start of the dead range written by this block
    if (threadIdx.x == 0) {
      const int nact = oa + ta;
      new_start[m] = (int32_t)n;
      bstart[m] = ob + tb;
      const int dead_start = new_start[ntiles];
      ctr[C_ACTIVE] = nact;
      ctr[C_DEAD_START] = dead_start;
      ctr[C_BIN_ITEMS] = nact + ((int64_t)dead_start < n ? 1 : 0);
    }
  }
}

__global__ void bin_bucket(const uint32_t *__restrict__ knew, int ntiles, const int32_t *__restrict__ movers,
                           const int32_t *__restrict__ bstart, int32_t *__restrict__ bfill,
                           int32_t *__restrict__ bucket, const int32_t *__restrict__ ctr) {
  const int nm = ctr[C_MOVERS_SNAP];
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < nm; m += gridDim.x * blockDim.x) {
    const int i = movers[m];
    const int tn = min((int)(knew[i] >> LOCAL_BITS), ntiles);
    bucket[bstart[tn] + atomicAdd(&bfill[tn], 1)] = i;
  }
}

__device__ __forceinline__ int next_work(int32_t *ctr, int slot) {
  __shared__ int s_w;
  if (threadIdx.x == 0) s_w = atomicAdd(&ctr[slot], 1);
  __syncthreads();
  const int w = s_w;
  __syncthreads();
  return w;
}

__global__ void __launch_bounds__(BT) bin_tiles(BinLaunch B) {
  __shared__ int cnt[CELLS_PER_TILE];
  __shared__ int base[CELLS_PER_TILE];
  __shared__ int running[CELLS_PER_TILE];
  __shared__ uint16_t wcnt[BT_WARPS][CELLS_PER_TILE + 1];
  __shared__ int sb_in[BUCKET_SMEM];
  __shared__ int sb_out[BUCKET_SMEM];
  __shared__ int s_nl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const int ntiles = B.ntiles;
  for (int i = tid; i < BT_WARPS * (CELLS_PER_TILE + 1); i += BT) (&wcnt[0][0])[i] = 0;
  __syncthreads();

  for (;;) {
    const int w = next_work(B.s.ctr, C_WORK_BIN);
    if (w >= B.s.ctr[C_BIN_ITEMS]) break;
    const int t = (w < B.s.ctr[C_ACTIVE]) ? B.s.active[w] : ntiles;
    const int os = B.old_start[t], oe = B.old_start[t + 1];
    const int bs = B.s.bucket_start[t], be = B.s.bucket_start[t + 1];
    const int nbk = be - bs;
    const int ns = B.new_start[t];

    // arrivals sorted by storage position (positions are distinct)
    const int *sorted;
    if (nbk <= BUCKET_SMEM) {
      for (int i = tid; i < nbk; i += BT) sb_in[i] = B.s.bucket[bs + i];
      __syncthreads();
      for (int i = tid; i < nbk; i += BT) {
        const int p = sb_in[i];
        int r = 0;
        for (int j = 0; j < nbk; ++j) r += sb_in[j] < p;
        sb_out[r] = p;
      }
      sorted = sb_out;
    } else {
      const int32_t *src = B.s.bucket + bs;
      for (int i = tid; i < nbk; i += BT) {
        const int p = src[i];
        int r = 0;
        for (int j = 0; j < nbk; ++j) r += src[j] < p;
        B.s.bucket_sorted[bs + r] = p;
      }
      sorted = B.s.bucket_sorted + bs;
    }
    if (tid < CELLS_PER_TILE) {
      cnt[tid] = 0;
      running[tid] = 0;
    }
    __syncthreads();
    if (tid == 0) {  // arrivals stored before the old range come first
      int lo = 0, hi = nbk;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sorted[mid] < os) lo = mid + 1; else hi = mid;
      }
      s_nl = lo;
    }
    __syncthreads();
    const int nl = s_nl;
    const int nr = oe - os;
    const int S = nbk + nr;

    // histogram of local cells (warp-aggregated shared atomics)
    for (int c0 = 0; c0 < S; c0 += BT) {
      const int s = c0 + tid;
      int d = CELLS_PER_TILE;
      if (s < S) {
        const bool in_range = s >= nl && s < nl + nr;
        const int pos = in_range ? os + (s - nl) : sorted[s < nl ? s : s - nr];
        const uint32_t k = B.knew[pos];
        if (!in_range || (int)min((int)(k >> LOCAL_BITS), ntiles) == t)
          d = (t == ntiles) ? 0 : (int)(k & (CELLS_PER_TILE - 1));
      }
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      if (d < CELLS_PER_TILE && (peers & lt_mask) == 0) atomicAdd(&cnt[d], __popc(peers));
    }
    __syncthreads();
    if (warp == 0) {
      const int a = cnt[lane], b = cnt[lane + 32];
      const int ia = warp_incl(a);
      const int tot_a = __shfl_sync(0xffffffffu, ia, 31);
      const int ib = warp_incl(b);
      base[lane] = ia - a;
      base[lane + 32] = tot_a + ib - b;
    }
    __syncthreads();

    // stable scatter in storage order
    for (int c0 = 0; c0 < S; c0 += BT) {
      const int s = c0 + tid;
      int d = CELLS_PER_TILE;
      int pos = 0;
      uint32_t k = 0;
      if (s < S) {
        const bool in_range = s >= nl && s < nl + nr;
        pos = in_range ? os + (s - nl) : sorted[s < nl ? s : s - nr];
        k = B.knew[pos];
        if (!in_range || (int)min((int)(k >> LOCAL_BITS), ntiles) == t)
          d = (t == ntiles) ? 0 : (int)(k & (CELLS_PER_TILE - 1));
      }
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const int rank = __popc(peers & lt_mask);
      if (rank == 0) wcnt[warp][d] = (uint16_t)__popc(peers);
      __syncthreads();
      if (d < CELLS_PER_TILE) {
        int dst = ns + base[d] + running[d] + rank;
        for (int k2 = 0; k2 < warp; ++k2) dst += wcnt[k2][d];
        B.perm_out[dst] = pos;
        B.keys_out[dst] = k;
      }
      __syncthreads();
      if (tid <= CELLS_PER_TILE) {
        int add = 0;
#pragma unroll
        for (int k2 = 0; k2 < BT_WARPS; ++k2) {
          add += wcnt[k2][tid];
          wcnt[k2][tid] = 0;
        }
        if (tid < CELLS_PER_TILE) running[tid] += add;
      }
      __syncthreads();
    }
  }
}

template <int D>
__global__ void permute_k(int64_t n, PBuf A, PBuf B, const int32_t *__restrict__ perm) {
  constexpr int NS = nstress<D>();
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int j = perm[q];
    B.key[q] = A.key[j];
    B.id[q] = A.id[j];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      B.off[k][q] = A.off[k][j];
      B.vel[k][q] = A.vel[k][j];
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      B.sig[i][q] = A.sig[i][j];
      B.eps[i][q] = A.eps[i][j];
    }
    B.mass[q] = A.mass[j];
    B.jm1[q] = A.jm1[j];
    B.epsp[q] = A.epsp[j];
    if (A.coh) B.coh[q] = A.coh[j];
  }
}

}  // namespace

cudaError_t bin_step(const BinLaunch &B, cudaStream_t st) {
  if (B.n <= 0) return cudaSuccess;
  const int gridp = (int)((B.n + 255) / 256 < B.grid * 4 ? (B.n + 255) / 256 : B.grid * 4);
  bin_movers<<<gridp, 256, 0, st>>>(B.knew, B.kold, B.n, B.ntiles, B.s.in_cnt, B.s.out_cnt, B.s.movers, B.s.ctr);
  const int sblocks = (B.ntiles + 1 + SCAN_T * SCAN_ITEMS - 1) / (SCAN_T * SCAN_ITEMS);
  bin_scan_totals<<<sblocks, SCAN_T, 0, st>>>(B.ntiles, B.old_start, B.s.in_cnt, B.s.out_cnt, B.s.scan_tot);
  bin_scan_apply<<<sblocks, SCAN_T, 0, st>>>(B.n, B.ntiles, B.old_start, B.new_start, B.s.in_cnt, B.s.out_cnt,
                                             B.s.bucket_start, B.s.bucket_fill, B.s.active, B.s.scan_tot, B.s.ctr);
  bin_bucket<<<B.grid, 256, 0, st>>>(B.knew, B.ntiles, B.s.movers, B.s.bucket_start, B.s.bucket_fill, B.s.bucket,
                                     B.s.ctr);
  bin_tiles<<<B.grid, BT, 0, st>>>(B);
  return cudaGetLastError();
}

cudaError_t permute_state(int dim, int64_t n, const PBuf &A, const PBuf &B, const int32_t *perm, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192);
  if (dim == 3)
    permute_k<3><<<blocks, 256, 0, st>>>(n, A, B, perm);
  else
    permute_k<2><<<blocks, 256, 0, st>>>(n, A, B, perm);
  return cudaGetLastError();
}

}  // namespace mpm
