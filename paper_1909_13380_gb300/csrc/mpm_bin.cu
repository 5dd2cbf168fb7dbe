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
//   (G2P of the previous step counts and lists the particles that changed
//   tile; bin_movers recounts them from the keys when a caller needs it)
//   bin_scan_lb      one pass over the tiles (decoupled look-back): new tile
//                    ranges = old ranges - leavers + arrivals (exclusive scan
//                    over tiles), arrival bucket offsets, the active tile
//                    list, counter resets; the last block to finish computes
//                    the work prefixes over the instances of the group;
//   bin_scan_one     (instead, when every instance has at most SCAN1_MAX
//                    tiles) one CTA per instance scans all of its tiles in
//                    one pass;
//   bin_bucket       groups the arrivals by destination tile;
//   bin_tiles        one CTA per tile: the tile's particles are the stayers
//                    of its old range plus its arrivals; a stable counting
//                    sort by local cell, in storage order, writes the
//                    permutation and the keys in binning order.
// The result is exactly the stable sort of the new keys by storage position
// (arrivals from lower tiles precede the stayers, arrivals from higher tiles
// follow them), i.e. the same permutation a full stable radix sort gives, at
// the cost of reading each key twice instead of several sort passes.
// Every kernel runs over a table of independent instances (a single mesh is
// a table of one); blocks and work items map to instances through prefix
// arrays.
#include <climits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mpm_internal.h"

namespace mpm {
namespace {

constexpr int BUCKET_SMEM = 1024;
constexpr int SCAN_T = 256;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_CHUNK = SCAN_T * SCAN_ITEMS;  // tiles per scan block
constexpr int SCAN1_T = 1024;                    // one-CTA scan: threads
constexpr int SCAN1_K = MPM_SCAN1_K;             // one-CTA scan: tiles per thread at most
static_assert(SCAN1_T * SCAN1_K == SCAN1_MAX, "the one-CTA scan covers SCAN1_MAX tiles");

// Instance of item x: the largest i with prefix[i] <= x (prefix[0] = 0).
__device__ __forceinline__ int find_inst(const int32_t *prefix, int ninst, int x) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void bin_movers(GroupArgs G) {
  const int i = find_inst(G.pblk, G.ninst, blockIdx.x);
  const InstArgs &I = G.inst[i];
  const int64_t p = (int64_t)(blockIdx.x - G.pblk[i]) * blockDim.x + threadIdx.x;
  if (p >= I.n) return;
  const int ntiles = I.ntiles;
  const int tn = min((int)(I.A.key()[p] >> LOCAL_BITS), ntiles);
  const int to = min((int)(I.s.keys_sorted[p] >> LOCAL_BITS), ntiles);
  if (tn != to) {
    atomicAdd(&I.s.in_cnt[tn], 1);
    atomicAdd(&I.s.out_cnt[to], 1);
    I.s.movers[atomicAdd(&I.s.ctr[C_MOVERS], 1)] = (int32_t)p;
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

// The same for NV values per thread at once (NV scans, one set of
// barriers); v becomes the NV prefixes.  The CTA has at most 32 warps.
constexpr int NSCAN = 4;  // new count, arrivals, active tiles, residual P2G items
__device__ __forceinline__ void cta_excl4(int v[NSCAN], int (*wsum)[32], int total[NSCAN]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int inc[NSCAN];
#pragma unroll
  for (int k = 0; k < NSCAN; ++k) {
    inc[k] = warp_incl(v[k]);
    if (lane == 31) wsum[k][w] = inc[k];
  }
  __syncthreads();
  if (w < NSCAN) {
    int s = lane < nw ? wsum[w][lane] : 0;
    s = warp_incl(s);
    if (lane < nw) wsum[w][lane] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NSCAN; ++k) {
    total[k] = wsum[k][nw - 1];
    v[k] = (w ? wsum[k][w - 1] : 0) + inc[k] - v[k];
  }
  __syncthreads();
}

// Per tile e (tiles plus the dead range): new count = old count - leavers +
// arrivals; arrivals; active flag; residual flag: an active tile whose
// next-step P2G the previous G2P did not complete -- its partial sums are
// not for this step (`step`), or particles arrived from other tiles.
// A frozen instance (a bounded wait of an earlier scan gave up, its binning
// is not valid) has every particle in the dead range, so the step carries its
// state over unchanged and its kernels touch nothing else.
__device__ __forceinline__ void tile_counts(const InstArgs &I, int e, int step, bool frozen, int &cn, int &cb,
                                            int &ca, int &cr) {
  if (frozen) {
    cn = e == I.ntiles ? (int)I.n : 0;
    cb = ca = cr = 0;
    return;
  }
  const int in = I.s.in_cnt[e], out = I.s.out_cnt[e];
  cn = (I.old_start[e + 1] - I.old_start[e]) - out + in;
  cb = in;
  ca = (e < I.ntiles && cn > 0) ? 1 : 0;
  cr = (ca && (in > 0 || I.s.fepoch[e] != step)) ? 1 : 0;
}

// Prefixes of the binning tiles and the active tiles over the instances, and
// reset of the group's dynamic work counters.
__device__ __forceinline__ void group_prefix_body(const GroupArgs &G, int *wsum) {
  int cb = 0, ca = 0, cr = 0;
  for (int c0 = 0; c0 < G.ninst; c0 += blockDim.x) {
    const int j = c0 + threadIdx.x;
    int b = 0, a = 0, r = 0;
    if (j < G.ninst) {
      const int32_t *ctr = G.inst[j].s.ctr;
      // an instance whose scan gave up a wait this step does no more work in it
      if (!(__ldcg(ctr + C_STATUS) & ST_TIMEOUT)) {
        b = __ldcg(ctr + C_BIN_ITEMS);
        a = __ldcg(ctr + C_ACTIVE);
        r = __ldcg(ctr + C_RESID);
      }
    }
    int tb, ta, tr;
    const int pb = cta_excl(b, wsum, tb) + cb;
    const int pa = cta_excl(a, wsum, ta) + ca;
    const int pr = cta_excl(r, wsum, tr) + cr;
    if (j < G.ninst) {
      G.bin_items[j] = pb;
      G.act_items[j] = pa;
      G.res_items[j] = pr;
    }
    cb += tb;
    ca += ta;
    cr += tr;
  }
  if (threadIdx.x == 0) {
    G.bin_items[G.ninst] = cb;
    G.act_items[G.ninst] = ca;
    G.res_items[G.ninst] = cr;
  }
  if (threadIdx.x < W_COUNT) G.work[threadIdx.x] = 0;
}

// Scan over tiles in one pass with decoupled look-back (Merrill & Garland,
// "Single-pass parallel prefix scan with decoupled look-back", 2016).  Each
// block takes a ticket in start order, which names its chunk of SCAN_CHUNK
// tiles; it publishes its chunk's totals of (count, arrivals, active,
// residual), then one warp reads the chunks before it 32 at a time, adding
// their published totals up to the nearest one that has published its
// inclusive prefix.  A block waits only on chunks whose blocks took lower
// tickets and are therefore already running, so every wait ends; each wait
// is nonetheless bounded, and gives up with ST_TIMEOUT set.  Then it writes
// new ranges, arrival offsets, the active and residual lists and the counter
// resets of its tiles, and the block that finishes last advances the step
// index, computes the group's prefixes and clears the chunk flags for the
// next step.
// Per chunk k, scan_tot[SCAN_REC k ..] = flag (0 none, 1 totals, 2
// inclusive), totals (4), inclusive prefix (4).
constexpr int SCAN_REC = 16;

__device__ __forceinline__ int ld_volatile(const int32_t *p) { return *(const volatile int32_t *)p; }

template <bool ONE>
__global__ void __launch_bounds__(SCAN_T) bin_scan_lb(const __grid_constant__ GroupArgs G) {
  __shared__ int wsum4[NSCAN][32];
  __shared__ int s_ticket, s_last;
  __shared__ int s_excl[NSCAN];
  __shared__ InstArgs sI;
  pdl_trigger();
  pdl_wait();
  if (threadIdx.x == 0) s_ticket = atomicAdd(&G.work[W_SCAN_TICKET], 1);
  __syncthreads();
  const int tk = s_ticket;
  const int i = ONE ? 0 : find_inst(G.sblk, G.ninst, tk);
  if (!ONE) {
    copy_inst(G.inst, i, &sI);
    __syncthreads();
  }
  const InstArgs &I = inst_ref<ONE>(G, sI);
  const int c = ONE ? tk : tk - G.sblk[i];
  const int nchunks = ONE ? G.nblk_s : G.sblk[i + 1] - G.sblk[i];
  const int m = I.ntiles + 1;
  const int step = __ldcg(I.s.ctr + C_STEP) + 1;  // this step's index (the last block stores it)
  const bool frozen = (__ldcg(I.s.ctr + C_STATUS) & ST_TIMEOUT) != 0;
  int32_t *st = I.s.scan_tot;
  const int e0 = c * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
  int cn[SCAN_ITEMS], cb[SCAN_ITEMS], ca[SCAN_ITEMS], cr[SCAN_ITEMS];
  int pv[NSCAN] = {0, 0, 0, 0};
#pragma unroll
  for (int r = 0; r < SCAN_ITEMS; ++r) {
    const int e = e0 + r;
    cn[r] = cb[r] = ca[r] = cr[r] = 0;
    if (e < m) tile_counts(I, e, step, frozen, cn[r], cb[r], ca[r], cr[r]);
    pv[0] += cn[r];
    pv[1] += cb[r];
    pv[2] += ca[r];
    pv[3] += cr[r];
  }
  int tot[NSCAN];
  cta_excl4(pv, wsum4, tot);
  if (threadIdx.x < 32) {  // warp 0: publish, look back 32 chunks at a time, publish the prefix
    const int lane = threadIdx.x;
    int32_t *me = st + SCAN_REC * c;
    int ex[NSCAN] = {0, 0, 0, 0};
    const bool publish = c != I.lb_withhold;  // always, but for the failure-detection test hook
    if (c > 0) {
      if (lane == 0 && publish) {
#pragma unroll
        for (int k = 0; k < NSCAN; ++k) me[1 + k] = tot[k];
        __threadfence();
        atomicExch(me, 1);
      }
      for (int hi = c - 1; hi >= 0; hi -= 32) {
        const int q = hi - lane;  // lane 0 is the nearest predecessor
        int f = 0;
        if (q >= 0) {
          for (int it = 0; it < I.lb_spin && f == 0; ++it) f = ld_volatile(st + SCAN_REC * q);
          if (f == 0) atomicOr(&I.s.ctr[C_STATUS], ST_TIMEOUT);  // gave up: this step is invalid
        }
        __threadfence();
        const unsigned inc = __ballot_sync(0xffffffffu, q >= 0 && f == 2);
        const int upto = inc ? __ffs(inc) - 1 : 31;
        int vals[NSCAN] = {0, 0, 0, 0};
        if (q >= 0 && lane <= upto && f != 0) {
          const int o = (f == 2) ? 1 + NSCAN : 1;
#pragma unroll
          for (int k = 0; k < NSCAN; ++k) vals[k] = ld_volatile(st + SCAN_REC * q + o + k);
        }
#pragma unroll
        for (int k = 0; k < NSCAN; ++k) ex[k] += __reduce_add_sync(0xffffffffu, vals[k]);
        if (inc) break;
      }
    }
    if (lane == 0) {
      if (publish) {
#pragma unroll
        for (int k = 0; k < NSCAN; ++k) me[1 + NSCAN + k] = ex[k] + tot[k];
        __threadfence();
        atomicExch(me, 2);
      }
#pragma unroll
      for (int k = 0; k < NSCAN; ++k) s_excl[k] = ex[k];
    }
  }
  __syncthreads();
  int pn = pv[0] + s_excl[0], pb = pv[1] + s_excl[1], pa = pv[2] + s_excl[2], pr = pv[3] + s_excl[3];
  const int ob = s_excl[1], oa = s_excl[2], orr = s_excl[3];
#pragma unroll
  for (int r = 0; r < SCAN_ITEMS; ++r) {
    const int e = e0 + r;
    if (e < m) {
      I.new_start[e] = pn;
      I.s.bucket_start[e] = pb;
      if (ca[r] || (e == I.ntiles && cn[r] > 0)) {  // a binning item (the dead range comes last)
        I.s.active[pa] = make_int4(e, pn, pn + cn[r], INT_MIN);
        I.s.bin_rec[pa] = make_int4(I.old_start[e], I.old_start[e + 1], pb, pb + cb[r]);
        if (cr[r]) I.s.resid[pr] = pa;
      }
      I.s.in_cnt[e] = 0;
      I.s.out_cnt[e] = 0;
      I.s.bucket_fill[e] = 0;
    }
    pn += cn[r];
    pb += cb[r];
    pa += ca[r];
    pr += cr[r];
  }
  if (threadIdx.x == 0 && c == 0) {
    I.s.ctr[C_MOVERS_SNAP] = I.s.ctr[C_MOVERS];
    I.s.ctr[C_MOVERS] = 0;
    I.s.ctr[C_APEX] = 0;
  }
  __syncthreads();  // new_start of the dead range is written (last chunk)
  if (threadIdx.x == 0) {
    if (c == nchunks - 1) {
      const int nact = oa + tot[2];
      I.new_start[m] = (int32_t)I.n;
      I.s.bucket_start[m] = ob + tot[1];
      const int dead_start = I.new_start[I.ntiles];
      I.s.ctr[C_ACTIVE] = nact;
      I.s.ctr[C_RESID] = orr + tot[3];
      I.s.ctr[C_DEAD_START] = dead_start;
      I.s.ctr[C_BIN_ITEMS] = nact + ((int64_t)dead_start < I.n ? 1 : 0);
    }
    __threadfence();
    s_last = atomicAdd(&G.work[W_SCAN_DONE], 1) == G.nblk_s - 1;
  }
  __syncthreads();
  if (s_last) {  // every chunk of the group has finished its look-back (and read the step index)
    __threadfence();
    for (int ii = 0; ii < G.ninst; ++ii) {
      const InstArgs &J = ONE ? I : G.inst[ii];
      int32_t *sti = J.s.scan_tot;
      for (int k = threadIdx.x; k < G.sblk[ii + 1] - G.sblk[ii]; k += blockDim.x) sti[SCAN_REC * k] = 0;
      if (threadIdx.x == 0) J.s.ctr[C_STEP] = __ldcg(J.s.ctr + C_STEP) + 1;
    }
    group_prefix_body(G, wsum4[0]);
  }
}

template <bool ONE>
__global__ void bin_bucket(const __grid_constant__ GroupArgs G) {
  __shared__ InstArgs sI;
  pdl_trigger();
  const int i = ONE ? 0 : find_inst(G.mblk, G.ninst, blockIdx.x);  // host-written tables
  if (!ONE) copy_inst(G.inst, i, &sI);
  pdl_wait();
  if (!ONE) __syncthreads();
  const InstArgs &I = inst_ref<ONE>(G, sI);
  const int lb = ONE ? blockIdx.x : blockIdx.x - G.mblk[i];
  const int nb = ONE ? G.nblk_m : G.mblk[i + 1] - G.mblk[i];
  const int nm = I.s.ctr[C_MOVERS_SNAP];
  for (int m = lb * blockDim.x + threadIdx.x; m < nm; m += nb * blockDim.x) {
    const int p = I.s.movers[m];
    const int tn = min((int)(I.A.key()[p] >> LOCAL_BITS), I.ntiles);
    I.s.bucket[I.s.bucket_start[tn] + atomicAdd(&I.s.bucket_fill[tn], 1)] = p;
  }
}

// One CTA per instance (instances of at most SCAN1_MAX tiles): the whole scan
// over the instance's tiles in one pass -- new ranges, arrival offsets, the
// active and residual lists, counter resets.  Warp w owns the K consecutive
// 32-tile chunks from tile 32 K w (K = ceil(tiles / SCAN1_T) <= SCAN1_K);
// lane l holds tile l of each chunk, so every load and store is coalesced and
// all the loads are in flight at once.  The warps' totals go through one CTA
// scan, then each warp scans its chunks in order with a running offset.  The
// CTA then advances the instance's step index.  For a group of one the CTA
// writes the group's prefixes itself; otherwise the CTA that finishes last
// (counted on a work counter, no waiting) computes them.
template <bool ONE>
__global__ void __launch_bounds__(SCAN1_T) bin_scan_one(const __grid_constant__ GroupArgs G) {
  __shared__ int wsum4[NSCAN][32];
  __shared__ int s_last;
  __shared__ InstArgs sI;
  pdl_trigger();
  if (!ONE) copy_inst(G.inst, blockIdx.x, &sI);  // host-written table
  pdl_wait();
  if (!ONE) __syncthreads();
  const InstArgs &I = inst_ref<ONE>(G, sI);
  const int m = I.ntiles + 1;
  const int lane = threadIdx.x & 31;
  const int K = (m + SCAN1_T - 1) / SCAN1_T;       // <= SCAN1_K: the host checks m <= SCAN1_MAX
  const int seg0 = (threadIdx.x >> 5) * K * 32;  // this warp's first tile
  const int step = __ldcg(I.s.ctr + C_STEP) + 1;  // this step's index (thread 0 stores it at the end)
  const bool frozen = (__ldcg(I.s.ctr + C_STATUS) & ST_TIMEOUT) != 0;
  int cn[SCAN1_K], cb[SCAN1_K], cr[SCAN1_K];
  int v[NSCAN] = {0, 0, 0, 0};  // this lane's count, arrivals, active tiles, residual items
#pragma unroll
  for (int r = 0; r < SCAN1_K; ++r) {
    const int e = seg0 + r * 32 + lane;
    cn[r] = cb[r] = cr[r] = 0;
    if (r < K && e < m) {
      int ca;
      tile_counts(I, e, step, frozen, cn[r], cb[r], ca, cr[r]);
      v[2] += ca;
    }
    v[0] += cn[r];
    v[1] += cb[r];
    v[3] += cr[r];
  }
  // offsets of the warps: a CTA scan of the warp totals (held by lane 0)
  int tot[NSCAN];
#pragma unroll
  for (int k = 0; k < NSCAN; ++k) {
    v[k] = __reduce_add_sync(0xffffffffu, v[k]);
    if (lane) v[k] = 0;
  }
  cta_excl4(v, wsum4, tot);
  int on = __shfl_sync(0xffffffffu, v[0], 0);
  int ob = __shfl_sync(0xffffffffu, v[1], 0);
  int oa = __shfl_sync(0xffffffffu, v[2], 0);
  int orr = __shfl_sync(0xffffffffu, v[3], 0);
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < SCAN1_K; ++r) {
    if (r < K) {  // warp-uniform
      const int e = seg0 + r * 32 + lane;
      const int in_n = warp_incl(cn[r]), in_b = warp_incl(cb[r]);
      const bool act = e < I.ntiles && cn[r] > 0;
      const unsigned am = __ballot_sync(0xffffffffu, act);
      const unsigned rm = __ballot_sync(0xffffffffu, cr[r] != 0);
      if (e < m) {
        const int pn = on + in_n - cn[r], pb = ob + in_b - cb[r];
        I.new_start[e] = pn;
        I.s.bucket_start[e] = pb;
        if (act || (e == I.ntiles && cn[r] > 0)) {  // a binning item (the dead range comes last)
          const int k = oa + __popc(am & lt_mask);
          I.s.active[k] = make_int4(e, pn, pn + cn[r], INT_MIN);
          I.s.bin_rec[k] = make_int4(I.old_start[e], I.old_start[e + 1], pb, pb + cb[r]);
          if (cr[r]) I.s.resid[orr + __popc(rm & lt_mask)] = k;
        }
        I.s.in_cnt[e] = 0;
        I.s.out_cnt[e] = 0;
        I.s.bucket_fill[e] = 0;
      }
      on += __shfl_sync(0xffffffffu, in_n, 31);
      ob += __shfl_sync(0xffffffffu, in_b, 31);
      oa += __popc(am);
      orr += __popc(rm);
    }
  }
  const int ob_all = tot[1], oa_all = tot[2], or_all = tot[3];
  __syncthreads();  // new_start of the dead range is written; every thread has read the step index
  if (threadIdx.x == 0) {
    I.s.ctr[C_MOVERS_SNAP] = I.s.ctr[C_MOVERS];
    I.s.ctr[C_MOVERS] = 0;
    I.s.ctr[C_APEX] = 0;
    I.s.ctr[C_STEP] = step;
    I.new_start[m] = (int32_t)I.n;
    I.s.bucket_start[m] = ob_all;
    const int dead_start = I.new_start[I.ntiles];
    I.s.ctr[C_ACTIVE] = oa_all;
    I.s.ctr[C_RESID] = or_all;
    I.s.ctr[C_DEAD_START] = dead_start;
    const int bin_items = oa_all + ((int64_t)dead_start < I.n ? 1 : 0);
    I.s.ctr[C_BIN_ITEMS] = bin_items;
    if (ONE) {  // the group's prefixes are this instance's counts
      G.bin_items[0] = 0;
      G.bin_items[1] = bin_items;
      G.act_items[0] = 0;
      G.act_items[1] = oa_all;
      G.res_items[0] = 0;
      G.res_items[1] = or_all;
    } else {
      __threadfence();
      s_last = atomicAdd(&G.work[W_SCAN_DONE], 1) == G.ninst - 1;
    }
  }
  if (ONE) {
    if (threadIdx.x < W_COUNT) G.work[threadIdx.x] = 0;
    return;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    group_prefix_body(G, wsum4[0]);
  }
}


// NT threads per CTA, one tile at a time; the grid holds 2048 threads per SM
// (NT = 256 for groups whose active tiles are about as many as the CTAs, 128
// for large groups, where more tiles in flight per SM shorten the pass).
template <bool ONE, int NT>
__global__ void __launch_bounds__(NT) bin_tiles(const __grid_constant__ GroupArgs G) {
  static_assert(NT > CELLS_PER_TILE && NT % 32 == 0 && 2048 % NT == 0, "bin_tiles block");
  constexpr int NW = NT / 32;
  __shared__ int cnt[CELLS_PER_TILE];
  __shared__ int base[CELLS_PER_TILE];
  __shared__ int running[CELLS_PER_TILE];
  __shared__ uint16_t wcnt[NW][CELLS_PER_TILE + 1];
  __shared__ int sb_in[BUCKET_SMEM];
  __shared__ int sb_out[BUCKET_SMEM];
  __shared__ int s_nl;
  __shared__ InstArgs sI;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  __shared__ int s_work[2];
  pdl_trigger();
  for (int k = tid; k < NW * (CELLS_PER_TILE + 1); k += NT) (&wcnt[0][0])[k] = 0;
  pdl_wait();
  // items: first the CTA's own (blockIdx.x), then gridDim.x + the work counter
  const int total = G.bin_items[G.ninst];
  if (tid == 0) s_work[0] = blockIdx.x;
  __syncthreads();
  int loaded = -1;

  for (int it = 0;; ++it) {
    const int w = s_work[it & 1];
    if (w >= total) break;
    // the next work item is fetched now and published at the end of this one
    int wnext = 0;
    if (tid == 0) wnext = (int)gridDim.x + atomicAdd(&G.work[W_BIN], 1);
    const int ii = ONE ? 0 : find_inst(G.bin_items, G.ninst, w);
    if (!ONE && ii != loaded) {  // uniform
      copy_inst(G.inst, ii, &sI);
      loaded = ii;
      __syncthreads();
    }
    const InstArgs &I = inst_ref<ONE>(G, sI);
    const int local = ONE ? w : w - G.bin_items[ii];
    const int ntiles = I.ntiles;
    const int4 item = I.s.active[local], rec = I.s.bin_rec[local];  // one round of loads
    const int t = item.x, ns = item.y;
    const int os = rec.x, oe = rec.y, bs = rec.z, be = rec.w;
    const int nbk = be - bs;
    const uint32_t *knew = I.A.key();

    // No arrivals, and the old range still holds only this tile's keys in
    // ascending order (no particle left the tile or changed cell out of
    // order): the stable sort is the identity on the range.
    if (nbk == 0 && t < ntiles) {
      const int nr = oe - os;
      // the first KPT keys of each thread load at once and stay in registers
      // for the write-through (a tile of up to KPT * NT particles; 64M-slope
      // binning 272 -> 252 us); the batch kernel, whose registers this would
      // raise from 47 to 56, keeps one key at a time
      constexpr int KPT = ONE ? 4 : 0;
      uint32_t kk[KPT > 0 ? KPT : 1];
      bool sorted = true;
#pragma unroll
      for (int i = 0; i < KPT; ++i) {
        const int k = tid + i * NT;
        if (k < nr) {
          kk[i] = knew[os + k];
          const uint32_t kp = k > 0 ? knew[os + k - 1] : 0u;
          sorted = sorted && (int)(kk[i] >> LOCAL_BITS) == t && kp <= kk[i];
        }
      }
      for (int k = tid + KPT * NT; k < nr; k += NT) {
        const uint32_t kq = knew[os + k];
        sorted = sorted && (int)(kq >> LOCAL_BITS) == t && (k == 0 || knew[os + k - 1] <= kq);
      }
      if (__syncthreads_and(sorted)) {
#pragma unroll
        for (int i = 0; i < KPT; ++i) {
          const int k = tid + i * NT;
          if (k < nr) {
            I.perm_out[ns + k] = os + k;
            I.keys_out[ns + k] = kk[i];
          }
        }
        for (int k = tid + KPT * NT; k < nr; k += NT) {
          I.perm_out[ns + k] = os + k;
          I.keys_out[ns + k] = knew[os + k];
        }
        // the range moved as a whole: P2G maps positions to slots without the permutation
        if (tid == 0) reinterpret_cast<int *>(I.s.active + local)[3] = os - ns;
        if (tid == 0) s_work[(it + 1) & 1] = wnext;
        __syncthreads();
        continue;
      }
    }

    // arrivals sorted by storage position (positions are distinct)
    const int *sorted;
    if (nbk <= BUCKET_SMEM) {
      for (int k = tid; k < nbk; k += NT) sb_in[k] = I.s.bucket[bs + k];
      __syncthreads();
      for (int k = tid; k < nbk; k += NT) {
        const int p = sb_in[k];
        int r = 0;
        for (int j = 0; j < nbk; ++j) r += sb_in[j] < p;
        sb_out[r] = p;
      }
      sorted = sb_out;
    } else {
      const int32_t *src = I.s.bucket + bs;
      for (int k = tid; k < nbk; k += NT) {
        const int p = src[k];
        int r = 0;
        for (int j = 0; j < nbk; ++j) r += src[j] < p;
        I.s.bucket_sorted[bs + r] = p;
      }
      sorted = I.s.bucket_sorted + bs;
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
    for (int c0 = 0; c0 < S; c0 += NT) {
      const int s = c0 + tid;
      int d = CELLS_PER_TILE;
      if (s < S) {
        const bool in_range = s >= nl && s < nl + nr;
        const int pos = in_range ? os + (s - nl) : sorted[s < nl ? s : s - nr];
        const uint32_t k = knew[pos];
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
    for (int c0 = 0; c0 < S; c0 += NT) {
      const int s = c0 + tid;
      int d = CELLS_PER_TILE;
      int pos = 0;
      uint32_t k = 0;
      if (s < S) {
        const bool in_range = s >= nl && s < nl + nr;
        pos = in_range ? os + (s - nl) : sorted[s < nl ? s : s - nr];
        k = knew[pos];
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
        I.perm_out[dst] = pos;
        I.keys_out[dst] = k;
      }
      __syncthreads();
      if (tid <= CELLS_PER_TILE) {
        int add = 0;
#pragma unroll
        for (int k2 = 0; k2 < NW; ++k2) {
          add += wcnt[k2][tid];
          wcnt[k2][tid] = 0;
        }
        if (tid < CELLS_PER_TILE) running[tid] += add;
      }
      __syncthreads();
    }
    if (tid == 0) s_work[(it + 1) & 1] = wnext;
    __syncthreads();
  }
}

template <int D>
__global__ void permute_k(int64_t n, PBuf A, PBuf B, const int32_t *__restrict__ perm) {
  constexpr int NS = nstress<D>();
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int j = perm[q];
    B.key()[q] = A.key()[j];
    B.id()[q] = A.id()[j];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      B.off(k)[q] = A.off(k)[j];
      B.vel(k)[q] = A.vel(k)[j];
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      B.sig(i)[q] = A.sig(i)[j];
      B.eps(i)[q] = A.eps(i)[j];
    }
    B.mass()[q] = A.mass()[j];
    B.jm1()[q] = A.jm1()[j];
    B.epsp()[q] = A.epsp()[j];
    if (A.coh()) B.coh()[q] = A.coh()[j];
  }
}

template <bool ONE>
cudaError_t bin_launch(const GroupArgs &G, cudaStream_t st) {
  cudaError_t e = G.scan_one ? launch_dep(bin_scan_one<ONE>, G.ninst, SCAN1_T, 0, st, G)
                             : launch_dep(bin_scan_lb<ONE>, G.nblk_s, SCAN_T, 0, st, G);
  if (e == cudaSuccess) e = launch_dep(bin_bucket<ONE>, G.nblk_m, 256, 0, st, G);
  if (e == cudaSuccess)
    e = G.bin_t == 128 ? launch_dep(bin_tiles<ONE, 128>, G.grid * 2, 128, 0, st, G)
                       : launch_dep(bin_tiles<ONE, 256>, G.grid, 256, 0, st, G);
  return e;
}

}  // namespace

cudaError_t count_movers(const GroupArgs &G, cudaStream_t st) {
  if (G.ninst <= 0 || G.nblk_p <= 0) return cudaSuccess;
  bin_movers<<<G.nblk_p, 256, 0, st>>>(G);
  return cudaGetLastError();
}

cudaError_t bin_group(int dim, const GroupArgs &G, cudaStream_t st) {
  (void)dim;
  if (G.ninst <= 0 || G.nblk_p <= 0) return cudaSuccess;
  return G.ninst == 1 ? bin_launch<true>(G, st) : bin_launch<false>(G, st);
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
