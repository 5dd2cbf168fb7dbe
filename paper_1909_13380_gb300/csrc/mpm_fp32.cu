// mpm_fp32.cu -- FP32 mixed-precision explicit MPM step.
//
// Paper (arXiv 1909.13380): INTRODUCTION (particle <-> node transfers with the
// same shape functions, nodal values reset each step), CODE OVERVIEW (Node,
// Cell with linear quad/hex, Material, USF/USL), DATA STRUCTURES (a node
// aggregates the particles of all cells around it and must be protected
// against races -- the paper uses a mutex per node), ISOPARAMETRIC MESH
// (nodal velocity and frictional conditions).
//
// GPU design (replaces the per-node mutex), after the binning of mpm_bin.cu:
//   p2g_tile   one CTA per 4x4x4 (8x8) cell tile: loads the tile's particles
//              in binning order (coalesced), evaluates each particle's corner
//              contributions once, sums them per cell in a fixed sequential
//              order through a shared-memory staging buffer (compensated
//              sums), sums cells into the tile's node box and writes the box
//              to the tile's own slot -- no atomics, bit-reproducible;
//   node_tile  one CTA per tile: final nodal values of the box, summing the
//              slots of the (at most 2^D) tiles that share each node in
//              ascending tile order, then v = P/m, a = f/m + g, v' = v + a dt
//              and the boundary conditions; written to dense node arrays
//              (nodes shared by boxes get bit-identical values);
//   g2p        one thread per particle in binning order: FLIP velocity,
//              advection, strain, stress, volume and relocation into the new
//              cell, written in binning order so the next step reads
//              contiguously.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mpm_internal.h"

namespace mpm {
namespace {

constexpr int P2G_T = 128;  // threads per P2G CTA
constexpr int P2G_W = P2G_T / 32;
constexpr int NODE_T = 128;
constexpr int G2P_T = 256;

// Instance of item x: the largest i with prefix[i] <= x (prefix[0] = 0).
__device__ __forceinline__ int find_inst(const int32_t *prefix, int ninst, int x) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int next_tile(int32_t *ctr, int slot) {
  __shared__ int s_w;
  if (threadIdx.x == 0) s_w = atomicAdd(&ctr[slot], 1);
  __syncthreads();
  const int w = s_w;
  __syncthreads();
  return w;
}

// Start of warp w's share of [s, e): the first cell boundary at or after
// s + w (e - s) / NW, so that no cell is split between warps.
template <int NW>
__device__ __forceinline__ int warp_split(const uint32_t *keys, int s, int e, int w) {
  if (w <= 0) return s;
  if (w >= NW) return e;
  int p = s + (int)(((int64_t)(e - s) * w) / NW);
  if (p <= s) p = s + 1;
  const int lane = threadIdx.x & 31;
  for (;;) {
    if (p >= e) return e;
    const int q = p + lane;
    const bool brk = (q >= e) || (keys[q] != keys[q - 1]);
    const unsigned m = __ballot_sync(0xffffffffu, brk);
    if (m) return p + __ffs(m) - 1;
    p += 32;
  }
}

__device__ __forceinline__ void tile_coords(const Geo &g, int t, int tc[3]) {
  tc[0] = t % g.nt[0];
  tc[1] = (t / g.nt[0]) % g.nt[1];
  tc[2] = t / (g.nt[0] * g.nt[1]);
}

template <int D>
__device__ __forceinline__ void local_coords(uint32_t key, int lc[3]) {
  const int l = key & (CELLS_PER_TILE - 1);
  lc[0] = l % Tile<D>::TX;
  lc[1] = (l / Tile<D>::TX) % Tile<D>::TY;
  lc[2] = l / (Tile<D>::TX * Tile<D>::TY);
}

// Corner weights of the linear element at natural coordinates xi = 2u:
// w0[k] = (1 - xi_k)/2, w1[k] = (1 + xi_k)/2.  N_a and its gradient are
// products of these (shape_fn in mpm_device.cuh writes them out in full).
template <int D>
__device__ __forceinline__ void corner_weights(const float u[D], float w0[D], float w1[D]) {
#pragma unroll
  for (int k = 0; k < D; ++k) {
    w0[k] = 0.5f - u[k];
    w1[k] = 0.5f + u[k];
  }
}

template <int D>
__device__ __forceinline__ void corner_shape(int a, const float w0[D], const float w1[D], float inv_h, float &N,
                                             float G[D]) {
  float w[D];
#pragma unroll
  for (int k = 0; k < D; ++k) w[k] = ((a >> k) & 1) ? w1[k] : w0[k];
  N = w[0];
#pragma unroll
  for (int k = 1; k < D; ++k) N *= w[k];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    float g = ((a >> k) & 1) ? inv_h : -inv_h;
#pragma unroll
    for (int j = 0; j < D; ++j)
      if (j != k) g *= w[j];
    G[k] = g;
  }
}

// ---------------------------------------------------------------------------
// P2G: value index v = corner * NCH + channel; channels USL (m, P_k, f_k),
// MOM (m, P_k), FORCE (f_k), f_k = -V sum_j sig_kj dN/dx_j.
// ---------------------------------------------------------------------------
template <int D, int MODE>
constexpr size_t p2g_smem() {
  return sizeof(float) * (CELLS_PER_TILE * (1 << D) * p2g_channels<D, MODE>() + P2G_W * 32 * 33);
}

template <int D, int MODE>
__global__ void __launch_bounds__(P2G_T, 4) p2g_tile(GroupArgs G, int work_slot) {
  constexpr int NC = 1 << D;
  constexpr int NCH = p2g_channels<D, MODE>();
  constexpr int NV = NC * NCH;
  constexpr int NPASS = (NV + 31) / 32;
  constexpr int BN = box_nodes<D>();
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  constexpr bool HAS_M = MODE != P2G_FORCE;
  constexpr bool HAS_F = MODE != P2G_MOM;
  extern __shared__ float sm[];
  float *cellP = sm;  // [64][NV]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float *wst = sm + CELLS_PER_TILE * NV + warp * 32 * 33;  // [32][33]
  const int total = G.act_items[G.ninst];
  __shared__ InstArgs sI;

  for (;;) {
    const int wi = next_tile(G.work, work_slot);
    if (wi >= total) break;
    const int ii = find_inst(G.act_items, G.ninst, wi);
    copy_inst(G.inst, ii, &sI);
    for (int i = threadIdx.x; i < CELLS_PER_TILE * NV; i += P2G_T) cellP[i] = 0.f;
    __syncthreads();
    const InstArgs &I = sI;
    const Geo &g = I.geo;
    float *slots_out = MODE == P2G_FORCE ? I.s.slots2 : I.s.slots1;
    const int t = I.s.active[wi - G.act_items[ii]];
    const int s = I.new_start[t], e = I.new_start[t + 1];
    const int ws = warp_split<P2G_W>(I.keys_out, s, e, warp);
    const int we = warp_split<P2G_W>(I.keys_out, s, e, warp + 1);

    for (int b0 = ws; b0 < we; b0 += 32) {
      const int q = b0 + lane;
      const bool valid = q < we;
      const int nb = min(32, we - b0);
      int lc = CELLS_PER_TILE + lane;
      float w0[D], w1[D];
      float mm = 0.f, mv[D], sv[D][D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        w0[k] = w1[k] = mv[k] = 0.f;
#pragma unroll
        for (int j = 0; j < D; ++j) sv[k][j] = 0.f;
      }
      if (valid) {
        lc = I.keys_out[q] & (CELLS_PER_TILE - 1);
        const int j = I.perm_out[q];
        float u[D];
#pragma unroll
        for (int k = 0; k < D; ++k) u[k] = I.A.off(k)[j];
        corner_weights<D>(u, w0, w1);
        mm = I.A.mass()[j];
        if (HAS_M) {
#pragma unroll
          for (int k = 0; k < D; ++k) mv[k] = mm * I.A.vel(k)[j];
        }
        if (HAS_F) {
          // FORCE (USF) reads the stress updated earlier this step, stored in
          // binning order; USL reads the stress at the start of the step
          const PBuf &S = (MODE == P2G_FORCE) ? I.B : I.A;
          const int js = (MODE == P2G_FORCE) ? q : j;
          const float nV = -mm * g.inv_rho * (1.f + S.jm1()[js]);
          if (D == 3) {
            const float sxx = S.sig(0)[js], syy = S.sig(1)[js], szz = S.sig(2)[js];
            const float sxy = S.sig(3)[js], syz = S.sig(4)[js], sxz = S.sig(5)[js];
            const float t3[3][3] = {{sxx, sxy, sxz}, {sxy, syy, syz}, {sxz, syz, szz}};
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
              for (int b = 0; b < D; ++b) sv[a][b] = nV * t3[a][b];
          } else {
            const float sxx = S.sig(0)[js], syy = S.sig(1)[js], sxy = S.sig(3)[js];
            const float t2[2][2] = {{sxx, sxy}, {sxy, syy}};
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
              for (int b = 0; b < D; ++b) sv[a][b] = nV * t2[a][b];
          }
        }
      }
      // run ends inside this batch: lane k ends a run when the next lane's
      // cell differs or it is the last valid lane
      const int lc_next = __shfl_down_sync(0xffffffffu, lc, 1);
      const unsigned ends = __ballot_sync(0xffffffffu, valid && (lane == nb - 1 || lc_next != lc));

#pragma unroll
      for (int pass = 0; pass < NPASS; ++pass) {
        // stage this pass's values of my particle: wst[v][lane]
#pragma unroll
        for (int a = 0; a < NC; ++a) {
          if (a * NCH + NCH <= pass * 32 || a * NCH >= pass * 32 + 32) continue;
          float N, G[D];
          corner_shape<D>(a, w0, w1, g.inv_h, N, G);
#pragma unroll
          for (int ch = 0; ch < NCH; ++ch) {
            const int v = a * NCH + ch;
            if (v < pass * 32 || v >= pass * 32 + 32) continue;
            float val;
            if (HAS_M && ch == 0) {
              val = mm * N;
            } else if (HAS_M && ch <= D) {
              val = mv[ch - 1] * N;
            } else {
              const int k = HAS_M ? ch - 1 - D : ch;
              float f = 0.f;
#pragma unroll
              for (int jj = 0; jj < D; ++jj) f += sv[k][jj] * G[jj];
              val = f;
            }
            wst[(v - pass * 32) * 33 + lane] = val;
          }
        }
        __syncwarp();
        // lane = value index: sum the batch in particle order (at most 32
        // terms, plain FP32), flush at run ends
        const int v = pass * 32 + lane;
        const float *row = wst + lane * 33;
        float acc = 0.f;
#pragma unroll 8
        for (int k = 0; k < nb; ++k) {
          acc += row[k];
          if ((ends >> k) & 1u) {
            const int ck = __shfl_sync(0xffffffffu, lc, k);
            if (v < NV) cellP[ck * NV + v] += acc;
            acc = 0.f;
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();

    // cells -> node box (ascending local cell order), compensated; -> slot
    for (int b = threadIdx.x; b < BN; b += P2G_T) {
      const int bx = b % (TX + 1);
      const int by = (b / (TX + 1)) % (TY + 1);
      const int bz = D == 3 ? b / ((TX + 1) * (TY + 1)) : 0;
      TwoAcc<float> acc[NCH];
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) acc[ch].init();
#pragma unroll
      for (int dz = (D == 3 ? 1 : 0); dz >= 0; --dz)
#pragma unroll
        for (int dy = 1; dy >= 0; --dy)
#pragma unroll
          for (int dx = 1; dx >= 0; --dx) {
            const int cx = bx - dx, cy = by - dy, cz = bz - dz;
            if (cx < 0 || cx >= TX || cy < 0 || cy >= TY || cz < 0 || cz >= TZ) continue;
            const int cl = cx + TX * (cy + TY * cz);
            const int a = dx + 2 * dy + 4 * dz;
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) acc[ch].add(cellP[cl * NV + a * NCH + ch]);
          }
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) slots_out[((int64_t)t * NCH + ch) * BN + b] = acc[ch].value();
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Nodes
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ int node_faces(const Geo &g, const int I[3]) {
  int m = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (I[k] == 0) m |= 1 << (2 * k);
    if (I[k] == g.nc[k]) m |= 1 << (2 * k + 1);
  }
  return m;
}

// Sum channels of node I over the slots of every active tile whose box holds
// it, in ascending tile order (every tile computes a shared node the same way).
template <int D, int NOUT>
__device__ __forceinline__ void gather_node(const Geo &g, const int32_t *tile_start, const float *slots, int nch,
                                            const int I[3], const int tc[3], float out[NOUT]) {
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  constexpr int BN = box_nodes<D>();
  const int T[3] = {TX, TY, TZ};
  int lo[3], hi[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lo[k] = hi[k] = tc[k];
    if (k < D) {
      const int l = I[k] - tc[k] * T[k];
      if (l == 0 && tc[k] > 0) lo[k] = tc[k] - 1;
      if (l == T[k] && tc[k] + 1 < g.nt[k]) hi[k] = tc[k] + 1;
    }
  }
  TwoAcc<float> acc[NOUT];
#pragma unroll
  for (int c = 0; c < NOUT; ++c) acc[c].init();
  for (int z = lo[2]; z <= hi[2]; ++z)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int x = lo[0]; x <= hi[0]; ++x) {
        const int t2 = x + g.nt[0] * (y + g.nt[1] * z);
        if (tile_start[t2 + 1] <= tile_start[t2]) continue;
        const int bx = I[0] - x * TX, by = I[1] - y * TY, bz = D == 3 ? I[2] - z * TZ : 0;
        const int bl = bx + (TX + 1) * (by + (TY + 1) * bz);
#pragma unroll
        for (int c = 0; c < NOUT; ++c) acc[c].add(slots[((int64_t)t2 * nch + c) * BN + bl]);
      }
#pragma unroll
  for (int c = 0; c < NOUT; ++c) out[c] = acc[c].value();
}

template <int D, int NMODE>
__global__ void __launch_bounds__(NODE_T) node_tile(GroupArgs G, int work_slot) {
  constexpr int BN = box_nodes<D>();
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  constexpr int NCH1 = NMODE == NODE_USL ? 1 + 2 * D : 1 + D;
  const int total = G.act_items[G.ninst];
  __shared__ InstArgs sI;
  for (;;) {
    const int wi = next_tile(G.work, work_slot);
    if (wi >= total) break;
    const int ii = find_inst(G.act_items, G.ninst, wi);
    copy_inst(G.inst, ii, &sI);
    __syncthreads();
    const InstArgs &I = sI;
    const Geo &g = I.geo;
    const int t = I.s.active[wi - G.act_items[ii]];
    int tc[3];
    tile_coords(g, t, tc);
    for (int b = threadIdx.x; b < BN; b += NODE_T) {
      const int bx = b % (TX + 1);
      const int by = (b / (TX + 1)) % (TY + 1);
      const int bz = D == 3 ? b / ((TX + 1) * (TY + 1)) : 0;
      const int Ig[3] = {tc[0] * TX + bx, tc[1] * TY + by, D == 3 ? tc[2] * TZ + bz : 0};
      bool inside = true;
#pragma unroll
      for (int k = 0; k < D; ++k) inside = inside && Ig[k] <= g.nc[k];
      if (!inside) continue;
      float v[D], a[D], vn[D];
#pragma unroll
      for (int k = 0; k < D; ++k) v[k] = a[k] = vn[k] = 0.f;
      float c1[1 + 2 * D];
      if (NMODE == NODE_USL)
        gather_node<D, 1 + 2 * D>(g, I.new_start, I.s.slots1, NCH1, Ig, tc, c1);
      else
        gather_node<D, 1 + D>(g, I.new_start, I.s.slots1, NCH1, Ig, tc, c1);
      const float m = c1[0];
      const int faces = node_faces<D>(g, Ig);
      if (m > g.mass_tol) {
        const float inv_m = 1.f / m;
#pragma unroll
        for (int k = 0; k < D; ++k) v[k] = c1[1 + k] * inv_m;
        if (NMODE == NODE_USL) {
#pragma unroll
          for (int k = 0; k < D; ++k) {
            a[k] = c1[1 + D + k] * inv_m + g.g[k];
            vn[k] = v[k] + a[k] * g.dt;
          }
          bc_full<D, float>(faces, g.bc, g.mu, g.dt, v, a, vn);
        } else if (NMODE == NODE_USF_V) {
          bc_velocity<D, float>(faces, g.bc, v);
        } else {
          float f[D];
          gather_node<D, D>(g, I.new_start, I.s.slots2, D, Ig, tc, f);
          bc_velocity<D, float>(faces, g.bc, v);
#pragma unroll
          for (int k = 0; k < D; ++k) {
            a[k] = f[k] * inv_m + g.g[k];
            vn[k] = v[k] + a[k] * g.dt;
          }
          bc_full<D, float>(faces, g.bc, g.mu, g.dt, v, a, vn);
        }
      }
      const int gi = Ig[0] + I.ns0 * Ig[1] + I.ns1 * Ig[2];
      const float *w = NMODE == NODE_USF_V ? v : vn;
      if (D == 3) {
        I.s.node[2 * gi] = make_float4(w[0], w[1], w[D - 1], 0.f);
        I.s.node[2 * gi + 1] = make_float4(a[0], a[1], a[D - 1], 0.f);
      } else {
        I.s.node[gi] = make_float4(w[0], w[1], a[0], a[1]);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// G2P: one thread per particle in binning order
// ---------------------------------------------------------------------------
template <int D, int GMODE>
__global__ void __launch_bounds__(G2P_T, 3) g2p(GroupArgs G) {
  constexpr int NC = 1 << D;
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  constexpr int NS = nstress<D>();
  __shared__ InstArgs sI;
  const int ii = find_inst(G.pblk, G.ninst, blockIdx.x);
  copy_inst(G.inst, ii, &sI);
  __syncthreads();
  const InstArgs &I = sI;
  const Geo &g = I.geo;
  const int64_t q = (int64_t)(blockIdx.x - G.pblk[ii]) * G2P_T + threadIdx.x;
  if (q >= I.n) return;
  const int j = I.perm_out[q];
  const int dead_start = I.s.ctr[C_DEAD_START];
  if (q >= dead_start) {  // left the mesh earlier: carried over unchanged
    if (GMODE != G2P_USF_STRESS) {
      I.B.key()[q] = I.A.key()[j];
      I.B.id()[q] = I.A.id()[j];
      I.B.mass()[q] = I.A.mass()[j];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        I.B.off(k)[q] = I.A.off(k)[j];
        I.B.vel(k)[q] = I.A.vel(k)[j];
      }
      if (I.A.coh()) I.B.coh()[q] = I.A.coh()[j];
    }
    if (GMODE != G2P_USF_ADVECT) {
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        I.B.sig(i)[q] = I.A.sig(i)[j];
        I.B.eps(i)[q] = I.A.eps(i)[j];
      }
      I.B.jm1()[q] = I.A.jm1()[j];
      I.B.epsp()[q] = I.A.epsp()[j];
    }
    return;
  }
  const uint32_t key = I.keys_out[q];
  const int t = key >> LOCAL_BITS;
  int tc[3], lc[3];
  tile_coords(g, t, tc);
  local_coords<D>(key, lc);
  int cell[3] = {tc[0] * TX + lc[0], tc[1] * TY + lc[1], D == 3 ? tc[2] * TZ + lc[2] : 0};
  float u[D], w0[D], w1[D];
#pragma unroll
  for (int k = 0; k < D; ++k) u[k] = I.A.off(k)[j];
  corner_weights<D>(u, w0, w1);
  float dv[D], vb[D], L[D][D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    dv[k] = vb[k] = 0.f;
#pragma unroll
    for (int l = 0; l < D; ++l) L[k][l] = 0.f;
  }
  const int gi0 = cell[0] + I.ns0 * cell[1] + I.ns1 * cell[2];
#pragma unroll
  for (int a = 0; a < NC; ++a) {
    float N, G[D];
    corner_shape<D>(a, w0, w1, g.inv_h, N, G);
    const int gi = gi0 + (a & 1) + I.ns0 * ((a >> 1) & 1) + (D == 3 ? I.ns1 * ((a >> 2) & 1) : 0);
    float nv[D], na[D];
    if (D == 3) {
      const float4 r0 = I.s.node[2 * gi];
      nv[0] = r0.x;
      nv[1] = r0.y;
      nv[D - 1] = r0.z;
      if (GMODE != G2P_USF_STRESS) {
        const float4 r1 = I.s.node[2 * gi + 1];
        na[0] = r1.x;
        na[1] = r1.y;
        na[D - 1] = r1.z;
      }
    } else {
      const float4 r0 = I.s.node[gi];
      nv[0] = r0.x;
      nv[1] = r0.y;
      na[0] = r0.z;
      na[1] = r0.w;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (GMODE != G2P_USF_STRESS) {
        dv[k] += N * na[k];
        vb[k] += N * nv[k];
      }
#pragma unroll
      for (int l = 0; l < D; ++l) L[k][l] += nv[k] * G[l];
    }
  }

  // Every load of the particle's state is issued before the first store: the
  // compiler cannot tell A from B, so a load placed after a store would wait
  // for the value before it (one memory latency per field).
  constexpr bool KIN = GMODE != G2P_USF_STRESS, STR = GMODE != G2P_USF_ADVECT;
  float v0[D], sg[6], ep[6], jm1 = 0.f, epsp = 0.f, mass = 0.f, coh = I.mat.c;
  int32_t pid = 0;
  const bool has_coh = I.A.coh() != nullptr;
  if (KIN) {
#pragma unroll
    for (int k = 0; k < D; ++k) v0[k] = I.A.vel(k)[j];
    mass = I.A.mass()[j];
    pid = I.A.id()[j];
  }
  if (has_coh && (KIN || STR)) coh = I.A.coh()[j];
  if (STR) {
#pragma unroll
    for (int i = 0; i < 6; ++i) sg[i] = ep[i] = 0.f;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      sg[i] = I.A.sig(i)[j];
      ep[i] = I.A.eps(i)[j];
    }
    jm1 = I.A.jm1()[j];
    epsp = I.A.epsp()[j];
  }

  int status = 0;
  // FLIP velocity, advection in cell units, relocation
  if (KIN) {
    bool dead = false;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float vk = v0[k] + g.dt * dv[k];
      I.B.vel(k)[q] = vk;
      if (!isfinite(vk)) status |= ST_NONFINITE;
      float un = u[k] + g.dt * vb[k] * g.inv_h;
      if (!isfinite(un)) {
        status |= ST_NONFINITE;
        dead = true;
        un = 0.f;
      }
      // one cell crossing is an exact subtraction (Sterbenz), so the offset
      // stays in [-0.5, 0.5) and the cell is exact
      if (un >= 0.5f) {
        un -= 1.f;
        cell[k] += 1;
      } else if (un < -0.5f) {
        un += 1.f;
        cell[k] -= 1;
      }
      if (!(un >= -0.5f && un < 0.5f)) {  // more than one cell per step
        const float sh = floorf(un + 0.5f);
        un -= sh;
        cell[k] += (int)sh;
        if (un >= 0.5f) {
          un -= 1.f;
          cell[k] += 1;
        } else if (un < -0.5f) {
          un += 1.f;
          cell[k] -= 1;
        }
      }
      if (cell[k] < 0 || cell[k] >= g.nc[k]) dead = true;
      I.B.off(k)[q] = un;
    }
    uint32_t nkey = g.dead_key;
    if (!dead) {
      const int t2 = cell[0] / TX + g.nt[0] * (cell[1] / TY + g.nt[1] * (D == 3 ? cell[2] / TZ : 0));
      const int l2 = cell[0] % TX + TX * (cell[1] % TY + TY * (D == 3 ? cell[2] % TZ : 0));
      nkey = (uint32_t)t2 * CELLS_PER_TILE + (uint32_t)l2;
    } else {
      status |= ST_LEFT_MESH;
    }
    I.B.key()[q] = nkey;
    I.B.mass()[q] = mass;
    I.B.id()[q] = pid;
    if (has_coh) I.B.coh()[q] = coh;
  }
  if (STR) {
    // strain increment de = sym(L) dt, strain, volume ratio, stress
    float de[6] = {0, 0, 0, 0, 0, 0};
    de[0] = L[0][0] * g.dt;
    de[1] = L[1][1] * g.dt;
    de[3] = 0.5f * (L[0][1] + L[1][0]) * g.dt;
    if (D == 3) {
      de[2] = L[D - 1][D - 1] * g.dt;
      de[4] = 0.5f * (L[1][D - 1] + L[D - 1][1]) * g.dt;
      de[5] = 0.5f * (L[0][D - 1] + L[D - 1][0]) * g.dt;
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) I.B.eps(i)[q] = ep[i] + de[i];
    // V = V0 (1 + jm1):  (1 + jm1)(1 + tr) - 1 = jm1 + tr + jm1 tr
    const float tr = de[0] + de[1] + de[2];
    I.B.jm1()[q] = jm1 + (tr + jm1 * tr);
    material_update(I.mat, I.matd, coh, sg, de, epsp);
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      I.B.sig(i)[q] = sg[i];
      if (!isfinite(sg[i])) status |= ST_NONFINITE;
    }
    I.B.epsp()[q] = epsp;
  }
  if (status) atomicOr(&I.s.ctr[C_STATUS], status);
}

template <int D, int MODE>
cudaError_t launch_p2g(const GroupArgs &G, int work_slot, cudaStream_t st) {
  p2g_tile<D, MODE><<<G.grid, P2G_T, p2g_smem<D, MODE>(), st>>>(G, work_slot);
  return cudaGetLastError();
}

template <int D, int MODE>
cudaError_t prepare_p2g() {
  return cudaFuncSetAttribute(p2g_tile<D, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)p2g_smem<D, MODE>());
}

template <int D, int NMODE>
cudaError_t launch_node(const GroupArgs &G, int work_slot, cudaStream_t st) {
  node_tile<D, NMODE><<<G.grid, NODE_T, 0, st>>>(G, work_slot);
  return cudaGetLastError();
}

template <int D, int GMODE>
cudaError_t launch_g2p(const GroupArgs &G, cudaStream_t st) {
  g2p<D, GMODE><<<G.nblk_p, G2P_T, 0, st>>>(G);
  return cudaGetLastError();
}

template <int D>
cudaError_t step_dim(int scheme, const GroupArgs &G, cudaEvent_t *ev, cudaStream_t st) {
  cudaError_t e;
  // phase events 0 (start) and 1 (after binning) are recorded by the
  // caller; 2.. follow each kernel here
  if (scheme == 1) {  // USL
    if ((e = launch_p2g<D, P2G_USL>(G, W_P2G, st)) != cudaSuccess) return e;
    if ((e = phase_mark(ev, 2, st)) != cudaSuccess) return e;
    if ((e = launch_node<D, NODE_USL>(G, W_NODE, st)) != cudaSuccess) return e;
    if ((e = phase_mark(ev, 3, st)) != cudaSuccess) return e;
    if ((e = launch_g2p<D, G2P_USL>(G, st)) != cudaSuccess) return e;
    return phase_mark(ev, 4, st);
  }
  // USF
  if ((e = launch_p2g<D, P2G_MOM>(G, W_P2G, st)) != cudaSuccess) return e;
  if ((e = phase_mark(ev, 2, st)) != cudaSuccess) return e;
  if ((e = launch_node<D, NODE_USF_V>(G, W_NODE, st)) != cudaSuccess) return e;
  if ((e = phase_mark(ev, 3, st)) != cudaSuccess) return e;
  if ((e = launch_g2p<D, G2P_USF_STRESS>(G, st)) != cudaSuccess) return e;
  if ((e = phase_mark(ev, 4, st)) != cudaSuccess) return e;
  if ((e = launch_p2g<D, P2G_FORCE>(G, W_P2G2, st)) != cudaSuccess) return e;
  if ((e = phase_mark(ev, 5, st)) != cudaSuccess) return e;
  if ((e = launch_node<D, NODE_USF_A>(G, W_NODE2, st)) != cudaSuccess) return e;
  if ((e = phase_mark(ev, 6, st)) != cudaSuccess) return e;
  if ((e = launch_g2p<D, G2P_USF_ADVECT>(G, st)) != cudaSuccess) return e;
  return phase_mark(ev, 7, st);
}

// ---------------------------------------------------------------------------
// Conservation sums (FP64, deterministic two-level), export
// ---------------------------------------------------------------------------
constexpr int CONS_BLOCKS = 1024;
constexpr int CONS_VALS = 7;

template <int D>
__global__ void cons_partial(int64_t n, PBuf P, uint32_t dead_key, float inv_rho, double *part) {
  constexpr int NS = nstress<D>();
  double acc[CONS_VALS] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    if (P.key()[q] >= dead_key) continue;
    const double m = P.mass()[q];
    acc[0] += m;
    double ke = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double v = P.vel(k)[q];
      acc[1 + k] += m * v;
      ke += v * v;
    }
    acc[4] += 0.5 * m * ke;
    double se = 0;
#pragma unroll
    for (int i = 0; i < NS; ++i) se += (i >= 3 ? 2.0 : 1.0) * (double)P.sig(i)[q] * (double)P.eps(i)[q];
    const double vol = m * (double)inv_rho * (1.0 + (double)P.jm1()[q]);
    acc[5] += 0.5 * vol * se;
    acc[6] += 1.0;
  }
  __shared__ double red[CONS_VALS][256];
#pragma unroll
  for (int c = 0; c < CONS_VALS; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int c = 0; c < CONS_VALS; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < CONS_VALS) part[blockIdx.x * CONS_VALS + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void cons_final(const double *part, int nb, double *out) {
  if (threadIdx.x < CONS_VALS) {
    double s = 0;
    for (int b = 0; b < nb; ++b) s += part[b * CONS_VALS + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

template <int D>
__global__ void export_k(int64_t n, PBuf P, Geo g, double o0, double o1, double o2, double h, double rho,
                         double *pos, double *vel, double *sig, double *eps, double *vol, double *epsp,
                         int64_t *cell) {
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  constexpr int NS = nstress<D>();
  const double org[3] = {o0, o1, o2};
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t id = P.id()[q];
    const uint32_t key = P.key()[q];
    const bool dead = key >= g.dead_key;
    int c[3] = {0, 0, 0};
    if (!dead) {
      int tc[3], lc[3];
      tile_coords(g, (int)(key >> LOCAL_BITS), tc);
      local_coords<D>(key, lc);
      c[0] = tc[0] * TX + lc[0];
      c[1] = tc[1] * TY + lc[1];
      c[2] = D == 3 ? tc[2] * TZ + lc[2] : 0;
    }
    if (pos)
#pragma unroll
      for (int k = 0; k < D; ++k)
        pos[id * D + k] = dead ? __longlong_as_double(0x7ff8000000000000ll)
                               : org[k] + ((double)c[k] + 0.5 + (double)P.off(k)[q]) * h;
    if (vel)
#pragma unroll
      for (int k = 0; k < D; ++k) vel[id * D + k] = P.vel(k)[q];
    if (sig || eps) {
      double s6[6] = {0, 0, 0, 0, 0, 0}, e6[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        s6[i] = P.sig(i)[q];
        e6[i] = P.eps(i)[q];
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        if (sig) sig[id * 6 + i] = s6[i];
        if (eps) eps[id * 6 + i] = e6[i];
      }
    }
    if (vol) vol[id] = (double)P.mass()[q] / rho * (1.0 + (double)P.jm1()[q]);
    if (epsp) epsp[id] = P.epsp()[q];
    if (cell) cell[id] = dead ? -1 : (int64_t)c[0] + (int64_t)g.nc[0] * ((int64_t)c[1] + (int64_t)g.nc[1] * c[2]);
  }
}

__global__ void mat_update_f32_k(MatConst<float> m, MatConst<double> md, int64_t n, const float *sig,
                                 const float *de, const float *coh, float *out, float *depsp) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float s[6], d[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      s[k] = sig[i * 6 + k];
      d[k] = de[i * 6 + k];
    }
    float ep = 0.f;
    material_update(m, md, coh ? coh[i] : m.c, s, d, ep);
#pragma unroll
    for (int k = 0; k < 6; ++k) out[i * 6 + k] = s[k];
    if (depsp) depsp[i] = ep;
  }
}

}  // namespace

cudaError_t f32_prepare(int dim) {
  cudaError_t e;
  if (dim == 3) {
    if ((e = prepare_p2g<3, P2G_USL>()) != cudaSuccess) return e;
    if ((e = prepare_p2g<3, P2G_MOM>()) != cudaSuccess) return e;
    return prepare_p2g<3, P2G_FORCE>();
  }
  if ((e = prepare_p2g<2, P2G_USL>()) != cudaSuccess) return e;
  if ((e = prepare_p2g<2, P2G_MOM>()) != cudaSuccess) return e;
  return prepare_p2g<2, P2G_FORCE>();
}

__global__ void gather_status_k(const InstArgs *tab, int ninst, int32_t *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ninst; i += gridDim.x * blockDim.x)
    out[i] = tab[i].s.ctr[C_STATUS];
}

cudaError_t gather_status(const InstArgs *tab, int ninst, int32_t *out, cudaStream_t st) {
  if (ninst <= 0) return cudaSuccess;
  gather_status_k<<<(ninst + 255) / 256, 256, 0, st>>>(tab, ninst, out);
  return cudaGetLastError();
}

cudaError_t f32_group_step(int dim, int scheme, const GroupArgs &G, cudaEvent_t *ev, cudaStream_t st) {
  if (G.ninst <= 0 || G.nblk_p <= 0) return cudaSuccess;
  return dim == 3 ? step_dim<3>(scheme, G, ev, st) : step_dim<2>(scheme, G, ev, st);
}

cudaError_t f32_conservation(int dim, int64_t n, const PBuf &P, uint32_t dead_key, float inv_rho, double *d_out,
                             double *d_partials, cudaStream_t st) {
  if (dim == 3)
    cons_partial<3><<<CONS_BLOCKS, 256, 0, st>>>(n, P, dead_key, inv_rho, d_partials);
  else
    cons_partial<2><<<CONS_BLOCKS, 256, 0, st>>>(n, P, dead_key, inv_rho, d_partials);
  cons_final<<<1, 32, 0, st>>>(d_partials, CONS_BLOCKS, d_out);
  return cudaGetLastError();
}

cudaError_t f32_export(int dim, int64_t n, const PBuf &P, const Geo &g, const double origin[3], double h,
                       double rho, double *pos, double *vel, double *sig, double *eps, double *vol, double *epsp,
                       int64_t *cell, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (dim == 3)
    export_k<3><<<blocks, 256, 0, st>>>(n, P, g, origin[0], origin[1], origin[2], h, rho, pos, vel, sig, eps, vol,
                                        epsp, cell);
  else
    export_k<2><<<blocks, 256, 0, st>>>(n, P, g, origin[0], origin[1], origin[2], h, rho, pos, vel, sig, eps, vol,
                                        epsp, cell);
  return cudaGetLastError();
}

cudaError_t material_update_f32(const MatConst<float> &m, const MatConst<double> &md, int64_t n, const float *sig,
                                const float *de, const float *coh, float *out, float *depsp, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  mat_update_f32_k<<<blocks, 256, 0, st>>>(m, md, n, sig, de, coh, out, depsp);
  return cudaGetLastError();
}

}  // namespace mpm
