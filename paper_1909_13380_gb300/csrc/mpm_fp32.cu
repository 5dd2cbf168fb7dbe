// mpm_fp32.cu -- FP32 mixed-precision explicit MPM step on tiles of 256 cells.
//
// Paper (arXiv 1909.13380): INTRODUCTION (particle <-> node transfers with the
// same shape functions, nodal values reset each step), CODE OVERVIEW (Node,
// Cell with linear quad/hex, Material, USF/USL), DATA STRUCTURES (nodal
// updates aggregate the particles of all cells around a node and must be
// protected against races -- the paper uses a mutex per node),
// ISOPARAMETRIC MESH (nodal velocity and frictional conditions).
//
// GPU design (replaces the per-node mutex): particles are binned by a
// tile-major cell key (mpm_sort.cu).  One CTA owns one tile:
//   p2g_tile   loads the tile's particles in key order (coalesced), evaluates
//              every particle's corner contributions once, reduces them per
//              cell in a fixed sequential order through a shared-memory
//              staging buffer (compensated sums), sums cells into the tile's
//              node box, and writes that box to the tile's own slot -- no
//              atomics, no zeroing pass, bit-reproducible.
//   g2p_tile   rebuilds the final node values of its box by summing the slots
//              of the (at most 2^D) tiles that share each node, in ascending
//              tile order (so every tile sees bit-identical node values),
//              applies the boundary conditions, then streams its particles
//              once: FLIP velocity, advection, strain, stress, volume and
//              relocation into the new cell, writing the new state in key
//              order so the next step's reads stay coalesced.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mpm_internal.h"

namespace mpm {
namespace {

constexpr int NT = 256;  // threads per tile CTA
constexpr int NWARP = NT / 32;

template <int D>
struct P2GArgs {
  Geo geo;
  PBuf A;              // particle storage (read through perm)
  PBuf B;              // FORCE mode: stress/volume already updated, key order
  const uint32_t *keys;
  const int32_t *perm;
  const int32_t *tile_start;
  const int32_t *active;
  int32_t *ctr;
  int work_slot;
  float *slots;
};

template <int D>
struct G2PArgs {
  Geo geo;
  MatConst<float> mat;
  MatConst<double> matd;
  PBuf A, B;
  const uint32_t *keys;
  const int32_t *perm;
  const int32_t *tile_start;
  const int32_t *active;
  int32_t *ctr;
  int work_slot;
  const float *slots1;  // m, P (and f_int in USL)
  const float *slots2;  // f_int (USF advect)
  int nch1;
};

__device__ __forceinline__ int next_tile(int32_t *ctr, int slot) {
  __shared__ int s_w;
  if (threadIdx.x == 0) s_w = atomicAdd(&ctr[slot], 1);
  __syncthreads();
  const int w = s_w;
  __syncthreads();
  return w;
}

// Start of warp w's share of [s, e): the first cell boundary at or after
// s + w (e - s) / NWARP, so that no cell is split between warps.
__device__ __forceinline__ int warp_split(const uint32_t *keys, int s, int e, int w) {
  if (w <= 0) return s;
  if (w >= NWARP) return e;
  int p = s + (int)(((int64_t)(e - s) * w) / NWARP);
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

template <int D>
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

// ---------------------------------------------------------------------------
// P2G: contributions of a particle to its cell's 2^D nodes.
// value index v = corner * NCH + channel;  channels: USL (m, P_k, f_k),
// MOM (m, P_k), FORCE (f_k) with f_k = -V sum_j sig_kj dN/dx_j.
// ---------------------------------------------------------------------------
template <int D, int MODE>
__global__ void __launch_bounds__(NT, 2) p2g_tile(P2GArgs<D> A) {
  constexpr int NC = 1 << D;
  constexpr int NCH = p2g_channels<D, MODE>();
  constexpr int NV = NC * NCH;
  constexpr int NPASS = (NV + 31) / 32;
  constexpr int BN = box_nodes<D>();
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY;
  constexpr bool HAS_M = MODE != P2G_FORCE;
  constexpr bool HAS_F = MODE != P2G_MOM;
  extern __shared__ float sm[];
  float *cellP = sm;                               // [256][NV]
  float *stage = sm + CELLS_PER_TILE * NV;         // [NWARP][32][33]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float *wst = stage + warp * 32 * 33;
  const Geo &g = A.geo;

  for (;;) {
    const int wi = next_tile(A.ctr, A.work_slot);
    if (wi >= A.ctr[0]) break;
    const int t = A.active[wi];
    const int s = A.tile_start[t], e = A.tile_start[t + 1];
    for (int i = threadIdx.x; i < CELLS_PER_TILE * NV; i += NT) cellP[i] = 0.f;
    const int ws = warp_split(A.keys, s, e, warp);
    const int we = warp_split(A.keys, s, e, warp + 1);
    __syncthreads();

    for (int b0 = ws; b0 < we; b0 += 32) {
      const int q = b0 + lane;
      const bool valid = q < we;
      const int nb = min(32, we - b0);
      int lc = CELLS_PER_TILE + lane;
      float N[NC], G[NC][D];
      float mm = 0.f, mv[D], sv[D][D];
      if (valid) {
        const uint32_t key = A.keys[q];
        lc = key & (CELLS_PER_TILE - 1);
        const int j = A.perm[q];
        float xi[D];
#pragma unroll
        for (int k = 0; k < D; ++k) xi[k] = 2.f * A.A.off[k][j];
        shape_fn<D, float>(xi, g.inv_h, N, G);
        if (HAS_M) {
          mm = A.A.mass[j];
#pragma unroll
          for (int k = 0; k < D; ++k) mv[k] = mm * A.A.vel[k][j];
        }
        if (HAS_F) {
          const PBuf &S = (MODE == P2G_FORCE) ? A.B : A.A;
          const int js = (MODE == P2G_FORCE) ? q : j;
          const float nV = -S.vol[js];
          if (D == 3) {
            const float sxx = S.sig[0][js], syy = S.sig[1][js], szz = S.sig[2][js];
            const float sxy = S.sig[3][js], syz = S.sig[4][js], sxz = S.sig[5][js];
            const float t3[3][3] = {{sxx, sxy, sxz}, {sxy, syy, syz}, {sxz, syz, szz}};
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
              for (int b = 0; b < D; ++b) sv[a][b] = nV * t3[a][b];
          } else {
            const float sxx = S.sig[0][js], syy = S.sig[1][js], sxy = S.sig[3][js];
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
        // stage this pass's 32 values of my particle: wst[v][lane]
#pragma unroll
        for (int vv = 0; vv < 32; ++vv) {
          const int v = pass * 32 + vv;
          if (v < NV) {
            const int a = v / NCH, ch = v % NCH;
            float val = 0.f;
            if (valid) {
              if (HAS_M && ch == 0) {
                val = mm * N[a];
              } else if (HAS_M && ch <= D) {
                val = mv[ch - 1] * N[a];
              } else {
                const int k = HAS_M ? ch - 1 - D : ch;
                float f = 0.f;
#pragma unroll
                for (int jj = 0; jj < D; ++jj) f += sv[k][jj] * G[a][jj];
                val = f;
              }
            }
            wst[vv * 33 + lane] = val;
          }
        }
        __syncwarp();
        // lane = value index: sum the batch in particle order, flush at run ends
        const int v = pass * 32 + lane;
        TwoAcc<float> acc;
        acc.init();
        for (int k = 0; k < nb; ++k) {
          if (v < NV) acc.add(wst[lane * 33 + k]);
          if ((ends >> k) & 1u) {
            const int ck = __shfl_sync(0xffffffffu, lc, k);
            if (v < NV) cellP[ck * NV + v] += acc.value();
            acc.init();
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();

    // cells -> node box (ascending local cell order), compensated; -> slot
    for (int b = threadIdx.x; b < BN; b += NT) {
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
            if (cx < 0 || cx >= TX || cy < 0 || cy >= TY || cz < 0 || cz >= Tile<D>::TZ) continue;
            const int cl = cx + TX * (cy + TY * cz);
            const int a = dx + 2 * dy + 4 * dz;
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) acc[ch].add(cellP[cl * NV + a * NCH + ch]);
          }
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) A.slots[((int64_t)t * NCH + ch) * BN + b] = acc[ch].value();
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// G2P
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

// Sum channel `ch` of node I over the slots of every active tile whose box
// holds it, in ascending tile order.
template <int D>
__device__ __forceinline__ void gather_node(const Geo &g, const int32_t *tile_start, const float *slots,
                                            int nch, const int I[3], const int tc[3], float *out,
                                            int nout) {
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
  TwoAcc<float> acc[2 * 3 + 1];
  for (int c = 0; c < nout; ++c) acc[c].init();
  for (int z = lo[2]; z <= hi[2]; ++z)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int x = lo[0]; x <= hi[0]; ++x) {
        const int t2 = x + g.nt[0] * (y + g.nt[1] * z);
        if (tile_start[t2 + 1] <= tile_start[t2]) continue;
        const int bx = I[0] - x * TX, by = I[1] - y * TY, bz = D == 3 ? I[2] - z * TZ : 0;
        if (bx < 0 || bx > TX || by < 0 || by > TY || bz < 0 || bz > (D == 3 ? TZ : 0)) continue;
        const int bl = bx + (TX + 1) * (by + (TY + 1) * bz);
        for (int c = 0; c < nout; ++c) acc[c].add(slots[((int64_t)t2 * nch + c) * BN + bl]);
      }
  for (int c = 0; c < nout; ++c) out[c] = acc[c].value();
}

template <int D, int GMODE>
__global__ void __launch_bounds__(NT, 2) g2p_tile(G2PArgs<D> A) {
  constexpr int NC = 1 << D;
  constexpr int BN = box_nodes<D>();
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  constexpr int NS = nstress<D>();
  __shared__ float sV[BN][D];   // v' (USL, USF advect) or v (USF stress)
  __shared__ float sA[BN][D];   // a
  const Geo &g = A.geo;

  for (;;) {
    const int wi = next_tile(A.ctr, A.work_slot);
    if (wi >= A.ctr[0]) break;
    const int t = A.active[wi];
    const int s = A.tile_start[t], e = A.tile_start[t + 1];
    int tc[3];
    tile_coords<D>(g, t, tc);

    // node box: final nodal values and boundary conditions
    for (int b = threadIdx.x; b < BN; b += NT) {
      const int bx = b % (TX + 1);
      const int by = (b / (TX + 1)) % (TY + 1);
      const int bz = D == 3 ? b / ((TX + 1) * (TY + 1)) : 0;
      const int I[3] = {tc[0] * TX + bx, tc[1] * TY + by, D == 3 ? tc[2] * TZ + bz : 0};
      float v[D], a[D], vn[D];
#pragma unroll
      for (int k = 0; k < D; ++k) v[k] = a[k] = vn[k] = 0.f;
      bool inside = true;
#pragma unroll
      for (int k = 0; k < D; ++k) inside = inside && I[k] <= g.nc[k];
      if (inside) {
        float ch1[1 + 2 * D];
        const int n1 = GMODE == G2P_USL ? 1 + 2 * D : 1 + D;
        gather_node<D>(g, A.tile_start, A.slots1, A.nch1, I, tc, ch1, n1);
        const float m = ch1[0];
        const int faces = node_faces<D>(g, I);
        if (m > g.mass_tol) {
          const float inv_m = 1.f / m;
#pragma unroll
          for (int k = 0; k < D; ++k) v[k] = ch1[1 + k] * inv_m;
          if (GMODE == G2P_USL) {
#pragma unroll
            for (int k = 0; k < D; ++k) {
              a[k] = ch1[1 + D + k] * inv_m + g.g[k];
              vn[k] = v[k] + a[k] * g.dt;
            }
            bc_full<D, float>(faces, g.bc, g.mu, g.dt, v, a, vn);
          } else if (GMODE == G2P_USF_STRESS) {
            bc_velocity<D, float>(faces, g.bc, v);
          } else {
            float f[3];
            gather_node<D>(g, A.tile_start, A.slots2, D, I, tc, f, D);
            bc_velocity<D, float>(faces, g.bc, v);
#pragma unroll
            for (int k = 0; k < D; ++k) {
              a[k] = f[k] * inv_m + g.g[k];
              vn[k] = v[k] + a[k] * g.dt;
            }
            bc_full<D, float>(faces, g.bc, g.mu, g.dt, v, a, vn);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        sV[b][k] = GMODE == G2P_USF_STRESS ? v[k] : vn[k];
        sA[b][k] = a[k];
      }
    }
    __syncthreads();

    for (int q = s + threadIdx.x; q < e; q += NT) {
      const uint32_t key = A.keys[q];
      const int j = A.perm[q];
      int lc[3];
      local_coords<D>(key, lc);
      float u[D], xi[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        u[k] = A.A.off[k][j];
        xi[k] = 2.f * u[k];
      }
      float N[NC], G[NC][D];
      shape_fn<D, float>(xi, g.inv_h, N, G);
      float dv[D], vb[D], L[D][D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        dv[k] = vb[k] = 0.f;
#pragma unroll
        for (int l = 0; l < D; ++l) L[k][l] = 0.f;
      }
#pragma unroll
      for (int a = 0; a < NC; ++a) {
        const int b = (lc[0] + (a & 1)) + (TX + 1) * ((lc[1] + ((a >> 1) & 1)) + (TY + 1) * (D == 3 ? lc[2] + ((a >> 2) & 1) : 0));
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float vk = sV[b][k];
          if (GMODE != G2P_USF_STRESS) {
            dv[k] += N[a] * sA[b][k];
            vb[k] += N[a] * vk;
          }
#pragma unroll
          for (int l = 0; l < D; ++l) L[k][l] += vk * G[a][l];
        }
      }

      int status = 0;
      if (GMODE != G2P_USF_ADVECT) {
        // strain increment, volume, stress
        float de[6] = {0, 0, 0, 0, 0, 0};
        de[0] = L[0][0] * g.dt;
        de[1] = L[1][1] * g.dt;
        de[3] = 0.5f * (L[0][1] + L[1][0]) * g.dt;
        if (D == 3) {
          de[2] = L[D - 1][D - 1] * g.dt;
          de[4] = 0.5f * (L[1][D - 1] + L[D - 1][1]) * g.dt;
          de[5] = 0.5f * (L[0][D - 1] + L[D - 1][0]) * g.dt;
        }
        float sg[6], ep[NS];
        if (D == 3) {
#pragma unroll
          for (int i = 0; i < 6; ++i) sg[i] = A.A.sig[i][j];
        } else {
          sg[0] = A.A.sig[0][j]; sg[1] = A.A.sig[1][j]; sg[2] = A.A.sig[2][j]; sg[3] = A.A.sig[3][j];
          sg[4] = sg[5] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < NS; ++i) ep[i] = A.A.eps[i][j] + de[i];
        float vol = A.A.vol[j] * (1.f + de[0] + de[1] + de[2]);
        float epsp = A.A.epsp[j];
        const float coh = A.A.coh ? A.A.coh[j] : A.mat.c;
        material_update(A.mat, A.matd, coh, sg, de, epsp);
#pragma unroll
        for (int i = 0; i < NS; ++i) {
          A.B.sig[i][q] = sg[i];
          A.B.eps[i][q] = ep[i];
          if (!isfinite(sg[i])) status |= ST_NONFINITE;
        }
        A.B.vol[q] = vol;
        A.B.epsp[q] = epsp;
      }
      if (GMODE != G2P_USF_STRESS) {
        // FLIP velocity, advection in cell units, relocation
        int cell[3] = {tc[0] * TX + lc[0], tc[1] * TY + lc[1], D == 3 ? tc[2] * TZ + lc[2] : 0};
        bool dead = false;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float vk = A.A.vel[k][j] + g.dt * dv[k];
          A.B.vel[k][q] = vk;
          if (!isfinite(vk)) status |= ST_NONFINITE;
          float un = u[k] + g.dt * vb[k] * g.inv_h;
          if (!isfinite(un)) {
            status |= ST_NONFINITE;
            dead = true;
            un = 0.f;
          }
          // relocation: one cell crossing is an exact subtraction (Sterbenz),
          // so the offset stays in [-0.5, 0.5) and the cell is exact
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
          A.B.off[k][q] = un;
        }
        uint32_t nkey = g.dead_key;
        if (!dead) {
          const int t2 = cell[0] / TX + g.nt[0] * (cell[1] / TY + g.nt[1] * (D == 3 ? cell[2] / TZ : 0));
          const int l2 = cell[0] % TX + TX * (cell[1] % TY + TY * (D == 3 ? cell[2] % TZ : 0));
          nkey = (uint32_t)t2 * CELLS_PER_TILE + (uint32_t)l2;
        } else {
          status |= ST_LEFT_MESH;
        }
        A.B.key[q] = nkey;
        A.B.mass[q] = A.A.mass[j];
        A.B.id[q] = A.A.id[j];
        if (A.A.coh) A.B.coh[q] = A.A.coh[j];
      }
      if (status) atomicOr(&A.ctr[8], status);
    }
    __syncthreads();
  }
}

// Particles that left the mesh sit after all tiles in key order: carried over.
template <int D>
__global__ void copy_dead(PBuf A, PBuf B, const int32_t *perm, const int32_t *tile_start, int ntiles,
                          int64_t n) {
  const int s = tile_start[ntiles];
  constexpr int NS = nstress<D>();
  for (int64_t q = s + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
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
    B.vol[q] = A.vol[j];
    B.epsp[q] = A.epsp[j];
    if (A.coh) B.coh[q] = A.coh[j];
  }
}

template <int D, int MODE>
constexpr size_t p2g_smem() {
  return sizeof(float) * (CELLS_PER_TILE * (1 << D) * p2g_channels<D, MODE>() + NWARP * 32 * 33);
}

template <int D, int MODE>
cudaError_t launch_p2g(const F32Launch &L, float *slots, int work_slot, cudaStream_t st) {
  P2GArgs<D> a;
  a.geo = L.geo;
  a.A = L.A;
  a.B = L.B;
  a.keys = L.s.keys_sorted;
  a.perm = L.s.perm;
  a.tile_start = L.s.tile_start;
  a.active = L.s.active;
  a.ctr = L.s.ctr;
  a.work_slot = work_slot;
  a.slots = slots;
  p2g_tile<D, MODE><<<L.grid, NT, p2g_smem<D, MODE>(), st>>>(a);
  return cudaGetLastError();
}

template <int D, int MODE>
cudaError_t prepare_p2g() {
  return cudaFuncSetAttribute(p2g_tile<D, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)p2g_smem<D, MODE>());
}

template <int D, int GMODE>
cudaError_t launch_g2p(const F32Launch &L, int work_slot, int nch1, cudaStream_t st) {
  G2PArgs<D> a;
  a.geo = L.geo;
  a.mat = L.mat;
  a.matd = L.matd;
  a.A = L.A;
  a.B = L.B;
  a.keys = L.s.keys_sorted;
  a.perm = L.s.perm;
  a.tile_start = L.s.tile_start;
  a.active = L.s.active;
  a.ctr = L.s.ctr;
  a.work_slot = work_slot;
  a.slots1 = L.s.slots1;
  a.slots2 = L.s.slots2;
  a.nch1 = nch1;
  g2p_tile<D, GMODE><<<L.grid, NT, 0, st>>>(a);
  return cudaGetLastError();
}

template <int D>
cudaError_t step_dim(const F32Launch &L, cudaStream_t st) {
  cudaError_t e;
  const int blocks = L.grid;
  // phase events 0..2 are recorded by the caller (start, after sort, after
  // tile bounds); the tile kernels add 3.. after each launch
  if (L.scheme == 1) {  // USL
    if ((e = launch_p2g<D, P2G_USL>(L, L.s.slots1, 1, st)) != cudaSuccess) return e;
    if ((e = phase_mark(L.ev, 3, st)) != cudaSuccess) return e;
    if ((e = launch_g2p<D, G2P_USL>(L, 2, 1 + 2 * D, st)) != cudaSuccess) return e;
  } else {  // USF
    if ((e = launch_p2g<D, P2G_MOM>(L, L.s.slots1, 1, st)) != cudaSuccess) return e;
    if ((e = phase_mark(L.ev, 3, st)) != cudaSuccess) return e;
    if ((e = launch_g2p<D, G2P_USF_STRESS>(L, 2, 1 + D, st)) != cudaSuccess) return e;
    if ((e = phase_mark(L.ev, 4, st)) != cudaSuccess) return e;
    if ((e = launch_p2g<D, P2G_FORCE>(L, L.s.slots2, 3, st)) != cudaSuccess) return e;
    if ((e = phase_mark(L.ev, 5, st)) != cudaSuccess) return e;
    if ((e = launch_g2p<D, G2P_USF_ADVECT>(L, 4, 1 + D, st)) != cudaSuccess) return e;
  }
  copy_dead<D><<<blocks, 256, 0, st>>>(L.A, L.B, L.s.perm, L.s.tile_start, L.geo.ntiles, L.n);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return phase_mark(L.ev, L.scheme == 1 ? 4 : 6, st);
}

// ---------------------------------------------------------------------------
// Conservation sums (FP64, deterministic two-level), export, keys
// ---------------------------------------------------------------------------
constexpr int CONS_BLOCKS = 1024;
constexpr int CONS_VALS = 7;

template <int D>
__global__ void cons_partial(int64_t n, PBuf P, uint32_t dead_key, double *part) {
  constexpr int NS = nstress<D>();
  double acc[CONS_VALS] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    if (P.key[q] >= dead_key) continue;
    const double m = P.mass[q];
    acc[0] += m;
    double ke = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double v = P.vel[k][q];
      acc[1 + k] += m * v;
      ke += v * v;
    }
    acc[4] += 0.5 * m * ke;
    double se = 0;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      const int i6 = (D == 2 && i == 3) ? 3 : i;
      const double w = (i6 >= 3) ? 2.0 : 1.0;
      se += w * (double)P.sig[i][q] * (double)P.eps[i][q];
    }
    acc[5] += 0.5 * (double)P.vol[q] * se;
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
__global__ void export_k(int64_t n, PBuf P, Geo g, double o0, double o1, double o2, double h, double *pos,
                         double *vel, double *sig, double *eps, double *vol, double *epsp, int64_t *cell) {
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  constexpr int NS = nstress<D>();
  const double org[3] = {o0, o1, o2};
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t id = P.id[q];
    const uint32_t key = P.key[q];
    const bool dead = key >= g.dead_key;
    int c[3] = {0, 0, 0};
    if (!dead) {
      const int t = key / CELLS_PER_TILE;
      int tc[3];
      tc[0] = t % g.nt[0];
      tc[1] = (t / g.nt[0]) % g.nt[1];
      tc[2] = t / (g.nt[0] * g.nt[1]);
      int lc[3];
      local_coords<D>(key, lc);
      c[0] = tc[0] * TX + lc[0];
      c[1] = tc[1] * TY + lc[1];
      c[2] = D == 3 ? tc[2] * TZ + lc[2] : 0;
    }
    if (pos)
#pragma unroll
      for (int k = 0; k < D; ++k)
        pos[id * D + k] = dead ? __longlong_as_double(0x7ff8000000000000ll)
                               : org[k] + ((double)c[k] + 0.5 + (double)P.off[k][q]) * h;
    if (vel)
#pragma unroll
      for (int k = 0; k < D; ++k) vel[id * D + k] = P.vel[k][q];
    if (sig || eps) {
      double s6[6] = {0, 0, 0, 0, 0, 0}, e6[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        s6[i] = P.sig[i][q];
        e6[i] = P.eps[i][q];
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        if (sig) sig[id * 6 + i] = s6[i];
        if (eps) eps[id * 6 + i] = e6[i];
      }
    }
    if (vol) vol[id] = P.vol[q];
    if (epsp) epsp[id] = P.epsp[q];
    if (cell) cell[id] = dead ? -1 : (int64_t)c[0] + (int64_t)g.nc[0] * ((int64_t)c[1] + (int64_t)g.nc[1] * c[2]);
  }
}

__global__ void keys_copy(int64_t n, const uint32_t *src, uint32_t *dst) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    dst[q] = src[q];
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

cudaError_t f32_step(const F32Launch &L, cudaStream_t st) {
  if (L.n <= 0) return cudaSuccess;
  return L.dim == 3 ? step_dim<3>(L, st) : step_dim<2>(L, st);
}

cudaError_t f32_conservation(int dim, int64_t n, const PBuf &P, uint32_t dead_key, double *d_out,
                             double *d_partials, cudaStream_t st) {
  if (dim == 3)
    cons_partial<3><<<CONS_BLOCKS, 256, 0, st>>>(n, P, dead_key, d_partials);
  else
    cons_partial<2><<<CONS_BLOCKS, 256, 0, st>>>(n, P, dead_key, d_partials);
  cons_final<<<1, 32, 0, st>>>(d_partials, CONS_BLOCKS, d_out);
  return cudaGetLastError();
}

cudaError_t f32_export(int dim, int64_t n, const PBuf &P, const Geo &g, const double origin[3], double h,
                       double *pos, double *vel, double *sig, double *eps, double *vol, double *epsp,
                       int64_t *cell, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (dim == 3)
    export_k<3><<<blocks, 256, 0, st>>>(n, P, g, origin[0], origin[1], origin[2], h, pos, vel, sig, eps, vol, epsp, cell);
  else
    export_k<2><<<blocks, 256, 0, st>>>(n, P, g, origin[0], origin[1], origin[2], h, pos, vel, sig, eps, vol, epsp, cell);
  return cudaGetLastError();
}

cudaError_t f32_keys(int dim, int64_t n, const PBuf &P, uint32_t *keys_out, cudaStream_t st) {
  (void)dim;
  if (n <= 0) return cudaSuccess;
  keys_copy<<<1024, 256, 0, st>>>(n, P.key, keys_out);
  return cudaGetLastError();
}

cudaError_t material_update_f32(const MatConst<float> &m, const MatConst<double> &md, int64_t n,
                                const float *sig, const float *de, const float *coh, float *out,
                                float *depsp, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  mat_update_f32_k<<<blocks, 256, 0, st>>>(m, md, n, sig, de, coh, out, depsp);
  return cudaGetLastError();
}

}  // namespace mpm
