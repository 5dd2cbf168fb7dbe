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
//   p2g_tile   one CTA per 4x4x4 (8x8) cell tile, each thread owning
//              corners of one cell: stages the tile's particles (binning
//              order, coalesced) in shared memory, each thread sums its
//              corners' contributions over its cell's particles in order in
//              registers, cells are summed into the tile's node box
//              (compensated sums) and the box is written to the tile's own
//              slot -- no atomics, bit-reproducible;
//   node_tile  one warp per slice of a tile's box: final nodal values,
//              summing the slots of the (at most 2^D) tiles that share each
//              node in ascending tile order, then v = P/m, a = f/m + g,
//              v' = v + a dt and the boundary conditions; each node is
//              computed once (by its lowest active tile) into dense node
//              records;
//   g2p        one thread per particle in binning order: FLIP velocity,
//              advection, strain, stress, volume and relocation into the new
//              cell, written in binning order so the next step reads
//              contiguously; particles that change tile are counted and
//              listed for the next step's binning.
#include <climits>
#include <type_traits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mpm_internal.h"
#include "mpm_iso.cuh"

namespace mpm {
namespace {

constexpr int NODE_T = 128;
#ifndef MPM_G2P_T
#define MPM_G2P_T 128
#endif
constexpr int G2P_T = MPM_G2P_T;        // G2P threads per CTA
constexpr int G2P_SUB = 256 / G2P_T;    // G2P CTAs per 256-particle block of the group prefix
#ifndef MPM_P2G_MINB
#define MPM_P2G_MINB 5  // resident P2G CTAs per SM the register budget is sized for
#endif
#ifndef MPM_NODE_MINB
#define MPM_NODE_MINB 8  // resident node CTAs per SM for a single mesh (a batch's kernel: 8)
#endif
#ifndef MPM_G2P_MINB
#define MPM_G2P_MINB 8  // resident G2P CTAs per SM the register budget is sized for
#endif

// Instance of item x: the largest i with prefix[i] <= x (prefix[0] = 0).
__device__ __forceinline__ int find_inst(const int32_t *prefix, int ninst, int x) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void tile_coords(const Geo &g, int t, int tc[3]) {
  const int tz = g.div_nt01.div(t);
  const int r = t - tz * (g.nt[0] * g.nt[1]);
  const int ty = g.div_nt0.div(r);
  tc[0] = r - ty * g.nt[0];
  tc[1] = ty;
  tc[2] = tz;
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

// Shape values and gradients of the corners a P2G thread owns, at offset u.
// The corners share their x and y bits (bits 0 and 1 of cp; sx, sy = +1 for
// the upper node of the cell along that axis) and, in 3D, are the lower (r =
// 0) and the upper (r = 1) node along z.  ThreadCorners holds the factors
// they share; corner(r) forms the products of corner_shape in the same order,
// so the values are identical to it.
template <int D>
struct ThreadCorners {
  float wxy, gx, gy, gz, wz[2];
  __device__ __forceinline__ ThreadCorners(const float *u, int cp, float inv_h) {
    const bool ux = cp & 1, uy = cp & 2;  // upper node along x, y (predicates, loop-invariant)
    const float wx = ux ? 0.5f + u[0] : 0.5f - u[0], wy = uy ? 0.5f + u[1] : 0.5f - u[1];
    wxy = wx * wy;
    const float tx = inv_h * wy, ty = inv_h * wx;  // (-a) b = -(a b) exactly
    gx = ux ? tx : -tx;
    gy = uy ? ty : -ty;
    gz = D == 3 ? ty * wy : 0.f;
    wz[0] = D == 3 ? 0.5f - u[D - 1] : 1.f;
    wz[1] = D == 3 ? 0.5f + u[D - 1] : 1.f;
  }
  __device__ __forceinline__ void corner(int r, float &N, float G[D]) const {
    if constexpr (D == 2) {
      N = wxy;
      G[0] = gx;
      G[1] = gy;
    } else {
      N = wxy * wz[r];
      G[0] = gx * wz[r];
      G[1] = gy * wz[r];
      G[2] = r ? gz : -gz;
    }
  }
};

// Four corners per thread (3D): the x bit is the thread's (cp & 1), corner r
// has y bit r & 1 and z bit r >> 1.  The products are those of
// ThreadCorners (and so of corner_shape), formed once per y bit.
struct ThreadCorners4 {
  float wxy[2], gx[2], gy[2], gz[2], wz[2];
  __device__ __forceinline__ ThreadCorners4(const float *u, int cp, float inv_h) {
    const bool ux = cp & 1;
    const float wx = ux ? 0.5f + u[0] : 0.5f - u[0];
    const float ty = inv_h * wx;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const float wy = b ? 0.5f + u[1] : 0.5f - u[1];
      wxy[b] = wx * wy;
      const float tx = inv_h * wy;
      gx[b] = ux ? tx : -tx;
      gy[b] = b ? ty : -ty;
      gz[b] = ty * wy;
    }
    wz[0] = 0.5f - u[2];
    wz[1] = 0.5f + u[2];
  }
  __device__ __forceinline__ void corner(int r, float &N, float G[3]) const {
    const int b = r & 1, z = r >> 1;
    N = wxy[b] * wz[z];
    G[0] = gx[b] * wz[z];
    G[1] = gy[b] * wz[z];
    G[2] = z ? gz[b] : -gz[b];
  }
};
template <int D, int CPT>
using CornersOf = typename std::conditional<CPT == 4, ThreadCorners4, ThreadCorners<D>>::type;

// ---------------------------------------------------------------------------
// Mapped (isoparametric) cells (ISOPARAMETRIC MESH) in the FP32 path.  A
// particle's offset u is half its natural coordinates (u in [-0.5, 0.5)^D);
// relative to the cell's centre and in units of h the cell maps u to
// x(u) = sum_a N_a(u) P_a, P_a its corners (Geo::cgeo), with Jacobian
// J = dx/du = sum_a P_a (x) dN_a/du.  A shape gradient is then
// dN_a/dx = (dN_a/du K) / h with K = J^-1, so the transfers run the
// Cartesian arithmetic on dN/du and multiply by K once per particle.  Every
// position is kept in the frame of the particle's own cell, so FP32 resolves
// it as finely as the Cartesian offset does.
// ---------------------------------------------------------------------------
// Face-stress forces of a mapped mesh's boundary node (Geo::fload), added to ft.
template <int D>
__device__ __forceinline__ void add_face_loads(const Geo &g, int faces, const int I[3], float ft[D]) {
#pragma unroll
  for (int f = 0; f < 2 * D; ++f)
    if ((faces >> f) & 1) {
      const float4 q = __ldg(g.fload + g.fnoff[f] + face_node_index<D>(f, I, g.nc));
      ft[0] += q.x;
      ft[1] += q.y;
      if (D == 3) ft[D - 1] += q.z;
    }
}

template <int D>
__device__ __forceinline__ int cell_lin(const Geo &g, const int c[3]) {
  return c[0] + g.nc[0] * (c[1] + g.nc[1] * (D == 3 ? c[2] : 0));
}

template <int D>
__device__ __forceinline__ void load_cgeo(const Geo &g, int cid, float P[1 << D][D]) {
  constexpr int NF = CGEO_F4<D>();
  float f[4 * NF];
#pragma unroll
  for (int m = 0; m < NF; ++m) {
    const float4 q = __ldg(g.cgeo + (int64_t)NF * cid + m);
    f[4 * m] = q.x;
    f[4 * m + 1] = q.y;
    f[4 * m + 2] = q.z;
    f[4 * m + 3] = q.w;
  }
#pragma unroll
  for (int a = 0; a < (1 << D); ++a)
#pragma unroll
    for (int k = 0; k < D; ++k) P[a][k] = f[D * a + k];
}

// x(u) and J(u) of a mapped cell.
template <int D>
__device__ __forceinline__ void cgeo_map(const float P[1 << D][D], const float u[D], float x[D], float J[D][D]) {
  float w0[D], w1[D];
  corner_weights<D>(u, w0, w1);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    x[k] = 0.f;
#pragma unroll
    for (int m = 0; m < D; ++m) J[k][m] = 0.f;
  }
#pragma unroll
  for (int a = 0; a < (1 << D); ++a) {
    float N, G[D];
    corner_shape<D>(a, w0, w1, 1.f, N, G);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      x[k] = fmaf(N, P[a][k], x[k]);
#pragma unroll
      for (int m = 0; m < D; ++m) J[k][m] = fmaf(P[a][k], G[m], J[k][m]);
    }
  }
}

// K = J^-1 by cofactors; false if J is singular or not finite.  Explicitly
// rounded operations (never contracted into FMAs), so that a mesh alone and
// in a batch round alike.
template <int D>
__device__ __forceinline__ bool inv_jac(const float J[D][D], float K[D][D]) {
  if constexpr (D == 2) {
    const float det = __fsub_rn(__fmul_rn(J[0][0], J[1][1]), __fmul_rn(J[0][1], J[1][0]));
    if (!(fabsf(det) > 0.f) || !isfinite(det)) return false;
    const float r = __frcp_rn(det);
    K[0][0] = __fmul_rn(J[1][1], r);
    K[0][1] = -__fmul_rn(J[0][1], r);
    K[1][0] = -__fmul_rn(J[1][0], r);
    K[1][1] = __fmul_rn(J[0][0], r);
  } else {
    float C[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        C[i][j] = __fsub_rn(__fmul_rn(J[i1][j1], J[i2][j2]), __fmul_rn(J[i1][j2], J[i2][j1]));
      }
    const float det =
        __fadd_rn(__fadd_rn(__fmul_rn(J[0][0], C[0][0]), __fmul_rn(J[0][1], C[0][1])), __fmul_rn(J[0][2], C[0][2]));
    if (!(fabsf(det) > 0.f) || !isfinite(det)) return false;
    const float r = __frcp_rn(det);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) K[i][j] = __fmul_rn(C[j][i], r);
  }
  return true;
}

// Newton-Raphson in one cell for the offset whose image is T (the cell's
// frame), from un: at most 8 iterations, until a step is below 1e-7 cell.
template <int D>
__device__ __forceinline__ void cgeo_solve(const float P[1 << D][D], const float T[D], float un[D]) {
  for (int it = 0; it < 8; ++it) {
    float x[D], J[D][D], K[D][D];
    cgeo_map<D>(P, un, x, J);
    if (!inv_jac<D>(J, K)) return;
    float r[D], st = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) r[k] = x[k] - T[k];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      float d = 0.f;
#pragma unroll
      for (int m = 0; m < D; ++m) d = fmaf(K[k][m], r[m], d);
      un[k] -= d;
      st = fmaxf(st, fabsf(d));
    }
    if (!(st > 1e-7f)) return;  // converged, or not finite (the caller checks)
  }
}

// ---------------------------------------------------------------------------
// P2G: one CTA per tile; each thread owns CPT corners of one cell (3D: two
// corners, 256 threads, or four and 128 threads for the USF mass/momentum
// P2G; 2D: one corner, 256 threads).  The tile's particles (binning order,
// so grouped by cell) are staged in shared memory in chunks of 256
// particles (512 in the USF mass/momentum P2G), one to four per thread:
// offset u, and the per-particle factors of the
// channels -- m and m v (mass, momentum), nV sig with nV = -V (internal
// force f_k = -V sum_j sig_kj dN/dx_j).  Then the thread of (cell c, corner
// a) runs over the particles of c in binning order and accumulates its
// corners' channels in registers: each (cell, corner, channel) sum is a plain
// sequential FP32 sum, independent of the launch.  Cell sums go to the node
// box (compensated, ascending cell order) and the box to the tile's slot.
// Value index v = corner * NCH + channel; channels USL (m, P_k, f_k), MOM
// (m, P_k), FORCE (f_k).
// ---------------------------------------------------------------------------
// WIDE (3D): four corners per thread, two threads per cell, 128 threads per
// tile, each staging several particles of a chunk.  The four-channel
// mass/momentum P2G stages 512 particles a chunk (64M slope 758 -> 730 us);
// the USL and force P2G were slower so (1117 -> 1155, 872 -> 897 us).
template <int D, int MODE, bool MAP = false, bool WIDE = false>
struct P2GRec {
  static_assert(!WIDE || D == 3, "four corners per thread: 3D");
  static constexpr bool HAS_M = MODE != P2G_FORCE, HAS_F = MODE != P2G_MOM;
  // nV sig (xx yy zz xy yz xz | xx yy xy); on a mapped mesh the full D x D
  // matrix nV sig K^T (row-major), K the inverse of the cell map's Jacobian
  static constexpr int NSV = MAP ? D * D : (D == 3 ? 6 : 3);
  static constexpr int NF = D + (HAS_M ? 1 + D : 0) + (HAS_F ? NSV : 0);
  static constexpr int NQ = (NF + 3) / 4;                      // float4 chunks per particle
  static constexpr int CPT = D == 3 ? (WIDE ? 4 : 2) : 1;      // corners per thread
  static constexpr int CPC = (1 << D) / CPT;                   // threads per cell
  static constexpr int NT = CELLS_PER_TILE * CPC;              // threads
  static constexpr int CH = (WIDE && MODE == P2G_MOM) ? 512 : 256;  // particles per chunk
  static constexpr int PPT = CH / NT;                          // particles each thread stages
  static constexpr int NV = (1 << D) * p2g_channels<D, MODE>();
  static constexpr size_t REC_BYTES = sizeof(float4) * NQ * CH;
  static constexpr size_t CELLP_BYTES = sizeof(float) * CELLS_PER_TILE * NV;
  static constexpr size_t SMEM = (REC_BYTES > CELLP_BYTES ? REC_BYTES : CELLP_BYTES);
};

// Resident P2G CTAs per SM the register budget is sized for: MPM_P2G_MINB
// (48 registers at 5), except the 3D USL kernel of a batch, which reads its
// instance from shared memory and would spill at 48: 4 (64 registers).
template <int D, int MODE, bool ONE>
constexpr int p2g_min_blocks() {
  return (D == 3 && MODE == P2G_USL && !ONE) ? 4 : MPM_P2G_MINB;
}
#ifndef MPM_P2G_WIDE_MINB
#define MPM_P2G_WIDE_MINB 8  // resident 128-thread P2G CTAs per SM (64 registers)
#endif

template <int D, int MODE>
constexpr size_t p2g_smem() {
  return P2GRec<D, MODE>::SMEM;
}
template <int D>
constexpr int p2g_threads() {
  return P2GRec<D, P2G_USL>::NT;
}
// Four corners per thread: the Cartesian 3D mass and momentum P2G of USF
// (64M slope 786 -> 759 us; with the seven channels of USL it was slower,
// 1116 -> 1268 us at 64 registers, and the force-only P2G no faster).
template <int D, int MODE, bool MAP>
constexpr bool p2g_wide() {
  return D == 3 && !MAP && MODE == P2G_MOM;
}
template <int D, int MODE, bool MAP>
using P2GTile = P2GRec<D, MODE, MAP, p2g_wide<D, MODE, MAP>()>;

// Resident G2P CTAs per SM the register budget is sized for: MPM_G2P_MINB
// (64 registers at 8) for the 3D USL and USF stress kernels; nine (56
// registers) for the USF advection stage and in 2D, which measured faster
// so (64M slope advection 1348 -> 1262 us, 256 batched 2D columns 0.507 ->
// 0.494 ms per step) while the 3D USL G2P was slower (2348 -> 2395 us).
template <int D, int GMODE, bool MAP>
constexpr int g2p_min_blocks() {
  return MAP ? 4 : ((D == 3 && GMODE != G2P_USF_ADVECT) ? MPM_G2P_MINB : 9);
}

// 4- and 16-byte asynchronous global -> shared copies (each thread later reads only
// what it copied itself, so a wait on its own copies is all it needs).
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// The active-tile record (tile, new start, new end, slot shift or INT_MIN) of
// P2G work item w.
template <bool ONE>
__device__ __forceinline__ const int4 *act_rec(const GroupArgs &G, int w) {
  if constexpr (ONE) {
    return G.one.s.active + w;
  } else {
    const int i = find_inst(G.act_items, G.ninst, w);
    return G.inst[i].s.active + (w - G.act_items[i]);
  }
}

// Slot of particle i of a chunk: the low three bits are XORed with the next
// three, so that the cells of a warp, whose current particles are often a
// multiple of eight apart, read different shared-memory banks.
__device__ __forceinline__ int rec_slot(int i) { return (i & ~7) | ((i ^ (i >> 3)) & 7); }

// The P2G record of one particle: offset u, and the per-particle factors of
// the channels -- m and m v (mass, momentum), nV sig with nV = -V (internal
// force f_k = -V sum_j sig_kj dN/dx_j).  The same arithmetic wherever a record
// is formed (from stored state, or in G2P from the state it has just
// computed), so a particle's contributions do not depend on where.
template <int D, int MODE>
__device__ __forceinline__ void p2g_record(const float *u, float mm, const float *v, float jm1, const float *sg,
                                           float inv_rho, float f[4 * P2GRec<D, MODE>::NQ]) {
  using R = P2GRec<D, MODE>;
#pragma unroll
  for (int k = 0; k < 4 * R::NQ; ++k) f[k] = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) f[k] = u[k];
  if (R::HAS_M) {
    f[D] = mm;
#pragma unroll
    for (int k = 0; k < D; ++k) f[D + 1 + k] = mm * v[k];
  }
  if (R::HAS_F) {
    const float nV = -mm * inv_rho * (1.f + jm1);
    constexpr int o = R::HAS_M ? 2 * D + 1 : D;
    if (D == 3) {
#pragma unroll
      for (int k = 0; k < 6; ++k) f[o + k] = nV * sg[k];
    } else {
      f[o] = nV * sg[0];
      f[o + 1] = nV * sg[1];
      f[o + 2] = nV * sg[3];
    }
  }
}

// Add record i to the channels of the thread's corners (my_cp + r * CPC).
template <int D, int MODE>
__device__ __forceinline__ void accumulate_rec(const float4 *rec, int i, int my_cp, float inv_h,
                                               float acc[P2GRec<D, MODE>::CPT][p2g_channels<D, MODE>()]) {
  using R = P2GRec<D, MODE>;
  constexpr int NQ = R::NQ, CH = R::CH, CPT = R::CPT, CPC = R::CPC;
  constexpr bool HAS_M = R::HAS_M, HAS_F = R::HAS_F;
  {
    const int sl = rec_slot(i);
    float f[4 * NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const float4 rv = rec[k * CH + sl];
      f[4 * k] = rv.x;
      f[4 * k + 1] = rv.y;
      f[4 * k + 2] = rv.z;
      f[4 * k + 3] = rv.w;
    }
    static_assert(CPT == (D == 3 ? 2 : 1) && CPC == 4, "corners my_cp + 4 r: z bit = r");
    const ThreadCorners<D> tc(f, my_cp, inv_h);
#pragma unroll
    for (int r = 0; r < CPT; ++r) {
      float N, Gr[D];
      tc.corner(r, N, Gr);
      if (HAS_M) {
        acc[r][0] = fmaf(f[D], N, acc[r][0]);
#pragma unroll
        for (int k = 0; k < D; ++k) acc[r][1 + k] = fmaf(f[D + 1 + k], N, acc[r][1 + k]);
      }
      if (HAS_F) {
        constexpr int o = HAS_M ? 2 * D + 1 : D;
        constexpr int a0 = HAS_M ? 1 + D : 0;
        if (D == 3) {
          // nV sig: xx yy zz xy yz xz
          const float t3[3][3] = {{f[o], f[o + 3], f[o + 5]}, {f[o + 3], f[o + 1], f[o + 4]},
                                  {f[o + 5], f[o + 4], f[o + 2]}};
#pragma unroll
          for (int k = 0; k < D; ++k)
#pragma unroll
            for (int jj = 0; jj < D; ++jj) acc[r][a0 + k] = fmaf(t3[k][jj], Gr[jj], acc[r][a0 + k]);
        } else {
          const float t2[2][2] = {{f[o], f[o + 2]}, {f[o + 2], f[o + 1]}};
#pragma unroll
          for (int k = 0; k < D; ++k)
#pragma unroll
            for (int jj = 0; jj < D; ++jj) acc[r][a0 + k] = fmaf(t2[k][jj], Gr[jj], acc[r][a0 + k]);
        }
      }
    }
  }
}

// Accumulate the records i0..i1-1 of one cell, in order (plain sequential
// FP32 sums per channel).
template <int D, int MODE>
__device__ __forceinline__ void accumulate_cell(const float4 *rec, int i0, int i1, int my_cp, float inv_h,
                                                float acc[P2GRec<D, MODE>::CPT][p2g_channels<D, MODE>()]) {
  for (int i = i0; i < i1; ++i) accumulate_rec<D, MODE>(rec, i, my_cp, inv_h, acc);
}

// Cell sums (cellP[cell][corner][channel]) -> the tile's node box, summed in
// ascending local cell order with compensated (TwoSum) accumulation, written
// to the tile's slot.  Every thread of the CTA (nthreads) takes part.
template <int D, int NCH>
__device__ __forceinline__ void cells_to_slot(const float *cellP, float *slots_out, int t, int nthreads) {
  constexpr int BN = box_nodes<D>();
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  constexpr int NV = (1 << D) * NCH;
  for (int b = threadIdx.x; b < BN; b += nthreads) {
    const int bx = b % (TX + 1);
    const int by = (b / (TX + 1)) % (TY + 1);
    const int bz = D == 3 ? b / ((TX + 1) * (TY + 1)) : 0;
    TwoAcc<float> ta[NCH];
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) ta[ch].init();
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
          for (int ch = 0; ch < NCH; ++ch) ta[ch].add(cellP[cl * NV + a * NCH + ch]);
        }
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) slots_out[((int64_t)t * NCH + ch) * BN + b] = ta[ch].value();
  }
}

template <int D, int MODE, bool ONE, bool MAP = false>
__global__ void __launch_bounds__(P2GTile<D, MODE, MAP>::NT,
                                  MAP ? 4 : (p2g_wide<D, MODE, MAP>() ? MPM_P2G_WIDE_MINB : p2g_min_blocks<D, MODE, ONE>()))
    p2g_tile(const __grid_constant__ GroupArgs G, int work_slot) {
  using R = P2GTile<D, MODE, MAP>;
  constexpr int NCH = p2g_channels<D, MODE>();
  constexpr int NV = R::NV;
  constexpr int CH = R::CH, NT = R::NT, PPT = R::PPT;
  constexpr int NQ = R::NQ;
  constexpr int CPT = R::CPT, CPC = R::CPC;
  constexpr int BN = box_nodes<D>();
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  constexpr bool HAS_M = R::HAS_M, HAS_F = R::HAS_F;
  extern __shared__ float4 sm4[];
  float4 *rec = sm4;                              // [NQ][CH] float4
  float *cellP = reinterpret_cast<float *>(sm4);  // [64][NV], after the chunks
  __shared__ int cs[CELLS_PER_TILE], ce[CELLS_PER_TILE], stamp[CELLS_PER_TILE];
  __shared__ int s_work[2];
  __shared__ int4 s_ar[2];  // the item's active-tile record; the next one lands during the box phase
  __shared__ InstArgs sI;
  const int tid = threadIdx.x;
  const int my_cell = tid / CPC, my_cp = tid % CPC;  // corners my_cp + r * CPC
  pdl_trigger();
  if (tid < CELLS_PER_TILE) stamp[tid] = -1;
  pdl_wait();
  // items: first the CTA's own (blockIdx.x), then gridDim.x + the work counter
  const int total = G.act_items[G.ninst];
  if (tid == 0) {
    s_work[0] = blockIdx.x;
    if ((int)blockIdx.x < total) s_ar[0] = *act_rec<ONE>(G, blockIdx.x);
  }
  __syncthreads();
  int chunk_id = 0, loaded = -1;

  for (int it = 0;; ++it) {
    const int wi = s_work[it & 1];
    if (wi >= total) break;
    // the next work item is fetched now and published at the end of this one
    int wnext = 0;
    if (tid == 0) wnext = (int)gridDim.x + atomicAdd(&G.work[work_slot], 1);
    const int ii = ONE ? 0 : find_inst(G.act_items, G.ninst, wi);
    if (!ONE && ii != loaded) {  // uniform
      copy_inst(G.inst, ii, &sI);
      loaded = ii;
      __syncthreads();
    }
    const InstArgs &I = inst_ref<ONE>(G, sI);
    const Geo &g = I.geo;
    float *slots_out = MODE == P2G_FORCE ? I.s.slots2 : I.s.slots1;
    const int4 ar = s_ar[it & 1];
    const int t = ar.x, s = ar.y, e = ar.z;
    int tco[3] = {0, 0, 0};
    if (MAP) tile_coords(g, t, tco);
    float acc[CPT][NCH];
#pragma unroll
    for (int r = 0; r < CPT; ++r)
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) acc[r][ch] = 0.f;

    for (int c0 = s; c0 < e; c0 += CH) {
      // ---- stage this chunk: particles q = c0 + ps, ps = tid + pp * NT
      const int c1 = min(e, c0 + CH);
#pragma unroll
      for (int pp = 0; pp < PPT; ++pp) {
      const int ps = tid + pp * NT;
      const int q = c0 + ps;
      if (q < c1) {
        // the binning moved the tile's range as a whole (slot q + dj holds
        // position q): the loads need not wait for the permutation
        const int dj = s_ar[it & 1].w;
        const int j = dj != INT_MIN ? q + dj : I.perm_out[q];
        const int lc = I.keys_out[q] & (CELLS_PER_TILE - 1);
        float f[4 * NQ];
#pragma unroll
        for (int k = 0; k < 4 * NQ; ++k) f[k] = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) f[k] = I.A.off(k)[j];
        const float mm = I.A.mass()[j];
        if (HAS_M) {
          f[D] = mm;
#pragma unroll
          for (int k = 0; k < D; ++k) f[D + 1 + k] = mm * I.A.vel(k)[j];
        }
        if (HAS_F) {
          // FORCE (USF) reads the stress updated earlier this step, stored in
          // binning order; USL reads the stress at the start of the step
          const PBuf &S = (MODE == P2G_FORCE) ? I.B : I.A;
          const int js = (MODE == P2G_FORCE) ? q : j;
          const float nV = -mm * g.inv_rho * (1.f + S.jm1()[js]);
          constexpr int o = HAS_M ? 2 * D + 1 : D;
          if constexpr (MAP) {
            // nV sig K^T at the particle's offset, K = J^-1 of its cell's map
            int l3[3], cc[3];
            local_coords<D>((uint32_t)lc, l3);
            cc[0] = tco[0] * TX + l3[0];
            cc[1] = tco[1] * TY + l3[1];
            cc[2] = D == 3 ? tco[2] * TZ + l3[2] : 0;
            float P[1 << D][D], xl[D], J[D][D], K[D][D];
            load_cgeo<D>(g, cell_lin<D>(g, cc), P);
            cgeo_map<D>(P, f, xl, J);
            if (!inv_jac<D>(J, K)) {
#pragma unroll
              for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = 0; b < D; ++b) K[a][b] = 0.f;
            }
            float sm[D][D];
            if (D == 3) {
              const float s0 = S.sig(0)[js], s1 = S.sig(1)[js], s2 = S.sig(2)[js];
              const float s3 = S.sig(3)[js], s4 = S.sig(4)[js], s5 = S.sig(5)[js];
              const float t3[3][3] = {{s0, s3, s5}, {s3, s1, s4}, {s5, s4, s2}};
#pragma unroll
              for (int a = 0; a < D; ++a)
#pragma unroll
                for (int b = 0; b < D; ++b) sm[a][b] = t3[a][b];
            } else {
              sm[0][0] = S.sig(0)[js];
              sm[1][1] = S.sig(1)[js];
              sm[0][1] = sm[1][0] = S.sig(3)[js];
            }
#pragma unroll
            for (int k = 0; k < D; ++k)
#pragma unroll
              for (int m = 0; m < D; ++m) {
                float acc_km = 0.f;
#pragma unroll
                for (int jj = 0; jj < D; ++jj) acc_km = fmaf(sm[k][jj], K[m][jj], acc_km);
                f[o + D * k + m] = nV * acc_km;
              }
          } else if (D == 3) {
#pragma unroll
            for (int k = 0; k < 6; ++k) f[o + k] = nV * S.sig(k)[js];
          } else {
            f[o] = nV * S.sig(0)[js];
            f[o + 1] = nV * S.sig(1)[js];
            f[o + 2] = nV * S.sig(3)[js];
          }
        }
        const int sl = rec_slot(ps);
#pragma unroll
        for (int k = 0; k < NQ; ++k) rec[k * CH + sl] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
        // run boundaries of the cell within the chunk
        const bool first = q == c0 || (int)(I.keys_out[q - 1] & (CELLS_PER_TILE - 1)) != lc;
        const bool last = q == c1 - 1 || (int)(I.keys_out[q + 1] & (CELLS_PER_TILE - 1)) != lc;
        if (first) {
          cs[lc] = ps;
          stamp[lc] = chunk_id;
        }
        if (last) ce[lc] = ps + 1;
      }
      }
      __syncthreads();
      // ---- accumulate my (cell, corner) pairs over the cell's particles in order
      if (stamp[my_cell] == chunk_id) {
        const int i0 = cs[my_cell], i1 = ce[my_cell];
        for (int i = i0; i < i1; ++i) {
          const int sl = rec_slot(i);
          float f[4 * NQ];
#pragma unroll
          for (int k = 0; k < NQ; ++k) {
            const float4 rv = rec[k * CH + sl];
            f[4 * k] = rv.x;
            f[4 * k + 1] = rv.y;
            f[4 * k + 2] = rv.z;
            f[4 * k + 3] = rv.w;
          }
          static_assert(CPT == 4 ? (D == 3 && CPC == 2) : (CPT == (D == 3 ? 2 : 1) && CPC == 4),
                        "corners my_cp + CPC r");
          const CornersOf<D, CPT> tc(f, my_cp, g.inv_h);
#pragma unroll
          for (int r = 0; r < CPT; ++r) {
            float N, Gr[D];
            tc.corner(r, N, Gr);
            if (HAS_M) {
              acc[r][0] = fmaf(f[D], N, acc[r][0]);
#pragma unroll
              for (int k = 0; k < D; ++k) acc[r][1 + k] = fmaf(f[D + 1 + k], N, acc[r][1 + k]);
            }
            if (HAS_F) {
              constexpr int o = HAS_M ? 2 * D + 1 : D;
              constexpr int a0 = HAS_M ? 1 + D : 0;
              if constexpr (MAP) {
#pragma unroll
                for (int k = 0; k < D; ++k)
#pragma unroll
                  for (int m = 0; m < D; ++m) acc[r][a0 + k] = fmaf(f[o + D * k + m], Gr[m], acc[r][a0 + k]);
              } else if (D == 3) {
                // nV sig: xx yy zz xy yz xz
                const float t3[3][3] = {{f[o], f[o + 3], f[o + 5]}, {f[o + 3], f[o + 1], f[o + 4]},
                                        {f[o + 5], f[o + 4], f[o + 2]}};
#pragma unroll
                for (int k = 0; k < D; ++k)
#pragma unroll
                  for (int jj = 0; jj < D; ++jj) acc[r][a0 + k] = fmaf(t3[k][jj], Gr[jj], acc[r][a0 + k]);
              } else {
                const float t2[2][2] = {{f[o], f[o + 2]}, {f[o + 2], f[o + 1]}};
#pragma unroll
                for (int k = 0; k < D; ++k)
#pragma unroll
                  for (int jj = 0; jj < D; ++jj) acc[r][a0 + k] = fmaf(t2[k][jj], Gr[jj], acc[r][a0 + k]);
              }
            }
          }
        }
      }
      ++chunk_id;
      __syncthreads();  // the next chunk overwrites the records
    }

    // ---- cells -> node box (ascending local cell order), compensated; -> slot
#pragma unroll
    for (int r = 0; r < CPT; ++r)
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) cellP[my_cell * NV + (my_cp + r * CPC) * NCH + ch] = acc[r][ch];
    if (tid == 0 && wnext < total) {  // the next item's record, in flight during the box phase
      cp_async16(&s_ar[(it + 1) & 1], act_rec<ONE>(G, wnext));
      cp_async_commit();
    }
    __syncthreads();
    for (int b = tid; b < BN; b += NT) {
      const int bx = b % (TX + 1);
      const int by = (b / (TX + 1)) % (TY + 1);
      const int bz = D == 3 ? b / ((TX + 1) * (TY + 1)) : 0;
      TwoAcc<float> ta[NCH];
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) ta[ch].init();
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
            for (int ch = 0; ch < NCH; ++ch) ta[ch].add(cellP[cl * NV + a * NCH + ch]);
          }
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) slots_out[((int64_t)t * NCH + ch) * BN + b] = ta[ch].value();
    }
    if (tid == 0) {
      s_work[(it + 1) & 1] = wnext;
      cp_async_wait_all();
    }
    __syncthreads();
  }
}


// Residual P2G of the fused USL step (RES): the items are the active tiles whose
// next-step P2G the previous G2P did not complete (the scan's residual
// list): a tile without valid sums for this step (fepoch != step) sums all
// its particles into slots1 (fepoch = step); a tile with valid sums sums only
// the particles that arrived from other tiles -- those outside the tile's old
// range -- into slots_a (aepoch = step).  Staged particles are compacted in
// binning order, so the cells' runs stay contiguous.
template <int D, int MODE, bool ONE, bool RES>
__global__ void __launch_bounds__(P2GRec<D, MODE>::CH, p2g_min_blocks<D, MODE, ONE>())
    p2g_resid(const __grid_constant__ GroupArgs G, int work_slot) {
  static_assert(RES && MODE == P2G_USL, "the residual P2G is the USL one");
  using R = P2GRec<D, MODE>;
  constexpr int NCH = p2g_channels<D, MODE>();
  constexpr int NV = R::NV;
  constexpr int CH = R::CH;
  constexpr int NQ = R::NQ;
  constexpr int CPT = R::CPT, CPC = R::CPC;
  constexpr int NW = CH / 32;
  extern __shared__ float4 sm4[];
  float4 *rec = sm4;                              // [NQ][CH] float4
  float *cellP = reinterpret_cast<float *>(sm4);  // [64][NV], after the chunks
  __shared__ int cs[CELLS_PER_TILE], ce[CELLS_PER_TILE], stamp[CELLS_PER_TILE];
  __shared__ int s_work[2];
  __shared__ int ccell[RES ? CH : 1];
  __shared__ int wkeep[NW + 1];
  __shared__ InstArgs sI;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int my_cell = tid / CPC, my_cp = tid % CPC;  // corners my_cp + r * CPC
  pdl_trigger();
  if (tid < CELLS_PER_TILE) stamp[tid] = -1;
  pdl_wait();
  const int32_t *items = RES ? G.res_items : G.act_items;
  // items: first the CTA's own (blockIdx.x), then gridDim.x + the work counter
  const int total = items[G.ninst];
  if (tid == 0) s_work[0] = blockIdx.x;
  __syncthreads();
  int chunk_id = 0, loaded = -1;

  for (int it = 0;; ++it) {
    const int wi = s_work[it & 1];
    if (wi >= total) break;
    // the next work item is fetched now and published at the end of this one
    int wnext = 0;
    if (tid == 0) wnext = (int)gridDim.x + atomicAdd(&G.work[work_slot], 1);
    const int ii = ONE ? 0 : find_inst(items, G.ninst, wi);
    if (!ONE && ii != loaded) {  // uniform
      copy_inst(G.inst, ii, &sI);
      loaded = ii;
      __syncthreads();
    }
    const InstArgs &I = inst_ref<ONE>(G, sI);
    const Geo &g = I.geo;
    const int local = ONE ? wi : wi - items[ii];
    const int aidx = RES ? I.s.resid[local] : local;
    const int4 ar = I.s.active[aidx];
    const int t = ar.x, s = ar.y, e = ar.z;
    int os = 0, oe = 0, step = 0;
    bool full = true;
    if (RES) {
      const int4 br = I.s.bin_rec[aidx];
      os = br.x;
      oe = br.y;
      step = I.s.ctr[C_STEP];
      full = I.s.fepoch[t] != step;  // uniform
    }
    float *slots_out = MODE == P2G_FORCE ? I.s.slots2 : (RES && !full ? I.s.slots_a : I.s.slots1);
    float acc[CPT][NCH];
#pragma unroll
    for (int r = 0; r < CPT; ++r)
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) acc[r][ch] = 0.f;

    for (int c0 = s; c0 < e; c0 += CH) {
      // ---- stage this chunk: particle q = c0 + tid
      const int q = c0 + tid;
      const int c1 = min(e, c0 + CH);
      if constexpr (RES) {
        int j = 0, lc = 0;
        bool keep = false;
        if (q < c1) {
          j = I.perm_out[q];
          lc = I.keys_out[q] & (CELLS_PER_TILE - 1);
          keep = full || j < os || j >= oe;
        }
        // compaction in binning order: warp counts, then offsets over the warps
        const unsigned km = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wkeep[warp] = __popc(km);
        __syncthreads();
        int base = 0, nkeep = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const int c = wkeep[w];
          base += w < warp ? c : 0;
          nkeep += c;
        }
        const int idx = base + __popc(km & ((1u << lane) - 1u));
        if (keep) {
          const PBuf &A = I.A;
          float u[D], v[D], sg[6];
#pragma unroll
          for (int k = 0; k < D; ++k) {
            u[k] = A.off(k)[j];
            v[k] = A.vel(k)[j];
          }
#pragma unroll
          for (int k = 0; k < 6; ++k) sg[k] = k < nstress<D>() ? A.sig(k)[j] : 0.f;
          float f[4 * NQ];
          p2g_record<D, MODE>(u, A.mass()[j], v, A.jm1()[j], sg, g.inv_rho, f);
          const int sl = rec_slot(idx);
#pragma unroll
          for (int k = 0; k < NQ; ++k)
            rec[k * CH + sl] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
          ccell[idx] = lc;
        }
        __syncthreads();
        if (keep) {  // run boundaries of the cell among the staged particles
          if (idx == 0 || ccell[idx - 1] != lc) {
            cs[lc] = idx;
            stamp[lc] = chunk_id;
          }
          if (idx == nkeep - 1 || ccell[idx + 1] != lc) ce[lc] = idx + 1;
        }
      } else if (q < c1) {
        const int j = I.perm_out[q];
        const int lc = I.keys_out[q] & (CELLS_PER_TILE - 1);
        // FORCE (USF) reads the stress updated earlier this step, stored in
        // binning order; USL and MOM read the state at the start of the step
        const PBuf &S = (MODE == P2G_FORCE) ? I.B : I.A;
        const int js = (MODE == P2G_FORCE) ? q : j;
        float u[D], v[D], sg[6];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          u[k] = I.A.off(k)[j];
          v[k] = R::HAS_M ? I.A.vel(k)[j] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) sg[k] = (R::HAS_F && k < nstress<D>()) ? S.sig(k)[js] : 0.f;
        float f[4 * NQ];
        p2g_record<D, MODE>(u, I.A.mass()[j], v, R::HAS_F ? S.jm1()[js] : 0.f, sg, g.inv_rho, f);
        const int sl = rec_slot(tid);
#pragma unroll
        for (int k = 0; k < NQ; ++k) rec[k * CH + sl] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
        // run boundaries of the cell within the chunk
        const bool first = q == c0 || (int)(I.keys_out[q - 1] & (CELLS_PER_TILE - 1)) != lc;
        const bool last = q == c1 - 1 || (int)(I.keys_out[q + 1] & (CELLS_PER_TILE - 1)) != lc;
        if (first) {
          cs[lc] = tid;
          stamp[lc] = chunk_id;
        }
        if (last) ce[lc] = tid + 1;
      }
      __syncthreads();
      // ---- accumulate my (cell, corner) pairs over the cell's particles in order
      if (stamp[my_cell] == chunk_id) accumulate_cell<D, MODE>(rec, cs[my_cell], ce[my_cell], my_cp, g.inv_h, acc);
      ++chunk_id;
      __syncthreads();  // the next chunk overwrites the records
    }

    // ---- cells -> node box (ascending local cell order), compensated; -> slot
#pragma unroll
    for (int r = 0; r < CPT; ++r)
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) cellP[my_cell * NV + (my_cp + r * CPC) * NCH + ch] = acc[r][ch];
    __syncthreads();
    cells_to_slot<D, NCH>(cellP, slots_out, t, CH);
    if (tid == 0) {
      if (RES) {
        if (full)
          I.s.fepoch[t] = step;
        else
          I.s.aepoch[t] = step;
      }
      s_work[(it + 1) & 1] = wnext;
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

// Active tiles whose box holds node I, in ascending tile order: bit i of the
// result is the i-th tile of the (at most 2 x 2 x 2) block lo..hi, `first`
// the lowest active tile index (-1 if none).  Activity comes from the
// 3 x 3 x 3 neighbourhood mask of tile tc (bit (dz + 1) 9 + (dy + 1) 3 +
// (dx + 1) set when that neighbour has particles).
template <int D>
__device__ __forceinline__ unsigned node_tiles_mask(const Geo &g, unsigned nmask, const int I[3], const int tc[3],
                                                    int lo[3], int hi[3], int &first) {
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  const int T[3] = {TX, TY, TZ};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lo[k] = hi[k] = tc[k];
    if (k < D) {
      const int l = I[k] - tc[k] * T[k];
      if (l == 0 && tc[k] > 0) lo[k] = tc[k] - 1;
      if (l == T[k] && tc[k] + 1 < g.nt[k]) hi[k] = tc[k] + 1;
    }
  }
  unsigned act = 0;
  int idx = 0;
  first = -1;
  for (int z = lo[2]; z <= hi[2]; ++z)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int x = lo[0]; x <= hi[0]; ++x, ++idx) {
        const int nb = (z - tc[2] + 1) * 9 + (y - tc[1] + 1) * 3 + (x - tc[0] + 1);
        if ((nmask >> nb) & 1u) {
          act |= 1u << idx;
          if (first < 0) first = x + g.nt[0] * (y + g.nt[1] * z);
        }
      }
  return act;
}

// Sum channels of node I over the slots of the active tiles `act` (from
// node_tiles_mask), in ascending tile order, so that the value does not depend on
// which tile computes it.  For up to four channels the loads of two holders
// are issued together before their sums, so a node held by two tiles (a box
// face node) waits for one memory latency, not two (measured: USF nodal
// stages 287 -> 277 and 316 -> 305 us on the 64M-particle slope; the same
// form of the USL gather, seven channels, was slower: 316 -> 349 us).
template <int D, int NOUT>
__device__ __forceinline__ void gather_node(const Geo &g, const float *slots, int nch, const int I[3], const int lo[3],
                                            const int hi[3], unsigned act, float out[NOUT]) {
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  constexpr int BN = box_nodes<D>();
  TwoAcc<float> acc[NOUT];
#pragma unroll
  for (int c = 0; c < NOUT; ++c) acc[c].init();
  if constexpr (NOUT > 4) {
    int idx = 0;
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x, ++idx) {
          if (!((act >> idx) & 1u)) continue;
          const int t2 = x + g.nt[0] * (y + g.nt[1] * z);
          const int bx = I[0] - x * TX, by = I[1] - y * TY, bz = D == 3 ? I[2] - z * TZ : 0;
          const int bl = bx + (TX + 1) * (by + (TY + 1) * bz);
#pragma unroll
          for (int c = 0; c < NOUT; ++c) acc[c].add(slots[((int64_t)t2 * nch + c) * BN + bl]);
        }
  } else {
    // the active holders in ascending tile order, as 3-bit offsets from lo
    unsigned codes = 0;
    int nh = 0, idx = 0;
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x, ++idx)
          if ((act >> idx) & 1u) {
            codes |= (unsigned)((x - lo[0]) | ((y - lo[1]) << 1) | ((z - lo[2]) << 2)) << (3 * nh);
            ++nh;
          }
    for (int h0 = 0; h0 < nh; h0 += 2) {
      float v[2][NOUT];
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (h0 + k < nh) {
          const unsigned cd = (codes >> (3 * (h0 + k))) & 7u;
          const int x = lo[0] + (int)(cd & 1u), y = lo[1] + (int)((cd >> 1) & 1u), z = lo[2] + (int)(cd >> 2);
          const int t2 = x + g.nt[0] * (y + g.nt[1] * z);
          const int bx = I[0] - x * TX, by = I[1] - y * TY, bz = D == 3 ? I[2] - z * TZ : 0;
          const int bl = bx + (TX + 1) * (by + (TY + 1) * bz);
#pragma unroll
          for (int c = 0; c < NOUT; ++c) v[k][c] = slots[((int64_t)t2 * nch + c) * BN + bl];
        }
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (h0 + k < nh)
#pragma unroll
          for (int c = 0; c < NOUT; ++c) acc[c].add(v[k][c]);
    }
  }
#pragma unroll
  for (int c = 0; c < NOUT; ++c) out[c] = acc[c].value();
}

// USL: sum channels of node I over the active tiles `act` in ascending tile
// order, taking each tile's sums of the particles that stayed (slots1) when
// they are for this step (bit of fmask27, the 3 x 3 x 3 neighbourhood of tc)
// and of the particles that arrived (slots_a) when those are (amask27).
template <int D, int NOUT>
__device__ __forceinline__ void gather_node_usl(const Geo &g, const float *slots, const float *slots_a, const int I[3],
                                                const int lo[3], const int hi[3], const int tc[3], unsigned act,
                                                unsigned fmask27, unsigned amask27, float out[NOUT]) {
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  constexpr int BN = box_nodes<D>();
  TwoAcc<float> acc[NOUT];
#pragma unroll
  for (int c = 0; c < NOUT; ++c) acc[c].init();
  int idx = 0;
  for (int z = lo[2]; z <= hi[2]; ++z)
    for (int y = lo[1]; y <= hi[1]; ++y)
      for (int x = lo[0]; x <= hi[0]; ++x, ++idx) {
        if (!((act >> idx) & 1u)) continue;
        const int nb = (z - tc[2] + 1) * 9 + (y - tc[1] + 1) * 3 + (x - tc[0] + 1);
        const int t2 = x + g.nt[0] * (y + g.nt[1] * z);
        const int bx = I[0] - x * TX, by = I[1] - y * TY, bz = D == 3 ? I[2] - z * TZ : 0;
        const int bl = bx + (TX + 1) * (by + (TY + 1) * bz);
        if ((fmask27 >> nb) & 1u)
#pragma unroll
          for (int c = 0; c < NOUT; ++c) acc[c].add(slots[((int64_t)t2 * NOUT + c) * BN + bl]);
        if ((amask27 >> nb) & 1u)
#pragma unroll
          for (int c = 0; c < NOUT; ++c) acc[c].add(slots_a[((int64_t)t2 * NOUT + c) * BN + bl]);
      }
#pragma unroll
  for (int c = 0; c < NOUT; ++c) out[c] = acc[c].value();
}

// The slot entries a tile needs for the nodes it owns when all its lower
// neighbours are active (its box's nodes at local 1..T on every axis): for
// each holder offset hd = dx + 2 dy + 4 dz (d in {0, 1}^D: ascending tile
// order), the owned nodes with b_k = T_k wherever d_k = 1, indexed over the
// other axes (x fastest).  They number exactly the box's nodes.
template <int D>
struct OwnEntries {
  __host__ __device__ static constexpr int T(int k) {
    return k == 0 ? Tile<D>::TX : (k == 1 ? Tile<D>::TY : (D == 3 ? Tile<D>::TZ : 1));
  }
  __host__ __device__ static constexpr int count(int hd) {
    int n = 1;
    for (int k = 0; k < D; ++k)
      if (!((hd >> k) & 1)) n *= T(k);
    return n;
  }
  __host__ __device__ static constexpr int base(int hd) {
    int b = 0;
    for (int h = 0; h < hd; ++h) b += count(h);
    return b;
  }
  static_assert(base(1 << D) == box_nodes<D>(), "one entry per box node");
  // entry of owned node b (local 1..T) and holder hd (b_k = T_k where d_k = 1)
  __device__ static __forceinline__ int entry(int hd, const int b[3]) {
    int e = 0, st = 1;
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (!((hd >> k) & 1)) {
        e += (b[k] - 1) * st;
        st *= T(k);
      }
    return base(hd) + e;
  }
};

// Stage the slot entries (NST channels of `slots`) of the nodes tile tc owns
// into sv[c][entry], two entries per lane with their loads in flight together,
// so the warp waits for two memory latencies per tile rather than one per
// holder of each of its nodes.  Entries of inactive holders are not loaded
// (never read).
template <int D, int NST>
__device__ __forceinline__ void stage_own_entries(const Geo &g, const float *slots, const int tc[3], unsigned nmask,
                                                  int lane, float (*sv)[box_nodes<D>()]) {
  using E = OwnEntries<D>;
  constexpr int BN = box_nodes<D>();
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY;
  constexpr int NI = (BN + 31) / 32;  // entries per lane
  constexpr int SG = 2;               // entries whose loads are in flight together
#pragma unroll
  for (int i0 = 0; i0 < NI; i0 += SG) {
    float v[SG][NST];
    int ent[SG];
#pragma unroll
    for (int i = 0; i < SG; ++i) {
      const int e = lane + 32 * (i0 + i);
      ent[i] = -1;
      if (i0 + i >= NI || e >= BN) continue;
      int hd = 0;
#pragma unroll
      for (int h = 1; h < (1 << D); ++h)
        if (e >= E::base(h)) hd = h;
      int r = e - E::base(hd), bh[3] = {0, 0, 0}, d[3] = {0, 0, 0};
#pragma unroll
      for (int k = 0; k < D; ++k) {
        d[k] = (hd >> k) & 1;
        if (!d[k]) {
          bh[k] = 1 + r % E::T(k);  // the node's local coordinate, also the holder's (d_k = 0)
          r /= E::T(k);
        }
      }
      const int nb = (d[2] + 1) * 9 + (d[1] + 1) * 3 + (d[0] + 1);
      if (!((nmask >> nb) & 1u)) continue;
      ent[i] = e;
      const int t2 = (tc[0] + d[0]) + g.nt[0] * ((tc[1] + d[1]) + g.nt[1] * (tc[2] + d[2]));
      const int bl = bh[0] + (TX + 1) * (bh[1] + (TY + 1) * bh[2]);
#pragma unroll
      for (int c = 0; c < NST; ++c) v[i][c] = slots[((int64_t)t2 * NST + c) * BN + bl];
    }
#pragma unroll
    for (int i = 0; i < SG; ++i)
      if (ent[i] >= 0)
#pragma unroll
        for (int c = 0; c < NST; ++c) sv[c][ent[i]] = v[i][c];
  }
}

// Sum the staged entries of owned node b (local 1..T) over its active
// holders in ascending tile order (the order of gather_node).
template <int D, int NOUT>
__device__ __forceinline__ void combine_own_entries(const float (*sv)[box_nodes<D>()], const int b[3], unsigned nmask,
                                                    float out[NOUT]) {
  using E = OwnEntries<D>;
  // the tile itself (hd = 0) holds every node it owns and comes first: its
  // entry starts the sums (what adding it to zero gives)
  TwoAcc<float> acc[NOUT];
  const int e0 = E::entry(0, b);
#pragma unroll
  for (int c = 0; c < NOUT; ++c) {
    acc[c].hi = sv[c][e0];
    acc[c].lo = 0.f;
  }
#pragma unroll
  for (int hd = 1; hd < (1 << D); ++hd) {
    bool holds = true;
#pragma unroll
    for (int k = 0; k < D; ++k)
      if ((hd >> k) & 1) holds = holds && b[k] == E::T(k);
    const int nb = (((hd >> 2) & 1) + 1) * 9 + (((hd >> 1) & 1) + 1) * 3 + ((hd & 1) + 1);
    if (holds && ((nmask >> nb) & 1u)) {
      const int e = E::entry(hd, b);
#pragma unroll
      for (int c = 0; c < NOUT; ++c) acc[c].add(sv[c][e]);
    }
  }
#pragma unroll
  for (int c = 0; c < NOUT; ++c) out[c] = acc[c].value();
}

// Work items dealt to the warps of the grid in turn (the work per item is
// uniform): a 32-node slice of an active tile's box when there are few
// active tiles, a whole box (four slices in turn) when there are enough to
// fill the grid.  The nodes whose lowest active holder is the tile -- every
// node is computed once -- get v = P/m, a = f/m + g, v' = v + a dt and the
// boundary conditions, written to the dense node records.
template <int D, int NMODE, bool ONE, bool MAP = false>
__global__ void __launch_bounds__(NODE_T, ONE ? MPM_NODE_MINB : 8) node_tile(const __grid_constant__ GroupArgs G, int work_slot) {
  constexpr int BN = box_nodes<D>();
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  constexpr int NCH1 = NMODE == NODE_USL ? 1 + 2 * D : 1 + D;
  constexpr int NW = NODE_T / 32;
  constexpr int NSL = (BN + 31) / 32;  // slices per tile
  constexpr int NOWN = CELLS_PER_TILE / 32;  // slices of the nodes at local 1..T on every axis
  static_assert(CELLS_PER_TILE % 32 == 0, "owned-node slices");
  // neighbourhood-mask bits of the lower neighbours (offsets in {-1, 0}^D, not all 0)
  constexpr unsigned LOWER = D == 3 ? (1u << 0) | (1u << 1) | (1u << 3) | (1u << 4) | (1u << 9) | (1u << 10) | (1u << 12)
                                    : (1u << 9) | (1u << 10) | (1u << 12);
  // channels staged per owned-node walk: the sums the node needs (the USF
  // force stage gathers only the forces; its mass and velocity are in the
  // record).  Staged: the USF stages (64M slope 275 -> 216 and 305 -> 232
  // us); the seven-channel USL sums were slower staged (311 -> 420 us) and
  // gather per node.
  constexpr int NST = NMODE == NODE_USF_A ? D : NCH1;
  constexpr bool STAGE = !MAP && NMODE != NODE_USL;
  __shared__ InstArgs sI[NW];
  __shared__ float sv_all[STAGE ? NW * NST * BN : 1];
  float(*const sv)[BN] = reinterpret_cast<float(*)[BN]>(sv_all + (STAGE ? (threadIdx.x >> 5) * NST * BN : 0));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const InstArgs &I = inst_ref<ONE>(G, sI[warp]);
  (void)work_slot;
  pdl_trigger();
  pdl_wait();
  int loaded = -1;
  const int stride = gridDim.x * NW;
  const int nact = G.act_items[G.ninst];
  const int split = nact * NSL <= 2 * stride ? NSL : 1;  // items per tile
  const int total = nact * split;
  for (int wi = blockIdx.x * NW + warp; wi < total; wi += stride) {
    const int item = wi / split, slice0 = wi % split;
    const int ii = ONE ? 0 : find_inst(G.act_items, G.ninst, item);
    if (!ONE && ii != loaded) {  // warp-uniform
      const unsigned long long *src = reinterpret_cast<const unsigned long long *>(G.inst + ii);
      unsigned long long *dst = reinterpret_cast<unsigned long long *>(&sI[warp]);
      for (int i = lane; i < (int)(sizeof(InstArgs) / 8); i += 32) dst[i] = __ldg(src + i);
      __syncwarp();
      loaded = ii;
    }
    const Geo &g = I.geo;
    const int t = I.s.active[ONE ? item : item - G.act_items[ii]].x;
    int tc[3];
    tile_coords(g, t, tc);
    // activity of the 27 tiles around t, one lane each (USL: and whether
    // their stayers' and arrivals' sums are for this step)
    bool nact = false, fv = false, av = false;
    if (lane < 27) {
      const int d[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
      const int n3[3] = {tc[0] + d[0], tc[1] + d[1], tc[2] + d[2]};
      bool in = D == 3 || d[2] == 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) in = in && n3[k] >= 0 && n3[k] < g.nt[k];
      if (in) {
        const int t2 = n3[0] + g.nt[0] * (n3[1] + g.nt[1] * n3[2]);
        nact = I.new_start[t2 + 1] > I.new_start[t2];
        if (NMODE == NODE_USL && MPM_FUSED_USL) {
          const int step = I.s.ctr[C_STEP];
          fv = I.s.fepoch[t2] == step;
          av = I.s.aepoch[t2] == step;
        }
      }
    }
    const unsigned nmask = __ballot_sync(0xffffffffu, nact);
    const unsigned fmask27 = __ballot_sync(0xffffffffu, fv), amask27 = __ballot_sync(0xffffffffu, av);
    // One warp walking a whole box whose lower neighbours are all active
    // computes just the nodes at local 1..T on every axis: a node on a lower
    // face (a local coordinate 0) is held by the active lower neighbour
    // along that axis, whose index is lower.  Otherwise, and for one slice
    // per warp, the walk is in box order with the ownership test below.
    const bool own_only = split == 1 && (nmask & LOWER) == LOWER;  // warp-uniform
    // such a walk stages the slot entries of all its nodes first
    const bool staged = STAGE && own_only;
    if (staged) {
      stage_own_entries<D, NST>(g, NMODE == NODE_USF_A ? I.s.slots2 : I.s.slots1, tc, nmask, lane, sv);
      __syncwarp();
    }
    for (int sl = slice0; sl < (split == 1 ? (own_only ? NOWN : NSL) : slice0 + 1); ++sl) do {  // a node per lane
      const int b = sl * 32 + lane;
      if (b >= BN) break;  // break: nothing to write for this lane
      const int bx = own_only ? 1 + b % TX : b % (TX + 1);
      const int by = own_only ? 1 + (b / TX) % TY : (b / (TX + 1)) % (TY + 1);
      const int bz = D == 3 ? (own_only ? 1 + b / (TX * TY) : b / ((TX + 1) * (TY + 1))) : 0;
      const int Ig[3] = {tc[0] * TX + bx, tc[1] * TY + by, D == 3 ? tc[2] * TZ + bz : 0};
      bool inside = true;
#pragma unroll
      for (int k = 0; k < D; ++k) inside = inside && Ig[k] <= g.nc[k];
      if (!inside) break;
      int lo[3], hi[3], first = t;
      unsigned act = 0;
      if (!staged) act = node_tiles_mask<D>(g, nmask, Ig, tc, lo, hi, first);  // (a staged walk owns its nodes)
      if (first != t) break;  // a lower active tile computes this node
      float v[D], a[D], vn[D];
#pragma unroll
      for (int k = 0; k < D; ++k) v[k] = a[k] = vn[k] = 0.f;
      const int gi = Ig[0] + I.ns0 * Ig[1] + I.ns1 * Ig[2];
      float c1[1 + 2 * D];
      if (NMODE == NODE_USL && MPM_FUSED_USL) {
        gather_node_usl<D, 1 + 2 * D>(g, I.s.slots1, I.s.slots_a, Ig, lo, hi, tc, act, fmask27, amask27, c1);
      } else if (NMODE != NODE_USF_A && staged) {
        const int bb[3] = {bx, by, bz};
        combine_own_entries<D, NCH1>(sv, bb, nmask, c1);
      } else if (NMODE == NODE_USL) {
        gather_node<D, 1 + 2 * D>(g, I.s.slots1, NCH1, Ig, lo, hi, act, c1);
      } else if (NMODE == NODE_USF_V) {
        gather_node<D, 1 + D>(g, I.s.slots1, NCH1, Ig, lo, hi, act, c1);
      } else {
        // the USF force stage: the node's mass and its constrained velocity
        // as the velocity stage left them in its record (the same values a
        // second gather of the mass and momentum would give)
        const float4 r = I.s.node[(D == 3 ? 2 : 1) * gi];
        c1[0] = D == 3 ? r.w : r.z;
        c1[1] = r.x;
        c1[2] = r.y;
        if (D == 3) c1[D] = r.z;
      }
      const float m = c1[0];
      const int faces = node_faces<D>(g, Ig);
      // a mapped mesh's boundary node: its faces' outward normals
      float nrm[6][3];
      if (MAP && faces) {
#pragma unroll
        for (int f = 0; f < 2 * D; ++f)
          if ((faces >> f) & 1) {
            const float4 q = __ldg(g.fnorm + g.fnoff[f] + face_node_index<D>(f, Ig, g.nc));
            nrm[f][0] = q.x;
            nrm[f][1] = q.y;
            nrm[f][2] = q.z;
          }
      }
      if (m > g.mass_tol) {
        const float inv_m = 1.f / m;
#pragma unroll
        for (int k = 0; k < D; ++k) v[k] = NMODE == NODE_USF_A ? c1[1 + k] : c1[1 + k] * inv_m;
        if (NMODE == NODE_USL) {
          float ft[D];
          if (g.loads) face_force<D, float>(faces, Ig, g.nc, g.h, g.trac, ft);
          if (MAP && g.loads && g.fload && faces) add_face_loads<D>(g, faces, Ig, ft);
#pragma unroll
          for (int k = 0; k < D; ++k) {
            a[k] = g.loads ? (c1[1 + D + k] + ft[k]) * inv_m + g.g[k] - g.damp * v[k] : c1[1 + D + k] * inv_m + g.g[k];
            vn[k] = v[k] + a[k] * g.dt;
          }
          if (MAP && faces)
            bc_full_n<D, float>(faces, g.bc, g.mu, g.dt, nrm, v, a, vn);
          else
            bc_full<D, float>(faces, g.bc, g.mu, g.dt, v, a, vn);
        } else if (NMODE == NODE_USF_V) {
          if (MAP && faces)
            bc_velocity_n<D, float>(faces, g.bc, nrm, v);
          else
            bc_velocity<D, float>(faces, g.bc, v);
        } else {
          float f[D];
          if (staged) {
            const int bb[3] = {bx, by, bz};
            combine_own_entries<D, D>(sv, bb, nmask, f);
          } else {
            gather_node<D, D>(g, I.s.slots2, D, Ig, lo, hi, act, f);
          }
          float ft[D];
          if (g.loads) face_force<D, float>(faces, Ig, g.nc, g.h, g.trac, ft);
          if (MAP && g.loads && g.fload && faces) add_face_loads<D>(g, faces, Ig, ft);
#pragma unroll
          for (int k = 0; k < D; ++k) {
            a[k] = g.loads ? (f[k] + ft[k]) * inv_m + g.g[k] - g.damp * v[k] : f[k] * inv_m + g.g[k];
            vn[k] = v[k] + a[k] * g.dt;
          }
          if (MAP && faces)
            bc_full_n<D, float>(faces, g.bc, g.mu, g.dt, nrm, v, a, vn);
          else
            bc_full<D, float>(faces, g.bc, g.mu, g.dt, v, a, vn);
        }
      }
      const float *w = NMODE == NODE_USF_V ? v : vn;
      // the velocity stage keeps the node's mass where the force stage reads
      // it (3D: the spare fourth component; 2D: the acceleration slot, unused
      // until the force stage writes it)
      const float ms = NMODE == NODE_USF_V ? m : 0.f;
      if (D == 3) {
        I.s.node[2 * gi] = make_float4(w[0], w[1], w[D - 1], ms);
        I.s.node[2 * gi + 1] = make_float4(a[0], a[1], a[D - 1], 0.f);
      } else {
        I.s.node[gi] = make_float4(w[0], w[1], NMODE == NODE_USF_V ? ms : a[0], a[1]);
      }
    } while (0);
    __syncwarp();  // the instance copy and the staged entries may be replaced next
  }
}


// ---------------------------------------------------------------------------
// G2P: one thread per particle in binning order, G2P_T-thread CTAs.  Right
// after reading its storage slot, each thread starts cp.async copies of its
// particle's state (all but the offset) into its own shared-memory column;
// they land while the node gather runs, and the thread waits only on its own
// copies.
// ---------------------------------------------------------------------------
template <int D, int GMODE, bool ONE, bool MAP = false>
__global__ void __launch_bounds__(G2P_T, g2p_min_blocks<D, GMODE, MAP>()) g2p(const __grid_constant__ GroupArgs G) {
  constexpr int NC = 1 << D;
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  constexpr int NS = nstress<D>();
  __shared__ InstArgs sI;
  pdl_trigger();
  const int unit = blockIdx.x / G2P_SUB;
  const int ii = ONE ? 0 : find_inst(G.pblk, G.ninst, unit);  // host-written tables
  if (!ONE) copy_inst(G.inst, ii, &sI);
  pdl_wait();
  if (!ONE) __syncthreads();
  const InstArgs &I = inst_ref<ONE>(G, sI);
  const Geo &g = I.geo;
  // the binning key travels with the permutation (both coalesced, in flight
  // at once): the cell, its node records and whether the particle is still
  // in the mesh are known while the offset and the state are on their way
  const int64_t q = (int64_t)(unit - (ONE ? 0 : G.pblk[ii])) * 256 + (blockIdx.x % G2P_SUB) * G2P_T + threadIdx.x;
  if (q >= I.n) return;
  const int j = I.perm_out[q];
  const uint32_t key = I.keys_out[q];
  const bool gone = (int)(key >> LOCAL_BITS) >= I.ntiles;  // left the mesh in an earlier step
  // the particle's state (all but its offset) travels to this thread's
  // shared-memory column while the node gather runs, without holding
  // registers: stress-stage fields (sig, eps, J-1, eps_p), then kinematic
  // ones (velocity, mass, id), then cohesion
  constexpr bool KIN = GMODE != G2P_USF_STRESS, STR = GMODE != G2P_USF_ADVECT;
  constexpr int S_VEL = STR ? 2 * NS + 2 : 0, S_MASS = S_VEL + D, S_ID = S_MASS + 1;
  constexpr int S_COH = KIN ? S_ID + 1 : S_VEL;
  __shared__ float stg[S_COH + 1][G2P_T];
  const bool has_coh = I.A.coh() != nullptr;
  if (!gone) {
    if (STR) {
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        cp_async4(&stg[i][threadIdx.x], I.A.sig(i) + j);
        cp_async4(&stg[NS + i][threadIdx.x], I.A.eps(i) + j);
      }
      cp_async4(&stg[2 * NS][threadIdx.x], I.A.jm1() + j);
      cp_async4(&stg[2 * NS + 1][threadIdx.x], I.A.epsp() + j);
    }
    if (KIN) {
#pragma unroll
      for (int k = 0; k < D; ++k) cp_async4(&stg[S_VEL + k][threadIdx.x], I.A.vel(k) + j);
      cp_async4(&stg[S_MASS][threadIdx.x], I.A.mass() + j);
      cp_async4(&stg[S_ID][threadIdx.x], I.A.id() + j);
    }
    if (has_coh) cp_async4(&stg[S_COH][threadIdx.x], I.A.coh() + j);
    cp_async_commit();
  }
  if (gone) {  // carried over unchanged
    if (GMODE != G2P_USF_STRESS) {
      I.B.key()[q] = key;
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
  const int t = key >> LOCAL_BITS;
  int tc[3], lc[3];
  tile_coords(g, t, tc);
  local_coords<D>(key, lc);
  int cell[3] = {tc[0] * TX + lc[0], tc[1] * TY + lc[1], D == 3 ? tc[2] * TZ + lc[2] : 0};
  {  // the cell's node records into L1 while the offset loads
    const int gp = cell[0] + I.ns0 * cell[1] + I.ns1 * cell[2];
#pragma unroll
    for (int r = 0; r < (D == 3 ? 4 : 2); ++r) {
      const float4 *nr = I.s.node + (D == 3 ? 2 : 1) * (gp + I.ns0 * (r & 1) + (D == 3 ? I.ns1 * (r >> 1) : 0));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(nr));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(nr + (D == 3 ? 3 : 1)));
    }
  }
  float u[D], w0[D], w1[D];
#pragma unroll
  for (int k = 0; k < D; ++k) u[k] = I.A.off(k)[j];
  corner_weights<D>(u, w0, w1);
  // mapped cell: its corners, the image of u and K = J^-1 at u
  float Pc[1 << D][D], K[D][D], xl[D];
  bool bad_cell = false;
  if constexpr (MAP) {
    float J[D][D];
    load_cgeo<D>(g, cell_lin<D>(g, cell), Pc);
    cgeo_map<D>(Pc, u, xl, J);
    if (!inv_jac<D>(J, K)) {
      bad_cell = true;
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) K[a][b] = 0.f;
    }
  }
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
    if constexpr (D == 3) {
      // paired FP32 FMAs: each lane is the same single-rounding FMA as the
      // scalar accumulation below, two per instruction
      if (GMODE != G2P_USF_STRESS) {
        const float2 NN = make_float2(N, N);
        const float2 a01 = __ffma2_rn(NN, make_float2(na[0], na[1]), make_float2(dv[0], dv[1]));
        const float2 v01 = __ffma2_rn(NN, make_float2(nv[0], nv[1]), make_float2(vb[0], vb[1]));
        dv[0] = a01.x;
        dv[1] = a01.y;
        dv[2] = fmaf(N, na[2], dv[2]);
        vb[0] = v01.x;
        vb[1] = v01.y;
        vb[2] = fmaf(N, nv[2], vb[2]);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float2 l01 = __ffma2_rn(make_float2(nv[k], nv[k]), make_float2(G[0], G[1]), make_float2(L[k][0], L[k][1]));
        L[k][0] = l01.x;
        L[k][1] = l01.y;
        L[k][2] = fmaf(nv[k], G[2], L[k][2]);
      }
    } else {
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
  }

  if constexpr (MAP) {  // velocity gradient: (sum_a v_a (x) dN_a/du) K / h
    float Lm[D][D];
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int l = 0; l < D; ++l) {
        float sacc = 0.f;
#pragma unroll
        for (int m = 0; m < D; ++m) sacc = fmaf(L[k][m], K[m][l], sacc);
        Lm[k][l] = sacc;
      }
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int l = 0; l < D; ++l) L[k][l] = Lm[k][l];
  }

  // Every load of the particle's state is issued before the first store: the
  // compiler cannot tell A from B, so a load placed after a store would wait
  // for the value before it (one memory latency per field).
  float v0[D], sg[6], ep[6], jm1 = 0.f, epsp = 0.f, mass = 0.f, coh = I.mat.c;
  int32_t pid = 0;
  cp_async_wait_all();
  if (KIN) {
#pragma unroll
    for (int k = 0; k < D; ++k) v0[k] = stg[S_VEL + k][threadIdx.x];
    mass = stg[S_MASS][threadIdx.x];
    pid = __float_as_int(stg[S_ID][threadIdx.x]);
  }
  if (has_coh) coh = stg[S_COH][threadIdx.x];
  if (STR) {
#pragma unroll
    for (int i = 0; i < 6; ++i) sg[i] = ep[i] = 0.f;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      sg[i] = stg[i][threadIdx.x];
      ep[i] = stg[NS + i][threadIdx.x];
    }
    jm1 = stg[2 * NS][threadIdx.x];
    epsp = stg[2 * NS + 1][threadIdx.x];
  }

  int status = bad_cell ? ST_NONFINITE : 0;
  // FLIP velocity, advection in cell units, relocation
  if (KIN) {
    bool dead = false;
    if constexpr (MAP) {
      // the target x(u) + dt vb / h in the cell's frame; Newton from the
      // step K dt vb / h; a solution outside [-0.5, 0.5) moves to the
      // neighbour across the face of the largest excess, the target into the
      // neighbour's frame (the shared node seen from both centres), and
      // solves again -- at most 8 cells per step
      float T[D], un[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float vk = v0[k] + g.dt * dv[k];
        I.B.vel(k)[q] = vk;
        if (!isfinite(vk)) status |= ST_NONFINITE;
        T[k] = g.dt * vb[k] * g.inv_h;
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        float d = 0.f;
#pragma unroll
        for (int m = 0; m < D; ++m) d = fmaf(K[k][m], T[m], d);
        un[k] = u[k] + d;
      }
#pragma unroll
      for (int k = 0; k < D; ++k) T[k] += xl[k];
      bool found = false;
      for (int hop = 0; hop < 8; ++hop) {
        cgeo_solve<D>(Pc, T, un);
        bool fin = true;
#pragma unroll
        for (int k = 0; k < D; ++k) fin = fin && isfinite(un[k]);
        if (!fin) {
          status |= ST_NONFINITE;
          dead = true;
          break;
        }
        int best = -1;
        float ex = -1.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float e = un[k] >= 0.5f ? un[k] - 0.5f : (un[k] < -0.5f ? -0.5f - un[k] : -1.f);
          if (e >= 0.f && e > ex) {
            ex = e;
            best = k;
          }
        }
        if (best < 0) {
          found = true;
          break;
        }
        // (indices stay compile-time constants: selects, not local memory)
        int sgn = 0;
        bool off_grid = false;
#pragma unroll
        for (int k = 0; k < D; ++k)
          if (k == best) {
            sgn = un[k] >= 0.5f ? 1 : -1;
            cell[k] += sgn;
            un[k] -= (float)sgn;
            off_grid = cell[k] < 0 || cell[k] >= g.nc[k];
          }
        if (off_grid) {
          dead = true;
          break;
        }
        float Pn[1 << D][D];
        load_cgeo<D>(g, cell_lin<D>(g, cell), Pn);
        const int ao = sgn > 0 ? (1 << best) : 0, an = sgn > 0 ? 0 : (1 << best);
#pragma unroll
        for (int a = 0; a < (1 << D); ++a)
#pragma unroll
          for (int k = 0; k < D; ++k) {
            if (a == ao) T[k] -= Pc[a][k];
            if (a == an) T[k] += Pn[a][k];
          }
#pragma unroll
        for (int a = 0; a < (1 << D); ++a)
#pragma unroll
          for (int k = 0; k < D; ++k) Pc[a][k] = Pn[a][k];
      }
      if (!found) dead = true;
#pragma unroll
      for (int k = 0; k < D; ++k) I.B.off(k)[q] = dead ? 0.f : un[k];
    }
#pragma unroll
    for (int k = 0; k < (MAP ? 0 : D); ++k) {
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
    // tile movers for the next step's binning; one append per warp
    const int tn = min((int)(nkey >> LOCAL_BITS), I.ntiles);
    const bool mover = tn != t;
    const unsigned am = __activemask();
    const unsigned mv = __ballot_sync(am, mover);
    if (mover) {
      const int lane = threadIdx.x & 31;
      const int leader = __ffs(mv) - 1;
      int base = 0;
      if (lane == leader) base = atomicAdd(&I.s.ctr[C_MOVERS], __popc(mv));
      base = __shfl_sync(mv, base, leader);
      atomicAdd(&I.s.in_cnt[tn], 1);
      atomicAdd(&I.s.out_cnt[t], 1);
      I.s.movers[base + __popc(mv & ((1u << lane) - 1u))] = (int32_t)q;
    }
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
    // a trial in the apex band keeps its trial stress here and is queued for
    // the FP64 return (apex_band_k, right after this kernel)
    if (material_update_inline(I.mat, coh, sg, de, epsp)) I.s.bucket_sorted[atomicAdd(&I.s.ctr[C_APEX], 1)] = (int32_t)q;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      I.B.sig(i)[q] = sg[i];
      if (!isfinite(sg[i])) status |= ST_NONFINITE;
    }
    I.B.epsp()[q] = epsp;
  }
  if (status) atomicOr(&I.s.ctr[C_STATUS], status);
}

// Every field of particle j of A copied to slot q of B (a particle that left
// the mesh earlier is carried over unchanged).
template <int D>
__device__ __forceinline__ void copy_particle(const PBuf &A, const PBuf &B, int j, int64_t q) {
  constexpr int NS = nstress<D>();
  B.key()[q] = A.key()[j];
  B.id()[q] = A.id()[j];
  B.mass()[q] = A.mass()[j];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    B.off(k)[q] = A.off(k)[j];
    B.vel(k)[q] = A.vel(k)[j];
  }
  if (A.coh()) B.coh()[q] = A.coh()[j];
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    B.sig(i)[q] = A.sig(i)[j];
    B.eps(i)[q] = A.eps(i)[j];
  }
  B.jm1()[q] = A.jm1()[j];
  B.epsp()[q] = A.epsp()[j];
}

__device__ __forceinline__ int warp_incl(int x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// ---------------------------------------------------------------------------
// USL G2P fused with the next step's P2G: one CTA per active tile (and one
// item for the particles that left the mesh earlier).  The CTA loads the node
// records of the tile's box into shared memory once; then, in chunks of one
// particle per thread (binning order), each thread runs the particle's whole
// G2P update -- FLIP velocity, advection and relocation, strain, stress,
// volume -- from the box, with the particle's state copied to shared memory
// by cp.async while the node gather runs.  A particle that stays in the tile
// then forms its P2G record for the next step (the same arithmetic as P2G
// from the stored state); the chunk's records are sorted by their new local
// cell: each thread of a (cell, corner pair) adds, to its running sums in
// shared memory, the records of the particles of its cell that stayed in it
// (the chunk is in binning order, so they form the cell's run), then those of
// the particles that moved into it from another cell of the tile (listed per
// warp, in binning order).  At the end the cells go to the tile's node box
// and the box to slots1, valid for the next step (fepoch = step + 1).
// Particles that leave the tile are left to the next step's residual P2G
// (they arrive in another tile), as are tiles whose FP64 apex-band returns
// change a stress after this kernel (apex_band_k invalidates their sums).
// While no particle changes cell, each (cell, corner) sums in the order the
// plain P2G of the stored state uses, so the sums are the same.  Two
// barriers per chunk.
// ---------------------------------------------------------------------------
#ifndef MPM_G2PF_MINB
#define MPM_G2PF_MINB 3  // resident fused G2P CTAs per SM the register budget is sized for
#endif
template <int D>
struct G2PF {
  using R = P2GRec<D, P2G_USL>;
  static constexpr int T = R::CH;  // threads: a particle each in G2P, a (cell, corner pair) each in P2G
  static constexpr int NCH = 1 + 2 * D, NV = R::NV, NQ = R::NQ, NS = nstress<D>();
  static constexpr int NREC = D == 3 ? 2 : 1;  // float4 node records per node
  static constexpr int BN = box_nodes<D>();
  // staged state: sig, eps, J-1, eps_p, velocity, mass, id, cohesion
  static constexpr int S_SIG = 0, S_EPS = NS, S_JM1 = 2 * NS, S_EPSP = 2 * NS + 1, S_VEL = 2 * NS + 2,
                       S_MASS = S_VEL + D, S_ID = S_MASS + 1, S_COH = S_ID + 1, NSTG = S_COH + 1;
  static constexpr size_t STG_BYTES = (sizeof(float) * NSTG * T + 15) / 16 * 16;
  static constexpr size_t REC_BYTES = sizeof(float4) * NQ * T;
  static constexpr size_t CELLP_BYTES = (sizeof(float) * CELLS_PER_TILE * NV + 15) / 16 * 16;
  static constexpr size_t NODES_BYTES = sizeof(float4) * BN * NREC;
  static constexpr size_t SMEM = REC_BYTES + STG_BYTES + CELLP_BYTES + NODES_BYTES;
};

template <int D, bool ONE>
__global__ void __launch_bounds__(G2PF<D>::T, MPM_G2PF_MINB) g2p_tile(const __grid_constant__ GroupArgs G) {
  using F = G2PF<D>;
  constexpr int T = F::T, NCH = F::NCH, NV = F::NV, NQ = F::NQ, NS = F::NS, NREC = F::NREC, BN = F::BN;
  constexpr int NC = 1 << D;
  constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ;
  constexpr int CPT = F::R::CPT, CPC = F::R::CPC;
  constexpr int NW = T / 32;
  extern __shared__ float4 sm4[];
  float4 *rec = sm4;                                                                  // [NQ][T] P2G records
  float *stg = reinterpret_cast<float *>(reinterpret_cast<char *>(sm4) + F::REC_BYTES);  // [NSTG][T] state
  float *cellP = reinterpret_cast<float *>(reinterpret_cast<char *>(sm4) + F::REC_BYTES + F::STG_BYTES);  // [64][NV]
  float4 *nodes_s =
      reinterpret_cast<float4 *>(reinterpret_cast<char *>(sm4) + F::REC_BYTES + F::STG_BYTES + F::CELLP_BYTES);
  __shared__ int cs[CELLS_PER_TILE], ce[CELLS_PER_TILE], stamp[CELLS_PER_TILE];  // runs of the old cells
  __shared__ uint8_t kind[T];      // 1: stays in its cell, 2: moves to another cell of the tile, 0: neither
  __shared__ uint8_t ncell[T];     // new local cell of a kind-2 particle
  __shared__ uint8_t mvw[NW][32];  // per warp: its kind-2 particles, in binning order
  __shared__ int cntw[NW];
  __shared__ int s_work[2];
  __shared__ InstArgs sI;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int my_cell = tid / CPC, my_cp = tid % CPC;  // corners my_cp + r * CPC
  pdl_trigger();
  if (tid < CELLS_PER_TILE) stamp[tid] = -1;
  pdl_wait();
  // items: first the CTA's own (blockIdx.x), then gridDim.x + the work counter
  const int total = G.bin_items[G.ninst];
  if (tid == 0) s_work[0] = blockIdx.x;
  __syncthreads();
  int loaded = -1, chunk_id = 0;

  for (int it = 0;; ++it) {
    const int wi = s_work[it & 1];
    if (wi >= total) break;
    int wnext = 0;
    if (tid == 0) wnext = (int)gridDim.x + atomicAdd(&G.work[W_G2P], 1);
    const int ii = ONE ? 0 : find_inst(G.bin_items, G.ninst, wi);
    if (!ONE && ii != loaded) {  // uniform
      copy_inst(G.inst, ii, &sI);
      loaded = ii;
      __syncthreads();
    }
    const InstArgs &I = inst_ref<ONE>(G, sI);
    const Geo &g = I.geo;
    const int4 ar = I.s.active[ONE ? wi : wi - G.bin_items[ii]];
    const int t = ar.x, s = ar.y, e = ar.z;
    if (t >= I.ntiles) {  // the particles that left the mesh earlier: carried over unchanged
      for (int q = s + tid; q < e; q += T) copy_particle<D>(I.A, I.B, I.perm_out[q], q);
      if (tid == 0) s_work[(it + 1) & 1] = wnext;
      __syncthreads();
      continue;
    }
    const int step = I.s.ctr[C_STEP];
    int tc[3];
    tile_coords(g, t, tc);
    // the node records of the tile's box (nodes beyond the mesh: zeros, never read)
    for (int b = tid; b < BN * NREC; b += T) {
      const int bn = b / NREC, r = b - bn * NREC;
      const int bx = bn % (TX + 1), by = (bn / (TX + 1)) % (TY + 1), bz = D == 3 ? bn / ((TX + 1) * (TY + 1)) : 0;
      const int I0 = tc[0] * TX + bx, I1 = tc[1] * TY + by, I2 = D == 3 ? tc[2] * TZ + bz : 0;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (I0 <= g.nc[0] && I1 <= g.nc[1] && (D == 2 || I2 <= g.nc[2]))
        v = I.s.node[(int64_t)NREC * (I0 + I.ns0 * I1 + I.ns1 * I2) + r];
      nodes_s[b] = v;
    }
#pragma unroll
    for (int r = 0; r < CPT; ++r)
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) cellP[my_cell * NV + (my_cp + r * CPC) * NCH + ch] = 0.f;
    __syncthreads();

    for (int c0 = s; c0 < e; c0 += T) {
      const int q = c0 + tid;
      const int c1 = min(e, c0 + T);
      int kd = 0;                 // kind of this thread's particle
      unsigned lcn = 0;           // its new local cell
      if (q < e) {
        const int j = I.perm_out[q];
        const uint32_t key = I.keys_out[q];
        const bool has_coh = I.A.coh() != nullptr;
        // the state (all but the offset) travels to this thread's shared
        // column while the node gather runs
#pragma unroll
        for (int i = 0; i < NS; ++i) {
          cp_async4(&stg[(F::S_SIG + i) * T + tid], I.A.sig(i) + j);
          cp_async4(&stg[(F::S_EPS + i) * T + tid], I.A.eps(i) + j);
        }
        cp_async4(&stg[F::S_JM1 * T + tid], I.A.jm1() + j);
        cp_async4(&stg[F::S_EPSP * T + tid], I.A.epsp() + j);
#pragma unroll
        for (int k = 0; k < D; ++k) cp_async4(&stg[(F::S_VEL + k) * T + tid], I.A.vel(k) + j);
        cp_async4(&stg[F::S_MASS * T + tid], I.A.mass() + j);
        cp_async4(&stg[F::S_ID * T + tid], I.A.id() + j);
        if (has_coh) cp_async4(&stg[F::S_COH * T + tid], I.A.coh() + j);
        cp_async_commit();
        int lc[3];
        local_coords<D>(key, lc);
        {  // runs of the old cells within the chunk (binning order groups them)
          const int lo = key & (CELLS_PER_TILE - 1);
          if (q == c0 || (int)(I.keys_out[q - 1] & (CELLS_PER_TILE - 1)) != lo) {
            cs[lo] = tid;
            stamp[lo] = chunk_id;
          }
          if (q == c1 - 1 || (int)(I.keys_out[q + 1] & (CELLS_PER_TILE - 1)) != lo) ce[lo] = tid + 1;
        }
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
        const int b0 = lc[0] + (TX + 1) * (lc[1] + (TY + 1) * lc[2]);
#pragma unroll
        for (int a = 0; a < NC; ++a) {
          float N, Gd[D];
          corner_shape<D>(a, w0, w1, g.inv_h, N, Gd);
          const int b = b0 + (a & 1) + (TX + 1) * ((a >> 1) & 1) + (D == 3 ? (TX + 1) * (TY + 1) * ((a >> 2) & 1) : 0);
          float nv[D], na[D];
          if (D == 3) {
            const float4 r0 = nodes_s[2 * b], r1 = nodes_s[2 * b + 1];
            nv[0] = r0.x;
            nv[1] = r0.y;
            nv[D - 1] = r0.z;
            na[0] = r1.x;
            na[1] = r1.y;
            na[D - 1] = r1.z;
          } else {
            const float4 r0 = nodes_s[b];
            nv[0] = r0.x;
            nv[1] = r0.y;
            na[0] = r0.z;
            na[1] = r0.w;
          }
          if constexpr (D == 3) {
            // paired FP32 FMAs: each lane is the same single-rounding FMA as
            // the scalar form, two per instruction
            const float2 NN = make_float2(N, N);
            const float2 a01 = __ffma2_rn(NN, make_float2(na[0], na[1]), make_float2(dv[0], dv[1]));
            const float2 v01 = __ffma2_rn(NN, make_float2(nv[0], nv[1]), make_float2(vb[0], vb[1]));
            dv[0] = a01.x;
            dv[1] = a01.y;
            dv[2] = fmaf(N, na[2], dv[2]);
            vb[0] = v01.x;
            vb[1] = v01.y;
            vb[2] = fmaf(N, nv[2], vb[2]);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              const float2 l01 =
                  __ffma2_rn(make_float2(nv[k], nv[k]), make_float2(Gd[0], Gd[1]), make_float2(L[k][0], L[k][1]));
              L[k][0] = l01.x;
              L[k][1] = l01.y;
              L[k][2] = fmaf(nv[k], Gd[2], L[k][2]);
            }
          } else {
#pragma unroll
            for (int k = 0; k < D; ++k) {
              dv[k] += N * na[k];
              vb[k] += N * nv[k];
#pragma unroll
              for (int l = 0; l < D; ++l) L[k][l] += nv[k] * Gd[l];
            }
          }
        }
        float v0[D], sg[6], ep[6];
        cp_async_wait_all();
#pragma unroll
        for (int k = 0; k < D; ++k) v0[k] = stg[(F::S_VEL + k) * T + tid];
        const float mass = stg[F::S_MASS * T + tid];
        const int32_t pid = __float_as_int(stg[F::S_ID * T + tid]);
        const float coh = has_coh ? stg[F::S_COH * T + tid] : I.mat.c;
#pragma unroll
        for (int i = 0; i < 6; ++i) sg[i] = ep[i] = 0.f;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
          sg[i] = stg[(F::S_SIG + i) * T + tid];
          ep[i] = stg[(F::S_EPS + i) * T + tid];
        }
        const float jm1 = stg[F::S_JM1 * T + tid];
        float epsp = stg[F::S_EPSP * T + tid];

        int status = 0;
        // FLIP velocity, advection in cell units, relocation
        bool dead = false;
        float vk[D], un[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          vk[k] = v0[k] + g.dt * dv[k];
          I.B.vel(k)[q] = vk[k];
          if (!isfinite(vk[k])) status |= ST_NONFINITE;
          un[k] = u[k] + g.dt * vb[k] * g.inv_h;
          if (!isfinite(un[k])) {
            status |= ST_NONFINITE;
            dead = true;
            un[k] = 0.f;
          }
          // one cell crossing is an exact subtraction (Sterbenz), so the
          // offset stays in [-0.5, 0.5) and the cell is exact
          if (un[k] >= 0.5f) {
            un[k] -= 1.f;
            cell[k] += 1;
          } else if (un[k] < -0.5f) {
            un[k] += 1.f;
            cell[k] -= 1;
          }
          if (!(un[k] >= -0.5f && un[k] < 0.5f)) {  // more than one cell per step
            const float sh = floorf(un[k] + 0.5f);
            un[k] -= sh;
            cell[k] += (int)sh;
            if (un[k] >= 0.5f) {
              un[k] -= 1.f;
              cell[k] += 1;
            } else if (un[k] < -0.5f) {
              un[k] += 1.f;
              cell[k] -= 1;
            }
          }
          if (cell[k] < 0 || cell[k] >= g.nc[k]) dead = true;
          I.B.off(k)[q] = un[k];
        }
        uint32_t nkey = g.dead_key;
        int l2 = 0;
        if (!dead) {
          const int t2 = cell[0] / TX + g.nt[0] * (cell[1] / TY + g.nt[1] * (D == 3 ? cell[2] / TZ : 0));
          l2 = cell[0] % TX + TX * (cell[1] % TY + TY * (D == 3 ? cell[2] % TZ : 0));
          nkey = (uint32_t)t2 * CELLS_PER_TILE + (uint32_t)l2;
        } else {
          status |= ST_LEFT_MESH;
        }
        I.B.key()[q] = nkey;
        I.B.mass()[q] = mass;
        I.B.id()[q] = pid;
        if (has_coh) I.B.coh()[q] = coh;
        // tile movers for the next step's binning; one append per warp
        const int tn = min((int)(nkey >> LOCAL_BITS), I.ntiles);
        const bool mover = tn != t;
        const unsigned am = __activemask();
        const unsigned mv = __ballot_sync(am, mover);
        if (mover) {
          const int leader = __ffs(mv) - 1;
          int base = 0;
          if (lane == leader) base = atomicAdd(&I.s.ctr[C_MOVERS], __popc(mv));
          base = __shfl_sync(mv, base, leader);
          atomicAdd(&I.s.in_cnt[tn], 1);
          atomicAdd(&I.s.out_cnt[t], 1);
          I.s.movers[base + __popc(mv & lt_mask)] = (int32_t)q;
        }
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
        const float jn = jm1 + (tr + jm1 * tr);
        I.B.jm1()[q] = jn;
        // a trial in the apex band keeps its trial stress here and is queued
        // for the FP64 return (apex_band_k, which also drops this tile's sums)
        if (material_update_inline(I.mat, coh, sg, de, epsp)) I.s.bucket_sorted[atomicAdd(&I.s.ctr[C_APEX], 1)] = (int32_t)q;
#pragma unroll
        for (int i = 0; i < NS; ++i) {
          I.B.sig(i)[q] = sg[i];
          if (!isfinite(sg[i])) status |= ST_NONFINITE;
        }
        I.B.epsp()[q] = epsp;
        if (status) atomicOr(&I.s.ctr[C_STATUS], status);
        if (!mover) {  // stays in the tile: its record for the next step's P2G
          float f[4 * NQ];
          p2g_record<D, P2G_USL>(un, mass, vk, jn, sg, g.inv_rho, f);
          const int sl = rec_slot(tid);
#pragma unroll
          for (int k = 0; k < NQ; ++k)
            rec[k * T + sl] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
          lcn = (unsigned)l2;
          kd = l2 == (int)(key & (CELLS_PER_TILE - 1)) ? 1 : 2;
        }
      }
      // the particles that moved to another cell of the tile, per warp in order
      const unsigned mv2 = __ballot_sync(0xffffffffu, kd == 2);
      if (kd == 2) {
        mvw[warp][__popc(mv2 & lt_mask)] = (uint8_t)tid;
        ncell[tid] = (uint8_t)lcn;
      }
      kind[tid] = (uint8_t)kd;
      if (lane == 0) cntw[warp] = __popc(mv2);
      __syncthreads();
      {  // my (cell, corner pair): the cell's stayers in order, then the particles that moved in
        float acc[CPT][NCH];
#pragma unroll
        for (int r = 0; r < CPT; ++r)
#pragma unroll
          for (int ch = 0; ch < NCH; ++ch) acc[r][ch] = cellP[my_cell * NV + (my_cp + r * CPC) * NCH + ch];
        if (stamp[my_cell] == chunk_id) {
          const int i1 = ce[my_cell];
          for (int i = cs[my_cell]; i < i1; ++i)
            if (kind[i] == 1) accumulate_rec<D, P2G_USL>(rec, i, my_cp, g.inv_h, acc);
        }
#pragma unroll 1
        for (int w = 0; w < NW; ++w) {
          const int nw = cntw[w];
          for (int k = 0; k < nw; ++k) {
            const int i = mvw[w][k];
            if (ncell[i] == my_cell) accumulate_rec<D, P2G_USL>(rec, i, my_cp, g.inv_h, acc);
          }
        }
#pragma unroll
        for (int r = 0; r < CPT; ++r)
#pragma unroll
          for (int ch = 0; ch < NCH; ++ch) cellP[my_cell * NV + (my_cp + r * CPC) * NCH + ch] = acc[r][ch];
      }
      ++chunk_id;
      __syncthreads();  // the records are read; the next chunk writes over them
    }
    cells_to_slot<D, NCH>(cellP, I.s.slots1, t, T);
    if (tid == 0) {
      I.s.fepoch[t] = step + 1;
      s_work[(it + 1) & 1] = wnext;
    }
    __syncthreads();
  }
}

// FP64 apex-band returns of the particles G2P queued (rare: trials within
// 1e-3 (|p| + c cot phi) of the apex, cohesive materials only).  G2P stored
// their trial stress; this completes it in place and adds the plastic strain
// increment.  Every CTA walks every instance's queue with a grid stride.
constexpr int APEX_T = 128;
template <int D, bool ONE>
__global__ void __launch_bounds__(APEX_T) apex_band_k(const __grid_constant__ GroupArgs G) {
  constexpr int NS = nstress<D>();
  pdl_trigger();
  pdl_wait();
  for (int ii = 0; ii < G.ninst; ++ii) {
    const InstArgs &I = ONE ? G.one : G.inst[ii];
    const int cnt = I.s.ctr[C_APEX];
    for (int e = blockIdx.x * APEX_T + threadIdx.x; e < cnt; e += gridDim.x * APEX_T) {
      const int q = I.s.bucket_sorted[e];
      const float c = I.A.coh() ? I.A.coh()[I.perm_out[q]] : I.mat.c;
      float st[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, out[6];
#pragma unroll
      for (int i = 0; i < NS; ++i) st[i] = I.B.sig(i)[q];
      float epsp = I.B.epsp()[q];
      mc_return_apex_band(I.matd, c, st, out, epsp);
      int status = 0;
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        I.B.sig(i)[q] = out[i];
        if (!isfinite(out[i])) status |= ST_NONFINITE;
      }
      I.B.epsp()[q] = epsp;
      if (status) atomicOr(&I.s.ctr[C_STATUS], status);
      // the fused USL G2P summed this particle's trial stress into its tile's
      // sums for the next step: those sums are no longer valid
      const uint32_t k2 = I.B.key()[q];
      if (k2 < I.geo.dead_key) I.s.fepoch[k2 >> LOCAL_BITS] = -1;
    }
  }
}

template <int D, int MODE, bool RES = false>
cudaError_t launch_p2g(const GroupArgs &G, int work_slot, cudaStream_t st) {
  if constexpr (RES)
    return G.ninst == 1 ? launch_dep(p2g_resid<D, MODE, true, true>, G.grid, p2g_threads<D>(), p2g_smem<D, MODE>(),
                                     st, G, work_slot)
                        : launch_dep(p2g_resid<D, MODE, false, true>, G.grid, p2g_threads<D>(), p2g_smem<D, MODE>(),
                                     st, G, work_slot);
  else {
    // a mapped mesh needs K only for the force
    if constexpr (MODE != P2G_MOM)
      if (G.mapped)
        return G.ninst == 1 ? launch_dep(p2g_tile<D, MODE, true, true>, G.grid, p2g_threads<D>(),
                                         P2GRec<D, MODE, true>::SMEM, st, G, work_slot)
                            : launch_dep(p2g_tile<D, MODE, false, true>, G.grid, p2g_threads<D>(),
                                         P2GRec<D, MODE, true>::SMEM, st, G, work_slot);
    // as many CTAs as are resident (G.grid is 8 per SM): a CTA's first item
    // is its block index, and a CTA waiting for a free slot would hold its
    // item back until the end of the pass
    constexpr int nt = P2GTile<D, MODE, false>::NT;
    constexpr bool wide = p2g_wide<D, MODE, false>();
    const int grid1 = G.grid / 8 * (wide ? MPM_P2G_WIDE_MINB : p2g_min_blocks<D, MODE, true>());
    const int gridn = G.grid / 8 * (wide ? MPM_P2G_WIDE_MINB : p2g_min_blocks<D, MODE, false>());
    return G.ninst == 1
               ? launch_dep(p2g_tile<D, MODE, true>, grid1, nt, P2GTile<D, MODE, false>::SMEM, st, G, work_slot)
               : launch_dep(p2g_tile<D, MODE, false>, gridn, nt, P2GTile<D, MODE, false>::SMEM, st, G, work_slot);
  }
}

template <int D, int MODE, bool RES = false>
cudaError_t prepare_p2g() {
  cudaError_t e;
  if constexpr (RES) {
    e = cudaFuncSetAttribute(p2g_resid<D, MODE, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)p2g_smem<D, MODE>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(p2g_resid<D, MODE, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)p2g_smem<D, MODE>());
  }
  e = cudaFuncSetAttribute(p2g_tile<D, MODE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)P2GTile<D, MODE, false>::SMEM);
  if (e != cudaSuccess) return e;
  if constexpr (MODE != P2G_MOM) {
    e = cudaFuncSetAttribute(p2g_tile<D, MODE, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)P2GRec<D, MODE, true>::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(p2g_tile<D, MODE, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)P2GRec<D, MODE, true>::SMEM);
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(p2g_tile<D, MODE, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)P2GTile<D, MODE, false>::SMEM);
}

template <int D>
cudaError_t prepare_g2p_tile() {
  cudaError_t e = cudaFuncSetAttribute(g2p_tile<D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)G2PF<D>::SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(g2p_tile<D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G2PF<D>::SMEM);
}

// The fused USL G2P (and, for cohesive materials, the FP64 apex-band return).
template <int D>
cudaError_t launch_g2p_tile(const GroupArgs &G, cudaStream_t st) {
  cudaError_t e = G.ninst == 1 ? launch_dep(g2p_tile<D, true>, G.grid, G2PF<D>::T, G2PF<D>::SMEM, st, G)
                               : launch_dep(g2p_tile<D, false>, G.grid, G2PF<D>::T, G2PF<D>::SMEM, st, G);
  if (e != cudaSuccess || !G.apex) return e;
  return G.ninst == 1 ? launch_dep(apex_band_k<D, true>, G.grid / 8, APEX_T, 0, st, G)
                      : launch_dep(apex_band_k<D, false>, G.grid / 8, APEX_T, 0, st, G);
}

template <int D, int NMODE>
cudaError_t launch_node(const GroupArgs &G, int work_slot, cudaStream_t st) {
  if (G.mapped)
    return G.ninst == 1 ? launch_dep(node_tile<D, NMODE, true, true>, G.grid, NODE_T, 0, st, G, work_slot)
                        : launch_dep(node_tile<D, NMODE, false, true>, G.grid, NODE_T, 0, st, G, work_slot);
  return G.ninst == 1 ? launch_dep(node_tile<D, NMODE, true>, G.grid, NODE_T, 0, st, G, work_slot)
                      : launch_dep(node_tile<D, NMODE, false>, G.grid, NODE_T, 0, st, G, work_slot);
}

template <int D, int GMODE>
cudaError_t launch_g2p(const GroupArgs &G, cudaStream_t st) {
  const int nb = G.nblk_p * G2P_SUB;
  cudaError_t e = G.mapped ? (G.ninst == 1 ? launch_dep(g2p<D, GMODE, true, true>, nb, G2P_T, 0, st, G)
                                            : launch_dep(g2p<D, GMODE, false, true>, nb, G2P_T, 0, st, G))
                           : G.ninst == 1 ? launch_dep(g2p<D, GMODE, true>, nb, G2P_T, 0, st, G)
                                          : launch_dep(g2p<D, GMODE, false>, nb, G2P_T, 0, st, G);
  if (e != cudaSuccess || !G.apex || GMODE == G2P_USF_ADVECT) return e;
  return G.ninst == 1 ? launch_dep(apex_band_k<D, true>, G.grid / 8, APEX_T, 0, st, G)
                      : launch_dep(apex_band_k<D, false>, G.grid / 8, APEX_T, 0, st, G);
}

template <int D>
cudaError_t step_dim(int scheme, const GroupArgs &G, cudaEvent_t *ev, cudaStream_t st) {
  cudaError_t e;
  // phase events 0 (start) and 1 (after binning) are recorded by the
  // caller; 2.. follow each kernel here
  if (scheme == 1) {
#if MPM_FUSED_USL
    // residual P2G, nodes, G2P fused with the next step's P2G
    if ((e = launch_p2g<D, P2G_USL, true>(G, W_P2G, st)) != cudaSuccess) return e;
    if ((e = phase_mark(ev, 2, st)) != cudaSuccess) return e;
    if ((e = launch_node<D, NODE_USL>(G, W_NODE, st)) != cudaSuccess) return e;
    if ((e = phase_mark(ev, 3, st)) != cudaSuccess) return e;
    if ((e = launch_g2p_tile<D>(G, st)) != cudaSuccess) return e;
#else
    // P2G, nodes, per-particle G2P
    if ((e = launch_p2g<D, P2G_USL>(G, W_P2G, st)) != cudaSuccess) return e;
    if ((e = phase_mark(ev, 2, st)) != cudaSuccess) return e;
    if ((e = launch_node<D, NODE_USL>(G, W_NODE, st)) != cudaSuccess) return e;
    if ((e = phase_mark(ev, 3, st)) != cudaSuccess) return e;
    if ((e = launch_g2p<D, G2P_USL>(G, st)) != cudaSuccess) return e;
#endif
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
constexpr int CONS_VALS = 8;  // mass, momentum (3), kinetic and strain energy, live count, volume

template <int D>
__global__ void cons_partial(int64_t n, PBuf P, uint32_t dead_key, float inv_rho, double *part) {
  constexpr int NS = nstress<D>();
  double acc[CONS_VALS] = {0, 0, 0, 0, 0, 0, 0, 0};
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
    acc[7] += vol;
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
    if (pos && g.X && !dead) {  // mapped: x(xi) of the cell, xi = 2 off
      double xi[D], xa[1 << D][D], x[D], J[D][D];
#pragma unroll
      for (int k = 0; k < D; ++k) xi[k] = 2.0 * (double)P.off(k)[q];
      const iso::IsoGrid M{g.X, {g.nc[0], g.nc[1], g.nc[2]}};
      iso::cell_xyz<D>(M, c, xa);
      iso::cell_map<D>(xa, xi, x, J);
#pragma unroll
      for (int k = 0; k < D; ++k) pos[id * D + k] = x[k];
    } else if (pos) {
#pragma unroll
      for (int k = 0; k < D; ++k)
        pos[id * D + k] = dead ? __longlong_as_double(0x7ff8000000000000ll)
                               : org[k] + ((double)c[k] + 0.5 + (double)P.off(k)[q]) * h;
    }
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
#if MPM_FUSED_USL
    if ((e = prepare_p2g<3, P2G_USL, true>()) != cudaSuccess) return e;
    if ((e = prepare_g2p_tile<3>()) != cudaSuccess) return e;
#endif
    if ((e = prepare_p2g<3, P2G_USL>()) != cudaSuccess) return e;
    if ((e = prepare_p2g<3, P2G_MOM>()) != cudaSuccess) return e;
    return prepare_p2g<3, P2G_FORCE>();
  }
#if MPM_FUSED_USL
  if ((e = prepare_p2g<2, P2G_USL, true>()) != cudaSuccess) return e;
  if ((e = prepare_g2p_tile<2>()) != cudaSuccess) return e;
#endif
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
