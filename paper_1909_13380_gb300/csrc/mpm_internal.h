// mpm_internal.h -- launch interfaces shared by the C-ABI (mpm_api.cu) and the
// kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mpm_device.cuh"

namespace mpm {

// Tiles of the FP32 path: 256 cells each, 8 x 8 x 4 hexahedra or 16 x 16 quads.
template <int D> struct Tile;
template <> struct Tile<3> {
  static constexpr int TX = 8, TY = 8, TZ = 4;
};
template <> struct Tile<2> {
  static constexpr int TX = 16, TY = 16, TZ = 1;
};
constexpr int CELLS_PER_TILE = 256;
template <int D> constexpr int box_x() { return Tile<D>::TX + 1; }
template <int D> constexpr int box_y() { return Tile<D>::TY + 1; }
template <int D> constexpr int box_z() { return D == 3 ? Tile<D>::TZ + 1 : 1; }
template <int D> constexpr int box_nodes() { return box_x<D>() * box_y<D>() * box_z<D>(); }
template <int D> constexpr int nstress() { return D == 3 ? 6 : 4; }

// P2G channel sets: USL (m, P, f_int), MOM (m, P), FORCE (f_int).
enum { P2G_USL = 0, P2G_MOM = 1, P2G_FORCE = 2 };
template <int D, int MODE> constexpr int p2g_channels() {
  return MODE == P2G_USL ? 1 + 2 * D : MODE == P2G_MOM ? 1 + D : D;
}
// G2P kernels: USL (full update), USF stress stage, USF advection stage.
enum { G2P_USL = 0, G2P_USF_STRESS = 1, G2P_USF_ADVECT = 2 };

// FP32 particle storage, SoA; every field has n entries.  Offsets are in cell
// units, centred: the particle sits at origin + (cell + 0.5 + off) h with
// off in [-0.5, 0.5).  Stresses/strains: 6 comps in 3D, (xx,yy,zz,xy) in 2D.
struct PBuf {
  uint32_t *key;
  int32_t *id;
  float *off[3];
  float *vel[3];
  float *sig[6];
  float *eps[6];
  float *mass, *vol, *epsp, *coh;  // coh may be nullptr
};

struct Geo {
  int nc[3];   // cells per axis (nc[2] = 1 in 2D)
  int nt[3];   // tiles per axis
  int ntiles;
  uint32_t dead_key;
  float h, inv_h, dt, mass_tol;
  float g[3];
  int bc[6];
  float mu[6];
};

// Device scratch of one binning + step of the FP32 path.
struct StepBufs {
  uint32_t *keys_sorted;  // n
  int32_t *perm;          // n
  int32_t *tile_start;    // ntiles + 2
  int32_t *active;        // ntiles
  int32_t *ctr;           // [0] active tiles, [1..7] work counters, [8] status
  float *slots1;          // ntiles * box * channels (P2G USL / MOM)
  float *slots2;          // ntiles * box * D        (P2G FORCE, USF)
};

// --- radix sort (mpm_sort.cu) ---------------------------------------------
// Scratch bytes for sorting n keys of key_bits bits.
size_t sort_scratch_bytes(int64_t n);
// Stable LSD sort: keys_in (unchanged) -> keys_out sorted, perm_out
// (index of the q-th smallest).  vals_in == nullptr means identity.
cudaError_t sort_pairs(const uint32_t *keys_in, const int32_t *vals_in, uint32_t *keys_out,
                       int32_t *perm_out, int64_t n, int key_bits, void *scratch, cudaStream_t st);
// tile_start / active tile list from sorted keys.
cudaError_t tile_bounds(const uint32_t *keys_sorted, int64_t n, int ntiles, int32_t *tile_start,
                        int32_t *active, int32_t *ctr, cudaStream_t st);

// --- FP32 tile kernels (mpm_fp32.cu) ----------------------------------------
struct F32Launch {
  int dim, scheme;
  int64_t n;
  Geo geo;
  MatConst<float> mat;
  MatConst<double> matd;
  PBuf A, B;  // A: state at the start of the step (storage order), B: out (sorted order)
  StepBufs s;
  int grid;   // persistent grid size for the tile kernels
  cudaEvent_t *ev;  // optional phase events (recorded after each tile kernel), or nullptr
};
// Record a phase boundary (works inside stream capture as an external node).
inline cudaError_t phase_mark(cudaEvent_t *ev, int i, cudaStream_t st) {
  return ev ? cudaEventRecordWithFlags(ev[i], st, cudaEventRecordExternal) : cudaSuccess;
}
cudaError_t f32_prepare(int dim);                           // once per process and dim
cudaError_t f32_step(const F32Launch &L, cudaStream_t st);  // everything after binning
cudaError_t f32_conservation(int dim, int64_t n, const PBuf &P, uint32_t dead_key, double *d_out,
                             double *d_partials, cudaStream_t st);
cudaError_t f32_export(int dim, int64_t n, const PBuf &P, const Geo &g, const double origin[3], double h,
                       double *pos, double *vel, double *sig, double *eps, double *vol, double *epsp,
                       int64_t *cell, cudaStream_t st);
cudaError_t f32_keys(int dim, int64_t n, const PBuf &P, uint32_t *keys_out, cudaStream_t st);

// --- FP64 plain kernels (mpm_fp64.cu) ----------------------------------------
struct D64State {
  double *x[3], *v[3], *sig[6], *eps[6];
  double *mass, *vol, *epsp, *coh;
  int32_t *alive;
};
struct D64Nodes {
  double *m, *P[3], *f[3], *v[3], *a[3], *vn[3];
};
struct D64Launch {
  int dim, scheme;
  int64_t n;
  int nc[3];
  double origin[3], h, dt, mass_tol, g[3];
  int bc[6];
  double mu[6];
  MatConst<double> mat;
  D64State P;
  D64Nodes N;
  int64_t nnodes;
  int32_t *status;
};
cudaError_t d64_step(const D64Launch &L, cudaStream_t st);
cudaError_t d64_conservation(const D64Launch &L, double *d_out, double *d_partials, cudaStream_t st);

// --- material update primitive (mpm_fp64.cu / mpm_fp32.cu) -------------------
cudaError_t material_update_f32(const MatConst<float> &m, const MatConst<double> &md, int64_t n,
                                const float *sig, const float *de, const float *coh, float *out,
                                float *depsp, cudaStream_t st);
cudaError_t material_update_f64(const MatConst<double> &m, int64_t n, const double *sig,
                                const double *de, const double *coh, double *out, double *depsp,
                                cudaStream_t st);

}  // namespace mpm
