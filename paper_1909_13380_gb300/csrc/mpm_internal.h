// mpm_internal.h -- launch interfaces shared by the C-ABI (mpm_api.cu) and the
// kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mpm_device.cuh"

namespace mpm {

// Tiles of the FP32 path: 64 cells each, 4 x 4 x 4 hexahedra or 8 x 8 quads.
// Binning key = tile * 64 + local cell, tile = tx + NTX (ty + NTY tz),
// local = lx + TX (ly + TY lz); particles that left the mesh carry the key
// NT * 64 (a virtual tile after all real ones).
template <int D> struct Tile;
template <> struct Tile<3> {
  static constexpr int TX = 4, TY = 4, TZ = 4;
};
template <> struct Tile<2> {
  static constexpr int TX = 8, TY = 8, TZ = 1;
};
constexpr int CELLS_PER_TILE = 64;
constexpr int LOCAL_BITS = 6;
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
// Node kernels: USL (v', a), USF velocity stage (v), USF force stage (v', a).
enum { NODE_USL = 0, NODE_USF_V = 1, NODE_USF_A = 2 };
// G2P kernels: USL (full update), USF stress stage, USF advection stage.
enum { G2P_USL = 0, G2P_USF_STRESS = 1, G2P_USF_ADVECT = 2 };

// FP32 particle storage, SoA; every field has n entries.  Offsets are in cell
// units, centred: the particle sits at origin + (cell + 0.5 + off) h with
// off in [-0.5, 0.5).  Volume is held as jm1 = V / V0 - 1 with V0 = m / rho,
// so that the tiny per-step volume changes keep FP32's relative precision.
// Stresses/strains: 6 comps in 3D, (xx, yy, zz, xy) in 2D.
// All fields live in one allocation, field f at base + f * stride (stride a
// multiple of 256 bytes), so a buffer is described by two values:
//   0 key, 1 id, 2-4 offset, 5-7 velocity, 8-13 stress, 14-19 strain,
//   20 mass, 21 J-1, 22 plastic strain, 23 cohesion (when present).
// 2D leaves the z offset/velocity and the last two stress/strain slots unused.
constexpr int PBUF_FIELDS = 24;
struct PBuf {
  char *base;
  int64_t stride;
  int has_coh;
  __host__ __device__ __forceinline__ uint32_t *key() const { return (uint32_t *)base; }
  __host__ __device__ __forceinline__ int32_t *id() const { return (int32_t *)(base + stride); }
  __host__ __device__ __forceinline__ float *fld(int f) const { return (float *)(base + f * stride); }
  __host__ __device__ __forceinline__ float *off(int k) const { return fld(2 + k); }
  __host__ __device__ __forceinline__ float *vel(int k) const { return fld(5 + k); }
  __host__ __device__ __forceinline__ float *sig(int i) const { return fld(8 + i); }
  __host__ __device__ __forceinline__ float *eps(int i) const { return fld(14 + i); }
  __host__ __device__ __forceinline__ float *mass() const { return fld(20); }
  __host__ __device__ __forceinline__ float *jm1() const { return fld(21); }
  __host__ __device__ __forceinline__ float *epsp() const { return fld(22); }
  __host__ __device__ __forceinline__ float *coh() const { return has_coh ? fld(23) : nullptr; }
};

// Division of 0 <= n < 2^26 by an invariant d >= 1 as a multiply and a
// shift (Granlund & Montgomery, "Division by invariant integers using
// multiplication", 1994): with l = ceil(log2 d), s = 32 + l and
// m = floor(2^s / d) + 1, floor(n m / 2^s) = floor(n / d) for every n < 2^32;
// n < 2^26 keeps n m below 2^64.
struct FastDiv {
  unsigned long long m;
  int s;
  __host__ __device__ __forceinline__ int div(int n) const {
    return (int)(((unsigned long long)(unsigned)n * m) >> s);
  }
};
inline FastDiv make_fastdiv(int d) {
  int l = 0;
  while ((1LL << l) < (long long)d) ++l;
  FastDiv f;
  f.s = 32 + l;
  f.m = (unsigned long long)(((unsigned __int128)1 << f.s) / (unsigned)d) + 1;
  return f;
}

struct Geo {
  int nc[3];   // cells per axis (nc[2] = 1 in 2D)
  int nt[3];   // tiles per axis
  FastDiv div_nt0, div_nt01;  // division by nt[0] and by nt[0] nt[1]
  int ntiles;
  uint32_t dead_key;
  float h, inv_h, dt, mass_tol, inv_rho;
  float g[3];
  int bc[6];
  float mu[6];
  int loads;           // face tractions or damping present (mpm_set_loads)
  float damp;          // alpha of a = f / m - alpha v
  float trac[6][3];    // traction per face
  // Mapped (isoparametric) mesh, else both null (ISOPARAMETRIC MESH).  cgeo:
  // per cell (id cx + nc0 (cy + nc1 cz)) the positions of its 2^D corners
  // relative to the cell's centre, in units of h, corner a's component k at
  // float D a + k of the cell's CGEO_F4<D> float4s.  The offset of a particle
  // is then half its natural coordinates, u = xi / 2.  X: the FP64 node
  // coordinates (3 per node) for the initial location and the export.
  const float4 *cgeo;
  const double *X;
  // mapped mesh: outward unit normal of face f at its node (i1, i2) -- the
  // node's indices along the face's two other axes, in increasing axis order
  // (2D: the one other axis) -- at fnorm[fnoff[f] + i1 + (n_i1 + 1) i2]
  const float4 *fnorm;
  int fnoff[6];
  // mapped 2D mesh under face stresses: the force on each face node, laid out
  // as fnorm (null: none)
  const float4 *fload;
};
template <int D> constexpr int CGEO_F4() { return D == 3 ? 6 : 2; }

// Counters of a step (int32, in StepBufs::ctr).
enum {
  C_ACTIVE = 0,     // active (non-empty) tiles this step
  C_MOVERS = 1,     // particles that changed tile (appended by G2P, or bin_movers)
  C_MOVERS_SNAP = 2,
  C_WORK_BIN = 3,   // dynamic tile counters of the per-tile kernels
  C_WORK_P2G = 4,
  C_WORK_NODE = 5,
  C_WORK_P2G2 = 6,
  C_WORK_NODE2 = 7,
  C_STATUS = 8,     // sticky device status bits (ST_*)
  C_BIN_ITEMS = 9,  // active tiles + 1 if the dead range is non-empty
  C_DEAD_START = 10,
  C_APEX = 11,      // particles queued by G2P for the FP64 apex-band return (in StepBufs::bucket_sorted)
  C_STEP = 12,      // step index, advanced by the tile scan (the epoch of the nodal partial sums)
  C_RESID = 13,     // binning items that need the residual P2G this step (USL)
  C_NCTR = 16
};

// Device storage of the FP32 path's binning and step.
struct StepBufs {
  uint32_t *keys_sorted;   // n: keys in binning order (old keys for the next binning)
  int32_t *perm;           // n: storage slot of the q-th particle in binning order
  int32_t *tile_start[2];  // ntiles + 2 each: old / new tile ranges (parity = step parity)
  int32_t *in_cnt;         // ntiles + 1: particles entering each tile
  int32_t *out_cnt;        // ntiles + 1: particles leaving each tile
  int32_t *bucket_start;   // ntiles + 2
  int32_t *bucket_fill;    // ntiles + 1
  int32_t *movers;         // n: storage slots of tile movers
  int32_t *bucket;         // n: movers grouped by destination tile
  int32_t *bucket_sorted;  // n: scratch for large buckets (binning), then the apex-band queue (G2P)
  int4 *active;            // ntiles + 2: active tiles in ascending order, (tile, new start, new end,
                           // old start - new start when the binning moved the tile's range as a whole,
                           // else INT_MIN), then the dead range (tile = ntiles) when it is not empty:
                           // the binning items
  int4 *bin_rec;           // ntiles + 2: per binning item (old start, old end, bucket start, bucket end)
  int32_t *scan_tot;       // 8 per chunk of the tile scan (look-back flag, totals, prefix)
  int32_t *ctr;            // C_NCTR counters
  float *slots1;           // ntiles * box * channels (P2G USL / MOM)
  float *slots2;           // ntiles * box * D        (P2G FORCE, USF)
  // USL: slots1 of a tile holds the next step's P2G of the particles that
  // stay in it, summed by the G2P that moved them (fepoch = the step those
  // sums are for), or the P2G of all its particles; slots_a the P2G of the
  // particles that arrived from other tiles (aepoch).  A tile's sums count
  // in a step only while their epoch equals that step's index (C_STEP).
  float *slots_a;          // ntiles * box * (1 + 2D)  (USL arrivals)
  int32_t *fepoch;         // ntiles
  int32_t *aepoch;         // ntiles
  int32_t *resid;          // ntiles + 2: binning items (active tiles) whose P2G is not complete
  // dense node values, one 16-byte record per node in 2D (v'x v'y ax ay) and
  // two in 3D (v'x v'y v'z -, ax ay az -); v' is v in the USF velocity stage
  float4 *node;
};

// --- radix sort (mpm_sort.cu) ---------------------------------------------
size_t sort_scratch_bytes(int64_t n);
// Stable LSD sort: keys_in (unchanged) -> keys_out sorted, perm_out
// (index of the q-th smallest).  vals_in == nullptr means identity.
cudaError_t sort_pairs(const uint32_t *keys_in, const int32_t *vals_in, uint32_t *keys_out,
                       int32_t *perm_out, int64_t n, int key_bits, void *scratch, cudaStream_t st);
// tile_start[u] = first position with key >= u * 64 (u = 0..ntiles), [ntiles+1] = n.
cudaError_t tile_bounds(const uint32_t *keys_sorted, int64_t n, int ntiles, int32_t *tile_start,
                        cudaStream_t st);

// --- one FP32 step over a group of instances ---------------------------------
// Every FP32 kernel works on a table of instances (a single mesh is a group of
// one).  Instances share no data, so each instance's result does not depend
// on what else is in the group.
struct InstArgs {
  int64_t n;        // particles
  int ntiles;
  Geo geo;
  MatConst<float> mat;
  MatConst<double> matd;
  PBuf A, B;        // A: state at the start of the step (storage order), B: out (binning order)
  StepBufs s;
  const int32_t *old_start;  // previous tile ranges
  int32_t *new_start;        // this step's tile ranges (written by the binning)
  uint32_t *keys_out;        // binning order keys (s.keys_sorted, or scratch)
  int32_t *perm_out;         // binning permutation (s.perm, or scratch)
  int ns0, ns1;              // node strides (nx+1), (nx+1)(ny+1)
  // failure detection test hook of the look-back tile scan: the chunk whose
  // flag is withheld (-1: none) and the polls a wait makes before it gives up
  int lb_withhold, lb_spin;
};

// Copy the table entry of instance ii into the block's shared copy (every
// thread of the block takes part; the caller synchronises before reading it).
// Kernels read instance constants from the shared copy: global stores cannot
// alias shared memory, so the compiler need not reload pointers and strides
// after every store, as it must for an entry read through a global pointer.
__device__ __forceinline__ void copy_inst(const InstArgs *tab, int ii, InstArgs *dst) {
  static_assert(sizeof(InstArgs) % 8 == 0, "InstArgs is copied as 8-byte words");
  const unsigned long long *src = reinterpret_cast<const unsigned long long *>(tab + ii);
  unsigned long long *d = reinterpret_cast<unsigned long long *>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(InstArgs) / 8); i += blockDim.x) d[i] = __ldg(src + i);
}

// USL step form.  0 (default): P2G of the stored state, the nodal solve, a
// G2P thread per particle.  1: G2P fused with the next step's P2G (one CTA
// per tile sums the P2G of the particles that stay in the tile while it
// moves them; a residual P2G adds arrivals) -- correct, but slower on every
// workload measured, so not the default.
#ifndef MPM_FUSED_USL
#define MPM_FUSED_USL 0
#endif

// Polls a wait of the look-back tile scan makes before it gives up (and sets
// ST_TIMEOUT); every wait is on a block that is already running, so it ends
// long before this.
constexpr int LB_SPIN_LIMIT = 1 << 20;

// Largest tile count (plus the dead range) scanned by one CTA per instance
// (1024 threads, at most MPM_SCAN1_K tiles each); larger instances take the
// look-back scan over many CTAs.
#ifndef MPM_SCAN1_K
#define MPM_SCAN1_K 4
#endif
constexpr int SCAN1_MAX = 1024 * MPM_SCAN1_K;

// Per-group launch description.  The prefix arrays map a block (or a work
// item) to its instance: entry i is the first block (item) of instance i and
// entry ninst the total.
enum { W_BIN = 0, W_P2G = 1, W_NODE = 2, W_P2G2 = 3, W_NODE2 = 4, W_SCAN_DONE = 5, W_SCAN_TICKET = 6, W_G2P = 7,
       W_COUNT = 8 };
struct GroupArgs {
  const InstArgs *inst;     // device table
  int ninst;
  const int32_t *pblk;      // blocks of the per-particle kernels (host-computed)
  const int32_t *sblk;      // blocks of the tile scan (host-computed)
  const int32_t *mblk;      // blocks of the mover bucketing (host-computed)
  int32_t *bin_items;       // device-computed prefix of binning tiles
  int32_t *act_items;       // device-computed prefix of active tiles
  int32_t *res_items;       // device-computed prefix of residual P2G items (USL)
  int32_t *work;            // W_COUNT dynamic work counters
  int nblk_p, nblk_s, nblk_m;
  int scan_one;             // every instance has at most SCAN1_MAX tiles: one-CTA scans
  int grid;                 // CTAs of the per-tile kernels
  int apex;                 // some instance can reach the FP64 apex band (cohesion > 0): run apex_band_k
  int bin_t;                // bin_tiles threads per CTA: 128 for groups of >= 4M particles, else 256
  int mapped;               // the instances have mapped cells (Geo::cgeo; a group of one)
  InstArgs one;             // a group of one: its table entry (inst[0]) by value
};

// The instance a kernel of the step reads.  For a group of one it is the copy
// inside the kernel's parameters (passed __grid_constant__): its constants are
// constant-bank operands of the arithmetic and cost no load instruction.
// Otherwise it is the block's (or warp's) shared-memory copy of its table
// entry, which costs a shared load wherever a constant is not kept in a
// register.
template <bool ONE>
__device__ __forceinline__ const InstArgs &inst_ref(const GroupArgs &G, const InstArgs &shared_copy) {
  if constexpr (ONE)
    return G.one;
  else
    return shared_copy;
}

// Programmatic dependent launch.  The kernels of a step are launched with
// launch_dep(), which lets a kernel's CTAs be scheduled while the kernel
// before it in the stream is still running, hiding the launch and the CTA
// ramp between dependent kernels.  A CTA so launched runs only code that
// reads what the host wrote before the step (the group's instance table and
// block prefixes), then pdl_wait(): it returns once the preceding kernel has
// completed and its writes are visible (that kernel passed its own pdl_wait,
// so every earlier kernel has completed too).  Every CTA calls pdl_wait()
// before it touches any other memory or exits, otherwise the grid could
// complete ahead of its predecessor.  pdl_trigger() releases the next kernel
// once every CTA of this grid has called it or exited; a kernel is released
// only when all of its predecessor's CTAs are running, so the waits always
// end.  Without a preceding kernel (a graph's first node, a copy, an event
// node) both are no-ops and the launch is an ordinary stream-ordered one.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Record a phase boundary (works inside stream capture as an external node).
inline cudaError_t phase_mark(cudaEvent_t *ev, int i, cudaStream_t st) {
  return ev ? cudaEventRecordWithFlags(ev[i], st, cudaEventRecordExternal) : cudaSuccess;
}

// --- incremental binning (mpm_bin.cu) ----------------------------------------
// The binning of a step starts from the tile movers (particles whose key left
// their tile), counted per tile and listed by the previous step's G2P; it
// consumes (zeroes) those counts.  count_movers recounts them from the keys
// (A's keys against the previous binning's keys), for callers that have just
// zeroed the counters (a binning into scratch buffers).
cudaError_t bin_group(int dim, const GroupArgs &G, cudaStream_t st);
cudaError_t count_movers(const GroupArgs &G, cudaStream_t st);
// Gather every field of A into B in the order perm (B[q] = A[perm[q]]).
cudaError_t permute_state(int dim, int64_t n, const PBuf &A, const PBuf &B, const int32_t *perm,
                          cudaStream_t st);

// --- FP32 step kernels (mpm_fp32.cu) -----------------------------------------
cudaError_t f32_prepare(int dim);  // once per process and dim
// Everything after the binning; phase events 2.. after each kernel if ev.
cudaError_t f32_group_step(int dim, int scheme, const GroupArgs &G, cudaEvent_t *ev, cudaStream_t st);
// out[i] = latched status bits of instance i of the table.
cudaError_t gather_status(const InstArgs *tab, int ninst, int32_t *out, cudaStream_t st);
cudaError_t f32_conservation(int dim, int64_t n, const PBuf &P, uint32_t dead_key, float inv_rho,
                             double *d_out, double *d_partials, cudaStream_t st);
// Positions: origin + (cell + 0.5 + off) h, or on a mapped mesh (g.X) the
// map of the cell at natural coordinates 2 off, in FP64.
cudaError_t f32_export(int dim, int64_t n, const PBuf &P, const Geo &g, const double origin[3], double h,
                       double rho, double *pos, double *vel, double *sig, double *eps, double *vol,
                       double *epsp, int64_t *cell, cudaStream_t st);

// --- FP64 plain kernels (mpm_fp64.cu) ----------------------------------------
struct D64State {
  double *x[3], *v[3], *sig[6], *eps[6];
  double *mass, *vol, *epsp, *coh;
  int32_t *alive;
  // mapped mesh only (ISOPARAMETRIC MESH), else null: each particle's cell
  // (linear id ix + nx (iy + ny iz)) and its natural coordinates there
  int32_t *cell;
  double *xi[3];
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
  int loads;
  double damp, trac[6][3];
  D64State P;
  D64Nodes N;
  int64_t nnodes;
  int32_t *status;
  const double *X;  // mapped mesh: node coordinates, 3 per node (x fastest); null: Cartesian
  const double *fnorm;  // mapped mesh: face normals (3 per face node, laid out as Geo::fnorm)
  const double *fload;  // mapped 2D mesh: face-stress force per face node (same layout), or null
  int64_t fnoff[6];
};
cudaError_t d64_step(const D64Launch &L, cudaStream_t st);
// Locate particles n0 .. n0 + n - 1 of a mapped mesh (L.X set) by the
// neighbourhood walk from their Cartesian guess cell; fills P.cell and P.xi
// and counts the ones found in no cell in *bad.
cudaError_t d64_locate(const D64Launch &L, int64_t n0, int64_t n, int32_t *bad, cudaStream_t st);
cudaError_t d64_conservation(const D64Launch &L, double *d_out, double *d_partials, cudaStream_t st);

// --- material update primitive (mpm_fp64.cu / mpm_fp32.cu) -------------------
cudaError_t material_update_f32(const MatConst<float> &m, const MatConst<double> &md, int64_t n,
                                const float *sig, const float *de, const float *coh, float *out,
                                float *depsp, cudaStream_t st);
cudaError_t material_update_f64(const MatConst<double> &m, int64_t n, const double *sig,
                                const double *de, const double *coh, double *out, double *depsp,
                                cudaStream_t st);

}  // namespace mpm
