// mpm_api.cu -- the C ABI declared in include/mpm.h.
//
// Host side of the library: validates descriptors, owns device storage,
// computes each particle's initial cell on the host in FP64 (cell =
// floor((x - origin)/h) per axis; the offset from the cell centre, in cell
// units, is rounded to FP32 for the mixed path), bins the particles once with
// a full stable radix sort when they are added, and enqueues steps.  The FP32
// kernels run over a table of instances: a mesh stepped alone is a group of
// one, a batch groups its meshes by dimension and scheme.  A step (or batched
// step) is replayed from a captured CUDA graph when the stream allows capture.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <algorithm>
#include <vector>

#include "../../include/mpm.h"
#include "mpm_internal.h"
#include "mpm_iso.cuh"

using namespace mpm;

namespace {

// Device tables of one group of instances (two step parities).
struct GroupDev {
  int ninst = 0, cap = 0;
  InstArgs *tab[2] = {nullptr, nullptr};
  int32_t *pfx = nullptr;     // pblk | sblk | mblk | bin_items | act_items (cap + 1 each) | work
  int32_t *status = nullptr;  // cap
  GroupArgs ga[2];
};

void free_group(GroupDev &g) {
  for (int p = 0; p < 2; ++p)
    if (g.tab[p]) cudaFree(g.tab[p]);
  if (g.pfx) cudaFree(g.pfx);
  if (g.status) cudaFree(g.status);
  g = GroupDev();
}

// FP64 inputs of add_particles, uploaded as given (row-major, as the ABI
// takes them); stress0 and cohesion may be null.
struct NewParticles {
  const double *pos, *vel, *vol, *stress0, *coh;
};

// The FP32 storage of new particles p (slot n0 + p) from their FP64 inputs:
// cell = floor((x - origin) / h) and offset s - cell - 0.5 in FP64 (the same
// IEEE operations as the oracle's locate), the offset rounded to FP32 and
// kept inside [-0.5, 0.5); key, id, FP32 velocity, stress (zero without
// stress0), mass = rho V, cohesion; strain, J-1 and eps_p zero.  On a
// mapped mesh (g.X) the cell is found by the FP64 neighbourhood walk from
// the Cartesian cell of origin and h (clamped to the grid) and the offset is
// half the natural coordinates there.  Points outside the mesh (or not
// finite) are counted in *bad and leave their slot unwritten.
template <int D>
__global__ void init_particles_k(int64_t n, int64_t n0, PBuf P, Geo g, double o0, double o1, double o2, double h,
                                 double rho, NewParticles in, int32_t *bad) {
  constexpr int NS = nstress<D>();
  constexpr int T[3] = {Tile<D>::TX, Tile<D>::TY, Tile<D>::TZ};
  const double org[3] = {o0, o1, o2};
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    int c[3] = {0, 0, 0};
    float u[3] = {0.f, 0.f, 0.f};
    bool ok = true;
    if (g.X) {
      double x[D], xi[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        x[k] = in.pos[p * D + k];
        ok = ok && isfinite(x[k]);
        const double f = ok ? floor((x[k] - org[k]) / h) : 0.0;
        c[k] = f < 0.0 ? 0 : (f >= (double)g.nc[k] ? g.nc[k] - 1 : (int)f);
      }
      ok = ok && iso::walk<D>(iso::IsoGrid{g.X, {g.nc[0], g.nc[1], g.nc[2]}}, x, c, xi);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        float uk = ok ? (float)(0.5 * xi[k]) : 0.f;
        if (uk >= 0.5f) uk = __int_as_float(0x3effffff);  // the float below 0.5
        if (uk < -0.5f) uk = -0.5f;
        u[k] = uk;
      }
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double sk = (in.pos[p * D + k] - org[k]) / h;
        const double f = floor(sk);
        ok = ok && sk >= 0.0 && f < (double)g.nc[k];
        c[k] = ok ? (int)f : 0;
        float uk = (float)(sk - f - 0.5);
        if (uk >= 0.5f) uk = __int_as_float(0x3effffff);  // the float below 0.5
        if (uk < -0.5f) uk = -0.5f;
        u[k] = uk;
      }
    }
    if (!ok) {
      atomicAdd(bad, 1);
      continue;
    }
    const int64_t q = n0 + p;
    const int t = c[0] / T[0] + g.nt[0] * (c[1] / T[1] + g.nt[1] * (c[2] / T[2]));
    const int l = c[0] % T[0] + T[0] * (c[1] % T[1] + T[1] * (c[2] % T[2]));
    P.key()[q] = (uint32_t)t * CELLS_PER_TILE + (uint32_t)l;
    P.id()[q] = (int32_t)q;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      P.off(k)[q] = u[k];
      P.vel(k)[q] = (float)in.vel[p * D + k];
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      P.sig(i)[q] = in.stress0 ? (float)in.stress0[p * 6 + i] : 0.f;
      P.eps(i)[q] = 0.f;
    }
    P.mass()[q] = (float)(rho * in.vol[p]);
    P.jm1()[q] = 0.f;
    P.epsp()[q] = 0.f;
    if (in.coh) P.coh()[q] = (float)in.coh[p];
  }
}

// The FP64 storage of new particles p (slot n0 + p): the inputs as given,
// mass = rho V, strain and eps_p zero, alive.
template <int D>
__global__ void init_particles64_k(int64_t n, int64_t n0, D64State P, double rho, NewParticles in) {
  constexpr int NS = nstress<D>();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = n0 + p;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      P.x[k][q] = in.pos[p * D + k];
      P.v[k][q] = in.vel[p * D + k];
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      P.sig[i][q] = in.stress0 ? in.stress0[p * 6 + i] : 0.0;
      P.eps[i][q] = 0.0;
    }
    P.mass[q] = rho * in.vol[p];
    P.vol[q] = in.vol[p];
    P.epsp[q] = 0.0;
    if (in.coh) P.coh[q] = in.coh[p];
    P.alive[q] = 1;
  }
}

// Copy the FP64 inputs of add_particles to one device scratch allocation
// (freed by the caller with cudaFreeAsync), with a zeroed int32 counter after
// them.  Stream-ordered; the host arrays are read before the call returns.
cudaError_t upload_inputs(cudaStream_t st, int64_t n, int D, const double *pos, const double *vel, const double *vol,
                          const double *stress0, const double *cohesion, double *&scratch, NewParticles &np,
                          int32_t *&counter) {
  const size_t w = (size_t)D * 2 + 1 + (stress0 ? 6 : 0) + (cohesion ? 1 : 0);  // doubles per particle
  scratch = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&scratch, sizeof(double) * w * n + 256, st);
  if (e != cudaSuccess) return e;
  double *at = scratch;
  auto put = [&](const double *src, size_t cnt, const double *&dst) -> cudaError_t {
    dst = at;
    at += cnt;
    return cudaMemcpyAsync(at - cnt, src, sizeof(double) * cnt, cudaMemcpyHostToDevice, st);
  };
  np.stress0 = np.coh = nullptr;
  e = put(pos, (size_t)n * D, np.pos);
  if (e == cudaSuccess) e = put(vel, (size_t)n * D, np.vel);
  if (e == cudaSuccess) e = put(vol, (size_t)n, np.vol);
  if (e == cudaSuccess && stress0) e = put(stress0, (size_t)n * 6, np.stress0);
  if (e == cudaSuccess && cohesion) e = put(cohesion, (size_t)n, np.coh);
  counter = (int32_t *)at;  // 256 spare bytes after the inputs
  if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(int32_t), st);
  return e;
}

}  // namespace

struct mpm_ctx {
  mpm_mesh_desc d;
  mpm_material mat;
  bool has_mat = false;
  bool has_coh = false;
  bool own_stream = false;
  cudaStream_t st = nullptr;
  cudaStream_t st_saved = nullptr;  // own stream while admitted to a batch
  mpm_batch_ctx *batch = nullptr;
  int64_t n = 0, cap = 0;
  int nsm = 152;
  std::string err;
  mpm_status sticky = MPM_OK;
  // FP32 mixed
  Geo geo{};
  int key_bits = 1;
  int64_t nnodes = 0;
  void *bufmem[2] = {nullptr, nullptr};
  PBuf buf[2];
  int cur = 0;  // state buf[cur], old tile ranges tile_start[cur]
  StepBufs s{};
  uint32_t *keys2 = nullptr;  // binning outputs of mpm_read_binning
  int32_t *perm2 = nullptr;
  void *sort_scratch = nullptr;
  GroupDev grp;       // this mesh as a group of one (tables indexed by absolute parity)
  GroupDev grp_bin;   // the same with scratch binning outputs (mpm_read_binning)
  bool grp_valid = false;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int32_t graph_kernels = -1;  // kernel nodes of the last captured step graph
  int32_t lb_withhold = -1, lb_spin = LB_SPIN_LIMIT;  // tile scan test hook (mpm_set_scan_fault)
  int loads = 0;                                     // face tractions and damping (mpm_set_loads)
  double damp = 0.0, trac[6][3] = {};
  bool timing = false;
  bool timed_step = false;
  cudaEvent_t ev[MPM_MAX_PHASES + 1] = {};
  // FP64 plain
  D64Launch L64{};
  void *pmem64 = nullptr;
  void *nmem64 = nullptr;
  double *X64 = nullptr;  // mapped mesh: node coordinates, 3 per node (mpm_set_node_coordinates)
  float4 *cgeo32 = nullptr;  // mapped FP32 mesh: corner positions per cell (Geo::cgeo)
  double *fn64 = nullptr;    // mapped FP64 mesh: face normals (D64Launch::fnorm)
  float4 *fn32 = nullptr;    // mapped FP32 mesh: face normals (Geo::fnorm)
  int64_t fnoff[6] = {};     // offset of each face's table
  double *fl64 = nullptr;    // mapped 2D mesh under face stresses: force per face node (D64Launch::fload)
  float4 *fl32 = nullptr;    // the same in FP32 (Geo::fload)
  double fstress[6][6] = {}; // the face stresses (mpm_set_face_stress)
  bool has_fstress = false;
  // shared
  int32_t *d_status = nullptr;  // FP64 path status word (FP32 path: s.ctr[C_STATUS])
  double *d_cons = nullptr;     // 8 results + partials
};

struct mpm_batch_ctx {
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int nsm = 152;
  int64_t budget = 0;            // device bytes the admitted meshes may hold together (0: no budget)
  int64_t used = 0;              // footprints of the admitted meshes
  int32_t max_slots = 1;
  std::vector<mpm_ctx *> slots;  // nullptr: empty slot
  std::vector<int64_t> slot_bytes;  // footprint of the slot's mesh at admission
  std::vector<int64_t> slot_steps;  // batched steps since admission
  int32_t graph_kernels = -1;
  struct Group {
    int dim, scheme;
    bool mapped;  // mapped FP32 meshes step in groups of their own (the MAP kernels)
    std::vector<mpm_ctx *> mem;
    std::vector<int> slot;
    GroupDev dev;
  };
  std::vector<Group> groups;
  bool dirty = true;
  int bpar = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
};

namespace {

mpm_status fail(mpm_ctx *h, mpm_status s, const std::string &msg) {
  if (h) {
    // a rejected call (malformed, or not valid in this state) changed nothing
    if (s != MPM_ERR_ARG && s != MPM_ERR_STATE && (h->sticky == MPM_OK || s == MPM_ERR_CUDA)) h->sticky = s;
    h->err = msg;
  }
  return s;
}

mpm_status cuda_fail(mpm_ctx *h, cudaError_t e, const char *where) {
  if (e == cudaErrorMemoryAllocation) return fail(h, MPM_ERR_OOM, std::string(where) + ": out of device memory");
  return fail(h, MPM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(expr, where)                                    \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) return cuda_fail(h, _e, where); \
  } while (0)

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

// Device allocations that an error return must release: freed on scope exit
// unless handed over with release().
struct DevGuard {
  void *p[2] = {nullptr, nullptr};
  ~DevGuard() {
    for (void *q : p)
      if (q) cudaFree(q);
  }
  void release() { p[0] = p[1] = nullptr; }
};

// One allocation holds the PBUF_FIELDS fields (the last one only with
// per-particle cohesion), each al256(4 cap) bytes apart.
size_t buf32_bytes(int dim, bool coh, int64_t cap) {
  (void)dim;
  return al256(4 * cap) * (PBUF_FIELDS - (coh ? 0 : 1));
}

void carve32(void *mem, int dim, bool coh, int64_t cap, PBuf &b) {
  (void)dim;
  b.base = (char *)mem;
  b.stride = (int64_t)al256(4 * cap);
  b.has_coh = coh ? 1 : 0;
}

int nfields64(int dim, bool coh, bool mapped) {
  const int ns = dim == 3 ? 6 : 4;
  return 2 * dim + 2 * ns + 3 + (coh ? 1 : 0) + (mapped ? dim : 0);  // + alive, cell (int, counted apart)
}

void carve64(void *mem, int dim, bool coh, bool mapped, int64_t cap, D64State &P) {
  char *p = (char *)mem;
  const size_t f = al256(8 * cap);
  memset(&P, 0, sizeof(P));
  for (int k = 0; k < dim; ++k) { P.x[k] = (double *)p; p += f; }
  for (int k = 0; k < dim; ++k) { P.v[k] = (double *)p; p += f; }
  const int ns = dim == 3 ? 6 : 4;
  for (int i = 0; i < ns; ++i) { P.sig[i] = (double *)p; p += f; }
  for (int i = 0; i < ns; ++i) { P.eps[i] = (double *)p; p += f; }
  P.mass = (double *)p; p += f;
  P.vol = (double *)p; p += f;
  P.epsp = (double *)p; p += f;
  if (coh) { P.coh = (double *)p; p += f; }
  if (mapped)
    for (int k = 0; k < dim; ++k) { P.xi[k] = (double *)p; p += f; }
  P.alive = (int32_t *)p;
  p += al256(4 * cap);
  if (mapped) P.cell = (int32_t *)p;
}

size_t buf64_bytes(int dim, bool coh, bool mapped, int64_t cap) {
  return al256(8 * cap) * nfields64(dim, coh, mapped) + al256(4 * cap) * (mapped ? 2 : 1);
}



template <typename T>
MatConst<T> mat_const(const mpm_material &m) {
  MatConst<T> c;
  c.model = m.model;
  c.E = (T)m.E;
  c.nu = (T)m.nu;
  c.G = (T)(m.E / (2.0 * (1.0 + m.nu)));
  const double G = m.E / (2.0 * (1.0 + m.nu)), lam = m.E * m.nu / ((1.0 + m.nu) * (1.0 - 2.0 * m.nu));
  // plane stress: the in-plane stiffness with lambda* = 2 lambda G / (lambda + 2 G)
  c.lam = (T)(m.model == MPM_PLANE_STRESS_ELASTIC ? 2.0 * lam * G / (lam + 2.0 * G) : lam);
  c.sphi = (T)sin(m.phi);
  c.cphi = (T)cos(m.phi);
  c.spsi = (T)sin(m.psi);
  c.c = (T)m.c;
  return c;
}

// The FP64 launch parameters from the handle (particle/node storage is kept
// in h->L64 as it is allocated).
void fill_launch64(const mpm_ctx *h, D64Launch &L) {
  L.dim = h->d.dim;
  L.scheme = h->d.scheme;
  L.n = h->n;
  for (int k = 0; k < 3; ++k) {
    L.nc[k] = h->d.ncells[k];
    L.origin[k] = h->d.origin[k];
    L.g[k] = h->d.gravity[k];
  }
  L.h = h->d.h;
  L.dt = h->d.dt;
  L.mass_tol = h->d.mass_tol;
  for (int f = 0; f < 6; ++f) {
    L.bc[f] = h->d.face_bc[f];
    L.mu[f] = h->d.face_mu[f];
  }
  L.mat = mat_const<double>(h->mat);
  L.loads = h->loads;
  L.damp = h->damp;
  for (int f = 0; f < 6; ++f)
    for (int k = 0; k < 3; ++k) L.trac[f][k] = h->trac[f][k];
  L.status = h->d_status;
  L.X = h->X64;
  L.fnorm = h->fn64;
  L.fload = h->fl64;
  for (int f = 0; f < 6; ++f) L.fnoff[f] = h->fnoff[f];
}

int tile_dim(int dim, int k) {
  if (dim == 3) return k == 0 ? Tile<3>::TX : k == 1 ? Tile<3>::TY : Tile<3>::TZ;
  return k == 0 ? Tile<2>::TX : k == 1 ? Tile<2>::TY : 1;
}

void destroy_graphs(cudaGraphExec_t g[2]) {
  for (int i = 0; i < 2; ++i)
    if (g[i]) {
      cudaGraphExecDestroy(g[i]);
      g[i] = nullptr;
    }
}

// Kernel nodes of a captured graph (-1 if the graph cannot be inspected).
int32_t count_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return -1;
  std::vector<cudaGraphNode_t> nodes(n);
  if (n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return -1;
  int32_t k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

// Instance arguments of mesh h whose state is in buf[c].
InstArgs make_inst(const mpm_ctx *h, int c, bool scratch_out) {
  InstArgs I;
  memset(&I, 0, sizeof(I));
  I.n = h->n;
  I.ntiles = h->geo.ntiles;
  I.geo = h->geo;
  I.mat = mat_const<float>(h->mat);
  I.matd = mat_const<double>(h->mat);
  I.A = h->buf[c];
  I.B = h->buf[c ^ 1];
  I.s = h->s;
  I.old_start = h->s.tile_start[c];
  I.new_start = h->s.tile_start[c ^ 1];
  I.keys_out = scratch_out ? h->keys2 : h->s.keys_sorted;
  I.perm_out = scratch_out ? h->perm2 : h->s.perm;
  I.ns0 = h->d.ncells[0] + 1;
  I.ns1 = I.ns0 * (h->d.ncells[1] + 1);
  I.lb_withhold = h->lb_withhold;
  I.lb_spin = h->lb_spin;
  return I;
}

// Upload the tables of a group.  relative: table p holds each member at its
// current parity flipped p times (batches); otherwise table p holds every
// member at absolute parity p (a mesh stepped alone).
cudaError_t build_group(GroupDev &g, const std::vector<mpm_ctx *> &mem, bool relative, bool scratch_out, int nsm,
                        cudaStream_t st) {
  const int n = (int)mem.size();
  cudaError_t e;
  if (n > g.cap) {
    free_group(g);
    const int cap = n < 8 ? 8 : n;
    for (int p = 0; p < 2; ++p)
      if ((e = cudaMalloc(&g.tab[p], sizeof(InstArgs) * cap)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&g.pfx, sizeof(int32_t) * (6 * (cap + 1) + W_COUNT))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&g.status, sizeof(int32_t) * cap)) != cudaSuccess) return e;
    if ((e = cudaMemset(g.pfx, 0, sizeof(int32_t) * (6 * (cap + 1) + W_COUNT))) != cudaSuccess) return e;
    g.cap = cap;
  }
  g.ninst = n;
  std::vector<InstArgs> tab[2];
  std::vector<int32_t> pre(3 * (g.cap + 1), 0);
  int32_t *pb = pre.data(), *sb = pb + (g.cap + 1), *mb = sb + (g.cap + 1);
  for (int i = 0; i < n; ++i) {
    const mpm_ctx *h = mem[i];
    for (int p = 0; p < 2; ++p) tab[p].push_back(make_inst(h, relative ? (h->cur ^ p) : p, scratch_out));
    pb[i + 1] = pb[i] + (int32_t)((h->n + 255) / 256);
    sb[i + 1] = sb[i] + (h->geo.ntiles + 1 + 1023) / 1024;
    int64_t m = h->n / 65536;
    mb[i + 1] = mb[i] + (int32_t)(m < 1 ? 1 : (m > 16 ? 16 : m));
  }
  for (int p = 0; p < 2 && n > 0; ++p)
    if ((e = cudaMemcpyAsync(g.tab[p], tab[p].data(), sizeof(InstArgs) * n, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return e;
  if ((e = cudaMemcpyAsync(g.pfx, pre.data(), sizeof(int32_t) * pre.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  for (int p = 0; p < 2; ++p) {
    GroupArgs &G = g.ga[p];
    G.inst = g.tab[p];
    G.ninst = n;
    G.pblk = g.pfx;
    G.sblk = g.pfx + (g.cap + 1);
    G.mblk = g.pfx + 2 * (g.cap + 1);
    G.bin_items = g.pfx + 3 * (g.cap + 1);
    G.act_items = g.pfx + 4 * (g.cap + 1);
    G.res_items = g.pfx + 5 * (g.cap + 1);
    G.work = g.pfx + 6 * (g.cap + 1);
    G.nblk_p = pb[n];
    G.nblk_s = sb[n];
    G.nblk_m = mb[n];
    G.grid = 8 * nsm;
    int max_m = 0;
    for (int i = 0; i < n; ++i) max_m = std::max(max_m, mem[i]->geo.ntiles + 1);
    G.scan_one = max_m <= SCAN1_MAX ? 1 : 0;
    G.mapped = (n > 0 && mem[0]->geo.cgeo) ? 1 : 0;  // a group is all mapped or all Cartesian
    int64_t np = 0;
    for (int i = 0; i < n; ++i) np += mem[i]->n;
    G.bin_t = np >= ((int64_t)1 << 22) ? 128 : 256;
    // the apex band of the FP32 return is empty without cohesion
    G.apex = 0;
    for (int i = 0; i < n; ++i)
      if (mem[i]->mat.model == MPM_MOHR_COULOMB && (mem[i]->has_coh || (float)mem[i]->mat.c != 0.f)) G.apex = 1;
    if (n == 1)
      G.one = tab[p][0];
    else
      memset(&G.one, 0, sizeof(G.one));
  }
  return cudaSuccess;
}

// One FP32 step of a group (enqueue only); phase events if ev.
cudaError_t enqueue_group_step(int dim, int scheme, const GroupArgs &G, cudaEvent_t *ev, cudaStream_t st) {
  cudaError_t e;
  if ((e = phase_mark(ev, 0, st)) != cudaSuccess) return e;
  if ((e = bin_group(dim, G, st)) != cudaSuccess) return e;
  if ((e = phase_mark(ev, 1, st)) != cudaSuccess) return e;
  return f32_group_step(dim, scheme, G, ev, st);
}

mpm_status check_handle(mpm_ctx *h) {
  if (!h) return MPM_ERR_ARG;
  if (h->sticky == MPM_ERR_CUDA || h->sticky == MPM_ERR_OOM) return h->sticky;
  return MPM_OK;
}

mpm_status device_status(mpm_ctx *h) {
  int32_t st = 0;
  cudaError_t e;
  if (h->d.precision == MPM_FP32_MIXED)
    e = cudaMemcpyAsync(&st, h->s.ctr + C_STATUS, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
  else
    e = cudaMemcpyAsync(&st, h->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return cuda_fail(h, e, "status read");
  if (st & ST_NONFINITE) return fail(h, MPM_ERR_NONFINITE, "a particle state became non-finite");
  if (st & ST_LEFT_MESH) return fail(h, MPM_ERR_LEFT_MESH, "a particle left the mesh");
  if (st & ST_TIMEOUT) return fail(h, MPM_ERR_TIMEOUT, "a bounded device wait gave up");
  return h->sticky;
}

mpm_status status_of_bits(int32_t st) {
  if (st & ST_NONFINITE) return MPM_ERR_NONFINITE;
  if (st & ST_LEFT_MESH) return MPM_ERR_LEFT_MESH;
  if (st & ST_TIMEOUT) return MPM_ERR_TIMEOUT;
  return MPM_OK;
}

void free_ptr(void *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <typename T>
void free_t(T *&p) {
  if (p) cudaFree((void *)p);
  p = nullptr;
}

// Device bytes of the FP32 step storage that does not scale with particles.
int64_t f32_fixed_bytes(const mpm_mesh_desc &d, int64_t nt, int64_t nn) {
  const int bn = d.dim == 3 ? box_nodes<3>() : box_nodes<2>();
  int64_t b = 4 * nt * bn * (1 + 2 * d.dim) * (d.scheme == MPM_USL && MPM_FUSED_USL ? 2 : 1) +
              (d.scheme == MPM_USF ? 4 * nt * bn * d.dim : 0);
  b += 9 * 4 * (nt + 2) + 2 * 16 * (nt + 2) + 16 * nn * (d.dim == 3 ? 2 : 1) + 4096;
  return b;
}

}  // namespace

extern "C" {

mpm_status mpm_create_mesh(const mpm_mesh_desc *desc, mpm_handle *out) {
  if (!desc || !out) return MPM_ERR_ARG;
  *out = nullptr;
  const mpm_mesh_desc &d = *desc;
  if (d.dim != 2 && d.dim != 3) return MPM_ERR_ARG;
  for (int k = 0; k < d.dim; ++k)
    if (d.ncells[k] < 1) return MPM_ERR_ARG;
  if (!(d.h > 0) || !(d.dt > 0) || !(d.mass_tol >= 0)) return MPM_ERR_ARG;
  if (d.scheme != MPM_USF && d.scheme != MPM_USL) return MPM_ERR_ARG;
  if (d.precision != MPM_FP64_PLAIN && d.precision != MPM_FP32_MIXED) return MPM_ERR_ARG;
  for (int f = 0; f < 6; ++f) {
    if (d.face_bc[f] < MPM_BC_FREE || d.face_bc[f] > MPM_BC_FRICTION) return MPM_ERR_ARG;
    if (d.face_bc[f] == MPM_BC_FRICTION && !(d.face_mu[f] >= 0)) return MPM_ERR_ARG;
  }
  int64_t nn = 1;
  for (int k = 0; k < d.dim; ++k) nn *= (int64_t)d.ncells[k] + 1;
  if (2 * nn >= ((int64_t)1 << 31)) return MPM_ERR_ARG;  // node records use 32-bit indices
  mpm_ctx *h = new mpm_ctx();
  h->d = d;
  if (d.dim == 2) h->d.ncells[2] = 1;
  h->nnodes = nn;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (d.stream) {
    h->st = (cudaStream_t)d.stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete h;
      return MPM_ERR_CUDA;
    }
    h->own_stream = true;
  }
  cudaError_t e = cudaMalloc(&h->d_cons, sizeof(double) * (8 + 8 * 1024));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_status, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int32_t));
  if (d.precision == MPM_FP32_MIXED && e == cudaSuccess) {
    Geo &g = h->geo;
    memset(&g, 0, sizeof(g));
    int64_t nt = 1;
    for (int k = 0; k < 3; ++k) {
      g.nc[k] = h->d.ncells[k];
      g.nt[k] = (g.nc[k] + tile_dim(d.dim, k) - 1) / tile_dim(d.dim, k);
      nt *= g.nt[k];
    }
    if ((nt + 1) * CELLS_PER_TILE >= (int64_t)1 << 31) {
      mpm_destroy(h);
      return MPM_ERR_ARG;
    }
    g.ntiles = (int)nt;
    g.div_nt0 = make_fastdiv(g.nt[0]);
    g.div_nt01 = make_fastdiv(g.nt[0] * g.nt[1]);
    g.dead_key = (uint32_t)(nt * CELLS_PER_TILE);
    int bits = 1;
    while (((uint64_t)1 << bits) <= g.dead_key) ++bits;
    h->key_bits = bits;
    g.h = (float)d.h;
    g.inv_h = (float)(1.0 / d.h);
    g.dt = (float)d.dt;
    g.mass_tol = (float)d.mass_tol;
    g.inv_rho = 1.f;
    for (int k = 0; k < 3; ++k) g.g[k] = (float)d.gravity[k];
    for (int f = 0; f < 6; ++f) {
      g.bc[f] = d.face_bc[f];
      g.mu[f] = (float)d.face_mu[f];
    }
    const int bn = d.dim == 3 ? box_nodes<3>() : box_nodes<2>();
    const size_t s1 = sizeof(float) * (size_t)nt * bn * (1 + 2 * d.dim);
    const size_t s2 = d.scheme == MPM_USF ? sizeof(float) * (size_t)nt * bn * d.dim : 0;
    StepBufs &S = h->s;
    const size_t ti = sizeof(int32_t) * (nt + 2);
    if (e == cudaSuccess) e = cudaMalloc(&S.slots1, s1);
    if (e == cudaSuccess && s2) e = cudaMalloc(&S.slots2, s2);
    if (e == cudaSuccess && d.scheme == MPM_USL && MPM_FUSED_USL) e = cudaMalloc(&S.slots_a, s1);
    if (e == cudaSuccess) e = cudaMalloc(&S.fepoch, sizeof(int32_t) * nt);
    if (e == cudaSuccess) e = cudaMalloc(&S.aepoch, sizeof(int32_t) * nt);
    if (e == cudaSuccess) e = cudaMalloc(&S.resid, sizeof(int32_t) * (nt + 2));
    if (e == cudaSuccess) e = cudaMemset(S.fepoch, 0xff, sizeof(int32_t) * nt);  // -1: no sums yet
    if (e == cudaSuccess) e = cudaMemset(S.aepoch, 0xff, sizeof(int32_t) * nt);
    for (int p = 0; p < 2 && e == cudaSuccess; ++p) e = cudaMalloc(&S.tile_start[p], ti);
    if (e == cudaSuccess) e = cudaMalloc(&S.in_cnt, ti);
    if (e == cudaSuccess) e = cudaMalloc(&S.out_cnt, ti);
    if (e == cudaSuccess) e = cudaMalloc(&S.bucket_start, ti);
    if (e == cudaSuccess) e = cudaMalloc(&S.bucket_fill, ti);
    if (e == cudaSuccess) e = cudaMalloc(&S.active, sizeof(int4) * (nt + 2));
    if (e == cudaSuccess) e = cudaMalloc(&S.bin_rec, sizeof(int4) * (nt + 2));
    const size_t stb = sizeof(int32_t) * 16 * ((nt + 1) / 1024 + 2);
    if (e == cudaSuccess) e = cudaMalloc(&S.scan_tot, stb);
    if (e == cudaSuccess) e = cudaMemset(S.scan_tot, 0, stb);
    if (e == cudaSuccess) e = cudaMalloc(&S.ctr, sizeof(int32_t) * C_NCTR);
    for (int p = 0; p < 2 && e == cudaSuccess; ++p) e = cudaMemset(S.tile_start[p], 0, ti);
    if (e == cudaSuccess) e = cudaMemset(S.in_cnt, 0, ti);
    if (e == cudaSuccess) e = cudaMemset(S.out_cnt, 0, ti);
    if (e == cudaSuccess) e = cudaMemset(S.bucket_fill, 0, ti);
    if (e == cudaSuccess) e = cudaMemset(S.ctr, 0, sizeof(int32_t) * C_NCTR);
    if (e == cudaSuccess) e = cudaMalloc(&S.node, sizeof(float4) * nn * (d.dim == 3 ? 2 : 1));
    if (e == cudaSuccess) e = f32_prepare(d.dim);
  } else if (e == cudaSuccess) {
    h->L64.nnodes = nn;
    const size_t f = al256(sizeof(double) * nn);
    e = cudaMalloc(&h->nmem64, f * (1 + 5 * d.dim));
    if (e == cudaSuccess) {
      char *p = (char *)h->nmem64;
      D64Nodes &N = h->L64.N;
      N.m = (double *)p; p += f;
      for (int k = 0; k < d.dim; ++k) { N.P[k] = (double *)p; p += f; }
      for (int k = 0; k < d.dim; ++k) { N.f[k] = (double *)p; p += f; }
      for (int k = 0; k < d.dim; ++k) { N.v[k] = (double *)p; p += f; }
      for (int k = 0; k < d.dim; ++k) { N.a[k] = (double *)p; p += f; }
      for (int k = 0; k < d.dim; ++k) { N.vn[k] = (double *)p; p += f; }
    }
  }
  if (e != cudaSuccess) {
    mpm_destroy(h);
    return e == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA;
  }
  *out = h;
  return MPM_OK;
}

mpm_status mpm_footprint(const mpm_mesh_desc *desc, int64_t n, int32_t has_cohesion, int64_t *bytes) {
  if (!desc || !bytes || n < 0 || (desc->dim != 2 && desc->dim != 3)) return MPM_ERR_ARG;
  const mpm_mesh_desc &d = *desc;
  int64_t nn = 1, nt = 1;
  for (int k = 0; k < d.dim; ++k) {
    if (d.ncells[k] < 1) return MPM_ERR_ARG;
    nn *= (int64_t)d.ncells[k] + 1;
    nt *= (d.ncells[k] + tile_dim(d.dim, k) - 1) / tile_dim(d.dim, k);
  }
  const bool coh = has_cohesion != 0;
  if (d.precision == MPM_FP32_MIXED)
    *bytes = 2 * (int64_t)buf32_bytes(d.dim, coh, n) + 7 * 4 * n + (int64_t)sort_scratch_bytes(n) +
             f32_fixed_bytes(d, nt, nn);
  else
    *bytes = (int64_t)buf64_bytes(d.dim, coh, false, n) + 8 * nn * (1 + 5 * d.dim) + 65536;
  return MPM_OK;
}

mpm_status mpm_add_particles(mpm_handle h, int64_t n, const double *pos, const double *vel, const double *vol,
                             const mpm_material *mat, const double *cohesion, const double *stress0,
                             int64_t *first_id) {
  mpm_status s0 = check_handle(h);
  if (s0 != MPM_OK) return s0;
  if (h->batch) return fail(h, MPM_ERR_STATE, "add_particles: the mesh is admitted to a batch");
  if (n < 0 || !mat || (n > 0 && (!pos || !vel || !vol))) return fail(h, MPM_ERR_ARG, "add_particles: bad arguments");
  if (mat->model != MPM_LINEAR_ELASTIC && mat->model != MPM_MOHR_COULOMB && mat->model != MPM_PLANE_STRESS_ELASTIC)
    return fail(h, MPM_ERR_ARG, "unknown material model");
  if (mat->model == MPM_PLANE_STRESS_ELASTIC && h->d.dim != 2)
    return fail(h, MPM_ERR_ARG, "plane stress is a 2D material");
  if (!(mat->E > 0) || !(mat->nu > -1.0 && mat->nu < 0.5) || !(mat->rho > 0))
    return fail(h, MPM_ERR_ARG, "material constants out of range");
  if (h->has_mat && memcmp(&h->mat, mat, sizeof(mpm_material)) != 0)
    return fail(h, MPM_ERR_ARG, "one material per mesh: a different material was passed");
  if (h->n > 0 && (cohesion != nullptr) != h->has_coh)
    return fail(h, MPM_ERR_ARG, "per-particle cohesion must be given for all particles or none");
  if (h->n + n >= ((int64_t)1 << 31) - 1) return fail(h, MPM_ERR_ARG, "too many particles");
  const int D = h->d.dim;
  const mpm_mesh_desc &d = h->d;
  // FP64 storage: reject points outside the mesh on the host (the FP32
  // storage is converted and checked on the device, init_particles_k; a
  // mapped mesh locates them on the device, d64_locate)
  if (h->d.precision != MPM_FP32_MIXED && !h->X64)
    for (int64_t p = 0; p < n; ++p)
      for (int k = 0; k < D; ++k) {
        const double s = (pos[p * D + k] - d.origin[k]) / d.h;
        if (!(s >= 0.0) || floor(s) >= (double)d.ncells[k])
          return fail(h, MPM_ERR_ARG, "a particle lies outside the mesh");
      }
  if (n == 0) {
    if (first_id) *first_id = h->n;
    h->mat = *mat;
    h->has_mat = true;
    return MPM_OK;
  }
  CK(cudaStreamSynchronize(h->st), "add_particles sync");
  const bool coh = cohesion != nullptr;
  const int64_t n0 = h->n, n1 = h->n + n;
  const int ns = D == 3 ? 6 : 4;
  auto cp = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, h->st) : cudaSuccess;
  };
  if (h->d.precision == MPM_FP32_MIXED) {
    const int64_t cap = n1;
    DevGuard guard;
    void **nm = guard.p;
    for (int b = 0; b < 2; ++b) CK(cudaMalloc(&nm[b], buf32_bytes(D, coh, cap)), "particle storage");
    PBuf nb[2];
    carve32(nm[0], D, coh, cap, nb[0]);
    carve32(nm[1], D, coh, cap, nb[1]);
    // nb[1] gathers old + new particles unsorted; nb[0] receives them binned
    const PBuf &ob = h->buf[h->cur];
    if (n0 > 0)
      for (int fi = 0; fi < PBUF_FIELDS - (coh ? 0 : 1); ++fi)
        CK(cp(nb[1].fld(fi), ob.fld(fi), 4 * n0), "copy");
    // the FP64 inputs go up once; one kernel forms every FP32 field
    {
      double *in64 = nullptr;
      int32_t *bad = nullptr;
      NewParticles np;
      cudaError_t e = upload_inputs(h->st, n, D, pos, vel, vol, stress0, cohesion, in64, np, bad);
      if (in64 == nullptr) CK(e, "upload scratch");
      const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8192);
      if (e == cudaSuccess) {
        if (D == 3)
          init_particles_k<3><<<blocks, 256, 0, h->st>>>(n, n0, nb[1], h->geo, d.origin[0], d.origin[1], d.origin[2],
                                                         d.h, mat->rho, np, bad);
        else
          init_particles_k<2><<<blocks, 256, 0, h->st>>>(n, n0, nb[1], h->geo, d.origin[0], d.origin[1], d.origin[2],
                                                         d.h, mat->rho, np, bad);
        e = cudaGetLastError();
      }
      int32_t nbad = 0;
      if (e == cudaSuccess) e = cudaMemcpyAsync(&nbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
      cudaFreeAsync(in64, h->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
      CK(e, "upload");
      if (nbad) return fail(h, MPM_ERR_ARG, "a particle lies outside the mesh");
    }
    // per-particle scratch of the binning
    StepBufs &S = h->s;
    free_t(S.keys_sorted);
    free_t(S.perm);
    free_t(S.movers);
    free_t(S.bucket);
    free_t(S.bucket_sorted);
    free_t(h->keys2);
    free_t(h->perm2);
    free_ptr(h->sort_scratch);
    CK(cudaMalloc(&S.keys_sorted, 4 * cap), "scratch");
    CK(cudaMalloc(&S.perm, 4 * cap), "scratch");
    CK(cudaMalloc(&S.movers, 4 * cap), "scratch");
    CK(cudaMalloc(&S.bucket, 4 * cap), "scratch");
    CK(cudaMalloc(&S.bucket_sorted, 4 * cap), "scratch");
    CK(cudaMalloc(&h->keys2, 4 * cap), "scratch");
    CK(cudaMalloc(&h->perm2, 4 * cap), "scratch");
    CK(cudaMalloc(&h->sort_scratch, sort_scratch_bytes(cap)), "scratch");
    // full stable binning once: sort keys, gather the state in key order
    CK(sort_pairs(nb[1].key(), nullptr, S.keys_sorted, S.perm, n1, h->key_bits, h->sort_scratch, h->st), "binning");
    CK(permute_state(D, n1, nb[1], nb[0], S.perm, h->st), "binning");
    CK(tile_bounds(S.keys_sorted, n1, h->geo.ntiles, S.tile_start[0], h->st), "binning");
    const size_t ti = sizeof(int32_t) * (h->geo.ntiles + 2);
    CK(cudaMemsetAsync(S.in_cnt, 0, ti, h->st), "binning");
    CK(cudaMemsetAsync(S.out_cnt, 0, ti, h->st), "binning");
    CK(cudaMemsetAsync(S.bucket_fill, 0, ti, h->st), "binning");
    CK(cudaMemsetAsync(S.ctr, 0, sizeof(int32_t) * C_STATUS, h->st), "binning");
    // the particle set changed: no tile holds valid partial sums of the next P2G
    CK(cudaMemsetAsync(S.fepoch, 0xff, sizeof(int32_t) * h->geo.ntiles, h->st), "binning");
    CK(cudaMemsetAsync(S.aepoch, 0xff, sizeof(int32_t) * h->geo.ntiles, h->st), "binning");
    CK(cudaStreamSynchronize(h->st), "binning");
    for (int b = 0; b < 2; ++b) free_ptr(h->bufmem[b]);
    h->bufmem[0] = nm[0];
    h->bufmem[1] = nm[1];
    guard.release();
    h->buf[0] = nb[0];
    h->buf[1] = nb[1];
    h->cur = 0;
    h->cap = cap;
    h->geo.inv_rho = (float)(1.0 / mat->rho);
  } else {
    const int64_t cap = n1;
    DevGuard guard;
    void *&nmem = guard.p[0];
    const bool mapped = h->X64 != nullptr;
    CK(cudaMalloc(&nmem, buf64_bytes(D, coh, mapped, cap)), "particle storage");
    D64State P;
    carve64(nmem, D, coh, mapped, cap, P);
    const D64State &O = h->L64.P;
    if (n0 > 0) {
      const size_t b8 = 8 * n0;
      for (int k = 0; k < D; ++k) {
        CK(cp(P.x[k], O.x[k], b8), "copy");
        CK(cp(P.v[k], O.v[k], b8), "copy");
      }
      for (int i = 0; i < ns; ++i) {
        CK(cp(P.sig[i], O.sig[i], b8), "copy");
        CK(cp(P.eps[i], O.eps[i], b8), "copy");
      }
      CK(cp(P.mass, O.mass, b8), "copy");
      CK(cp(P.vol, O.vol, b8), "copy");
      CK(cp(P.epsp, O.epsp, b8), "copy");
      if (coh) CK(cp(P.coh, O.coh, b8), "copy");
      CK(cp(P.alive, O.alive, 4 * n0), "copy");
      if (mapped) {
        CK(cp(P.cell, O.cell, 4 * n0), "copy");
        for (int k = 0; k < D; ++k) CK(cp(P.xi[k], O.xi[k], b8), "copy");
      }
    }
    {  // the FP64 inputs go up once; one kernel fills the new slots
      double *in64 = nullptr;
      int32_t *bad = nullptr;
      NewParticles np;
      cudaError_t e = upload_inputs(h->st, n, D, pos, vel, vol, stress0, cohesion, in64, np, bad);
      if (in64 == nullptr) CK(e, "upload scratch");
      const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8192);
      if (e == cudaSuccess) {
        if (D == 3)
          init_particles64_k<3><<<blocks, 256, 0, h->st>>>(n, n0, P, mat->rho, np);
        else
          init_particles64_k<2><<<blocks, 256, 0, h->st>>>(n, n0, P, mat->rho, np);
        e = cudaGetLastError();
      }
      int32_t nbad = 0;
      if (e == cudaSuccess && mapped) {  // the initial cells by the neighbourhood walk
        D64Launch L = h->L64;
        fill_launch64(h, L);
        L.P = P;
        e = d64_locate(L, n0, n, bad, h->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&nbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
      }
      cudaFreeAsync(in64, h->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
      CK(e, "upload");
      if (nbad > 0) return fail(h, MPM_ERR_ARG, "a particle lies outside the mapped mesh");
    }
    free_ptr(h->pmem64);
    h->pmem64 = nmem;
    guard.release();
    h->L64.P = P;
    h->cap = cap;
  }
  destroy_graphs(h->graph);
  h->grp_valid = false;
  h->n = n1;
  h->has_coh = coh;
  h->mat = *mat;
  h->has_mat = true;
  if (first_id) *first_id = n0;
  return MPM_OK;
}

mpm_status mpm_step(mpm_handle h, int64_t nsteps) {
  mpm_status s0 = check_handle(h);
  if (s0 != MPM_OK) return s0;
  if (h->batch) return fail(h, MPM_ERR_STATE, "step: the mesh is admitted to a batch");
  if (nsteps < 0) return fail(h, MPM_ERR_ARG, "nsteps < 0");
  if (nsteps == 0 || h->n == 0) return h->sticky;
  if (h->d.precision == MPM_FP32_MIXED) {
    if (!h->grp_valid) {
      std::vector<mpm_ctx *> one(1, h);
      CK(build_group(h->grp, one, false, false, h->nsm, h->st), "group tables");
      h->grp_valid = true;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(h->st, &cs);
    const bool use_graph = cs == cudaStreamCaptureStatusNone;
    cudaEvent_t *ev = h->timing ? h->ev : nullptr;
    for (int64_t s = 0; s < nsteps; ++s) {
      const int cur = h->cur;
      if (use_graph) {
        if (!h->graph[cur]) {
          cudaGraph_t g = nullptr;
          CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal), "graph capture");
          cudaError_t e = enqueue_group_step(h->d.dim, h->d.scheme, h->grp.ga[cur], ev, h->st);
          cudaError_t e2 = cudaStreamEndCapture(h->st, &g);
          if (e != cudaSuccess) return cuda_fail(h, e, "step enqueue");
          CK(e2, "graph capture");
          h->graph_kernels = count_kernel_nodes(g);
          e = cudaGraphInstantiate(&h->graph[cur], g, 0);
          cudaGraphDestroy(g);
          CK(e, "graph instantiate");
        }
        CK(cudaGraphLaunch(h->graph[cur], h->st), "graph launch");
      } else {
        CK(enqueue_group_step(h->d.dim, h->d.scheme, h->grp.ga[cur], ev, h->st), "step enqueue");
      }
      h->cur ^= 1;
    }
    if (h->timing) h->timed_step = true;
  } else {
    D64Launch &L = h->L64;
    fill_launch64(h, L);
    for (int64_t s = 0; s < nsteps; ++s) CK(d64_step(L, h->st), "step enqueue");
  }
  return h->sticky;
}

mpm_status mpm_sync(mpm_handle h) {
  if (!h) return MPM_ERR_ARG;
  return device_status(h);
}

mpm_status mpm_num_particles(mpm_handle h, int64_t *n) {
  if (!h || !n) return MPM_ERR_ARG;
  *n = h->n;
  return MPM_OK;
}

mpm_status mpm_read_particles(mpm_handle h, double *pos, double *vel, double *stress, double *strain, double *vol,
                              double *epsp, int64_t *cell) {
  mpm_status s0 = check_handle(h);
  if (s0 != MPM_OK) return s0;
  const int64_t n = h->n;
  const int D = h->d.dim;
  if (n == 0) return device_status(h);
  if (h->d.precision == MPM_FP32_MIXED) {
    // one export of every requested field into device scratch, then the copies
    const PBuf &P = h->buf[h->cur];
    struct Item {
      void *host;
      int width;
    };
    const Item items[7] = {{pos, D}, {vel, D}, {stress, 6}, {strain, 6}, {vol, 1}, {epsp, 1}, {cell, 1}};
    size_t words = 0;
    for (const Item &it : items)
      if (it.host) words += (size_t)it.width * n;
    double *tmp = nullptr;
    CK(cudaMallocAsync((void **)&tmp, sizeof(double) * words, h->st), "read scratch");
    double *o[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    size_t at = 0;
    for (int i = 0; i < 7; ++i)
      if (items[i].host) {
        o[i] = tmp + at;
        at += (size_t)items[i].width * n;
      }
    cudaError_t e = f32_export(D, n, P, h->geo, h->d.origin, h->d.h, h->mat.rho, o[0], o[1], o[2], o[3], o[4], o[5],
                               (int64_t *)o[6], h->st);
    for (int i = 0; i < 7 && e == cudaSuccess; ++i)
      if (items[i].host)
        e = cudaMemcpyAsync(items[i].host, o[i], sizeof(double) * items[i].width * n, cudaMemcpyDeviceToHost, h->st);
    cudaFreeAsync(tmp, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "read_particles");
  } else {
    const D64State &P = h->L64.P;
    const int ns = D == 3 ? 6 : 4;
    std::vector<double> col((size_t)n);
    std::vector<int32_t> alive((size_t)n);
    CK(cudaMemcpyAsync(alive.data(), P.alive, 4 * n, cudaMemcpyDeviceToHost, h->st), "read");
    auto get = [&](const double *src) -> cudaError_t {
      cudaError_t e = cudaMemcpyAsync(col.data(), src, 8 * n, cudaMemcpyDeviceToHost, h->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
      return e;
    };
    const bool mapped = h->X64 != nullptr;
    if (cell)
      for (int64_t p = 0; p < n; ++p) cell[p] = 0;
    if (cell && mapped) {  // the cells the neighbourhood walk keeps
      std::vector<int32_t> c32((size_t)n);
      CK(cudaMemcpyAsync(c32.data(), P.cell, 4 * n, cudaMemcpyDeviceToHost, h->st), "read");
      CK(cudaStreamSynchronize(h->st), "read");
      for (int64_t p = 0; p < n; ++p) cell[p] = alive[p] ? c32[p] : -1;
    }
    for (int k = 0; k < D; ++k) {
      if (pos || (cell && !mapped)) {
        CK(get(P.x[k]), "read");
        if (pos)
          for (int64_t p = 0; p < n; ++p) pos[p * D + k] = col[p];
        if (cell && !mapped) {
          int64_t mul = 1;
          for (int j = 0; j < k; ++j) mul *= h->d.ncells[j];
          for (int64_t p = 0; p < n; ++p) {
            const double s = (col[p] - h->d.origin[k]) / h->d.h;
            const double c = floor(s);
            if (!alive[p] || !(s >= 0) || c >= h->d.ncells[k]) cell[p] = -1;
            if (cell[p] >= 0) cell[p] += (int64_t)c * mul;
          }
        }
      }
      if (vel) {
        CK(get(P.v[k]), "read");
        for (int64_t p = 0; p < n; ++p) vel[p * D + k] = col[p];
      }
    }
    for (int i = 0; i < 6; ++i) {
      if (stress) {
        if (i < ns) {
          CK(get(P.sig[i]), "read");
          for (int64_t p = 0; p < n; ++p) stress[p * 6 + i] = col[p];
        } else {
          for (int64_t p = 0; p < n; ++p) stress[p * 6 + i] = 0.0;
        }
      }
      if (strain) {
        if (i < ns) {
          CK(get(P.eps[i]), "read");
          for (int64_t p = 0; p < n; ++p) strain[p * 6 + i] = col[p];
        } else {
          for (int64_t p = 0; p < n; ++p) strain[p * 6 + i] = 0.0;
        }
      }
    }
    if (vol) {
      CK(get(P.vol), "read");
      memcpy(vol, col.data(), 8 * n);
    }
    if (epsp) {
      CK(get(P.epsp), "read");
      memcpy(epsp, col.data(), 8 * n);
    }
    if (pos)
      for (int64_t p = 0; p < n; ++p)
        if (!alive[p])
          for (int k = 0; k < D; ++k) pos[p * D + k] = NAN;
  }
  return device_status(h);
}

mpm_status mpm_conservation(mpm_handle h, double out[8]) {
  mpm_status s0 = check_handle(h);
  if (s0 != MPM_OK) return s0;
  if (!out) return fail(h, MPM_ERR_ARG, "conservation: null out");
  if (h->n == 0) {
    for (int i = 0; i < 8; ++i) out[i] = 0.0;
    return device_status(h);
  }
  if (h->d.precision == MPM_FP32_MIXED)
    CK(f32_conservation(h->d.dim, h->n, h->buf[h->cur], h->geo.dead_key, h->geo.inv_rho, h->d_cons, h->d_cons + 8,
                        h->st),
       "conservation");
  else
    CK(d64_conservation(h->L64, h->d_cons, h->d_cons + 8, h->st), "conservation");
  double tmp[8];
  CK(cudaMemcpyAsync(tmp, h->d_cons, sizeof(double) * 8, cudaMemcpyDeviceToHost, h->st), "conservation");
  CK(cudaStreamSynchronize(h->st), "conservation");
  for (int i = 0; i < 8; ++i) out[i] = tmp[i];
  return device_status(h);
}

mpm_status mpm_read_binning(mpm_handle h, int32_t *key, int32_t *perm, int32_t *tile_dims) {
  mpm_status s0 = check_handle(h);
  if (s0 != MPM_OK) return s0;
  if (h->d.precision != MPM_FP32_MIXED) return fail(h, MPM_ERR_STATE, "read_binning: FP32_MIXED handles only");
  if (tile_dims)
    for (int k = 0; k < 3; ++k) tile_dims[k] = tile_dim(h->d.dim, k);
  if (h->n == 0) return device_status(h);
  // the production binning of the stored particles, written to scratch so
  // that the next step's binning (which reads the previous binning) is intact
  // (the binning consumes the mover counts left by the last G2P: recount
  // them from the keys before and after, so the next step finds them intact)
  std::vector<mpm_ctx *> one(1, h);
  CK(build_group(h->grp_bin, one, false, true, h->nsm, h->st), "binning tables");
  const GroupArgs &G = h->grp_bin.ga[h->cur];
  const size_t ti = sizeof(int32_t) * (h->geo.ntiles + 2);
  for (int pass = 0; pass < 2; ++pass) {
    CK(cudaMemsetAsync(h->s.in_cnt, 0, ti, h->st), "binning");
    CK(cudaMemsetAsync(h->s.out_cnt, 0, ti, h->st), "binning");
    CK(cudaMemsetAsync(h->s.ctr + C_MOVERS, 0, sizeof(int32_t), h->st), "binning");
    CK(count_movers(G, h->st), "binning");
    if (pass == 0) CK(bin_group(h->d.dim, G, h->st), "binning");
  }
  if (key) CK(cudaMemcpyAsync(key, h->buf[h->cur].key(), 4 * h->n, cudaMemcpyDeviceToHost, h->st), "binning");
  if (perm) CK(cudaMemcpyAsync(perm, h->perm2, 4 * h->n, cudaMemcpyDeviceToHost, h->st), "binning");
  CK(cudaStreamSynchronize(h->st), "binning");
  return device_status(h);
}

mpm_status mpm_set_phase_timing(mpm_handle h, int32_t enable) {
  mpm_status s0 = check_handle(h);
  if (s0 != MPM_OK) return s0;
  if (h->d.precision != MPM_FP32_MIXED) return fail(h, MPM_ERR_STATE, "phase timing: FP32_MIXED handles only");
  const bool on = enable != 0;
  if (on == h->timing) return MPM_OK;
  CK(cudaStreamSynchronize(h->st), "phase timing");
  if (on && !h->ev[0])
    for (int i = 0; i <= MPM_MAX_PHASES; ++i) CK(cudaEventCreate(&h->ev[i]), "phase timing");
  h->timing = on;
  h->timed_step = false;
  destroy_graphs(h->graph);  // recapture with / without the event nodes
  return MPM_OK;
}

mpm_status mpm_phase_times(mpm_handle h, float *ms, int32_t *nphase) {
  mpm_status s0 = check_handle(h);
  if (s0 != MPM_OK) return s0;
  if (!ms || !nphase) return fail(h, MPM_ERR_ARG, "phase_times: null output");
  if (!h->timing || !h->timed_step) return fail(h, MPM_ERR_STATE, "phase_times: no timed step");
  const int np = h->d.scheme == MPM_USL ? 4 : 7;
  CK(cudaEventSynchronize(h->ev[np]), "phase timing");
  for (int i = 0; i < np; ++i) CK(cudaEventElapsedTime(&ms[i], h->ev[i], h->ev[i + 1]), "phase timing");
  *nphase = np;
  return MPM_OK;
}

mpm_status mpm_set_loads(mpm_handle h, const double *face_traction, double damping) {
  mpm_status s0 = check_handle(h);
  if (s0 != MPM_OK) return s0;
  if (h->batch) return fail(h, MPM_ERR_STATE, "set_loads: the mesh is admitted to a batch");
  if (!(damping >= 0.0) || !std::isfinite(damping)) return fail(h, MPM_ERR_ARG, "set_loads: damping must be >= 0");
  double t[6][3] = {};
  int any = damping > 0.0;
  for (int f = 0; f < 6; ++f)
    for (int k = 0; k < 3; ++k) {
      t[f][k] = face_traction ? face_traction[3 * f + k] : 0.0;
      if (!std::isfinite(t[f][k])) return fail(h, MPM_ERR_ARG, "set_loads: traction not finite");
      if (f >= 2 * h->d.dim || k >= h->d.dim) t[f][k] = 0.0;
      if (t[f][k] != 0.0 && h->X64) return fail(h, MPM_ERR_ARG, "set_loads: no face tractions on a mapped mesh");
      any |= t[f][k] != 0.0;
    }
  CK(cudaStreamSynchronize(h->st), "set_loads");
  h->loads = any || h->has_fstress;
  h->damp = damping;
  memcpy(h->trac, t, sizeof(t));
  Geo &g = h->geo;
  g.loads = h->loads;
  g.damp = (float)damping;
  for (int f = 0; f < 6; ++f)
    for (int k = 0; k < 3; ++k) g.trac[f][k] = (float)t[f][k];
  destroy_graphs(h->graph);  // the instance (and its loads) is captured in the step graph
  h->grp_valid = false;
  return MPM_OK;
}

mpm_status mpm_set_node_coordinates(mpm_handle h, const double *node_xyz) {
  mpm_status s0 = check_handle(h);
  if (s0 != MPM_OK) return s0;
  if (h->batch) return fail(h, MPM_ERR_STATE, "node coordinates: the mesh is admitted to a batch");
  if (h->n > 0) return fail(h, MPM_ERR_STATE, "node coordinates: set before the first particles");
  if (!node_xyz) return fail(h, MPM_ERR_ARG, "node coordinates: null");
  for (int f = 0; f < 6; ++f)
    for (int k = 0; k < 3; ++k)
      if (h->trac[f][k] != 0.0) return fail(h, MPM_ERR_ARG, "node coordinates: the mesh carries face tractions");
  if (h->has_fstress) return fail(h, MPM_ERR_STATE, "node coordinates: set them before the face stresses");
  const int D = h->d.dim;
  const int64_t nx = h->d.ncells[0] + 1, ny = h->d.ncells[1] + 1, nz = D == 3 ? h->d.ncells[2] + 1 : 1;
  const int64_t nn = nx * ny * nz;
  std::vector<double> X3((size_t)(3 * nn), 0.0);
  for (int64_t i = 0; i < nn; ++i)
    for (int k = 0; k < D; ++k) {
      const double v = node_xyz[i * D + k];
      if (!std::isfinite(v)) return fail(h, MPM_ERR_ARG, "node coordinates: not finite");
      X3[3 * i + k] = v;
    }
  // every cell must map the reference cell one-to-one and keep its
  // orientation: the Jacobian determinant of the map is positive at each of
  // the cell's corners (there it is the cross product of the edges meeting
  // at the corner)
  auto at = [&](int64_t i, int64_t j, int64_t k, int c) { return X3[3 * (i + nx * (j + ny * k)) + c]; };
  for (int64_t k = 0; k + 1 < nz || (D == 2 && k == 0); ++k)
    for (int64_t j = 0; j + 1 < ny; ++j)
      for (int64_t i = 0; i + 1 < nx; ++i)
        for (int a = 0; a < (1 << D); ++a) {
          const int64_t ci = i + (a & 1), cj = j + ((a >> 1) & 1), ck = k + ((a >> 2) & 1);
          double e[3][3];  // edges from the corner along +axis (reversed at upper corners)
          for (int ax = 0; ax < D; ++ax) {
            const int up = (a >> ax) & 1;
            int64_t o[3] = {ci, cj, ck};
            o[ax] += up ? -1 : 1;
            for (int c = 0; c < D; ++c) {
              const double d = at(o[0], o[1], o[2], c) - at(ci, cj, ck, c);
              e[ax][c] = up ? -d : d;
            }
          }
          double det;
          if (D == 2)
            det = e[0][0] * e[1][1] - e[0][1] * e[1][0];
          else
            det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                  e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                  e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
          if (!(det > 0.0)) return fail(h, MPM_ERR_ARG, "node coordinates: a cell is degenerate or inverted");
        }
  // Outward unit normal of every face at each of its nodes (ISOPARAMETRIC
  // MESH: nodal conditions on irregular surfaces): the normals of the
  // boundary facets next to the node -- 2D edges (as long as the edge), 3D
  // bilinear facets (the cross product of their two edges at the node) --
  // summed, oriented away from the mesh edge that leads inside, normalised.
  // Face f's table runs over the node's indices along the other axes in
  // increasing axis order (Geo::fnorm).
  const int64_t ncl[3] = {h->d.ncells[0], h->d.ncells[1], D == 3 ? h->d.ncells[2] : 0};
  std::vector<double> fnv;
  int64_t fnoff[6] = {0, 0, 0, 0, 0, 0};
  for (int f = 0; f < 2 * D; ++f) {
    const int k = f / 2, up = f & 1;
    int ax[2] = {0, 0}, na = 0;
    for (int c = 0; c < D; ++c)
      if (c != k) ax[na++] = c;
    const int64_t n1 = ncl[ax[0]] + 1, n2 = D == 3 ? ncl[ax[1]] + 1 : 1;
    fnoff[f] = (int64_t)fnv.size() / 3;
    for (int64_t i2 = 0; i2 < n2; ++i2)
      for (int64_t i1 = 0; i1 < n1; ++i1) {
        int64_t ijk[3] = {0, 0, 0};
        ijk[k] = up ? ncl[k] : 0;
        ijk[ax[0]] = i1;
        if (D == 3) ijk[ax[1]] = i2;
        int64_t in[3] = {ijk[0], ijk[1], ijk[2]};
        in[k] += up ? -1 : 1;
        double din[3], acc[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < 3; ++c) din[c] = at(in[0], in[1], in[2], c) - at(ijk[0], ijk[1], ijk[2], c);
        auto edge = [&](int axis, int sgn, double e[3]) -> bool {
          int64_t nb[3] = {ijk[0], ijk[1], ijk[2]};
          nb[axis] += sgn;
          if (nb[axis] < 0 || nb[axis] > ncl[axis]) return false;
          for (int c = 0; c < 3; ++c) e[c] = at(nb[0], nb[1], nb[2], c) - at(ijk[0], ijk[1], ijk[2], c);
          return true;
        };
        if (D == 2) {
          for (int sgn = -1; sgn <= 1; sgn += 2) {
            double e[3];
            if (!edge(ax[0], sgn, e)) continue;
            double q0 = e[1], q1 = -e[0];
            if (q0 * din[0] + q1 * din[1] > 0.0) {
              q0 = -q0;
              q1 = -q1;
            }
            acc[0] += q0;
            acc[1] += q1;
          }
        } else {
          for (int s1 = -1; s1 <= 1; s1 += 2)
            for (int s2 = -1; s2 <= 1; s2 += 2) {
              double ea[3], eb[3];
              if (!edge(ax[0], s1, ea) || !edge(ax[1], s2, eb)) continue;
              double q[3] = {ea[1] * eb[2] - ea[2] * eb[1], ea[2] * eb[0] - ea[0] * eb[2],
                             ea[0] * eb[1] - ea[1] * eb[0]};
              const double sd = q[0] * din[0] + q[1] * din[1] + q[2] * din[2];
              for (int c = 0; c < 3; ++c) acc[c] += sd > 0.0 ? -q[c] : q[c];
            }
        }
        const double len = std::sqrt(acc[0] * acc[0] + acc[1] * acc[1] + acc[2] * acc[2]);
        for (int c = 0; c < 3; ++c) fnv.push_back(acc[c] / len);
      }
  }
  // FP32 path: per cell the corners relative to the cell's centre, in units
  // of h, computed in FP64 and rounded once (Geo::cgeo)
  std::vector<float4> cg;
  if (h->d.precision == MPM_FP32_MIXED) {
    const int nf = D == 3 ? CGEO_F4<3>() : CGEO_F4<2>();
    const int64_t ncx = h->d.ncells[0], ncy = h->d.ncells[1], ncz = D == 3 ? h->d.ncells[2] : 1;
    cg.assign((size_t)(ncx * ncy * ncz * nf), make_float4(0.f, 0.f, 0.f, 0.f));
    for (int64_t k = 0; k < ncz; ++k)
      for (int64_t j = 0; j < ncy; ++j)
        for (int64_t i = 0; i < ncx; ++i) {
          double ctr[3] = {0.0, 0.0, 0.0}, xa[8][3];
          for (int a = 0; a < (1 << D); ++a)
            for (int c = 0; c < D; ++c) {
              xa[a][c] = at(i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1), c);
              ctr[c] += xa[a][c];
            }
          float f[24] = {};
          for (int a = 0; a < (1 << D); ++a)
            for (int c = 0; c < D; ++c) f[D * a + c] = (float)((xa[a][c] - ctr[c] / (1 << D)) / h->d.h);
          float4 *dst = &cg[(size_t)((i + ncx * (j + ncy * k)) * nf)];
          for (int m = 0; m < nf; ++m) dst[m] = make_float4(f[4 * m], f[4 * m + 1], f[4 * m + 2], f[4 * m + 3]);
        }
  }
  double *dX = nullptr, *dN64 = nullptr;
  float4 *dG = nullptr, *dN32 = nullptr;
  const size_t nfn = fnv.size() / 3;
  CK(cudaStreamSynchronize(h->st), "node coordinates");
  CK(cudaMalloc(&dX, sizeof(double) * 3 * nn), "node coordinates");
  cudaError_t e = cudaMemcpy(dX, X3.data(), sizeof(double) * 3 * nn, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !cg.empty()) {
    e = cudaMalloc(&dG, sizeof(float4) * cg.size());
    if (e == cudaSuccess) e = cudaMemcpy(dG, cg.data(), sizeof(float4) * cg.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && h->d.precision == MPM_FP32_MIXED) {
    std::vector<float4> f4(nfn);
    for (size_t i = 0; i < nfn; ++i)
      f4[i] = make_float4((float)fnv[3 * i], (float)fnv[3 * i + 1], (float)fnv[3 * i + 2], 0.f);
    e = cudaMalloc(&dN32, sizeof(float4) * nfn);
    if (e == cudaSuccess) e = cudaMemcpy(dN32, f4.data(), sizeof(float4) * nfn, cudaMemcpyHostToDevice);
  } else if (e == cudaSuccess) {
    e = cudaMalloc(&dN64, sizeof(double) * 3 * nfn);
    if (e == cudaSuccess) e = cudaMemcpy(dN64, fnv.data(), sizeof(double) * 3 * nfn, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cudaFree(dX);
    if (dG) cudaFree(dG);
    if (dN32) cudaFree(dN32);
    if (dN64) cudaFree(dN64);
    return cuda_fail(h, e, "node coordinates");
  }
  if (h->X64) cudaFree(h->X64);
  if (h->cgeo32) cudaFree(h->cgeo32);
  if (h->fn64) cudaFree(h->fn64);
  if (h->fn32) cudaFree(h->fn32);
  h->X64 = dX;
  h->cgeo32 = dG;
  h->fn64 = dN64;
  h->fn32 = dN32;
  for (int f = 0; f < 6; ++f) {
    h->fnoff[f] = fnoff[f];
    h->geo.fnoff[f] = (int)fnoff[f];
  }
  h->geo.X = h->d.precision == MPM_FP32_MIXED ? dX : nullptr;
  h->geo.cgeo = dG;
  h->geo.fnorm = dN32;
  destroy_graphs(h->graph);  // the instance (and its geometry) is captured in the step graph
  h->grp_valid = false;
  return MPM_OK;
}

mpm_status mpm_set_face_stress(mpm_handle h, const double *face_stress) {
  mpm_status s0 = check_handle(h);
  if (s0 != MPM_OK) return s0;
  if (h->batch) return fail(h, MPM_ERR_STATE, "face stress: the mesh is admitted to a batch");
  if (!h->X64 || h->d.dim != 2) return fail(h, MPM_ERR_ARG, "face stress: mapped 2D meshes only");
  double S[6][6] = {};
  bool any = false;
  for (int f = 0; f < 6; ++f)
    for (int k = 0; k < 6; ++k) {
      S[f][k] = face_stress ? face_stress[6 * f + k] : 0.0;
      if (!std::isfinite(S[f][k])) return fail(h, MPM_ERR_ARG, "face stress: not finite");
      if (f >= 4) S[f][k] = 0.0;
      any |= S[f][k] != 0.0;
    }
  // node coordinates back from the device copy (3 per node)
  const int64_t nx = h->d.ncells[0] + 1, ny = h->d.ncells[1] + 1;
  std::vector<double> X3((size_t)(3 * nx * ny));
  CK(cudaStreamSynchronize(h->st), "face stress");
  CK(cudaMemcpy(X3.data(), h->X64, sizeof(double) * X3.size(), cudaMemcpyDeviceToHost), "face stress");
  auto at = [&](int64_t i, int64_t j, int c) { return X3[3 * (i + nx * j) + c]; };
  // the force of face f's stress on each of its nodes: for each boundary
  // edge of f at the node, sigma_f . (the edge turned outward) / 2 -- the
  // traction sigma . n of the uniform stress over the edge, half to each end
  const int64_t nn = h->fnoff[3] + (h->d.ncells[0] + 1);  // the four faces' tables
  std::vector<double> fl((size_t)(3 * nn), 0.0);
  for (int f = 0; f < 4; ++f) {
    const double *sf = S[f];
    if (sf[0] == 0.0 && sf[1] == 0.0 && sf[3] == 0.0) continue;
    const int k = f / 2, t = 1 - k, up = f & 1;
    const int64_t nt_ = h->d.ncells[t] + 1;
    for (int64_t it = 0; it < nt_; ++it) {
      int64_t ij[2];
      ij[k] = up ? h->d.ncells[k] : 0;
      ij[t] = it;
      int64_t in[2] = {ij[0], ij[1]};
      in[k] += up ? -1 : 1;
      const double dx = at(in[0], in[1], 0) - at(ij[0], ij[1], 0), dy = at(in[0], in[1], 1) - at(ij[0], ij[1], 1);
      double fx = 0.0, fy = 0.0;
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        int64_t nb[2] = {ij[0], ij[1]};
        nb[t] += sgn;
        if (nb[t] < 0 || nb[t] > h->d.ncells[t]) continue;
        double qx = at(nb[0], nb[1], 1) - at(ij[0], ij[1], 1), qy = -(at(nb[0], nb[1], 0) - at(ij[0], ij[1], 0));
        if (qx * dx + qy * dy > 0.0) {
          qx = -qx;
          qy = -qy;
        }
        fx += 0.5 * (sf[0] * qx + sf[3] * qy);
        fy += 0.5 * (sf[3] * qx + sf[1] * qy);
      }
      const int64_t e = h->fnoff[f] + it;
      fl[3 * e] += fx;
      fl[3 * e + 1] += fy;
    }
  }
  double *d64 = nullptr;
  float4 *d32 = nullptr;
  cudaError_t e = cudaSuccess;
  if (any && h->d.precision == MPM_FP32_MIXED) {
    std::vector<float4> f4((size_t)nn);
    for (int64_t i = 0; i < nn; ++i) f4[i] = make_float4((float)fl[3 * i], (float)fl[3 * i + 1], 0.f, 0.f);
    e = cudaMalloc(&d32, sizeof(float4) * nn);
    if (e == cudaSuccess) e = cudaMemcpy(d32, f4.data(), sizeof(float4) * nn, cudaMemcpyHostToDevice);
  } else if (any) {
    e = cudaMalloc(&d64, sizeof(double) * 3 * nn);
    if (e == cudaSuccess) e = cudaMemcpy(d64, fl.data(), sizeof(double) * 3 * nn, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    if (d32) cudaFree(d32);
    if (d64) cudaFree(d64);
    return cuda_fail(h, e, "face stress");
  }
  if (h->fl64) cudaFree(h->fl64);
  if (h->fl32) cudaFree(h->fl32);
  h->fl64 = d64;
  h->fl32 = d32;
  memcpy(h->fstress, S, sizeof(S));
  h->has_fstress = any;
  bool trac_any = false;
  for (int f = 0; f < 6; ++f)
    for (int k = 0; k < 3; ++k) trac_any |= h->trac[f][k] != 0.0;
  h->loads = any || trac_any || h->damp > 0.0;
  h->geo.loads = h->loads;
  h->geo.fload = d32;
  destroy_graphs(h->graph);  // the instance (and its loads) is captured in the step graph
  h->grp_valid = false;
  return MPM_OK;
}

mpm_status mpm_set_scan_fault(mpm_handle h, int32_t withhold_chunk, int32_t spin_limit) {
  mpm_status s0 = check_handle(h);
  if (s0 != MPM_OK) return s0;
  if (h->d.precision != MPM_FP32_MIXED) return fail(h, MPM_ERR_STATE, "scan fault: FP32_MIXED handles only");
  if (h->batch) return fail(h, MPM_ERR_STATE, "scan fault: the mesh is admitted to a batch");
  if (withhold_chunk < -1 || spin_limit < 1 || spin_limit > LB_SPIN_LIMIT)
    return fail(h, MPM_ERR_ARG, "scan fault: bad arguments");
  CK(cudaStreamSynchronize(h->st), "scan fault");
  h->lb_withhold = withhold_chunk;
  h->lb_spin = spin_limit;
  destroy_graphs(h->graph);  // the instance (and its hook) is captured in the step graph
  h->grp_valid = false;
  return MPM_OK;
}

mpm_status mpm_step_kernels(mpm_handle h, int32_t *kernels) {
  if (!h || !kernels) return MPM_ERR_ARG;
  if (h->d.precision != MPM_FP32_MIXED || h->graph_kernels < 0) return MPM_ERR_STATE;
  *kernels = h->graph_kernels;
  return MPM_OK;
}

const char *mpm_last_error(mpm_handle h) {
  if (!h) return "null handle";
  return h->err.empty() ? "no error" : h->err.c_str();
}

mpm_status mpm_destroy(mpm_handle h) {
  if (!h) return MPM_OK;
  if (h->batch) {  // leave the batch first
    mpm_batch_ctx *b = h->batch;
    for (size_t i = 0; i < b->slots.size(); ++i)
      if (b->slots[i] == h) mpm_batch_evict(b, (int32_t)i);
  }
  if (h->st) cudaStreamSynchronize(h->st);
  destroy_graphs(h->graph);
  free_group(h->grp);
  free_group(h->grp_bin);
  StepBufs &S = h->s;
  void *ptrs[] = {h->bufmem[0], h->bufmem[1], S.keys_sorted, S.perm, S.tile_start[0], S.tile_start[1], S.in_cnt,
                  S.out_cnt, S.bucket_start, S.bucket_fill, S.movers, S.bucket, S.bucket_sorted, S.active,
                  S.bin_rec, S.scan_tot, S.ctr, S.slots1, S.slots2, S.slots_a, S.fepoch, S.aepoch, S.resid, S.node,
                  h->keys2, h->perm2, h->sort_scratch,
                  h->pmem64, h->nmem64, h->X64, h->cgeo32, h->fn64, h->fn32, h->fl64, h->fl32, h->d_status,
                  h->d_cons};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (int i = 0; i <= MPM_MAX_PHASES; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  if (h->own_stream && h->st) cudaStreamDestroy(h->st);
  delete h;
  return MPM_OK;
}

// ---- batches ---------------------------------------------------------------

mpm_status mpm_batch_create(int64_t hbm_budget_bytes, int32_t max_slots, void *stream, mpm_batch *out) {
  if (!out) return MPM_ERR_ARG;
  *out = nullptr;
  if (hbm_budget_bytes < 0 || max_slots < 1) return MPM_ERR_ARG;
  mpm_batch_ctx *b = new mpm_batch_ctx();
  b->budget = hbm_budget_bytes;
  b->max_slots = max_slots;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  if (stream) {
    b->st = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return MPM_ERR_CUDA;
    }
    b->own_stream = true;
  }
  *out = b;
  return MPM_OK;
}

mpm_status mpm_batch_admit(mpm_batch b, mpm_handle h, int32_t *slot) {
  if (!b || !h) return MPM_ERR_ARG;
  mpm_status s0 = check_handle(h);
  if (s0 != MPM_OK) return s0;
  if (h->d.precision != MPM_FP32_MIXED) return fail(h, MPM_ERR_ARG, "batch: FP32_MIXED meshes only");
  if (h->batch) return fail(h, MPM_ERR_STATE, "batch: the mesh is already admitted to a batch");
  // room: a free slot, and the mesh's footprint within what the budget has left
  int s = -1;
  for (size_t i = 0; i < b->slots.size(); ++i)
    if (!b->slots[i]) {
      s = (int)i;
      break;
    }
  if (s < 0 && (int32_t)b->slots.size() >= b->max_slots) {
    h->err = "batch admit: every slot is taken";
    return MPM_ERR_OOM;  // not latched: the mesh is unchanged
  }
  int64_t fp = 0;
  if (mpm_footprint(&h->d, h->n, h->has_coh ? 1 : 0, &fp) != MPM_OK) return fail(h, MPM_ERR_ARG, "batch admit: footprint");
  if (b->budget > 0 && fp > b->budget - b->used) {
    h->err = "batch admit: the mesh does not fit the batch's memory budget";
    return MPM_ERR_OOM;  // not latched: the mesh is unchanged
  }
  CK(cudaStreamSynchronize(h->st), "batch admit");
  CK(cudaStreamSynchronize(b->st), "batch admit");
  h->st_saved = h->st;
  h->st = b->st;
  h->batch = b;
  if (s < 0) {
    s = (int)b->slots.size();
    b->slots.push_back(nullptr);
    b->slot_bytes.push_back(0);
    b->slot_steps.push_back(0);
  }
  b->slots[s] = h;
  b->slot_bytes[s] = fp;
  b->slot_steps[s] = 0;
  b->used += fp;
  b->dirty = true;
  if (slot) *slot = s;
  return MPM_OK;
}

mpm_status mpm_batch_evict(mpm_batch b, int32_t slot) {
  if (!b || slot < 0 || slot >= (int32_t)b->slots.size() || !b->slots[slot]) return MPM_ERR_ARG;
  if (cudaStreamSynchronize(b->st) != cudaSuccess) return MPM_ERR_CUDA;
  mpm_ctx *h = b->slots[slot];
  h->st = h->st_saved;
  h->batch = nullptr;
  b->slots[slot] = nullptr;
  b->used -= b->slot_bytes[slot];
  b->slot_bytes[slot] = 0;
  b->dirty = true;
  return MPM_OK;
}

mpm_status mpm_batch_step(mpm_batch b, int64_t nsteps) {
  if (!b || nsteps < 0) return MPM_ERR_ARG;
  if (nsteps == 0) return MPM_OK;
  if (b->dirty) {
    if (cudaStreamSynchronize(b->st) != cudaSuccess) return MPM_ERR_CUDA;
    destroy_graphs(b->graph);
    for (auto &g : b->groups) free_group(g.dev);
    b->groups.clear();
    for (size_t i = 0; i < b->slots.size(); ++i) {
      mpm_ctx *h = b->slots[i];
      if (!h || h->n == 0) continue;
      mpm_batch_ctx::Group *gp = nullptr;
      const bool mapped = h->geo.cgeo != nullptr;
      for (auto &g : b->groups)
        if (g.dim == h->d.dim && g.scheme == h->d.scheme && g.mapped == mapped) gp = &g;
      if (!gp) {
        b->groups.push_back(mpm_batch_ctx::Group{h->d.dim, h->d.scheme, mapped, {}, {}, GroupDev()});
        gp = &b->groups.back();
      }
      gp->mem.push_back(h);
      gp->slot.push_back((int)i);
    }
    for (auto &g : b->groups)
      if (build_group(g.dev, g.mem, true, false, b->nsm, b->st) != cudaSuccess) return MPM_ERR_CUDA;
    b->bpar = 0;
    b->dirty = false;
  }
  if (b->groups.empty()) return MPM_OK;
  for (int64_t s = 0; s < nsteps; ++s) {
    const int p = b->bpar;
    if (!b->graph[p]) {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MPM_ERR_CUDA;
      cudaError_t e = cudaSuccess;
      for (auto &gr : b->groups)
        if (e == cudaSuccess) e = enqueue_group_step(gr.dim, gr.scheme, gr.dev.ga[p], nullptr, b->st);
      cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return MPM_ERR_CUDA;
      }
      b->graph_kernels = count_kernel_nodes(g);
      e = cudaGraphInstantiate(&b->graph[p], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return MPM_ERR_CUDA;
    }
    if (cudaGraphLaunch(b->graph[p], b->st) != cudaSuccess) return MPM_ERR_CUDA;
    b->bpar ^= 1;
    for (auto &gr : b->groups)
      for (mpm_ctx *h : gr.mem) h->cur ^= 1;
  }
  for (auto &gr : b->groups)
    for (int sl : gr.slot) b->slot_steps[sl] += nsteps;
  return MPM_OK;
}

mpm_status mpm_batch_poll(mpm_batch b, int32_t nslots, int32_t *slot_status, int64_t *slot_steps) {
  if (!b || nslots < 0 || (nslots > 0 && !slot_status)) return MPM_ERR_ARG;
  for (int i = 0; i < nslots; ++i) slot_status[i] = MPM_ERR_STATE;
  if (slot_steps)
    for (int i = 0; i < nslots; ++i)
      slot_steps[i] = (i < (int)b->slots.size() && b->slots[i]) ? b->slot_steps[i] : -1;
  std::vector<int32_t> bits;
  for (auto &gr : b->groups) {
    if (b->dirty) break;
    if (gather_status(gr.dev.tab[0], gr.dev.ninst, gr.dev.status, b->st) != cudaSuccess) return MPM_ERR_CUDA;
    bits.resize(gr.dev.ninst);
    if (cudaMemcpyAsync(bits.data(), gr.dev.status, sizeof(int32_t) * gr.dev.ninst, cudaMemcpyDeviceToHost, b->st) !=
        cudaSuccess)
      return MPM_ERR_CUDA;
    if (cudaStreamSynchronize(b->st) != cudaSuccess) return MPM_ERR_CUDA;
    for (int k = 0; k < gr.dev.ninst; ++k)
      if (gr.slot[k] < nslots) slot_status[gr.slot[k]] = status_of_bits(bits[k]);
  }
  if (cudaStreamSynchronize(b->st) != cudaSuccess) return MPM_ERR_CUDA;
  // meshes admitted since the last batched step (or with no particles)
  for (int i = 0; i < nslots && i < (int)b->slots.size(); ++i) {
    mpm_ctx *h = b->slots[i];
    if (h && slot_status[i] == MPM_ERR_STATE) {
      int32_t st = 0;
      if (cudaMemcpy(&st, h->s.ctr + C_STATUS, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
        return MPM_ERR_CUDA;
      slot_status[i] = status_of_bits(st);
    }
  }
  return MPM_OK;
}

mpm_status mpm_batch_room(mpm_batch b, int64_t *free_bytes, int32_t *free_slots) {
  if (!b) return MPM_ERR_ARG;
  int32_t taken = 0;
  for (mpm_ctx *h : b->slots) taken += h ? 1 : 0;
  if (free_bytes) *free_bytes = b->budget > 0 ? b->budget - b->used : INT64_MAX;
  if (free_slots) *free_slots = b->max_slots - taken;
  return MPM_OK;
}

mpm_status mpm_batch_step_kernels(mpm_batch b, int32_t *kernels) {
  if (!b || !kernels) return MPM_ERR_ARG;
  if (b->graph_kernels < 0) return MPM_ERR_STATE;
  *kernels = b->graph_kernels;
  return MPM_OK;
}

mpm_status mpm_batch_destroy(mpm_batch b) {
  if (!b) return MPM_OK;
  for (size_t i = 0; i < b->slots.size(); ++i)
    if (b->slots[i]) mpm_batch_evict(b, (int32_t)i);
  cudaStreamSynchronize(b->st);
  destroy_graphs(b->graph);
  for (auto &g : b->groups) free_group(g.dev);
  if (b->own_stream) cudaStreamDestroy(b->st);
  delete b;
  return MPM_OK;
}

// ---- standalone primitives ---------------------------------------------------

mpm_status mpm_sort_keys(const uint32_t *d_keys, int32_t *d_perm, int64_t n, int32_t key_bits, void *stream) {
  if (n < 0 || key_bits < 1 || key_bits > 32 || (n > 0 && (!d_keys || !d_perm))) return MPM_ERR_ARG;
  if (n >= ((int64_t)1 << 31)) return MPM_ERR_ARG;
  if (n == 0) return MPM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  void *scratch = nullptr;
  uint32_t *kout = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, sort_scratch_bytes(n), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&kout, 4 * n, st);
  if (e == cudaSuccess) e = sort_pairs(d_keys, nullptr, kout, d_perm, n, key_bits, scratch, st);
  if (kout) cudaFreeAsync(kout, st);
  if (scratch) cudaFreeAsync(scratch, st);
  cudaError_t e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  if (e == cudaErrorMemoryAllocation) return MPM_ERR_OOM;
  return e == cudaSuccess ? MPM_OK : MPM_ERR_CUDA;
}

mpm_status mpm_material_update(const mpm_material *mat, int32_t precision, int64_t n, const double *sig,
                               const double *deps, const double *cohesion, double *sig_out, double *depsp_out,
                               void *stream) {
  if (!mat || n < 0 || (n > 0 && (!sig || !deps || !sig_out))) return MPM_ERR_ARG;
  if (precision != MPM_FP64_PLAIN && precision != MPM_FP32_MIXED) return MPM_ERR_ARG;
  if (n == 0) return MPM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (precision == MPM_FP64_PLAIN) {
    double *d = nullptr;
    const size_t nb = sizeof(double) * n;
    e = cudaMallocAsync((void **)&d, nb * 20, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA;
    double *ds = d, *dd = d + 6 * n, *dc = d + 12 * n, *dout = d + 13 * n, *dep = d + 19 * n;
    e = cudaMemcpyAsync(ds, sig, nb * 6, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dd, deps, nb * 6, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && cohesion) e = cudaMemcpyAsync(dc, cohesion, nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = material_update_f64(mat_const<double>(*mat), n, ds, dd, cohesion ? dc : nullptr, dout, dep, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sig_out, dout, nb * 6, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && depsp_out) e = cudaMemcpyAsync(depsp_out, dep, nb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d, st);
    cudaStreamSynchronize(st);
  } else {
    std::vector<float> hs(6 * n), hd(6 * n), hc(cohesion ? n : 0), ho(6 * n), he(n);
    for (int64_t i = 0; i < 6 * n; ++i) {
      hs[i] = (float)sig[i];
      hd[i] = (float)deps[i];
    }
    for (int64_t i = 0; i < (int64_t)hc.size(); ++i) hc[i] = (float)cohesion[i];
    float *d = nullptr;
    const size_t nb = sizeof(float) * n;
    e = cudaMallocAsync((void **)&d, nb * 20, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? MPM_ERR_OOM : MPM_ERR_CUDA;
    float *ds = d, *dd = d + 6 * n, *dc = d + 12 * n, *dout = d + 13 * n, *dep = d + 19 * n;
    e = cudaMemcpyAsync(ds, hs.data(), nb * 6, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dd, hd.data(), nb * 6, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && cohesion) e = cudaMemcpyAsync(dc, hc.data(), nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = material_update_f32(mat_const<float>(*mat), mat_const<double>(*mat), n, ds, dd, cohesion ? dc : nullptr,
                              dout, dep, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ho.data(), dout, nb * 6, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(he.data(), dep, nb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d, st);
    cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
      for (int64_t i = 0; i < 6 * n; ++i) sig_out[i] = ho[i];
      if (depsp_out)
        for (int64_t i = 0; i < n; ++i) depsp_out[i] = he[i];
    }
  }
  if (e == cudaErrorMemoryAllocation) return MPM_ERR_OOM;
  return e == cudaSuccess ? MPM_OK : MPM_ERR_CUDA;
}

}  // extern "C"
