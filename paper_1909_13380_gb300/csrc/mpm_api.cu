// mpm_api.cu -- the C ABI declared in include/mpm.h.
//
// Host side of the library: validates descriptors, owns device storage,
// computes each particle's initial cell on the host in FP64 (cell =
// floor((x - origin)/h) per axis; the offset from the cell centre, in cell
// units, is rounded to FP32 for the mixed path), bins the particles once with
// a full stable radix sort when they are added, enqueues steps on the
// handle's stream (replaying a captured CUDA graph per step when the stream
// allows capture), and converts the state back to FP64 in insertion order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/mpm.h"
#include "mpm_internal.h"

using namespace mpm;

struct mpm_ctx {
  mpm_mesh_desc d;
  mpm_material mat;
  bool has_mat = false;
  bool has_coh = false;
  bool own_stream = false;
  cudaStream_t st = nullptr;
  int64_t n = 0, cap = 0;
  int nsm = 152;
  std::string err;
  mpm_status sticky = MPM_OK;
  // FP32 mixed
  Geo geo;
  int key_bits = 1;
  int64_t nnodes = 0;
  void *bufmem[2] = {nullptr, nullptr};
  PBuf buf[2];
  int cur = 0;  // state buf[cur], old tile ranges tile_start[cur]
  StepBufs s{};
  uint32_t *keys2 = nullptr;  // binning outputs of mpm_read_binning
  int32_t *perm2 = nullptr;
  void *sort_scratch = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool timing = false;
  bool timed_step = false;
  cudaEvent_t ev[MPM_MAX_PHASES + 1] = {};
  // FP64 plain
  D64Launch L64{};
  void *pmem64 = nullptr;
  void *nmem64 = nullptr;
  // shared
  int32_t *d_status = nullptr;  // FP64 path status word (FP32 path: s.ctr[C_STATUS])
  double *d_cons = nullptr;     // 8 results + partials
};

namespace {

mpm_status fail(mpm_ctx *h, mpm_status s, const std::string &msg) {
  if (h) {
    if (s != MPM_ERR_ARG && (h->sticky == MPM_OK || s == MPM_ERR_CUDA)) h->sticky = s;
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

int nfields32(int dim, bool coh) {
  // off[D] vel[D] sig[NS] eps[NS] mass jm1 epsp (coh)
  const int ns = dim == 3 ? 6 : 4;
  return 2 * dim + 2 * ns + 3 + (coh ? 1 : 0);
}

size_t buf32_bytes(int dim, bool coh, int64_t cap) { return al256(4 * cap) * (2 + nfields32(dim, coh)); }

void carve32(void *mem, int dim, bool coh, int64_t cap, PBuf &b) {
  char *p = (char *)mem;
  const size_t f = al256(4 * cap);
  memset(&b, 0, sizeof(b));
  b.key = (uint32_t *)p; p += f;
  b.id = (int32_t *)p; p += f;
  for (int k = 0; k < dim; ++k) { b.off[k] = (float *)p; p += f; }
  for (int k = 0; k < dim; ++k) { b.vel[k] = (float *)p; p += f; }
  const int ns = dim == 3 ? 6 : 4;
  for (int i = 0; i < ns; ++i) { b.sig[i] = (float *)p; p += f; }
  for (int i = 0; i < ns; ++i) { b.eps[i] = (float *)p; p += f; }
  b.mass = (float *)p; p += f;
  b.jm1 = (float *)p; p += f;
  b.epsp = (float *)p; p += f;
  b.coh = coh ? (float *)p : nullptr;
}

int nfields64(int dim, bool coh) {
  const int ns = dim == 3 ? 6 : 4;
  return 2 * dim + 2 * ns + 3 + (coh ? 1 : 0);  // + alive (int, counted apart)
}

void carve64(void *mem, int dim, bool coh, int64_t cap, D64State &P) {
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
  P.alive = (int32_t *)p;
}

size_t buf64_bytes(int dim, bool coh, int64_t cap) { return al256(8 * cap) * nfields64(dim, coh) + al256(4 * cap); }

template <typename T>
MatConst<T> mat_const(const mpm_material &m) {
  MatConst<T> c;
  c.model = m.model;
  c.E = (T)m.E;
  c.nu = (T)m.nu;
  c.G = (T)(m.E / (2.0 * (1.0 + m.nu)));
  c.lam = (T)(m.E * m.nu / ((1.0 + m.nu) * (1.0 - 2.0 * m.nu)));
  c.sphi = (T)sin(m.phi);
  c.cphi = (T)cos(m.phi);
  c.spsi = (T)sin(m.psi);
  c.c = (T)m.c;
  return c;
}

void destroy_graphs(mpm_ctx *h) {
  for (int i = 0; i < 2; ++i)
    if (h->graph[i]) {
      cudaGraphExecDestroy(h->graph[i]);
      h->graph[i] = nullptr;
    }
}

int tile_dim(int dim, int k) {
  if (dim == 3) return k == 0 ? Tile<3>::TX : k == 1 ? Tile<3>::TY : Tile<3>::TZ;
  return k == 0 ? Tile<2>::TX : k == 1 ? Tile<2>::TY : 1;
}

BinLaunch bin_launch(mpm_ctx *h, int cur, uint32_t *keys_out, int32_t *perm_out) {
  BinLaunch B;
  B.n = h->n;
  B.ntiles = h->geo.ntiles;
  B.knew = h->buf[cur].key;
  B.kold = h->s.keys_sorted;
  B.old_start = h->s.tile_start[cur];
  B.new_start = h->s.tile_start[cur ^ 1];
  B.s = h->s;
  B.keys_out = keys_out;
  B.perm_out = perm_out;
  B.grid = 8 * h->nsm;
  return B;
}

// One FP32 step from buf[cur] to buf[cur ^ 1] (enqueue only).
cudaError_t enqueue_f32_step(mpm_ctx *h, int cur) {
  cudaError_t e;
  cudaEvent_t *ev = h->timing ? h->ev : nullptr;
  if ((e = phase_mark(ev, 0, h->st)) != cudaSuccess) return e;
  if ((e = bin_step(bin_launch(h, cur, h->s.keys_sorted, h->s.perm), h->st)) != cudaSuccess) return e;
  if ((e = phase_mark(ev, 1, h->st)) != cudaSuccess) return e;
  F32Launch L;
  L.dim = h->d.dim;
  L.scheme = h->d.scheme;
  L.n = h->n;
  L.geo = h->geo;
  L.mat = mat_const<float>(h->mat);
  L.matd = mat_const<double>(h->mat);
  L.A = h->buf[cur];
  L.B = h->buf[cur ^ 1];
  L.s = h->s;
  L.tile_start = h->s.tile_start[cur ^ 1];
  L.node_stride[0] = (int64_t)h->d.ncells[0] + 1;
  L.node_stride[1] = L.node_stride[0] * ((int64_t)h->d.ncells[1] + 1);
  L.grid = 8 * h->nsm;
  L.ev = ev;
  return f32_step(L, h->st);
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

void free_ptr(void *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

template <typename T>
void free_t(T *&p) {
  if (p) cudaFree((void *)p);
  p = nullptr;
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
  if (nn >= ((int64_t)1 << 34)) return MPM_ERR_ARG;
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
  cudaError_t e = cudaMalloc(&h->d_cons, sizeof(double) * (8 + 7 * 1024));
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
    for (int p = 0; p < 2 && e == cudaSuccess; ++p) e = cudaMalloc(&S.tile_start[p], ti);
    if (e == cudaSuccess) e = cudaMalloc(&S.in_cnt, ti);
    if (e == cudaSuccess) e = cudaMalloc(&S.out_cnt, ti);
    if (e == cudaSuccess) e = cudaMalloc(&S.bucket_start, ti);
    if (e == cudaSuccess) e = cudaMalloc(&S.bucket_fill, ti);
    if (e == cudaSuccess) e = cudaMalloc(&S.active, ti);
    if (e == cudaSuccess) e = cudaMalloc(&S.scan_tot, sizeof(int32_t) * 3 * ((nt + 1) / 1024 + 1));
    if (e == cudaSuccess) e = cudaMalloc(&S.ctr, sizeof(int32_t) * C_NCTR);
    for (int p = 0; p < 2 && e == cudaSuccess; ++p) e = cudaMemset(S.tile_start[p], 0, ti);
    if (e == cudaSuccess) e = cudaMemset(S.in_cnt, 0, ti);
    if (e == cudaSuccess) e = cudaMemset(S.out_cnt, 0, ti);
    if (e == cudaSuccess) e = cudaMemset(S.bucket_fill, 0, ti);
    if (e == cudaSuccess) e = cudaMemset(S.ctr, 0, sizeof(int32_t) * C_NCTR);
    if (2 * nn >= ((int64_t)1 << 31)) {  // node records are indexed with 32-bit ints
      mpm_destroy(h);
      return MPM_ERR_ARG;
    }
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

mpm_status mpm_add_particles(mpm_handle h, int64_t n, const double *pos, const double *vel, const double *vol,
                             const mpm_material *mat, const double *cohesion, const double *stress0,
                             int64_t *first_id) {
  mpm_status s0 = check_handle(h);
  if (s0 != MPM_OK) return s0;
  if (n < 0 || !mat || (n > 0 && (!pos || !vel || !vol))) return fail(h, MPM_ERR_ARG, "add_particles: bad arguments");
  if (mat->model != MPM_LINEAR_ELASTIC && mat->model != MPM_MOHR_COULOMB)
    return fail(h, MPM_ERR_ARG, "unknown material model");
  if (!(mat->E > 0) || !(mat->nu > -1.0 && mat->nu < 0.5) || !(mat->rho > 0))
    return fail(h, MPM_ERR_ARG, "material constants out of range");
  if (h->has_mat && memcmp(&h->mat, mat, sizeof(mpm_material)) != 0)
    return fail(h, MPM_ERR_ARG, "one material per mesh: a different material was passed");
  if (h->n > 0 && (cohesion != nullptr) != h->has_coh)
    return fail(h, MPM_ERR_ARG, "per-particle cohesion must be given for all particles or none");
  if (h->n + n >= ((int64_t)1 << 31) - 1) return fail(h, MPM_ERR_ARG, "too many particles");
  const int D = h->d.dim;
  const mpm_mesh_desc &d = h->d;
  // initial cells (FP64, host): floor((x - origin)/h); reject outside points
  std::vector<int32_t> cell((size_t)n * D);
  std::vector<double> off((size_t)n * D);
  for (int64_t p = 0; p < n; ++p)
    for (int k = 0; k < D; ++k) {
      const double s = (pos[p * D + k] - d.origin[k]) / d.h;
      if (!(s >= 0.0)) return fail(h, MPM_ERR_ARG, "a particle lies outside the mesh");
      const double f = floor(s);
      if (f >= (double)d.ncells[k]) return fail(h, MPM_ERR_ARG, "a particle lies outside the mesh");
      cell[p * D + k] = (int32_t)f;
      off[p * D + k] = s - f - 0.5;
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
    void *nm[2] = {nullptr, nullptr};
    for (int b = 0; b < 2; ++b) CK(cudaMalloc(&nm[b], buf32_bytes(D, coh, cap)), "particle storage");
    PBuf nb[2];
    carve32(nm[0], D, coh, cap, nb[0]);
    carve32(nm[1], D, coh, cap, nb[1]);
    // nb[1] gathers old + new particles unsorted; nb[0] receives them binned
    const PBuf &ob = h->buf[h->cur];
    if (n0 > 0) {
      const size_t b4 = 4 * n0;
      CK(cp(nb[1].key, ob.key, b4), "copy");
      CK(cp(nb[1].id, ob.id, b4), "copy");
      for (int k = 0; k < D; ++k) {
        CK(cp(nb[1].off[k], ob.off[k], b4), "copy");
        CK(cp(nb[1].vel[k], ob.vel[k], b4), "copy");
      }
      for (int i = 0; i < ns; ++i) {
        CK(cp(nb[1].sig[i], ob.sig[i], b4), "copy");
        CK(cp(nb[1].eps[i], ob.eps[i], b4), "copy");
      }
      CK(cp(nb[1].mass, ob.mass, b4), "copy");
      CK(cp(nb[1].jm1, ob.jm1, b4), "copy");
      CK(cp(nb[1].epsp, ob.epsp, b4), "copy");
      if (coh) CK(cp(nb[1].coh, ob.coh, b4), "copy");
    }
    std::vector<uint32_t> key(n);
    std::vector<int32_t> id(n);
    std::vector<float> f((size_t)n);
    for (int64_t p = 0; p < n; ++p) {
      int c[3] = {0, 0, 0};
      for (int k = 0; k < D; ++k) c[k] = cell[p * D + k];
      const int T0 = tile_dim(D, 0), T1 = tile_dim(D, 1), T2 = tile_dim(D, 2);
      const int t = c[0] / T0 + h->geo.nt[0] * (c[1] / T1 + h->geo.nt[1] * (c[2] / T2));
      const int l = c[0] % T0 + T0 * (c[1] % T1 + T1 * (c[2] % T2));
      key[p] = (uint32_t)t * CELLS_PER_TILE + (uint32_t)l;
      id[p] = (int32_t)(n0 + p);
    }
    CK(cudaMemcpyAsync(nb[1].key + n0, key.data(), 4 * n, cudaMemcpyHostToDevice, h->st), "upload");
    CK(cudaMemcpyAsync(nb[1].id + n0, id.data(), 4 * n, cudaMemcpyHostToDevice, h->st), "upload");
    auto up = [&](float *dst, auto get) -> cudaError_t {
      for (int64_t p = 0; p < n; ++p) f[p] = get(p);
      cudaError_t e = cudaMemcpyAsync(dst + n0, f.data(), 4 * n, cudaMemcpyHostToDevice, h->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);  // f is reused
      return e;
    };
    for (int k = 0; k < D; ++k) {
      CK(up(nb[1].off[k], [&](int64_t p) {
           float u = (float)off[p * D + k];
           if (u >= 0.5f) u = nextafterf(0.5f, 0.f);
           if (u < -0.5f) u = -0.5f;
           return u;
         }), "upload");
      CK(up(nb[1].vel[k], [&](int64_t p) { return (float)vel[p * D + k]; }), "upload");
    }
    for (int i = 0; i < ns; ++i) {
      CK(up(nb[1].sig[i], [&](int64_t p) { return stress0 ? (float)stress0[p * 6 + i] : 0.f; }), "upload");
      CK(up(nb[1].eps[i], [&](int64_t) { return 0.f; }), "upload");
    }
    CK(up(nb[1].mass, [&](int64_t p) { return (float)(mat->rho * vol[p]); }), "upload");
    CK(up(nb[1].jm1, [&](int64_t) { return 0.f; }), "upload");
    CK(up(nb[1].epsp, [&](int64_t) { return 0.f; }), "upload");
    if (coh) CK(up(nb[1].coh, [&](int64_t p) { return (float)cohesion[p]; }), "upload");
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
    CK(sort_pairs(nb[1].key, nullptr, S.keys_sorted, S.perm, n1, h->key_bits, h->sort_scratch, h->st), "binning");
    CK(permute_state(D, n1, nb[1], nb[0], S.perm, h->st), "binning");
    CK(tile_bounds(S.keys_sorted, n1, h->geo.ntiles, S.tile_start[0], h->st), "binning");
    const size_t ti = sizeof(int32_t) * (h->geo.ntiles + 2);
    CK(cudaMemsetAsync(S.in_cnt, 0, ti, h->st), "binning");
    CK(cudaMemsetAsync(S.out_cnt, 0, ti, h->st), "binning");
    CK(cudaMemsetAsync(S.bucket_fill, 0, ti, h->st), "binning");
    CK(cudaMemsetAsync(S.ctr, 0, sizeof(int32_t) * C_STATUS, h->st), "binning");
    CK(cudaStreamSynchronize(h->st), "binning");
    for (int b = 0; b < 2; ++b) free_ptr(h->bufmem[b]);
    h->bufmem[0] = nm[0];
    h->bufmem[1] = nm[1];
    h->buf[0] = nb[0];
    h->buf[1] = nb[1];
    h->cur = 0;
    h->cap = cap;
    h->geo.inv_rho = (float)(1.0 / mat->rho);
  } else {
    const int64_t cap = n1;
    void *nmem = nullptr;
    CK(cudaMalloc(&nmem, buf64_bytes(D, coh, cap)), "particle storage");
    D64State P;
    carve64(nmem, D, coh, cap, P);
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
    }
    std::vector<double> f((size_t)n);
    auto up = [&](double *dst, auto get) -> cudaError_t {
      for (int64_t p = 0; p < n; ++p) f[p] = get(p);
      cudaError_t e = cudaMemcpyAsync(dst + n0, f.data(), 8 * n, cudaMemcpyHostToDevice, h->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
      return e;
    };
    for (int k = 0; k < D; ++k) {
      CK(up(P.x[k], [&](int64_t p) { return pos[p * D + k]; }), "upload");
      CK(up(P.v[k], [&](int64_t p) { return vel[p * D + k]; }), "upload");
    }
    for (int i = 0; i < ns; ++i) {
      CK(up(P.sig[i], [&](int64_t p) { return stress0 ? stress0[p * 6 + i] : 0.0; }), "upload");
      CK(up(P.eps[i], [&](int64_t) { return 0.0; }), "upload");
    }
    CK(up(P.mass, [&](int64_t p) { return mat->rho * vol[p]; }), "upload");
    CK(up(P.vol, [&](int64_t p) { return vol[p]; }), "upload");
    CK(up(P.epsp, [&](int64_t) { return 0.0; }), "upload");
    if (coh) CK(up(P.coh, [&](int64_t p) { return cohesion[p]; }), "upload");
    std::vector<int32_t> one((size_t)n, 1);
    CK(cudaMemcpyAsync(P.alive + n0, one.data(), 4 * n, cudaMemcpyHostToDevice, h->st), "upload");
    CK(cudaStreamSynchronize(h->st), "upload");
    free_ptr(h->pmem64);
    h->pmem64 = nmem;
    h->L64.P = P;
    h->cap = cap;
  }
  destroy_graphs(h);
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
  if (nsteps < 0) return fail(h, MPM_ERR_ARG, "nsteps < 0");
  if (nsteps == 0 || h->n == 0) return h->sticky;
  if (h->d.precision == MPM_FP32_MIXED) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(h->st, &cs);
    const bool use_graph = cs == cudaStreamCaptureStatusNone;
    for (int64_t s = 0; s < nsteps; ++s) {
      const int cur = h->cur;
      if (use_graph) {
        if (!h->graph[cur]) {
          cudaGraph_t g = nullptr;
          CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal), "graph capture");
          cudaError_t e = enqueue_f32_step(h, cur);
          cudaError_t e2 = cudaStreamEndCapture(h->st, &g);
          if (e != cudaSuccess) return cuda_fail(h, e, "step enqueue");
          CK(e2, "graph capture");
          e = cudaGraphInstantiate(&h->graph[cur], g, 0);
          cudaGraphDestroy(g);
          CK(e, "graph instantiate");
        }
        CK(cudaGraphLaunch(h->graph[cur], h->st), "graph launch");
      } else {
        CK(enqueue_f32_step(h, cur), "step enqueue");
      }
      h->cur ^= 1;
    }
    if (h->timing) h->timed_step = true;
  } else {
    D64Launch &L = h->L64;
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
    L.status = h->d_status;
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
    double *tmp = nullptr;
    CK(cudaMallocAsync((void **)&tmp, sizeof(double) * 6 * n, h->st), "read scratch");
    const PBuf &P = h->buf[h->cur];
    struct Item {
      void *host;
      int width;
      int which;
    };
    const Item items[7] = {{pos, D, 0},  {vel, D, 1},  {stress, 6, 2}, {strain, 6, 3},
                           {vol, 1, 4},  {epsp, 1, 5}, {cell, 1, 6}};
    cudaError_t e = cudaSuccess;
    for (const Item &it : items) {
      if (!it.host || e != cudaSuccess) continue;
      double *o[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
      o[it.which] = tmp;
      e = f32_export(D, n, P, h->geo, h->d.origin, h->d.h, h->mat.rho, o[0], o[1], o[2], o[3], o[4], o[5],
                     (int64_t *)o[6], h->st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(it.host, tmp, sizeof(double) * it.width * n, cudaMemcpyDeviceToHost, h->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    }
    cudaFreeAsync(tmp, h->st);
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
    if (cell)
      for (int64_t p = 0; p < n; ++p) cell[p] = 0;
    for (int k = 0; k < D; ++k) {
      if (pos || cell) {
        CK(get(P.x[k]), "read");
        if (pos)
          for (int64_t p = 0; p < n; ++p) pos[p * D + k] = col[p];
        if (cell) {
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

mpm_status mpm_conservation(mpm_handle h, double out[7]) {
  mpm_status s0 = check_handle(h);
  if (s0 != MPM_OK) return s0;
  if (!out) return fail(h, MPM_ERR_ARG, "conservation: null out");
  if (h->n == 0) {
    for (int i = 0; i < 7; ++i) out[i] = 0.0;
    return device_status(h);
  }
  if (h->d.precision == MPM_FP32_MIXED)
    CK(f32_conservation(h->d.dim, h->n, h->buf[h->cur], h->geo.dead_key, h->geo.inv_rho, h->d_cons, h->d_cons + 8,
                        h->st),
       "conservation");
  else
    CK(d64_conservation(h->L64, h->d_cons, h->d_cons + 8, h->st), "conservation");
  double tmp[8];
  CK(cudaMemcpyAsync(tmp, h->d_cons, sizeof(double) * 7, cudaMemcpyDeviceToHost, h->st), "conservation");
  CK(cudaStreamSynchronize(h->st), "conservation");
  for (int i = 0; i < 7; ++i) out[i] = tmp[i];
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
  CK(bin_step(bin_launch(h, h->cur, h->keys2, h->perm2), h->st), "binning");
  if (key) CK(cudaMemcpyAsync(key, h->buf[h->cur].key, 4 * h->n, cudaMemcpyDeviceToHost, h->st), "binning");
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
  destroy_graphs(h);  // recapture with / without the event nodes
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

const char *mpm_last_error(mpm_handle h) {
  if (!h) return "null handle";
  return h->err.empty() ? "no error" : h->err.c_str();
}

mpm_status mpm_destroy(mpm_handle h) {
  if (!h) return MPM_OK;
  if (h->st) cudaStreamSynchronize(h->st);
  destroy_graphs(h);
  StepBufs &S = h->s;
  void *ptrs[] = {h->bufmem[0], h->bufmem[1], S.keys_sorted, S.perm, S.tile_start[0], S.tile_start[1], S.in_cnt,
                  S.out_cnt, S.bucket_start, S.bucket_fill, S.movers, S.bucket, S.bucket_sorted, S.active,
                  S.scan_tot, S.ctr,
                  S.slots1, S.slots2, S.node,
                  h->keys2, h->perm2, h->sort_scratch, h->pmem64, h->nmem64, h->d_status, h->d_cons};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (int i = 0; i <= MPM_MAX_PHASES; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  if (h->own_stream && h->st) cudaStreamDestroy(h->st);
  delete h;
  return MPM_OK;
}

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
