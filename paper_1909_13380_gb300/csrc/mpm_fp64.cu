// mpm_fp64.cu -- the plain FP64 explicit MPM step on the GPU.
//
// Paper (arXiv 1909.13380): INTRODUCTION (particle -> node mapping, nodal
// solve, node -> particle interpolation, nodal values reset each step),
// CODE OVERVIEW (USF / USL explicit schemes, linear quad/hex, Material),
// DATA STRUCTURES (particle updates are independent; nodal updates are
// aggregated with atomic updates per node), ISOPARAMETRIC MESH (nodal
// velocity and frictional conditions).
//
// This is the simplest correct GPU step and the comparison point of the
// FP32 mixed path: FP64 global positions, particles in insertion order,
// FP64 atomicAdd into a dense node grid that is cleared every step -- the
// GPU analogue of the paper's per-node atomic update.
//
// On a mapped (isoparametric) mesh (ISOPARAMETRIC MESH) the cells are the
// images of [-1, 1]^d under x(xi) = sum_a N_a(xi) X_a.  Each particle keeps
// its cell and its natural coordinates there; after advection a
// neighbourhood walk from the old cell finds the new ones (Newton-Raphson
// from the inverse bilinear solution in 2D, from the affine guess in 3D), so
// the transfers of the next step only evaluate N and dN/dx = dN/dxi J^-1.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mpm_internal.h"
#include "mpm_iso.cuh"

namespace mpm {
namespace {

constexpr int BS = 256;

inline int nblk(int64_t n) {
  int64_t b = (n + BS - 1) / BS;
  return (int)(b < 1 ? 1 : (b > 65535 * 4 ? 65535 * 4 : b));
}

template <int D>
__device__ __forceinline__ bool locate(const D64Launch &L, const double x[D], int c[3], double xi[D]) {
  c[0] = c[1] = c[2] = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double s = (x[k] - L.origin[k]) / L.h;
    if (!(s >= 0.0)) return false;
    const double f = floor(s);
    if (f >= (double)L.nc[k]) return false;
    c[k] = (int)f;
    xi[k] = 2.0 * (s - f) - 1.0;
  }
  return true;
}

template <int D>
__device__ __forceinline__ int64_t node_of(const D64Launch &L, const int c[3], int a) {
  const int64_t nx = L.nc[0] + 1, ny = L.nc[1] + 1;
  const int64_t i = c[0] + (a & 1), j = c[1] + ((a >> 1) & 1), k = D == 3 ? c[2] + ((a >> 2) & 1) : 0;
  return i + nx * (j + ny * k);
}

template <int D>
__device__ __forceinline__ void load_pos(const D64Launch &L, int64_t p, double x[D]) {
#pragma unroll
  for (int k = 0; k < D; ++k) x[k] = L.P.x[k][p];
}

__device__ __forceinline__ iso::IsoGrid iso_grid(const D64Launch &L) {
  return iso::IsoGrid{L.X, {L.nc[0], L.nc[1], L.nc[2]}};
}

// Shape values and physical gradients of particle p: on a Cartesian mesh
// from its position; on a mapped mesh from its stored cell and natural
// coordinates, G = dN/dxi J^-1.  False if the particle is in no cell.
template <int D, bool MAP>
__device__ __forceinline__ bool particle_basis(const D64Launch &L, int64_t p, int c[3], double N[1 << D],
                                               double G[1 << D][D]) {
  if (!MAP) {
    double x[D], xi[D];
    load_pos<D>(L, p, x);
    if (!locate<D>(L, x, c, xi)) return false;
    shape_fn<D, double>(xi, 1.0 / L.h, N, G);
    return true;
  }
  const iso::IsoGrid M = iso_grid(L);
  iso::cell_split(M, L.P.cell[p], c);
  double xi[D], xa[1 << D][D], xm[D], J[D][D], Ji[D][D], Gx[1 << D][D];
#pragma unroll
  for (int k = 0; k < D; ++k) xi[k] = L.P.xi[k][p];
  iso::cell_xyz<D>(M, c, xa);
  iso::cell_map<D>(xa, xi, xm, J);
  if (!iso::invert<D>(J, Ji)) return false;
  shape_fn<D, double>(xi, 0.5, N, Gx);
#pragma unroll
  for (int a = 0; a < (1 << D); ++a)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double g = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) g += Gx[a][k] * Ji[k][j];
      G[a][j] = g;
    }
  return true;
}

// mode: 0 mass+momentum+force, 1 mass+momentum, 2 force only.
template <int D, int MODE, bool MAP>
__global__ void p2g64(D64Launch L) {
  constexpr int NC = 1 << D;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < L.n; p += (int64_t)gridDim.x * blockDim.x) {
    if (!L.P.alive[p]) continue;
    int c[3];
    double N[NC], G[NC][D];
    if (!particle_basis<D, MAP>(L, p, c, N, G)) continue;
    const double m = L.P.mass[p];
    double s6[6] = {0, 0, 0, 0, 0, 0};
    if (MODE != 1) {
      if (D == 3) {
#pragma unroll
        for (int i = 0; i < 6; ++i) s6[i] = L.P.sig[i][p];
      } else {
        s6[0] = L.P.sig[0][p]; s6[1] = L.P.sig[1][p]; s6[3] = L.P.sig[3][p];
      }
    }
    const double T3[3][3] = {{s6[0], s6[3], s6[5]}, {s6[3], s6[1], s6[4]}, {s6[5], s6[4], s6[2]}};
    const double V = L.P.vol[p];
#pragma unroll
    for (int a = 0; a < NC; ++a) {
      const int64_t i = node_of<D>(L, c, a);
      if (MODE != 2) {
        atomicAdd(&L.N.m[i], N[a] * m);
#pragma unroll
        for (int k = 0; k < D; ++k) atomicAdd(&L.N.P[k][i], N[a] * m * L.P.v[k][p]);
      }
      if (MODE != 1) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
          double sg = 0.0;
#pragma unroll
          for (int k = 0; k < D; ++k) sg += T3[j][k] * G[a][k];
          atomicAdd(&L.N.f[j][i], -V * sg + N[a] * m * L.g[j]);
        }
      }
    }
  }
}

// stage 0: v from P with velocity conditions (USF);
// stage 1: USL (v from P, a, v', full conditions);
// stage 2: USF force stage (v kept, a, v', full conditions).
template <int D, int STAGE>
__global__ void node64(D64Launch L) {
  const int64_t nx = L.nc[0] + 1, ny = L.nc[1] + 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L.nnodes; i += (int64_t)gridDim.x * blockDim.x) {
    const int I[3] = {(int)(i % nx), (int)((i / nx) % ny), D == 3 ? (int)(i / (nx * ny)) : 0};
    int faces = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (I[k] == 0) faces |= 1 << (2 * k);
      if (I[k] == L.nc[k]) faces |= 1 << (2 * k + 1);
    }
    const double m = L.N.m[i];
    const bool active = m > L.mass_tol;
    double v[D], a[D], vn[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      v[k] = STAGE == 2 ? L.N.v[k][i] : (active ? L.N.P[k][i] / m : 0.0);
      a[k] = vn[k] = 0.0;
    }
    double nrm[6][3];  // a mapped mesh's boundary node: its faces' outward normals
    if (L.fnorm && faces) {
#pragma unroll
      for (int f = 0; f < 2 * D; ++f)
        if ((faces >> f) & 1) {
          const double *q = L.fnorm + 3 * (L.fnoff[f] + face_node_index<D>(f, I, L.nc));
          nrm[f][0] = q[0];
          nrm[f][1] = q[1];
          nrm[f][2] = q[2];
        }
    }
    if (STAGE == 0) {
      if (L.fnorm && faces)
        bc_velocity_n<D, double>(faces, L.bc, nrm, v);
      else
        bc_velocity<D, double>(faces, L.bc, v);
#pragma unroll
      for (int k = 0; k < D; ++k) L.N.v[k][i] = v[k];
      continue;
    }
    if (active) {
      double ft[D];
      if (L.loads) face_force<D, double>(faces, I, L.nc, L.h, L.trac, ft);
      if (L.loads && L.fload && faces)  // face stresses on a mapped mesh
#pragma unroll
        for (int f = 0; f < 2 * D; ++f)
          if ((faces >> f) & 1) {
            const double *q = L.fload + 3 * (L.fnoff[f] + face_node_index<D>(f, I, L.nc));
#pragma unroll
            for (int k = 0; k < D; ++k) ft[k] += q[k];
          }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        a[k] = L.loads ? (L.N.f[k][i] + ft[k]) / m - L.damp * v[k] : L.N.f[k][i] / m;
        vn[k] = v[k] + a[k] * L.dt;
      }
      if (L.fnorm && faces)
        bc_full_n<D, double>(faces, L.bc, L.mu, L.dt, nrm, v, a, vn);
      else
        bc_full<D, double>(faces, L.bc, L.mu, L.dt, v, a, vn);
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) v[k] = 0.0;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      L.N.v[k][i] = v[k];
      L.N.a[k][i] = a[k];
      L.N.vn[k][i] = vn[k];
    }
  }
}

// mode: 0 USL (everything), 1 USF stress stage, 2 USF advection stage.
template <int D, int MODE, bool MAP>
__global__ void g2p64(D64Launch L) {
  constexpr int NC = 1 << D;
  constexpr int NS = nstress<D>();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < L.n; p += (int64_t)gridDim.x * blockDim.x) {
    if (!L.P.alive[p]) continue;
    double x[D];
    int c[3];
    double N[NC], G[NC][D];
    if (!particle_basis<D, MAP>(L, p, c, N, G)) continue;
    load_pos<D>(L, p, x);
    double dv[D], vb[D], Lg[D][D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      dv[k] = vb[k] = 0.0;
#pragma unroll
      for (int l = 0; l < D; ++l) Lg[k][l] = 0.0;
    }
    double *const *vel = MODE == 1 ? L.N.v : L.N.vn;
#pragma unroll
    for (int a = 0; a < NC; ++a) {
      const int64_t i = node_of<D>(L, c, a);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double vk = vel[k][i];
        if (MODE != 1) {
          dv[k] += N[a] * L.N.a[k][i];
          vb[k] += N[a] * vk;
        }
#pragma unroll
        for (int l = 0; l < D; ++l) Lg[k][l] += vk * G[a][l];
      }
    }
    int status = 0;
    if (MODE != 2) {
      double de[6] = {0, 0, 0, 0, 0, 0};
      de[0] = Lg[0][0] * L.dt;
      de[1] = Lg[1][1] * L.dt;
      de[3] = 0.5 * (Lg[0][1] + Lg[1][0]) * L.dt;
      if (D == 3) {
        de[2] = Lg[D - 1][D - 1] * L.dt;
        de[4] = 0.5 * (Lg[1][D - 1] + Lg[D - 1][1]) * L.dt;
        de[5] = 0.5 * (Lg[0][D - 1] + Lg[D - 1][0]) * L.dt;
      }
      double sg[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        sg[i] = L.P.sig[i][p];
        L.P.eps[i][p] += de[i];
      }
      L.P.vol[p] *= 1.0 + de[0] + de[1] + de[2];
      double ep = L.P.epsp[p];
      material_update(L.mat, L.P.coh ? L.P.coh[p] : L.mat.c, sg, de, ep);
      L.P.epsp[p] = ep;
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        L.P.sig[i][p] = sg[i];
        if (!isfinite(sg[i])) status |= ST_NONFINITE;
      }
    }
    if (MODE != 1) {
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double vk = L.P.v[k][p] + L.dt * dv[k];
        L.P.v[k][p] = vk;
        x[k] += L.dt * vb[k];
        L.P.x[k][p] = x[k];
        if (!isfinite(vk)) status |= ST_NONFINITE;
      }
      int c2[3] = {c[0], c[1], c[2]};
      double xi2[D];
      bool found;
      if (MAP) {
        found = iso::walk<D>(iso_grid(L), x, c2, xi2);
        if (found) {
          L.P.cell[p] = iso::cell_id(iso_grid(L), c2);
#pragma unroll
          for (int k = 0; k < D; ++k) L.P.xi[k][p] = xi2[k];
        }
      } else {
        found = locate<D>(L, x, c2, xi2);
      }
      if (!found) {
        L.P.alive[p] = 0;
        status |= ST_LEFT_MESH;
      }
    }
    if (status) atomicOr(L.status, status);
  }
}

// Initial cells of new particles on a mapped mesh: the walk starts from the
// Cartesian cell of the mesh description's origin and h (clamped to the
// grid), which is the right cell for a mesh that only perturbs the grid.
template <int D>
__global__ void locate64_k(D64Launch L, int64_t n0, int64_t n, int32_t *bad) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = n0 + q;
    double x[D], xi[D];
    int c[3] = {0, 0, 0};
    load_pos<D>(L, p, x);
    bool finite = true;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      finite = finite && isfinite(x[k]);
      const double s = finite ? floor((x[k] - L.origin[k]) / L.h) : 0.0;
      c[k] = s < 0.0 ? 0 : (s >= (double)L.nc[k] ? L.nc[k] - 1 : (int)s);
    }
    if (finite && iso::walk<D>(iso_grid(L), x, c, xi)) {
      L.P.cell[p] = iso::cell_id(iso_grid(L), c);
#pragma unroll
      for (int k = 0; k < D; ++k) L.P.xi[k][p] = xi[k];
    } else {
      atomicAdd(bad, 1);
    }
  }
}

template <int D, bool MAP>
cudaError_t step_dim(const D64Launch &L, cudaStream_t st) {
  const size_t nb = sizeof(double) * L.nnodes;
  const int gp = nblk(L.n), gn = nblk(L.nnodes);
  cudaMemsetAsync(L.N.m, 0, nb, st);
  for (int k = 0; k < D; ++k) {
    cudaMemsetAsync(L.N.P[k], 0, nb, st);
    cudaMemsetAsync(L.N.f[k], 0, nb, st);
  }
  if (L.scheme == 1) {
    p2g64<D, 0, MAP><<<gp, BS, 0, st>>>(L);
    node64<D, 1><<<gn, BS, 0, st>>>(L);
    g2p64<D, 0, MAP><<<gp, BS, 0, st>>>(L);
  } else {
    p2g64<D, 1, MAP><<<gp, BS, 0, st>>>(L);
    node64<D, 0><<<gn, BS, 0, st>>>(L);
    g2p64<D, 1, MAP><<<gp, BS, 0, st>>>(L);
    p2g64<D, 2, MAP><<<gp, BS, 0, st>>>(L);
    node64<D, 2><<<gn, BS, 0, st>>>(L);
    g2p64<D, 2, MAP><<<gp, BS, 0, st>>>(L);
  }
  return cudaGetLastError();
}

constexpr int CONS_BLOCKS = 1024;

template <int D>
__global__ void cons64_partial(D64Launch L, double *part) {
  constexpr int NS = nstress<D>();
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // mass, momentum (3), KE, SE, live count, volume
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < L.n; p += (int64_t)gridDim.x * blockDim.x) {
    if (!L.P.alive[p]) continue;
    const double m = L.P.mass[p];
    acc[0] += m;
    double ke = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const double v = L.P.v[k][p];
      acc[1 + k] += m * v;
      ke += v * v;
    }
    acc[4] += 0.5 * m * ke;
    double se = 0;
#pragma unroll
    for (int i = 0; i < NS; ++i) se += (i >= 3 ? 2.0 : 1.0) * L.P.sig[i][p] * L.P.eps[i][p];
    acc[5] += 0.5 * L.P.vol[p] * se;
    acc[6] += 1.0;
    acc[7] += L.P.vol[p];
  }
  __shared__ double red[8][256];
#pragma unroll
  for (int c = 0; c < 8; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int c = 0; c < 8; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 8) part[blockIdx.x * 8 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void cons64_final(const double *part, int nb, double *out) {
  if (threadIdx.x < 8) {
    double s = 0;
    for (int b = 0; b < nb; ++b) s += part[b * 8 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

__global__ void mat_update_f64_k(MatConst<double> m, int64_t n, const double *sig, const double *de,
                                 const double *coh, double *out, double *depsp) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s[6], d[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      s[k] = sig[i * 6 + k];
      d[k] = de[i * 6 + k];
    }
    double ep = 0.0;
    material_update(m, coh ? coh[i] : m.c, s, d, ep);
#pragma unroll
    for (int k = 0; k < 6; ++k) out[i * 6 + k] = s[k];
    if (depsp) depsp[i] = ep;
  }
}

}  // namespace

cudaError_t d64_step(const D64Launch &L, cudaStream_t st) {
  if (L.n <= 0) return cudaSuccess;
  if (L.X) return L.dim == 3 ? step_dim<3, true>(L, st) : step_dim<2, true>(L, st);
  return L.dim == 3 ? step_dim<3, false>(L, st) : step_dim<2, false>(L, st);
}

cudaError_t d64_locate(const D64Launch &L, int64_t n0, int64_t n, int32_t *bad, cudaStream_t st) {
  if (n <= 0 || !L.X) return cudaSuccess;
  if (L.dim == 3)
    locate64_k<3><<<nblk(n), BS, 0, st>>>(L, n0, n, bad);
  else
    locate64_k<2><<<nblk(n), BS, 0, st>>>(L, n0, n, bad);
  return cudaGetLastError();
}

cudaError_t d64_conservation(const D64Launch &L, double *d_out, double *d_partials, cudaStream_t st) {
  if (L.dim == 3)
    cons64_partial<3><<<CONS_BLOCKS, 256, 0, st>>>(L, d_partials);
  else
    cons64_partial<2><<<CONS_BLOCKS, 256, 0, st>>>(L, d_partials);
  cons64_final<<<1, 32, 0, st>>>(d_partials, CONS_BLOCKS, d_out);
  return cudaGetLastError();
}

cudaError_t material_update_f64(const MatConst<double> &m, int64_t n, const double *sig, const double *de,
                                const double *coh, double *out, double *depsp, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  mat_update_f64_k<<<nblk(n) > 4096 ? 4096 : nblk(n), BS, 0, st>>>(m, n, sig, de, coh, out, depsp);
  return cudaGetLastError();
}

}  // namespace mpm
