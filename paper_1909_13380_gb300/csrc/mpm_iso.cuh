// mpm_iso.cuh -- mapped (isoparametric) cells in FP64 (ISOPARAMETRIC MESH).
//
// A cell of a mapped mesh is the image of [-1, 1]^d under
// x(xi) = sum_a N_a(xi) X_a.  The natural coordinates of a point are the root
// of x(xi) = x in its cell: Newton-Raphson from the closed-form inverse
// bilinear solution (2D) or the affine guess (3D).  A point is placed in a
// cell by a neighbourhood walk from a starting cell.  Used by the FP64 step
// and by the initial location of particles on either path.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mpm_device.cuh"

namespace mpm {
namespace iso {

// A mapped mesh as the walk sees it: node coordinates (3 per node, node
// ix + (nx+1) (iy + (ny+1) iz)) and the cells per axis.
struct IsoGrid {
  const double *X;
  int nc[3];
};

// Coordinates of the 2^D nodes of cell c (node a: bit k = upper along k).
template <int D>
__device__ __forceinline__ void cell_xyz(const IsoGrid &L, const int c[3], double xa[1 << D][D]) {
  const int64_t nx = L.nc[0] + 1, ny = L.nc[1] + 1;
#pragma unroll
  for (int a = 0; a < (1 << D); ++a) {
    const int64_t i = (c[0] + (a & 1)) + nx * ((c[1] + ((a >> 1) & 1)) + ny * (D == 3 ? c[2] + ((a >> 2) & 1) : 0));
#pragma unroll
    for (int k = 0; k < D; ++k) xa[a][k] = L.X[3 * i + k];
  }
}

// x(xi) and J[j][k] = dx_j / dxi_k of the cell's map.
template <int D>
__device__ __forceinline__ void cell_map(const double xa[1 << D][D], const double xi[D], double x[D],
                                         double J[D][D]) {
  double N[1 << D], G[1 << D][D];
  shape_fn<D, double>(xi, 0.5, N, G);  // inv_h = 1/2: G = dN/dxi
#pragma unroll
  for (int j = 0; j < D; ++j) {
    x[j] = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) J[j][k] = 0.0;
  }
#pragma unroll
  for (int a = 0; a < (1 << D); ++a)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      x[j] += N[a] * xa[a][j];
#pragma unroll
      for (int k = 0; k < D; ++k) J[j][k] += xa[a][j] * G[a][k];
    }
}

// Ji = J^-1 by cofactors; false when J is singular (or not finite).
template <int D>
__device__ __forceinline__ bool invert(const double J[D][D], double Ji[D][D]) {
  if constexpr (D == 2) {
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    if (!(fabs(det) > 0.0) || !isfinite(det)) return false;
    const double r = 1.0 / det;
    Ji[0][0] = J[1][1] * r;
    Ji[0][1] = -J[0][1] * r;
    Ji[1][0] = -J[1][0] * r;
    Ji[1][1] = J[0][0] * r;
    return true;
  } else {
    double C[3][3];  // cofactors
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        C[i][j] = J[i1][j1] * J[i2][j2] - J[i1][j2] * J[i2][j1];
      }
    const double det = J[0][0] * C[0][0] + J[0][1] * C[0][1] + J[0][2] * C[0][2];
    if (!(fabs(det) > 0.0) || !isfinite(det)) return false;
    const double r = 1.0 / det;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Ji[i][j] = C[j][i] * r;  // adjugate / det
    return true;
  }
}

// The affine guess: the map linearised at the cell centre.
template <int D>
__device__ __forceinline__ bool affine_guess(const double xa[1 << D][D], const double x[D], double xi[D]) {
  double x0[D], J[D][D], Ji[D][D];
#pragma unroll
  for (int k = 0; k < D; ++k) xi[k] = 0.0;
  cell_map<D>(xa, xi, x0, J);
  if (!invert<D>(J, Ji)) return false;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) s += Ji[j][k] * (x[k] - x0[k]);
    xi[j] = s;
  }
  return true;
}

// 2D: the inverse of the bilinear map in closed form.  With
// x = b0 + b1 xi + b2 eta + b3 xi eta, crossing x - b0 - b2 eta with
// b1 + b3 eta leaves A eta^2 + B eta + C = 0; the root nearer the cell is
// taken (the stable form of the quadratic formula) and xi follows by
// projection.  False when no real root exists (far outside the cell).
__device__ __forceinline__ bool inverse_bilinear(const double xa[4][2], const double x[2], double xi[2]) {
  double b0[2], b1[2], b2[2], b3[2], d[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    b0[k] = 0.25 * ((xa[0][k] + xa[1][k]) + (xa[2][k] + xa[3][k]));
    b1[k] = 0.25 * ((xa[1][k] - xa[0][k]) + (xa[3][k] - xa[2][k]));
    b2[k] = 0.25 * ((xa[2][k] - xa[0][k]) + (xa[3][k] - xa[1][k]));
    b3[k] = 0.25 * ((xa[0][k] - xa[1][k]) + (xa[3][k] - xa[2][k]));
    d[k] = x[k] - b0[k];
  }
  auto cross = [](const double *u, const double *v) { return u[0] * v[1] - u[1] * v[0]; };
  const double A = cross(b3, b2), B = cross(d, b3) + cross(b1, b2), C = cross(d, b1);
  double eta;
  if (fabs(A) <= 1e-13 * fabs(B)) {
    if (B == 0.0) return false;
    eta = -C / B;
  } else {
    const double disc = B * B - 4.0 * A * C;
    if (!(disc >= 0.0)) return false;
    const double q = -0.5 * (B + copysign(sqrt(disc), B));
    const double r1 = q / A, r2 = q != 0.0 ? C / q : r1;
    eta = fabs(r1) < fabs(r2) ? r1 : r2;
  }
  const double u[2] = {b1[0] + b3[0] * eta, b1[1] + b3[1] * eta};
  const double uu = u[0] * u[0] + u[1] * u[1];
  if (!(uu > 0.0)) return false;
  xi[0] = ((d[0] - b2[0] * eta) * u[0] + (d[1] - b2[1] * eta) * u[1]) / uu;
  xi[1] = eta;
  return isfinite(xi[0]) && isfinite(xi[1]);
}

// Natural coordinates of x in a cell: Newton-Raphson on x(xi) = x from the
// inverse bilinear solution (2D) or the affine guess (3D), until a step
// falls below 1e-12 and one more has been taken.  False if it does not
// converge; xi then holds the starting guess.
template <int D>
__device__ __forceinline__ bool natural(const double xa[1 << D][D], const double x[D], double xi[D]) {
  bool ok;
  if constexpr (D == 2)
    ok = inverse_bilinear(xa, x, xi) || affine_guess<D>(xa, x, xi);
  else
    ok = affine_guess<D>(xa, x, xi);
  if (!ok) return false;
  double x0[D];
#pragma unroll
  for (int k = 0; k < D; ++k) x0[k] = xi[k];
  bool polish = false;
  for (int it = 0; it < 40; ++it) {
    double xm[D], J[D][D], Ji[D][D];
    cell_map<D>(xa, xi, xm, J);
    if (!invert<D>(J, Ji)) break;
    double step = 0.0;
    double r[D];
#pragma unroll
    for (int k = 0; k < D; ++k) r[k] = xm[k] - x[k];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double dj = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) dj += Ji[j][k] * r[k];
      xi[j] -= dj;
      step = fmax(step, fabs(dj));
    }
    if (!isfinite(step)) break;
    if (step < 1e-12) {
      if (polish) return true;
      polish = true;
    }
  }
#pragma unroll
  for (int k = 0; k < D; ++k) xi[k] = x0[k];
  return false;
}

// The cell of x by a neighbourhood walk from c (updated): while the affine
// guess lies far outside the current cell (beyond [-2, 2]) it gives the
// direction, nearer the Newton root does; the walk steps to the neighbour
// across the face of the largest excess over [-1, 1), or of the next
// largest when that neighbour is beyond the grid.  xi = 1 belongs to the
// next cell.  False when the point is outside the mesh.
template <int D>
__device__ bool walk(const IsoGrid &L, const double x[D], int c[3], double xi[D]) {
  const int limit = 2 * (L.nc[0] + L.nc[1] + (D == 3 ? L.nc[2] : 0)) + 8;
  for (int s = 0; s < limit; ++s) {
    double xa[1 << D][D];
    cell_xyz<D>(L, c, xa);
    if (!affine_guess<D>(xa, x, xi)) return false;
    bool near = true;
#pragma unroll
    for (int k = 0; k < D; ++k) near = near && fabs(xi[k]) <= 2.0;
    const bool conv = near && natural<D>(xa, x, xi);
    double ex[D];
    bool inside = true;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      ex[k] = xi[k] < -1.0 ? -1.0 - xi[k] : (xi[k] >= 1.0 ? xi[k] - 1.0 : -1.0);
      inside = inside && ex[k] < 0.0;
    }
    if (inside) return conv;
    bool moved = false;
    for (int t = 0; t < D && !moved; ++t) {
      int best = -1;
#pragma unroll
      for (int k = 0; k < D; ++k)
        if (ex[k] >= 0.0 && (best < 0 || ex[k] > ex[best])) best = k;
      if (best < 0) break;
      const int nb = c[best] + (xi[best] < -1.0 ? -1 : 1);
      if (nb >= 0 && nb < L.nc[best]) {
        c[best] = nb;
        moved = true;
      } else {
        ex[best] = -1.0;
      }
    }
    if (!moved) return false;
  }
  return false;
}

__device__ __forceinline__ void cell_split(const IsoGrid &L, int32_t id, int c[3]) {
  c[0] = id % L.nc[0];
  c[1] = (id / L.nc[0]) % L.nc[1];
  c[2] = id / (L.nc[0] * L.nc[1]);
}

__device__ __forceinline__ int32_t cell_id(const IsoGrid &L, const int c[3]) {
  return c[0] + L.nc[0] * (c[1] + L.nc[1] * c[2]);
}

}  // namespace iso
}  // namespace mpm
