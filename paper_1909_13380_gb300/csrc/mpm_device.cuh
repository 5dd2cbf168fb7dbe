// mpm_device.cuh -- device-side arithmetic of one explicit MPM step shared by
// the FP64 plain kernels and the FP32 mixed kernels: linear quad/hex shape
// functions, nodal boundary conditions, and the material update
// (linear elastic, Mohr-Coulomb return in principal stresses).
//
// Paper: Kumar et al., arXiv 1909.13380.  CODE OVERVIEW names the linear
// 4-node quadrilateral / 8-node hexahedron, the Node with persistent
// friction/velocity constraints, and the Material that returns the stress
// for a strain increment; ISOPARAMETRIC MESH applies velocity and frictional
// (acceleration) conditions at the nodes.  The equations are the textbook
// explicit MPM (Sulsky et al. 1994) and the de Souza Neto et al. (2008)
// principal-space Mohr-Coulomb return.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mpm {

enum { BC_FREE = 0, BC_ROLLER = 1, BC_FIXED = 2, BC_FRICTION = 3 };
enum { ST_LEFT_MESH = 1, ST_NONFINITE = 2, ST_TIMEOUT = 4 };

// ---------------------------------------------------------------------------
// Material constants, precomputed on the host.
// ---------------------------------------------------------------------------
template <typename T>
struct MatConst {
  int model;          // 0 linear elastic, 1 Mohr-Coulomb, 2 plane-stress linear elastic (2D)
  T E, nu, G, lam;    // elastic constants (plane stress: lam = 2 lambda G / (lambda + 2 G))
  T sphi, cphi, spsi; // sin(phi), cos(phi), sin(psi)
  T c;                // cohesion (default when no per-particle value)
};

// ---------------------------------------------------------------------------
// Compensated summation: Knuth's TwoSum keeps the rounding error of every
// addition in a second float ("two-float" accumulator).
// ---------------------------------------------------------------------------
template <typename T>
struct TwoAcc {
  T hi, lo;
  __device__ __forceinline__ void init() { hi = T(0); lo = T(0); }
  __device__ __forceinline__ void add(T x) {
    T s = hi + x;
    T bp = s - hi;
    T err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
  }
  __device__ __forceinline__ T value() const { return hi + lo; }
};

// ---------------------------------------------------------------------------
// Shape functions of the linear element in natural coordinates xi in
// [-1,1]^D.  Local node a has xi^a_k = +1 when bit k of a is set (x fastest):
//   N_a = prod_k (1 + xi_k xi^a_k)/2,
//   dN_a/dx_k = (xi^a_k / h) prod_{j!=k} (1 + xi_j xi^a_j)/2.
// ---------------------------------------------------------------------------
template <int D, typename T>
__device__ __forceinline__ void shape_fn(const T xi[D], T inv_h, T N[1 << D], T G[1 << D][D]) {
  T wl[D], wh[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    wl[k] = T(0.5) * (T(1) - xi[k]);
    wh[k] = T(0.5) * (T(1) + xi[k]);
  }
#pragma unroll
  for (int a = 0; a < (1 << D); ++a) {
    T w[D];
#pragma unroll
    for (int k = 0; k < D; ++k) w[k] = ((a >> k) & 1) ? wh[k] : wl[k];
    T n = w[0];
#pragma unroll
    for (int k = 1; k < D; ++k) n *= w[k];
    N[a] = n;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      T g = ((a >> k) & 1) ? inv_h : -inv_h;
#pragma unroll
      for (int j = 0; j < D; ++j)
        if (j != k) g *= w[j];
      G[a][k] = g;
    }
  }
}

// ---------------------------------------------------------------------------
// Nodal boundary conditions.  `faces` has bit f set when the node lies on
// face f (-x,+x,-y,+y,-z,+z).  Fixed faces zero every component; roller
// faces zero the face-normal component; a friction face acts only while the
// node moves into it (w = outward . v' > 0): the normal component of v'
// becomes 0 and the tangential part shrinks by mu*w (to 0 when it is not
// larger: stick); the acceleration of the node is then reset to
// (v' - v)/dt so that v' = v + a dt keeps holding.
// ---------------------------------------------------------------------------
template <int D, typename T>
__device__ __forceinline__ void bc_velocity(int faces, const int *bc, T v[D]) {
#pragma unroll
  for (int f = 0; f < 2 * D; ++f)
    if (((faces >> f) & 1) && bc[f] == BC_FIXED) {
#pragma unroll
      for (int k = 0; k < D; ++k) v[k] = T(0);
      return;
    }
#pragma unroll
  for (int f = 0; f < 2 * D; ++f) {
    if (!((faces >> f) & 1)) continue;
    const int k = f >> 1;
    const T out = (f & 1) ? T(1) : T(-1);
    if (bc[f] == BC_ROLLER) v[k] = T(0);
    if (bc[f] == BC_FRICTION && out * v[k] > T(0)) v[k] = T(0);
  }
}

template <int D, typename T>
__device__ __forceinline__ void bc_full(int faces, const int *bc, const T *mu, T dt, T v[D], T a[D],
                                        T vn[D]) {
#pragma unroll
  for (int f = 0; f < 2 * D; ++f)
    if (((faces >> f) & 1) && bc[f] == BC_FIXED) {
#pragma unroll
      for (int k = 0; k < D; ++k) v[k] = a[k] = vn[k] = T(0);
      return;
    }
#pragma unroll
  for (int f = 0; f < 2 * D; ++f)
    if (((faces >> f) & 1) && bc[f] == BC_ROLLER) {
      const int k = f >> 1;
#pragma unroll
      for (int j = 0; j < D; ++j)
        if (j == k) v[j] = a[j] = vn[j] = T(0);
    }
#pragma unroll
  for (int f = 0; f < 2 * D; ++f) {
    if (!(((faces >> f) & 1) && bc[f] == BC_FRICTION)) continue;
    const int k = f >> 1;
    const T out = (f & 1) ? T(1) : T(-1);
    T w = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j)
      if (j == k) w = out * vn[j];
    if (!(w > T(0))) continue;
    T t2 = T(0);
#pragma unroll
    for (int j = 0; j < D; ++j)
      if (j != k) t2 += vn[j] * vn[j];
    const T tn = sqrt(t2);
    const T cap = mu[f] * w;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      if (j == k)
        vn[j] = T(0);
      else
        vn[j] = (tn <= cap) ? T(0) : vn[j] - cap * vn[j] / tn;
    }
#pragma unroll
    for (int j = 0; j < D; ++j) a[j] = (vn[j] - v[j]) / dt;
  }
}

// The same conditions on a node of a mapped mesh (ISOPARAMETRIC MESH: nodal
// conditions on irregular surfaces): nrm[f] is the outward unit normal of
// face f at the node (read only for the node's faces).  A roller removes the
// velocity along the roller normals, made orthonormal in face order; a
// friction face acts on w = n . v' and on the part of v' tangent to n.  With
// n = +-e_k these are the axis rules above.  Products and sums are written
// as explicit FMAs, so every kernel that inlines them (a mesh alone or in a
// batch) rounds them alike.
template <int D, typename T>
__device__ __forceinline__ T dotn(const T a[D], const T b[D]) {
  T s = T(0);
#pragma unroll
  for (int k = 0; k < D; ++k) s = fma(a[k], b[k], s);
  return s;
}

template <int D, typename T>
__device__ __forceinline__ int roller_basis_n(int faces, const int *bc, const T nrm[6][3], T B[D][D]) {
  int nb = 0;
#pragma unroll
  for (int f = 0; f < 2 * D; ++f) {
    if (!(((faces >> f) & 1) && bc[f] == BC_ROLLER)) continue;
    T n[D];
#pragma unroll
    for (int k = 0; k < D; ++k) n[k] = nrm[f][k];
#pragma unroll
    for (int b = 0; b < D; ++b)
      if (b < nb) {
        const T d = dotn<D, T>(n, B[b]);
#pragma unroll
        for (int k = 0; k < D; ++k) n[k] = fma(-d, B[b][k], n[k]);
      }
    const T len = sqrt(dotn<D, T>(n, n));
    if (!(len > T(1e-6))) continue;  // along an earlier roller normal
#pragma unroll
    for (int b = 0; b < D; ++b)
      if (b == nb)
#pragma unroll
        for (int k = 0; k < D; ++k) B[b][k] = n[k] / len;
    ++nb;
  }
  return nb;
}

template <int D, typename T>
__device__ __forceinline__ void bc_velocity_n(int faces, const int *bc, const T nrm[6][3], T v[D]) {
#pragma unroll
  for (int f = 0; f < 2 * D; ++f)
    if (((faces >> f) & 1) && bc[f] == BC_FIXED) {
#pragma unroll
      for (int k = 0; k < D; ++k) v[k] = T(0);
      return;
    }
  T B[D][D];
  const int nb = roller_basis_n<D, T>(faces, bc, nrm, B);
#pragma unroll
  for (int b = 0; b < D; ++b)
    if (b < nb) {
      const T d = dotn<D, T>(v, B[b]);
#pragma unroll
      for (int k = 0; k < D; ++k) v[k] = fma(-d, B[b][k], v[k]);
    }
#pragma unroll
  for (int f = 0; f < 2 * D; ++f) {
    if (!(((faces >> f) & 1) && bc[f] == BC_FRICTION)) continue;
    const T w = dotn<D, T>(v, nrm[f]);
    if (w > T(0))
#pragma unroll
      for (int k = 0; k < D; ++k) v[k] = fma(-w, nrm[f][k], v[k]);
  }
}

template <int D, typename T>
__device__ __forceinline__ void bc_full_n(int faces, const int *bc, const T *mu, T dt, const T nrm[6][3], T v[D],
                                          T a[D], T vn[D]) {
#pragma unroll
  for (int f = 0; f < 2 * D; ++f)
    if (((faces >> f) & 1) && bc[f] == BC_FIXED) {
#pragma unroll
      for (int k = 0; k < D; ++k) v[k] = a[k] = vn[k] = T(0);
      return;
    }
  T B[D][D];
  const int nb = roller_basis_n<D, T>(faces, bc, nrm, B);
#pragma unroll
  for (int b = 0; b < D; ++b)
    if (b < nb) {
      const T dv = dotn<D, T>(v, B[b]), da = dotn<D, T>(a, B[b]), dn = dotn<D, T>(vn, B[b]);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        v[k] = fma(-dv, B[b][k], v[k]);
        a[k] = fma(-da, B[b][k], a[k]);
        vn[k] = fma(-dn, B[b][k], vn[k]);
      }
    }
#pragma unroll
  for (int f = 0; f < 2 * D; ++f) {
    if (!(((faces >> f) & 1) && bc[f] == BC_FRICTION)) continue;
    const T w = dotn<D, T>(vn, nrm[f]);
    if (!(w > T(0))) continue;
#pragma unroll
    for (int k = 0; k < D; ++k) vn[k] = fma(-w, nrm[f][k], vn[k]);
    const T tn = sqrt(dotn<D, T>(vn, vn));
    const T cap = mu[f] * w;
#pragma unroll
    for (int k = 0; k < D; ++k) vn[k] = (tn <= cap) ? T(0) : vn[k] - cap * vn[k] / tn;
#pragma unroll
    for (int k = 0; k < D; ++k) a[k] = (vn[k] - v[k]) / dt;
  }
}

// Index of node I within the table of face f: its indices along the face's
// other axes in increasing axis order (nc: cells per axis).
template <int D>
__device__ __forceinline__ int64_t face_node_index(int f, const int I[3], const int nc[3]) {
  const int k = f >> 1;
  if (D == 2) return I[1 - k];
  const int t1 = k == 0 ? 1 : 0, t2 = k == 2 ? 1 : 2;
  return (int64_t)I[t1] + (int64_t)(nc[t1] + 1) * I[t2];
}

// ---------------------------------------------------------------------------
// Explicitly rounded operations for the FP32 material update.  Whether the
// compiler contracts a product and a sum into one FMA depends on the code
// around them, so the same source, inlined into two kernels (a mesh stepped
// alone, and in a batch), could round differently.  Written with explicit
// round-to-nearest operations -- never contracted or reassociated -- the
// FP32 material update rounds the same way in every kernel.  The FP64
// overloads are the plain operators: the FP64 plain step runs one mesh at a
// time, and the FP64 apex-band return is one out-of-line function, so each
// is compiled once, and the FP64 pipe keeps its fused multiply-adds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float xm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double xm(double a, double b) { return a * b; }
__device__ __forceinline__ float xa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double xa(double a, double b) { return a + b; }
__device__ __forceinline__ float xs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double xs(double a, double b) { return a - b; }
__device__ __forceinline__ float xf(float a, float b, float c) { return __fmaf_rn(a, b, c); }  // a b + c
__device__ __forceinline__ double xf(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float xd(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double xd(double a, double b) { return a / b; }
__device__ __forceinline__ float xsqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double xsqrt(double a) { return sqrt(a); }
// a b + c d + e f, and the dot product of two 3-vectors
template <typename T>
__device__ __forceinline__ T xdot3(T a, T b, T c, T d, T e, T f) {
  return xf(e, f, xf(c, d, xm(a, b)));
}

// ---------------------------------------------------------------------------
// Loads of a quasi-static run (the plate with a hole of BENCHMARK AND
// PERFORMANCE: uniform tension at the ends of a plane-stress strip).  A
// uniform traction on an end of the body acts as forces on the nodes of the
// mesh face that coincides with it: for every face f the node lies on,
// traction_f times the node's tributary length (area in 3D), h per tangent
// axis and h / 2 at the face's own edges.  The explicit run is brought to
// rest by mass-proportional viscous damping, a = f / m - alpha v.
// ---------------------------------------------------------------------------
template <int D, typename T>
__device__ __forceinline__ void face_force(int faces, const int I[3], const int nc[3], T h, const T (*trac)[3],
                                           T ft[D]) {
#pragma unroll
  for (int k = 0; k < D; ++k) ft[k] = T(0);
#pragma unroll
  for (int f = 0; f < 2 * D; ++f) {
    if (!((faces >> f) & 1)) continue;
    T trib = T(1);
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (k != f / 2) trib *= (I[k] == 0 || I[k] == nc[k]) ? T(0.5) * h : h;
#pragma unroll
    for (int k = 0; k < D; ++k) ft[k] += trac[f][k] * trib;
  }
}

// ---------------------------------------------------------------------------
// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (Golub & Van
// Loan, symmetric Schur decomposition).  A is overwritten (diagonal ->
// eigenvalues), Q accumulates the eigenvectors as columns.
// ---------------------------------------------------------------------------
template <typename T, int p, int q>
__device__ __forceinline__ void jacobi_rot(T A[3][3], T Q[3][3]) {
  constexpr int o = 3 - p - q;
  const T apq = A[p][q];
  if (apq == T(0)) return;
  const T theta = xd(xs(A[q][q], A[p][p]), xm(T(2), apq));
  const T t = xd(theta >= T(0) ? T(1) : T(-1), xa(fabs(theta), xsqrt(xf(theta, theta, T(1)))));
  // any c, s with c^2 + s^2 = 1 keep Q orthogonal; rsqrt is exact enough here
  const T c = sizeof(T) == 4 ? (T)rsqrtf((float)xf(t, t, T(1))) : xd(T(1), xsqrt(xf(t, t, T(1))));
  const T s = xm(t, c);
  const T aop = A[o][p], aoq = A[o][q];
  A[p][p] = xs(A[p][p], xm(t, apq));
  A[q][q] = xa(A[q][q], xm(t, apq));
  A[p][q] = A[q][p] = T(0);
  A[o][p] = A[p][o] = xs(xm(c, aop), xm(s, aoq));
  A[o][q] = A[q][o] = xa(xm(s, aop), xm(c, aoq));
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const T vp = Q[r][p], vq = Q[r][q];
    Q[r][p] = xs(xm(c, vp), xm(s, vq));
    Q[r][q] = xa(xm(s, vp), xm(c, vq));
  }
}

template <typename T>
__device__ __forceinline__ void eig_sym3(const T s[6], T lam[3], T Q[3][3]) {
  T A[3][3] = {{s[0], s[3], s[5]}, {s[3], s[1], s[4]}, {s[5], s[4], s[2]}};
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) Q[r][c] = (r == c) ? T(1) : T(0);
  // stop when the off-diagonal mass is below (1e-6)^2 (FP32) or (1e-16)^2
  // (FP64) of the diagonal; Jacobi converges quadratically, so the sweep
  // that crosses the bound leaves far less in practice
  const T tol = sizeof(T) == 4 ? T(1e-12) : T(1e-32);
  for (int sweep = 0; sweep < (sizeof(T) == 4 ? 6 : 20); ++sweep) {
    const T off = xdot3(A[0][1], A[0][1], A[0][2], A[0][2], A[1][2], A[1][2]);
    const T dia = xdot3(A[0][0], A[0][0], A[1][1], A[1][1], A[2][2], A[2][2]);
    if (off <= xm(tol, dia) || off == T(0)) break;
    jacobi_rot<T, 0, 1>(A, Q);
    jacobi_rot<T, 0, 2>(A, Q);
    jacobi_rot<T, 1, 2>(A, Q);
  }
  lam[0] = A[0][0];
  lam[1] = A[1][1];
  lam[2] = A[2][2];
}

// Mean stress p, deviator diagonal d, and J2 of a Voigt stress.
__device__ __forceinline__ void mean_dev_j2(const float s[6], float &p, float d[3], float &j2) {
  p = xm(xa(xa(s[0], s[1]), s[2]), 1.f / 3.f);
  d[0] = xs(s[0], p);
  d[1] = xs(s[1], p);
  d[2] = xs(s[2], p);
  j2 = xf(s[5], s[5], xf(s[4], s[4], xf(s[3], s[3], xm(0.5f, xdot3(d[0], d[0], d[1], d[1], d[2], d[2])))));
}

// Symmetric 3x3 eigen-decomposition in closed form with deflation (FP32).
// Work on the normalised deviator A = (s - p I) / r, r = sqrt(J2 / 3), whose
// eigenvalues are 2 cos(theta + 2 pi k / 3), cos(3 theta) = det(A) / 2.  Of
// the largest and the smallest, take the one farther from the middle value:
// its gap to both others is at least sqrt(3) / 2, so it is insensitive to the
// error of the arc-cosine (a stationary point of the cosine where the other
// two meet) and its eigenvector, the cross product of two rows of A - mu I
// (the pair of largest norm), is well conditioned.  The remaining pair is the
// 2x2 problem in the plane orthogonal to that vector, solved by one exact
// rotation (stable tangent formula), which keeps a near-double pair accurate.
// Eigenvalues come back as p + r mu, eigenvectors as the columns of Q.
__device__ __forceinline__ void eig_sym3_closed(const float s[6], float lam[3], float Q[3][3]) {
  float p, dv[3], j2;
  mean_dev_j2(s, p, dv, j2);
  if (!(j2 > 1e-30f)) {  // isotropic (or a deviator below any stress of interest)
    lam[0] = s[0];
    lam[1] = s[1];
    lam[2] = s[2];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) Q[r][c] = (r == c) ? 1.f : 0.f;
    return;
  }
  const float r = xsqrt(xm(j2, 1.f / 3.f));
  const float ir = xd(1.f, r);
  const float A[3][3] = {{xm(dv[0], ir), xm(s[3], ir), xm(s[5], ir)},
                         {xm(s[3], ir), xm(dv[1], ir), xm(s[4], ir)},
                         {xm(s[5], ir), xm(s[4], ir), xm(dv[2], ir)}};
  const float m0 = xs(xm(A[1][1], A[2][2]), xm(A[1][2], A[1][2]));
  const float m1 = xs(xm(A[0][1], A[2][2]), xm(A[1][2], A[0][2]));
  const float m2 = xs(xm(A[0][1], A[1][2]), xm(A[1][1], A[0][2]));
  const float det = xa(xs(xm(A[0][0], m0), xm(A[0][1], m1)), xm(A[0][2], m2));
  const float c3 = fminf(1.f, fmaxf(-1.f, xm(0.5f, det)));
  const float th = xm(acosf(c3), 1.f / 3.f);
  float sn, cs;
  sincosf(th, &sn, &cs);
  const float sq3 = 1.7320508f;
  const float mu1 = xm(2.f, cs), mu3 = xs(-cs, xm(sq3, sn)), mu2 = xa(-cs, xm(sq3, sn));
  const float mud0 = (xs(mu1, mu2) >= xs(mu2, mu3)) ? mu1 : mu3;
  // eigenvector of the distinct value: largest cross product of two rows
  float R[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) R[i][j] = i == j ? xs(A[i][j], mud0) : A[i][j];
  float n[3], best = -1.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int a = k == 2 ? 1 : 0, b = k == 0 ? 1 : 2;  // row pairs (0,1) (0,2) (1,2)
    const float cx = xs(xm(R[a][1], R[b][2]), xm(R[a][2], R[b][1]));
    const float cy = xs(xm(R[a][2], R[b][0]), xm(R[a][0], R[b][2]));
    const float cz = xs(xm(R[a][0], R[b][1]), xm(R[a][1], R[b][0]));
    const float m2c = xdot3(cx, cx, cy, cy, cz, cz);
    if (m2c > best) {
      best = m2c;
      n[0] = cx;
      n[1] = cy;
      n[2] = cz;
    }
  }
  if (!(best > 1e-30f)) {  // cannot happen for a rank-2 A - mu I; keep the iterative solver as a guard
    eig_sym3<float>(s, lam, Q);
    return;
  }
  const float inr = rsqrtf(best);
  n[0] = xm(n[0], inr);
  n[1] = xm(n[1], inr);
  n[2] = xm(n[2], inr);
  // orthonormal basis e1, e2 of the plane orthogonal to n
  float e1[3];
  if (fabsf(n[0]) >= fabsf(n[1])) {
    const float k = rsqrtf(xf(n[2], n[2], xm(n[0], n[0])));
    e1[0] = xm(-n[2], k);
    e1[1] = 0.f;
    e1[2] = xm(n[0], k);
  } else {
    const float k = rsqrtf(xf(n[2], n[2], xm(n[1], n[1])));
    e1[0] = 0.f;
    e1[1] = xm(n[2], k);
    e1[2] = xm(-n[1], k);
  }
  const float e2[3] = {xs(xm(n[1], e1[2]), xm(n[2], e1[1])), xs(xm(n[2], e1[0]), xm(n[0], e1[2])),
                       xs(xm(n[0], e1[1]), xm(n[1], e1[0]))};
  float An[3], A1[3], A2[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    An[i] = xdot3(A[i][0], n[0], A[i][1], n[1], A[i][2], n[2]);
    A1[i] = xdot3(A[i][0], e1[0], A[i][1], e1[1], A[i][2], e1[2]);
    A2[i] = xdot3(A[i][0], e2[0], A[i][1], e2[1], A[i][2], e2[2]);
  }
  const float mud = xdot3(n[0], An[0], n[1], An[1], n[2], An[2]);  // Rayleigh quotient
  const float b11 = xdot3(e1[0], A1[0], e1[1], A1[1], e1[2], A1[2]);
  const float b22 = xdot3(e2[0], A2[0], e2[1], A2[1], e2[2], A2[2]);
  const float b12 = xdot3(e1[0], A2[0], e1[1], A2[1], e1[2], A2[2]);
  float t = 0.f;
  if (b12 != 0.f) {
    const float tj = xd(xs(b22, b11), xm(2.f, b12));
    t = xd(tj >= 0.f ? 1.f : -1.f, xa(fabsf(tj), xsqrt(xf(tj, tj, 1.f))));
  }
  const float c = rsqrtf(xf(t, t, 1.f)), sr = xm(t, c);
  lam[0] = xf(r, mud, p);
  lam[1] = xf(r, xs(b11, xm(t, b12)), p);
  lam[2] = xf(r, xf(t, b12, b22), p);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Q[i][0] = n[i];
    Q[i][1] = xs(xm(c, e1[i]), xm(sr, e2[i]));
    Q[i][2] = xa(xm(sr, e1[i]), xm(c, e2[i]));
  }
}

// Principal stresses sorted s1 >= s2 >= s3 with their eigenvector columns
// (stable for ties: a swap only when strictly smaller).
template <typename T>
__device__ __forceinline__ void sort3_desc(T lam[3], T Q[3][3]) {
  auto sw = [&](int i, int j) {
    if (lam[i] < lam[j]) {
      T t = lam[i];
      lam[i] = lam[j];
      lam[j] = t;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        T u = Q[r][i];
        Q[r][i] = Q[r][j];
        Q[r][j] = u;
      }
    }
  };
  sw(0, 1);
  sw(1, 2);
  sw(0, 1);
}

// The Mohr-Coulomb function of a pair of principal stresses a >= b:
// (a - b) + (a + b) sin(phi) - 2 c cos(phi).
template <typename T>
__device__ __forceinline__ T mc_f(const MatConst<T> &m, T c, T a, T b) {
  return xs(xf(xa(a, b), m.sphi, xs(a, b)), xm(xm(T(2), c), m.cphi));
}

// Mohr-Coulomb return in principal stresses (tension positive, perfect
// plasticity): yield f = (s1 - s3) + (s1 + s3) sin(phi) - 2 c cos(phi);
// plastic potential of the same form with psi.  Order of de Souza Neto et
// al. (2008, Box 8.5): main plane; if the ordering s1 >= s2 >= s3 breaks,
// the edge where the first gap closes (s1 = s2 or s2 = s3) with both planes
// active; if that edge passes the apex, the apex c cot(phi).  Returns the
// branch (0 elastic, 1 plane, 2 edge s1 = s2, 3 edge s2 = s3, 4 apex),
// writes the principal results r[] and the equivalent plastic strain
// increment sqrt(2/3 |C (s_trial - s)|^2).
template <typename T>
__device__ __forceinline__ int mc_principal(const MatConst<T> &m, T c, const T s[3], T r[3],
                                            T &depsp) {
  const T f13 = mc_f(m, c, s[0], s[2]);
  if (!(f13 > T(0))) {
    r[0] = s[0];
    r[1] = s[1];
    r[2] = s[2];
    depsp = T(0);
    return 0;
  }
  const T G2 = xm(T(2), m.G);
  const T l2 = xm(xm(T(2), m.lam), m.spsi);
  const T up = xm(G2, xa(T(1), m.spsi)), dn = xm(G2, xs(T(1), m.spsi));
  // D N for the planes 1-3 (a), 2-3 (b), 1-2 (c)
  const T DNa[3] = {xa(l2, up), l2, xs(l2, dn)};
  const T DNb[3] = {l2, xa(l2, up), xs(l2, dn)};
  const T DNc[3] = {xa(l2, up), xs(l2, dn), l2};
  const T ll = xm(xm(xm(T(4), m.lam), m.sphi), m.spsi);
  const T a = xf(xm(T(4), m.G), xf(m.sphi, m.spsi, T(1)), ll);
  int branch = 1;
  const T g = xd(f13, a);
#pragma unroll
  for (int i = 0; i < 3; ++i) r[i] = xs(s[i], xm(g, DNa[i]));
  if (!(r[0] >= r[1] && r[1] >= r[2])) {
    const T crit = xs(xm(xs(T(1), m.spsi), xs(s[0], s[1])), xm(xa(T(1), m.spsi), xs(s[1], s[2])));
    if (crit <= T(0)) {
      const T fb = mc_f(m, c, s[1], s[2]);
      const T b = xf(xm(G2, xs(T(1), m.sphi)), xs(T(1), m.spsi), ll);
      const T det = xs(xm(a, a), xm(b, b));
      const T ga = xd(xs(xm(a, f13), xm(b, fb)), det), gb = xd(xs(xm(a, fb), xm(b, f13)), det);
#pragma unroll
      for (int i = 0; i < 3; ++i) r[i] = xs(xs(s[i], xm(ga, DNa[i])), xm(gb, DNb[i]));
      branch = 2;
    } else {
      const T fc = mc_f(m, c, s[0], s[1]);
      const T b = xf(xm(G2, xa(T(1), m.sphi)), xa(T(1), m.spsi), ll);
      const T det = xs(xm(a, a), xm(b, b));
      const T ga = xd(xs(xm(a, f13), xm(b, fc)), det), gc = xd(xs(xm(a, fc), xm(b, f13)), det);
#pragma unroll
      for (int i = 0; i < 3; ++i) r[i] = xs(xs(s[i], xm(ga, DNa[i])), xm(gc, DNc[i]));
      branch = 3;
    }
    if (m.sphi > T(0) && !(r[0] >= r[2])) {
      branch = 4;
      const T pa = xd(xm(c, m.cphi), m.sphi);
      r[0] = r[1] = r[2] = pa;
    }
  }
  T sq = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T d0 = xs(s[i], r[i]), d1 = xs(s[(i + 1) % 3], r[(i + 1) % 3]), d2 = xs(s[(i + 2) % 3], r[(i + 2) % 3]);
    const T e = xd(xs(d0, xm(m.nu, xa(d1, d2))), m.E);
    sq = xf(e, e, sq);
  }
  depsp = xsqrt(xm(T(2) / T(3), sq));
  return branch;
}

// Clearly inside the yield surface?  Principal stresses from the closed form
// of a symmetric 3x3 (mean p, J2, J3 and the Lode angle: s_k = p + 2 sqrt(J2/3)
// cos(theta - 2 pi k / 3)), then the yield function with a margin larger than
// the error of that form in FP32 (worst near repeated eigenvalues, where the
// arc-cosine loses about half the digits).  Only a cheap filter: a trial that
// is not clearly elastic goes through the full return (accurate eigenpairs,
// then the yield check), so the result is the same as without the filter.
__device__ __forceinline__ bool clearly_elastic(const MatConst<float> &m, float c, const float s[6]) {
  float p, d[3], j2;
  mean_dev_j2(s, p, d, j2);
  const float j3 = xa(xs(xm(d[0], xs(xm(d[1], d[2]), xm(s[4], s[4]))), xm(s[3], xs(xm(s[3], d[2]), xm(s[4], s[5])))),
                      xm(s[5], xs(xm(s[3], s[4]), xm(d[1], s[5]))));
  const float r = xsqrt(xm(j2, 1.f / 3.f));
  float c3 = r > 0.f ? xd(j3, xm(xm(xm(2.f, r), r), r)) : 0.f;
  c3 = fminf(1.f, fmaxf(-1.f, c3));
  const float th = xm(acosf(c3), 1.f / 3.f);
  const float r2 = xm(2.f, r);
  const float s1 = xf(r2, cosf(th), p);
  const float s3 = xf(r2, cosf(xa(th, 2.0943951f)), p);
  const float f = mc_f(m, c, s1, s3);
  const float margin = xf(1e-3f, c, xm(4e-3f, xa(r, fabsf(p))));
  return f < -margin;
}

// Elastic for certain, without trigonometry?  With the principal deviatoric
// stresses 2 r cos(theta + 2 pi k / 3), r = sqrt(J2 / 3), the yield function
// is f = 2 r (sqrt(3) sin(psi) + sin(phi) cos(psi)) + 2 p sin(phi)
// - 2 c cos(phi) with psi = theta + pi / 3, and over every Lode angle
// sqrt(3) sin(psi) + sin(phi) cos(psi) <= sqrt(3 + sin^2(phi)).  A trial
// whose bound stays below zero by more than the FP32 rounding of p and J2 is
// inside the surface whatever its Lode angle.
__device__ __forceinline__ bool bounded_elastic(const MatConst<float> &m, float c, const float s[6]) {
  float p, d[3], j2;
  mean_dev_j2(s, p, d, j2);
  const float r = xsqrt(xm(j2, 1.f / 3.f));
  const float fmax = xs(xf(xm(2.f, r), xsqrt(xf(m.sphi, m.sphi, 3.f)), xm(xm(2.f, p), m.sphi)),
                        xm(xm(2.f, c), m.cphi));
  return fmax < xm(-1e-4f, xa(xa(r, fabsf(p)), c));
}

// Trial stress -> returned stress (Voigt 6) for Mohr-Coulomb in precision T.
template <typename T>
__device__ __forceinline__ int mc_return(const MatConst<T> &m, T c, const T st[6], T out[6], T &depsp) {
  T lam[3], Q[3][3];
  if constexpr (sizeof(T) == 4)
    eig_sym3_closed(st, lam, Q);
  else
    eig_sym3<T>(st, lam, Q);
  sort3_desc<T>(lam, Q);
  T r[3];
  const int br = mc_principal<T>(m, c, lam, r, depsp);
  if (br == 0) {
#pragma unroll
    for (int i = 0; i < 6; ++i) out[i] = st[i];
  } else if (br == 4) {
    out[0] = out[1] = out[2] = r[0];
    out[3] = out[4] = out[5] = T(0);
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) out[i] = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const T n0 = Q[0][i], n1 = Q[1][i], n2 = Q[2][i];
      out[0] = xf(xm(r[i], n0), n0, out[0]);
      out[1] = xf(xm(r[i], n1), n1, out[1]);
      out[2] = xf(xm(r[i], n2), n2, out[2]);
      out[3] = xf(xm(r[i], n0), n1, out[3]);
      out[4] = xf(xm(r[i], n1), n2, out[4]);
      out[5] = xf(xm(r[i], n0), n2, out[5]);
    }
  }
  return br;
}

// Elastic trial sigma + D : de (isotropic, tensor shear strain).
template <typename T>
__device__ __forceinline__ void elastic_trial(const MatConst<T> &m, const T sig[6], const T de[6], T st[6]) {
  const T tr = xa(xa(de[0], de[1]), de[2]);
  const T lt = xm(m.lam, tr), G2 = xm(T(2), m.G);
#pragma unroll
  for (int i = 0; i < 3; ++i) st[i] = xf(G2, de[i], xa(sig[i], lt));
#pragma unroll
  for (int i = 3; i < 6; ++i) st[i] = xf(G2, de[i], sig[i]);
}

// Distance of the trial stress from the apex c cot(phi) within which the
// FP32 path redoes the return in FP64: 1e-3 (|p| + c cot(phi)).  Inside it the
// principal stresses minus the apex pressure lose more than three of FP32's
// seven digits to cancellation.  The band is relative only: with c = 0 the
// apex is the zero stress and FP32 loses nothing near it.
__device__ __forceinline__ bool near_apex(const float st[6], const MatConst<float> &m, float c) {
  if (!(m.sphi > 0.f) || c == 0.f) return false;  // c = 0: |sigma|^2 >= 3 p^2, the band is empty
  const float pa = xd(xm(c, m.cphi), m.sphi);
  const float p = xm(xa(xa(st[0], st[1]), st[2]), 1.f / 3.f);
  const float d0 = xs(st[0], pa), d1 = xs(st[1], pa), d2 = xs(st[2], pa);
  const float sh = xdot3(st[3], st[3], st[4], st[4], st[5], st[5]);
  const float dist2 = xf(2.f, sh, xdot3(d0, d0, d1, d1, d2, d2));
  const float band = xm(1e-3f, xa(fabsf(p), pa));
  return dist2 < xm(band, band);
}

// The FP64 return near the apex, kept out of line: it is rare, and inlining
// it would raise the register count of the kernel that calls it.  (The step
// runs it in a kernel of its own over the particles G2P queued.)
static __device__ __noinline__ void mc_return_apex_band(const MatConst<double> &md, float c, const float st[6], float out[6],
                                                 float &epsp) {
  double sd[6], od[6], dd;
#pragma unroll
  for (int i = 0; i < 6; ++i) sd[i] = (double)st[i];
  mc_return<double>(md, (double)c, sd, od, dd);
#pragma unroll
  for (int i = 0; i < 6; ++i) out[i] = (float)od[i];
  epsp += (float)dd;
}

// FP32 material update of one particle, sigma <- return(sigma + D:de), all
// in line (no call: a call site makes the caller save its live registers to
// the stack and constrains register allocation around it).  Returns true,
// with sig = the trial stress and epsp unchanged, for a trial inside the apex
// band: the caller completes it with mc_return_apex_band (FP64).
__device__ __forceinline__ bool material_update_inline(const MatConst<float> &m, float c, float sig[6],
                                                       const float de[6], float &epsp) {
  float st[6];
  elastic_trial<float>(m, sig, de, st);
#pragma unroll
  for (int i = 0; i < 6; ++i) sig[i] = st[i];
  if (m.model == 2) sig[2] = 0.f;  // plane stress
  if (m.model != 1 || bounded_elastic(m, c, st) || clearly_elastic(m, c, st)) return false;
  if (near_apex(st, m, c)) return true;
  float d;
  mc_return<float>(m, c, st, sig, d);
  epsp += d;
  return false;
}

// Full FP32 material update: FP32 arithmetic except the Mohr-Coulomb return
// inside the apex band, which runs in FP64.  The FP64 path: everything in FP64.
__device__ __forceinline__ void material_update(const MatConst<float> &m, const MatConst<double> &md,
                                                float c, float sig[6], const float de[6], float &epsp) {
  if (material_update_inline(m, c, sig, de, epsp)) {
    const float st[6] = {sig[0], sig[1], sig[2], sig[3], sig[4], sig[5]};
    mc_return_apex_band(md, c, st, sig, epsp);
  }
}

__device__ __forceinline__ void material_update(const MatConst<double> &m, double c, double sig[6],
                                                const double de[6], double &epsp) {
  double st[6];
  elastic_trial<double>(m, sig, de, st);
  if (m.model != 1) {
#pragma unroll
    for (int i = 0; i < 6; ++i) sig[i] = st[i];
    if (m.model == 2) sig[2] = 0.0;  // plane stress
    return;
  }
  double d;
  mc_return<double>(m, c, st, sig, d);
  epsp += d;
}

}  // namespace mpm
