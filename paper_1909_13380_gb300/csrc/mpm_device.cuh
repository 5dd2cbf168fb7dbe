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
  int model;          // 0 linear elastic, 1 Mohr-Coulomb
  T E, nu, G, lam;    // elastic constants
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
  const T theta = (A[q][q] - A[p][p]) / (T(2) * apq);
  const T t = (theta >= T(0) ? T(1) : T(-1)) / (fabs(theta) + sqrt(theta * theta + T(1)));
  // any c, s with c^2 + s^2 = 1 keep Q orthogonal; rsqrt is exact enough here
  const T c = sizeof(T) == 4 ? (T)rsqrtf((float)(t * t + T(1))) : T(1) / sqrt(t * t + T(1));
  const T s = t * c;
  const T aop = A[o][p], aoq = A[o][q];
  A[p][p] -= t * apq;
  A[q][q] += t * apq;
  A[p][q] = A[q][p] = T(0);
  A[o][p] = A[p][o] = c * aop - s * aoq;
  A[o][q] = A[q][o] = s * aop + c * aoq;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const T vp = Q[r][p], vq = Q[r][q];
    Q[r][p] = c * vp - s * vq;
    Q[r][q] = s * vp + c * vq;
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
    const T off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    const T dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off <= tol * dia || off == T(0)) break;
    jacobi_rot<T, 0, 1>(A, Q);
    jacobi_rot<T, 0, 2>(A, Q);
    jacobi_rot<T, 1, 2>(A, Q);
  }
  lam[0] = A[0][0];
  lam[1] = A[1][1];
  lam[2] = A[2][2];
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
  const float p = (s[0] + s[1] + s[2]) * (1.f / 3.f);
  const float d0 = s[0] - p, d1 = s[1] - p, d2 = s[2] - p;
  const float j2 = 0.5f * (d0 * d0 + d1 * d1 + d2 * d2) + s[3] * s[3] + s[4] * s[4] + s[5] * s[5];
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
  const float r = sqrtf(j2 * (1.f / 3.f));
  const float ir = 1.f / r;
  const float A[3][3] = {{d0 * ir, s[3] * ir, s[5] * ir}, {s[3] * ir, d1 * ir, s[4] * ir}, {s[5] * ir, s[4] * ir, d2 * ir}};
  const float det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[1][2]) - A[0][1] * (A[0][1] * A[2][2] - A[1][2] * A[0][2]) +
                    A[0][2] * (A[0][1] * A[1][2] - A[1][1] * A[0][2]);
  const float c3 = fminf(1.f, fmaxf(-1.f, 0.5f * det));
  const float th = acosf(c3) * (1.f / 3.f);
  float sn, cs;
  sincosf(th, &sn, &cs);
  const float sq3 = 1.7320508f;
  const float mu1 = 2.f * cs, mu3 = -cs - sq3 * sn, mu2 = -cs + sq3 * sn;
  const float mud0 = (mu1 - mu2 >= mu2 - mu3) ? mu1 : mu3;
  // eigenvector of the distinct value: largest cross product of two rows
  float R[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) R[i][j] = A[i][j] - (i == j ? mud0 : 0.f);
  float n[3], best = -1.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int a = k == 2 ? 1 : 0, b = k == 0 ? 1 : 2;  // row pairs (0,1) (0,2) (1,2)
    const float cx = R[a][1] * R[b][2] - R[a][2] * R[b][1];
    const float cy = R[a][2] * R[b][0] - R[a][0] * R[b][2];
    const float cz = R[a][0] * R[b][1] - R[a][1] * R[b][0];
    const float m2 = cx * cx + cy * cy + cz * cz;
    if (m2 > best) {
      best = m2;
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
  n[0] *= inr;
  n[1] *= inr;
  n[2] *= inr;
  // orthonormal basis e1, e2 of the plane orthogonal to n
  float e1[3];
  if (fabsf(n[0]) >= fabsf(n[1])) {
    const float k = rsqrtf(n[0] * n[0] + n[2] * n[2]);
    e1[0] = -n[2] * k;
    e1[1] = 0.f;
    e1[2] = n[0] * k;
  } else {
    const float k = rsqrtf(n[1] * n[1] + n[2] * n[2]);
    e1[0] = 0.f;
    e1[1] = n[2] * k;
    e1[2] = -n[1] * k;
  }
  const float e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
  float An[3], A1[3], A2[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    An[i] = A[i][0] * n[0] + A[i][1] * n[1] + A[i][2] * n[2];
    A1[i] = A[i][0] * e1[0] + A[i][1] * e1[1] + A[i][2] * e1[2];
    A2[i] = A[i][0] * e2[0] + A[i][1] * e2[1] + A[i][2] * e2[2];
  }
  const float mud = n[0] * An[0] + n[1] * An[1] + n[2] * An[2];  // Rayleigh quotient
  const float b11 = e1[0] * A1[0] + e1[1] * A1[1] + e1[2] * A1[2];
  const float b22 = e2[0] * A2[0] + e2[1] * A2[1] + e2[2] * A2[2];
  const float b12 = e1[0] * A2[0] + e1[1] * A2[1] + e1[2] * A2[2];
  float t = 0.f;
  if (b12 != 0.f) {
    const float tj = (b22 - b11) / (2.f * b12);
    t = (tj >= 0.f ? 1.f : -1.f) / (fabsf(tj) + sqrtf(tj * tj + 1.f));
  }
  const float c = rsqrtf(t * t + 1.f), sr = t * c;
  lam[0] = p + r * mud;
  lam[1] = p + r * (b11 - t * b12);
  lam[2] = p + r * (b22 + t * b12);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Q[i][0] = n[i];
    Q[i][1] = c * e1[i] - sr * e2[i];
    Q[i][2] = sr * e1[i] + c * e2[i];
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
  const T f13 = (s[0] - s[2]) + (s[0] + s[2]) * m.sphi - T(2) * c * m.cphi;
  if (!(f13 > T(0))) {
    r[0] = s[0];
    r[1] = s[1];
    r[2] = s[2];
    depsp = T(0);
    return 0;
  }
  const T G2 = T(2) * m.G;
  const T l2 = T(2) * m.lam * m.spsi;
  const T up = G2 * (T(1) + m.spsi), dn = G2 * (T(1) - m.spsi);
  // D N for the planes 1-3 (a), 2-3 (b), 1-2 (c)
  const T DNa[3] = {l2 + up, l2, l2 - dn};
  const T DNb[3] = {l2, l2 + up, l2 - dn};
  const T DNc[3] = {l2 + up, l2 - dn, l2};
  const T a = T(4) * m.G * (T(1) + m.sphi * m.spsi) + T(4) * m.lam * m.sphi * m.spsi;
  int branch = 1;
  const T g = f13 / a;
#pragma unroll
  for (int i = 0; i < 3; ++i) r[i] = s[i] - g * DNa[i];
  if (!(r[0] >= r[1] && r[1] >= r[2])) {
    const T crit = (T(1) - m.spsi) * (s[0] - s[1]) - (T(1) + m.spsi) * (s[1] - s[2]);
    if (crit <= T(0)) {
      const T fb = (s[1] - s[2]) + (s[1] + s[2]) * m.sphi - T(2) * c * m.cphi;
      const T b = T(4) * m.lam * m.sphi * m.spsi + G2 * (T(1) - m.sphi) * (T(1) - m.spsi);
      const T det = a * a - b * b;
      const T ga = (a * f13 - b * fb) / det, gb = (a * fb - b * f13) / det;
#pragma unroll
      for (int i = 0; i < 3; ++i) r[i] = s[i] - ga * DNa[i] - gb * DNb[i];
      branch = 2;
    } else {
      const T fc = (s[0] - s[1]) + (s[0] + s[1]) * m.sphi - T(2) * c * m.cphi;
      const T b = T(4) * m.lam * m.sphi * m.spsi + G2 * (T(1) + m.sphi) * (T(1) + m.spsi);
      const T det = a * a - b * b;
      const T ga = (a * f13 - b * fc) / det, gc = (a * fc - b * f13) / det;
#pragma unroll
      for (int i = 0; i < 3; ++i) r[i] = s[i] - ga * DNa[i] - gc * DNc[i];
      branch = 3;
    }
    if (m.sphi > T(0) && !(r[0] >= r[2])) {
      branch = 4;
      const T pa = c * m.cphi / m.sphi;
      r[0] = r[1] = r[2] = pa;
    }
  }
  T sq = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T d0 = s[i] - r[i], d1 = s[(i + 1) % 3] - r[(i + 1) % 3], d2 = s[(i + 2) % 3] - r[(i + 2) % 3];
    const T e = (d0 - m.nu * (d1 + d2)) / m.E;
    sq += e * e;
  }
  depsp = sqrt(T(2) / T(3) * sq);
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
  const float p = (s[0] + s[1] + s[2]) * (1.f / 3.f);
  const float d0 = s[0] - p, d1 = s[1] - p, d2 = s[2] - p;
  const float j2 = 0.5f * (d0 * d0 + d1 * d1 + d2 * d2) + s[3] * s[3] + s[4] * s[4] + s[5] * s[5];
  const float j3 = d0 * (d1 * d2 - s[4] * s[4]) - s[3] * (s[3] * d2 - s[4] * s[5]) + s[5] * (s[3] * s[4] - d1 * s[5]);
  const float r = sqrtf(j2 * (1.f / 3.f));
  float c3 = r > 0.f ? j3 / (2.f * r * r * r) : 0.f;
  c3 = fminf(1.f, fmaxf(-1.f, c3));
  const float th = acosf(c3) * (1.f / 3.f);
  const float s1 = p + 2.f * r * cosf(th);
  const float s3 = p + 2.f * r * cosf(th + 2.0943951f);
  const float f = (s1 - s3) + (s1 + s3) * m.sphi - 2.f * c * m.cphi;
  const float margin = 4e-3f * (r + fabsf(p)) + 1e-3f * c;
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
  const float p = (s[0] + s[1] + s[2]) * (1.f / 3.f);
  const float d0 = s[0] - p, d1 = s[1] - p, d2 = s[2] - p;
  const float j2 = 0.5f * (d0 * d0 + d1 * d1 + d2 * d2) + s[3] * s[3] + s[4] * s[4] + s[5] * s[5];
  const float r = sqrtf(j2 * (1.f / 3.f));
  const float fmax = 2.f * r * sqrtf(3.f + m.sphi * m.sphi) + 2.f * p * m.sphi - 2.f * c * m.cphi;
  return fmax < -1e-4f * (r + fabsf(p) + c);
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
      out[0] += r[i] * n0 * n0;
      out[1] += r[i] * n1 * n1;
      out[2] += r[i] * n2 * n2;
      out[3] += r[i] * n0 * n1;
      out[4] += r[i] * n1 * n2;
      out[5] += r[i] * n0 * n2;
    }
  }
  return br;
}

// Elastic trial sigma + D : de (isotropic, tensor shear strain).
template <typename T>
__device__ __forceinline__ void elastic_trial(const MatConst<T> &m, const T sig[6], const T de[6], T st[6]) {
  const T tr = de[0] + de[1] + de[2];
  const T lt = m.lam * tr, G2 = T(2) * m.G;
#pragma unroll
  for (int i = 0; i < 3; ++i) st[i] = sig[i] + lt + G2 * de[i];
#pragma unroll
  for (int i = 3; i < 6; ++i) st[i] = sig[i] + G2 * de[i];
}

// Distance of the trial stress from the apex c cot(phi) within which the
// FP32 path redoes the return in FP64: 1e-3 (|p| + c cot(phi)).  Inside it the
// principal stresses minus the apex pressure lose more than three of FP32's
// seven digits to cancellation.  The band is relative only: with c = 0 the
// apex is the zero stress and FP32 loses nothing near it.
__device__ __forceinline__ bool near_apex(const float st[6], const MatConst<float> &m, float c) {
  if (!(m.sphi > 0.f) || c == 0.f) return false;  // c = 0: |sigma|^2 >= 3 p^2, the band is empty
  const float pa = c * m.cphi / m.sphi;
  const float p = (st[0] + st[1] + st[2]) * (1.f / 3.f);
  const float d0 = st[0] - pa, d1 = st[1] - pa, d2 = st[2] - pa;
  const float dist2 = d0 * d0 + d1 * d1 + d2 * d2 + 2.f * (st[3] * st[3] + st[4] * st[4] + st[5] * st[5]);
  const float band = 1e-3f * (fabsf(p) + pa);
  return dist2 < band * band;
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
    return;
  }
  double d;
  mc_return<double>(m, c, st, sig, d);
  epsp += d;
}

}  // namespace mpm
