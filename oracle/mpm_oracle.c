/*
 * mpm_oracle.c -- plain, slow, FP64 CPU explicit material point method.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the parity oracle: only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg load it.  The
 * product path (the CUDA library) shares no code, header, table or helper
 * with it and must never call it.
 *
 * What it computes (Kumar et al., "Scalable and modular material point
 * method for large-scale simulations", arXiv 1909.13380):
 *   - INTRODUCTION: particles carry the state; the governing equations are
 *     solved on the nodes of a fixed background mesh whose nodal values are
 *     reset every step; particle -> node and node -> particle transfers use
 *     the same mapping (shape) functions.
 *   - CODE OVERVIEW: Node stores mass, momentum, velocity, acceleration and
 *     forces (reset every step) while friction and velocity constraints
 *     persist; Cell holds the linear 4-node quadrilateral / 8-node hexahedron
 *     element; Material turns a strain increment into a stress; the explicit
 *     Update-Stress-First (USF) and Update-Stress-Last (USL) schemes.
 *   - DATA STRUCTURES: stress and strain in 6-component Voigt form.
 *   - ISOPARAMETRIC MESH: velocity and frictional (acceleration) boundary
 *     conditions are applied at the nodes; particles are located in cells.
 * The paper states none of the equations.  They are the textbook explicit
 * MPM (Sulsky, Chen & Schreyer 1994; USF/USL ordering as analysed by
 * Bardenhagen 2002) and, for the Mohr-Coulomb material, the principal-space
 * multi-surface return of de Souza Neto, Peric & Owen (2008, ch. 8), with
 * the readings listed below.
 *
 * Readings where the paper is silent (each is stated again where it is used):
 *   R1  FLIP particle velocity update, v_p += dt * sum_i N_ip a_i; position
 *       advected with the updated nodal velocity.
 *   R2  a node is active when its mass exceeds mass_tol; inactive nodes carry
 *       v = a = v' = 0.
 *   R3  fixed face: all velocity/acceleration components zero; roller face:
 *       the normal component zero; friction face: Coulomb friction applied
 *       as an acceleration condition (node_constrain below).
 *   R4  Mohr-Coulomb: tension positive, perfect plasticity, yield
 *       f = (s1 - s3) + (s1 + s3) sin(phi) - 2 c cos(phi), plastic potential
 *       of the same form with psi, return to main plane / edge / apex.
 *   R5  small-strain hypoelastic stress increment, no objective rate;
 *       volume update V <- V (1 + tr de).
 *   R6  a particle exactly on a cell face belongs to the higher cell (floor);
 *       a particle at or beyond the upper mesh bound has left the mesh.
 *   R7  2D is plane strain: the stress keeps its zz component, strain zz = 0,
 *       unless the material is the plane-stress elastic one (R8).
 *   R8  plane stress (BENCHMARK AND PERFORMANCE: the plate with a hole is a
 *       "plane strip (plane stress)"): stress zz = 0 and the in-plane
 *       stiffness has lambda* = 2 lambda G / (lambda + 2 G) in place of
 *       lambda; the area follows the in-plane trace of the strain increment.
 *   R9  a uniform traction on an end of the body (the plate's "uniform
 *       tension ... applied at the ends"): a constant force on the nodes of
 *       the mesh face that coincides with that end, traction times the
 *       node's tributary length (area in 3D): h per tangent axis, half of
 *       it at the face's own edges.
 *   R10 a quasi-static protocol (the plate's static stress field; the paper
 *       gives none): mass-proportional viscous damping of the nodal motion,
 *       a = f / m - alpha v, so the explicit run settles to equilibrium.
 *   R11 mapped (isoparametric) mesh (ISOPARAMETRIC MESH): the logical grid
 *       of cells is the Cartesian one with moved nodes; the natural
 *       coordinates of a point are the root of x(xi) = x, found by Newton-
 *       Raphson from the affine guess; a particle keeps the cell the
 *       neighbourhood walk last found for it; a point on a face shared by
 *       two cells belongs to the higher one (xi = 1 is outside, as R6).
 *   R12 on a mapped mesh ("nodal boundary conditions on irregular
 *       surfaces") a node of a logical face takes the face's outward normal
 *       there (face_normal: the facet normals next to the node summed and
 *       normalised); a roller removes the velocity along the roller
 *       normals of the node (made orthonormal in face order), a friction
 *       face applies R3 with that normal; fixed faces as before; face
 *       tractions (R9) are not defined there.
 *   R13 a far-field stress on a face of a mapped 2D mesh (the plate's
 *       "uniform tension" at its end, when one logical face runs along the
 *       loaded end and a free edge): the traction sigma . n of a uniform
 *       stress sigma on each boundary edge of the face, lumped to the edge's
 *       two nodes -- node a gets sum over its edges e of sigma . n_e |e| / 2
 *       (n_e the outward normal).  On a Cartesian face it would be the
 *       traction sigma . n of R9.
 *
 * Layout: every particle vector is stored with 3 components and every
 * stress/strain with 6 Voigt components (xx, yy, zz, xy, yz, xz; tensor
 * shear strain, not engineering gamma), also in 2D, where the unused
 * components stay zero.  Nodes are numbered x fastest.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Status codes, mirrored in the Python wrapper. */
#define OM_OK 0
#define OM_LEFT_MESH (-4)
#define OM_NONFINITE (-5)
#define OM_ARG (-1)

enum { OM_BC_FREE = 0, OM_BC_ROLLER = 1, OM_BC_FIXED = 2, OM_BC_FRICTION = 3 };
enum { OM_USF = 0, OM_USL = 1 };
enum { OM_LINEAR_ELASTIC = 0, OM_MOHR_COULOMB = 1, OM_PLANE_STRESS_ELASTIC = 2 };

typedef struct {
  int32_t dim;        /* 2 (4-node quad, plane strain) or 3 (8-node hex) */
  int32_t n[3];       /* cells per axis */
  double h;           /* cell size */
  double origin[3];   /* coordinates of node (0,0,0) */
  int32_t face_bc[6]; /* -x,+x,-y,+y,-z,+z */
  double face_mu[6];  /* Coulomb coefficient of a FRICTION face */
  double g[3];        /* gravity */
  double dt;
  int32_t scheme;     /* OM_USF / OM_USL */
  double mass_tol;    /* R2 */
  double face_traction[6][3]; /* R9: traction on each face (force per length / area) */
  double damping;     /* R10: alpha, 1/s */
  double face_stress[6][6];   /* R13: a uniform stress loading each face of a mapped 2D mesh (Voigt) */
} om_mesh;

typedef struct {
  int32_t model;      /* OM_LINEAR_ELASTIC / OM_MOHR_COULOMB / OM_PLANE_STRESS_ELASTIC (2D) */
  double E, nu, rho;
  double phi, c, psi; /* radians, Pa, radians */
} om_material;

/* ------------------------------------------------------------------------ */
/* Mesh helpers                                                             */
/* ------------------------------------------------------------------------ */

static int64_t nodes_along(const om_mesh *M, int k) {
  return k < M->dim ? (int64_t)M->n[k] + 1 : 1;
}

int64_t oracle_num_nodes(const om_mesh *M) {
  return nodes_along(M, 0) * nodes_along(M, 1) * nodes_along(M, 2);
}

/* Scratch doubles needed by oracle_step: m, P[3], f[3], v[3], a[3], v'[3]. */
int64_t oracle_work_size(const om_mesh *M) { return 16 * oracle_num_nodes(M); }

static int64_t node_index(const om_mesh *M, const int ijk[3]) {
  return ijk[0] + nodes_along(M, 0) * (ijk[1] + nodes_along(M, 1) * (int64_t)ijk[2]);
}

/* Locate a point: cell = floor((x - origin) / h) per axis (R6); natural
 * coordinate xi in [-1, 1) measured from the cell centre.  Returns
 * OM_LEFT_MESH when the point is outside the mesh. */
int oracle_locate(const om_mesh *M, const double x[3], int32_t cell[3], double xi[3]) {
  for (int k = 0; k < 3; ++k) {
    cell[k] = 0;
    xi[k] = 0.0;
  }
  for (int k = 0; k < M->dim; ++k) {
    double s = (x[k] - M->origin[k]) / M->h;
    if (!(s >= 0.0)) return OM_LEFT_MESH; /* also catches NaN */
    double f = floor(s);
    if (f >= (double)M->n[k]) return OM_LEFT_MESH;
    cell[k] = (int32_t)f;
    xi[k] = 2.0 * (s - f) - 1.0;
  }
  return OM_OK;
}

/* Linear Lagrange shape functions of the 4-node quadrilateral (dim 2) and
 * the 8-node hexahedron (dim 3) in natural coordinates (CODE OVERVIEW:
 * "Linear" mapping functions of the quadrilateral / hexahedral elements).
 * Node a has natural coordinates xi^a_k = +1 if bit k of a is set, else -1,
 * so nodes are ordered x fastest.
 *   N_a = prod_k (1 + xi_k xi^a_k) / 2
 *   dN_a/dxi_k = (xi^a_k / 2) prod_{j != k} (1 + xi_j xi^a_j) / 2 */
void oracle_shape(int32_t dim, const double xi[3], double N[8], double dNdxi[24]) {
  int nn = 1 << dim;
  for (int a = 0; a < nn; ++a) {
    double w[3], dw[3];
    for (int k = 0; k < dim; ++k) {
      double sa = ((a >> k) & 1) ? 1.0 : -1.0;
      w[k] = 0.5 * (1.0 + sa * xi[k]);
      dw[k] = 0.5 * sa;
    }
    double prod = 1.0;
    for (int k = 0; k < dim; ++k) prod *= w[k];
    N[a] = prod;
    for (int k = 0; k < 3; ++k) {
      double d = 0.0;
      if (k < dim) {
        d = dw[k];
        for (int j = 0; j < dim; ++j)
          if (j != k) d *= w[j];
      }
      dNdxi[3 * a + k] = d;
    }
  }
  for (int a = nn; a < 8; ++a) {
    N[a] = 0.0;
    for (int k = 0; k < 3; ++k) dNdxi[3 * a + k] = 0.0;
  }
}

/* Voigt (xx, yy, zz, xy, yz, xz) -> symmetric 3x3 entry (j,k). */
static double voigt_at(const double s[6], int j, int k) {
  static const int map[3][3] = {{0, 3, 5}, {3, 1, 4}, {5, 4, 2}};
  return s[map[j][k]];
}

/* Node global index of local node a of a cell. */
static int64_t cell_node(const om_mesh *M, const int32_t cell[3], int a) {
  int ijk[3];
  for (int k = 0; k < 3; ++k) ijk[k] = cell[k] + (k < M->dim ? ((a >> k) & 1) : 0);
  return node_index(M, ijk);
}

/* ------------------------------------------------------------------------ */
/* Isoparametric (mapped) cells (ISOPARAMETRIC MESH).  The logical grid of  */
/* cells is the Cartesian one, but node i sits at X[3 i .. 3 i + 2], so a   */
/* cell is the image of [-1, 1]^d under x(xi) = sum_a N_a(xi) X_a.  A point */
/* is placed in a cell by inverting that map with Newton-Raphson from the   */
/* affine guess xi0 = J(0)^-1 (x - x(0)), and particles are located by a    */
/* neighbourhood walk from their current cell.                              */
/* ------------------------------------------------------------------------ */

/* Coordinates of the 2^d nodes of a cell (node a: bit k = upper along k). */
static void iso_cell_nodes(const om_mesh *M, const double *X, const int32_t cell[3], double xa[8][3]) {
  int nn = 1 << M->dim;
  for (int a = 0; a < nn; ++a) {
    int64_t i = cell_node(M, cell, a);
    for (int k = 0; k < 3; ++k) xa[a][k] = X[3 * i + k];
  }
}

/* x(xi) and the Jacobian J[j][k] = dx_j / dxi_k of the cell's map. */
static void iso_map(int dim, const double xa[8][3], const double xi[3], double x[3], double J[3][3]) {
  double N[8], dN[24];
  oracle_shape(dim, xi, N, dN);
  for (int j = 0; j < 3; ++j) {
    x[j] = 0.0;
    for (int k = 0; k < 3; ++k) J[j][k] = (j == k && j >= dim) ? 1.0 : 0.0;
  }
  for (int a = 0; a < (1 << dim); ++a)
    for (int j = 0; j < dim; ++j) {
      x[j] += N[a] * xa[a][j];
      for (int k = 0; k < dim; ++k) J[j][k] += xa[a][j] * dN[3 * a + k];
    }
}

/* Inverse of the leading dim x dim block of J (cofactors); 0 if singular. */
static int iso_inverse(int dim, const double J[3][3], double Ji[3][3]) {
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) Ji[j][k] = (j == k) ? 1.0 : 0.0;
  if (dim == 2) {
    double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    if (!(det != 0.0) || !isfinite(det)) return 0;
    Ji[0][0] = J[1][1] / det;
    Ji[0][1] = -J[0][1] / det;
    Ji[1][0] = -J[1][0] / det;
    Ji[1][1] = J[0][0] / det;
    return 1;
  }
  double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  if (!(det != 0.0) || !isfinite(det)) return 0;
  Ji[0][0] = c00 / det;
  Ji[1][0] = c01 / det;
  Ji[2][0] = c02 / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  return 1;
}

/* The affine guess of x's natural coordinates in a cell: the map
 * linearised at the cell centre, xi0 = J(0)^-1 (x - x(0)).  0 if J(0) is
 * singular. */
static int iso_affine(const om_mesh *M, const double xa[8][3], const double x[3], double xi[3]) {
  double x0[3], J[3][3], Ji[3][3];
  xi[0] = xi[1] = xi[2] = 0.0;
  iso_map(M->dim, xa, xi, x0, J);
  if (!iso_inverse(M->dim, J, Ji)) return 0;
  for (int j = 0; j < M->dim; ++j)
    for (int k = 0; k < M->dim; ++k) xi[j] += Ji[j][k] * (x[k] - x0[k]);
  return 1;
}

/* Natural coordinates of x in a cell: Newton-Raphson on x(xi) = x from the
 * affine guess.  Returns the iterations taken, or -1 if the map is singular
 * or Newton does not converge (50 iterations), with xi then the affine
 * guess.  Far outside the cell the extrapolated map may have other roots:
 * only a root inside (or near) the cell means anything. */
int oracle_iso_natural(const om_mesh *M, const double *X, const int32_t cell[3], const double x[3],
                       double xi[3]) {
  double xa[8][3], J[3][3], Ji[3][3];
  iso_cell_nodes(M, X, cell, xa);
  if (!iso_affine(M, xa, x, xi)) return -1;
  double guess[3] = {xi[0], xi[1], xi[2]};
  int done = 0;
  for (int it = 1; it <= 50; ++it) {
    double xm[3], r[3], step = 0.0;
    iso_map(M->dim, xa, xi, xm, J);
    if (!iso_inverse(M->dim, J, Ji)) break;
    for (int k = 0; k < M->dim; ++k) r[k] = xm[k] - x[k];
    for (int j = 0; j < M->dim; ++j) {
      double d = 0.0;
      for (int k = 0; k < M->dim; ++k) d += Ji[j][k] * r[k];
      xi[j] -= d;
      if (fabs(d) > step) step = fabs(d);
    }
    if (!isfinite(step)) break;
    /* converged to rounding: the residual's rounding, divided by J, keeps
     * the last steps near 1e-15; one more step after 1e-12 */
    if (step < 1e-12) {
      if (done) return it;
      done = 1;
    }
  }
  for (int j = 0; j < 3; ++j) xi[j] = guess[j];
  return -1;
}

/* Locate x by a neighbourhood walk from `cell` (updated).  In the current
 * cell take the affine guess of xi; while it lies well outside the cell
 * (beyond [-2, 2] on some axis) it sets the direction, otherwise Newton's
 * root does.  If some xi_k lies outside [-1, 1), step to the neighbour along
 * the axis of the largest excess (the next largest when that neighbour is
 * beyond the grid) and repeat.  A point on a face shared by two cells
 * belongs to the higher one (xi = 1 is outside); a point that needs a step
 * beyond the grid on every axis it lies outside of has left the mesh. */
int oracle_iso_locate(const om_mesh *M, const double *X, const double x[3], int32_t cell[3], double xi[3]) {
  int limit = 2 * (M->n[0] + M->n[1] + M->n[2]) + 8;
  for (int s = 0; s < limit; ++s) {
    double xa[8][3];
    iso_cell_nodes(M, X, cell, xa);
    if (!iso_affine(M, xa, x, xi)) return OM_LEFT_MESH;
    int far = 0, conv = 0;
    for (int k = 0; k < M->dim; ++k) far |= fabs(xi[k]) > 2.0;
    if (!far) conv = oracle_iso_natural(M, X, cell, x, xi) >= 0;
    double excess[3] = {0.0, 0.0, 0.0};
    int dir[3] = {0, 0, 0}, any = 0;
    for (int k = 0; k < M->dim; ++k) {
      if (xi[k] < -1.0) {
        excess[k] = -1.0 - xi[k];
        dir[k] = -1;
      } else if (xi[k] >= 1.0) {
        excess[k] = xi[k] - 1.0;
        dir[k] = 1;
      }
      any |= dir[k] != 0;
    }
    if (!any) return conv ? OM_OK : OM_LEFT_MESH;
    int moved = 0;
    for (int tries = 0; tries < M->dim && !moved; ++tries) {
      int best = -1;
      for (int k = 0; k < M->dim; ++k)
        if (dir[k] != 0 && (best < 0 || excess[k] > excess[best])) best = k;
      if (best < 0) break;
      int c = cell[best] + dir[best];
      if (c >= 0 && c < M->n[best]) {
        cell[best] = c;
        moved = 1;
      } else {
        dir[best] = 0;
      }
    }
    if (!moved) return OM_LEFT_MESH;
  }
  return OM_LEFT_MESH;
}

/* Shape values and physical gradients of a point in a mapped cell:
 * dN_a/dx_j = sum_k dN_a/dxi_k dxi_k/dx_j = sum_k dN_a/dxi_k Ji[k][j]. */
void oracle_iso_basis(const om_mesh *M, const double *X, const int32_t cell[3], const double xi[3],
                      double N[8], double G[24]) {
  double xa[8][3], xm[3], J[3][3], Ji[3][3], dN[24];
  iso_cell_nodes(M, X, cell, xa);
  iso_map(M->dim, xa, xi, xm, J);
  iso_inverse(M->dim, J, Ji);
  oracle_shape(M->dim, xi, N, dN);
  for (int a = 0; a < 8; ++a)
    for (int j = 0; j < 3; ++j) {
      double g = 0.0;
      if (a < (1 << M->dim) && j < M->dim)
        for (int k = 0; k < M->dim; ++k) g += dN[3 * a + k] * Ji[k][j];
      G[3 * a + j] = g;
    }
}

/* The basis of particle p.  Cartesian mesh (X == NULL): its cell by the
 * floor rule, G = dN/dxi (the caller multiplies by 2/h).  Mapped mesh: the
 * cell it is stored in (pcell), xi by Newton-Raphson, G = dN/dx. */
static int particle_basis(const om_mesh *M, const double *X, const int32_t *pcell, int64_t p, const double *x,
                          int32_t cell[3], double N[8], double G[24]) {
  double xi[3];
  if (!X) {
    if (oracle_locate(M, x, cell, xi) != OM_OK) return OM_LEFT_MESH;
    oracle_shape(M->dim, xi, N, G);
    return OM_OK;
  }
  for (int k = 0; k < 3; ++k) cell[k] = pcell[3 * p + k];
  if (oracle_iso_natural(M, X, cell, x, xi) < 0) return OM_LEFT_MESH;
  oracle_iso_basis(M, X, cell, xi, N, G);
  return OM_OK;
}

/* ------------------------------------------------------------------------ */
/* Particle -> grid (INTRODUCTION: "transferred from the material points to */
/* the nodes using mapping functions"; DATA STRUCTURES: nodal aggregation)  */
/*   m_i = sum_p N_ip m_p                                                   */
/*   P_i = sum_p N_ip m_p v_p                                               */
/*   f_i = sum_p [ -V_p sigma_p . grad N_ip + N_ip m_p g ]                  */
/* ------------------------------------------------------------------------ */
static void p2g(const om_mesh *M, const double *X, const int32_t *pcell, int64_t np, const double *x,
                const double *v, const double *sig, const double *m, const double *vol, const int32_t *alive,
                double *nm, double *nP, double *nf, int want_mass_mom, int want_force) {
  int nn = 1 << M->dim;
  for (int64_t p = 0; p < np; ++p) {
    if (!alive[p]) continue;
    int32_t cell[3];
    double N[8], dN[24];
    if (particle_basis(M, X, pcell, p, x + 3 * p, cell, N, dN) != OM_OK) continue;
    for (int a = 0; a < nn; ++a) {
      int64_t i = cell_node(M, cell, a);
      if (want_mass_mom) {
        nm[i] += N[a] * m[p];
        for (int k = 0; k < 3; ++k) nP[3 * i + k] += N[a] * m[p] * v[3 * p + k];
      }
      if (want_force) {
        double grad[3];
        for (int k = 0; k < 3; ++k) grad[k] = X ? dN[3 * a + k] : dN[3 * a + k] * 2.0 / M->h;
        for (int j = 0; j < 3; ++j) {
          double sg = 0.0;
          for (int k = 0; k < 3; ++k) sg += voigt_at(sig + 6 * p, j, k) * grad[k];
          double fint = (j < M->dim) ? -vol[p] * sg : 0.0;
          double fext = (j < M->dim) ? N[a] * m[p] * M->g[j] : 0.0;
          nf[3 * i + j] += fint + fext;
        }
      }
    }
  }
}

/* Exposed for the brute-force and conservation pins: nodal mass, momentum
 * and total (internal + external) force of the current particle state. */
void oracle_p2g(const om_mesh *M, int64_t np, const double *x, const double *v,
                const double *sig, const double *m, const double *vol, const int32_t *alive,
                double *nm, double *nP, double *nf) {
  int64_t nnodes = oracle_num_nodes(M);
  memset(nm, 0, sizeof(double) * nnodes);
  memset(nP, 0, sizeof(double) * 3 * nnodes);
  memset(nf, 0, sizeof(double) * 3 * nnodes);
  p2g(M, NULL, NULL, np, x, v, sig, m, vol, alive, nm, nP, nf, 1, 1);
}

/* ------------------------------------------------------------------------ */
/* Nodal boundary conditions (ISOPARAMETRIC MESH: "velocity constraints and */
/* acceleration (frictional) boundary conditions are applied at the        */
/* nodes"; CODE OVERVIEW: constraints persist while nodal values reset).    */
/* ------------------------------------------------------------------------ */

/* Which faces node ijk lies on: bit f set for face f (-x,+x,-y,+y,-z,+z). */
static int node_faces(const om_mesh *M, const int ijk[3]) {
  int mask = 0;
  for (int k = 0; k < M->dim; ++k) {
    if (ijk[k] == 0) mask |= 1 << (2 * k);
    if (ijk[k] == M->n[k]) mask |= 1 << (2 * k + 1);
  }
  return mask;
}

/* Velocity constraints on the pre-force nodal velocity (USF stage one):
 * fixed -> 0; roller -> normal component 0; friction face -> the normal
 * component is removed only when it points out of the mesh (no
 * penetration), tangential friction waits for the force stage. */
static void constrain_velocity(const om_mesh *M, int faces, double v[3]) {
  for (int f = 0; f < 2 * M->dim; ++f)
    if ((faces >> f & 1) && M->face_bc[f] == OM_BC_FIXED) {
      v[0] = v[1] = v[2] = 0.0;
      return;
    }
  for (int f = 0; f < 2 * M->dim; ++f) {
    if (!(faces >> f & 1)) continue;
    int k = f / 2;
    double out = (f & 1) ? 1.0 : -1.0;
    if (M->face_bc[f] == OM_BC_ROLLER) v[k] = 0.0;
    if (M->face_bc[f] == OM_BC_FRICTION && out * v[k] > 0.0) v[k] = 0.0;
  }
}

/* Full constraint at the force stage, on (v, a, v' = v + a dt).
 *  fixed face:    v = a = v' = 0 in every component;
 *  roller face:   v, a, v' = 0 in the face-normal component;
 *  friction face (reading R3): let w = out . v' be the speed into the wall
 *    (out = outward normal).  If w > 0 the node is in contact: the normal
 *    component of v' becomes 0, and the tangential part t of v' is reduced
 *    by the Coulomb limit mu * w (the normal velocity jump times mu), or to
 *    zero when |t| <= mu * w (stick).  The acceleration of every component
 *    changed by contact is reset to (v' - v) / dt so that v' = v + a dt
 *    still holds.  If w <= 0 the node is free.
 * Faces are visited in order -x,+x,-y,+y,-z,+z; a fixed face wins outright,
 * rollers act before friction faces. */
static void constrain_full(const om_mesh *M, int faces, double v[3], double a[3], double vn[3]) {
  for (int f = 0; f < 2 * M->dim; ++f)
    if ((faces >> f & 1) && M->face_bc[f] == OM_BC_FIXED) {
      for (int k = 0; k < 3; ++k) v[k] = a[k] = vn[k] = 0.0;
      return;
    }
  for (int f = 0; f < 2 * M->dim; ++f)
    if ((faces >> f & 1) && M->face_bc[f] == OM_BC_ROLLER) {
      int k = f / 2;
      v[k] = a[k] = vn[k] = 0.0;
    }
  for (int f = 0; f < 2 * M->dim; ++f) {
    if (!((faces >> f & 1) && M->face_bc[f] == OM_BC_FRICTION)) continue;
    int k = f / 2;
    double out = (f & 1) ? 1.0 : -1.0;
    double w = out * vn[k];
    if (!(w > 0.0)) continue;
    vn[k] = 0.0;
    double tnorm2 = 0.0;
    for (int j = 0; j < M->dim; ++j)
      if (j != k) tnorm2 += vn[j] * vn[j];
    double tnorm = sqrt(tnorm2);
    double cap = M->face_mu[f] * w;
    for (int j = 0; j < M->dim; ++j) {
      if (j == k) continue;
      if (tnorm <= cap)
        vn[j] = 0.0;
      else
        vn[j] -= cap * vn[j] / tnorm;
    }
    for (int j = 0; j < M->dim; ++j) a[j] = (vn[j] - v[j]) / M->dt;
  }
}

/* ---- conditions on the faces of a mapped mesh (R12) ---------------------- */

/* Outward unit normal of logical face f at its node ijk: the sum of the
 * outward normals of the boundary facets next to the node -- in 2D the
 * boundary edges, each normal as long as its edge; in 3D the bilinear facets,
 * each the cross product of its two edges at the node -- normalised.  The
 * inward direction is the mesh edge from the node into the mesh. */
static void face_normal(const om_mesh *M, const double *X, int f, const int ijk[3], double n[3]) {
  const int k = f / 2, up = f & 1;
  const double *x0 = X + 3 * node_index(M, ijk);
  int in3[3] = {ijk[0], ijk[1], ijk[2]};
  in3[k] += up ? -1 : 1;
  const double *xi = X + 3 * node_index(M, in3);
  double din[3], acc[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < 3; ++c) din[c] = xi[c] - x0[c];
  if (M->dim == 2) {
    const int t = 1 - k;
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      int nb[3] = {ijk[0], ijk[1], 0};
      nb[t] += sgn;
      if (nb[t] < 0 || nb[t] > M->n[t]) continue;
      const double *xb = X + 3 * node_index(M, nb);
      double e0 = xb[0] - x0[0], e1 = xb[1] - x0[1];
      double q0 = e1, q1 = -e0; /* perpendicular, |q| = |e| */
      if (q0 * din[0] + q1 * din[1] > 0.0) { q0 = -q0; q1 = -q1; }
      acc[0] += q0;
      acc[1] += q1;
    }
  } else {
    const int t1 = (k + 1) % 3, t2 = (k + 2) % 3;
    for (int s1 = -1; s1 <= 1; s1 += 2)
      for (int s2 = -1; s2 <= 1; s2 += 2) {
        int a3[3] = {ijk[0], ijk[1], ijk[2]}, b3[3] = {ijk[0], ijk[1], ijk[2]};
        a3[t1] += s1;
        b3[t2] += s2;
        if (a3[t1] < 0 || a3[t1] > M->n[t1] || b3[t2] < 0 || b3[t2] > M->n[t2]) continue;
        const double *xa = X + 3 * node_index(M, a3), *xb = X + 3 * node_index(M, b3);
        double ea[3], eb[3], q[3];
        for (int c = 0; c < 3; ++c) {
          ea[c] = xa[c] - x0[c];
          eb[c] = xb[c] - x0[c];
        }
        q[0] = ea[1] * eb[2] - ea[2] * eb[1];
        q[1] = ea[2] * eb[0] - ea[0] * eb[2];
        q[2] = ea[0] * eb[1] - ea[1] * eb[0];
        if (q[0] * din[0] + q[1] * din[1] + q[2] * din[2] > 0.0)
          for (int c = 0; c < 3; ++c) q[c] = -q[c];
        for (int c = 0; c < 3; ++c) acc[c] += q[c];
      }
  }
  double len = sqrt(acc[0] * acc[0] + acc[1] * acc[1] + acc[2] * acc[2]);
  for (int c = 0; c < 3; ++c) n[c] = acc[c] / len;
}

void oracle_face_normal(const om_mesh *M, const double *X, int32_t f, const int32_t ijk[3], double n[3]) {
  int c[3] = {ijk[0], ijk[1], ijk[2]};
  face_normal(M, X, f, c, n);
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* The roller normals of a node, made orthonormal in face order (Gram-Schmidt),
 * so that removing each removes the velocity along every roller normal. */
static int roller_basis(const om_mesh *M, const double *X, int faces, const int ijk[3], double B[3][3]) {
  int nb = 0;
  for (int f = 0; f < 2 * M->dim; ++f) {
    if (!((faces >> f & 1) && M->face_bc[f] == OM_BC_ROLLER)) continue;
    double n[3];
    face_normal(M, X, f, ijk, n);
    for (int b = 0; b < nb; ++b) {
      double d = dot3(n, B[b]);
      for (int c = 0; c < 3; ++c) n[c] -= d * B[b][c];
    }
    double len = sqrt(dot3(n, n));
    if (!(len > 1e-12)) continue; /* parallel to an earlier roller normal */
    for (int c = 0; c < 3; ++c) B[nb][c] = n[c] / len;
    ++nb;
  }
  return nb;
}

/* The velocity stage and the full constraint of a node of a mapped mesh:
 * the Cartesian rules with the face's outward normal n in place of the face
 * axis -- a roller removes the components along the roller normals, a
 * friction face acts on w = n . v' and the part of v' tangent to it. */
static void constrain_velocity_mapped(const om_mesh *M, const double *X, int faces, const int ijk[3], double v[3]) {
  for (int f = 0; f < 2 * M->dim; ++f)
    if ((faces >> f & 1) && M->face_bc[f] == OM_BC_FIXED) {
      v[0] = v[1] = v[2] = 0.0;
      return;
    }
  double B[3][3];
  int nb = roller_basis(M, X, faces, ijk, B);
  for (int b = 0; b < nb; ++b) {
    double d = dot3(v, B[b]);
    for (int c = 0; c < 3; ++c) v[c] -= d * B[b][c];
  }
  for (int f = 0; f < 2 * M->dim; ++f) {
    if (!((faces >> f & 1) && M->face_bc[f] == OM_BC_FRICTION)) continue;
    double n[3];
    face_normal(M, X, f, ijk, n);
    double w = dot3(v, n);
    if (w > 0.0)
      for (int c = 0; c < 3; ++c) v[c] -= w * n[c];
  }
}

static void constrain_full_mapped(const om_mesh *M, const double *X, int faces, const int ijk[3], double v[3],
                                  double a[3], double vn[3]) {
  for (int f = 0; f < 2 * M->dim; ++f)
    if ((faces >> f & 1) && M->face_bc[f] == OM_BC_FIXED) {
      for (int k = 0; k < 3; ++k) v[k] = a[k] = vn[k] = 0.0;
      return;
    }
  double B[3][3];
  int nb = roller_basis(M, X, faces, ijk, B);
  for (int b = 0; b < nb; ++b) {
    double dv = dot3(v, B[b]), da = dot3(a, B[b]), dn = dot3(vn, B[b]);
    for (int c = 0; c < 3; ++c) {
      v[c] -= dv * B[b][c];
      a[c] -= da * B[b][c];
      vn[c] -= dn * B[b][c];
    }
  }
  for (int f = 0; f < 2 * M->dim; ++f) {
    if (!((faces >> f & 1) && M->face_bc[f] == OM_BC_FRICTION)) continue;
    double n[3];
    face_normal(M, X, f, ijk, n);
    double w = dot3(vn, n);
    if (!(w > 0.0)) continue;
    for (int c = 0; c < 3; ++c) vn[c] -= w * n[c];
    double tnorm = sqrt(dot3(vn, vn));
    double cap = M->face_mu[f] * w;
    for (int c = 0; c < 3; ++c) {
      if (tnorm <= cap)
        vn[c] = 0.0;
      else
        vn[c] -= cap * vn[c] / tnorm;
    }
    for (int c = 0; c < M->dim; ++c) a[c] = (vn[c] - v[c]) / M->dt;
  }
}

/* Exposed for unit tests of a single node: node ijk, in/out v, a, v'. */
void oracle_constrain_node(const om_mesh *M, const int32_t ijk[3], double v[3], double a[3],
                           double vn[3]) {
  int c[3] = {ijk[0], ijk[1], ijk[2]};
  constrain_full(M, node_faces(M, c), v, a, vn);
}

/* ------------------------------------------------------------------------ */
/* Material: stress for a strain increment (CODE OVERVIEW: Material class)  */
/* ------------------------------------------------------------------------ */

/* Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix given in
 * Voigt order (Golub & Van Loan, symmetric Schur rotation).  On return
 * lam[i] are the eigenvalues and column i of V (V[3*r + i]) the unit
 * eigenvector. */
void oracle_eig_sym3(const double s[6], double lam[3], double V[9]) {
  double A[3][3];
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) A[j][k] = voigt_at(s, j, k);
  double Q[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  static const int P[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
    double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
    if (off == 0.0 || off <= 1e-34 * dia) break;
    for (int r = 0; r < 3; ++r) {
      int p = P[r][0], q = P[r][1];
      double apq = A[p][q];
      if (apq == 0.0) continue;
      double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
      double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
      int o = 3 - p - q; /* the remaining index */
      double aop = A[o][p], aoq = A[o][q];
      A[p][p] -= t * apq;
      A[q][q] += t * apq;
      A[p][q] = A[q][p] = 0.0;
      A[o][p] = A[p][o] = c * aop - sn * aoq;
      A[o][q] = A[q][o] = sn * aop + c * aoq;
      for (int rr = 0; rr < 3; ++rr) {
        double vp = Q[rr][p], vq = Q[rr][q];
        Q[rr][p] = c * vp - sn * vq;
        Q[rr][q] = sn * vp + c * vq;
      }
    }
  }
  for (int i = 0; i < 3; ++i) {
    lam[i] = A[i][i];
    for (int r = 0; r < 3; ++r) V[3 * r + i] = Q[r][i];
  }
}

/* Mohr-Coulomb return mapping in principal stresses (reading R4), following
 * the order of de Souza Neto, Peric & Owen (2008), Box 8.5: elastic check,
 * main plane, then one of the two edges, then the apex.
 * sig_tr: elastic trial stress (Voigt).  Returns the branch taken:
 *   0 elastic, 1 main plane, 2 edge s1 = s2, 3 edge s2 = s3, 4 apex.
 * depsp (may be NULL) receives the equivalent plastic strain increment
 * sqrt(2/3 |de^p|^2) with de^p = C (sig_tr - sig) in principal axes. */
int oracle_mc_return(double E, double nu, double phi, double psi, double c, const double sig_tr[6],
                     double sig_out[6], double *depsp) {
  double G = E / (2.0 * (1.0 + nu));
  double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  double sphi = sin(phi), cphi = cos(phi), spsi = sin(psi);

  double ev[3], V[9];
  oracle_eig_sym3(sig_tr, ev, V);
  /* order s1 >= s2 >= s3, ties keep the solver order (stable) */
  int ord[3] = {0, 1, 2};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j + 1 < 3 - i; ++j)
      if (ev[ord[j]] < ev[ord[j + 1]]) {
        int t = ord[j];
        ord[j] = ord[j + 1];
        ord[j + 1] = t;
      }
  double s1 = ev[ord[0]], s2 = ev[ord[1]], s3 = ev[ord[2]];

  double f13 = (s1 - s3) + (s1 + s3) * sphi - 2.0 * c * cphi;
  if (!(f13 > 0.0)) {
    for (int i = 0; i < 6; ++i) sig_out[i] = sig_tr[i];
    if (depsp) *depsp = 0.0;
    return 0;
  }

  /* D N for the three plastic potentials (principal components):
   *   Na = (1+sp, 0, -(1-sp))   plane s1-s3 (main)
   *   Nb = (0, 1+sp, -(1-sp))   plane s2-s3 (edge with s1 = s2)
   *   Nc = (1+sp, -(1-sp), 0)   plane s1-s2 (edge with s2 = s3)
   * D N = lam tr(N) 1 + 2 G N,  tr N = 2 sp. */
  double l2 = 2.0 * lam * spsi;
  double DNa[3] = {l2 + 2.0 * G * (1.0 + spsi), l2, l2 - 2.0 * G * (1.0 - spsi)};
  double DNb[3] = {l2, l2 + 2.0 * G * (1.0 + spsi), l2 - 2.0 * G * (1.0 - spsi)};
  double DNc[3] = {l2 + 2.0 * G * (1.0 + spsi), l2 - 2.0 * G * (1.0 - spsi), l2};
  /* a = dfa . D Na ; the same for b and c (all planes share it) */
  double a = 4.0 * G * (1.0 + sphi * spsi) + 4.0 * lam * sphi * spsi;

  double r[3];
  int branch;
  /* main plane */
  double dg = f13 / a;
  for (int i = 0; i < 3; ++i) r[i] = (i == 0 ? s1 : i == 1 ? s2 : s3) - dg * DNa[i];
  branch = 1;
  if (!(r[0] >= r[1] && r[1] >= r[2])) {
    /* which ordering is lost first along the main-plane return decides the
     * edge: gap12 closes at rate 2G(1+sp), gap23 at 2G(1-sp). */
    double crit = (1.0 - spsi) * (s1 - s2) - (1.0 + spsi) * (s2 - s3);
    double fa = f13;
    if (crit <= 0.0) {
      /* edge s1 = s2: planes a (1-3) and b (2-3) */
      double fb = (s2 - s3) + (s2 + s3) * sphi - 2.0 * c * cphi;
      double b = 4.0 * lam * sphi * spsi + 2.0 * G * (1.0 - sphi) * (1.0 - spsi);
      double det = a * a - b * b;
      double ga = (a * fa - b * fb) / det, gb = (a * fb - b * fa) / det;
      double tr[3] = {s1, s2, s3};
      for (int i = 0; i < 3; ++i) r[i] = tr[i] - ga * DNa[i] - gb * DNb[i];
      branch = 2;
      if (sphi > 0.0 && !(r[0] >= r[2])) branch = 4;
    } else {
      /* edge s2 = s3: planes a (1-3) and c (1-2) */
      double fc = (s1 - s2) + (s1 + s2) * sphi - 2.0 * c * cphi;
      double b = 4.0 * lam * sphi * spsi + 2.0 * G * (1.0 + sphi) * (1.0 + spsi);
      double det = a * a - b * b;
      double ga = (a * fa - b * fc) / det, gc = (a * fc - b * fa) / det;
      double tr[3] = {s1, s2, s3};
      for (int i = 0; i < 3; ++i) r[i] = tr[i] - ga * DNa[i] - gc * DNc[i];
      branch = 3;
      if (sphi > 0.0 && !(r[0] >= r[2])) branch = 4;
    }
    if (branch == 4) {
      double pa = c * cphi / sphi; /* apex at c cot(phi) */
      r[0] = r[1] = r[2] = pa;
    }
  }

  if (branch == 4) {
    sig_out[0] = sig_out[1] = sig_out[2] = r[0];
    sig_out[3] = sig_out[4] = sig_out[5] = 0.0;
  } else {
    for (int i = 0; i < 6; ++i) sig_out[i] = 0.0;
    for (int i = 0; i < 3; ++i) {
      int e = ord[i];
      double n0 = V[0 + e], n1 = V[3 + e], n2 = V[6 + e];
      sig_out[0] += r[i] * n0 * n0;
      sig_out[1] += r[i] * n1 * n1;
      sig_out[2] += r[i] * n2 * n2;
      sig_out[3] += r[i] * n0 * n1;
      sig_out[4] += r[i] * n1 * n2;
      sig_out[5] += r[i] * n0 * n2;
    }
  }
  if (depsp) {
    double ds[3] = {s1 - r[0], s2 - r[1], s3 - r[2]};
    double sq = 0.0;
    for (int i = 0; i < 3; ++i) {
      double e = (ds[i] - nu * (ds[(i + 1) % 3] + ds[(i + 2) % 3])) / E;
      sq += e * e;
    }
    *depsp = sqrt(2.0 / 3.0 * sq);
  }
  return branch;
}

/* sigma <- sigma + D : de (trial), then the material's return.  Plane stress
 * (R8): lambda* = 2 lambda G / (lambda + 2 G), and sigma_zz stays 0. */
static void stress_update(const om_material *mat, double coh, double sig[6], const double de[6],
                          double *epsp) {
  double G = mat->E / (2.0 * (1.0 + mat->nu));
  double lam = mat->E * mat->nu / ((1.0 + mat->nu) * (1.0 - 2.0 * mat->nu));
  if (mat->model == OM_PLANE_STRESS_ELASTIC) {
    double ls = 2.0 * lam * G / (lam + 2.0 * G);
    double tr2 = de[0] + de[1];
    sig[0] += ls * tr2 + 2.0 * G * de[0];
    sig[1] += ls * tr2 + 2.0 * G * de[1];
    sig[2] = 0.0;
    sig[3] += 2.0 * G * de[3];
    return;
  }
  double tr = de[0] + de[1] + de[2];
  double st[6];
  for (int i = 0; i < 3; ++i) st[i] = sig[i] + lam * tr + 2.0 * G * de[i];
  for (int i = 3; i < 6; ++i) st[i] = sig[i] + 2.0 * G * de[i];
  if (mat->model == OM_MOHR_COULOMB) {
    double d = 0.0;
    oracle_mc_return(mat->E, mat->nu, mat->phi, mat->psi, coh, st, sig, &d);
    *epsp += d;
  } else {
    for (int i = 0; i < 6; ++i) sig[i] = st[i];
  }
}

/* Exposed: one material-point stress update from a strain increment. */
void oracle_stress_update(const om_material *mat, double coh, double sig[6], const double de[6],
                          double *epsp) {
  stress_update(mat, coh, sig, de, epsp);
}

/* ------------------------------------------------------------------------ */
/* The explicit step                                                        */
/* ------------------------------------------------------------------------ */

static int finite6(const double *s) {
  for (int i = 0; i < 6; ++i)
    if (!isfinite(s[i])) return 0;
  return 1;
}

/* Strain increment from the nodal velocity field vel (3 per node):
 *   L_jk = sum_a vel_a,j dN_a/dx_k ;  de = dt (L + L^T) / 2  (Voigt, tensor
 * shear).  In 2D only the in-plane components are non-zero (R7). */
static void strain_increment(const om_mesh *M, int mapped, const int32_t cell[3], const double dN[24],
                             const double *vel, double de[6]) {
  double L[3][3] = {{0}};
  int nn = 1 << M->dim;
  for (int a = 0; a < nn; ++a) {
    int64_t i = cell_node(M, cell, a);
    for (int j = 0; j < M->dim; ++j)
      for (int k = 0; k < M->dim; ++k)
        L[j][k] += mapped ? vel[3 * i + j] * dN[3 * a + k] : vel[3 * i + j] * dN[3 * a + k] * 2.0 / M->h;
  }
  de[0] = L[0][0] * M->dt;
  de[1] = L[1][1] * M->dt;
  de[2] = L[2][2] * M->dt;
  de[3] = 0.5 * (L[0][1] + L[1][0]) * M->dt;
  de[4] = 0.5 * (L[1][2] + L[2][1]) * M->dt;
  de[5] = 0.5 * (L[0][2] + L[2][0]) * M->dt;
}

static void material_point_update(const om_mesh *M, const om_material *mat, double coh,
                                  const double de[6], double *sig, double *eps, double *vol,
                                  double *epsp) {
  for (int i = 0; i < 6; ++i) eps[i] += de[i];
  *vol *= 1.0 + de[0] + de[1] + de[2];
  stress_update(mat, coh, sig, de, epsp);
  (void)M;
}

/* Force of the face tractions on node ijk (R9): for every face f the node
 * lies on, traction_f times the node's tributary length (area): h per
 * tangent axis of the face, h / 2 where the node is at the face's edge. */
static void face_force(const om_mesh *M, const int ijk[3], int faces, double ft[3]) {
  ft[0] = ft[1] = ft[2] = 0.0;
  for (int f = 0; f < 2 * M->dim; ++f) {
    if (!(faces >> f & 1)) continue;
    double trib = 1.0;
    for (int k = 0; k < M->dim; ++k) {
      if (k == f / 2) continue;
      trib *= (ijk[k] == 0 || ijk[k] == M->n[k]) ? 0.5 * M->h : M->h;
    }
    for (int k = 0; k < 3; ++k) ft[k] += M->face_traction[f][k] * trib;
  }
}

/* R13: the force of the face stresses on node ijk of a mapped 2D mesh, added
 * to ft -- for each face f of the node and each boundary edge e of f at the
 * node: sigma_f . (n_e |e|) / 2, n_e |e| the edge vector turned outward. */
static void face_stress_force(const om_mesh *M, const double *X, const int ijk[3], int faces, double ft[3]) {
  if (M->dim != 2) return;
  const double *x0 = X + 3 * node_index(M, ijk);
  for (int f = 0; f < 4; ++f) {
    if (!(faces >> f & 1)) continue;
    const double *S = M->face_stress[f]; /* xx yy zz xy yz xz */
    if (S[0] == 0.0 && S[1] == 0.0 && S[3] == 0.0) continue;
    const int k = f / 2, t = 1 - k;
    int in3[3] = {ijk[0], ijk[1], 0};
    in3[k] += (f & 1) ? -1 : 1;
    const double *xin = X + 3 * node_index(M, in3);
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      int nb[3] = {ijk[0], ijk[1], 0};
      nb[t] += sgn;
      if (nb[t] < 0 || nb[t] > M->n[t]) continue;
      const double *xb = X + 3 * node_index(M, nb);
      double q0 = xb[1] - x0[1], q1 = -(xb[0] - x0[0]); /* the edge turned, |q| = |e| */
      if (q0 * (xin[0] - x0[0]) + q1 * (xin[1] - x0[1]) > 0.0) {
        q0 = -q0;
        q1 = -q1;
      }
      ft[0] += 0.5 * (S[0] * q0 + S[3] * q1);
      ft[1] += 0.5 * (S[3] * q0 + S[1] * q1);
    }
  }
}

/* Nodal solve: v = P/m, a = f/m, v' = v + a dt for active nodes (R2); the
 * constraints follow. stage: 0 = velocity only (USF stage one),
 * 1 = USL (v from P), 2 = USF force stage (v already set).  The force
 * includes the face tractions (R9), and the damping (R10) takes alpha v
 * from the acceleration: a = (f + f_traction) / m - alpha v. */
static void node_solve(const om_mesh *M, const double *X, double *nm, double *nP, double *nf, double *nv,
                       double *na, double *nvn, int stage) {
  int64_t nx = nodes_along(M, 0), ny = nodes_along(M, 1), nz = nodes_along(M, 2);
  for (int64_t kz = 0; kz < nz; ++kz)
    for (int64_t ky = 0; ky < ny; ++ky)
      for (int64_t kx = 0; kx < nx; ++kx) {
        int ijk[3] = {(int)kx, (int)ky, (int)kz};
        int64_t i = node_index(M, ijk);
        int faces = node_faces(M, ijk);
        int active = nm[i] > M->mass_tol;
        double *v = nv + 3 * i, *a = na + 3 * i, *vn = nvn + 3 * i;
        if (stage == 0) {
          for (int k = 0; k < 3; ++k) v[k] = active ? nP[3 * i + k] / nm[i] : 0.0;
          if (X && faces)
            constrain_velocity_mapped(M, X, faces, ijk, v);
          else
            constrain_velocity(M, faces, v);
          continue;
        }
        double ft[3];
        face_force(M, ijk, faces, ft);
        if (X && faces) face_stress_force(M, X, ijk, faces, ft);
        for (int k = 0; k < 3; ++k) {
          if (stage == 1) v[k] = active ? nP[3 * i + k] / nm[i] : 0.0;
          a[k] = active ? (nf[3 * i + k] + ft[k]) / nm[i] - M->damping * v[k] : 0.0;
          vn[k] = active ? v[k] + a[k] * M->dt : 0.0;
        }
        if (!active) {
          for (int k = 0; k < 3; ++k) v[k] = a[k] = vn[k] = 0.0;
          continue;
        }
        if (X && faces)
          constrain_full_mapped(M, X, faces, ijk, v, a, vn);
        else
          constrain_full(M, faces, v, a, vn);
      }
}

/* One explicit step.  USL: reset, P2G (m, P, f), nodal solve with
 * constraints, then per particle FLIP velocity, position, strain from v',
 * stress, volume and relocation.  USF: reset, P2G (m, P), nodal velocity
 * with velocity constraints, per particle strain from that velocity and
 * stress, P2G of forces from the new stress, nodal acceleration with the
 * full constraints, then per particle FLIP velocity, position, relocation.
 */
static int step_once(const om_mesh *M, const double *X, int32_t *pcell, const om_material *mat, int64_t np,
                     double *x, double *v, double *sig, double *eps, const double *m, double *vol, double *epsp,
                     const double *coh, int32_t *alive, double *work) {
  int64_t N = oracle_num_nodes(M);
  double *nm = work, *nP = work + N, *nf = work + 4 * N, *nv = work + 7 * N, *na = work + 10 * N,
         *nvn = work + 13 * N;
  memset(work, 0, sizeof(double) * 16 * N);
  int status = OM_OK;
  int nn = 1 << M->dim;

  if (M->scheme == OM_USL) {
    p2g(M, X, pcell, np, x, v, sig, m, vol, alive, nm, nP, nf, 1, 1);
    node_solve(M, X, nm, nP, nf, nv, na, nvn, 1);
  } else {
    p2g(M, X, pcell, np, x, v, sig, m, vol, alive, nm, nP, nf, 1, 0);
    node_solve(M, X, nm, nP, nf, nv, na, nvn, 0);
    for (int64_t p = 0; p < np; ++p) {
      if (!alive[p]) continue;
      int32_t cell[3];
      double N8[8], dN[24], de[6];
      if (particle_basis(M, X, pcell, p, x + 3 * p, cell, N8, dN) != OM_OK) continue;
      strain_increment(M, X != NULL, cell, dN, nv, de);
      material_point_update(M, mat, coh ? coh[p] : mat->c, de, sig + 6 * p, eps + 6 * p, vol + p,
                            epsp + p);
    }
    p2g(M, X, pcell, np, x, v, sig, m, vol, alive, nm, nP, nf, 0, 1);
    node_solve(M, X, nm, nP, nf, nv, na, nvn, 2);
  }

  for (int64_t p = 0; p < np; ++p) {
    if (!alive[p]) continue;
    int32_t cell[3];
    double N8[8], dN[24];
    if (particle_basis(M, X, pcell, p, x + 3 * p, cell, N8, dN) != OM_OK) continue;
    double dv[3] = {0, 0, 0}, vb[3] = {0, 0, 0};
    for (int a = 0; a < nn; ++a) {
      int64_t i = cell_node(M, cell, a);
      for (int k = 0; k < 3; ++k) {
        dv[k] += N8[a] * na[3 * i + k];
        vb[k] += N8[a] * nvn[3 * i + k];
      }
    }
    if (M->scheme == OM_USL) {
      double de[6];
      strain_increment(M, X != NULL, cell, dN, nvn, de);
      material_point_update(M, mat, coh ? coh[p] : mat->c, de, sig + 6 * p, eps + 6 * p, vol + p,
                            epsp + p);
    }
    for (int k = 0; k < M->dim; ++k) {
      v[3 * p + k] += M->dt * dv[k];
      x[3 * p + k] += M->dt * vb[k];
    }
    int32_t c2[3];
    double xi2[3];
    int where;
    if (X) {  /* the neighbourhood walk from the particle's cell */
      for (int k = 0; k < 3; ++k) c2[k] = cell[k];
      where = oracle_iso_locate(M, X, x + 3 * p, c2, xi2);
      if (where == OM_OK)
        for (int k = 0; k < 3; ++k) pcell[3 * p + k] = c2[k];
    } else {
      where = oracle_locate(M, x + 3 * p, c2, xi2);
    }
    if (where != OM_OK) {
      alive[p] = 0;
      status = OM_LEFT_MESH;
    }
    if (!finite6(sig + 6 * p) || !isfinite(v[3 * p]) || !isfinite(v[3 * p + 1]) ||
        !isfinite(v[3 * p + 2]))
      if (status == OM_OK) status = OM_NONFINITE;
  }
  return status;
}

/* Run nsteps explicit steps in place.  work: oracle_work_size(M) doubles.
 * coh: per-particle cohesion or NULL for the material's c.  Returns the
 * first non-OK status seen (particles that left the mesh are marked dead
 * and the run continues), or OM_ARG on a malformed mesh. */
int oracle_step(const om_mesh *M, const om_material *mat, int64_t np, double *x, double *v,
                double *sig, double *eps, const double *m, double *vol, double *epsp,
                const double *coh, int32_t *alive, double *work, int64_t nsteps) {
  if (!M || !mat || (M->dim != 2 && M->dim != 3) || M->h <= 0.0 || M->dt <= 0.0) return OM_ARG;
  int status = OM_OK;
  for (int64_t s = 0; s < nsteps; ++s) {
    int st = step_once(M, NULL, NULL, mat, np, x, v, sig, eps, m, vol, epsp, coh, alive, work);
    if (status == OM_OK) status = st;
  }
  return status;
}

/* The same steps on a mapped mesh (node coordinates X, 3 per node): pcell
 * (3 per particle) holds each particle's cell, located beforehand with
 * oracle_iso_locate and kept up to date by the walk after advection. */
int oracle_step_mapped(const om_mesh *M, const double *X, const om_material *mat, int64_t np, double *x,
                       double *v, double *sig, double *eps, const double *m, double *vol, double *epsp,
                       const double *coh, int32_t *alive, int32_t *pcell, double *work, int64_t nsteps) {
  if (!M || !X || !pcell || !mat || (M->dim != 2 && M->dim != 3) || M->dt <= 0.0) return OM_ARG;
  for (int f = 0; f < 6; ++f)  /* R12 */
    for (int k = 0; k < 3; ++k)
      if (M->face_traction[f][k] != 0.0) return OM_ARG;
  for (int f = 0; f < 6; ++f)  /* R13: 2D only */
    for (int k = 0; k < 6; ++k)
      if (M->face_stress[f][k] != 0.0 && M->dim != 2) return OM_ARG;
  int status = OM_OK;
  for (int64_t s = 0; s < nsteps; ++s) {
    int st = step_once(M, X, pcell, mat, np, x, v, sig, eps, m, vol, epsp, coh, alive, work);
    if (status == OM_OK) status = st;
  }
  return status;
}

/* Global sums over live particles: out[0] mass, out[1..3] momentum,
 * out[4] kinetic energy, out[5] elastic strain energy sum 1/2 V sigma:eps,
 * out[6] number of live particles. */
void oracle_conservation(int64_t np, const double *v, const double *sig, const double *eps,
                         const double *m, const double *vol, const int32_t *alive, double out[7]) {
  for (int i = 0; i < 7; ++i) out[i] = 0.0;
  for (int64_t p = 0; p < np; ++p) {
    if (!alive[p]) continue;
    out[0] += m[p];
    double ke = 0.0;
    for (int k = 0; k < 3; ++k) {
      out[1 + k] += m[p] * v[3 * p + k];
      ke += v[3 * p + k] * v[3 * p + k];
    }
    out[4] += 0.5 * m[p] * ke;
    const double *s = sig + 6 * p, *e = eps + 6 * p;
    double se = s[0] * e[0] + s[1] * e[1] + s[2] * e[2] + 2.0 * (s[3] * e[3] + s[4] * e[4] + s[5] * e[5]);
    out[5] += 0.5 * vol[p] * se;
    out[6] += 1.0;
  }
}
