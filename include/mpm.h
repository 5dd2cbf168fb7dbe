/*
 * mpm.h -- C ABI of the GB300 explicit material point method library
 * (libmpm.so).  Plain C types only: no C++ or PyTorch types cross it.
 *
 * The operation is one explicit MPM time step as described in Kumar et al.,
 * "Scalable and modular material point method for large-scale simulations"
 * (arXiv 1909.13380):
 *   INTRODUCTION   particles carry all state; the equations are solved on the
 *                  nodes of a fixed background mesh, whose nodal values are
 *                  reset every step; particle->node and node->particle
 *                  transfers use the same shape functions.
 *   CODE OVERVIEW  Node (mass, momentum, velocity, acceleration, forces;
 *                  persistent friction/velocity constraints), Cell with the
 *                  linear 4-node quadrilateral / 8-node hexahedron, Material
 *                  (stress from a strain increment), Mesh, and the explicit
 *                  USF / USL algorithms.
 *   DATA STRUCTURES  6-component Voigt stress/strain.
 *   ISOPARAMETRIC MESH  nodal velocity and frictional boundary conditions;
 *                  locating particles in cells.
 * The paper prints no equations; the library computes the textbook explicit
 * MPM (Sulsky et al. 1994; USF/USL after Bardenhagen 2002) with a
 * Mohr-Coulomb return in principal stresses (de Souza Neto et al. 2008).
 *
 * Conventions
 *   - Faces are numbered -x, +x, -y, +y, -z, +z.  Vectors have `dim`
 *     components; stresses and strains have 6 Voigt components
 *     (xx, yy, zz, xy, yz, xz) with tensor (not engineering) shear strain,
 *     also in 2D (plane strain: strain zz = 0, stress zz kept; yz = xz = 0).
 *   - Tension is positive.  Angles are in radians.
 *   - Cells are Cartesian cubes/squares of side h; node (i,j,k) sits at
 *     origin + (i,j,k) h.  A particle's cell is floor((x - origin)/h) per
 *     axis; a particle on a face belongs to the higher cell, and one at or
 *     beyond the upper mesh bound has left the mesh.
 *   - Host pointers are copied; the caller keeps ownership.  The library
 *     owns all device memory of a handle and frees it in mpm_destroy.
 *   - Every call returns an mpm_status.  MPM_ERR_ARG and MPM_ERR_STATE (a
 *     call rejected before it did anything) leave the handle as it was;
 *     every other error is sticky per handle until mpm_destroy.
 *     mpm_last_error gives a message.  Device-side conditions
 *     (a particle left the mesh, a non-finite value) are latched in a device
 *     status word and reported at the next synchronising call.
 *   - A handle is not thread-safe; different handles may be used from
 *     different host threads.
 */
#ifndef MPM_GB300_H
#define MPM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpm_ctx *mpm_handle;

typedef enum {
  MPM_OK = 0,
  MPM_ERR_ARG = -1,       /* malformed argument; nothing was changed */
  MPM_ERR_OOM = -2,       /* device allocation failed */
  MPM_ERR_CUDA = -3,      /* a CUDA runtime call or launch failed */
  MPM_ERR_LEFT_MESH = -4, /* a particle left the mesh; it is dropped from the step */
  MPM_ERR_NONFINITE = -5, /* a particle state became NaN/Inf */
  MPM_ERR_TIMEOUT = -6,   /* a bounded device wait gave up */
  MPM_ERR_STATE = -7      /* call not valid in the handle's current state */
} mpm_status;

enum { MPM_BC_FREE = 0, MPM_BC_ROLLER = 1, MPM_BC_FIXED = 2, MPM_BC_FRICTION = 3 };
enum { MPM_USF = 0, MPM_USL = 1 };
enum { MPM_FP64_PLAIN = 0, MPM_FP32_MIXED = 1 };
enum { MPM_LINEAR_ELASTIC = 0, MPM_MOHR_COULOMB = 1, MPM_PLANE_STRESS_ELASTIC = 2 };

/* Background mesh and step parameters (CODE OVERVIEW: Mesh, Node, Cell;
 * the explicit USF/USL algorithm).
 *   dim        2 (4-node quads, plane strain) or 3 (8-node hexahedra)
 *   ncells     cells per axis (ncells[2] ignored in 2D); each >= 1
 *   h          cell size (> 0); origin: coordinates of node (0,0,0)
 *   face_bc    per face: MPM_BC_FREE / ROLLER (normal velocity 0) /
 *              FIXED (all velocity 0) / FRICTION (Coulomb, coefficient
 *              face_mu; contact only while the node moves into the face)
 *   gravity    body acceleration; dt: time step (> 0)
 *   scheme     MPM_USF or MPM_USL
 *   precision  MPM_FP64_PLAIN: FP64 global positions, unsorted particles,
 *              FP64 atomics on a dense node grid.
 *              MPM_FP32_MIXED: FP32 state with each position held as an
 *              integer cell plus an FP32 offset, particles binned by cell
 *              every step, deterministic tile reductions with compensated
 *              sums, FP64 only in the Mohr-Coulomb return near the apex and
 *              in the conservation sums.
 *   mass_tol   a node is active when its mass exceeds this (e.g. 1e-12 kg)
 *   stream     cudaStream_t to enqueue on (NULL: the handle creates its own
 *              non-blocking stream and destroys it in mpm_destroy) */
typedef struct {
  int32_t dim;
  int32_t ncells[3];
  double h;
  double origin[3];
  int32_t face_bc[6];
  double face_mu[6];
  double gravity[3];
  double dt;
  int32_t scheme;
  int32_t precision;
  double mass_tol;
  void *stream;
} mpm_mesh_desc;

/* Material of the particles (CODE OVERVIEW: Material).  Linear elastic uses
 * E, nu; Mohr-Coulomb adds friction angle phi, cohesion c and dilation
 * angle psi (perfect plasticity).  MPM_PLANE_STRESS_ELASTIC (2D meshes only;
 * BENCHMARK AND PERFORMANCE: the plate with a hole is a plane-stress strip)
 * is linear elastic with stress zz = 0: in-plane stiffness with
 * lambda* = 2 lambda G / (lambda + 2 G).  rho gives particle mass
 * rho * volume. */
typedef struct {
  int32_t model;
  double E, nu, rho;
  double phi, c, psi;
} mpm_material;

/* Create a mesh.  Validates desc (MPM_ERR_ARG on nonsense) and allocates the
 * node/tile storage on the current CUDA device.  *out receives the handle. */
mpm_status mpm_create_mesh(const mpm_mesh_desc *desc, mpm_handle *out);

/* Add n particles (CODE OVERVIEW: material points with a Material).
 *   pos, vel   n*dim doubles, row-major (host)
 *   vol        n doubles, initial volume (area per unit thickness in 2D)
 *   mat        material; every call on a handle must pass the same one
 *   cohesion   n doubles overriding mat->c per particle, or NULL
 *   stress0    n*6 initial stresses, or NULL for zero
 *   first_id   out: id of the first new particle (ids are 0,1,2,... in
 *              insertion order), may be NULL
 * Particles outside the mesh (or with a non-finite position) are rejected
 * (MPM_ERR_ARG, none added, the mesh unchanged).  The initial cell is
 * computed in FP64 by the rule above: on the host for FP64_PLAIN, on the
 * device for FP32_MIXED (the inputs are copied up once and every FP32 field
 * is formed there).  The host arrays are only read during the call.  Must
 * not be called while steps are in flight (it synchronises the stream). */
mpm_status mpm_add_particles(mpm_handle h, int64_t n, const double *pos, const double *vel,
                             const double *vol, const mpm_material *mat, const double *cohesion,
                             const double *stress0, int64_t *first_id);

/* Mapped (isoparametric) mesh (ISOPARAMETRIC MESH: cells that follow
 * non-prismatic geometry such as a landslide's terrain), FP64_PLAIN and
 * FP32_MIXED handles, before the first mpm_add_particles and outside a
 * batch (MPM_ERR_STATE otherwise).
 *   node_xyz   host, (nodes, dim) row-major doubles: the coordinates of node
 *              ix + (nx+1) (iy + (ny+1) iz) -- the logical grid of
 *              mpm_mesh_desc keeps its cells, only the nodes move.  Read
 *              during the call; the handle keeps a device copy.
 * Every cell must keep the orientation of the logical grid (the Jacobian
 * determinant of its map positive at each corner) and the coordinates must
 * be finite (MPM_ERR_ARG, nothing changed).  A cell is then the image of
 * [-1, 1]^dim under x(xi) = sum_a N_a(xi) X_a, and:
 *   - a particle's natural coordinates are the root of x(xi) = x; shape
 *     gradients are dN/dx = dN/dxi J^-1;
 *   - mpm_add_particles locates new particles by a neighbourhood walk from
 *     the Cartesian cell of desc.origin and desc.h (which serve no other
 *     purpose on a mapped mesh), solving for xi by Newton-Raphson from the
 *     inverse bilinear solution (2D) or the affine guess (3D), in FP64; a
 *     particle in no cell rejects the call (MPM_ERR_ARG, none added);
 *   - each step, after advection, a particle moves from its cell to the
 *     neighbour across the face its natural coordinates leave by until they
 *     lie in [-1, 1) (xi = 1 belongs to the next cell); a particle that
 *     would leave the grid has left the mesh (MPM_ERR_LEFT_MESH).  FP64:
 *     the walk above from the new position.  FP32_MIXED: the offset is
 *     xi / 2 and every cell holds its corners relative to its centre in
 *     FP32 (rounded once from FP64); the particle's new offset is solved in
 *     the frame of its own cell and carried into each neighbour's frame
 *     through the node they share, at most 8 cells per step (beyond that
 *     the particle is dropped as having left the mesh);
 *   - face conditions act along each face's outward normal at the node
 *     (nodal conditions on irregular surfaces): the normals of the boundary
 *     facets next to the node (2D edges, weighted by length; 3D bilinear
 *     facets, the cross product of their edges at the node) summed and
 *     normalised.  A roller removes the velocity along the node's roller
 *     normals (made orthonormal in face order: -x,+x,-y,+y,-z,+z); a
 *     friction face applies the Coulomb rule to w = n . v' and the part of
 *     v' tangent to n; a fixed face zeroes the velocity.  Face tractions are
 *     not defined: mpm_set_loads rejects them, and a mesh that carries them
 *     rejects this call (MPM_ERR_ARG).  Damping is allowed;
 *   - in a batch, mapped and Cartesian meshes step in groups of their own
 *     kind; every mesh's result is the same as stepping it alone.
 * mpm_read_particles' position is x(xi) of the particle's cell and its cell
 * the walk's.  mpm_footprint does not include the mapped storage: 24 bytes
 * per node, and per particle 4 + 8 dim (FP64_PLAIN), or per cell 32 (2D) or
 * 96 (3D) bytes (FP32_MIXED).  Calling it again before the first particles
 * replaces the coordinates. */
mpm_status mpm_set_node_coordinates(mpm_handle h, const double *node_xyz);

/* Far-field stresses on the faces of a mapped 2D mesh (BENCHMARK AND
 * PERFORMANCE: the plate's uniform tension at its ends, where one logical
 * face of a mesh fitted to the hole runs along the loaded end and a free
 * edge).  face_stress: host, 6 faces (-x,+x,-y,+y,-z,+z) x 6 Voigt
 * components (xx, yy, zz, xy, yz, xz), read during the call; NULL clears.
 * The load of face f is the traction sigma_f . n of that uniform stress on
 * each boundary edge of the face, lumped half to each end node (n the edge's
 * outward normal): node a gets sum over its edges e of sigma_f . n_e |e| / 2.
 * Added to the nodal force like the tractions of mpm_set_loads (whose
 * damping applies too).  Mapped 2D meshes only, after
 * mpm_set_node_coordinates (MPM_ERR_ARG otherwise; a Cartesian face takes
 * sigma . n as a traction through mpm_set_loads); MPM_ERR_STATE while the
 * mesh is admitted to a batch.  mpm_set_node_coordinates is not valid once
 * face stresses are set (MPM_ERR_STATE). */
mpm_status mpm_set_face_stress(mpm_handle h, const double *face_stress);

/* Enqueue nsteps explicit steps on desc.stream and return without waiting.
 * Returns a latched error, if any, or MPM_OK.  Zero particles is valid. */
mpm_status mpm_step(mpm_handle h, int64_t nsteps);

/* Wait for enqueued work and return the latched device status. */
mpm_status mpm_sync(mpm_handle h);

/* Number of particles added so far (live or not). */
mpm_status mpm_num_particles(mpm_handle h, int64_t *n);

/* Copy particle state to host arrays in insertion order (synchronises).
 * Any pointer may be NULL.  pos/vel: n*dim; stress/strain: n*6; vol, epsp
 * (accumulated equivalent plastic strain): n; cell: n linear cell ids
 * ix + nx*(iy + ny*iz), -1 for particles that left the mesh. */
mpm_status mpm_read_particles(mpm_handle h, double *pos, double *vel, double *stress,
                              double *strain, double *vol, double *epsp, int64_t *cell);

/* FP64 global sums over live particles (deterministic order): out[0] mass,
 * out[1..3] momentum, out[4] kinetic energy, out[5] strain energy
 * sum 1/2 V sigma:eps, out[6] number of live particles, out[7] total volume
 * sum V.  Synchronises. */
mpm_status mpm_conservation(mpm_handle h, double out[8]);

/* Particle binning (step a1 of the path; ISOPARAMETRIC MESH: locating the
 * particles in cells), FP32_MIXED handles only.  Runs the binning of the
 * current particle storage and copies to the host: key[n] the binning key of
 * each stored particle (tile-major cell id, see below; dead particles carry
 * the largest key) and perm[n] the stable sort permutation (perm[q] is the
 * storage slot of the q-th particle in key order; ties keep storage order).
 * Tile-major key: tiles of TX x TY x TZ cells (8 x 8 in 2D, 4 x 4 x 4 in
 * 3D), tile t = tx + NTX*(ty + NTY*tz), local l = lx + TX*(ly + TY*lz),
 * key = t * (TX*TY*TZ) + l; dead key = NT * (TX*TY*TZ).  tile_dims receives
 * (TX, TY, TZ) if not NULL. */
mpm_status mpm_read_binning(mpm_handle h, int32_t *key, int32_t *perm, int32_t *tile_dims);

/* Per-phase device timing of the FP32_MIXED step (measurement support; the
 * paper reports wall times only, BENCHMARK AND PERFORMANCE).  When enabled,
 * every enqueued step records CUDA events (cudaEventRecordExternal, so they
 * also fire inside the captured step graph) at its phase boundaries.
 * mpm_phase_times synchronises and writes the durations in milliseconds of
 * the most recent step's phases to ms[0..*nphase-1]:
 *   USL (4): binning, P2G, nodal solve, G2P (+ carry of dead particles)
 *   USF (7): binning, P2G mass/momentum, nodal velocity, G2P stress,
 *            P2G internal force, nodal solve, G2P advection
 * With cohesion, a G2P phase that updates stresses includes the FP64
 * apex-band return that follows it.  The event nodes also serialise the
 * step's kernels (which otherwise overlap their launches), so the phases
 * add up to more than an untimed step.  ms must hold MPM_MAX_PHASES floats.
 * MPM_ERR_STATE on FP64_PLAIN handles or when timing is off or no step ran
 * since it was enabled. */
#define MPM_MAX_PHASES 8
mpm_status mpm_set_phase_timing(mpm_handle h, int32_t enable);
mpm_status mpm_phase_times(mpm_handle h, float *ms, int32_t *nphase);

/* Estimated device bytes a FP32_MIXED or FP64_PLAIN mesh of desc holding n
 * particles (with per-particle cohesion if has_cohesion) allocates; for
 * admission control by free memory. */
mpm_status mpm_footprint(const mpm_mesh_desc *desc, int64_t n, int32_t has_cohesion, int64_t *bytes);

/* ---- batched steps of independent meshes (serving) ---------------------
 * A batch advances many independent FP32_MIXED meshes together: every phase
 * of the step is one kernel launch over all admitted meshes (their tiles and
 * particles form one work list), and a batched step is one CUDA graph
 * replay.  Meshes share no data, so each mesh's result is bit-identical to
 * stepping it alone.  The paper has no batching; it runs one simulation per
 * process (CODE OVERVIEW, DATA STRUCTURES).
 *   mpm_batch_create   hbm_budget_bytes: device bytes the admitted meshes may
 *                      hold together, counted as mpm_footprint of each mesh
 *                      at its admission (0: no memory budget); max_slots:
 *                      most meshes admitted at once (>= 1); stream:
 *                      cudaStream_t for all batch work (NULL: a private
 *                      stream).  MPM_ERR_ARG for a negative budget or
 *                      max_slots < 1.
 *   mpm_batch_admit    adds an idle FP32_MIXED mesh (its pending work is
 *                      finished first); from then on the mesh's own calls
 *                      run on the batch stream and mpm_step on it returns
 *                      MPM_ERR_STATE until it is evicted.  *slot receives a
 *                      stable slot id in 0..max_slots-1.  MPM_ERR_OOM when
 *                      every slot is taken or the mesh's footprint exceeds
 *                      what the budget has left; the mesh and the batch are
 *                      then unchanged and the error is not latched on the
 *                      mesh (admit it later, after an eviction).
 *   mpm_batch_room     what is left: *free_bytes of the budget (INT64_MAX
 *                      without a budget) and *free_slots; either may be NULL.
 *   mpm_batch_evict    removes the mesh of a slot (after the batch's pending
 *                      work) and returns its footprint to the budget; the
 *                      mesh keeps its state and can be read, stepped alone or
 *                      admitted again.
 *   mpm_batch_step     enqueues nsteps batched steps of every admitted mesh.
 *   mpm_batch_poll     synchronises and writes, for slots 0..nslots-1, the
 *                      latched status of the slot's mesh (MPM_OK,
 *                      MPM_ERR_LEFT_MESH, MPM_ERR_NONFINITE, MPM_ERR_TIMEOUT)
 *                      or MPM_ERR_STATE for an empty slot, and, if
 *                      slot_steps is not NULL, the batched steps the slot's
 *                      mesh has taken since its admission (-1 for an empty
 *                      slot).
 *   mpm_batch_step_kernels  kernel launches of one batched step: the kernel
 *                      nodes of the last captured batched-step graph
 *                      (MPM_ERR_STATE before the first batched step).
 *   mpm_batch_destroy  evicts every mesh (they stay valid) and frees the batch.
 * A batch is not thread-safe. */
typedef struct mpm_batch_ctx *mpm_batch;
mpm_status mpm_batch_create(int64_t hbm_budget_bytes, int32_t max_slots, void *stream, mpm_batch *out);
mpm_status mpm_batch_admit(mpm_batch b, mpm_handle mesh, int32_t *slot);
mpm_status mpm_batch_room(mpm_batch b, int64_t *free_bytes, int32_t *free_slots);
mpm_status mpm_batch_evict(mpm_batch b, int32_t slot);
mpm_status mpm_batch_step(mpm_batch b, int64_t nsteps);
mpm_status mpm_batch_poll(mpm_batch b, int32_t nslots, int32_t *slot_status, int64_t *slot_steps);
mpm_status mpm_batch_step_kernels(mpm_batch b, int32_t *kernels);
mpm_status mpm_batch_destroy(mpm_batch b);

/* Loads of a quasi-static run (BENCHMARK AND PERFORMANCE: a strip "subjected
 * to uniform tension ... applied at the ends"; the paper gives no protocol
 * for reaching the static state).
 *   face_traction  18 doubles, the traction (force per unit length in 2D,
 *                  per unit area in 3D; dim components used) on each face
 *                  -x,+x,-y,+y,-z,+z, or NULL for none.  It acts on the
 *                  nodes of that mesh face, so the loaded end of the body
 *                  must lie on it: each active node gets the traction times
 *                  its tributary length (area), h per tangent axis, h / 2 at
 *                  the face's own edges.
 *   damping        alpha >= 0 of a mass-proportional viscous damping of the
 *                  nodes, a = (f + f_traction) / m - alpha v, which brings
 *                  an explicit run to rest; 0 for none.
 * Both act from the next step on, in both precisions and both schemes (the
 * USF velocity stage is undamped).  Not for a mesh admitted to a batch.
 * MPM_ERR_ARG for a negative or non-finite value. */
mpm_status mpm_set_loads(mpm_handle h, const double *face_traction, double damping);

/* Failure-detection test hook (the paper has no counterpart).  The FP32
 * tile scan of meshes with more than 4095 tiles runs one pass over chunks of
 * 1024 tiles in which each chunk waits, on the device, for the prefix its
 * predecessors publish; every such wait is bounded and gives up with
 * MPM_ERR_TIMEOUT (latched, reported by mpm_sync) instead of hanging.  This
 * call makes that happen on purpose: chunk withhold_chunk (0-based; -1 = none)
 * never publishes, and a wait polls at most spin_limit times (1..2^20; 2^20
 * is the default).  A mesh whose scan gave up a wait is frozen: from then on
 * its steps carry its particles over unchanged and touch nothing else, and
 * its status stays MPM_ERR_TIMEOUT until mpm_destroy.  Other meshes are not
 * affected.  FP32_MIXED meshes not admitted to a batch; MPM_ERR_ARG for
 * out-of-range values. */
mpm_status mpm_set_scan_fault(mpm_handle h, int32_t withhold_chunk, int32_t spin_limit);

/* Kernel launches one mpm_step of h enqueues (measurement support): the
 * kernel nodes of the step graph the library captured for h, FP32_MIXED
 * only.  MPM_ERR_STATE before the first captured step or for FP64_PLAIN. */
mpm_status mpm_step_kernels(mpm_handle h, int32_t *kernels);

/* Human-readable description of the last error on h (never NULL). */
const char *mpm_last_error(mpm_handle h);

/* Free all device storage of h.  NULL is accepted. */
mpm_status mpm_destroy(mpm_handle h);

/* ---- standalone path primitives ---------------------------------------- */

/* Stable LSD radix sort by key on the device (the binning step a1 as a
 * primitive).  d_keys: n uint32 keys < 2^key_bits (device, unchanged);
 * d_perm: n int32 out (device), perm[q] = index of the q-th smallest key,
 * equal keys in index order.  key_bits in 1..32.  Allocates its scratch with
 * cudaMallocAsync on `stream` and frees it before returning (the call
 * synchronises the stream). */
mpm_status mpm_sort_keys(const uint32_t *d_keys, int32_t *d_perm, int64_t n, int32_t key_bits,
                         void *stream);

/* The same stable key sort as mpm_sort_keys for callers that cannot
 * allocate device memory: for example a host program whose own allocator
 * already holds all of the GPU's free memory, or a loop that must not
 * allocate once it is running.  The paper has no counterpart; this is a
 * service of this library.
 *   The scratch is a fixed array in the library's device memory (about
 *   22 MiB, held on every GPU that loads the library until the process
 *   exits), so this call allocates and frees nothing.  n above
 *   MPM_SORT_STATIC_MAX_KEYS is rejected with MPM_ERR_ARG before any device
 *   work.  Every call looks up the array's device address in the current
 *   device's context (cudaGetSymbolAddress); the first call on a device also
 *   loads the library's device code there, so make that first call before
 *   any stream capture.
 *   The call only enqueues work on `stream` and returns; d_perm is ready
 *   when the stream reaches that point.  All calls share the one array, so
 *   calls whose work overlaps on the GPU (different streams, or different
 *   host threads) race and give wrong results: order them on one stream.
 *   Every scratch word is written before it is read, so nothing needs to
 *   be cleared between calls. */
#define MPM_SORT_STATIC_MAX_KEYS (1 << 20)
mpm_status mpm_sort_keys_static(const uint32_t *d_keys, int32_t *d_perm, int64_t n, int32_t key_bits,
                                void *stream);

/* Material-point stress update on the GPU (CODE OVERVIEW: Material, "the
 * updated stresses for a given strain tensor"), for n independent points.
 *   sig, deps   n*6 host doubles: stress before, strain increment
 *   cohesion    n host doubles or NULL (mat->c)
 *   sig_out     n*6 host doubles out; depsp_out n doubles out (equivalent
 *               plastic strain increment), may be NULL
 *   precision   MPM_FP64_PLAIN computes in FP64; MPM_FP32_MIXED rounds the
 *               inputs to FP32 and computes as the FP32 step does (FP64
 *               only near the Mohr-Coulomb apex).
 * Synchronous; allocates and frees its own device buffers. */
mpm_status mpm_material_update(const mpm_material *mat, int32_t precision, int64_t n,
                               const double *sig, const double *deps, const double *cohesion,
                               double *sig_out, double *depsp_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MPM_GB300_H */
