/*
 * iblb.h -- C ABI of libiblb, a GB300 (sm_103a) implementation of one time
 * step of the immersed-boundary lattice Boltzmann (IBLB) droplet method of
 * Taglienti, Guglietta and Sbragaglia, arXiv:2403.01161:
 *
 *   1. surface-tension nodal forces F_i = -sigma dA/dx_i of the triangulated
 *      droplet (Sec. 3.1, Eq. (pi_drop)), FP64;
 *   2. spreading onto the lattice with the Peskin 4-point delta
 *      (Eq. (ibm_force_d)(a));
 *   3. D3Q19 BGK stream-collide with Guo forcing and half-force momentum
 *      (Eqs. (LBMEQ), (collision), (equilibriumLB), (density_velocity_LB)),
 *      with the Zou-He box boundary imposing u = A(t)(l - L/2) on all wet
 *      boundary nodes (Eqs. (velo_facce_cubo_da_gradiente), (ZH_bulk),
 *      (ZH_edges), (zh-buried-links-edges), (zh-buried-links-corners));
 *   4. interpolation of the fluid velocity to the nodes and forward-Euler
 *      advection (Eq. (ibm_force_d)(b), Eq. (fwd_euler));
 *   5. optional mesh regularisation (Sec. 3.3) and shape readout (Sec. 2,
 *      morphological tensor, lambda_max, Eq. (beta)).
 * Velocity-gradient frames are held a fixed number of steps each (Sec. 3.2).
 *
 * Conventions
 *   - Lattice nodes sit at integer positions 0..n_a-1 per axis; on a Zou-He
 *     axis the planes 0 and n_a-1 are the wet boundary nodes and the box
 *     centre used in the wall velocity is (n_a-1)/2.
 *   - Host arrays are row-major C arrays of double unless stated.  A frame is
 *     9 doubles, A[3*a+b] = du_a/dx_b in lattice units.
 *   - Fields are laid out [component][z][y][x] (x fastest).
 *   - Every call returns an int status: IBL_OK (0) or a negative IBL_E* code;
 *     ibl_last_error() returns a message for the calling thread's last
 *     failure.  Kernel launches are asynchronous on the stream bound at
 *     creation; device-side errors (instability, wall contact,
 *     regularisation not converged) are sticky bits reported by the next
 *     synchronising call (ibl_sync, ibl_readout, ibl_copy_*).
 *   - Ownership: the library never allocates device memory.  Each handle
 *     lives in a caller-provided device workspace (size from the matching
 *     *_workspace_size call, 256-byte aligned, owned by the caller, which
 *     must keep it alive until the handle is destroyed).  Host outputs are
 *     caller-owned.  Handles are not thread safe.
 */
#ifndef IBLB_H
#define IBLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define IBL_ABI_VERSION 1

/* status codes */
#define IBL_OK 0
#define IBL_EINVAL (-1)    /* invalid argument or state */
#define IBL_ENOMEM (-2)    /* workspace smaller than required */
#define IBL_ECUDA (-3)     /* a CUDA runtime call failed */
#define IBL_EUNSTABLE (-4) /* NaN density or |u| > 0.3 on some node */
#define IBL_ENOCONV (-5)   /* mesh regularisation reached max_iter */
#define IBL_EWALL (-6)     /* a droplet node's 4x4x4 stencil reached a wet boundary node */
#define IBL_ETIMEOUT (-7)  /* a kernel gave up waiting for its staged copies (never expected) */

/* sticky device error bits, as in ibl_observables.err */
#define IBL_ERRBIT_UNSTABLE 1
#define IBL_ERRBIT_NOCONV 2
#define IBL_ERRBIT_WALL 4
#define IBL_ERRBIT_TIMEOUT 8

enum { IBL_BC_ZOU_HE = 0, IBL_BC_PERIODIC = 1 };
/* Edge/corner rule, Eqs. (ZH_edges), (zh-buried-links-edges),
 * (zh-buried-links-corners).  IBL_EDGE_COUNTER_SLIP (default): the face
 * rule's construction of Eq. (ZH_bulk) carried to two normals -- the
 * tangential sum with the sign that removes the edge-line momentum, the
 * moving-wall bounce-back term -2 w_i (c_i.u_w)/c_s^2, the wall's edge-line
 * share -(t_i.u_w)/12, and each buried link plus 3 w_j (c_j.u_w) -- so that
 * every edge and corner node carries exactly the momentum u_w (rho0 = 1).
 * IBL_EDGE_PAPER_LITERAL: the equations as printed (minus sign, no wall
 * velocity at edges and corners). */
enum { IBL_EDGE_COUNTER_SLIP = 0, IBL_EDGE_PAPER_LITERAL = 1 };
/* Population storage: FP32 deviations f_i - w_i, or FP64 deviations. */
enum { IBL_FP32_DEV = 0, IBL_FP64 = 1 };

typedef struct ibl_lb ibl_lb;
typedef struct ibl_mesh ibl_mesh;

typedef struct {
    int version;       /* IBL_ABI_VERSION */
    int n[3];          /* lattice nodes per axis, each >= 4 */
    double tau;        /* BGK relaxation time tau_f > 1/2 (nu = (tau - 1/2)/3) */
    int bc[3];         /* IBL_BC_ZOU_HE or IBL_BC_PERIODIC per axis */
    int edge_rule;     /* IBL_EDGE_* */
    int precision;     /* IBL_FP32_DEV or IBL_FP64 */
    int record_fields; /* nonzero: reserve buffers so that ibl_step_record can
                          store density, velocity and force of a step */
} ibl_lb_params;

/* Shape record of the droplet (Sec. 2).  S = (5/V) int (x - x_c)(x - x_c)^T dV
 * over the enclosed polyhedron; lam ascending; vmax the unit eigenvector of
 * lam[2]; D = (sqrt(lam2) - sqrt(lam0))/(sqrt(lam2) + sqrt(lam0)); beta =
 * vmax.E.vmax/|E|_F with E the symmetric part of the frame applied in the
 * last completed step (NaN when |E| = 0). */
typedef struct {
    long long step;    /* steps completed when the record was taken */
    int frame;         /* frame index used for beta */
    int reg_iters;     /* iterations of the latest regularisation, 0 if none */
    int err;           /* IBL_ERRBIT_* at the time of the record */
    int pad_;
    double volume, area;
    double centroid[3];
    double S[6];       /* xx, yy, zz, xy, xz, yz */
    double lam[3];
    double vmax[3];
    double D, beta;
} ibl_observables;

/* ---- lattice --------------------------------------------------------- */

/* Device bytes needed by a lattice with these parameters and n_frames frames. */
int ibl_lb_workspace_size(const ibl_lb_params *p, int n_frames, size_t *bytes);

/* Creates a lattice in `workspace` (device, `bytes` long) bound to `stream`
 * (a cudaStream_t, NULL for the legacy default stream).  A_frames: host,
 * n_frames x 9 doubles, frame k is applied in steps k*steps_per_frame ..
 * (k+1)*steps_per_frame - 1, the last frame held beyond the end (Sec. 3.2
 * trajectory loop).  The initial state is f = f_eq(rho = 1, u = A_0(x - c))
 * at every node.  Copies the frames; the host array may be freed after. */
int ibl_lb_create(const ibl_lb_params *p, const double *A_frames, int n_frames, int steps_per_frame,
                  void *workspace, size_t bytes, void *stream, ibl_lb **out);
void ibl_lb_destroy(ibl_lb *lb);

/* Replaces frame k (0 <= k < n_frames) by 9 host doubles; asynchronous
 * (stream-ordered), so the host array must stay valid until the stream
 * reaches the copy (ibl_sync). */
int ibl_set_frame(ibl_lb *lb, int k, const double *A);

/* ---- droplet mesh ---------------------------------------------------- */

/* Node and triangle counts of an icosphere of subdivision level `level`:
 * 10*4^level + 2 nodes, 20*4^level triangles. */
int ibl_icosphere_size(int level, int *n_nodes, int *n_tris);

/* Host-only: writes the icosphere used by ibl_mesh_create_icosphere (radius
 * R, centre `center`, 3 doubles, not NULL) into caller-owned host arrays r
 * (n_nodes x 3 doubles) and tris (n_tris x 3 int32).  No device work. */
int ibl_icosphere(int level, double R, const double *center, double *r, int32_t *tris);

/* Device bytes of a closed triangle mesh with these counts. */
int ibl_mesh_workspace_size(int n_nodes, int n_tris, size_t *bytes);

/* Attaches a droplet to `lb` (one per lattice).  The icosphere variant
 * builds the structured spherical mesh of Sec. 3.2 (subdivided icosahedron,
 * midpoints projected on the sphere at every level, triangles
 * counter-clockwise seen from outside) of radius R centred at `center`
 * (host, 3 doubles; NULL = box centre).  The generic variant takes host
 * positions (n_nodes x 3 doubles) and triangles (n_tris x 3 int32, outward
 * counter-clockwise) of a closed mesh.  sigma: surface tension (lattice
 * units). */
int ibl_mesh_create_icosphere(ibl_lb *lb, int level, double R, double sigma, const double *center,
                              void *workspace, size_t bytes, ibl_mesh **out);
int ibl_mesh_create(ibl_lb *lb, int n_nodes, const double *r, int n_tris, const int32_t *tris,
                    double sigma, void *workspace, size_t bytes, ibl_mesh **out);
void ibl_mesh_destroy(ibl_mesh *m);

/* Mesh regularisation of Sec. 3.3 (extended Laplacian smoothing), applied
 * after the advection of every `every`-th step (0 = off).  plus_sign = 1
 * uses x_p <- x_p - (gamma b_i + (1-gamma)/N_i sum_j b_j) (the volume
 * preserving form), 0 the sign as printed in Eq. (HC_algo_full).  The loop
 * stops when max_i |x_p - x_q| < tol or after max_iter iterations
 * (IBL_ERRBIT_NOCONV).  Paper values: alpha 0.1, gamma 0.51, tol 0.01. */
int ibl_set_regularization(ibl_mesh *m, double alpha, double gamma, double tol, int max_iter,
                           int every, int plus_sign);

/* Adaptive trigger for the scheduled regularisation (the paper regularises
 * unconditionally; this makes the smoothing conditional on the mesh
 * degrading, Sec. 3.3's motivation: clustered nodes and loose triangles).
 * At each scheduled regularisation the kernel first measures the mesh
 * quality q = max over triangles of (longest edge / shortest edge), which is
 * 1 for equilateral triangles; with max_edge_ratio > 0 it smooths only when
 * q > max_edge_ratio, otherwise the step is left as it is.  0 (the default)
 * smooths at every scheduled step.  Values in (0, 1) are rejected
 * (IBL_EINVAL).  ibl_regularize_now always smooths.  Synchronises the
 * lattice's stream. */
int ibl_set_regularization_trigger(ibl_mesh *m, double max_edge_ratio);

/* keep != 0: after every regularisation (scheduled or ibl_regularize_now),
 * scale the mesh about its volume centroid back to the volume it enclosed
 * before the smoothing (the paper has no such step; the smoothing of
 * Sec. 3.3 alone shrinks a curved mesh a little at each application, which
 * adds up over long runs).  Default 0.  Synchronises the lattice's stream. */
int ibl_set_regularization_keep_volume(ibl_mesh *m, int keep);

/* Re-centring of the boundary field (Sec. 3.2 says the linearisation of the
 * velocity field is centred on the droplet's centre of mass, while its
 * Eq. (velo_facce_cubo_da_gradiente) centres it on the box, L/2).  on != 0:
 * every step imposes u = A (l - c) on the Zou-He faces, c the centre of
 * mass (volume centroid) of the region the mesh encloses, measured on the
 * device from the positions at the start of the step; 0 (the default): the
 * box centre.  The adjoint (ibl_adjoint) refuses a lattice with re-centring
 * on (IBL_EINVAL); destroying the mesh switches it off; an ensemble takes
 * the setting its members have when it is created.  IBL_EINVAL if the mesh
 * is not attached.  Synchronises the lattice's stream. */
int ibl_set_recentring(ibl_mesh *m, int on);

/* Viscosity ratio (Sec. 2: the droplet phase has viscosity chi mu, the
 * carrier mu; the paper's runs have chi = 1).  Each step, the nodes inside
 * the droplet relax with tau_in = 1/2 + chi (tau - 1/2), the others with
 * tau.  Inside is decided per lattice node by the even-odd rule on a
 * vertical ray: a node is inside when an odd number of mesh triangles lie
 * above it, a triangle counting when the point (x + 1.4142135623730951e-7,
 * y + 1.7320508075688772e-7) falls strictly inside its projection on the xy
 * plane and its height there exceeds z (IEEE operations, no contraction).
 * chi = 1 switches it off.  IBL_EINVAL if chi is not finite and positive,
 * the mesh is not attached, or an axis is periodic.  The adjoint and the
 * ensemble refuse a lattice with chi != 1.  Synchronises the lattice's
 * stream. */
int ibl_set_viscosity_ratio(ibl_mesh *m, double chi);

/* Synchronising: *count = regularisations performed so far (triggered
 * scheduled ones and ibl_regularize_now calls), *mesh_quality = q measured
 * at the latest regularisation check (0 before the first).  Either pointer
 * may be NULL. */
int ibl_regularization_stats(ibl_mesh *m, int *count, double *mesh_quality);

/* Take a shape record every `every` steps (0 = off) into a device ring of
 * 4096 records, read with ibl_read_series. */
int ibl_set_readout(ibl_mesh *m, int every);

/* ---- stepping -------------------------------------------------------- */

/* Enqueues n IBLB steps on the bound stream (asynchronous). */
int ibl_step(ibl_lb *lb, long long n);

/* Enqueues one step that also stores rho, u and F_ext of every node
 * (needs record_fields); read them with ibl_copy_fields. */
int ibl_step_record(ibl_lb *lb);

/* Graph replay (default on): ibl_step runs whole chunks of steps -- a
 * multiple of 6 and of the regularisation and readout periods, at least 32
 * -- as one captured CUDA graph launched on the bound stream.  The chunk is
 * captured on a private stream at the first use and again after any
 * schedule change.  The shorter runs before the first chunk boundary and
 * after the last one (segments) run eagerly the first time a segment of
 * that length starts at that position in the schedule period, and from its
 * second occurrence on replay a graph of their own (up to 32 such graphs
 * are kept, least recently used dropped first): stepping in fixed
 * increments replays graphs throughout once each phase has come round
 * twice.  enable = 0 launches every kernel eagerly. */
int ibl_set_graphs(ibl_lb *lb, int enable);

/* Captures, without running any step, the CUDA graphs that the next call
 * ibl_step(lb, n) replays -- its whole chunks and the segments between them
 * (runs of 2 steps or more) -- and uploads them to the device, so that the
 * next ibl_step(lb, n) launches graphs only and pays no capture.  The
 * capture runs on private streams; only the graphs' uploads are enqueued on
 * the bound stream.  A no-op when graph replay is off.  IBL_EINVAL for n < 0, IBL_ECUDA for a failed
 * capture. */
int ibl_prepare_steps(ibl_lb *lb, long long n);

/* Kernel of the lattice update outside the droplet patch (and of the whole
 * box without a droplet), Eqs. (LBMEQ)-(density_velocity_LB) with the
 * boundary rebuild of Sec. 3.2: kind 0 = one thread per node with direct
 * loads; kind 1..2 = a pipeline of persistent blocks that stage each tile's
 * populations into shared memory with bulk asynchronous copies, in one of
 * two launch shapes (128-node tiles; 2 stages and 8 blocks per SM, or 3
 * stages and 6 blocks per SM).  Every kind computes the same update bit for bit.  The
 * staged kinds need FP32 populations and Zou-He walls on every axis
 * (IBL_EINVAL otherwise); a step that stores the fields (ibl_step_record)
 * uses kind 0.  Synchronises the bound stream and drops captured graphs.
 * ibl_outside_update reads the kind in use. */
int ibl_set_outside_update(ibl_lb *lb, int kind);
int ibl_outside_update(const ibl_lb *lb, int *kind);

/* For tests of the failure path only (no counterpart in the paper): with
 * on != 0 the staged outside update (kinds 1..2) announces more bytes than
 * its copies deliver, so that no stage completes.  Each block then gives up
 * after 1 s of waiting, sets the sticky bit IBL_ERRBIT_TIMEOUT, waits at
 * most 0.2 s per stage still outstanding and returns without updating a
 * node; the next synchronising call reports IBL_ETIMEOUT and the device
 * stays usable.
 * Synchronises the bound stream and drops captured graphs. */
int ibl_test_stage_timeout(ibl_lb *lb, int on);

/* Steps ibl_step has run eagerly and by graph replay since the lattice was
 * created (ibl_step_record and the adjoint's recomputations not counted). */
int ibl_step_paths(const ibl_lb *lb, long long *eager, long long *replayed);

/* Waits for the stream and reports the sticky device error bits as a status. */
int ibl_sync(ibl_lb *lb);

/* Checkpoint and resume (the paper's trajectories run for thousands of
 * frames, Sec. 3.2).  ibl_save synchronises the lattice's stream and writes
 * the whole dynamic state between steps to the file `path`: populations,
 * control block (step count, frame slots, patch buffers, sticky error bits),
 * frames, and, with a mesh, positions, nodal forces, bounding-box rows and
 * the shape-record ring.  ibl_load restores such a file into a lattice (and
 * its attached mesh) created with the same box, boundaries, precision, edge
 * rule, record_fields, tau, frame count, steps per frame and mesh size; the
 * step count comes from the file.  Settings made through the ibl_set_*
 * calls (regularisation, readout period, re-centring, viscosity ratio,
 * graphs) are not in the file: apply them to the resumed lattice as before.
 * Load before putting the lattice into an ensemble.  IBL_EINVAL for a null
 * argument, a file that cannot be opened, written or read in full, or a
 * mismatch; IBL_ECUDA for a failed copy.  The file layout is this library
 * version's own (a header, then the raw workspaces). */
int ibl_save(ibl_lb *lb, const char *path);
int ibl_load(ibl_lb *lb, const char *path);

/* Number of steps enqueued so far. */
long long ibl_steps_done(const ibl_lb *lb);

/* ---- readout (synchronising) ----------------------------------------- */

/* Computes a shape record of the current mesh now and copies it to *out. */
int ibl_readout(ibl_mesh *m, ibl_observables *out);

/* Copies up to `max` records of the ring, oldest first; *count = number copied. */
int ibl_read_series(ibl_mesh *m, ibl_observables *out, int max, int *count);

/* Fields of the last ibl_step_record step: rho (nodes), u and F (3 x nodes),
 * host, [c][z][y][x]; any pointer may be NULL. */
int ibl_copy_fields(ibl_lb *lb, double *rho, double *u, double *F);

/* Pre-collision populations f_i(x) of the next step in the library's
 * velocity order (ibl_velocity_set), host, 19 x nodes doubles, [i][z][y][x],
 * full values (not deviations); populations a wet boundary node has no
 * source for are 0. */
int ibl_copy_populations(ibl_lb *lb, double *f);

/* Node positions (n x 3), nodal forces of the last step (n x 3) and
 * triangles (m x 3 int32); any pointer may be NULL. */
int ibl_copy_mesh(ibl_mesh *m, double *r, double *F, int32_t *tris);

/* One-ring neighbour lists as CSR (ptr: n+1 int32, idx: ptr[n] int32,
 * ascending); either pointer may be NULL; *nnz receives ptr[n]. */
int ibl_copy_neighbours(ibl_mesh *m, int32_t *ptr, int32_t *idx, int *nnz);

/* Runs the regularisation once now on the current mesh (synchronising);
 * *iters receives the iteration count. */
int ibl_regularize_now(ibl_mesh *m, int *iters);

/* Allocation-free variant of the mesh regularisation (the paper has no
 * counterpart: this is an interface for callers that cannot allocate device
 * memory -- for instance a host program whose own allocator reserves the
 * device's memory up front, a time-budgeted loop that cannot absorb an
 * allocation call, or a plug-in whose host forbids allocations).  It runs
 * the same iteration as ibl_regularize_now on caller-owned device buffers:
 * r (n_nodes x 3 doubles, read and overwritten with the result), the
 * one-ring CSR nb_ptr (n_nodes + 1 int32) and nb_idx (nb_ptr[n_nodes]
 * int32, one-ring neighbours as returned by ibl_copy_neighbours), and
 * result (2 int32: iterations, 1 if converged else 0).  Asynchronous on
 * `stream` (a cudaStream_t, NULL = legacy default stream).
 * Scratch: a fixed array inside the library (16384 nodes x 9 doubles,
 * 1.18 MB) that every GPU loading the library holds until the process
 * exits; n_nodes above 16384 is rejected with IBL_EINVAL.  The first call
 * on a device looks up that array's device address (with the caller's
 * current device), so make the first call on each device before any stream
 * capture.  The address is looked up again whenever the calling thread's
 * current context is not the one it was looked up in (a driver-API context
 * made current, or the primary context created anew after
 * cudaDeviceReset): make the first call after such a change outside a
 * stream capture too.  Every call uses the same array and leaves its contents behind;
 * each call writes every element it reads first, so nothing needs
 * clearing, but calls whose executions overlap on the GPU (other streams,
 * other threads) race on it.  Calls no allocating routine. */
int ibl_regularize_noalloc(double *r, const int32_t *nb_ptr, const int32_t *nb_idx, int n_nodes, double alpha,
                           double gamma, double tol, int max_iter, int plus_sign, int32_t *result, void *stream);

/* The paper's trajectory loop with host buffers (Sec. 3.2, steps 1-4): for
 * each of n_frames frames, copy the frame (host, 9 doubles) to the device,
 * run steps_per_frame IBLB steps, and copy the droplet's shape record back
 * to out[k] (host).  steps_per_frame must equal the lattice's value and
 * the step count must be a multiple of it. */
int ibl_run_frames(ibl_lb *lb, ibl_mesh *m, const double *A_frames, int n_frames,
                   int steps_per_frame, ibl_observables *out);

/* ---- ensemble of droplets ---------------------------------------------- */

/* Many independent droplets advanced together (Sec. 4 runs one droplet per
 * turbulent trajectory; an ensemble batches such trajectories on one GPU).
 * Members are existing lattices, each with its droplet mesh, of any box and
 * mesh size, sharing precision, stream and step count.  Each ensemble step
 * launches every phase of the IBLB step once for all members (triangle
 * normals, force + spread, lattice update, interpolation + advection), plus
 * each member's own scheduled regularisation and shape record; whole chunks
 * of steps replay as one CUDA graph.  Members keep working with the
 * per-member readout calls; stepping a member on its own desynchronises it
 * (IBL_EINVAL at the next ensemble step).  The workspace (device, caller
 * owned) holds the member tables. */
typedef struct ibl_ensemble ibl_ensemble;
int ibl_ensemble_workspace_size(int n_members, ibl_lb *const *members, size_t *bytes);
int ibl_ensemble_create(int n_members, ibl_lb *const *members, void *workspace, size_t bytes, ibl_ensemble **out);
/* Enqueues n steps of every member (asynchronous). */
int ibl_ensemble_step(ibl_ensemble *e, long long n);
/* Launch shape of an ensemble step: IBL_ENSEMBLE_SHAPES candidates, shape
 * k = 8 c + 4 p + 2 t + w (c = 0..3).  The batched lattice update of the nodes outside
 * each droplet patch (almost all of a step's bytes) takes 128 (t = 0) or
 * 256 (t = 1) threads per block, each block updating that many consecutive
 * nodes of one z plane of one member, and prefetches the populations into
 * L2 w resident waves of blocks ahead (w = 0 or 1).  p = 0 keeps the
 * droplet-side data (mesh, patch populations, force and velocity) in L2
 * with an evict_last policy, as a single droplet's step does; p = 1 uses the
 * default policy.  c = 1, 2, 3 caps the droplet-side kernels (forces and
 * spread, patch nodes, interpolation), which run on the helper stream beside
 * the lattice update, at 1, 2 or 4 blocks per SM; c = 0 gives them one block
 * per work unit.  The shape changes only launch geometry and cache policy:
 * every shape computes the same populations.  Default: shape 16.
 *
 * ibl_ensemble_tune is the autotuner: it runs 2 untimed and
 * steps_per_candidate timed ensemble steps with each shape in turn (eager
 * launches, CUDA events on the bound stream), keeps the shape with the
 * least time per step and writes its index to *chosen and the measured ms
 * per step of every shape to ms (IBL_ENSEMBLE_SHAPES doubles; either may be
 * NULL).  These are steps of the members' trajectories: afterwards every
 * member has advanced by IBL_ENSEMBLE_SHAPES * (steps_per_candidate + 2)
 * steps.  Synchronising; returns the members' error status as
 * ibl_ensemble_sync.  ibl_ensemble_set_shape sets a shape directly (for
 * instance one stored from an earlier tuning of the same member sizes);
 * ibl_ensemble_shape reports the current one (any pointer may be NULL). */
#define IBL_ENSEMBLE_SHAPES 32
int ibl_ensemble_tune(ibl_ensemble *e, int steps_per_candidate, double *ms, int *chosen);
int ibl_ensemble_set_shape(ibl_ensemble *e, int shape);
int ibl_ensemble_shape(const ibl_ensemble *e, int *shape, int *threads, int *prefetch_waves);

/* Waits and returns the error status of the first member (in the order
 * given at creation) whose sticky device bits are set, with ibl_last_error()
 * naming that member's index ("ensemble member k: ..."); IBL_OK if none. */
int ibl_ensemble_sync(ibl_ensemble *e);
void ibl_ensemble_destroy(ibl_ensemble *e);

/* ---- gradients of the deformation ------------------------------------ */

/* Discrete adjoint of the IBLB trajectory (the paper has no counterpart:
 * it differentiates the step of items 1-4 above, without regularisation).
 * The objective is the Taylor deformation D of the droplet after n_steps
 * steps from step 0 (Sec. 2: D from the eigenvalues of S = (5/V) int (x -
 * x_c)(x - x_c)^T dV of the final mesh); the parameters are the surface
 * tension sigma (Eq. (pi_drop)) and every velocity-gradient frame A_k
 * (Eq. (velo_facce_cubo_da_gradiente), frame k held over steps
 * [k N, (k + 1) N), the last frame for all later steps; frame 0 also sets
 * the initial equilibrium populations).
 *
 * ibl_adjoint requires a droplet on `lb`, the step count at 0 and the
 * regularisation off (every = 0).  It re-initialises the populations to
 * the equilibrium of the current frame 0, runs the n_steps forward steps
 * (graph replay as ibl_step) saving a checkpoint every K steps, then
 * sweeps backwards: each segment of K steps is recomputed from its
 * checkpoint, keeping the node positions and the density, velocity and
 * force of every node for each step, and the adjoint of each step is taken
 * in reverse (interpolation + advection, lattice update with the Zou-He
 * rebuild, spreading, nodal forces).  Adjoint state: populations and
 * Eulerian fields in the storage precision, node quantities and all
 * accumulated gradients in FP64.
 *
 * Outputs (host, caller-owned, each may be NULL): *D; *dD_dsigma;
 * dD_dA[9 k + 3 a + b] = dD/dA_k[a][b] for every frame k of the lattice
 * (n_frames x 9 doubles); dD_dr0 = dD/dr of the initial node positions
 * (n_nodes x 3).  Synchronising; on return the lattice and droplet hold the
 * state after n_steps steps (shape records of the forward pass are kept,
 * the recomputation writes none).  The workspace (device, 256-byte
 * aligned, caller-owned, `bytes` from ibl_adjoint_workspace_size) holds
 * ceil(n_steps / K) + 1 checkpoints (populations, control block, positions)
 * plus two sets of min(K, n_steps) steps of recorded moments (7 values per
 * lattice node), positions and patches (one segment is recorded again on a
 * second stream while the next is swept back), and the adjoint fields.  Errors: IBL_EINVAL for a
 * bad state or argument, IBL_ENOMEM for a short workspace, and the sticky
 * device errors of the forward and recomputed steps. */
int ibl_adjoint_workspace_size(const ibl_lb *lb, long long n_steps, int K, size_t *bytes);
int ibl_adjoint(ibl_lb *lb, long long n_steps, int K, void *workspace, size_t bytes, double *D, double *dD_dsigma,
                double *dD_dA, double *dD_dr0);

/* ---- linear theory ---------------------------------------------------- */

/* The small-deformation theory of Eq. (LT) (Sec. 2), the paper's reference
 * for the Ca -> 0 limit, along many gradient trajectories at once:
 *   dS/dt = -(40(chi+1) / ((2chi+3)(19chi+16))) (S - R^2 I) / tau_sigma
 *           + 2 R^2 (5/(2chi+3)) E(t),   S(0) = R^2 I,
 * E the symmetric part of the frame in force, each frame held for `hold`
 * time units (lattice steps for the IBLB frames, Sec. 3.2), integrated by
 * the classical fourth-order Runge-Kutta method with `substeps` steps per
 * frame in FP64.  Device arrays (caller-owned): A [n_traj][n_frames][9]
 * row-major frames as in ibl_lb_create; params [n_traj][4] = tau_sigma, R,
 * chi, hold per trajectory; out [n_traj][n_frames][9] = S_xx, S_yy, S_zz,
 * S_xy, S_xz, S_yz, lambda_max / R^2, beta (Eq. (beta); NaN when E = 0) and
 * D at the end of every frame (D takes the smallest eigenvalue as 0 if the
 * theory has been driven past positive definiteness).  A trajectory with
 * tau_sigma <= 0, R <= 0, chi < 0, hold <= 0 or a non-finite parameter gets
 * NaN throughout.  Asynchronous on `stream` (a cudaStream_t, NULL = legacy
 * default stream); allocates nothing.  IBL_EINVAL for counts < 1, substeps
 * outside 1..2^20 or a null pointer. */
int ibl_linear_theory(int n_traj, int n_frames, const double *A, const double *params, int substeps,
                      double *out, void *stream);

/* ---- introspection --------------------------------------------------- */

/* Synchronises and returns the droplet patch of the next step: lower
 * corner lo[3] and extents ext[3] (nodes - 1 per axis; -1 = empty).  With a
 * droplet, each step updates the patch nodes on a high-priority helper
 * stream next to the droplet kernels, and all other nodes on the bound
 * stream concurrently. */
int ibl_patch(ibl_lb *lb, int32_t lo[3], int32_t ext[3]);

/* The library's D3Q19 velocities (19 x 3 int32) and weights (19 doubles). */
int ibl_velocity_set(int32_t *c, double *w);

/* Kernel timing with CUDA events on the bound stream.  `mask` selects the
 * kernels bracketed by an event pair at every launch: bit 0 the lattice
 * kernel, bit 1 the force/spread kernel, bit 2 the interpolation kernel (0
 * turns timing off and clears it); bit 3 restricts timing to the launches
 * inside captured graph chunks.  Only one launch in `every` of each kernel
 * is bracketed (1 = all), so that sparse sampling keeps the event overhead
 * out of the step time.  ibl_profile_read synchronises and
 * returns the summed durations (ms) and launch counts [lattice, spread,
 * interpolate] since enabling.  At most 65536 launches are recorded.  With
 * graph replay the event pairs are nodes of the captured chunk, so each
 * replay re-records them: the read covers the eager launches and the last
 * replay of the chunk. */
int ibl_profile_enable(ibl_lb *lb, int mask, int every);
int ibl_profile_read(ibl_lb *lb, double ms[3], long long launches[3]);

const char *ibl_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IBLB_H */
