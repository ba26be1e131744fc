/*
 * mevp.h -- C ABI of the GB300 mEVP momentum-subcycle library (libmevp.so).
 *
 * The library advances the viscous-plastic sea-ice momentum equation (Eq. 2 of
 * Jendersie, Lessig, Richter, "Towards a GPU-Parallelization of the neXtSIM-DG
 * Dynamical Core", PASC'24) with the mEVP pseudo-time iteration (Eq. 3) on one
 * GPU.  One subcycle is the four stages of the paper's Table 1 -- strain,
 * stress, divergence, velocity -- in two kernel launches in FP64 (element
 * stages, then the node gather and velocity update) and in one fused launch
 * per subcycle in the mixed precision.  The discretisation is the one of
 * Sec. 2.1: CG2 (Q2) velocity on a structured quadrilateral mesh (rectilinear,
 * general bilinear or curved isoparametric elements), tensor-valued DG stress
 * (DG1 = 3, DG2 = 6 or the 8-dof space of App. A per component), and DG ice
 * height H and concentration A with n_adv in {1, 3, 6} dofs (DG0, DG1, DG2).
 * The stress update per element is the one printed in Listing 1 / App. A
 * (generalised to any ellipse ratio e), with the element map computed from
 * the mesh geometry (Sec. 3.2, "on-the-fly map").
 *
 * Conventions shared by every call:
 *   - Every call returns an int status (MEVP_OK or a negative MEVP_ERR_*);
 *     no C++ exception crosses this boundary.  mevp_last_error() returns a
 *     thread-local, human-readable message for the last failing call of the
 *     calling thread (valid until that thread's next failing call).
 *   - Argument checks are synchronous.  Kernel launches are asynchronous on
 *     the state's CUDA stream; an asynchronous CUDA error surfaces as
 *     MEVP_ERR_CUDA at the next call that synchronises (mevp_sync,
 *     mevp_read_field to host) or checks for launch errors.
 *   - Handles are created and freed by the library; destroying NULL is a
 *     no-op.  Input pointers are borrowed only for the duration of the call.
 *   - "on_device" = 0: the pointer is host memory; the data are copied on the
 *     state's stream into a staging buffer and checked there for non-finite
 *     values (MEVP_ERR_NAN, the state unchanged), and the call returns once
 *     the host buffer has been read; the move into the state is enqueued.
 *     "on_device" = 1: the pointer is device memory of the state's device; the
 *     copy is enqueued on the state's stream (the caller keeps the buffer
 *     alive and unmodified until the stream reaches it).
 *
 * External array layouts (fixed, independent of the internal layout):
 *   N_e = nx*ny elements, element id K = ky*nx + kx;
 *   N_n = (2nx+1)(2ny+1) CG2 nodes, node id = iy*(2nx+1) + ix;
 *   N_v = (nx+1)(ny+1) vertices, vertex id = jy*(nx+1) + jx.
 *   velocity, wind stress, ocean velocity, forces: [2][N_n] (x row, then y)
 *   stress, strain: [3][n_stress][N_e], component order 11, 12, 22
 *   H, A: [n_adv][N_e]
 *   vertex coordinates: [N_v][2] (x, y) pairs
 * DG coefficients refer to the orthogonal basis on the reference square,
 * with xh = xi - 1/2, eh = eta - 1/2:
 *   {1, xh, eh, xh^2 - 1/12, xh*eh, eh^2 - 1/12, (xh^2 - 1/12)*eh,
 *    xh*(eh^2 - 1/12)}   (first 3 for DG1, first 6 for DG2)
 * Values at points, forces and velocities do not depend on this choice.
 */
#ifndef MEVP_GB300_C_ABI_H
#define MEVP_GB300_C_ABI_H

#include <stddef.h>

#if defined(__GNUC__)
#define MEVP_API __attribute__((visibility("default")))
#else
#define MEVP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mevp_mesh mevp_mesh;   /* opaque, library-owned */
typedef struct mevp_state mevp_state; /* opaque, library-owned */

/* Physical and iteration parameters.  Pstar, C, e (hard-coded 2 in the
 * paper's code) and DeltaMin enter the stress update of Listing 1 / App. A;
 * alpha is the stress relaxation of Eq. 3 in the relaxation form of the
 * paper's code, S <- (1 - 1/alpha) S + (1/alpha) M^-1 (...); beta, dt,
 * rho_ice, rho_water, Cw and coriolis_f enter the velocity update of Eq. 2. */
typedef struct {
  double Pstar;      /* ice strength P* [N/m^2] (> = 0)                  */
  double C;          /* ice strength concentration parameter (>= 0)      */
  double e;          /* yield-ellipse aspect ratio (> 0)                 */
  double DeltaMin;   /* Delta_min [1/s] (> 0)                            */
  double alpha;      /* stress relaxation (>= 1)                         */
  double beta;       /* velocity relaxation (>= 0)                       */
  double dt;         /* outer time step [s] (> 0)                        */
  double rho_ice;    /* ice density [kg/m^3] (> 0)                       */
  double rho_water;  /* water density [kg/m^3] (>= 0)                    */
  double Cw;         /* ocean drag coefficient (>= 0)                    */
  double coriolis_f; /* Coriolis parameter [1/s]                         */
} mevp_params;

enum { MEVP_FP64 = 0, MEVP_MIXED = 1 };

enum {
  MEVP_OK = 0,
  MEVP_ERR_ARG = -1,         /* invalid argument (synchronous)                */
  MEVP_ERR_CUDA = -2,        /* CUDA runtime or launch error                  */
  MEVP_ERR_OOM = -3,         /* allocation failed or workspace too small      */
  MEVP_ERR_STATE = -4,       /* call out of order (e.g. run before set_params) */
  MEVP_ERR_NAN = -5,         /* non-finite value detected                     */
  MEVP_ERR_TIMEOUT = -6,     /* bounded device wait gave up                   */
  MEVP_ERR_UNSUPPORTED = -7, /* valid input the library does not handle       */
  MEVP_ERR_BOUNDS = -8       /* a kernel index left its buffer (only builds
                                compiled with -DMEVP_CHECKED test for this;
                                reported by mevp_sync with the access site) */
};

enum mevp_field {
  MEVP_U = 0,          /* velocity x   [N_n]                                 */
  MEVP_V = 1,          /* velocity y   [N_n]                                 */
  MEVP_S11 = 2,        /* stress 11    [n_stress][N_e]                       */
  MEVP_S12 = 3,        /* stress 12    [n_stress][N_e]                       */
  MEVP_S22 = 4,        /* stress 22    [n_stress][N_e]                       */
  MEVP_E11 = 5,        /* strain rate 11 of the current velocity [n_stress][N_e] */
  MEVP_E12 = 6,        /* strain rate 12 (tensor component)                  */
  MEVP_E22 = 7,        /* strain rate 22                                     */
  MEVP_FORCE_X = 8,    /* nodal stress-divergence force of the current stress [N_n] */
  MEVP_FORCE_Y = 9,
  MEVP_H = 10,         /* ice height  [n_adv][N_e]                           */
  MEVP_A = 11,         /* ice concentration [n_adv][N_e]                     */
  MEVP_NODAL_MASS = 12 /* lumped nodal mass rho_ice int max(0,H) phi_j [N_n] (after begin_step) */
};

/* Create a structured nx x ny quadrilateral mesh (Sec. 2.1).  vertex_xy is
 * [N_v][2] host memory (copied), or NULL for a uniform mesh of [0,Lx] x [0,Ly]
 * (Lx, Ly ignored when vertex_xy is given).  A rectilinear vertex set
 * (x depends only on jx, y only on jy) must be strictly increasing in both
 * directions and runs on the rectilinear kernels.  Any other vertex set is a
 * general mesh: each element is the bilinear (Q1) image of the reference
 * square, evaluated on the fly per Gauss point (Sec. 3.2), and must be a
 * convex quadrilateral with counter-clockwise vertices (Jacobian determinant
 * positive at its four corners, hence everywhere), else MEVP_ERR_ARG.
 * No device memory is allocated.
 * nx, ny >= 1 and (2nx+1)(2ny+1) < 2^31. */
MEVP_API int mevp_mesh_create(int nx, int ny, double Lx, double Ly, const double *vertex_xy,
                     mevp_mesh **out);
/* Create a structured nx x ny mesh of curved (isoparametric) quadrilaterals:
 * node_xy [N_n][2] host memory (copied) holds the positions of all CG2 nodes,
 * node id = iy*(2nx+1) + ix, and each element is the image of the reference
 * square under the Q2 interpolant of its 9 nodes -- the element map from the
 * velocity's finite element space (Sec. 2.1).  The local mass matrices use
 * the Gauss rule of App. A (det J is then a higher-degree polynomial).
 * MEVP_ERR_ARG for non-finite positions or an element whose det J is not
 * positive at its 5 x 5 reference sample points.  FP64 and mixed states
 * (the mixed path keeps FP32 node offsets from each element's centre node). */
MEVP_API int mevp_mesh_create_nodes(int nx, int ny, const double *node_xy, mevp_mesh **out);
MEVP_API void mevp_mesh_destroy(mevp_mesh *mesh);

/* Device workspace a state needs, in bytes (all internal buffers). */
MEVP_API int mevp_state_workspace_bytes(const mevp_mesh *mesh, int n_stress, int n_adv, int precision,
                               size_t *bytes);

/* Create a state for n_stress in {3, 6, 8} (DG1, DG2 and the 8-dof stress of
 * App. A; Gauss rule 2x2, 3x3, 3x3), n_adv in {1, 3, 6} (DG0, DG1, DG2 H and
 * A; with DG1/DG2 the ice strength of Listing 1 varies over the Gauss points)
 * and precision MEVP_FP64 or MEVP_MIXED, bound to the current CUDA device and to cuda_stream (a
 * cudaStream_t; NULL = legacy default stream).  MEVP_MIXED computes strain,
 * viscosities, stress and element forces in FP32 (the FP32 stress update of
 * Sec. 4, extended to every element stage), keeps the velocity state as
 * compensated FP32 pairs and sums nodal forces with compensation; inputs and
 * outputs at this boundary stay FP64.  workspace: device memory of at least
 * mevp_state_workspace_bytes(), 256-byte aligned, owned by the caller and
 * kept alive until mevp_state_destroy; or NULL, in which case the library
 * allocates (cudaMalloc) and frees it.  The mesh must outlive the state.
 * All fields start at zero; parameters must be set before running. */
MEVP_API int mevp_state_create(const mevp_mesh *mesh, int n_stress, int n_adv, int precision,
                      void *cuda_stream, void *workspace, size_t workspace_bytes,
                      mevp_state **out);
MEVP_API void mevp_state_destroy(mevp_state *state);

/* Parameters (copied; see mevp_params for the passages that define each:
 * Listing 1 / App. A for Pstar, C, e and DeltaMin, Eq. 3 for alpha, Eq. 2
 * and the mEVP velocity relaxation for beta, dt, the densities, Cw and
 * coriolis_f).  Every field must be finite and in the range noted there,
 * else MEVP_ERR_ARG.  Takes effect at the next mevp_begin_step. */
MEVP_API int mevp_set_params(mevp_state *state, const mevp_params *params);

/* H and A, [n_adv][N_e] FP64 each.  Takes effect at the next mevp_begin_step. */
MEVP_API int mevp_set_ice(mevp_state *state, const double *H, const double *A, int on_device);

/* Per-element ice strength parameter P* [N_e] (N/m^2, replacing
 * params.Pstar element by element; NULL returns to params.Pstar).  Enters the
 * ice strength P = P* max(0,H) exp(-C (1 - clamp(A,0,1))) of Listing 1 at
 * the next mevp_begin_step. */
MEVP_API int mevp_set_strength_field(mevp_state *state, const double *Pstar, int on_device);

/* Nodal wind stress tau [2][N_n] (N/m^2) and ocean velocity [2][N_n] (m/s)
 * or NULL for an ocean at rest.  Takes effect at the next mevp_begin_step. */
MEVP_API int mevp_set_forcing(mevp_state *state, const double *tau, const double *v_ocean,
                     int on_device);

/* Velocity [2][N_n]: the CG2 velocity v of Eq. 2 and the iterate v^{p-1}
 * of the mEVP iteration (Eq. 3).  Boundary entries are stored as given but
 * every subcycle writes 0 there (Dirichlet).  Does not change v^n (that is
 * mevp_begin_step's).  MEVP_ERR_NAN for a non-finite host value (the state
 * keeps its previous velocity). */
MEVP_API int mevp_set_velocity(mevp_state *state, const double *uv, int on_device);

/* Stress [3][n_stress][N_e]: the DG coefficients of sigma, the iterate
 * sigma^{p-1} of Eq. 3 (Listing 1's S11, S12, S22).  MEVP_ERR_NAN for a
 * non-finite host value (the state keeps its previous stress). */
MEVP_API int mevp_set_stress(mevp_state *state, const double *S, int on_device);

/* Advect H and A by n_steps >= 0 steps of length params.dt with the
 * state's current velocity held fixed: the transport equations of Sec. 2
 * (zero sources) discretised as Sec. 2.1 states, discontinuous Galerkin in
 * the n_adv-dof space of H, A with the standard upwind flux (chosen pointwise
 * at the edge quadrature points; on the domain boundary the element's own
 * trace) and explicit Runge-Kutta in time: forward Euler for DG0, Heun's
 * method for DG1, the three-stage Shu-Osher scheme for DG2.  Quadrature:
 * 3 x 3 points per element and 3 per edge for DG0/DG1, 4 x 4 and 4 for DG2.
 * No limiter: the clamps of the stress update (max(0,H), clamp(A,0,1))
 * absorb undershoots.  Asynchronous on the state's stream; the new H, A
 * take effect at the next mevp_begin_step.  MEVP_ERR_STATE without
 * parameters. */
MEVP_API int mevp_advect(mevp_state *state, int n_steps);

/* Start an outer time step: v^n := current velocity, and recompute from H, A,
 * the forcing and the parameters the per-element ice strength
 * P = P* max(0,H) exp(-C (1 - clamp(A,0,1))) and the per-node constants of
 * the velocity update (lumped mass, forcing).  Asynchronous. */
MEVP_API int mevp_begin_step(mevp_state *state);

/* n >= 0 mEVP subcycles (Sec. 2: the momentum equation and Eq. 3 subcycled
 * within one outer step) from the current velocity and stress, with v^n and
 * the forcing of the last mevp_begin_step.  Asynchronous on the state's
 * stream; FP64: two kernel launches per subcycle, MEVP_MIXED: one (see
 * MEVP_OPT_FUSED); replayed as CUDA graphs (MEVP_OPT_GRAPHS).  The first
 * call after a parameter change captures its graphs: do not call it while
 * the state's stream is itself being captured. */
MEVP_API int mevp_run_subcycles(mevp_state *state, int n);

/* Copy a field (enum mevp_field) to dst, FP64, `count` = number of doubles
 * of dst (must be >= the field's size).  The fields are the outputs of the
 * stages of Table 1: velocity (the velocity stage), stress (the stress
 * update of Listing 1), strain (the strain stage's E, here of the current
 * velocity) and nodal force (the divergence stage, of the current stress);
 * the strain and force fields are computed by diagnostic kernels in FP64
 * (also for MEVP_MIXED states, from their FP32/compensated state).  With
 * on_device = 0 the call waits for the state's stream.  MEVP_ERR_ARG for an
 * unknown field, a NULL dst or a short count. */
MEVP_API int mevp_read_field(mevp_state *state, int field, double *dst, size_t count, int on_device);

/* Wait for all work on the state's stream; reports asynchronous errors. */
MEVP_API int mevp_sync(mevp_state *state);

/* Options of a state (mevp_set_option). */
enum {
  /* MEVP_MIXED only: 1 (default) = one fused launch per subcycle (element
   * work for a tile plus a one-element halo, forces through shared memory,
   * node update in the same CTA); 0 = two launches (element kernel writing
   * per-element forces to global memory, node kernel gathering them).  Both
   * give bitwise identical results. */
  MEVP_OPT_FUSED = 1,
  /* 1 (default) = mevp_run_subcycles replays runs of 4 or more subcycles as
   * CUDA graphs (chunks of up to 512, captured on the state's stream at first
   * use and kept until the parameters, the ocean forcing or an option
   * change); 0 = one launch at a time.  States on the legacy default stream
   * (cuda_stream = NULL) always launch one at a time. */
  MEVP_OPT_GRAPHS = 2,
  /* k > 0: after every k subcycles a watchdog kernel scans the velocity for
   * NaN/Inf and raises a device flag, which the next mevp_sync reports as
   * MEVP_ERR_NAN (and clears); 0 (default) = off. */
  MEVP_OPT_NAN_CHECK = 3,
  /* Failure-detection test hook, MEVP_MIXED fused launches only: 1 = the
   * tiles' shared-memory staging barrier expects 16 bytes more than its
   * copies deliver, so its bounded wait runs out; the tiles skip their node
   * stage (the velocity is then not updated) and the next mevp_sync returns
   * MEVP_ERR_TIMEOUT (and clears the flag).  0 (default) = off. */
  MEVP_OPT_STALL_TEST = 4
};
MEVP_API int mevp_set_option(mevp_state *state, int option, int value);

/* ---- Ensembles ------------------------------------------------------------
 * Many independent domains advanced together, for ensembles of uneven
 * domains (sizes, stress dofs, ice degree, mesh kind and parameters may
 * differ per member).  The members are existing states that share one
 * precision, one device and one stream; the ensemble borrows them (they must
 * outlive it) and they remain usable on their own.  The members on
 * rectilinear meshes with 3 or 6 stress dofs and DG0 ice are batched: per
 * subcycle, MEVP_MIXED issues one persistent launch over their (member, tile)
 * work list, MEVP_FP64 one persistent element launch per stress space over
 * their element blocks and one persistent node launch over all members.  The
 * remaining members run their single-state launches (FP64: the element
 * launch) in the same stream (and CUDA graphs).  Results
 * are bitwise those of stepping each member alone.  The ensemble allocates
 * small device tables (cudaMalloc) for its member descriptors and work
 * lists. */
typedef struct mevp_ensemble mevp_ensemble; /* opaque, library-owned */

MEVP_API int mevp_ensemble_create(mevp_state *const *members, int n, mevp_ensemble **out);
MEVP_API void mevp_ensemble_destroy(mevp_ensemble *ensemble);

/* mevp_begin_step on every member. */
MEVP_API int mevp_ensemble_begin_step(mevp_ensemble *ensemble);

/* n subcycles of every member (runs of 4 or more replayed as CUDA graphs on
 * a non-default stream, as for a single state).  Asynchronous. */
MEVP_API int mevp_ensemble_run_subcycles(mevp_ensemble *ensemble, int n);

/* Work decomposition candidates: MEVP_MIXED tile shapes (elements, x by y),
 * MEVP_FP64 element block sizes (threads, 1).  dims receives up to max
 * (x, y) pairs; count the number of candidates. */
MEVP_API int mevp_ensemble_shapes(int precision, int *dims, int max, int *count);
MEVP_API int mevp_ensemble_set_shape(mevp_ensemble *ensemble, int shape);

/* Time trial_subcycles (after 2 warm-up subcycles) with every candidate
 * shape on the ensemble itself, keep the fastest and return its index in
 * *best (may be NULL).  The members' velocity and stress are copied to a
 * temporary device buffer (cudaMalloc) first and restored afterwards, so the
 * trials leave no trace in the results.  Synchronises the stream. */
MEVP_API int mevp_ensemble_autotune(mevp_ensemble *ensemble, int trial_subcycles, int *best);

/* 1 (default): replay runs of subcycles as CUDA graphs; 0: direct launches. */
MEVP_API int mevp_ensemble_set_graphs(mevp_ensemble *ensemble, int on);

/* Size of the static device scratch used by mevp_run_subcycles_noalloc. */
#define MEVP_NOALLOC_SCRATCH_BYTES (8u << 20)

/* mevp_run_subcycles_noalloc -- one outer step (v^n := vel at entry) of n
 * mEVP subcycles, in place, WITHOUT allocating any device memory.
 *
 * The paper has no counterpart; this entry point exists for callers that
 * cannot allocate: a host model or coupler that owns a fixed device-memory
 * pool and hands this library only raw device pointers, a language runtime
 * with no binding to a CUDA allocator, or a time-critical loop that must
 * not call cudaMalloc/cudaFree because they can synchronise the device and
 * stall other streams.  It calls no cudaMalloc, cudaFree or allocating
 * library routine.  Results match mevp_begin_step + mevp_run_subcycles on a
 * state with the same inputs (FP64 only).
 *
 * All arrays are device memory of the current device, in the external
 * layouts above: xline [nx+1] and yline [ny+1] are the strictly increasing
 * vertex coordinates of a rectilinear mesh; H, A [N_e] (DG0); tau [2][N_n];
 * v_ocean [2][N_n] or NULL (ocean at rest); vel [2][N_n] and
 * S [3][n_stress][N_e] (n_stress 3, 6 or 8) are read and overwritten.
 * The library cannot see the lengths of these raw pointers: each must hold
 * at least the stated number of doubles (shorter buffers are read and
 * written past their end).  params is host memory.
 * Work is enqueued on cuda_stream (a cudaStream_t, NULL = legacy default
 * stream).  The call checks on the device that xline and yline increase
 * strictly and waits for that check (4 bytes read back; this waits for the
 * work already queued on cuda_stream, not for the device); it then enqueues
 * the subcycles and returns without waiting.  MEVP_ERR_ARG when a line does
 * not increase strictly.
 *
 * No NaN watchdog runs here (MEVP_OPT_NAN_CHECK belongs to states).  In a
 * library compiled with -DMEVP_CHECKED the call also waits at the end and
 * returns MEVP_ERR_BOUNDS for a kernel access that left its buffer; a normal
 * build does not test kernel indices.
 *
 * Scratch: a file-scope static device array of MEVP_NOALLOC_SCRATCH_BYTES
 * (8 MiB), which every process that loads the library holds on every device
 * it uses until exit.  A mesh needs 19 N_e + 9 N_n + 2 (nx + ny) doubles
 * and 4 status words (each region 256-byte aligned): meshes up to
 * 128 x 128 elements fit; larger ones return MEVP_ERR_ARG with the sizes in
 * the message.  All calls on a device share that one array and it keeps the
 * last call's contents: each call clears the status words first, and every
 * other word a call reads is written by the same call before.
 * Calls whose work overlaps on the GPU (other streams, other host threads)
 * race on the scratch: serialise them, e.g. on one stream.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it; make that
 * first call before any stream capture on the device.  Errors: MEVP_ERR_ARG
 * for bad sizes, parameters, coordinate lines or non-device pointers;
 * MEVP_ERR_CUDA for a failed lookup, copy or launch. */
MEVP_API int mevp_run_subcycles_noalloc(int nx, int ny, int n_stress, const mevp_params *params,
                                        const double *xline, const double *yline,
                                        const double *H, const double *A, const double *tau,
                                        const double *v_ocean, double *vel, double *S, int n,
                                        void *cuda_stream);

/* Gradient of the kinetic energy J = 1/2 sum_j m_j |v_j|^2 (m_j the lumped
 * nodal mass) after n >= 1 subcycles from the current state, with respect to
 * the per-element P* field (mevp_set_strength_field; params.Pstar where none
 * is set) and the nodal wind stress tau, for an FP64 state after
 * mevp_begin_step.  A hand-written reverse mode of the subcycle (Table 1's
 * four stages: strain, the stress update of Listing 1, divergence, velocity):
 * the forward sweep keeps checkpoints (v, S) every checkpoint_every
 * subcycles, and each segment's velocities are recomputed before it is
 * reversed; the last segment's velocities are recorded during the forward
 * sweep, so checkpoint_every >= n stores every velocity and recomputes
 * nothing.  The drag's kink |v_o - v| = 0 takes derivative 0.  Outputs (any
 * may be NULL): *J; dJ_dPstar [N_e]; dJ_dtau [2][N_n]; host memory with
 * on_device = 0 (the call then waits), device memory with on_device = 1.
 * Afterwards the state holds the result of the n subcycles, as after
 * mevp_run_subcycles(n).  Allocates its working memory (cudaMalloc):
 * about (n/k) (2 N_n + 3 n_stress N_e) + (k + 8) 2 N_n + 40 N_e doubles,
 * k = min(checkpoint_every, n).  Any stress dofs and ice degree; with DG1/DG2
 * ice the strength at each Gauss point is P*_K times that point's
 * max(0, h) exp(-C (1 - clamp(a))).  Any mesh: on general and curved
 * elements the reverse mode follows the Gauss-point form of the forward
 * kernels.  MEVP_ERR_UNSUPPORTED for MEVP_MIXED. */
MEVP_API int mevp_adjoint_kinetic_energy(mevp_state *state, int n, int checkpoint_every,
                                         double *J, double *dJ_dPstar, double *dJ_dtau,
                                         int on_device);

/* Per-kernel timing with CUDA events, for benchmarks.  With on = k > 0 the
 * launches of every k-th subcycle of mevp_run_subcycles are bracketed by
 * events on the state's stream (k = 1: every subcycle; 0 switches off).
 * mevp_timing_read waits for the stream and returns, for kernel 0 (element
 * kernel) and kernel 1 (node kernel), the summed milliseconds and the number
 * of timed launches since the last read (or since timing was switched on),
 * then resets both.  ms and launches point to 2 host values each. */
MEVP_API int mevp_timing_enable(mevp_state *state, int on);
MEVP_API int mevp_timing_read(mevp_state *state, double *ms, long long *launches);

/* Thread-local message of the calling thread's last failing call. */
MEVP_API const char *mevp_last_error(void);

/* Library version string. */
MEVP_API const char *mevp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MEVP_GB300_C_ABI_H */
