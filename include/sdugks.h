/*
 * sdugks.h -- C-ABI of libsdugks: the simplified discrete unified gas kinetic scheme
 * (S-DUGKS, arXiv:2007.07347) D2Q9 time step on finite-volume quad meshes, run by
 * hand-written CUDA kernels on one GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Status.     Every int-returning call returns SDUGKS_OK (0) or a negative
 *             SDUGKS_ERR_* code; sdugks_last_error() then holds a one-line message
 *             (thread-local, valid until the next failing call on that thread).
 *             No call aborts the process or traps the device.
 * Ownership.  Input arrays are caller-owned and only read during the call (the mesh
 *             is copied).  Handles are library-owned: create/destroy pairs.
 *             Host output arrays are caller-owned and must hold the stated size.
 * Memory.     "host" pointers are ordinary (pageable or pinned) CPU memory; "device"
 *             pointers are CUDA global memory of the solver's device.
 * Streams.    A solver issues all its work on the CUDA stream given at creation
 *             (NULL = legacy default stream).  Calls marked "async" return before the
 *             GPU is done; calls that write host memory synchronise that stream.
 * Threads.    One solver must not be used from two threads at once; distinct
 *             solvers are independent.
 * Lattice.    D2Q9, c = 1, c_s^2 = 1/3.  Velocity index a = 0..8:
 *             (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1),
 *             weights 4/9, 1/9 (a = 1..4), 1/36 (a = 5..8).
 * Layouts.    Cell-major, in the caller's cell numbering: f[n_cells][9],
 *             W[n_cells][3] = (rho, rho*u_x, rho*u_y), u[n_cells][2].
 */
#ifndef SDUGKS_H
#define SDUGKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------------- */
#define SDUGKS_OK 0
#define SDUGKS_ERR_INVALID_ARG (-1)  /* NULL handle/pointer, size or value out of range */
#define SDUGKS_ERR_INVALID_MESH (-2) /* inconsistent face/cell arrays, open or degenerate cell */
#define SDUGKS_ERR_BAD_BC (-3)       /* missing boundary condition, unmatched periodic face */
#define SDUGKS_ERR_OOM (-4)          /* device or host allocation failed */
#define SDUGKS_ERR_DIVERGED (-5)     /* non-finite value found by the residual reduction */
#define SDUGKS_ERR_TIMEOUT (-6)      /* a bounded device wait gave up */
#define SDUGKS_ERR_CUDA (-7)         /* any other CUDA runtime error (message has the name) */
#define SDUGKS_ERR_STATE (-8)        /* call out of order, e.g. step before init */
#define SDUGKS_ERR_FULL (-9)         /* a batch has no room (device memory or instance slots) */

/* ---- boundary kinds (Sec. III) ------------------------------------------------- */
#define SDUGKS_BC_UNSET 0
#define SDUGKS_BC_PERIODIC 1    /* params: partner patch, shift_x, shift_y             */
#define SDUGKS_BC_WALL 2        /* no-slip wall at rest; params unused                 */
#define SDUGKS_BC_MOVING_WALL 3 /* no-slip wall moving at (u_x, u_y); params: u_x, u_y */
#define SDUGKS_BC_FARFIELD 4    /* inlet / free stream; params: rho_inf, u_x, u_y      */
#define SDUGKS_BC_OUTLET 5      /* rho and u of the inner cell; params unused          */
#define SDUGKS_BC_SYMMETRY 6    /* mirror ghost cell (same rho, mirrored u); the patch's
                                   faces must be lines of constant x or y; params unused */

/* ---- storage/compute precision of f ------------------------------------------- */
#define SDUGKS_FP64 0          /* f stored and computed in FP64                          */
#define SDUGKS_FP32 1          /* f stored and computed in FP32                          */
#define SDUGKS_FP32_BF16DEV 2  /* f stored as bf16 d = (f - feq(W)) / w, computed in FP32 */
#define SDUGKS_FP32_FP16DEV 3  /* f stored as fp16 d / s with s = 2^-10, computed in FP32  */
/* W (and the macroscopic-flux accumulation, residual and mass) is FP64 in every mode.
 * Inside the library the FP32-compute modes work in a deviation form: the distribution
 * is handled as f - w (w the lattice weights: the rest equilibrium of unit density) and
 * the density as rho - 1, so that face fluxes and their moments are sums of small
 * terms.  Every call of this header takes and returns f and rho themselves. */

/* ---- kernel selection ---------------------------------------------------------- */
#define SDUGKS_KERNEL_AUTO 0      /* Cartesian kernel when the mesh is a uniform grid  */
#define SDUGKS_KERNEL_TILED 1     /* unstructured tiled kernel on any quad mesh        */
#define SDUGKS_KERNEL_CARTESIAN 2 /* structured kernel; INVALID_ARG if not a grid      */

/* ---- staging of the Cartesian kernel's interior blocks --------------------------- */
#define SDUGKS_STAGING_LOADS 0    /* every thread loads its staged position (default)  */
#define SDUGKS_STAGING_TMA 1      /* two TMA tensor copies per block (Cartesian only;  */
                                  /* the same results; 1-6 % slower on GB300)          */

typedef struct sdugks_mesh sdugks_mesh;
typedef struct sdugks_solver sdugks_solver;

/* Flow and launch parameters.  tau = nu / c_s^2 = 3 nu; dt is the time step
 * (sdugks_mesh_cfl_dt gives a CFL-limited value). */
typedef struct sdugks_params {
    double tau;          /* relaxation time, > 0                                   */
    double dt;           /* time step, > 0                                         */
    int32_t precision;   /* SDUGKS_FP64 | SDUGKS_FP32 | SDUGKS_FP32_BF16DEV | _FP16DEV */
    int32_t kernel;      /* SDUGKS_KERNEL_*                                        */
    int32_t tile_cells;  /* tiled kernel: cells per tile (16..128); Cartesian kernel (FP32,
                            bf16 and fp16 storage): 256, 224 or 128 for 16x16, 16x14 or 16x8 blocks;
                            0 = chosen from the grid size (Cartesian) or 128 (tiled) */
    int32_t graph_steps; /* steps per captured CUDA graph in sdugks_step, 0 = auto, <0 = off */
    int32_t staging;     /* SDUGKS_STAGING_*; TMA requires the Cartesian kernel (else
                            INVALID_ARG).  A TMA copy that does not land within the wait
                            limit below makes the block give up, and the next
                            sdugks_residual reports SDUGKS_ERR_TIMEOUT */
    int32_t tma_wait_us; /* wait limit of a TMA staging copy in microseconds:
                            0 = 200000 (0.2 s); < 0 = give up at once without waiting,
                            which exercises the timeout path (the block still waits, up
                            to 0.2 s, for its copies to land before it exits) */
} sdugks_params;

/* What a solver chose and holds (sdugks_solver_info). */
typedef struct sdugks_info {
    int64_t n_cells, n_faces;     /* after periodic faces are merged pairwise          */
    int64_t n_tiles;              /* CTAs per step                                     */
    int64_t halo_cells;           /* summed over tiles (ring 1 + ring 2)               */
    int64_t steps_done;           /* steps since init / set_state                      */
    int64_t device_bytes;         /* device memory held by the solver                  */
    double state_bytes_per_cell_step; /* f and W read and written once per cell and step */
    double mesh_bytes_per_cell_step;  /* mesh data the kernel reads per cell and step  */
    int32_t kernel;               /* SDUGKS_KERNEL_TILED or SDUGKS_KERNEL_CARTESIAN    */
    int32_t precision;
    int32_t tile_cells;
    int32_t nx, ny;               /* Cartesian kernel: grid size, else 0               */
    int32_t staging;              /* SDUGKS_STAGING_* in use                           */
    int32_t one_code_path;        /* Cartesian kernel: 1 when the grid runs in one wave and
                                     every block takes the general code path; 0 when interior
                                     blocks take the compile-time interior variant      */
    int64_t n_boundary_faces;     /* faces on non-periodic patches: the rows of
                                     sdugks_step_boundary_flux                          */
} sdugks_info;

/* ---- mesh ---------------------------------------------------------------------- */

/* Build a 2-D finite-volume mesh from face-based owner/neighbour arrays (the
 * unstructured FV form the paper's cases use, Sec. IV).
 *   xy[n_points][2]        point coordinates (host)
 *   face_pts[n_faces][2]   end points of each straight face (host)
 *   owner[n_faces]         cell on one side, 0 <= owner < n_cells (host)
 *   neighbour[n_faces]     cell on the other side, or -1 - patch for a face of
 *                          boundary patch `patch` (0 <= patch < 64) (host)
 * Every cell must be a closed convex polygon with 3 or 4 faces.  Geometry (face
 * normals, areas, centroids) is computed here in FP64.  Errors: INVALID_ARG,
 * INVALID_MESH (open cell, repeated point, more than 4 faces), OOM. */
int sdugks_mesh_create(int64_t n_points, const double *xy, int64_t n_faces, const int64_t *face_pts,
                       const int64_t *owner, const int64_t *neighbour, int64_t n_cells,
                       sdugks_mesh **out);

/* Boundary condition of one patch (Sec. III: no-slip/moving wall and inlet by
 * non-equilibrium extrapolation, outlet, symmetric, periodic).  params[3] as listed
 * with the SDUGKS_BC_* kinds (host; may be NULL for WALL, OUTLET and SYMMETRY).  A
 * SYMMETRY face acts as an interior face to the mirror image of its cell (fbar+ of
 * the mirrored velocity, reflected gradient, also a neighbour in the cell's LLSR);
 * a slanted symmetry face is rejected with BAD_BC when a solver is created.  A PERIODIC patch
 * must name a PERIODIC partner whose faces sit at this patch's face centres plus
 * (shift_x, shift_y); pairing is checked when a solver is created.
 * Errors: INVALID_ARG (patch or kind out of range). */
int sdugks_set_bc(sdugks_mesh *mesh, int32_t patch, int32_t kind, const double *params);

/* CFL time step dt = cfl * dx_min / |xi|_max with |xi|_max = sqrt(2) (the diagonal
 * D2Q9 velocity) and dx_min = min over cells of area / longest face (Sec. I: the
 * step is limited only by the CFL condition). */
int sdugks_mesh_cfl_dt(const sdugks_mesh *mesh, double cfl, double *dt);

/* Number of cells and faces as given, and the number of boundary patches used. */
int sdugks_mesh_sizes(const sdugks_mesh *mesh, int64_t *n_cells, int64_t *n_faces, int32_t *n_patches);

void sdugks_mesh_destroy(sdugks_mesh *mesh);

/* ---- solver -------------------------------------------------------------------- */

/* Create a solver on the current CUDA device: pairs periodic faces, builds the LLSR
 * normal matrices of Sec. II, orders cells into tiles and uploads everything.
 * `stream` is a cudaStream_t (NULL = default stream).  The mesh may be destroyed
 * afterwards.  Errors: INVALID_ARG, BAD_BC, INVALID_MESH, OOM, CUDA. */
int sdugks_solver_create(const sdugks_mesh *mesh, const sdugks_params *params, void *stream,
                         sdugks_solver **out);

/* Initial state: W = (rho, rho u), f = feq(W).
 * rho[n_cells], u[n_cells][2] (host); NULL rho means 1, NULL u means 0.
 * Also takes the residual snapshot.  Synchronises the stream. */
int sdugks_init(sdugks_solver *s, const double *rho, const double *u);

/* Advance n >= 0 steps (Sec. II, the eleven-step update; async).  Long runs replay
 * a captured CUDA graph of params.graph_steps steps.  Errors: STATE before init. */
int sdugks_step(sdugks_solver *s, int64_t n);

/* One step (as sdugks_step(s, 1)) that also returns the force on every boundary
 * patch: force[2 p], force[2 p + 1] (host, [64][2]) = the momentum leaving the fluid
 * through the faces of patch p in that step, sum over its faces of
 * sum_a xi_a (xi_a . n l) f_b,a (n out of the fluid), per unit depth and time in the
 * solver's units.  For a wall this is the force of the fluid on it, from which drag
 * and lift coefficients follow (C = F / (0.5 rho U^2 D), Sec. IV).  Periodic patches
 * read 0.  Synchronises.  The FP64 sums use atomics, so the last bits can vary from
 * run to run; the state update itself is unchanged. */
int sdugks_step_forces(sdugks_solver *s, double *force);

/* One step (as sdugks_step(s, 1)) that also returns the momentum leaving the fluid
 * through every boundary face, the face-by-face form of the forces of Sec. IV:
 *   face_flux[2 i], face_flux[2 i + 1] (host, [n_boundary_faces][2], FP64) for the i-th
 *   face of the mesh (in the caller's face order) whose neighbour is < 0 and whose
 *   patch is not periodic (sdugks_info.n_boundary_faces rows):
 *     F_i = sum_a xi_a (xi_a . n_i l_i) f_b,a,
 *   n_i the unit normal out of the fluid, l_i the face length, f_b the interface
 *   distribution of the step (Eq. f_t_n+1 with the rules of Sec. III).
 * The patch sums of F_i are the forces of sdugks_step_forces; the normal part
 * F_i . n_i / l_i is the normal momentum flux, i.e. the surface pressure at a no-slip
 * wall (where the normal velocity and normal viscous stress vanish), from which
 * C_p = (F_i . n_i / l_i - rho_inf c_s^2) / (0.5 rho_inf U^2) (Sec. IV); the tangential
 * part over l_i is the wall shear stress.  Symmetry faces are included.
 * force: NULL, or as in sdugks_step_forces (per patch, summed with atomics).
 * face_flux: NULL, or the caller's buffer; each row is written once, in FP64 (FP32
 * modes: the FP32 sum converted).  Synchronises.  Errors: INVALID_ARG, STATE. */
int sdugks_step_boundary_flux(sdugks_solver *s, double *force, double *face_flux);

/* Macroscopic fields at the current step: rho[n_cells], u[n_cells][2] (host;
 * synchronises).  Either pointer may be NULL. */
int sdugks_get_macros(sdugks_solver *s, double *rho, double *u);

/* Same into device memory (async): d_rho[n_cells], d_u[n_cells][2], FP64. */
int sdugks_get_macros_device(sdugks_solver *s, double *d_rho, double *d_u);

/* Convergence residual of Sec. IV against the snapshot taken at the previous call
 * (or at init/set_state):
 *   eps = sqrt(sum_i (U_i - U0_i)^2 + (V_i - V0_i)^2) / sqrt(sum_i U0_i^2 + V0_i^2)
 * with U, V = rho u / rho; +inf when the snapshot is at rest.  *mass = sum_i V_i rho_i.
 * Then the snapshot is refreshed.  FP64 device reduction with a fixed order.
 * Synchronises.  Returns DIVERGED (with eps = NaN) if any W is not finite.
 * Returns TIMEOUT if a bounded staging wait of a step since the previous call gave
 * up: the blocks that gave up skipped their update, so the whole state is invalid;
 * the solver then needs sdugks_init or sdugks_set_state before it steps again (STATE
 * until then). */
int sdugks_residual(sdugks_solver *s, double *eps, double *mass);

/* Checkpoint of the state at t_n (host, FP64, caller's cell order):
 *   f[n_cells][9]  cell distribution
 *   W[n_cells][3]  conserved variables
 * get synchronises; set replaces the state (f is rounded to the storage precision)
 * and refreshes the residual snapshot.  A run resumed from a checkpoint equals the
 * uninterrupted run bit for bit with FP64 and FP32 storage. */
int sdugks_get_state(sdugks_solver *s, double *f, double *W);
int sdugks_set_state(sdugks_solver *s, const double *f, const double *W);

/* Checkpoint in the solver's own storage: a 32-byte header (layout of the solver), then
 * the distribution in the storage precision and W in FP64, both in the solver's internal
 * cell order.  The FP32-compute precisions store f as its deviation from the lattice
 * weights and W[0] as rho - 1 (see the precision notes above); the FP64 f and rho of
 * sdugks_get_state can round those stored values in their last place, while this form
 * restores bit for bit in every precision.
 *   buf    host; get: NULL to query the size into *bytes; else *bytes is its capacity,
 *          and receives the size written
 *   bytes  set: the size of buf, which must be the size get reports for this solver
 * set accepts only a state taken from a solver of the same layout (same mesh, precision,
 * kernel and tile size: INVALID_ARG otherwise), replaces the state and refreshes the
 * residual snapshot.  Both synchronise.  Errors: INVALID_ARG, STATE (get before init). */
int sdugks_get_state_raw(sdugks_solver *s, void *buf, int64_t *bytes);
int sdugks_set_state_raw(sdugks_solver *s, const void *buf, int64_t bytes);

/* The residual and mass reduction of sdugks_residual, for callers that may not
 * allocate device memory: over caller-owned device arrays, with the reduction's
 * scratch (per-block partial sums) in a fixed array inside the library instead of
 * memory it allocates.  This is a facility of this library; the paper has no
 * counterpart.  It is for code that must not call cudaMalloc or any allocating
 * routine -- a loop whose device memory is owned and budgeted by another runtime,
 * or a latency-critical path that must not enter the allocator.
 *   n          number of cells, 1 <= n <= 4,194,304 (larger n: INVALID_ARG; the
 *              fixed scratch holds one partial row per 1024 cells, 4096 rows)
 *   d_W        device, [n][3] FP64 (rho, rho u_x, rho u_y)            (read)
 *   d_vol      device, [n] FP64 cell areas                            (read)
 *   d_snap     device, [n][2] FP64 (U0, V0) snapshot: read, then overwritten
 *              with the current (U, V), as sdugks_residual refreshes its own
 *   d_out      device, [3] FP64: eps (+inf when the snapshot is at rest), the mass
 *              sum V rho, and the count of cells with non-finite or zero-density W
 *   stream     cudaStream_t (NULL = default stream); the call is asynchronous
 * No memory is allocated and nothing is freed.  The scratch is 128 KiB of device
 * memory held on every GPU that loads the library until the process exits.  The
 * first call on a device (with that device current) looks up the scratch's device
 * address; make that first call before any stream capture on that device.  All calls
 * share the scratch, and every call overwrites the rows it uses before reading them,
 * so calls that run one after another need no clearing; calls that overlap on the
 * GPU (different streams, no ordering) race on the scratch and give wrong results.
 * Errors: INVALID_ARG, CUDA (message in sdugks_last_error()). */
int sdugks_residual_noalloc(int64_t n, const double *d_W, const double *d_vol, double *d_snap, double *d_out,
                            void *stream);

int sdugks_solver_info(const sdugks_solver *s, sdugks_info *out);

/* ---- autotuner ------------------------------------------------------------------ */
/* A facility of this library (the paper has no counterpart): the launch configuration
 * of a solve chosen by timing it on the current device. */
typedef struct sdugks_tune_info {
    double ns_per_step;   /* measured time of one step with the chosen configuration   */
    int32_t candidates;   /* configurations timed (0 when the result came from the cache) */
    int32_t from_cache;   /* 1: an earlier call tuned the same mesh on this device        */
    int32_t kernel;       /* SDUGKS_KERNEL_TILED or SDUGKS_KERNEL_CARTESIAN                */
    int32_t pad_;
} sdugks_tune_info;

/* Time the candidate launch configurations of a solve of mesh m with base's tau, dt,
 * precision and kernel request, and return in *best a copy of *base with the fastest
 * tile_cells, graph_steps and staging.  Candidates: on the Cartesian kernel the block
 * shapes 16x16, 16x14, 16x8 (FP64: 16x16) with per-thread loads or TMA staging; on the
 * tiled kernel tiles of 64, 96, 108, 120 and 128 cells; each with graphs of 32, 64 and
 * 128 steps.  Each candidate is a temporary solver at rest (the work of a step does not
 * depend on the state) timed over `steps` steps, rounded up to whole graphs, with CUDA
 * events on `stream` (a cudaStream_t; NULL = default stream), after one graph of warm-up.
 * The result is cached per (device, mesh and boundary rules, precision, kernel request)
 * for the life of the process; later calls return it without timing.  Choosing among
 * these does not change the method: every configuration runs the same sums per cell
 * (FP64 results are bit-identical across tile sizes, graph lengths and stagings; FP32
 * results agree to rounding across Cartesian block shapes).  Synchronises.  Allocates
 * and frees the candidates' device memory.  Errors: INVALID_ARG, OOM, CUDA. */
int sdugks_autotune(const sdugks_mesh *m, const sdugks_params *base, int64_t steps, void *stream,
                    sdugks_params *best, sdugks_tune_info *info);

/* Forget every cached autotuning result. */
void sdugks_autotune_clear(void);

/* ---- batched solves ----------------------------------------------------------- */
/* Many independent uniform-grid solves (cavities, channels) of different sizes and
 * Reynolds numbers advanced together: every step is one launch over the (instance,
 * 16x8 block) work list of all instances, one CTA per item (or, if the autotuner
 * prefers it, a fixed grid of CTAs walking the list), with the S-DUGKS update of
 * Sec. II per block; steps replay a captured CUDA graph.  Each
 * instance's arithmetic is the same as a single solver's Cartesian kernel on the
 * same mesh, so its results do not depend on what else is in the batch.  Instances
 * are admitted while the batch's device pool has room for their state (admission
 * by device-memory footprint) and can be removed at any step boundary, which frees
 * their memory for new ones (continuous batching). */
typedef struct sdugks_batch sdugks_batch;

typedef struct sdugks_batch_status {
    int64_t instances;       /* active instances                                    */
    int64_t cells;           /* cells over active instances                         */
    int64_t items;           /* (instance, block) work items per step               */
    int64_t pool_bytes;      /* device pool size                                    */
    int64_t pool_used;       /* bytes held by active instances                      */
    int64_t steps;           /* batch steps since creation                          */
    int32_t grid;            /* CTAs per step launch (the item count if per_item)   */
    int32_t ctas_per_sm;     /* resident CTAs per SM of the batched kernel          */
    int32_t graph_steps;     /* steps per captured graph                            */
    int32_t precision;
    int32_t per_item;        /* 1: one CTA per work item; 0: a fixed grid walks the
                                work list                                           */
} sdugks_batch_status;

/* Create a batch with a device pool of pool_bytes and room for max_instances
 * instances.  precision: SDUGKS_FP32, SDUGKS_FP32_BF16DEV or SDUGKS_FP32_FP16DEV.  stream as for
 * solvers.  Errors: INVALID_ARG, OOM, CUDA. */
int sdugks_batch_create(int64_t pool_bytes, int32_t precision, int32_t max_instances, void *stream,
                        sdugks_batch **out);

/* Bytes of pool an instance on this mesh would take (state f, W and the residual
 * snapshot, padded).  INVALID_ARG if the mesh is not a uniform Cartesian grid. */
int sdugks_batch_footprint(const sdugks_batch *b, const sdugks_mesh *mesh, int64_t *bytes);

/* Admit a solve on a uniform Cartesian grid (sides: walls, moving walls, far field,
 * outlet or periodic pairs) with relaxation time tau and time step dt, started from
 * rho[nx*ny], u[nx*ny][2] (host, cell order of the mesh; NULL = 1 and 0).  *id is
 * its handle.  FULL when the pool or the instance table has no room; INVALID_ARG if
 * the mesh is not a uniform grid.  The residual snapshot is taken at admission. */
int sdugks_batch_add(sdugks_batch *b, const sdugks_mesh *mesh, double tau, double dt, const double *rho,
                     const double *u, int64_t *id);

/* Remove an instance (its memory returns to the pool).  INVALID_ARG for an unknown id. */
int sdugks_batch_remove(sdugks_batch *b, int64_t id);

/* Advance every active instance by n steps (async). */
int sdugks_batch_step(sdugks_batch *b, int64_t n);

/* Residual and mass of every active instance against its snapshot, which is then
 * refreshed (as sdugks_residual).  ids, eps, mass: host arrays of at least
 * max_instances entries (any may be NULL); *count = active instances.  Steps taken
 * by instance ids[k] since admission go to steps[k] if steps is not NULL.
 * Synchronises.  Non-finite states are reported as eps = NaN (no error). */
int sdugks_batch_residual(sdugks_batch *b, int64_t *ids, double *eps, double *mass, int64_t *steps, int64_t *count);

/* rho[nx*ny], u[nx*ny][2] of one instance (host; synchronises). */
int sdugks_batch_get_macros(sdugks_batch *b, int64_t id, double *rho, double *u);

/* Time `steps` steps of each candidate launch form and keep the fastest: one CTA per
 * work item (the default), or a fixed grid of 1, 2 or 4 times the resident CTAs that
 * walks the work list (see sdugks_batch_status.per_item and .grid).  Call with
 * instances admitted.  With one CTA per item, the step graph is captured again after
 * the item count changes (instances admitted or removed). */
int sdugks_batch_autotune(sdugks_batch *b, int64_t steps);

int sdugks_batch_info(const sdugks_batch *b, sdugks_batch_status *out);

void sdugks_batch_destroy(sdugks_batch *b);

void sdugks_solver_destroy(sdugks_solver *s);

/* ---- rarefied flow on a discrete velocity grid (Sec. IV, micro cavity) ----------
 * The same step (Sec. II) with the D2Q9 lattice replaced by nv x nv velocity nodes at
 * the midpoints of a uniform partition of [-vmax, vmax]^2 (weights (2 vmax/nv)^2),
 * the Maxwellian of Eq. Feq (exponent |xi - u|^2 / (2 R T), two dimensions) and
 * W = (rho, rho u, rho E) with psi = (1, xi, xi^2/2) (Eq. Macro), R T = E - |u|^2/2.
 * Boundary faces must be PERIODIC (paired), WALL or MOVING_WALL; walls scatter
 * diffusely (Sec. III): velocities entering the gas take the wall Maxwellian at
 * R T_wall with the density that makes the wall pass no mass (Eqs. 6001-6002),
 * leaving ones the characteristic reconstruction from the inner cell.  Any other
 * boundary kind gives BAD_BC at creation.  f is stored [cell][velocity] (weighted
 * values f_q = w_q f(xi_q)), W [cell][4] in FP64.  Device memory: about
 * 4 x (2 n_cells + n_faces) x Q bytes (FP32). */
typedef struct sdugks_dvm sdugks_dvm;

typedef struct {
    int32_t nv;          /* velocity nodes per axis (Q = nv^2), 2..1024 */
    double vmax;         /* the grid spans [-vmax, vmax]^2 */
    double RT_wall;      /* R T of the walls (and the default initial state) */
    double tau, dt;      /* relaxation time and time step (lattice units) */
    int32_t precision;   /* SDUGKS_FP64 or SDUGKS_FP32 (f and the scratch arrays) */
    int32_t graph_steps; /* steps per captured CUDA graph: 0 = 32, < 0 = no graphs */
} sdugks_dvm_params;

/* Create on the current device; stream may be NULL (legacy default stream).
 * Errors: INVALID_ARG (NULL, nv out of range, non-positive vmax/RT_wall/tau/dt,
 * precision), INVALID_MESH (more than 4 faces per cell), BAD_BC, OOM, CUDA. */
int sdugks_dvm_create(const sdugks_mesh *mesh, const sdugks_dvm_params *params, void *stream, sdugks_dvm **out);

/* Initial state W = (rho, rho u, rho (|u|^2/2 + R T)), f = feq(W).  rho[n], u[n][2],
 * RT[n] host arrays in user cell order; NULL gives 1, (0, 0) and RT_wall. */
int sdugks_dvm_init(sdugks_dvm *d, const double *rho, const double *u, const double *RT);

/* n steps, asynchronous on the solver's stream. */
int sdugks_dvm_step(sdugks_dvm *d, int64_t n);

/* rho[n], u[n][2], RT[n] from W (host; any may be NULL; synchronises). */
int sdugks_dvm_get_macros(sdugks_dvm *d, double *rho, double *u, double *RT);

/* f[n][Q] (weighted, FP64) and W[n][4] (host; either may be NULL; synchronises). */
int sdugks_dvm_get_state(sdugks_dvm *d, double *f, double *W);

/* Sizes: cells, faces (periodic pairs merged), Q, device bytes. */
int sdugks_dvm_sizes(const sdugks_dvm *d, int64_t *n_cells, int64_t *n_faces, int64_t *n_velocities,
                     int64_t *device_bytes);

void sdugks_dvm_destroy(sdugks_dvm *d);

/* Message of the last failed call on this thread ("" if none). */
const char *sdugks_last_error(void);

/* Library version string, e.g. "sdugks 0.1 sm_103a". */
const char *sdugks_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SDUGKS_H */
