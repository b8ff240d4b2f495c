/*
 * rich.h - C ABI of the GB300 moving-Voronoi-mesh hydrodynamics sweep.
 *
 * One time step of the moving-mesh Godunov scheme of Yalinewich, Steinberg &
 * Sari, "RICH: Open Source Hydrodynamic Simulation on a Moving Voronoi Mesh"
 * (arXiv:1410.3219), Section 2, with the "extrapolated fluxes" time
 * advancement of Section 2.3:
 *
 *   a0  host: ghost images + Delaunay triangulation by point insertion with
 *       exact, tie-broken in-circle predicates (Section 2.1)
 *   a1  Voronoi geometry: circumcentres, areas, centres of mass, edge lengths,
 *       midpoints, normals, c_ij (quantities defined under Eq. 1)
 *   a2  primitive variables rho, v, p and sound speed (ideal gas)
 *   a3  Green-Gauss gradients (Eq. 1)
 *   a4  AREPO limiter (Eqs. 3-5), TESS limiter (Eq. 6), per-cell switch (Eqs. 7-8)
 *   a5  mesh-point velocities with cell rounding (Section 6)
 *   a6  Courant time step (Section 2.3)
 *   a7  per edge: linear extrapolation (Eq. 2), half-step prediction, boost
 *       into the moving edge's frame (Section 1), rotation, HLLC (Section 2.4)
 *   a8  conservative update U_i -= dt * sum_j L_ij F_ij (Section 5)
 *   a9  advance the mesh-generating points
 *
 * Steps a1-a9 run as CUDA kernels on the device (sm_103a); a0 runs on the host.
 *
 * Conventions
 *  - All arrays passed in or out are HOST arrays unless a name says "device".
 *    The library copies on entry and exit; the caller keeps ownership.
 *  - Per-cell arrays are indexed by the caller's point order (the library
 *    renumbers cells internally along a Hilbert curve and maps back).
 *  - Return value: RICH_OK (0) or a negative RICH_E* code; rich_strerror()
 *    gives a message, rich_last_error() the detail of the last failure on the
 *    calling thread.  No C++ exception crosses this boundary.
 *  - A rich_sim is used by one host thread at a time.
 */
#ifndef RICH_H
#define RICH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RICH_OK 0
#define RICH_EINVAL -1     /* bad argument: n < 3, point outside the box, rho/p <= 0, NaN, gamma <= 1 */
#define RICH_EDUPLICATE -2 /* two generating points coincide */
#define RICH_ETESS -3      /* tessellation failed (inconsistent connectivity) */
#define RICH_ETOOFEW -4    /* too few points for the ghost band to close every cell */
#define RICH_ENEGATIVE -5  /* a step produced m <= 0 or thermal energy <= 0, or moved a point so far
                              that reflecting it at a rigid wall leaves it outside; the state stays
                              at the last good step */
#define RICH_ENAN -6       /* a step produced a non-finite value; state kept as for RICH_ENEGATIVE */
#define RICH_ENOMEM -7     /* device or host allocation failed */
#define RICH_ECUDA -8      /* CUDA runtime error (see rich_last_error) */
#define RICH_ENODEV -9     /* no CUDA device */
#define RICH_ESTATE -10    /* call not valid in the current state */

#define RICH_BC_REFLECTIVE 0 /* rigid walls (mirror ghosts) */
#define RICH_BC_PERIODIC 1

#define RICH_MESH_LAGRANGIAN 0 /* w = v plus the Section 6 rounding velocity */
#define RICH_MESH_EULERIAN 1   /* w = 0 */

#define RICH_LIM_SWITCHED 0 /* AREPO, TESS where Eqs. 7-8 flag a shock (paper default) */
#define RICH_LIM_AREPO 1
#define RICH_LIM_TESS 2

#define RICH_SCHEME_EXTRAPOLATED 0 /* Section 2.3 "extrapolated fluxes": one sweep per step, edge
                                      states advanced half a step in time */
#define RICH_SCHEME_TIME_CENTRED 1 /* Section 2.3 "time centred fluxes" (the paper's own): a half
                                      step with spatially extrapolated edge states, the mesh rebuilt
                                      at the half-step points, then the full step from the
                                      start-of-step state with the half-step fluxes and mesh
                                      velocities; two tessellations and two sweeps per step.
                                      Single simulations only (batches and the server reject it). */

#define RICH_FP64 0       /* every step in FP64 */
#define RICH_FP32_SPLIT 1 /* primitives, gradients, limiter, mesh velocity, edge states and HLLC in
                             FP32; positions, Voronoi vertices, areas, centres of mass, coordinate
                             differences and the conserved variables (with the flux sums) in FP64 */

typedef struct rich_sim rich_sim;

/* Scheme parameters.  Paper defaults: cfl 0.3 (Section 2.3); theta 0.5,
   delta_v 0.2, delta_p 0.7 (Section 2.2); chi 0.15, eta 0.02 (Section 6). */
typedef struct {
    double gamma;                   /* ideal-gas adiabatic index, > 1 */
    double cfl;                     /* Courant number */
    int32_t boundary;               /* RICH_BC_* */
    double x0, x1, y0, y1;          /* domain box */
    int32_t motion;                 /* RICH_MESH_* */
    double chi, eta;                /* cell-rounding speed (units of c_s) and trigger distance (units of R_i) */
    double theta, delta_v, delta_p; /* TESS factor and shock-switch thresholds */
    int32_t limiter;                /* RICH_LIM_* */
    int32_t scheme;                 /* RICH_SCHEME_* */
    int32_t precision;              /* RICH_FP64 | RICH_FP32_SPLIT */
} rich_config;

typedef struct {
    int64_t steps_done; /* steps completed by this call */
    double t;           /* simulation time after the call */
    double dt_last;     /* last time step */
    double sweep_ms;    /* device time of steps a1-a9 summed over the call (CUDA events) */
    double tess_ms;     /* host time of a0 summed over the call */
    double copy_ms;     /* host time spent in host<->device copies and waits */
    int64_t n_ghost, n_tri, n_edges, n_slots; /* size of the last tessellation */
} rich_step_info;

/* Fill cfg with the paper's defaults (gamma 5/3, unit periodic box). */
void rich_default_config(rich_config *cfg);

/* Create a simulation from n generating points (x, y) inside the box and the
   primitive fields rho, vx, vy, p at those points (the problem statement of
   Sections 3-4: generating points, primitive fields, gamma, CFL, boundary).
   Tessellates, computes the initial cell areas and stores the extensive
   conserved variables (m, momentum, E) = (rho, rho v, p/(gamma-1) + rho|v|^2/2) * A
   on the device.  Points must lie strictly inside a walled box (periodic:
   x0 <= x < x1).  *out receives the handle; it owns all device memory and a
   CUDA stream.  Errors: RICH_EINVAL, RICH_EDUPLICATE, RICH_ETOOFEW,
   RICH_ENOMEM, RICH_ENODEV, RICH_ECUDA. */
int rich_init_mesh(const rich_config *cfg, int64_t n, const double *x, const double *y, const double *rho,
                   const double *vx, const double *vy, const double *p, rich_sim **out);

/* Advance up to max_steps steps, stopping early once the time reaches t_end
   (the last step is shortened to land on t_end).  Each step: a0 on the host
   for the current points, then a1-a9 on the device (twice, with a0 for the
   half-step points in between, in the time-centred scheme).  The points'
   motion (a9) needs only the mesh velocity and dt, known after the geometry
   stage, so each sweep writes the moved points first; the call reads them
   back then and runs a0 for them on the host while the device computes the
   gradients, fluxes and update.  A step that does not land on t_end thus
   leaves the mesh of its points built, and the next step or call starts
   with the sweep.  Results equal those of rich_tessellate / rich_sweep /
   rich_sync in turn, bit for bit.  info may be NULL.
   Errors: RICH_ENEGATIVE / RICH_ENAN (state left at the last good step),
   RICH_ETESS, RICH_EDUPLICATE, RICH_ECUDA. */
int rich_step(rich_sim *s, int32_t max_steps, double t_end, rich_step_info *info);

/* Primitive fields and cell areas on the current generating points (each
   output may be NULL; n must equal the simulation's size).  If the points
   moved since the last tessellation this tessellates and recomputes the
   geometry first.  Between the two sweeps of a time-centred step (pieces
   API below) the current points and state are the half-step ones; the same
   holds for rich_get_conserved. */
int rich_get_state(rich_sim *s, int64_t n, double *x, double *y, double *rho, double *vx, double *vy,
                   double *p, double *area);

/* Extensive conserved variables and generating points (each may be NULL). */
int rich_get_conserved(rich_sim *s, int64_t n, double *x, double *y, double *m, double *px, double *py,
                       double *E);

/* ---- checkpoint and restart (no counterpart in the paper) ---------------
   A checkpoint taken between steps is the configuration, rich_time, the
   points and conserved variables of rich_get_conserved, and the cell order
   of rich_get_order.  rich_init_conserved restarts from it; the restarted
   simulation then repeats the uninterrupted one bit for bit (same precision,
   scheme and device).  order may be NULL: cells are then renumbered along a
   Hilbert curve of the given points (a valid restart, not bit-identical).
   Errors as rich_init_mesh; RICH_EINVAL also for a non-positive mass or
   thermal energy, or an order that is not a permutation of 0..n-1. */
int rich_init_conserved(const rich_config *cfg, int64_t n, const double *x, const double *y, const double *m,
                        const double *px, const double *py, const double *E, double t, const int64_t *order,
                        rich_sim **out);
/* order[k] = the caller's index of the simulation's k-th internal cell. */
int rich_get_order(const rich_sim *s, int64_t n, int64_t *order);
/* Simulation time (-1 for a NULL handle). */
double rich_time(const rich_sim *s);

/* Release the handle and all its device memory.  NULL is ignored. */
void rich_destroy(rich_sim *s);

const char *rich_strerror(int code);
const char *rich_last_error(void);

/* ---- pieces of a step, for measurement and inspection ------------------- */

/* Launch all device work of this handle on the given cudaStream_t (NULL:
   the handle's own stream).  The caller keeps the stream alive. */
int rich_set_stream(rich_sim *s, void *cuda_stream);

/* a0 for the current points: copy points device->host, tessellate on the
   host, upload the rings (with each cell's first owned triangle and edge)
   and build the triangle and edge lists from them on the device.
   Synchronous.  RICH_ETESS if the device lists do not close. */
int rich_tessellate(rich_sim *s, rich_step_info *info);

/* Enqueue a1-a9 for one step on the current connectivity (asynchronous; no
   host synchronisation).  Requires a current tessellation.  In the
   time-centred scheme a step takes two rounds of rich_tessellate /
   rich_sweep / rich_sync: the first sweep (half step) leaves the half-step
   points current, the second completes the step. */
int rich_sweep(rich_sim *s, double t_end);

/* Wait for the enqueued sweep, read time step, time and status flags.
   Returns RICH_ENEGATIVE / RICH_ENAN if the last sweep failed (then the
   state is rolled back to before that sweep). */
int rich_sync(rich_sim *s, rich_step_info *info);

/* Per-cell diagnostics of the last sweep, caller's order, n doubles:
   0 area, 1-2 centre of mass, 3-6 rho vx vy p, 7 c_s, 8-15 unlimited gradient
   (d/dx, d/dy of rho, vx, vy, p), 16-23 limited gradient, 24-25 w,
   26 TESS flag, 27-30 alpha (rho, vx, vy, p), 31 dt (same value in every cell).
   A later tessellation leaves them alone; rich_get_state's geometry pass
   replaces fields 0-7 with those of the current points. */
int rich_get_field(rich_sim *s, int32_t field, int64_t n, double *out);

/* Write (on, the default) or skip (off) the inspection-only per-cell arrays
   of a sweep: unlimited gradient, alpha and TESS flag (fields 8-15, 26-30
   of rich_get_field).  The step's results do not depend on it. */
int rich_set_diagnostics(rich_sim *s, int32_t on);

/* Per-stage device times of the last synchronised sweep, from CUDA events
   recorded on the launching stream between the stages (enabled by
   rich_set_profiling; off by default).  Stages, in launch order:
   k_circumcentre, k_geometry (edge and cell geometry with the primitives,
   mesh velocity and Courant candidates, in one launch), k_advance_points,
   k_cell_gradient, k_edge_flux, k_cell_update.  *count receives the number of
   stages; up to cap values (milliseconds) are written to ms. */
int rich_set_profiling(rich_sim *s, int32_t on);
int rich_kernel_times(rich_sim *s, int32_t cap, double *ms, int32_t *count);
const char *rich_kernel_name(int32_t stage);

/* Wall time (ms) of the phases of the handle's last host tessellation (a0):
   ms[0] ghost images, point copies, bounding box and bucket grid; ms[1] the
   tiles (triangulation or in-place update, star checks, rings); ms[2]
   triangle and ring assembly; ms[3] edge counts and processing order. */
int rich_tess_phases(const rich_sim *s, double *ms);

/* Number of cells of the handle. */
int64_t rich_num_cells(const rich_sim *s);

/* ---- batches of independent simulations ---------------------------------- */

/* A batch advances many independent simulations (different sizes, problems
   and scheme parameters, one precision) with ONE device sweep per step over
   all their cells: each step tessellates every simulation on a pool of host
   threads, packs the meshes into one index space with a per-cell simulation
   id, and runs steps a1-a9 once; every simulation keeps its own time step,
   end time, step budget and status.  A cell's arithmetic depends only on its
   own simulation, so results are identical alone and in any mix.  The batch
   owns its device memory and stream. */
typedef struct rich_batch rich_batch;

#define RICH_SIM_PENDING 0  /* admitted, not yet stepped */
#define RICH_SIM_RUNNING 1
#define RICH_SIM_DONE 2     /* reached t_end or max_steps; state kept for reading */
#define RICH_SIM_FAILED 3   /* a step or a tessellation failed; last good state kept */

/* max_cells: admission budget (cells of pending + running simulations);
   device memory grows to about 1 KiB per admitted cell.  host_threads <= 0:
   one per hardware thread.  Errors: RICH_EINVAL, RICH_ENODEV, RICH_ECUDA. */
int rich_batch_create(int32_t precision, int64_t max_cells, int32_t host_threads, rich_batch **out);

/* Admit a simulation (arguments as rich_init_mesh, cfg->precision must equal
   the batch's) that runs until t_end or max_steps steps.  It joins the
   device sweep at the next rich_batch_step.  *id receives its handle.
   Errors: RICH_EINVAL, RICH_ENOMEM when the cell budget would be exceeded. */
int rich_batch_add(rich_batch *b, const rich_config *cfg, int64_t n, const double *x, const double *y,
                   const double *rho, const double *vx, const double *vy, const double *p, double t_end,
                   int64_t max_steps, int32_t *id);

/* One step of every pending or running simulation.  With the staged
   launch, the moved points are read back once the point motion is done and
   the simulations that go on are tessellated for the next step while the
   device finishes the sweep (the next call then tessellates only newly
   admitted ones); results equal those without this overlap, bit for bit.
   info (nullable): steps_done = simulations stepped, sweep_ms = device time
   of the sweep, tess_ms = host tessellation wall time (both tessellations),
   copy_ms = other host time outside the sweep. */
int rich_batch_step(rich_batch *b, rich_step_info *info);

/* State (RICH_SIM_*), error code of a failed simulation, its time and steps
   taken, and for finished ones the wall time from rich_batch_add to the end
   of its last step (ms; -1 while running).  Each output may be NULL. */
int rich_batch_query(rich_batch *b, int32_t id, int32_t *state, int32_t *error, double *t, int64_t *steps,
                     double *latency_ms);

/* Generating points and extensive conserved variables of a running or
   finished simulation, caller's point order (each output may be NULL). */
int rich_batch_get_conserved(rich_batch *b, int32_t id, int64_t n, double *x, double *y, double *m, double *px,
                             double *py, double *E);

/* Forget a simulation (running ones leave the batch at the next step). */
int rich_batch_remove(rich_batch *b, int32_t id);

/* As rich_set_diagnostics, for the batch (off by default). */
int rich_batch_set_diagnostics(rich_batch *b, int32_t on);

/* Cells of pending + running simulations. */
int64_t rich_batch_cells(const rich_batch *b);

/* How a batch launches its sweep.  mode 0 (default): autotune; the first
   eight steps each try one of {stage by stage, persistent with 128, 256, 512
   threads per block} twice, and the fastest is kept.  mode 1: stage by stage
   (one kernel per stage).  mode 2: persistent with `block` threads (128,
   256 or 512): all stages in one cooperative kernel launch, grid-stride
   loops, one block per co-resident slot on every SM, stages separated by
   grid barriers whose waits give up after about a second (the step is then
   redone stage by stage and mode 1 is kept).  The persistent launch is
   recorded once as a CUDA graph and replayed every step (the mesh sizes are
   read from device memory); it is recorded again when a device buffer
   moves.  Results do not depend on the mode. */
int rich_batch_set_launch(rich_batch *b, int32_t mode, int32_t block);

/* The launch shape in use (persistent 0/1, block, grid of the last
   persistent launch, tuning finished 0/1, graph replay available 0/1) and
   counts[4] = {staged steps, persistent steps, graph replays, graph
   recordings}; each output may be NULL. */
int rich_batch_launch_info(const rich_batch *b, int32_t *persistent, int32_t *block, int32_t *grid, int32_t *tuned,
                           int32_t *graph, int64_t *counts);

/* Failure detection of the persistent sweep (no counterpart in the paper).
   Its grid barriers wait a bounded number of polls; a wait that runs out
   stops the sweep with the step's inputs untouched, and the batch redoes
   the step with staged launches and keeps them.  With spin_limit > 0 the
   next persistent sweep is made to fail that way: its barrier waits for one
   block more than it launched, and every wait gives up after spin_limit
   polls (about 0.1-1 us each).  *timeouts_seen (nullable) receives the
   number of persistent sweeps whose barrier timed out so far.
   Errors: RICH_EINVAL. */
int rich_batch_inject_barrier_timeout(rich_batch *b, int32_t spin_limit, int64_t *timeouts_seen);

void rich_batch_destroy(rich_batch *b);

/* ---- continuous-batching server -------------------------------------------- */

/* A request loop over a batch: submitted simulations wait in arrival order
   and are admitted at the next tick at which their cells fit in the device
   budget; each tick advances every admitted simulation by one step in one
   batched sweep, and finished ones free their cells at once.  State stays on
   the device between ticks.  Per request the server records queueing time
   (submission to admission) and latency (submission to the end of its last
   step), host wall clock in milliseconds. */
typedef struct rich_server rich_server;

#define RICH_REQ_QUEUED 0
#define RICH_REQ_RUNNING 1
#define RICH_REQ_DONE 2
#define RICH_REQ_FAILED 3

/* As rich_batch_create; max_cells is the admission budget. */
int rich_server_create(int32_t precision, int64_t max_cells, int32_t host_threads, rich_server **out);

/* Queue a simulation (inputs are copied; arguments as rich_batch_add).
   *req receives the request id.  Errors: RICH_EINVAL (also for n above the
   budget); invalid simulation parameters surface as a failed request. */
int rich_server_submit(rich_server *s, const rich_config *cfg, int64_t n, const double *x, const double *y,
                       const double *rho, const double *vx, const double *vy, const double *p, double t_end,
                       int64_t max_steps, int64_t *req);

/* Admit what fits, then one batched step.  info as rich_batch_step; the
   counts of requests admitted this tick, still running, and still queued
   (each output may be NULL). */
int rich_server_tick(rich_server *s, rich_step_info *info, int32_t *admitted, int32_t *running, int32_t *queued);

/* State (RICH_REQ_*), error code of a failed request, steps taken, queueing
   time (-1 while queued) and latency (-1 until finished). */
int rich_server_query(rich_server *s, int64_t req, int32_t *state, int32_t *error, int64_t *steps, double *queue_ms,
                      double *latency_ms);

/* Results of a finished request (as rich_batch_get_conserved), then forget it. */
int rich_server_fetch(rich_server *s, int64_t req, int64_t n, double *x, double *y, double *m, double *px,
                      double *py, double *E);

/* Hand the server to lane threads (asynchronous mode; no counterpart in the
   paper): `lanes` (1-4) threads each step their own batch, with its own CUDA
   stream, in a loop for as long as it has admitted requests; the lanes share
   the server's host threads task by task, the lanes of larger requests
   first.  A request goes to lane k when its cell count is at
   least split_cells * 8^(k-1) (lane 0 below split_cells), so small requests
   never wait on the host tessellation of large ones, and one lane's host
   tessellation overlaps another's device sweep.  Admission takes each
   lane's queue in arrival order against the shared cell budget; the lane of
   the largest requests also holds at most top_lane_cells cells at once (a
   larger request alone; 0: no limit but the budget), so that its requests
   run nearly one at a time with the whole worker pool instead of all
   sharing it for their whole run.  Each lane's device memory grows to the
   cells it has held.  Call it before any request is admitted; afterwards
   rich_server_tick returns RICH_ESTATE and the caller polls
   rich_server_query.  Errors: RICH_EINVAL, RICH_ESTATE. */
int rich_server_start(rich_server *s, int32_t lanes, int64_t split_cells, int64_t top_lane_cells);

/* Totals over the server's steps (each output may be NULL): batched steps
   taken by all lanes, summed device sweep time, host tessellation time and
   other host time (ms), and the wall time since rich_server_start (ms; 0 in
   tick mode).  (sweep + tessellation) / wall above one shows host and
   device work overlapping. */
int rich_server_stats(rich_server *s, int64_t *steps, double *sweep_ms, double *tess_ms, double *other_ms,
                      double *wall_ms);

/* The batch of lane 0 (for rich_batch_set_launch / launch_info). */
rich_batch *rich_server_batch(rich_server *s);

void rich_server_destroy(rich_server *s);

/* ---- time step without allocation ---------------------------------------- */

/* Largest n accepted by rich_courant_dt_noalloc. */
#define RICH_NOALLOC_MAX_CELLS (1 << 24)

/* The paper has no counterpart to this entry point.  It serves callers that
   cannot allocate GPU memory when they need the time step: code running
   inside a memory pool or arena that owns the device, and code that must not
   trigger the device synchronisation an allocation or free can cause.

   Computes the Courant time step of the sweep (step a6) in FP64, before the
   step is shortened to land on an end time:
   dt = cfg->cfl * min_i R_i / (c_i + |v_i - w_i|), R_i = sqrt(area_i/pi),
   c_i = sqrt(gamma p_i/rho_i) (w = 0 for RICH_MESH_EULERIAN, when wx, wy may
   be NULL), over n cells whose values are DEVICE arrays of doubles owned by
   the caller, and writes it to the DEVICE double *dt_out, asynchronously on
   the cudaStream_t stream (NULL: the default stream).  The FP64 formula is
   used whatever cfg->precision says (a RICH_FP32_SPLIT sweep evaluates it in
   FP32).  Cells whose time step is +inf are skipped, as the sweep skips
   them; a cell whose time step is NaN, negative or -0.0 (a negative or NaN
   pressure or density) makes *dt_out a NaN instead of being skipped.
   It allocates nothing: its scratch (one partial minimum per block of 256
   cells and a completion counter, 512 KiB) is a fixed array in the
   library's device image, which every GPU that loads the library holds until
   the process exits.  The first call on each device looks up that array's
   address (cudaGetSymbolAddress), so make it before any stream capture.
   Every call shares the array and clears its counter: calls that overlap on
   the GPU (other streams, other host threads) race and must not be issued.
   Returns RICH_EINVAL for a configuration that rich_init_mesh rejects, a
   NULL array, or n outside [1, RICH_NOALLOC_MAX_CELLS], RICH_ECUDA if the
   set-up or launch fails (rich_last_error gives the reason). */
int rich_courant_dt_noalloc(const rich_config *cfg, int64_t n, const double *area, const double *rho,
                            const double *vx, const double *vy, const double *p, const double *wx,
                            const double *wy, double *dt_out, void *stream);

/* ---- measurement ----------------------------------------------------------- */

/* Measured arithmetic peaks of the current device (no counterpart in the
   paper): independent chains of FP64 and of FP32 fused multiply-adds, timed
   with CUDA events (best of three after a warm-up launch), in TFLOP/s
   counting a fused multiply-add as two operations.  Synchronous; allocates
   a few KiB for the duration of the call.  Errors: RICH_EINVAL (NULL
   output), RICH_ECUDA. */
int rich_probe_pipe_peaks(double *fp64_tflops, double *fp32_tflops);

/* ---- host-only entry points (no GPU needed) ----------------------------- */

/* Delaunay triangulation of n distinct points with the library's host
   builder (exact, tie-broken predicates).  Writes up to cap triangles (3
   point ids each; ids >= n are the corners of the enclosing triangle) and
   sets *ntri.  Returns RICH_EDUPLICATE, RICH_ETESS or RICH_EINVAL (cap too
   small, *ntri then holds the size needed). */
int rich_delaunay_host(int64_t n, const double *x, const double *y, int64_t cap, int32_t *tris, int64_t *ntri);

/* Voronoi neighbour rings of the n real cells of a box with ghosts (host a0
   only): ptr[n+1] offsets, and for each ring slot the neighbour's position
   (nbx, nby) and its source cell (caller order) in counter-clockwise order.
   cap is the capacity of nbx/nby/nbsrc; *nslots receives the size needed. */
int rich_rings_host(const rich_config *cfg, int64_t n, const double *x, const double *y, int64_t cap,
                    int64_t *ptr, double *nbx, double *nby, int64_t *nbsrc, int64_t *nslots);

/* The device's edge-list and triangle-list builders against the host's
   (a0 support; needs a GPU): builds the mesh of the n points on the host with
   its own lists, runs the device builders on the same rings, and counts the
   entries of the slot-to-edge map and of the edge arrays (left and right
   points, the two Voronoi vertices) that differ, and the vertices of each
   ring slot's triangle that differ (the triangles' numbering differs: the
   host's is per tile, the device's per owning cell).  *edges receives the
   number of edges.
   Errors: RICH_EINVAL, RICH_ENODEV, RICH_ECUDA, tessellation errors. */
int rich_edge_list_check(const rich_config *cfg, int64_t n, const double *x, const double *y, int64_t *edges,
                         int64_t *mismatched);

/* Check of the host builder's in-place update (a0 keeps each tile's last
   triangulation, moves its vertices, flips to Delaunay and inserts new
   points, rebuilding a tile only when a triangle turned over): builds the
   meshes of `steps` successive point sets (xs, ys: steps x n, row-major,
   the same cells in each) once with one reused workspace and once afresh
   each, with `threads` host threads, and counts the steps whose sweep
   inputs differ (rings, their neighbours and triangles, the edge list and
   each cell's first owned edge, ghosts) or whose first owned edges do not
   match the edge list.  A third reused workspace builds the sequence as a
   simulation does (rings only, read off incrementally, with each cell's
   first owned edge and triangle for the device's lists); a step whose
   rings, ghosts, first owned edges or processing order differ from the
   fresh build's counts as well.  *updated and *rebuilt receive the tile counts of the reused
   workspace over all steps, *reinserted the vertices it took out and put
   back where triangles would have turned over.  Returns RICH_EINVAL for bad
   arguments or the builder's error. */
int rich_mesh_update_check(const rich_config *cfg, int64_t n, int32_t steps, const double *xs, const double *ys,
                           int32_t threads, int32_t *mismatched, int64_t *updated, int64_t *rebuilt,
                           int64_t *reinserted);

#ifdef __cplusplus
}
#endif
#endif
