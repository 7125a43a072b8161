/*
 * cgks.h -- C ABI of libcgks: the compact 8th-order gas-kinetic scheme of
 * Zhao, Ji, Shyy, Xu, "An acoustic and shock wave capturing compact high-order
 * gas-kinetic scheme with spectral-like resolution" (arXiv 2001.01570), on one
 * GPU, in FP64.
 *
 * What one time step computes (every step runs entirely in CUDA kernels):
 *   - dt from the CFL condition, dt = CFL * min over cells of
 *     min(dx/(|U|+c+2 nu/dx), dy/(|V|+c+2 nu/dy)) (Sec. 4; nu = mu/rho, 0 for
 *     inviscid flow);
 *   - at every cell interface: the linear compact 8th-order reconstruction of
 *     the equilibrium state (Sec. 3.2, Eq. recons-8th-val) and the nonlinear
 *     WENO-Z compact reconstruction of the non-equilibrium left/right states
 *     (Sec. 3.3, Eq. sub-stencil, WENO-Z-w, smooth-indicator), from cell
 *     averages and cell-averaged gradients on the stencil {I_i-1..I_i+2};
 *   - the gas-kinetic evolution at two Gauss points per face (Sec. 2.1,
 *     Eq. 3rd-simplify-flux) with collision time
 *     tau = eps_tau*dt + c_tau*|p_l-p_r|/(p_l+p_r)*dt for inviscid flow, or
 *     tau = mu/p + c_tau*|p_l-p_r|/(p_l+p_r)*dt for viscous flow (Sec. 4),
 *     giving the time-accurate flux, its time derivative and the interface
 *     state;
 *   - the two-stage fourth-order update of cell averages (Sec. 2.2,
 *     Eq. step-hyper-1) and of the cell-averaged gradients by the Gauss
 *     theorem on the interface states (Sec. 3.1, Eq. compact-deriv-1).
 *
 * State layout ("planes"): structure of arrays of FP64, conservative
 * variables, row-major with x fastest:
 *   dim 2: 12 planes of ny*nx:  rho, rhoU, rhoV, rhoE,
 *                               d/dx of the four, d/dy of the four
 *          (cell averages and cell-averaged gradients), plane p, cell (i,j)
 *          at planes[p*ny*nx + j*nx + i];
 *   dim 1: 6 planes of nx:      rho, rhoU, rhoE, then their d/dx.
 *
 * Ownership: the library owns all device memory it allocates.  Pointers the
 * caller passes (host or device) are only read or written during the call
 * (or, for asynchronous calls, until the solver's stream reaches that point);
 * they are never retained.
 *
 * Errors: every entry point returns a cgks_status; nothing aborts or traps.
 * cgks_last_error() gives a thread-local human-readable detail for the last
 * failing call on the calling thread.  A solve that meets a non-physical state
 * (rho <= 0, p <= 0 or NaN in a reconstructed or updated state) stops with
 * CGKS_E_NONPHYSICAL and keeps its last valid state readable.
 */
#ifndef CGKS_H
#define CGKS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CGKS_OK = 0,
    CGKS_E_INVAL = 1,        /* invalid argument */
    CGKS_E_NOMEM = 2,        /* device or host allocation failed */
    CGKS_E_BUDGET = 3,       /* a served request can never fit the memory budget */
    CGKS_E_CUDA = 4,         /* a CUDA runtime call failed (detail in cgks_last_error) */
    CGKS_E_NONPHYSICAL = 5,  /* rho <= 0, p <= 0 or NaN met; the solve stopped */
    CGKS_E_TIMEOUT = 6,      /* a bounded wait expired */
    CGKS_E_BUSY = 7,         /* the object is in use (e.g. a server still running) */
    CGKS_E_NOTFOUND = 8      /* unknown request id */
} cgks_status;

/* boundary types of Sec. 4 (periodic, reflecting wall, supersonic inflow, outflow) */
typedef enum {
    CGKS_BC_PERIODIC = 0,  /* wrap around */
    CGKS_BC_REFLECT = 1,   /* mirror, normal momentum and the matching gradients odd */
    CGKS_BC_INFLOW = 2,    /* fixed state cgks_problem.inflow[side], zero gradients */
    CGKS_BC_OUTFLOW = 3    /* copy of the boundary cell, zero normal gradient */
} cgks_bc;

/* Statement of an Euler problem on a uniform grid (Sec. 2.1, Sec. 4). */
typedef struct {
    int dim;                 /* 1 or 2 */
    int nx, ny;              /* cells; ny is ignored (taken as 1) when dim == 1 */
    double x0, x1, y0, y1;   /* domain [x0,x1] x [y0,y1]; y0, y1 ignored when dim == 1 */
    double gamma;            /* ratio of specific heats, 1 < gamma < 3 (2D: < 2) */
    double cfl;              /* CFL number, > 0 */
    int bc[4];               /* cgks_bc for x-low, x-high, y-low, y-high */
    double inflow[4][4];     /* per side (x-low, x-high, y-low, y-high): primitive rho, u, v, p
                                of the fixed state on a CGKS_BC_INFLOW side (other sides ignore
                                theirs); rho > 0 and p > 0 are required where used */
    double eps_tau;          /* tau = eps_tau*dt + c_tau*|dp|/(sum p)*dt; paper: 0.01 */
    double c_tau;            /* paper: 1 */
    double weno_eps;         /* epsilon of the WENO-Z weights; paper tests 1e-6, 1e-4 */
    double mu;               /* dynamic viscosity; > 0 selects the viscous collision time
                                tau = mu/p + c_tau*|dp|/(sum p)*dt (Sec. 4; Navier-Stokes with
                                Prandtl number 1); 0: inviscid, tau from eps_tau */
    int recon_vars;          /* nonlinear (WENO-Z) reconstruction in 0: conservative variables,
                                1: characteristic variables of the normal flux Jacobian at the
                                mean of the two cells sharing the face (Sec. 3.2 allows either;
                                the linear reconstruction is the same in both) */
    int order;               /* spatial order of the compact reconstruction: 0 or 8 selects the
                                paper's 8th-order scheme (Sec. 3.2-3.3); 6 the compact 6th-order
                                variant that Sec. 3.2 names without printing: the linear
                                reconstruction is the degree-5 polynomial fixed by the four cell
                                averages and the slopes of the two cells next to the face, and
                                the WENO-Z step keeps the candidates q_0..q_6 with the linear
                                weights d = (3, 5, 8, 7, 7, 20, 20)/70 that recombine them into
                                that polynomial's interface value */
} cgks_problem;

typedef struct cgks_solver cgks_solver;   /* opaque; owns the device planes of one grid */

/* Create a solver for `prob` on the current CUDA device.  `cuda_stream` is a
 * cudaStream_t (NULL: the legacy default stream); all work of this solver is
 * ordered on it.  Allocates 3 x 12 planes of nx*ny doubles on the device.
 * Errors: CGKS_E_INVAL (bad dims, gamma, cfl, bc; a reflecting side needs at
 * least 2 cells), CGKS_E_NOMEM, CGKS_E_CUDA. */
cgks_status cgks_create(const cgks_problem* prob, void* cuda_stream, cgks_solver** out);

/* Free the solver and its device memory (synchronises its stream). */
cgks_status cgks_destroy(cgks_solver* s);

/* Copy an initial state (planes as described above) in, set time t and reset
 * the step count and error status.  `on_device` != 0: `planes` is a device
 * pointer.  Computes the CFL bound of the new state on the device. */
cgks_status cgks_set_state(cgks_solver* s, const double* planes, int on_device, double t);

/* Resume from a checkpoint: like cgks_set_state, but the step count starts at
 * `steps` (>= 0), the count cgks_get_state returned with the saved planes and
 * time.  The CFL bound of the restored state is computed with the same
 * rounding as at the end of a step, so that N steps, a checkpoint, a restore
 * into a new solver (same problem) and M more steps give the same bits as
 * N + M steps without interruption.  Errors: CGKS_E_INVAL, CGKS_E_CUDA. */
cgks_status cgks_restore_state(cgks_solver* s, const double* planes, int on_device, double t, long steps);

/* Copy the current state out (synchronises the stream).  t and steps may be
 * NULL.  Returns the solve's sticky status (CGKS_OK or CGKS_E_NONPHYSICAL). */
cgks_status cgks_get_state(cgks_solver* s, double* planes, int on_device, double* t, long* steps);

/* Advance `nsteps` S2O4 steps.  t_end > 0: the last step is shortened so that
 * t reaches t_end exactly and no step runs past it.  Synchronises the stream
 * before returning; *t_out (may be NULL) receives the new time.
 * Errors: CGKS_E_NONPHYSICAL (state kept at the last valid step), CGKS_E_CUDA. */
cgks_status cgks_step(cgks_solver* s, int nsteps, double t_end, double* t_out);

/* cgks_step with both stages of each step in one kernel launch (the temporal
 * fusion of the two-stage fourth-order step, Sec. 2.2, Eq. step-hyper-1): per
 * 16 x 8 tile, stage 1 runs on the tile widened by two cells and W* stays in
 * shared memory.  Same arguments, results (the same bits as cgks_step),
 * errors and step count; 2D only (CGKS_E_INVAL for 1D).  Every tile recomputes
 * the stage-1 work of its widened region, so on this FP64-bound path it is
 * slower than cgks_step. */
cgks_status cgks_step_fused(cgks_solver* s, int nsteps, double t_end, double* t_out);

/* Advance `n` independent solvers (any sizes and boundary types) by `nsteps`
 * steps each, each with its own dt, through one persistent launch per stage
 * over a flattened tile queue, replayed as a CUDA graph.  All solvers must live
 * on the current device; the work is ordered on the first solver's stream.
 * Synchronises before returning.  The status of each solver stays readable
 * through cgks_get_state. */
cgks_status cgks_batch_step(cgks_solver* const* solvers, int n, int nsteps);

/* Cells per CTA tile of the stage kernels for this solver's plain steps:
 * 0: 16x8, 1: 8x16, 2: 32x4, 3: 64x1, 4: 16x7, 5: 7x16, 6: 14x8, 7: 24x8,
 * 8: 16x14, 9: 20x11, 10: 15x15, 11: 22x10, 12: 18x12, 13: 20x12, 14: 15x16,
 * 15: 17x14, 16: 16x16, 17: 24x16, 18: 32x12; -1
 * restores the default (64x1 in 1D; in 2D 8x16, or 14x8 where it needs no more
 * passes of the persistent grid, as on small grids).  The shape changes only the
 * decomposition of the work, never the results.  Errors: CGKS_E_INVAL (1D
 * solvers take only 64x1; 2D solvers any other shape). */
cgks_status cgks_set_tile_shape(cgks_solver* s, int shape);

/* The solver's current tile shape (numbered as for cgks_set_tile_shape); -1
 * for a NULL solver. */
int cgks_tile_shape(const cgks_solver* s);

/* Tile shape (numbered as for cgks_set_tile_shape) that the autotuner of
 * cgks_batch_step chose for this exact batch, or -1 while it is still timing
 * the candidates.  The tuner times, on the first steps of a new batch
 * composition, the flux kernel's tile shapes 8x16, 14x8, 16x8 and 16x16 (with
 * 2, 1.75, 2 and 4 face segments per thread), then the update kernel at 2
 * and 4 cells per thread with the best shape (12 steps in all); neither choice
 * changes a result. */
int cgks_batch_tile_shape(cgks_solver* const* solvers, int n);

/* Cells per thread of the update kernel (1, 2 or 4) that the autotuner chose
 * for this exact batch, or -1 while it is still timing the candidates. */
int cgks_batch_update_cpt(cgks_solver* const* solvers, int n);

/* Same as cgks_step(s, nsteps, 0, NULL), but with CUDA events recorded on the
 * solver's stream around every kernel of every step; stage_ms[0..7] receive
 * the average duration in milliseconds of the step-begin, stage-1 record,
 * stage-1 flux, stage-1 update, stage-2 record, stage-2 flux, stage-2 update
 * and step-end kernels.  For measurement only (the events serialise nothing
 * but add host work per launch). */
cgks_status cgks_step_profiled(cgks_solver* s, int nsteps, double stage_ms[8]);

/* Device bytes a solver of this problem holds: three sets of 12 state planes
 * (current, next, intermediate), the face-row records of the stage in flight
 * (28 doubles per face row: x-faces 0..nx on rows -2..ny+1 and, in 2D, y-faces
 * 0..ny on columns -2..nx+1), the face results of the stage in flight (16
 * doubles per face) and 4 KB of descriptors.  The server admits a
 * request while these bytes fit its budget.  Returns 0 for a NULL or empty
 * problem. */
double cgks_problem_device_bytes(const cgks_problem* prob);

/* Kernel launch count of the most recent cgks_step / cgks_batch_step call on
 * the calling thread (for throughput accounting). */
long cgks_last_launch_count(void);

const char* cgks_status_string(cgks_status st);
const char* cgks_last_error(void);

/* ------------------------------------------------------------------------
 * Allocation-free stepping.  (The paper has no counterpart: this entry point
 * exists for callers of this library, not for the method.)
 *
 * Some callers cannot let a library call cudaMalloc: applications that manage
 * all device memory through their own pool or allocator, or embeddings with a
 * fixed device footprint where the allocator must not be re-entered.  cgks_step_noalloc advances a 2D problem whose state
 * the caller already holds in device memory and allocates nothing: the second
 * state buffer, the intermediate state, the face-row records, the control
 * block and the work queues live in fixed-size device arrays of the library
 * (file-scope __device__ storage, about 12.6 MB of state, 34 MB of face-row
 * records, 17 MB of face results and 300 KB of queues), which every GPU that
 * loads the library holds until the process exits.
 *
 * prob:        2D problem, nx*ny <= CGKS_NOALLOC_MAX_CELLS, nx and ny <=
 *              CGKS_NOALLOC_MAX_SIDE, at most CGKS_NOALLOC_MAX_TILES tiles of
 *              16x8 cells
 * planes:      device pointer, 12 planes of ny*nx doubles (layout above); read
 *              as the initial state and overwritten with the state after the
 *              steps (or the last valid state on CGKS_E_NONPHYSICAL)
 * nsteps:      S2O4 steps to take (dt from the CFL condition each step)
 * t_inout:     time of the state in, time after the steps out
 * cuda_stream: stream for all work (NULL: the legacy default stream); the
 *              call reads the control block back and synchronises the stream
 *              before returning, so it must not be called while a stream
 *              capture is active
 * Errors: CGKS_E_INVAL (3D/1D problem, grid larger than the maximum, bad
 * parameters), CGKS_E_NONPHYSICAL, CGKS_E_CUDA.
 * The first call on a device looks up the addresses of the fixed arrays and
 * sets kernel attributes.
 * All calls share the same arrays: calls whose work overlaps on the GPU (from
 * several threads or streams) race and must be serialised by the caller.
 * Each call re-initialises the control block and overwrites the scratch it
 * reads, so no state carries over from one call to the next. */
#define CGKS_NOALLOC_MAX_CELLS 65536
#define CGKS_NOALLOC_MAX_SIDE 4096
#define CGKS_NOALLOC_MAX_TILES 16384
cgks_status cgks_step_noalloc(const cgks_problem* prob, double* planes, int nsteps, double* t_inout,
                              void* cuda_stream);

/* Detail of the last failing cgks_step_noalloc call on the calling thread. */
const char* cgks_noalloc_last_error(void);

/* ------------------------------------------------------------------------
 * Serving: a continuous-batching solve server.  Requests (2D problems with an
 * initial state and a step count) may be submitted from any thread at any
 * time.  The server admits them in arrival order while fewer than max_active
 * solves are admitted and their device bytes (cgks_problem_device_bytes) fit
 * hbm_budget_bytes; it copies an admitted request's state to the GPU while
 * other solves run and adds it to the batched launch at the next round
 * boundary; all active solves advance together in rounds of steps_per_round
 * steps of that launch (each with its own dt and step target; the captured
 * step graphs are kept across changes of the active set, whose work queues are
 * rewritten in place); a finished solve is copied to host memory and its
 * device memory returned to the server's pool while later rounds run, so
 * waiting requests can enter.  A solve's result is the same whatever it
 * shares the launch with. */
typedef struct cgks_server cgks_server;

typedef struct {
    double hbm_budget_bytes;   /* device bytes the server may hold for solver state */
    int max_active;            /* at most this many solves share a launch */
    int steps_per_round;       /* steps between admission / retirement points */
    int tile_shape;            /* -1: autotune on the first batch; else a fixed shape */
    void* cuda_stream;         /* cudaStream_t of the rounds (NULL: a stream of the server's own);
                                  the copies run on two further streams of the server */
    const char* log_path;      /* NULL, or a file to which the server appends one JSON line per
                                  finished request: id, grid, steps, status, and the times (s since
                                  cgks_serve_start) of arrival, admission, first round and result */
    int order;                 /* which admitted solves a round computes:
                                  CGKS_SERVE_ALL_ACTIVE: every one (all advance at the same step rate);
                                  CGKS_SERVE_LEAST_WORK_FIRST: those with the fewest remaining
                                  cell-updates, as many as it takes to reach fill_cells cells (at least
                                  one); the others wait, state untouched, until they are among them.
                                  The order changes latencies, never a result. */
    double fill_cells;         /* cells a least-work-first round aims for (enough to fill the GPU:
                                  4e6 is the 2048^2 grid) */
} cgks_serve_cfg;

#define CGKS_SERVE_ALL_ACTIVE 0
#define CGKS_SERVE_LEAST_WORK_FIRST 1

typedef struct {
    cgks_problem prob;         /* dim must be 2 */
    const double* init_planes; /* host, 12 planes of ny*nx; copied during the call */
    int nsteps;                /* S2O4 steps to run */
} cgks_request;

typedef struct {
    long submitted, completed, rejected, failed, active, pending, rounds;
    double cell_updates;        /* completed solves: sum of cells x steps */
    double wall_s;              /* first arrival to last completion */
    double busy_s;              /* time during which at least one solve was active on the GPU */
    double cell_updates_per_s;  /* cell_updates / wall_s */
    double p50_s, p99_s, mean_s;/* solve latency, arrival to result on the host */
    double hbm_in_use, hbm_peak;/* bytes of admitted solves */
    int tile_shape;             /* flux-kernel tile shape in use (-1 while the tuner runs) */
    int update_cpt;             /* cells per thread of the update kernel (-1 while the tuner runs) */
    double gpu_s;               /* device time of all rounds (CUDA events around each round) */
    double round_overhead;      /* 1 - gpu_s / busy_s: share of the time with active solves in
                                   which the GPU ran none of their steps */
    long graph_captures;        /* step graphs captured so far (one per tuner candidate; changes
                                   of the active set capture none) */
} cgks_serve_stats_t;

/* Start a server (spawns its scheduler, upload and download threads).  Errors:
 * CGKS_E_INVAL (non-positive budget, slots or steps per round, an unknown tile
 * shape or order, fill_cells <= 0 with CGKS_SERVE_LEAST_WORK_FIRST, a log file
 * that cannot be opened). */
cgks_status cgks_serve_start(const cgks_serve_cfg* cfg, cgks_server** out);

/* Queue a request; *req_id receives its id.  The initial planes are copied.
 * Errors: CGKS_E_BUDGET if the request alone exceeds the budget (it could
 * never be admitted), CGKS_E_INVAL, CGKS_E_BUSY while stopping.  Otherwise the
 * request waits in the queue until it can be admitted. */
cgks_status cgks_serve_submit(cgks_server* srv, const cgks_request* req, long* req_id);

/* *done = 1 when the request has finished.  If so and out_planes is not NULL,
 * the final state (12 planes) is copied there and the request is forgotten.
 * Returns the request's status (CGKS_E_NOTFOUND for an unknown id). */
cgks_status cgks_serve_poll(cgks_server* srv, long req_id, double* out_planes, int* done);

/* Wait at most timeout_s seconds for a request, then behave like poll.
 * Returns CGKS_E_TIMEOUT if it has not finished by then. */
cgks_status cgks_serve_wait(cgks_server* srv, long req_id, double timeout_s, double* out_planes);

/* Throughput and latency statistics so far (always CGKS_OK for a valid
 * server: a failure of the server's scheduler is reported to new submissions,
 * to the requests it could not finish and by cgks_serve_stop). */
cgks_status cgks_serve_stats(cgks_server* srv, cgks_serve_stats_t* out);

/* Stop accepting requests, finish the queued and active ones, join the
 * server's threads and free the server.  Returns CGKS_OK, or the CUDA error
 * status that stopped the scheduler (its queued requests then completed with
 * that status). */
cgks_status cgks_serve_stop(cgks_server* srv);

/* Detail of the last failing cgks_serve_* call on the calling thread. */
const char* cgks_serve_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CGKS_H */
