/*
 * cgks.h -- C ABI of libcgks: the compact 8th-order gas-kinetic scheme of
 * Zhao, Ji, Shyy, Xu, "An acoustic and shock wave capturing compact high-order
 * gas-kinetic scheme with spectral-like resolution" (arXiv 2001.01570), on one
 * GPU, in FP64.
 *
 * What one time step computes (every step runs entirely in CUDA kernels):
 *   - dt from the CFL condition, dt = CFL * min over cells of
 *     min(dx/(|U|+c), dy/(|V|+c)) (Sec. 4);
 *   - at every cell interface: the linear compact 8th-order reconstruction of
 *     the equilibrium state (Sec. 3.2, Eq. recons-8th-val) and the nonlinear
 *     WENO-Z compact reconstruction of the non-equilibrium left/right states
 *     (Sec. 3.3, Eq. sub-stencil, WENO-Z-w, smooth-indicator), from cell
 *     averages and cell-averaged gradients on the stencil {I_i-1..I_i+2};
 *   - the gas-kinetic evolution at two Gauss points per face (Sec. 2.1,
 *     Eq. 3rd-simplify-flux) with collision time
 *     tau = eps_tau*dt + c_tau*|p_l-p_r|/(p_l+p_r)*dt (Sec. 4), giving the
 *     time-accurate flux, its time derivative and the interface state;
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
    CGKS_BC_INFLOW = 2,    /* fixed state cgks_problem.inflow, zero gradients */
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
    double inflow[4];        /* primitive rho, u, v, p used on CGKS_BC_INFLOW sides */
    double eps_tau;          /* tau = eps_tau*dt + c_tau*|dp|/(sum p)*dt; paper: 0.01 */
    double c_tau;            /* paper: 1 */
    double weno_eps;         /* epsilon of the WENO-Z weights; paper tests 1e-6, 1e-4 */
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

/* Copy the current state out (synchronises the stream).  t and steps may be
 * NULL.  Returns the solve's sticky status (CGKS_OK or CGKS_E_NONPHYSICAL). */
cgks_status cgks_get_state(cgks_solver* s, double* planes, int on_device, double* t, long* steps);

/* Advance `nsteps` S2O4 steps.  t_end > 0: the last step is shortened so that
 * t reaches t_end exactly and no step runs past it.  Synchronises the stream
 * before returning; *t_out (may be NULL) receives the new time.
 * Errors: CGKS_E_NONPHYSICAL (state kept at the last valid step), CGKS_E_CUDA. */
cgks_status cgks_step(cgks_solver* s, int nsteps, double t_end, double* t_out);

/* Advance `n` independent solvers (any sizes and boundary types) by `nsteps`
 * steps each, each with its own dt, through one persistent launch per stage
 * over a flattened tile queue, replayed as a CUDA graph.  All solvers must live
 * on the current device; the work is ordered on the first solver's stream.
 * Synchronises before returning.  The status of each solver stays readable
 * through cgks_get_state. */
cgks_status cgks_batch_step(cgks_solver* const* solvers, int n, int nsteps);

/* Same as cgks_step(s, nsteps, 0, NULL), but with CUDA events recorded on the
 * solver's stream around every kernel of every step; stage_ms[0..3] receive
 * the average duration in milliseconds of the step-begin, stage-1, stage-2 and
 * step-end kernels.  For measurement only (the events serialise nothing but
 * add host work per launch). */
cgks_status cgks_step_profiled(cgks_solver* s, int nsteps, double stage_ms[4]);

/* Kernel launch count of the most recent cgks_step / cgks_batch_step call on
 * the calling thread (for throughput accounting). */
long cgks_last_launch_count(void);

const char* cgks_status_string(cgks_status st);
const char* cgks_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CGKS_H */
