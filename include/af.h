/*
 * af.h -- C ABI of the GB300 (sm_103a) implementation of one time step of the
 * fully discrete Active Flux method with transported acoustic increments
 * (RB-TAI), with the additive Roe-Barsukow (RB) point update as a switch, for
 * the 2D compressible Euler equations (gamma-law gas) on a periodic Cartesian
 * grid of square cells (arXiv 2605.12915).
 *
 * Conventions for every entry point:
 *  - Status codes only; nothing throws, aborts or traps across this ABI.
 *  - Errors found on the device (acoustic CFL above 1/2, foot outside the
 *    supported reach, non-positive density or pressure, non-finite values) are
 *    latched in a device word and reported by af_step (as soon as the step that
 *    raised them has completed), af_sync, af_get_state and af_reduce_invariants.
 *  - The library never frees, and never keeps pointers to, caller memory.
 *  - Every array is a plane of nx*ny values in row-major order, index j*nx+i.
 *
 * Degrees of freedom (Sec. 2, Fig. 1) of cell C_ij = [x_i,x_{i+1}] x [y_j,y_{j+1}]:
 *   avg[4] conservative cell average (rho, rho u, rho v, E) of C_ij,
 *   vtx[4] primitive (rho, u, v, p) at the vertex        (x_i,       y_j),
 *   ev[4]  primitive (rho, u, v, p) at the x-edge midpoint (x_i,     y_{j+1/2}),
 *   eh[4]  primitive (rho, u, v, p) at the y-edge midpoint (x_{i+1/2}, y_j),
 * with E = p/(gamma-1) + rho (u^2+v^2)/2.
 */
#ifndef AF_H
#define AF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct af_handle af_handle; /* opaque; owns the device state and scratch */

typedef enum {
  AF_OK = 0,
  AF_ERR_ARG = 1,         /* invalid argument (null pointer, size, dt, enum) */
  AF_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  AF_ERR_ALLOC = 3,       /* device or pinned host allocation failed */
  AF_ERR_CFL = 4,         /* c dt / h > 1/2 at a node, or a convective foot beyond one cell */
  AF_ERR_NONPHYSICAL = 5, /* rho <= 0 or p <= 0 where a sound speed is needed */
  AF_ERR_NONFINITE = 6,   /* NaN or Inf produced */
  AF_ERR_STATE = 7,       /* handle unusable (a previous CUDA error) */
  AF_ERR_TIMEOUT = 8,     /* a kernel's bounded wait for its own asynchronous copies ran
                             out; the kernel stopped early and the step's result is invalid */
  AF_ERR_BOUNDS = 9       /* debug builds only (compiled with AF_BOUNDS_CHECK): a checked
                             shared-memory index of the fused step left its region; the
                             access used a valid index instead and the result is invalid */
} af_status;

typedef enum {
  AF_FP64 = 0,     /* all arithmetic and storage in double */
  AF_FP32 = 1,     /* all stencil arithmetic and storage in float */
  AF_FP32_COMP = 2 /* as AF_FP32, cell averages kept as float hi+lo pairs updated
                      by error-free sums of the edge-flux increments */
} af_precision;

typedef enum {
  AF_TAI = 0, /* transported acoustic increments, Eq. (transported-update) */
  AF_RB = 1,  /* additive point update, Eq. (barsukow-additive) */
  AF_FC = 2   /* foot-centred exact acoustic update (Appendix C): the acoustic
                 disk of radius c_* tau centred at the convective foot, state
                 frozen there, density from the linear closure of Sec. 3.1 at
                 the foot; FP64 only (an analytical reference: the paper puts
                 its cost at about 1000x the node-centred update); needs the
                 compact footprint |F - P| + c_* tau < h/2 per axis
                 (Eq. fc-half-footprint), else the step reports AF_ERR_CFL */
} af_variant;

typedef enum { AF_HOST = 0, AF_DEVICE = 1 } af_memory;

typedef struct {
  int32_t nx, ny; /* cells in x and y, each >= 2 */
  double h;       /* cell side, > 0 */
} af_grid;

typedef struct {
  double *avg[4];
  double *vtx[4];
  double *ev[4];
  double *eh[4];
} af_state_f64;

/* Indices of af_reduce_invariants' output (all FP64):
 *  mass, momentum, energy = h^2 sum of the cell averages (conserved by the
 *  flux-difference update, Eq. af-average-update); entropy functional
 *  -int rho log(p / rho^gamma) dA (Sec. 6) by tensor Simpson on each cell's
 *  nine nodes, and from the cell averages; kinetic energy of the averages;
 *  max of |u| + c and min of rho, p over vertex, edge and centre nodes;
 *  int (v_x - u_y) dA by Simpson along cell edges; the latched error bits. */
enum {
  AF_INV_MASS = 0,
  AF_INV_MOMX = 1,
  AF_INV_MOMY = 2,
  AF_INV_ENERGY = 3,
  AF_INV_ENTROPY = 4,
  AF_INV_ENTROPY_AVG = 5,
  AF_INV_KINETIC = 6,
  AF_INV_MAX_SPEED = 7,
  AF_INV_MIN_RHO = 8,
  AF_INV_MIN_P = 9,
  AF_INV_VORTICITY = 10,
  AF_INV_FLAGS = 11,
  AF_NINV = 12
};

/* Create a solver for grid g and copy the initial state in (Sec. 6: averages by
 * quadrature, point values sampled -- prepared by the caller).  `state` arrays
 * are read on `where` (AF_HOST: pageable or pinned host memory; AF_DEVICE:
 * device memory of the current device); the caller keeps ownership.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream) on which every
 * later call of this handle runs.  On error *out is NULL.
 *
 * The handle allocates two states and the step's scratch planes here (about
 * 88 planes of nx * ny values of the working precision); af_adjoint_step
 * allocates its own work area (92 planes) on its first call, host transfers
 * of pageable planes a staging buffer of 16 FP64 planes on their first use,
 * af_exchange_state another 16 FP64 planes and a second stream with host
 * planes; af_destroy frees all of them.  Kernel choices, read from the environment when the handle is created
 * (the results are the same up to rounding; they exist for comparison and
 * testing): AF_PATH=ref runs the FP32 modes on the kernel-per-stage path
 * instead of the fused kernel; AF_PIPE=0 replaces the persistent pipelined
 * fused kernel by one CTA per tile, AF_PIPE=n caps its grid at n CTAs;
 * AF_TMA=0 stages every tile by cp.async instead of tensor copies;
 * AF_PREFETCH=0 disables the L2 prefetch of the one-CTA-per-tile kernel;
 * AF_ZERO_COPY=0 copies pinned host planes through a staging buffer instead
 * of converting them in place; AF_TEST_LATE_WAIT=1 (testing the timeout
 * path only) makes the handle's first pipelined FP32 step give up its first
 * wait for a tensor-copied tile at once, so that the step reports
 * AF_ERR_TIMEOUT (the CTA still drains its copies before it stops).
 * AF_ADJ_FUSED=0, read by each af_adjoint_step call, selects its
 * stage-by-stage sweep. */
af_status af_init(af_handle **out, const af_grid *g, double gamma, const af_state_f64 *state,
                  af_memory where, af_precision prec, af_variant var, void *cuda_stream);

/* Advance n_steps >= 0 steps of size dt > 0 (Sec. 6.1, Algorithm): point values
 * at t^n + dt/2 and t^n + dt from the time-n reconstruction, then the
 * conservative space-time Simpson average update.  Asynchronous on the
 * handle's stream; returns the first latched device error of steps that have
 * already completed (AF_OK otherwise). */
af_status af_step(af_handle *h, double dt, int32_t n_steps);

/* Wait for the handle's stream and return the latched device error, if any. */
af_status af_sync(af_handle *h);

/* Copy the current state out as FP64 (AF_FP32_COMP: averages as hi + lo).
 * Synchronises the stream.  AF_HOST planes in pinned (page-locked) memory are
 * written directly by the conversion kernel; pageable planes go through a
 * device staging buffer and a copy. */
af_status af_get_state(af_handle *h, const af_state_f64 *out, af_memory where);

/* Replace the current state (converted to the handle's precision) and clear the
 * latched device error.  AF_HOST planes in pinned memory are read directly by
 * the conversion kernel, pageable ones are copied first. */
af_status af_set_state(af_handle *h, const af_state_f64 *in, af_memory where);

/* Hands the current state out into `out` and takes `in` in as the new current
 * state (as af_get_state then af_set_state), for callers that stream states
 * through the handle: set, step, then exchange the result for the next input.
 * `out` and `in` are FP64 planes on `where`, owned by the caller, and may not
 * share a byte (AF_ERR_ARG).  The call returns once the new state is in place
 * (the latched device error cleared).
 * AF_DEVICE: `out` is complete on return too.
 * AF_HOST: both transfers run on copy engines on two streams of the handle, so
 * that they overlap on the host-device link with each other and with a step
 * still running (one copy per direction when the sixteen planes are
 * consecutive in memory, in plane order, else one per plane): `in` is copied into a device staging buffer at once, the
 * outgoing state is converted into a second one (16 FP64 planes each,
 * allocated on first use, held until af_destroy) and copied into `out`.  That
 * last copy may still be in flight on return; later calls of this handle that
 * touch it are ordered after it (af_step does not wait for it, so the next
 * step overlaps it), but the caller itself may read or write `out` only once
 * af_sync, or any other call of this handle but af_step and
 * af_exchange_state, has returned.  `in` is read before the call returns. */
af_status af_exchange_state(af_handle *h, const af_state_f64 *out, const af_state_f64 *in,
                            af_memory where);

/* Asynchronous form of af_exchange_state for host planes (pinned or pageable),
 * for callers that stream states through the solver: `out` <- the current
 * state, then the current state <- `in`, all enqueued without waiting, so that
 * consecutive calls keep both directions of the host-device link busy.  The
 * incoming planes are copied into one of two device staging buffers and the
 * outgoing state is converted into one of two others (16 FP64 planes each,
 * allocated on the first call, held until af_destroy); alternate calls use
 * alternate buffers, each reused once its earlier copy and conversion are done.
 * The handle's later steps run on the new state.  The call returns before the
 * transfers end: the caller may modify `in` or read `out` only after af_sync
 * (or any other call of this handle except af_step and the exchanges) has
 * returned.  An incoming plane that shares memory with the target of an
 * earlier exchange's outgoing copy is read after that copy.  Unlike
 * af_exchange_state it leaves the latched device error as it is (af_sync
 * reports it; af_set_state clears it).  `out` and `in` may not share a byte
 * (AF_ERR_ARG). */
af_status af_exchange_state_async(af_handle *h, const af_state_f64 *out, const af_state_f64 *in);

/* FP64 global diagnostics of the current state, out[AF_NINV] in host memory.
 * Synchronises the stream. */
af_status af_reduce_invariants(af_handle *h, double *out);

/* Discrete adjoint of one step (Sec. 6.1, differentiated by hand, stage by
 * stage): lam_out = (d state^{n+1} / d state^n)^T lam_in, linearised about the
 * handle's current state (state^n), which is left unchanged.  lam_in holds the
 * adjoint of the state after one step of size dt, lam_out receives the adjoint
 * of the current state; both are FP64 arrays in the state layout above, on
 * `where`, owned by the caller (they may not overlap).  Adjoints are with
 * respect to the stored variables (cell averages and primitive point values).
 * The step's forward intermediates are recomputed in the handle's precision:
 * in the FP32 modes on grids the pipelined fused kernel accepts, one launch
 * recomputes each tile's step and reverses its fluxes and point updates in
 * shared memory.  Synchronises the stream; returns the latched device error,
 * if any. AF_FC handles are refused with AF_ERR_ARG (no adjoint of the
 * foot-centred update is provided). */
af_status af_adjoint_step(af_handle *h, double dt, const af_state_f64 *lam_in,
                          const af_state_f64 *lam_out, af_memory where);

/* Release the handle's device memory and streams' resources.  NULL is a no-op. */
void af_destroy(af_handle *h);

/* Static text for a status code. */
const char *af_status_string(af_status s);

/* Largest grid, in cells (nx * ny), that af_step_noalloc accepts. */
#define AF_NOALLOC_MAX_CELLS (128 * 128)

/* One FP64 step that allocates nothing.  The paper has no counterpart: this
 * serves callers that may not allocate device memory at all -- code running
 * under a fixed, pre-reserved device-memory budget, or inside a host runtime
 * that owns every allocation on the device.  The caller passes the state at
 * t^n (`in`) and receives the state at t^n + dt (`out`), both FP64 device
 * arrays in the layout above, on the current device, not overlapping.  The
 * intermediate values live in one work area compiled into the library (a
 * static device array of about 6.3 MB that every GPU loading the library holds
 * until the process exits); no cudaMalloc, cudaFree or other allocating call
 * is made.  The first call on a device looks up the work area's address on
 * that device.  Every call shares the one work area: calls that overlap on the GPU (other streams,
 * other threads) race and must be serialised by the caller.  Every call clears
 * the work area's error word, enqueues the step on `cuda_stream`, then copies
 * the error word to the host and synchronises `cuda_stream` before it returns
 * the step's error status.  nx * ny > AF_NOALLOC_MAX_CELLS, `in` and `out`
 * sharing any byte, or any other invalid argument returns AF_ERR_ARG without
 * touching the GPU. */
af_status af_step_noalloc(const af_grid *g, double gamma, double dt, af_variant var,
                          const af_state_f64 *in, const af_state_f64 *out, void *cuda_stream);

/* ---- Batched ensembles ----------------------------------------------------
 * Many independent grids (each with its own size, cell side, time step and
 * state) advanced together: every step is one launch of the fused FP32 kernel
 * over a table of the tiles of all grids, and the launches of an af_batch_step
 * call are captured once in a CUDA graph (re-captured when n_steps changes).
 * Geometries (AF_BATCH_GEOMS): 0, 1, 2 launch one CTA per tile of 32x32,
 * 24x16 or 16x16 cells; 3 launches persistent CTAs (one per SM) that step
 * through the 32x32 tiles of all grids, staging each next tile (tensor copies
 * inside a grid, cp.async on its periodic boundary) while the current one
 * finishes -- offered when every grid has nx a multiple of 4, nx >= 40 and
 * ny >= 38.  The first af_batch_step times the geometries on the actual
 * ensemble (states are snapshotted and restored around the trials) and keeps
 * the fastest; AF_BATCH_GEOM=g in the environment of af_batch_init fixes
 * geometry g instead (for comparison and testing).  Per-grid results are
 * bitwise those of af_step on a lone handle. */
#define AF_BATCH_GEOMS 4
typedef struct af_batch af_batch;

/* n grids; grids[k], states[k] as in af_init; prec must be AF_FP32 or
 * AF_FP32_COMP.  cuda_stream NULL: the batch creates (and later destroys) a
 * private non-blocking stream, since the legacy stream cannot be captured into
 * a graph.  On error *out is NULL. */
af_status af_batch_init(af_batch **out, int32_t n, const af_grid *grids, double gamma,
                        const af_state_f64 *states, af_memory where, af_precision prec,
                        af_variant var, void *cuda_stream);

/* n_steps steps of every grid k with time step dts[k] (host array of n).
 * Asynchronous; returns a latched device error of an earlier call, if any. */
af_status af_batch_step(af_batch *b, const double *dts, int32_t n_steps);

/* Wait for the stream; the first latched device error of any grid. */
af_status af_batch_sync(af_batch *b);

/* State of grid k (as af_get_state). */
af_status af_batch_get_state(af_batch *b, int32_t k, const af_state_f64 *out, af_memory where);

/* The tile geometry in use (index, -1 before the first step) and, if tune_ms is
 * not NULL, the per-step time of each candidate as timed by the autotuner
 * (AF_BATCH_GEOMS floats; -1 for a geometry not timed). */
af_status af_batch_info(af_batch *b, int32_t *geometry, float *tune_ms);

void af_batch_destroy(af_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* AF_H */
