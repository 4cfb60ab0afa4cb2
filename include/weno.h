/*
 * weno.h -- C-ABI of libweno: the WENO-ZA6 finite-difference right-hand side
 * and third-order SSP Runge-Kutta stepping, in CUDA for GB300 (sm_103a).
 *
 * Method: Gu, Wang, Don, Jung, "A Family of Even-Order Central-Upwind WENO
 * Schemes with Averaged Downwind and Novel Global Smoothness Indicators",
 * arXiv 2603.26272.  The sixth-order scheme WENO-ZA6 is Section 3; its
 * ingredients are the general framework of Section 2.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * State layout: U is a contiguous array of doubles [nbatch][ncomp][ny][nx],
 *   x fastest, holding nbatch independent problems of the same shape.
 *   ncomp = 1 for the scalar equations (u), 3 for 1D Euler (rho, rho u, E),
 *   4 for 2D Euler (rho, rho u, rho v, E); ny = 1 in 1D.  Cells are uniform:
 *   dx = (x1 - x0) / nx, dy = (y1 - y0) / ny (Section 2: x_{i+1/2} = a + i dx).
 * Memory: every array argument named U, dUdt, alpha or ws is DEVICE memory
 *   owned by the caller (for instance a PyTorch tensor), except where an
 *   entry point says "host".  The library never allocates device memory;
 *   scratch space is the caller's workspace `ws` of at least
 *   weno_workspace_bytes(d) bytes, 256-byte aligned, passed with its size.
 *   A workspace may be reused by consecutive calls on one stream; calls that
 *   share a workspace must not run concurrently.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  All
 *   work is enqueued on it; entry points that return values to the host
 *   synchronise that stream and say so.
 * Errors: every entry point returns a weno_status and never aborts.  On an
 *   error, weno_last_error() returns a message for the calling host thread.
 *   Device-side failures (a nonphysical state: rho <= 0, p <= 0, a
 *   non-positive Roe sound speed or a non-finite value) are recorded in the
 *   workspace and reported at the next synchronising call.
 */
#ifndef WENO_H
#define WENO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WENO_OK = 0,
  WENO_ERR_ARG = 1,         /* invalid descriptor, pointer or size            */
  WENO_ERR_CUDA = 2,        /* a CUDA runtime call failed                     */
  WENO_ERR_NONPHYSICAL = 3, /* rho <= 0, p <= 0, c^2 <= 0 or non-finite met   */
  WENO_ERR_NOMEM = 4,       /* workspace smaller than weno_workspace_bytes    */
  WENO_ERR_TIMEOUT = 5,     /* a bounded device wait gave up                  */
  WENO_ERR_MAXSTEPS = 6     /* weno_solve stopped at max_steps before t_final */
} weno_status;

enum {
  WENO_SYS_ADVECTION = 0,       /* u_t + a u_x = 0                                    */
  WENO_SYS_EULER = 1,           /* Euler equations, gamma-law gas (Section 4.2, 4.3)  */
  WENO_SYS_BURGERS = 2,         /* u_t + (u^2/2)_x = 0 (Section 4.1, Table 5)         */
  WENO_SYS_BUCKLEY_LEVERETT = 3 /* u_t + (u^2/(u^2 + (1-u)^2/4))_x = 0 (Table 5)      */
};
enum { WENO_BC_TRANSMISSIVE = 0, WENO_BC_PERIODIC = 1 };
enum { WENO_PREC_FP64 = 0, WENO_PREC_FP32_RECON = 1 };
enum { WENO_ALPHA_FIELD = 0, WENO_ALPHA_SINGLE = 1 };

/* Problem descriptor.  Defaults of the paper: eps = 1e-40 (Section 4
 * preamble), mu0 = 1e-40 (eq. (22)), p = 1 (Section 4 preamble; L = q = 1
 * are fixed, Section 2.1 after Table 1), gamma = 1.4 (Section 4.2). */
typedef struct weno_desc {
  int32_t system;     /* WENO_SYS_*; the scalar equations are 1D                  */
  int32_t ndim;       /* 1 or 2 (advection: 1)                                    */
  int64_t nbatch;     /* number of independent problems, >= 1                     */
  int64_t nx, ny;     /* cells per axis, nx >= 1, ny >= 1 (ny = 1 when ndim = 1)  */
  double x0, x1;      /* domain [x0, x1]                                          */
  double y0, y1;      /* domain [y0, y1] (ignored in 1D)                          */
  int32_t bc_x, bc_y; /* WENO_BC_*: r ghost cells per side, zero-gradient or wrap */
  double gamma;       /* ratio of specific heats (Euler)                          */
  double cfl;         /* CFL number of the time step rule                         */
  double eps;         /* sensitivity epsilon of eq. (21); with ai = 1, >= 1e-250  */
  double mu0;         /* mu_0 of eq. (22); with ai = 1, 16 eps mu0^2 >= 1e-300    */
  double p;           /* power parameter p of eq. (21), > 0 (the paper: 1, 3/2, 2) */
  int32_t ai;         /* 1: affine-invariant descaler mu[f] of eq. (22); 0: mu = 1 */
  int32_t precision;  /* WENO_PREC_FP64, or WENO_PREC_FP32_RECON: the indicators, */
                      /* weights and candidates of eqs. (11)-(22) in FP32 on the  */
                      /* mu-normalised stencil differences (needs ai = 1, order   */
                      /* 6); projections, fluxes and RK accumulation stay FP64    */
  int32_t alpha_mode; /* WENO_ALPHA_FIELD: GLF speed per characteristic field;    */
                      /* WENO_ALPHA_SINGLE: one speed max|u|+c for all fields     */
  int32_t order;      /* 2r, the order of the central-upwind scheme: 0 or 6 =      */
                      /* WENO-ZA6 (Section 3); 4, 8, 10 = the schemes of the      */
                      /* Appendix (tables of c_k, d_k, B_k, c_tau for r = 2, 4, 5) */
                      /* with the same weights, eqs. (16)-(22).  WENO_PREC_FP32_  */
                      /* RECON and the serving engine take order 6 only.          */
  double adv_speed;   /* a of the advection equation                              */
} weno_desc;

/* Bytes of device workspace that weno_rhs / weno_step / weno_solve need for d:
 * two stage states, the reduction slots and the per-problem clocks.  Returns
 * 0 if d is invalid (see weno_last_error). */
size_t weno_workspace_bytes(const weno_desc *d);

/* Global Lax-Friedrichs speeds of eq. (6) for the state U:
 * alpha[b*8 + dir*4 + m] = max over all cells of problem b of |lambda_m|
 * (dir 0 = x, 1 = y; m = characteristic field in the order u-c, u, u(, u+c);
 * unused slots 0), and the CFL time step dt[b] (1D: cfl dx / max(|u|+c);
 * 2D: cfl / (max(|u|+c)/dx + max(|v|+c)/dy); scalar: cfl dx / alpha).
 * For a scalar flux alpha[b*8] = max |f'(u)| over the range [min u, max u]
 * of the data (for Buckley-Leverett f' peaks inside that range).
 * alpha and dt are DEVICE arrays of nbatch*8 and nbatch doubles.
 * Asynchronous. */
weno_status weno_wavespeeds(const weno_desc *d, const double *U, double *alpha, double *dt,
                            void *ws, size_t ws_bytes, void *stream);

/* Tile autotuning (2D, order 6).  weno_rhs, weno_step and weno_solve choose
 * among eleven tile shapes of the 2D stage kernel (all give bitwise the same
 * result).  The first such call on a new problem shape (nx, ny, nbatch,
 * precision, ai, p == 1) in a process times them on the caller's data: two
 * launches of each shape on `stream`, writing only the workspace, with CUDA
 * events, and it synchronises the stream before it returns.  Later calls on
 * that shape are asynchronous as stated.  The environment variable
 * WENO_TILE2D = 0..10 forces one shape and skips the timing (use it when the
 * first call must not synchronise, e.g. inside a stream capture). */

/* Right-hand side of one Runge-Kutta stage, L(U) (eq. (5) dimension by
 * dimension: dU/dt = -(F_{i+1/2} - F_{i-1/2})/dx - (G_{j+1/2} - G_{j-1/2})/dy),
 * with the interface fluxes of WENO-ZA6 (Section 3) after global
 * Lax-Friedrichs splitting (eq. (6)), characteristic-wise on Roe-averaged
 * eigenvectors for Euler (Section 4.2), and the GLF speeds taken from U.
 * dUdt has U's layout and must not overlap U.  Asynchronous (but see the
 * tile autotuning note above for the first 2D call on a new shape). */
weno_status weno_rhs(const weno_desc *d, const double *U, double *dUdt, void *ws,
                     size_t ws_bytes, void *stream);

/* One third-order SSP (TVD) Runge-Kutta step of every problem, in place
 * (Section 4 preamble):
 *   U1 = U + dt L(U);  U2 = 3/4 U + 1/4 (U1 + dt L(U1));
 *   U <- 1/3 U + 2/3 (U2 + dt L(U2)).
 * dt > 0: that step for every problem; dt <= 0: each problem's own CFL step
 * (as in weno_wavespeeds).  dt_used: NULL (asynchronous call, apart from the
 * first 2D call on a new shape, see the tile autotuning note) or a HOST
 * array of nbatch doubles that receives the steps taken; then the call
 * synchronises the stream and also reports device-side errors. */
weno_status weno_step(const weno_desc *d, double *U, double dt, double *dt_used, void *ws,
                      size_t ws_bytes, void *stream);

/* Advance every problem from t0 to t_final with CFL steps, clipping each
 * problem's last step to land on t_final, taking at most max_steps steps.
 * t_out / steps_out: HOST arrays of nbatch (may be NULL) receiving each
 * problem's reached time and step count.  Synchronises the stream.
 * Returns WENO_ERR_MAXSTEPS if a problem had not reached t_final; on
 * WENO_ERR_NONPHYSICAL, U holds the state in which the bad value appeared. */
weno_status weno_solve(const weno_desc *d, double *U, double t0, double t_final,
                       int64_t max_steps, double *t_out, int64_t *steps_out, void *ws,
                       size_t ws_bytes, void *stream);

/* weno_step on a HOST state: copies U_host (nbatch*ncomp*ny*nx doubles) to
 * the device, takes one step as weno_step does, and copies the result back
 * into U_host.  The workspace must hold weno_workspace_bytes_host(d) bytes.
 * dt_used: NULL or a HOST array of nbatch doubles.  Synchronises the stream. */
weno_status weno_step_host(const weno_desc *d, double *U_host, double dt, double *dt_used,
                           void *ws, size_t ws_bytes, void *stream);

/* weno_solve on a HOST state: copies U_host to the device, solves, copies the
 * result back into U_host.  The workspace must hold
 * weno_workspace_bytes_host(d) bytes (the device copy of U lives there).
 * U_host may be pageable, but pinned memory gives full copy bandwidth.
 * Synchronises the stream. */
size_t weno_workspace_bytes_host(const weno_desc *d);
weno_status weno_solve_host(const weno_desc *d, double *U_host, double t0, double t_final,
                            int64_t max_steps, double *t_out, int64_t *steps_out, void *ws,
                            size_t ws_bytes, void *stream);

/* Synchronise the stream and report the device-side status recorded in the
 * workspace by the previous asynchronous calls (WENO_OK or
 * WENO_ERR_NONPHYSICAL with the problem, cell and stage in weno_last_error). */
weno_status weno_sync_status(const weno_desc *d, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Domain decomposition in y: a 2D Euler grid split into strips of rows, one
 * per process (GPU).  d is the GLOBAL descriptor (its ny, x0..y1, bc_x, bc_y,
 * scheme); a strip holds nrows consecutive rows, r <= nrows <= ny, r = order/2
 * (3 for WENO-ZA6), as U = [nbatch][4][nrows][nx] with its own workspace of
 * weno_workspace_bytes(d with ny = nrows) bytes.  One SSP-RK3 step of a strip:
 *   weno_dd_begin(U)                 local speed maxima of U (into the slot
 *                                    stage 1 reads) and U's first / last r rows
 *                                    into send_lo / send_hi;
 *   for stage = 1, 2, 3:
 *     weno_dd_speeds(stage)          device pointer to nbatch x 8 uint64: the
 *                                    caller replaces them in place by their
 *                                    maximum over all strips (they are the bit
 *                                    patterns of non-negative doubles, so an
 *                                    integer max is the numeric max; eq. (6)
 *                                    takes its GLF speeds over the whole grid);
 *     exchange                       the caller sends send_lo to the strip
 *                                    below (its halo_hi) and send_hi to the
 *                                    strip above (its halo_lo);
 *     weno_dd_stage(stage, halos)    the stage, reading the r rows beyond each
 *                                    side from halo_lo / halo_hi (rows in
 *                                    increasing order, [nbatch][4][r][nx]), or
 *                                    from the boundary condition bc_y where a
 *                                    halo pointer is NULL (a side of the global
 *                                    domain); it writes its output's first /
 *                                    last r rows into send_lo / send_hi (NULL:
 *                                    skipped) for the next exchange.
 * dt > 0 fixes the step; dt <= 0 takes the CFL step of eq. (6)'s global
 * speeds, the same on every strip.  Stage 3 leaves the new state in U.  The
 * arithmetic of every cell is that of weno_step on the whole grid, so the
 * strips together reproduce it bit for bit.  All calls are asynchronous on
 * `stream` (weno_dd_speeds enqueues nothing); weno_sync_status with the
 * strip's descriptor reports device-side errors.  The paper solves on one
 * CPU; this is how its 2D right-hand side shares out over GPUs. */
weno_status weno_dd_begin(const weno_desc *d, int64_t nrows, const double *U, double *send_lo,
                          double *send_hi, void *ws, size_t ws_bytes, void *stream);
weno_status weno_dd_speeds(const weno_desc *d, int64_t nrows, int stage, void *ws,
                           size_t ws_bytes, uint64_t **speeds);
weno_status weno_dd_stage(const weno_desc *d, int64_t nrows, int stage, double *U, double dt,
                          const double *halo_lo, const double *halo_hi, double *send_lo,
                          double *send_hi, void *ws, size_t ws_bytes, void *stream);

/* L(U) as weno_rhs computes it, for callers that cannot allocate device
 * memory or pass a workspace (a plug-in whose host owns all allocations, a
 * loop that must never enter the allocator, a fixed memory budget).  The
 * paper has no counterpart: this is a deployment variant, not a step of the
 * method.  Its scratch (a status word and one slot of speed maxima per
 * problem) is a fixed 64 KiB device array inside the library, present on every
 * GPU that loads it until the process exits; the call allocates nothing.
 * Limits: nbatch <= 1020 (larger batches return WENO_ERR_ARG with a message;
 * use weno_rhs).  The first call on each device looks up the array's address
 * (make it before any stream capture on that device).  All calls share the
 * array and clear what they need; calls that overlap on the GPU race and must
 * be serialised by the caller.  U, dUdt: DEVICE arrays as for weno_rhs.  Every
 * call ends by synchronising `stream` to read the shared status word back, and
 * returns WENO_ERR_NONPHYSICAL for a nonphysical input. */
weno_status weno_rhs_noalloc(const weno_desc *d, const double *U, double *dUdt, void *stream);

/* ---------------------------------------------------------------------------
 * Serving engine: continuous batching of independent solves on one GPU.
 * Each admitted problem ("slot": one Euler problem, nbatch = 1, ai = 1,
 * p = 1, FP64 or FP32_RECON, 1D or 2D of any size) advances with its own CFL
 * step to its own t_final; all admitted slots advance together, every engine
 * step being one SSP-RK3 step of each unfinished slot (three launches of a
 * persistent kernel over a device work list of all slots' tiles, replayed as
 * one CUDA graph).  A slot marked fast (weno_engine_set_fast) advances
 * WENO_ENGINE_FAST_STEPS SSP-RK3 steps per engine step: the graph then holds
 * that many sub-steps, the first over every slot, the others over the fast
 * slots only, so small or urgent solves need not wait for the pace of the
 * largest.  Problems can be admitted and retired between runs.  The paper
 * has no serving layer: this is how many of its solves share a GPU.
 *
 * Memory: `arena` is caller-owned DEVICE memory (256-byte aligned).  Its first
 * weno_engine_control_bytes(max_slots, max_tiles) bytes hold the engine's
 * tables; the rest is a heap for the slots' states (weno_engine_slot_bytes
 * each).  Admission fails with WENO_ERR_NOMEM when no slot, work-list entry
 * or heap block is free; the engine never calls the allocator.
 * The engine works on a CUDA stream of its own, created with the device's
 * highest stream priority (a large solve the caller runs beside it on a
 * stream of lower priority yields the SMs to the engine's blocks as its own
 * blocks finish); run() is asynchronous, admit/poll/retire synchronise it.
 * One host thread per engine.
 * --------------------------------------------------------------------------- */
typedef struct weno_engine weno_engine;

size_t weno_engine_control_bytes(int max_slots, int64_t max_tiles);
/* Heap bytes one problem described by d occupies (3 states), 0 if invalid. */
size_t weno_engine_slot_bytes(const weno_desc *d);
/* stream: reserved, pass NULL. */
weno_status weno_engine_create(void *arena, size_t arena_bytes, int max_slots, int64_t max_tiles,
                               void *stream, weno_engine **out);
/* Copy the HOST state U_host (layout of d, nbatch = 1) in, compute its speeds
 * and give it a slot (slot_out).  t_final > 0: the problem's end time. */
weno_status weno_engine_admit(weno_engine *e, const weno_desc *d, const double *U_host,
                              double t_final, int *slot_out);
/* Enqueue nsteps engine steps (asynchronous). */
weno_status weno_engine_run(weno_engine *e, int nsteps);
/* CUDA stream priority of the engine's runs (lower numbers are higher
 * priorities, clamped to the device's range; the engine starts at the
 * highest).  run() then launches on a stream of that priority, ordered after
 * the engine's own stream and before its next poll/admit/retire, so a caller
 * running other solves beside the engine can let one of them go first. */
weno_status weno_engine_set_priority(weno_engine *e, int priority);
/* SSP-RK3 steps per engine step of a fast slot. */
#define WENO_ENGINE_FAST_STEPS 4
/* Mark an admitted slot fast (fast = 1: WENO_ENGINE_FAST_STEPS steps per
 * engine step) or normal (0: one step).  Takes effect at the next run(); a
 * slot's results are the same bit for bit either way. */
weno_status weno_engine_set_fast(weno_engine *e, int slot, int fast);
/* Wait for the enqueued steps; done[0..min(*n_done, max_done)) receives the
 * slots that reached t_final or met a nonphysical state; n_active (may be
 * NULL) the number of admitted slots. */
weno_status weno_engine_poll(weno_engine *e, int *done, int max_done, int *n_done,
                             int *n_active);
/* Copy a slot's state to U_host (may be NULL), report its time and step
 * count, and free the slot.  Returns WENO_ERR_NONPHYSICAL for a slot that
 * met a nonphysical state (the other slots are unaffected). */
weno_status weno_engine_retire(weno_engine *e, int slot, double *U_host, double *t_out,
                               int64_t *steps_out);
/* Free heap bytes, the largest free block and the work-list entries in use. */
weno_status weno_engine_info(const weno_engine *e, size_t *heap_free_bytes,
                             size_t *heap_largest, int64_t *tiles_in_use);
weno_status weno_engine_destroy(weno_engine *e);

/* Measured FMA throughput of the current GPU, the peak of the stage kernels'
 * roofline (they are bound by FP64 instruction issue; no step of the method
 * is a dense contraction, and their HBM traffic is far below the memory
 * roof).  The paper has no counterpart: it reports CPU times only.
 * kind 0: FP64 FMA chains on full-mantissa values (the operands of a real
 *         solve; on GB300 the FP64 rate depends on the operands' bits),
 *      1: FP64 FMA chains that settle on 1.0 (a mantissa of zeros),
 *      2: FP32 FMA chains.
 * One launch of 8 blocks x 256 threads per SM, each thread running 8
 * independent chains of `iters` FMAs (1 .. 2^24; 4096 takes about 20 ms in
 * FP64 on GB300), timed with CUDA events on `stream` after a short warm-up.
 * *flops_per_s (HOST) receives 2 x FMAs / second.  Allocates no device
 * memory; synchronises the stream. */
weno_status weno_fma_rate(int kind, int iters, double *flops_per_s, void *stream);

/* Message describing the last error on the calling host thread ("" if none). */
const char *weno_last_error(void);

/* Library version string. */
const char *weno_version(void);

#ifdef __cplusplus
}
#endif
#endif /* WENO_H */
