/*
 * enoao.h -- C interface of the GB300 ENO-AO library.
 *
 * The library advances hyperbolic conservation laws u_t + f(u)_x = 0 (and
 * their dimension-by-dimension extension to 2D and 3D) with the ENO schemes
 * of adaptive order of H. Shen, "A class of ENO schemes with adaptive order
 * for solving hyperbolic conservation laws" (arXiv 2108.12742):
 *   - conservative finite-difference form L(u)_j = -(F_{j+1/2}-F_{j-1/2})/dx
 *     (Sec. 2, Eq. 1DWENOFD), summed over the axes (Sec. 2);
 *   - global Lax-Friedrichs splitting f^{+-} = (f +- alpha u)/2 (Sec. 2,
 *     Eq. LF_Flux_Split), alpha the maximum of |f'(u)| over the mesh;
 *   - for the Euler equations, projection onto characteristic fields with the
 *     Roe average at each face (Sec. 4);
 *   - ENO-AO interface values: candidate stencils from first order up to the
 *     designed order 5 or 7, chosen by the indicator IS = MIN(delta_L,
 *     delta_R) of Eq. (New_Smoothness_Indicator) and the selection principle
 *     with threshold delta (Sec. 3.2, Tables 1, 4, 5, Appendix A);
 *   - third-order TVD Runge-Kutta time stepping (Sec. 2).
 * Every step of that path runs in hand-written CUDA kernels for sm_103a.
 *
 * Conventions for every entry point:
 *   - A state array U holds the conserved variables as a structure of arrays,
 *     U[v][k][j][i] (i along x fastest, j along y, k along z), float64.  For
 *     the Euler equations v = (rho, rho*u, [rho*v], [rho*w], rho*e), nv =
 *     ndim + 2; for scalar advection nv = 1.
 *   - Pointers flagged "on_device" point to CUDA device memory of the device
 *     that was current at enoao_create; otherwise they point to host memory.
 *     The library copies from and to the caller's buffers and never keeps a
 *     caller pointer beyond the call.
 *   - Work is ordered on the CUDA stream given at creation (0 = the legacy
 *     default stream): a call's device work starts after the stream's earlier
 *     work and the stream's later work sees its results.  Calls that return
 *     data to the host, and enoao_advance*, synchronise before returning.
 *   - No exception or abort crosses this interface: every failure returns a
 *     status code and leaves a message readable with enoao_last_error.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef ENOAO_H
#define ENOAO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct enoao_ctx enoao_ctx;

typedef enum {
  ENOAO_OK = 0,
  ENOAO_EINVAL = 1,    /* invalid argument or configuration */
  ENOAO_ENOMEM = 2,    /* device or host allocation failed */
  ENOAO_ECUDA = 3,     /* a CUDA call failed (message has the CUDA error) */
  ENOAO_ENONPHYS = 4,  /* non-physical state met: rho <= 0, p <= 0 or NaN */
  ENOAO_ETIMEOUT = 5   /* a bounded device wait gave up */
} enoao_status;

enum { ENOAO_SCALAR_ADVECTION = 0, ENOAO_EULER = 1 };
enum { ENOAO_PERIODIC = 0, ENOAO_TRANSMISSIVE = 1 };
enum { ENOAO_FP64 = 0, ENOAO_FP32_BULK = 1 };
/* When alpha of the Lax-Friedrichs splitting (Sec. 2: the maximum of |f'(u)|
 * over the mesh) is taken for the Euler equations: once per step from U^n
 * for all three Runge-Kutta stages (the default), or per stage from that
 * stage's input state.  PER_FIELD: once per step from U^n, but each
 * characteristic field k splits with its own alpha_k = max |lambda_k| (per axis
 * max |u_d - c|, max |u_d| for the entropy and shear fields, max |u_d + c|),
 * the component-wise reading; single-problem contexts only (batched contexts
 * and enoao_step_noalloc return ENOAO_EINVAL), and FP32 bulk then re-decides
 * its near-ties inside the sweep whatever enoao_set_redecide says.  dt always
 * follows the CFL rule with alpha = max |u_d| + c of U^n. */
enum { ENOAO_ALPHA_PER_STEP = 0, ENOAO_ALPHA_PER_STAGE = 1, ENOAO_ALPHA_PER_FIELD = 2 };

typedef struct {
  int ndim;        /* 1, 2 or 3 */
  int system;      /* ENOAO_SCALAR_ADVECTION (f = adv_speed * u) or ENOAO_EULER */
  int order;       /* designed order: 5 (ENO-AO5) or 7 (ENO-AO7) */
  int precision;   /* ENOAO_FP64, or ENOAO_FP32_BULK: reconstruction, indicators
                      and projections in FP32, state and Runge-Kutta
                      accumulation in FP64, near-tie choices re-decided in FP64 */
  int64_t n[3];    /* cells per axis; unused axes must be 1 */
  double lo[3];    /* domain [lo, hi] per axis; dx = (hi - lo) / n */
  double hi[3];
  int bc[3];       /* ENOAO_PERIODIC or ENOAO_TRANSMISSIVE (zero-gradient) per axis */
  int alpha_mode;  /* ENOAO_ALPHA_PER_STEP, _PER_STAGE or _PER_FIELD */
  double adv_speed;  /* scalar advection speed a */
  double gamma;      /* ratio of specific heats (Euler) */
  double delta;      /* selection threshold, 1e-5 in the paper (Sec. 3.2 remark) */
  double tie_rel;    /* FP32_BULK: relative margin under which an indicator
                        comparison is re-done in FP64 */
} enoao_config;

/* Run statistics of a context. */
typedef struct {
  double t;                   /* simulated time reached */
  int64_t steps;              /* Runge-Kutta steps taken since enoao_init_state */
  double alpha[3];            /* Lax-Friedrichs alpha per axis of the last step */
  double dt;                  /* last step size */
  uint64_t fp64_fallbacks;    /* FP32_BULK: indicator decisions re-done in FP64 */
  uint64_t decisions;         /* stencil decisions taken (2 per field per face) */
} enoao_stats;

/* Fills a configuration with defaults: 1D, Euler, order 5, FP64, periodic,
 * gamma 1.4, adv_speed 1, delta 1e-5, tie_rel 1e-3, one cell per axis. */
void enoao_config_default(enoao_config *cfg);

/* Creates a context for one problem -- the conservation law u_t + f(u)_x = 0
 * on a uniform grid of n cells per axis (Sec. 2; dimension by dimension in 2D
 * and 3D) -- and allocates its device memory (three state buffers: U^n and
 * the two intermediate Runge-Kutta stages, and one right-hand-side buffer) on
 * the current device.
 * cuda_stream: a cudaStream_t (may be 0).  Errors: ENOAO_EINVAL for an
 * invalid configuration (ndim not 1..3, order not 5 or 7, fewer cells along
 * a swept axis than the stencil needs (11), non-positive dx, gamma <= 1,
 * delta < 0), ENOAO_ENOMEM, ENOAO_ECUDA.  *out is NULL on failure. */
enoao_status enoao_create(const enoao_config *cfg, void *cuda_stream, enoao_ctx **out);

/* Creates a context for nprob independent 1D problems of uneven lengths n[i]
 * on [lo[i], hi[i]] that share proto's system, order, precision, boundary
 * conditions and constants; each problem keeps its own alpha and time step.
 * States are concatenated: U[v][offset_i + i], offset_i = sum_{k<i} n[k].
 * They advance together in one persistent launch (enoao_batch_advance_steps).
 * Only 1D Euler or scalar problems; errors as enoao_create. */
enoao_status enoao_batch_create(const enoao_config *proto, int nprob, const int64_t *n,
                                const double *lo, const double *hi, void *cuda_stream,
                                enoao_ctx **out);

/* ---- Domain decomposition: a sub-domain of a grid split along its last axis.
 * The conservation form (Sec. 2, Eq. 1DWENOFD) needs, per Runge-Kutta stage,
 * the G = order/2 + 2 cells beyond a cell on each side of every axis, and
 * alpha of the global splitting is the maximum of |f'(u)| over the whole mesh
 * (Sec. 2).  A sub-domain context owns the layers [offset, offset + n_local)
 * of the last axis of the global problem (2D: rows, 3D: planes) and keeps G
 * ghost layers on each side of that axis in its arrays.  A step is then:
 * alpha = max over sub-domains of enoao_local_alpha, enoao_set_step_alpha,
 * dt = cfl / sum_d alpha_d / dx_d, and per stage k = 0, 1, 2: fill the ghost
 * layers of stage state k (enoao_halo_export on the neighbour, exchange,
 * enoao_halo_import here; enoao_halo_fill_transmissive at a transmissive edge
 * of the global grid; a periodic edge exchanges with the sub-domain at the
 * other end), then enoao_rk_stage(ctx, k, dt).  Results equal the undivided
 * grid's bit for bit.  enoao_init_state / enoao_get_state /
 * enoao_get_stage_state take the sub-domain's interior ([nv][n_local layers]);
 * non-physical cells are reported by their interior index.
 *
 * Creates the context of layers [offset, offset + n_local) of the 2D or 3D
 * problem global (its n, lo, hi, bc and constants).  Errors: as
 * enoao_create; ENOAO_EINVAL for a 1D problem, alpha_mode other than
 * ENOAO_ALPHA_PER_STEP, n_local < G or a range outside the grid.  Sub-domains
 * step stage by stage only (enoao_advance* return ENOAO_EINVAL) and FP32 bulk
 * re-decides its near-ties inside the sweep. */
enoao_status enoao_create_subdomain(const enoao_config *global, int64_t offset, int64_t n_local,
                                    void *cuda_stream, enoao_ctx **out);

/* Halo layers of stage state k (0: U^n, 1: U^(1), 2: U^(2)) on side 0 (low
 * index) or 1 (high index) of the split axis.  The buffer holds
 * [nv][G][plane] doubles, layers in increasing index order, plane the cells
 * of one layer (2D: n[0], 3D: n[0] n[1]).  Export copies the G interior
 * layers next to the side out; import writes the G ghost layers beyond it.
 * Both synchronise.  ENOAO_EINVAL for a context that is not a sub-domain, k
 * outside 0..2 or side not 0 or 1. */
enoao_status enoao_halo_export(enoao_ctx *ctx, int k, int side, double *buf, int on_device);
enoao_status enoao_halo_import(enoao_ctx *ctx, int k, int side, const double *buf,
                               int on_device);

/* Zero-gradient ghost layers (the transmissive boundary, each ghost layer a
 * copy of the edge layer) beyond side of stage state k; for a sub-domain at
 * a transmissive edge of the global grid.  Synchronises. */
enoao_status enoao_halo_fill_transmissive(enoao_ctx *ctx, int k, int side);

/* The maximum over this context's cells of the Lax-Friedrichs alpha per axis
 * (Sec. 2: |u_d| + c for the Euler equations, |a| for advection) for the
 * current U^n, in the arithmetic of the context's precision; for a
 * sub-domain, the value to take the maximum over all sub-domains of.
 * Synchronises; ENOAO_ENONPHYS if U^n holds a non-physical cell. */
enoao_status enoao_local_alpha(enoao_ctx *ctx, double *alpha);

/* Sets the alpha per axis that the next step (enoao_rk_stage stage 0) splits
 * with, in place of this context's own maximum -- the global maximum of a
 * decomposed grid.  ENOAO_EINVAL for negative or non-finite values, batched
 * contexts and alpha modes other than ENOAO_ALPHA_PER_STEP. */
enoao_status enoao_set_step_alpha(enoao_ctx *ctx, const double *alpha);

/* Time reached, the Lax-Friedrichs alpha its last step split with (Sec. 2:
 * the maximum of |f'(u)| over that problem's mesh) and the last step size of
 * problem p of a batched context (synchronises).  Null outputs are skipped.
 * ENOAO_EINVAL for a context that is not batched or p outside 0..nprob-1. */
enoao_status enoao_batch_problem_stats(enoao_ctx *ctx, int p, double *t, double *alpha,
                                       double *dt);

/* Releases every resource of the context (NULL is ignored). */
void enoao_destroy(enoao_ctx *ctx);

/* Message of the last failure on this context ("" if none); valid until the
 * next call on the context.  ctx may be NULL (message of the last failed
 * create, or of the last failed enoao_step_noalloc, on this host thread). */
const char *enoao_last_error(const enoao_ctx *ctx);

/* Sets the state U^n (conserved variables, layout above; for the Euler
 * equations of Sec. 4 rho, momenta and total energy) and resets time and
 * step count.  Computes alpha of the new state (Sec. 2: the maximum of
 * |f'(u)| over the mesh), with the arithmetic the steps take it in.
 * ENOAO_ENONPHYS if the state has rho <= 0, p <= 0 or NaN (Euler), with
 * the first such cell in the message. */
enoao_status enoao_init_state(enoao_ctx *ctx, const double *U, int on_device);

/* Copies the current state U^n out (same layout): the numerical solution
 * u_j of Sec. 2 at the time reached (enoao_get_stats). */
enoao_status enoao_get_state(enoao_ctx *ctx, double *U, int on_device);

/* Copies a Runge-Kutta stage state out (same layout): k = 0 is U^n (as
 * enoao_get_state), k = 1 and 2 are U^(1) = U^n + dt L(U^n) and U^(2) of
 * Sec. 2's third-order TVD scheme as the stages last wrote them -- after
 * enoao_rk_stage(ctx, 0 or 1, dt) the state the next stage starts from, after
 * a whole step the last step's.  For checking a step stage by stage.
 * ENOAO_EINVAL for k outside 0..2 and for batched contexts. */
enoao_status enoao_get_stage_state(enoao_ctx *ctx, int k, double *U, int on_device);

/* Interface fluxes F_{j+1/2} of Eq. (1DWENOFD) along axis dir for the current
 * state, with alpha of the current state (Sec. 2, 3, 4).  Fhat has the state's
 * layout with n[dir] replaced by n[dir]+1 faces; face f lies between cells
 * f-1 and f (periodic: faces 0 and n[dir] coincide).  stencil_idx (may be
 * NULL) receives the chosen candidate (priority index 0..8: S_j^j, S_j^{j+1},
 * S_{j-1}^{j+1}, S_{j-2}^{j+1}, S_{j-1}^{j+2}, S_{j-2}^{j+2}, S_{j-3}^{j+2},
 * S_{j-2}^{j+3}, S_{j-3}^{j+3}) per characteristic field v (Euler order:
 * u-c, entropy, shear..., u+c), sign s (0: f^+, 1: f^-) and face at
 * stencil_idx[(v*2 + s)*nfaces + face].  Not available for batched contexts.
 * With host buffers (on_device = 0) the results pass through device scratch
 * that the context keeps: the first call (or one that needs more of it)
 * allocates it, enoao_destroy frees it. */
enoao_status enoao_reconstruct_fluxes(enoao_ctx *ctx, int dir, double *Fhat,
                                      int8_t *stencil_idx, int on_device);

/* One stage (0, 1 or 2) of the third-order TVD Runge-Kutta step (Sec. 2):
 *   stage 0: U1 = U^n + dt L(U^n)      (alpha recomputed from U^n)
 *   stage 1: U2 = 3/4 U^n + 1/4 (U1 + dt L(U1))
 *   stage 2: U^{n+1} = 1/3 U^n + 2/3 (U2 + dt L(U2))
 * Stages must be called in order; after stage 2 the state is U^{n+1} and the
 * step count and time advance by one step and dt.  In FP32 bulk the stages
 * are evaluated as each stage's input plus an FP32 increment (U2 = U1 +
 * 1/4 dt L(U1) - 3/4 I0, U^{n+1} = U2 + 2/3 dt L(U2) - 1/12 I1, with I0 =
 * dt L(U^n) and I1 = I0 + dt L(U1) kept by the context), equal to the forms
 * above up to an FP32 rounding of the increment. */
enoao_status enoao_rk_stage(enoao_ctx *ctx, int stage, double dt);

/* Advances to t_end with dt = cfl / sum_d(alpha_d / dx_d), alpha from U^n of
 * each step, the last step shortened to land on t_end; or with the fixed
 * step dt_fixed when dt_fixed > 0.  Stops after max_steps steps when
 * max_steps > 0.  Steps run as CUDA-graph replays; alpha and dt never leave
 * the device.  Returns the time reached and the steps taken (nullable). */
enoao_status enoao_advance(enoao_ctx *ctx, double t_end, double cfl, double dt_fixed,
                           int64_t max_steps, double *t_out, int64_t *steps_out);

/* Advances exactly nsteps third-order TVD Runge-Kutta steps (Sec. 2) with
 * dt = cfl / sum_d(alpha_d / dx_d), alpha from U^n of each step (no end
 * time).  For batched contexts every problem takes nsteps steps with its own
 * alpha and dt in one persistent launch. */
enoao_status enoao_advance_steps(enoao_ctx *ctx, int64_t nsteps, double cfl);

/* Same as enoao_advance_steps but only enqueues the work on the stream and
 * returns without synchronising or reading the error word (for timing
 * loops); check with enoao_sync. */
enoao_status enoao_advance_steps_async(enoao_ctx *ctx, int64_t nsteps, double cfl);

/* Waits for the context's work and reports ENOAO_ENONPHYS / ENOAO_ETIMEOUT
 * raised by kernels since the last check. */
enoao_status enoao_sync(enoao_ctx *ctx);

/* Reads the run statistics (synchronises). */
enoao_status enoao_get_stats(enoao_ctx *ctx, enoao_stats *out);

/* Number of CUDA kernel launches one step issues (per graph replay step). */
int enoao_launches_per_step(const enoao_ctx *ctx);

/* Tile shape of the sweep kernels along each axis: lines per tile (ta) and
 * faces per tile (ts).  Set by the autotuner or by hand; 0 keeps the current
 * value.  Errors: ENOAO_EINVAL for shapes the kernels do not support. */
enoao_status enoao_set_tiles(enoao_ctx *ctx, int dir, int ta, int ts);
enoao_status enoao_get_tiles(const enoao_ctx *ctx, int dir, int *ta, int *ts);

/* Where FP32_BULK re-decides its near-tie stencil choices in FP64 (the
 * selection of Sec. 3.2 taken again from the FP64 state when the FP32
 * indicators cannot order it).  IN_SWEEP: inside the sweep, by the tile that
 * meets the choice.  GRID: each sweep lists the faces with such choices and a
 * pass over the whole GPU re-decides them after it, then applies the changed
 * choices to the two cells of each face (two extra launches per sweep; the
 * choices cluster at discontinuities, in tiles whose SMs would otherwise set
 * the sweep's length).  GRID pays where near-ties reach a few per cent of
 * the cells per step (shock and slip-line dominated flows such as the 2D
 * Riemann problems); elsewhere the pass, which has no FP32 work to hide its
 * FP64 work behind, costs more than it saves.  AUTO (default): IN_SWEEP.
 * Both give the same choices; the state differs by FP32 rounding of the
 * correction.  Either way results do not depend on tile shapes.  GRID needs
 * 8 + 4 nv + 4 bytes per face of the axis with most faces, allocated here.
 * The FP64 precision has no near-ties and ignores the mode.  GRID on a grid
 * with 2^32 or more faces along an axis falls back to IN_SWEEP.
 * Errors: ENOAO_EINVAL for an unknown mode or GRID on a batched context,
 * ENOAO_ENOMEM when the list cannot be allocated (the mode is then kept). */
enum { ENOAO_REDECIDE_AUTO = 0, ENOAO_REDECIDE_IN_SWEEP = 1, ENOAO_REDECIDE_GRID = 2 };
enoao_status enoao_set_redecide(enoao_ctx *ctx, int mode);
/* 1 when the context's steps use the grid-wide pass, else 0. */
int enoao_uses_grid_redecide(const enoao_ctx *ctx);

/* Whether FP32-bulk sweeps stage each tile's raw state (every component of
 * the tile's cells and halo) into shared memory with one TMA bulk tensor copy
 * per tile, issued a tile ahead (on = 1), or load it cell by cell (0, the
 * default: measured faster on GB300, the box's shared memory costing more
 * resident blocks than the copy saves).  Shapes TMA cannot address (row
 * strides not a multiple of 16 bytes, boxes beyond 256 cells, sub-domains,
 * the per-field and grid re-decision variants) load directly either way.
 * The results are the same bits. */
enoao_status enoao_set_tma(enoao_ctx *ctx, int on);

/* Whether each Runge-Kutta stage of a 2D problem runs as one launch for both
 * axes (on = 1; Sec. 2: L(u) is the unsplit sum of the two axes' flux
 * differences) instead of one launch per axis (0, the default).  A block
 * takes a 2D tile of x_cells x y_cells cells: the x part of L(u) on it in
 * tiles of x_lines rows x x_cells cells, then the y part in tiles of y_lines
 * columns x y_cells cells, which adds the x part the block just stored and
 * combines.  x_lines: 1, 2, 4 or 8; y_lines: 8, 16, 32 or 64; y_cells a
 * multiple of x_lines and x_cells of y_lines; all four 0 keeps the current
 * tiles (4, 64, 8, 48 by default).  It applies to FP32-bulk contexts with one
 * alpha and in-sweep re-decisions, without TMA staging, of 2D scalar
 * advection or Euler, ENO-AO5 or AO7, on a whole grid; other contexts keep
 * one launch per axis.  The results are the same bits either way.
 * ENOAO_EINVAL for a 3D or 1D context, bad tiles or a batched context. */
enoao_status enoao_set_fused_stage(enoao_ctx *ctx, int on, int x_lines, int x_cells, int y_lines,
                                   int y_cells);

/* Fault-injection knob for tests (the paper has no counterpart): bounds the
 * passes in which a warp re-decides its flagged FP32-bulk choices inside the
 * sweep (the default, -1, is 64 nv passes, which every warp needs at most
 * 2 nv of).  A warp that reaches a smaller bound stops waiting, keeps the FP32
 * pick of the choices left and sets the device error word, so that the next
 * synchronising call returns ENOAO_ETIMEOUT; nothing traps and the context
 * stays usable (enoao_init_state clears the error).  ENOAO_EINVAL for
 * batched contexts and for limits below -1. */
enoao_status enoao_set_redecide_pass_limit(enoao_ctx *ctx, int passes);

/* One third-order TVD Runge-Kutta step of a 1D problem that allocates no
 * device memory.  The paper has no counterpart: this is a deployment aid for
 * callers that cannot let a library allocate -- applications that reserve
 * all device memory up front for their own allocator or run under a fixed
 * memory budget, and time loops that must not pay the implicit device-wide
 * synchronisation cudaMalloc/cudaFree may cause.
 *   cfg    : 1D problem (ndim 1, n[0] cells, Euler or scalar advection, order,
 *            precision, bc[0], gamma / adv_speed, delta, tie_rel as in
 *            enoao_config); at most 262144 cells -- larger problems return
 *            ENOAO_EINVAL with a message naming the limit.
 *   U_in   : device pointer, U^n as [nv][n] float64 (not modified).
 *   U_out  : device pointer, receives U^{n+1} in the same layout; may equal
 *            U_in.
 *   dt     : step size; alpha is computed from U_in.
 *   stream : cudaStream_t the work is ordered on (0 = legacy default).
 * U_in and U_out must be device memory of the current device (checked:
 * ENOAO_EINVAL otherwise); their size cannot be checked from a pointer, so
 * each must hold nv * n[0] doubles.
 * The two intermediate stage states, the two FP32 stage increments of the
 * FP32 bulk combine and the step's device-side state live in
 * one fixed file-scope device array (18 MiB per GPU, held until the process
 * exits).  The first call on a device loads the library's device code there
 * (CUDA loads modules lazily by default), which brings the array into
 * existence, and looks up its device address (cudaGetSymbolAddress); make
 * that first call during set-up, before any stream capture.  The address is
 * kept for the life of the process, so do not use this entry point on a
 * device after cudaDeviceReset.  Every call shares the array and finds the
 * previous call's contents there (whatever must start at zero is cleared by
 * the call), so calls that overlap on the GPU -- from other streams or
 * threads -- race: serialise them.  The call waits for its stream to finish
 * the step and returns ENOAO_ENONPHYS for rho <= 0, p <= 0 or NaN (with the
 * first such cell in the message) and ENOAO_ETIMEOUT when a bounded device
 * wait gave up; messages are read with enoao_last_error(NULL). */
enoao_status enoao_step_noalloc(const enoao_config *cfg, const double *U_in, double *U_out,
                                double dt, void *cuda_stream);

/* Measurement helper: launches the sweep kernel of axis dir for Runge-Kutta
 * stage 0 on the current state nrep times back to back on the library's
 * stream, timed with CUDA events recorded on that stream, and returns the
 * mean duration of one launch in milliseconds.  The state U^n is not
 * modified (stage 0 writes U1). */
enoao_status enoao_time_sweep(enoao_ctx *ctx, int dir, int nrep, float *ms_per_launch);

/* Measurement helper (the paper has no counterpart): the arithmetic peak the
 * roofline of the sweep kernels divides by.  kind ENOAO_PEAK_FP32 (scalar
 * FP32 fused multiply-add), ENOAO_PEAK_FP32X2 (packed pairs, two per
 * instruction) or ENOAO_PEAK_FP64.  Every thread of a grid of 8 blocks of 256
 * threads per SM runs 8 independent multiply-add chains for trips x 64 steps;
 * one warm-up launch, then one launch timed with CUDA events on cuda_stream.
 * Returns the rate in TFLOP/s (2 flops per multiply-add) and the launch time
 * in ms, at whatever clock the GPU ran (no clock is set).  Allocates 8 MiB of
 * scratch for the duration of the call.  ENOAO_EINVAL for an unknown kind. */
enum { ENOAO_PEAK_FP32 = 0, ENOAO_PEAK_FP32X2 = 1, ENOAO_PEAK_FP64 = 2 };
enoao_status enoao_measure_fma_peak(int kind, int trips, void *cuda_stream, double *tflops,
                                    float *ms);

/* Times every supported tile shape of every axis on the current state
 * (restored afterwards) with CUDA events and keeps the fastest. */
enoao_status enoao_autotune(enoao_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* ENOAO_H */
