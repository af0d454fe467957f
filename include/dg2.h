/*
 * dg2.h -- C ABI of the GB300 DG2 flood solver.
 *
 * The solver advances the slope-decoupled second-order discontinuous Galerkin
 * (DG2) solution of the 2D shallow water equations of Ayog et al.,
 * "Second-order discontinuous Galerkin flood model" (Sec. 2.1): per cell an
 * average and an x- and y-slope coefficient of h, hu, hv (Eq. 2), topography
 * coefficients from DEM corner nodes (Eq. 3), explicit two-stage RK2 steps of
 * the operators of Eqs. 4-5 with HLL fluxes, implicit Manning friction
 * (Sec. 2.1.3), optional local slope limiting (Eqs. 6-7) and a global
 * Courant-number time step.
 *
 * Conventions
 *  - Grid: nx cells along x (west -> east), ny along y (south -> north); cell
 *    (i, j) spans [i dx, (i+1) dx] x [j dy, (j+1) dy].  Host arrays are
 *    row-major with the x index fastest.
 *  - State planes (host side, dense, ny*nx each), in this order:
 *    h0, h1x, h1y, qx0, qx1x, qx1y, qy0, qy1x, qy1y  (Eq. 2 coefficients).
 *  - Corner arrays (DEM, initial free surface) are (ny+1) x (nx+1).
 *  - Every function returns DG2_OK (0) or a negative DG2_E_* code; the text
 *    of the last error of the calling thread is in dg2_last_error().
 *  - Host input arrays are copied before the call returns; the caller keeps
 *    ownership.  Host output arrays are caller-allocated.
 *  - Device memory: the caller provides one device workspace of at least
 *    dg2_workspace_bytes() bytes (e.g. a torch uint8 tensor) and keeps it alive
 *    until dg2_destroy().  The library allocates no device memory itself.
 *  - Stream: every kernel and copy is issued on the caller's stream (a
 *    cudaStream_t passed as void*; NULL = legacy default stream).  Calls that
 *    return host data synchronise that stream.
 *  - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef DG2_H
#define DG2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    DG2_OK = 0,
    DG2_E_ARG = -1,        /* invalid argument (size, pointer, range)          */
    DG2_E_STATE = -2,      /* call order (e.g. stepping before dg2_set_dem)     */
    DG2_E_CUDA = -3,       /* a CUDA runtime call or kernel launch failed       */
    DG2_E_NONFINITE = -4,  /* a NaN/Inf or a time step <= 0 appeared on device  */
    DG2_E_NOMEM = -5,      /* workspace smaller than dg2_workspace_bytes()      */
    DG2_E_OVERFLOW = -7    /* gauge sample buffer full; extra samples dropped   */
};

enum { DG2_NL = 0, DG2_LL = 1 };            /* DG2-NL: no limiting; DG2-LL: Eqs. 6-7 */
/* Arithmetic of the bulk update.  DG2_FP64: FP64 depth modes, the form of
 * Eqs. 4-5.  DG2_FP32: FP32 free-surface modes eta = h + z with the momentum
 * terms regrouped around each limit's own hydrostatic pressure (algebraically
 * Eqs. 4-5, exactly still at rest in FP32); time, step size, reductions and
 * the mass ledger stay FP64 in both.  State I/O is FP64 depth modes in both. */
enum { DG2_FP64 = 0, DG2_FP32 = 1 };
enum { DG2_WALL = 0, DG2_OPEN = 1 };        /* edge types                            */
enum { DG2_HLL = 0, DG2_ROE = 1 };          /* Riemann solvers                       */
/* Spatial schemes: the slope-decoupled DG2 (Sec. 2.1) or the finite-volume
 * comparators of Sec. 2.2 (MUSCL-FV2: Eqs. 8-10, RK2; FV1: first order,
 * forward Euler) */
enum { DG2_SCHEME_DG2 = 0, DG2_SCHEME_FV2 = 1, DG2_SCHEME_FV1 = 2 };
/* DG2 face revision of partially wet cells (wet cells whose planar depth is
 * negative at a face): DG2_WD_POSITIVE (default) scales such a cell's clipped
 * face depths to average h0 and revises its faces on the free surface
 * (Sec. 2.2.2) so that averages stay near non-negative and still water stays
 * still; DG2_WD_PRINTED is Sec. 2.1.2 as printed (h* = max(0, h)).  Fully wet
 * cells take the printed revision under both. */
enum { DG2_WD_POSITIVE = 0, DG2_WD_PRINTED = 1 };
enum { DG2_WEST = 0, DG2_EAST = 1, DG2_SOUTH = 2, DG2_NORTH = 3 };

typedef struct dg2_params {
    double g;           /* gravity, m/s^2 (default 9.80665)                         */
    double cfl;         /* Courant number Cr (Sec. 2.1.2; default 0.3)               */
    double tol_dry;     /* drying tolerance on h (Sec. 2.1.3; default 1e-5 m)        */
    double ds_thresh;   /* shock-detector threshold of Eq. 6 (default 10)            */
    double dt_max;      /* time step when no cell is wet, and upper cap (default 1 s)*/
    int variant;        /* DG2_NL or DG2_LL                                          */
    int precision;      /* DG2_FP64 or DG2_FP32                                      */
    int bc[4];          /* DG2_WALL or DG2_OPEN per edge, indexed by DG2_WEST..NORTH */
    int max_gauges;     /* capacity of the gauge table (default 64)                  */
    int max_samples;    /* capacity of the gauge sample buffer in rows (default 4096)*/
    int skip_dry_tiles; /* 1 (default): leave 32 x 8 tiles of still, dry cells with
                           still, dry neighbours untouched -- they are exact fixed
                           points of a step, so results are bit-identical; 0: compute
                           every tile */
    int flux;           /* Riemann solver: DG2_HLL (default) or DG2_ROE (Roe's solver
                           named in Sec. 2.1.2, Harten's entropy fix; DG2_FP64 only) */
    int scheme;         /* DG2_SCHEME_DG2 (default), or DG2_SCHEME_FV2 / DG2_SCHEME_FV1
                           (Sec. 2.2): cell averages only (the slope planes of the
                           state are zeroed by dg2_set_dem and otherwise left as
                           they are), Sweby's limiter with beta = 1.25 for FV2,
                           friction on the averages; DG2_FP64 and DG2_NL only */
    int wetdry;         /* DG2_WD_POSITIVE (default) or DG2_WD_PRINTED; see above */
} dg2_params;

typedef struct dg2_ctx dg2_ctx;

/* Fills *p with the defaults listed above (variant NL, FP64, all walls). */
void dg2_default_params(dg2_params *p);

/* Text of the last error raised on the calling thread ("" if none). */
const char *dg2_last_error(void);

/* Device workspace needed for an nx x ny grid under *p (bytes; 0 on bad args).
 * Holds the state, one stage state, limited-slope scratch (DG2_LL), topography,
 * Manning n, per-block partials, the gauge buffers and device scalars. */
size_t dg2_workspace_bytes(int nx, int ny, const dg2_params *p);

/* Creates a context on the current CUDA device for the uniform Cartesian grid
 * of Sec. 2.1.1 (cells Q_c of size dx x dy, the stencil of Fig. 1).
 * nx, ny >= 1; dx, dy > 0; p may be NULL for defaults.  dev_workspace must be
 * 256-byte aligned device memory of ws_bytes >= dg2_workspace_bytes().  The
 * grid starts dry and flat until dg2_set_dem().  *out receives the context. */
int dg2_init_grid(dg2_ctx **out, int nx, int ny, double dx, double dy, const dg2_params *p,
                  void *dev_workspace, size_t ws_bytes, void *cuda_stream);

/* Topography, roughness and initial water (Sec. 2.1.1: DEM values at the corner
 * nodes, face-centred node values by averaging, modes by Eq. 3; Manning n of
 * the friction term of Eq. 1).
 * z_corner: (ny+1)*(nx+1) DEM at corner nodes (m), required.
 * manning: ny*nx per-cell Manning n (s m^-1/3), or NULL to use n_uniform.
 * eta_corner: (ny+1)*(nx+1) initial free-surface elevation at corners, or NULL
 *   for a dry start.  Corner depths eta - z are averaged to face nodes and
 *   turned into modes by Eq. 3 without clipping; a cell whose average depth
 *   is not positive starts dry.  Discharges start at zero.
 * Resets t = 0, the mass ledger and the gauge buffer, and computes the first
 * time step. */
int dg2_set_dem(dg2_ctx *ctx, const double *z_corner, const double *manning, double n_uniform,
                const double *eta_corner);

/* Adds an inflow hydrograph Q(t) (m^3/s, piecewise linear in t_knots, held
 * constant outside them): the discharge hydrographs imposed at a breach or a
 * west boundary in the paper's test cases (Sec. 3; Figs. 8, 11 and 14 show
 * them; Fig. 5b is a water-level hydrograph, which this call does not model).
 * It acts on the faces of `edge` whose centres lie in
 * [s0_m, s0_m + len_m] along the edge.  The discharge per unit width is Q
 * divided by the total length of those faces; it enters through a
 * critical-depth ghost state.  At most 8 inflows, 4096 knots each, t_knots
 * strictly increasing.  DG2_E_ARG if no face lies in the segment. */
int dg2_set_bc_inflow(dg2_ctx *ctx, int edge, double s0_m, double len_m, const double *t_knots,
                      const double *q_knots, int nknots);

/* Uniform rainfall (m/s) during [rain_t0, rain_t1) and a point inflow
 * q_point_m3s at (px, py), both added to the average depth equation.  These
 * sources are not in the paper; they drive the urban-style workloads. */
int dg2_set_sources(dg2_ctx *ctx, double rain_mps, double rain_t0, double rain_t1, double px,
                    double py, double q_point_m3s);

/* One RK2 time step (Sec. 2.1.2: two Runge-Kutta stages of the operators of
 * Eqs. 4-5 with the revised face limits; Sec. 2.1.3: friction by implicit
 * splitting before the step and, for DG2_LL, local limiting by Eqs. 6-7 before
 * each stage; wet-dry flags by h0 against tol_dry).  dt > 0 forces that step
 * size; dt <= 0 takes the Courant-number step (Cr of Sec. 2.1.2) computed from
 * the current state.  The step
 * taken is written to *dt_taken (may be NULL; writing it synchronises). */
int dg2_step(dg2_ctx *ctx, double dt, double *dt_taken);

/* Advances until t_end with Courant-number RK2 steps (as dg2_step, Sec. 2.1.2),
 * landing exactly on t_end (the output time T of Table 2) and on every gauge
 * sample time, so the time series of Sec. 3 (water level and velocity
 * hydrographs at sampling points, compared by Eqs. 13-14) are recorded at
 * exact times.  Runs on the device with no host round
 * trip per step (chunks of steps; a device flag stops work past t_end).
 * *steps_taken (may be NULL) receives the number of steps. */
int dg2_run_to(dg2_ctx *ctx, double t_end, int64_t *steps_taken);

/* Gauges: the sampling points of Sec. 3 (red dots of Figs. 5a, 8, 11, 14),
 * whose depth time series the paper compares.  xy = ngauge (x, y) pairs in
 * metres; depth max(0, planar h) of the containing cell's piecewise-planar
 * solution (Eq. 2) is recorded at every multiple of sample_every_s reached by
 * dg2_run_to.  Replaces earlier gauges and clears the sample buffer. */
int dg2_set_gauges(dg2_ctx *ctx, const double *xy, int ngauge, double sample_every_s);

/* The recorded gauge time series (Sec. 3), copied out; clears the buffer: t_out[cap],
 * h_out[cap][ngauge]; *nsamp = rows written.  DG2_E_OVERFLOW if samples were
 * dropped since the last read (the rows kept are still returned). */
int dg2_read_gauges(dg2_ctx *ctx, double *t_out, double *h_out, int cap, int *nsamp);

/* Domain mass sum(h0) dx dy (Eq. 11) and the ledger: initial mass plus the
 * volume that boundaries and sources added since dg2_set_dem/dg2_set_state.
 * Either pointer may be NULL. */
int dg2_mass(dg2_ctx *ctx, double *mass_m3, double *ledger_m3);

/* State in and out: planes = 9 dense ny*nx host planes in the order above. */
int dg2_get_state(dg2_ctx *ctx, double *planes, double *t);
int dg2_set_state(dg2_ctx *ctx, const double *planes, double t);

/* Topography modes z0, z1x, z1y (3 dense planes) as computed from the DEM. */
int dg2_get_topo(dg2_ctx *ctx, double *planes3);

/* Current time and the step size the next Courant step would take. */
int dg2_get_time(dg2_ctx *ctx, double *t, double *dt_next);

/* Per-kernel timing with CUDA events on the context's stream.  While enabled,
 * each dg2_step records an event before and after each of its three kernels
 * (friction, stage 1, stage 2) -- at most 8192 steps between reads.
 * dg2_kernel_times() synchronises the stream, writes the summed milliseconds
 * of each kernel to ms[0..2] and the number of steps timed to *nsteps, and
 * starts a new count.  dg2_run_to is never timed this way. */
int dg2_enable_kernel_timing(dg2_ctx *ctx, int enable);
int dg2_kernel_times(dg2_ctx *ctx, double *ms3, int64_t *nsteps);

/* Completed steps since the last dg2_set_dem / dg2_set_state (also those an
 * ensemble took for this member).  Synchronises the stream. */
int dg2_get_steps(dg2_ctx *ctx, int64_t *steps);

/* Number of kernels this context has launched (for launch accounting). */
int64_t dg2_launch_count(const dg2_ctx *ctx);

/* Cells per tile of the context's exact dry-tile skipping, the tiles that
 * dg2_tile_stats counts: writes the width (x) and height (y) of a tile, 32 x 8
 * for FP64 contexts; for FP32 ones 16 x 8 on grids of up to 2^23 cells and
 * 32 x 8 on larger ones.  Either pointer may be NULL.
 * Errors: DG2_E_ARG (null context). */
int dg2_tile_shape(dg2_ctx *ctx, int *w, int *h);

/* Tile accounting of the exact dry-tile skipping (tiles of dg2_tile_shape):
 * writes the number of tiles of the grid, the tiles the next step will compute and
 * copy (frontier), and the running total of tiles computed by all completed
 * steps (the units the stage kernels processed).  Any pointer may be NULL.
 * Synchronises the context's stream.  Errors: DG2_E_ARG (null context). */
int dg2_tile_stats(dg2_ctx *ctx, int *ntiles, int *n_active, int *n_frontier,
                   int64_t *tiles_computed);

/* Largest grid height (rows) that dg2_mass_noalloc accepts. */
#define DG2_NOALLOC_MAX_ROWS 65536

/* Domain mass sum(h0) * dx * dy of a depth-average plane, computed without
 * allocating any device memory.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory themselves
 * (a fixed memory pool they do not own, a plugin given only raw pointers).
 *   h0_dev   device pointer to ny rows of pitch doubles (row j at h0_dev + j*pitch;
 *            the first nx of each row are summed), e.g. plane 0 of a state.
 *   mass_dev device pointer to one double that receives the mass (m^3).
 *   cuda_stream  the stream the reduction runs on (void* cudaStream_t, NULL =
 *            legacy default stream); the call returns before it finishes.
 * Scratch: one partial per grid row and a block counter in a fixed
 * file-scope __device__ array (DG2_NOALLOC_MAX_ROWS doubles, 512 KiB), held by
 * every GPU that loads the library until the process exits.  Each call looks
 * up that array's device address in the current context (cudaGetSymbolAddress,
 * not cached, so a recreated context is followed); the first call on a device
 * may load the module, so make it before any stream capture.  Every call
 * shares the array, so calls that overlap on the GPU race; the counter is
 * cleared at the start of each call.  DG2_E_ARG if ny > DG2_NOALLOC_MAX_ROWS,
 * nx or ny < 1, pitch < nx, dx or dy <= 0, or a pointer is NULL.  Calls no
 * cudaMalloc, cudaFree or other allocating routine. */
int dg2_mass_noalloc(const double *h0_dev, int nx, int ny, int pitch, double dx, double dy,
                     double *mass_dev, void *cuda_stream);

/* Releases the host-side context (the workspace stays the caller's). */
int dg2_destroy(dg2_ctx *ctx);

/* Measured FP64 arithmetic peak of the current GPU, the denominator of the FP64
 * stage kernels' roofline (they are bound by the FP64 pipe, not by HBM; the paper
 * has no counterpart).  Launches blocks_per_sm (1..8) blocks of 256 threads per SM,
 * each thread running 8 independent chains of iters FP64 fused multiply-adds, once
 * untimed and once timed with CUDA events on cuda_stream (void* cudaStream_t, NULL =
 * legacy default stream); writes 2 x FMAs / time in GFLOP/s to *gflops and the
 * timed kernel's milliseconds to *ms (may be NULL).  Synchronises the stream.
 * Allocates nothing.  Errors: DG2_E_ARG (bad counts, gflops NULL), DG2_E_CUDA. */
int dg2_fp64_fma_peak(int blocks_per_sm, int iters, void *cuda_stream, double *gflops,
                      double *ms);

/* ------------------------------------------------------------------------
 * Ensembles: many FP32 problems advanced together.
 *
 * An ensemble gathers existing DG2_FP32 contexts ("members", all of one
 * variant, each already given its DEM or state, inflows, sources and gauges)
 * and advances all of them with one set of launches per step: one list of
 * (member, tile) work items per step, each member with its own Courant step,
 * time, ledger, gauges and landing on t_end.  Each member's result is bit for
 * bit the one dg2_run_to on that member alone gives (same cell arithmetic; the
 * tile shape changes only the summation order of the mass ledger's boundary
 * fluxes).  Members are read through their contexts while the ensemble runs:
 * do not step, reconfigure or destroy a member during an ensemble call; the
 * ensemble re-reads the members' parameters and recomputes every tile once at
 * the start of each dg2_ens_run_to.  State, time, mass and gauges are read
 * back through the member contexts (dg2_get_state, dg2_mass, ...).
 * ---------------------------------------------------------------------- */
typedef struct dg2_ens dg2_ens;

/* Device workspace bytes for an ensemble of these members (0 if a member is
 * NULL or not FP32, or nmembers is not 1..512).  Tile bookkeeping for every
 * tile shape the ensemble can take, the work lists and member descriptors. */
size_t dg2_ens_workspace_bytes(dg2_ctx *const *members, int nmembers);

/* Creates an ensemble of nmembers contexts (copied pointer array; the
 * contexts stay owned by the caller and must outlive the ensemble).  The
 * device workspace (>= dg2_ens_workspace_bytes, 256-byte aligned) and the
 * stream (void* cudaStream_t; a non-NULL stream enables CUDA-graph replay)
 * are the caller's.  Tile shape 32 x 8.  DG2_E_ARG: a NULL, duplicate or
 * non-FP32 member, mixed variants, bad workspace; DG2_E_STATE: a member
 * without DEM or state; DG2_E_NOMEM: workspace too small. */
int dg2_ens_create(dg2_ens **out, dg2_ctx *const *members, int nmembers, void *dev_workspace,
                   size_t ws_bytes, void *cuda_stream);

/* Advances every member to simulated time t_end (s) with its own Courant
 * steps, landing exactly on t_end and on its gauge sample times.  Members
 * already at or past t_end stay.  *steps_taken (may be NULL) = ensemble steps
 * replayed (the longest member's count, rounded up to the last chunk).
 * DG2_E_NONFINITE if a member's state or step became non-finite. */
int dg2_ens_run_to(dg2_ens *ens, double t_end, int64_t *steps_taken);

/* Picks the tile shape by timing: runs two passes over the supported shapes
 * (32x8, 32x4, 16x8, 64x4, 16x16 cells), each trial one untimed and
 * steps_per_trial (>= 4) timed steps of the run toward t_end (these are real
 * steps: the members advance), keeps the fastest shape and writes it to
 * *tile_w, *tile_h (may be NULL).  dg2_ens_tune_times gives the trial times. */
int dg2_ens_autotune(dg2_ens *ens, double t_end, int steps_per_trial, int *tile_w, int *tile_h);

/* Sets / reads the tile shape (one of the shapes listed above). */
int dg2_ens_set_tile_shape(dg2_ens *ens, int tile_w, int tile_h);
int dg2_ens_tile_shape(const dg2_ens *ens, int *tile_w, int *tile_h);

/* Milliseconds per step of each shape's best autotune trial (in the order
 * listed above; negative before dg2_ens_autotune).  Writes min(cap, count)
 * entries and returns the count of shapes. */
int dg2_ens_tune_times(const dg2_ens *ens, double *ms, int cap);

/* Number of kernels the ensemble has launched. */
int64_t dg2_ens_launch_count(const dg2_ens *ens);

/* Releases the ensemble (members and workspace stay the caller's). */
int dg2_ens_destroy(dg2_ens *ens);

/* ------------------------------------------------------------------------
 * Discrete adjoint of the DG2-NL step (Sec. 2.1.2-2.1.3), FP64 or FP32.
 *
 * Problem: nsteps DG2-NL steps (friction, the two RK stages of Eqs. 4-5, the
 * wet-dry treatment) from a given state with a given sequence of step sizes
 * (frozen: no derivative through the Courant step), one optional inflow
 * segment with a piecewise-linear hydrograph, and the misfit
 *     J = sum_s sum_g (h_g(U^{k_s}) - obs[s][g])^2
 * of gauge depths h_g = max(0, h0 + xi h1x + eta h1y) sampled after step
 * counts k_s (0..nsteps).  dg2_adj_gradient gives dJ/dn for the Manning n of
 * every cell and dJ/dq for every hydrograph knot discharge, by a reverse
 * sweep through each step's stages with the wet-dry, revision, HLL-regime
 * and ghost branches of the forward state frozen, and binomial checkpointing
 * of the step states in nsnap snapshot slots.  Under the default face revision
 * each face's revision depends on both cells' four depth limits (the partially
 * wet scale) and the cell's own terms on its faces' revised depths and beds;
 * both enter the reverse sweep.  Rain and point sources are not
 * part of the problem.  Planes are dense (ny rows of nx, x fastest).
 * Precision (dg2_params.precision): DG2_FP64, or DG2_FP32 -- the same step and
 * reverse sweep with every device buffer (state, checkpoints, adjoints, face
 * Jacobians, topography, Manning n, gradients) stored in FP32 and the
 * arithmetic kept in FP64 registers (the depth form's pressure / bed-term
 * balance does not survive FP32 arithmetic); half the checkpoint memory.  Host
 * arrays are FP64 in both.
 * ---------------------------------------------------------------------- */
typedef struct dg2_adj dg2_adj;

/* Workspace bytes (0 if a size is invalid: nx, ny, nsnap, max_steps >= 1,
 * max_gauges >= 0).  About (nsnap + 15) state-sized buffers of 9 planes: the
 * snapshots, the step's states and adjoints, the own terms' and faces'
 * adjoints and the revised faces of the step being reversed. */
size_t dg2_adj_workspace_bytes(int nx, int ny, int nsnap, int max_gauges, int max_steps);

/* params: g, tol_dry, bc[4], wetdry (the step's face revision, either) and
 * precision (DG2_FP64 or DG2_FP32) are used; variant must be DG2_NL, flux
 * DG2_HLL and scheme DG2_SCHEME_DG2 (DG2_E_ARG otherwise).  Workspace and
 * stream as for dg2_init_grid (dg2_adj_workspace_bytes serves both precisions). */
int dg2_adj_create(dg2_adj **out, int nx, int ny, double dx, double dy, const dg2_params *params,
                   int nsnap, int max_gauges, int max_steps, void *dev_workspace,
                   size_t ws_bytes, void *cuda_stream);

/* The problem: topography modes z3 (3 planes z0, z1x, z1y, as dg2_get_topo
 * returns), the initial state (9 planes, as dg2_get_state returns) at time
 * t0, the Manning n of every cell, the inflow segment (inflow_edge < 0: none;
 * segment [s0, s0 + len] along the edge, nknots increasing times and
 * discharges m^3/s) and ngauge gauge positions (x, y) in metres.  Host
 * arrays, copied.  DG2_E_ARG on a NULL required array, bad knots, an empty
 * segment or ngauge outside 0..max_gauges. */
int dg2_adj_set_problem(dg2_adj *adj, const double *z3, const double *state9, double t0,
                        const double *manning, int inflow_edge, double s0, double len,
                        const double *t_knots, const double *q_knots, int nknots,
                        const double *gauge_xy, int ngauge);

/* Replaces the parameters (either may be NULL): Manning n of every cell and
 * the knot discharges (same count as set). */
int dg2_adj_set_params(dg2_adj *adj, const double *manning, const double *q_knots);

/* Step sizes dts[nsteps] (> 0, nsteps <= max_steps), the step count after
 * which each of nsamples samples is taken (0..nsteps) and the observed depths
 * obs[nsamples][ngauge]. */
int dg2_adj_set_schedule(dg2_adj *adj, const double *dts, int nsteps, const int *sample_steps,
                         int nsamples, const double *obs);

/* Runs the forward steps: *loss = J; gauge_h (may be NULL) receives the
 * sampled depths [nsamples][ngauge]. */
int dg2_adj_forward(dg2_adj *adj, double *loss, double *gauge_h);

/* Forward and reverse sweeps: *loss = J, grad_manning[ny*nx] = dJ/dn,
 * grad_q[nknots] = dJ/dq (either may be NULL).  DG2_E_NONFINITE if J is not
 * finite. */
int dg2_adj_gradient(dg2_adj *adj, double *loss, double *grad_manning, double *grad_q);

/* Forward steps and reverse steps executed so far (checkpointing cost). */
int dg2_adj_counts(const dg2_adj *adj, int64_t *forward_steps, int64_t *reverse_steps);

int dg2_adj_destroy(dg2_adj *adj);

#ifdef __cplusplus
}
#endif
#endif /* DG2_H */
