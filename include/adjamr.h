/*
 * adjamr.h -- C ABI of the GB300 (sm_103a) implementation of the data-parallel
 * hot path of adjoint-guided block-structured AMR for linear hyperbolic
 * waves (Davis & LeVeque, "Adjoint methods for guiding adaptive mesh
 * refinement in wave propagation problems").
 *
 * Conventions for every call:
 *  - returns adjamr_status (0 = OK); adjamr_last_error(ctx) gives text;
 *    no C++ exception crosses this ABI;
 *  - input pointers are borrowed for the duration of the call only (the
 *    library copies what it keeps); output buffers are caller-allocated;
 *  - the context owns all device memory it allocates; adjoint snapshot sets
 *    are reference-counted handles that several contexts may share;
 *  - work is stream-ordered on the context's CUDA stream (a cudaStream_t
 *    passed as void*, NULL = the legacy default stream); calls that return
 *    host data synchronise that stream, the others do not;
 *  - one context must not be used by two host threads at the same time.
 *
 * Fields are FP64.  State layout seen through this ABI: per patch, field-
 * major, row-major interior cells: q[f][j][i] (1D: q[f][i]).
 * Field order: acoustics (p, u[, v]); shallow water (eta, mu, gamma).
 */
#ifndef ADJAMR_H
#define ADJAMR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADJAMR_MAX_LEVELS 8

typedef enum adjamr_status {
    ADJAMR_OK = 0,
    ADJAMR_EINVAL = 1,   /* invalid argument */
    ADJAMR_ENOMEM = 2,   /* device or host allocation failed */
    ADJAMR_EBUDGET = 3,  /* request does not fit the memory budget */
    ADJAMR_ECFL = 4,     /* Courant number exceeded cfl_max during the call */
    ADJAMR_ETIMEOUT = 5, /* a bounded device wait gave up */
    ADJAMR_ECUDA = 6,    /* a CUDA runtime call failed */
    ADJAMR_ESTATE = 7,   /* call not valid in the current state */
    ADJAMR_ENEST = 8     /* hierarchy not properly nested (internal invariant) */
} adjamr_status;

/* Systems (Sec. 2 Eq. eq:qtAqx; Sec. 5.1-5.3 matrices; adjoints Sec. 2 Eq.
 * adjoint1, time-reversed as in Sec. 4). */
enum {
    ADJAMR_ACOUSTICS = 0,          /* q_t + A q_x (+ B q_y) = 0, wave form */
    ADJAMR_ACOUSTICS_ADJOINT = 1,  /* q~_t - (A^T q~)_x (- (B^T q~)_y) = 0, f-wave */
    ADJAMR_SW = 2,                 /* linearised shallow water, f-wave with bathymetry */
    ADJAMR_SW_ADJOINT = 3          /* its adjoint, f-wave */
};

/* Physical boundary conditions (Sec. 5.1-5.2 walls; Sec. 5.2.3 outflow). */
enum { ADJAMR_BC_EXTRAP = 0, ADJAMR_BC_WALL = 1, ADJAMR_BC_PERIODIC = 2 };

/* Flag test.  Adjoint flagging (Sec. 4), with the time combination of the
 * adjoint snapshots (both bracketing snapshots count): maximum over the bracketing
 * snapshots, or q^ linear in time between snapshots.  The standard flaggers
 * the paper compares against: DIFFERENCE flags a cell when the undivided
 * centred difference |q_f(i+1) - q_f(i-1)| of some component in some
 * direction exceeds tol (Sec. 5.2.4, "pressure-flagging"; neighbours from the
 * level's ghost cells at the current time); SURFACE when |q_0| exceeds tol
 * (Sec. 5.3, "surface-flagging").  The standard flaggers need no adjoint.
 * ERROR (Sec. 7, the refinement the paper proposes as future work: the
 * forward solution's error estimated by Richardson extrapolation, its effect
 * on J by the adjoint) flags a cell when the maximum over the bracketing
 * snapshots of |q^ . tau| exceeds tol, tau being the cell's estimate of one
 * step's local error (adjamr_error_estimate).  It needs the adjoint, and it
 * nests refined levels ceil(4/r) + 1 cells of the coarser level deep (3 for
 * r = 2, 3) instead of 2, so that the estimate's ring stays on that level.
 * RICHARDSON is the standard flagger of that estimate (Sec. 1, AMRClaw's
 * Richardson error estimation): flag when the largest component of |tau|
 * exceeds tol, wherever that is; it needs no adjoint and nests as ERROR does. */
enum {
    ADJAMR_FLAG_BRACKET_MAX = 0,
    ADJAMR_FLAG_LINEAR = 1,
    ADJAMR_FLAG_DIFFERENCE = 2,
    ADJAMR_FLAG_SURFACE = 3,
    ADJAMR_FLAG_ERROR = 4,
    ADJAMR_FLAG_RICHARDSON = 5
};

enum { ADJAMR_MEDIUM_LAYERED = 1, ADJAMR_MEDIUM_DENSE = 2 };

/* Step launch modes: one launch per level over the whole tile work-list
 * (the default), a persistent grid of (#SMs x occupancy) CTAs striding over
 * the work-list, one launch per patch (the comparison baseline), or a
 * persistent grid whose CTAs take the next tile from an atomic counter
 * (dynamic balancing).  SUBSTEPS, on the finest level of a 2D hierarchy with
 * 8x8, 16x8, 16x12 or 16x16 kernel tiles: all r substeps of one coarser step in one
 * launch, each tile starting a substep as soon as the tiles its halo reads
 * have finished the previous one (ghost ring computed in the kernel); on any
 * other level it acts as DYNAMIC.  Every mode computes the same bits. */
enum {
    ADJAMR_LAUNCH_WORKLIST = 0,
    ADJAMR_LAUNCH_PERSISTENT = 1,
    ADJAMR_LAUNCH_PER_PATCH = 2,
    ADJAMR_LAUNCH_DYNAMIC = 3,
    ADJAMR_LAUNCH_SUBSTEPS = 4
};

/* Initial condition callback: fills q_out[f*n + k] for the n cell centres
 * (xc[k], yc[k]) of level `level` (yc = 0 in 1D).  Called on the host by
 * adjamr_init_grid_hierarchy and by an initial regrid. */
typedef void (*adjamr_qinit_fn)(int level, int n, const double *xc, const double *yc, double *q_out,
                                void *user);

/* Run parameters (Sec. 3: levels, ratios, regridding; Sec. 4/5: flagging
 * tolerance and time range of interest [ts, tf]). */
typedef struct adjamr_params {
    int dim;                     /* 1 or 2 */
    int eqn;                     /* ADJAMR_ACOUSTICS .. ADJAMR_SW_ADJOINT */
    double lo[2], hi[2];         /* domain [lo, hi] (y ignored in 1D) */
    int n0[2];                   /* level-0 cells per direction */
    int nlevels;                 /* 1 .. ADJAMR_MAX_LEVELS */
    int ratio[ADJAMR_MAX_LEVELS];/* ratio[l]: refinement from level l to l+1, space and time (2..16) */
    int bc[4];                   /* x-lo, x-hi, y-lo, y-hi */
    double cfl;                  /* desired Courant number: sets dt_0 */
    double cfl_max;              /* ADJAMR_ECFL if exceeded */
    double cmax;                 /* maximum wave speed of the medium */
    double dt0;                  /* > 0: use this level-0 step instead of the CFL rule */
    double t0, tf, ts;           /* start, final time, start of the time range of interest */
    double tol;                  /* flag tolerance: flag iff max |q^ . q| > tol (ERROR: max |q^ . tau| > tol;
                                    RICHARDSON: max_f |tau_f| > tol) */
    int regrid_interval;         /* regrid finer levels every k steps of a level (0 = never) */
    int buffer;                  /* flag buffer width (cells) */
    double cluster_eff;          /* Berger-Rigoutsos efficiency cut-off */
    int min_patch, max_patch;    /* patch edge range on refined levels (cells of that level) */
    int max_patch0;              /* level-0 tile edge */
    int flag_mode;               /* ADJAMR_FLAG_* */
    adjamr_qinit_fn qinit;       /* may be NULL (state starts at zero) */
    void *qinit_user;
    void *stream;                /* cudaStream_t or NULL */
    int tile_x, tile_y;          /* step-kernel tile size (0 = default 16 x 12; see adjamr_set_level_kernel) */
    int launch_mode;             /* ADJAMR_LAUNCH_* */
    int reflux;                  /* 1: conservation fix-up at coarse-fine interfaces (Sec. 3, AMR after
                                    Berger and LeVeque): after the fine substeps and the average-down,
                                    every uncovered coarse cell beside a fine patch is corrected so that
                                    it receives, through that side, the mean over the substeps and fine
                                    edges of (A-dQ + A+dQ of the Riemann problem between it and the fine
                                    cell) minus what the fine cell received there, in place of what the
                                    coarse step gave it; 0: off (the default) */
} adjamr_params;

/* Medium (Sec. 5.1/5.2 piecewise-constant layers; Sec. 5.3 bathymetry).
 * LAYERED (acoustics): layer k holds cells whose centre coordinate along
 *   `axis` (0 = x, 1 = y) satisfies iface[k-1] <= c < iface[k]; f0 = rho,
 *   f1 = K per layer.
 * DENSE: dense[l] points to [nmed][M_l][N_l] doubles covering level l's whole
 *   index space (acoustics nmed = 2: rho, K; shallow water nmed = 1: hbar).
 * Ghost cells outside the domain take the medium of the boundary-mapped
 * cell. */
typedef struct adjamr_medium {
    int kind;
    int axis, nlayers;
    const double *iface, *f0, *f1;
    const double *const *dense;
    int ndense;
} adjamr_medium;

/* phi = weight * indicator([x0,x1] x [y0,y1]) on field 0 (Sec. 2 Eq.
 * eq:J_general; Sec. 5.1 Eq. eq:phi_1d / Sec. 5.2 Eq. eq:phi_2d). */
typedef struct adjamr_target { double x0, x1, y0, y1, weight; } adjamr_target;

typedef struct adjamr_patch { int level, ilo, jlo, nx, ny; } adjamr_patch;

/* Counters since creation (cell-updates count interior cells advanced one
 * step on their level). */
typedef struct adjamr_stats {
    long long cell_updates;
    long long adjoint_cell_updates;
    long long kernel_launches;
    long long regrids;
    double cfl_max_seen;
    double step_kernel_ms;       /* CUDA-event time of the step kernels alone, if timing enabled */
    long long step_kernel_launches;
    double regrid_host_ms;       /* host wall time inside regrids (includes their synchronisations) */
    double cluster_host_ms;      /* of which: buffering, nesting and Berger-Rigoutsos on the host */
    long long level_rebuilds;    /* levels rebuilt by regrids */
    /* host wall time by regrid phase: [0] flag kernel + count/box readback (waits for queued work),
     * [1] flag-window copy, [2] clustering, [3] arena allocation and descriptor upload,
     * [4] builder kernels (medium, init, ghost and average-down maps), [5] release of the old arena */
    double regrid_phase_ms[6];
    /* per level: CUDA-event time of its step kernels (if timing enabled),
     * their launches, and the cell updates they made */
    double level_step_ms[ADJAMR_MAX_LEVELS];
    long long level_step_launches[ADJAMR_MAX_LEVELS];
    long long level_cell_updates[ADJAMR_MAX_LEVELS];
    /* host wall time inside clustering (regrid_phase_ms[2]): [0] buffer
     * dilation and nesting mask, [1] integral images, [2] Berger-Rigoutsos
     * bisection, [3] splitting to the maximum patch size and ordering */
    double cluster_phase_ms[4];
    /* per level: CUDA-event time of its ghost work outside the step kernels
     * (the separate ghost fill and the coarse stencil values), if timing
     * enabled; level_step_ms counts the step kernels alone */
    double level_ghost_ms[ADJAMR_MAX_LEVELS];
    /* regrids that found a level's new boxes equal to its current ones over an
     * unchanged coarser level (an empty level staying empty included) and kept
     * it as it was: the rebuild would have reproduced it bit for bit */
    long long level_rebuilds_skipped;
} adjamr_stats;

typedef struct adjamr_ctx adjamr_ctx;
typedef struct adjamr_adjoint adjamr_adjoint;

/* Create a hierarchy (Sec. 3: block-structured nested levels carrying the
 * linear system of Sec. 2): level 0 tiles the domain with near-equal patches of at
 * most max_patch0 cells per side; its state is sampled from p->qinit at cell
 * centres.  Finer levels are created by adjamr_regrid.  Errors: EINVAL for
 * inconsistent parameters, ENOMEM, ECUDA. */
adjamr_status adjamr_init_grid_hierarchy(const adjamr_params *p, adjamr_ctx **out);

/* Set the medium (Secs. 5.1-5.3: layered rho, K; bathymetry hbar); copies the
 * layer table or the dense per-level arrays to
 * the device and fills the per-cell coefficients of existing patches
 * (impedance, sound speed, edge coefficients).  Must precede stepping. */
adjamr_status adjamr_set_medium(adjamr_ctx *ctx, const adjamr_medium *m);

/* Adjoint snapshots (Sec. 4): snaps[nsnap][m][ay][ax] in FORWARD time order,
 * snapshot n at t_n = t0 + n (tf - t0)/(nsnap - 1), on a uniform ax x ay grid
 * covering the domain; wet[ay][ax] (NULL = all wet).  snaps_on_device != 0:
 * `snaps` is a device pointer (copied device-to-device).  The returned
 * handle holds a device copy and one reference; it is attached to ctx.
 * When the set ctx holds has the same shape and nothing else holds it, its
 * device buffers take the new values (after ctx's queued work; the returned
 * handle is then that set) instead of a new allocation.  Errors: EINVAL for
 * bad sizes, ENOMEM, ECUDA (a failed refill detaches the set from ctx). */
adjamr_status adjamr_load_adjoint_snapshots(adjamr_ctx *ctx, const double *snaps, int nsnap, int ax, int ay,
                                            const unsigned char *wet, int snaps_on_device,
                                            adjamr_adjoint **out);

/* Solve the adjoint (eqn = adjoint system) on the grid described by ap from
 * q~(x, 0) = phi (host [m][ay][ax] on the level-0 grid of ap) and store
 * nsnap snapshots of that grid on the device (Sec. 4: q^(x, tf - t_n) =
 * q~(x, t_n)).  The level-0 step is dt = dT/ceil(dT/dt_cfl), dT = (tf -
 * t0)/(nsnap - 1).  ap->nlevels = 1: a fixed grid, as in the paper.
 * ap->nlevels > 1: the adjoint solved with AMR (Sec. 7 proposes it for a
 * more accurate inner product): finer levels by ap->ratio, flagged by the
 * standard flagger ap->flag_mode (DIFFERENCE, SURFACE or RICHARDSON; EINVAL otherwise)
 * at ap->tol and regridded every ap->regrid_interval steps as in a forward
 * run; their initial cells are interpolated from phi on level 0; each
 * level-0 step is a full Berger-Oliger step, so the snapshot is level 0
 * holding the composite solution averaged onto it.  The handle is attached
 * to ctx (ctx may be NULL: then it is only returned). */
adjamr_status adjamr_solve_adjoint(adjamr_ctx *ctx, const adjamr_params *ap, const adjamr_medium *am,
                                   const double *phi, int nsnap, adjamr_adjoint **out);

/* Attach a (shared) snapshot set (Sec. 4) to ctx; takes a reference. */
adjamr_status adjamr_set_adjoint(adjamr_ctx *ctx, adjamr_adjoint *adj);
/* Copy snapshots (Sec. 4) to the host: dst[nsnap][m][ay][ax]. */
adjamr_status adjamr_adjoint_read(adjamr_adjoint *adj, double *dst, size_t cap);
/* Drop one reference to a snapshot set (Sec. 4); frees the device copy with
 * the last one. */
void adjamr_adjoint_release(adjamr_adjoint *adj);

/* Start a new solve in the same context: finer levels dropped, every level
 * back at t0, level 0 re-sampled from qinit (zero without it), the CFL record,
 * the device error word, gauge records and statistics cleared; the layout of
 * level 0, the medium, the attached adjoint set, the gauges' points and the
 * per-level kernel choices stay.  A solve after a reset gives the bits of a
 * solve in a new context (tested); the context keeps its cached device blocks,
 * so repeated solves skip the allocations of a new context.  Synchronises.
 * (No counterpart in the paper: context reuse.) */
adjamr_status adjamr_reset(adjamr_ctx *ctx);

/* Rebuild levels base_level+1 .. nlevels-1 top-down (Sec. 3, regridding):
 * adjoint flags on level l, buffered, properly nested, clustered by
 * Berger-Rigoutsos, split to max_patch, refined; new cells copied from old
 * patches of the same level or interpolated from level l (init != 0: sampled
 * from qinit).  Synchronises the stream (flags are clustered on the host). */
adjamr_status adjamr_regrid(adjamr_ctx *ctx, int base_level, int init);

/* Advance the hierarchy by nsteps level-0 steps (Berger-Oliger recursion,
 * Sec. 3: coarse step, r fine steps with time-interpolated ghost cells,
 * average down; regrid every regrid_interval steps).  level must be 0 (EINVAL
 * otherwise): a finer level advances only inside a step of the coarser one,
 * whose old and new states its ghost cells interpolate between, so every
 * advance starts at level 0 and recurses below it.
 * Returns ECFL if the Courant number exceeded cfl_max. */
adjamr_status adjamr_advance_level(adjamr_ctx *ctx, int level, int nsteps);

/* Adjoint flags of the interior cells of `level` at its current time t for
 * the time range of interest [t_s, tf] (Sec. 4, Sec. 5.1.2: flag iff the
 * maximum of |q^(tau) . q| over tau in [t, min(t + tf - t_s, tf)] exceeds
 * tol; t_s = tf is a time point of interest): flags_out[k] in patch order,
 * row-major per patch (may be NULL); *nflag = number flagged.  The standard
 * flaggers (params.flag_mode DIFFERENCE / SURFACE) ignore t_s.  The regrids
 * of adjamr_advance_level use params.ts.  EINVAL unless t0 <= t_s <= tf.
 * Synchronises. */
adjamr_status adjamr_flag_cells(adjamr_ctx *ctx, int level, double tol, double t_s, unsigned char *flags_out,
                                long long *nflag);

/* J = sum over the composite grid of weight * q0 * |cell ∩ box| (Sec. 2 Eq.
 * eq:J_general), fixed pairwise summation order.  Synchronises. */
adjamr_status adjamr_integrate_functional(adjamr_ctx *ctx, const adjamr_target *phi, double *J_out);

/* Patch layout of a level (Sec. 3, regridding), sorted by (jlo, ilo).  *n = number of patches
 * (written even if cap is too small; then EINVAL). */
adjamr_status adjamr_get_patches(adjamr_ctx *ctx, int level, adjamr_patch *out, int cap, int *n);

/* Interior state of a level (Sec. 3), patch by patch (q[f][j][i] per patch).
 * cap in doubles.  Synchronises. */
adjamr_status adjamr_read_level(adjamr_ctx *ctx, int level, double *dst, size_t cap);
/* Overwrite the interior state of a level (Sec. 3; same layout). */
adjamr_status adjamr_write_level(adjamr_ctx *ctx, int level, const double *src, size_t count);

/* Richardson estimate tau of one step's local error on `level` at its current
 * time (Sec. 7, future work: the error estimate that adjoint-weighted flagging
 * would weigh; ADJAMR_FLAG_ERROR flags with it).  Every patch is extended to
 * even extents with a ring of 4 cells (filled as ghost cells are: the level's
 * own cells, else the coarse space-time interpolation, boundary-mapped),
 * advanced two steps of dt, and, coarsened by 2 in every direction (mean of
 * the children, medium included), one step of 2 dt;
 *   tau = (coarsened two-step state - coarse step) / 6
 * on every 2 x 2 (1D: 2) block, the local error of one step of a
 * second-order method being C dx^3 and that of the coarse step 8 C dx^3.
 * Layout as adjamr_read_level; cap in doubles.  A level above level 0 must be
 * nested as ADJAMR_FLAG_ERROR nests it (else ADJAMR_ENEST).  The step
 * counters and the CFL record are unchanged.  Synchronises. */
adjamr_status adjamr_error_estimate(adjamr_ctx *ctx, int level, double *dst, size_t cap);

/* Fill the ghost cells of `level` for its current time (Sec. 3: same-level
 * copies, boundary conditions, coarse space-time interpolation; as a step would). */
adjamr_status adjamr_fill_ghosts(adjamr_ctx *ctx, int level);

/* Ghosted storage of patch k of `level` (Sec. 3): q[m][sy][sx] with sx = nx + 4,
 * sy = ny + 4 (1D: 1); med[nmed][sy][sx] = primary medium (rho, K | hbar). */
adjamr_status adjamr_read_patch_ghosted(adjamr_ctx *ctx, int level, int k, double *q, double *med);

/* Step every patch of `level` once (the Sec. 3 wave-propagation step),
 * without recursion, regrid or ghost fill (for sampled parity checks). */
adjamr_status adjamr_step_level_only(adjamr_ctx *ctx, int level);

/* Counters and timings of the context (no counterpart in the paper:
 * measurement). */
adjamr_status adjamr_get_stats(adjamr_ctx *ctx, adjamr_stats *out);
/* Enable/disable CUDA-event timing of step kernels (adds events only; no
 * counterpart in the paper: measurement). */
adjamr_status adjamr_set_timing(adjamr_ctx *ctx, int enable);
/* Step-kernel configuration of one level (level = -1: every level), used
 * from the next step on: the tile size the level's patches are cut to
 * (near-equal tiles of at most tile_x x tile_y cells; the kernel compiled for
 * the smallest of 8x8, 16x8, 16x12, 32x8, 16x16, 64x8, 32x16 that holds them runs
 * them; 1D: tile_x <= 256, tile_y ignored), whether the kernel computes the
 * level's ghost ring (same-level copies and coarse space-time interpolation,
 * Sec. 3) while staging its tiles (fuse_ghosts = 1, the default) or a
 * separate ghost-fill kernel runs before it (0), and the launch mode
 * (ADJAMR_LAUNCH_*; -1 keeps the level's current one).  Every choice
 * computes the same bits; it changes only speed (tile counts near whole
 * waves of resident CTAs, and small tiles on small levels, fill the GPU
 * better).  Errors: EINVAL for a tile no compiled kernel holds, or a bad mode
 * or level. */
adjamr_status adjamr_set_level_kernel(adjamr_ctx *ctx, int level, int tile_x, int tile_y, int fuse_ghosts,
                                      int launch_mode);
/* Check of the bounded waits of ADJAMR_LAUNCH_SUBSTEPS (no counterpart in
 * the paper: the failure path of this GPU launch mode): one substep launch
 * (2 substeps) of the finest level in which every tile's second substep
 * waits on a completion counter that nothing advances.  The waits give up
 * after about 1 s; the call returns ADJAMR_ETIMEOUT and the elapsed device
 * time in *wait_ms, and clears the failure, so the context stays usable.  The
 * level's current state (q[cur]) is not changed.  ESTATE when the finest
 * level cannot run substep launches or has no patches. */
adjamr_status adjamr_substep_wait_selftest(adjamr_ctx *ctx, double *wait_ms);
/* Gauges (time series at points, Sec. 5.2.4 and Sec. 5.3): n points (x[k],
 * y[k]; y is ignored in 1D) recorded on the device after every level-0 step
 * of adjamr_advance_level: the level-0 time, then the m values of the cell
 * holding the point (index floor((x - lo)/dx), clamped to the level) on the
 * finest level with a patch there.  Replaces earlier gauges and drops their
 * records.  Errors: EINVAL (n < 0, or null points with n > 0), ENOMEM. */
adjamr_status adjamr_set_gauges(adjamr_ctx *ctx, int n, const double *x, const double *y);
/* Gauge records so far (Sec. 5.2.4, Sec. 5.3): out[r][k][1 + m] for r < min(*nrec, cap) (out may be
 * null with cap = 0); *nrec = number of records held.  Synchronises the
 * context's stream. */
adjamr_status adjamr_read_gauges(adjamr_ctx *ctx, double *out, long long cap, long long *nrec);
/* Berger-Rigoutsos clustering (Sec. 3, regridding) as the regrid runs it, on
 * the host: flags[M][N] (0/1; the regrid clears flags where no patch may lie
 * before it clusters) and nestable[M][N] (nonzero where a patch may cover the
 * cell: a box over another cell is split; NULL: everywhere) in, boxes out as
 * (i0, i1, j0, j1)
 * inclusive, sorted by (j0, i0), for at most cap boxes; *nboxes = the number
 * of boxes (more than cap: only cap written).  min_cells = smallest side a
 * split may leave, efficiency = flagged fraction a box must reach.  No GPU is
 * involved.  Errors: EINVAL. */
adjamr_status adjamr_cluster_boxes(const unsigned char *flags, const unsigned char *nestable, int N, int M, int dim,
                                   int min_cells, double efficiency, int *boxes, int cap, int *nboxes);
/* Level-0 step and number of level-0 steps to reach tf (Sec. 3: the levels'
 * steps are dt0 / (r_0 ... r_{l-1})). */
adjamr_status adjamr_time_info(adjamr_ctx *ctx, double *dt0, int *nsteps_to_tf);
/* Text of the context's last error (no counterpart in the paper). */
const char *adjamr_last_error(adjamr_ctx *ctx);
/* Free the context and its device memory; drops its snapshot-set reference
 * (no counterpart in the paper). */
void adjamr_destroy(adjamr_ctx *ctx);

/* Measurement utility (no counterpart in the paper): FP64 instruction
 * throughput of this GPU, kind 0 = DFMA (2 flops), 1 = DADD, 2 = DMUL, from
 * 8 independent chains per thread over 8 CTAs of 256 threads per SM,
 * `iters` iterations, timed with CUDA events on the legacy stream.  Writes
 * flop/s and the timed kernel's milliseconds. */
adjamr_status adjamr_fp64_peak(int kind, int iters, double *flops_per_s, double *ms);

/* ------------------------------------------------------------------ */
/* Batched independent patches (uneven sizes, mixed levels): every patch is */
/* its own domain with extrapolation ghosts; one step advances all of them  */
/* with their own dt.  Used for the fused-vs-per-patch comparison.          */
/* ------------------------------------------------------------------ */
typedef struct adjamr_batch adjamr_batch;

/* (No counterpart in the paper: batching; every patch advances by the Sec. 3
 * step.)  npatch patches, 2D acoustics: patch k covers [x0[k], x1[k]] x [y0[k], y1[k]]
 * with nx[k] x ny[k] cells (dx = (x1 - x0)/nx as on a level) and steps with
 * dt[k]; medium_id[k] indexes `media` (LAYERED only); q0 = interiors
 * concatenated in patch order (q[3][ny][nx] each). */
adjamr_status adjamr_batch_create(int npatch, const int *nx, const int *ny, const double *x0, const double *y0,
                                  const double *x1, const double *y1, const double *dt, const int *medium_id,
                                  const adjamr_medium *media, int nmedia, const double *q0, void *stream,
                                  adjamr_batch **out);
/* Order of the tile work-list: patch order given here (a permutation; no
 * counterpart in the paper). */
adjamr_status adjamr_batch_set_order(adjamr_batch *b, const int *order);
/* (No counterpart in the paper.)  Ghost ring of the batch's patches computed inside the step kernel while
 * it stages its tiles (1) or by a separate ghost-fill kernel launched before
 * it (0, the default).  Same bits either way. */
adjamr_status adjamr_batch_set_ghost_fusion(adjamr_batch *b, int fuse_ghosts);
/* Advance all patches nsteps steps of Sec. 3 with the given launch mode and
 * tile size (as in adjamr_set_level_kernel). */
adjamr_status adjamr_batch_step(adjamr_batch *b, int nsteps, int launch_mode, int tile_x, int tile_y);
/* Capture one step (ghost fill + fused step of Sec. 3) in a CUDA graph and
 * replay it nsteps times. */
adjamr_status adjamr_batch_step_graph(adjamr_batch *b, int nsteps, int launch_mode, int tile_x, int tile_y);
/* Interiors of all patches, concatenated as q0 was (no counterpart in the paper). */
adjamr_status adjamr_batch_read(adjamr_batch *b, double *dst, size_t cap);
/* Interior cells of the batch (no counterpart in the paper). */
adjamr_status adjamr_batch_cells(adjamr_batch *b, long long *cells);
/* Free the batch (no counterpart in the paper). */
void adjamr_batch_destroy(adjamr_batch *b);

/* ------------------------------------------------------------------ */
/* Weighted sum without device allocation.                                 */
/* ------------------------------------------------------------------ */
/* No counterpart in the paper: this is a service for callers that cannot
 * allocate device memory at the point where they need J-type sums -- for
 * instance code running while its stream is being captured into a CUDA
 * graph (an allocation there would break or serialise the capture), a
 * solver loop with a fixed memory plan whose device memory all belongs to
 * another framework's pool, or a latency-critical path that must never
 * reach the allocator.
 *
 * *out = pairwise sum over k < n of weight*(q[k]*w[k]) -- the same terms and
 * the same fixed pairwise tree as adjamr_integrate_functional (pairs (2i,
 * 2i+1), an odd tail carried up), so the result equals that entry point's J
 * for the same terms.  q, w: device arrays of n doubles; out: device pointer
 * to one double; stream: cudaStream_t (NULL = legacy default stream).
 * Stream-ordered, does not synchronise.
 *
 * Allocates nothing: its scratch is a static device array of
 * ADJAMR_NOALLOC_MAX_TERMS doubles (8 MiB) that every GPU loading the
 * library holds until the process exits.  n > ADJAMR_NOALLOC_MAX_TERMS is
 * rejected with ADJAMR_EBUDGET before any work is issued.  Every call whose
 * stream is not being captured looks up the array's device address on the
 * current device (cudaGetSymbolAddress), so a device reset in between does
 * no harm; a call made during a stream capture uses the address found by the
 * last such call on that device: make the first call on a device before any
 * stream capture (otherwise ADJAMR_ESTATE, with nothing issued).  All calls share
 * the one array, so calls whose work overlaps on the GPU (different streams,
 * no ordering between them) race and give wrong results; calls ordered on
 * one stream are safe.  Nothing in the array needs clearing: each call writes
 * every entry it reads before reading it. */
#define ADJAMR_NOALLOC_MAX_TERMS (1 << 20)
adjamr_status adjamr_weighted_sum_noalloc(const double *q, const double *w, long long n, double weight, double *out,
                                          void *stream);

/* ------------------------------------------------------------------ */
/* Serving: many forward solves against shared device-resident adjoint     */
/* snapshot sets.  Requests are admitted in arrival order as soon as a     */
/* slot is free and their projected device memory fits the budget; every   */
/* slot runs on its own CUDA stream so admitted requests overlap on the    */
/* device.  A request's result does not depend on the other requests.      */
/* ------------------------------------------------------------------ */
typedef struct adjamr_server adjamr_server;

typedef struct adjamr_request {
    adjamr_params params;      /* params.stream is ignored (the slot's stream is used) */
    adjamr_medium medium;      /* LAYERED; the layer table is copied at submit */
    adjamr_adjoint *adjoint;   /* shared snapshot set; a reference is held until done */
    adjamr_target target;      /* J is computed at tf */
} adjamr_request;

typedef struct adjamr_result {
    int done;
    adjamr_status status;
    double J;
    long long cell_updates, kernel_launches;
    double t_submit, t_admit, t_finish;  /* seconds on the server's steady clock */
    size_t bytes_reserved;
    char error[128];
} adjamr_result;

/* (No counterpart in the paper: serving, as every serving call below.)
 * Projected device bytes of one solve (upper bound: every level fully
 * refined), used for admission.  0 for parameters no hierarchy accepts
 * (nlevels outside 1 .. ADJAMR_MAX_LEVELS, a refinement ratio outside
 * 2 .. 16); adjamr_server_submit refuses those requests with EINVAL. */
size_t adjamr_estimate_bytes(const adjamr_params *p);
/* Serving (no counterpart in the paper): max_slots worker threads on the
 * current device; budget in bytes. */
adjamr_status adjamr_server_create(size_t budget_bytes, int max_slots, adjamr_server **out);
/* Queue a request (serving; no counterpart in the paper); EBUDGET if it can never fit the budget, EINVAL if its
 * parameters are refused (adjamr_estimate_bytes gives 0). */
adjamr_status adjamr_server_submit(adjamr_server *srv, const adjamr_request *rq, long long *ticket);
/* Non-blocking status of a ticket (res.done = 0 while queued or running;
 * serving, no counterpart in the paper). */
adjamr_status adjamr_server_poll(adjamr_server *srv, long long ticket, adjamr_result *out);
/* Block until the ticket is done (serving, no counterpart in the paper). */
adjamr_status adjamr_server_wait(adjamr_server *srv, long long ticket, adjamr_result *out);
/* Reserved bytes, running and queued requests (serving, no counterpart in
 * the paper). */
adjamr_status adjamr_server_info(adjamr_server *srv, size_t *used_bytes, int *active, int *queued);
/* Seconds since the server was created: the clock of the results' times
 * (serving, no counterpart in the paper). */
double adjamr_server_now(adjamr_server *srv);
/* Stops the workers after the running requests finish; queued requests are
 * dropped (status ESTATE; serving, no counterpart in the paper). */
void adjamr_server_destroy(adjamr_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* ADJAMR_H */
