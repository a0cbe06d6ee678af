/*
 * icarus.h - C ABI of libicarus, a GB300 (sm_103a) implementation of the
 * explicit finite-volume update of the Icarus heliospheric MHD model
 * (arXiv 2211.12867): ideal MHD in the frame co-rotating with the Sun on a
 * block-structured spherical (r, theta, phi) grid with radial stretching and
 * solution-adaptive mesh refinement.
 *
 * Method passages (paper section / equation / table):
 *   Sect. 2.1  ideal MHD in the co-rotating frame; TVDLF scheme, second order
 *              in space and time, Woodward limiter, parabolic div B
 *              cleaning; domain 0.1-2 AU, +-60 deg, 360 deg; two ghost
 *              layers; inner boundary fixed in the rotating frame.
 *   Eqs. 1-4   cone CME injected through the inner boundary.
 *   Sect. 2.2, Eq. 5, Tables 1 and 3   radial grid stretching.
 *   Sect. 3    block AMR: factor 2 per level in every direction, adjacent
 *              blocks differ by at most one level, blocks coarsen again when
 *              the criterion fails.
 *
 * Units.  Everything crossing this ABI is in normalised units: length 1 AU,
 * speed 100 km/s, density m_p per cm^3, pressure rho0 v0^2, magnetic field
 * sqrt(mu0 rho0 v0^2) (mu0 absorbed), time 1 AU / (100 km/s).  Angles are
 * radians; theta is the colatitude.
 *
 * Variables.  Conserved U = (rho, m_r, m_th, m_ph, e, B_r, B_th, B_ph);
 * primitive W = (rho, v_r, v_th, v_ph, p, B_r, B_th, B_ph); vector components
 * in the local orthonormal basis.
 *
 * Host state layout.  State arrays exchanged with the host are FP64,
 * [leaf][variable][i][j][k] over the interior cells of each leaf block, leaves
 * of one member in Morton order (see icarus_get_tree), i = r index (slowest),
 * k = phi index (fastest).
 *
 * Ownership.  The caller owns the device arena and the CUDA stream; the
 * library allocates no device memory and keeps only small host-side
 * bookkeeping behind the context.  Calls are asynchronous on the stream except
 * those that return host data, which synchronise the stream.
 *
 * Errors.  Every call returns a status; nothing throws or exits.  Device
 * kernels record non-physical states (NaN, density or pressure below the
 * floors beyond the floor budget) in a sticky device word that is read at
 * synchronising calls.  After ICARUS_ERR_NONPHYSICAL or ICARUS_ERR_TIMEOUT the
 * context accepts only icarus_get_state, icarus_status_word and
 * icarus_destroy.  One host thread per context; no internal locking.
 */
#ifndef ICARUS_H
#define ICARUS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct icarus_ctx icarus_ctx;

typedef enum {
  ICARUS_OK = 0,
  ICARUS_ERR_ARG = 1,          /* invalid argument or descriptor */
  ICARUS_ERR_ARENA = 2,        /* caller arena too small / misaligned */
  ICARUS_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  ICARUS_ERR_NONPHYSICAL = 4,  /* NaN or floor budget exceeded on the device */
  ICARUS_ERR_TIMEOUT = 5,      /* a bounded device wait gave up */
  ICARUS_ERR_STATE = 6,        /* call out of order / context poisoned */
  ICARUS_ERR_CAPACITY = 7      /* block pool too small for the refined tree */
} icarus_status;

enum { ICARUS_FP64 = 0, ICARUS_FP32_MIXED = 1 };
enum { ICARUS_SPHERICAL = 0, ICARUS_CARTESIAN = 1 };
enum { ICARUS_BC_PERIODIC = 0, ICARUS_BC_OUTFLOW = 1, ICARUS_BC_REFLECT = 2, ICARUS_BC_INNER = 3 };
enum {
  ICARUS_FLAG_PLAIN = 0,
  ICARUS_FLAG_LEARNED = 1,
  ICARUS_FLAG_BOTH = 2,
  ICARUS_FLAG_SHOCK = 3,
  ICARUS_FLAG_TRACER = 4,
  ICARUS_FLAG_COMBINED = 5
};

/* Grid descriptor.
 *   n_cells      base-level cells (r, theta, phi); must be multiples of block.
 *   block        interior cells per block and direction, even, 4 .. 1020.
 *   max_level    finest level (1 = no refinement); per member, see
 *                icarus_set_member_max_level.  At most 8.
 *   radial_stretch  1: geometric radial faces r_I = r_in (r_out/r_in)^(I/N)
 *                (Sect. 2.2); 0: equidistant.
 *   geometry     ICARUS_SPHERICAL or ICARUS_CARTESIAN (test problems).
 *   x_min/x_max  r [AU], colatitude, longitude (x, y, z in Cartesian mode).
 *   gamma, omega (rotation rate, normalised), cfl, divb_cd (cleaning
 *                coefficient, 0 disables), p_floor, rho_floor.
 *   precision    ICARUS_FP64 or ICARUS_FP32_MIXED (FP32 state and stencil,
 *                FP64 pressure recovery in low-beta / thermally poor cells,
 *                FP64 time-step reduction and conservation sums).
 *   n_members    independent ensemble members sharing the grid geometry.
 *   bc_lo/bc_hi  boundary kind per direction (ICARUS_BC_*); periodic must be
 *                set on both sides; ICARUS_BC_INNER only at r low.
 *   max_blocks   capacity of the block pool (all members); 0 = base blocks.
 *   arena        caller-owned device memory, 256-byte aligned.
 *   stream       cudaStream_t (NULL = legacy default stream).
 *   tracer       1: store and advect the CME density tracer rho X (Sect. 3.1;
 *                see icarus_get_tracer), one more variable per cell; 0: none. */
typedef struct {
  int n_cells[3];
  int block[3];
  int max_level;
  int radial_stretch;
  int geometry;
  double x_min[3], x_max[3];
  double gamma, omega, cfl, divb_cd;
  double p_floor, rho_floor;
  int precision;
  int n_members;
  int bc_lo[3], bc_hi[3];
  int max_blocks;
  void *arena;
  size_t arena_bytes;
  void *stream;
  int tracer;
} icarus_grid_desc;

/* Cone CME (Eqs. 1-4): injected while t_start <= t <= t_start + t_max and the
 * CME sphere still crosses the inner boundary.  colat/lon: launch direction in
 * the co-rotating frame; half_width = omega_CME / 2; v = injection speed; rho,
 * p: CME plasma (B = 0, radial flow). */
typedef struct {
  double t_start, t_max, colat, lon, half_width, v, rho, p;
} icarus_cone;

/* Refinement criterion.
 * ICARUS_FLAG_PLAIN: Loehner second-derivative estimator E of density and
 * pressure (diagonal form, index space, noise parameter eps).  A block is
 * flagged +1 (refine) if some interior cell has E > e_refine and
 * v_r > v_r,background + dv; -1 (coarsen) if no cell has E > e_coarsen with
 * that gate; 0 otherwise.  _LEARNED: the plain flags, set to +1 where the
 * MLP pre-flagger's probability exceeds 1/2 on a block below its member's
 * finest level.  _BOTH: both computed, plain flags returned.
 * ICARUS_FLAG_SHOCK (Sect. 3.2): a cell counts where the velocity divergence
 * (central differences at cell centres, spherical form) is below -div_thr
 * (the paper's criterion is div_thr = 0) and its centre lies within
 * dlon_earth of Earth's longitude, within dcolat_earth of Earth's colatitude
 * (see icarus_set_earth) and within dlon_cme of the member's CME longitude
 * (the paper: 30, 10 and 90 degrees; a half width <= 0 switches that window
 * off).  A block is flagged +1 if some interior cell counts, -1 (coarsen:
 * the criterion no longer holds) otherwise.  Evaluated in FP64 with
 * explicitly rounded operations.  ICARUS_ERR_ARG for div_thr < 0 or a half
 * width >= pi.
 * ICARUS_FLAG_TRACER (Sect. 3.1; needs a descriptor with tracer = 1): a cell
 * counts where its CME tracer fraction X = (rho X) / rho exceeds x_thr (the
 * paper refines where X is non-zero: x_thr = 0), inside the same windows
 * (the paper applies none here: set the half widths to 0).
 * ICARUS_FLAG_COMBINED (Sect. 3.3): a cell counts where X > x_thr or the
 * velocity divergence is below -div_thr, inside the windows.  Both: +1 if
 * some interior cell counts, -1 otherwise; ICARUS_ERR_STATE without tracer.
 * The fields after mode are read in these three modes only. */
typedef struct {
  double e_refine, e_coarsen, eps, dv;
  int mode;
  double div_thr, dlon_earth, dcolat_earth, dlon_cme;
  double x_thr;
} icarus_refine;

/* Bytes of device arena that icarus_init_grid needs for this descriptor
 * (arena/arena_bytes/stream fields are ignored). */
icarus_status icarus_arena_bytes(const icarus_grid_desc *desc, size_t *bytes);

/* Create a context on the caller's arena and stream: geometry tables for all
 * levels, base-level blocks for every member, state zeroed.  *out receives
 * the context (free with icarus_destroy).
 * Passages: Sect. 2.1 (domain 0.1-2 AU, +-60 deg latitude, 360 deg longitude,
 * two ghost layers at the boundaries); Sect. 2.2 and Eq. 5 (radial stretching:
 * a cell's radial width grows in proportion to its radius, so the faces are
 * geometric); Tables 1 and 3 (resolutions per level); Sect. 3 (every level
 * halves the cells in all three directions).
 * Errors: ICARUS_ERR_ARG for an inconsistent descriptor, ICARUS_ERR_ARENA if
 * arena_bytes is below icarus_arena_bytes or the arena is not 256-byte
 * aligned, ICARUS_ERR_CUDA if a CUDA call fails; *out is then NULL. */
icarus_status icarus_init_grid(const icarus_grid_desc *desc, icarus_ctx **out);

/* Inner-boundary primitive map of one member (Sect. 2.1: boundary values
 * constant in time in the co-rotating frame, two ghost layers): host FP64
 * [8][n_theta][n_phi] at the base-level angular cells, copied (the caller
 * keeps its array).  Both inner ghost layers of every level take the value of
 * the containing base cell (not rescaled in r).  ICARUS_ERR_ARG for a bad
 * member or a NULL map. */
icarus_status icarus_set_inner_boundary(icarus_ctx *ctx, int member, const double *prim);

/* Start a cone CME on one member (Sect. 2.1, Eqs. 1-4: the cone's
 * cross-section with the inner boundary grows and shrinks as the CME sphere
 * passes through it) and record the member's background radial speed per
 * base cell from the current state (the gate of the refinement criterion).
 * cme (host) is copied.  All leaves of the member must be at level 1
 * (ICARUS_ERR_STATE otherwise). */
icarus_status icarus_inject_cone_cme(icarus_ctx *ctx, int member, const icarus_cone *cme);

/* Advance every member by up to n_steps steps of the midpoint
 * predictor-corrector (each step: ghost fill, half step, ghost fill, full
 * step with parabolic cleaning, reflux at coarse-fine faces, CFL time step).
 * Passage: Sect. 2.1 (ideal MHD in the co-rotating frame, TVDLF scheme second
 * order in space and time with the Woodward limiter, parabolic cleaning of
 * div B); the refinement levels of Sect. 3 advance with one shared time step.
 * t_stop[n_members] (host): a member's dt is clipped so that it lands on
 * t_stop, after which it stops.  When every t_stop is finite the call reads
 * the members' times back every 8 steps (synchronising) and returns early
 * once all have landed.  t_out[n_members] (host, may be NULL) receives the
 * members' times; passing it synchronises the stream.
 * Errors: the status word (NaN, floor budget, bounded wait) is checked at
 * every synchronisation of the call.  A call with t_out == NULL and infinite
 * stop times does not synchronise: it leaves a copy of the status word on
 * its way to the host, and the next icarus_step reports what it holds
 * (ICARUS_ERR_NONPHYSICAL or ICARUS_ERR_TIMEOUT) as soon as it has landed. */
icarus_status icarus_step(icarus_ctx *ctx, int n_steps, const double *t_stop, double *t_out);

/* Evaluate the refinement criterion on every leaf of every member (after a
 * ghost fill at the current time).  flags_out (host, optional): one int8 per
 * leaf in global leaf order (member-major, Morton within a member).
 * Passage: Sect. 3 (refine where the solution meets the criterion, coarsen
 * again once it no longer does); Sect. 3.2 for ICARUS_FLAG_SHOCK.  The flags
 * stay on the device for icarus_regrid.  Synchronises when flags_out is set. */
icarus_status icarus_flag_refine(icarus_ctx *ctx, const icarus_refine *crit, int8_t *flags_out);

/* Replace the current flags (host int8, global leaf order), e.g. to replay a
 * decision taken elsewhere. */
icarus_status icarus_set_flags(icarus_ctx *ctx, const int8_t *flags);

/* Apply the current flags: refine +1 leaves by one level, coarsen complete
 * sibling families all flagged -1 (refinement wins), enforce 2:1 balance over
 * faces, edges and corners (least balanced refinement), prolong new children
 * conservatively, restrict coarsened parents, renumber leaves in Morton order.
 * Passage: Sect. 3 (a refinement splits the cells in two in all three
 * directions; adjacent blocks differ by at most one level; blocks coarsen
 * when the criterion is no longer met).  ICARUS_ERR_STATE without flags.
 * Errors: ICARUS_ERR_CAPACITY if the new tree of all members needs more
 * blocks than max_blocks; the tree, the state and the flags are then left as
 * they were (the caller may retry at a later regrid). */
icarus_status icarus_regrid(icarus_ctx *ctx);

/* Sample primitives at n_pts points rtp[n_pts][3] (host: r, colat, lon) by
 * trilinear interpolation between cell centres of the finest leaf containing
 * each point; prim_out[n_pts][8] (host).  Points outside the domain give NaN.
 * Passage: Sect. 3.1-3.3 (time series of speed and density at Earth, from
 * which the shock arrival time, shock width and peak speed are read).
 * ICARUS_ERR_ARG for a bad member or n_pts < 0 or > 4096.  Synchronises. */
icarus_status icarus_probe(icarus_ctx *ctx, int member, int n_pts, const double *rtp, double *prim_out);

/* ---- helpers used by the harness and the parity tests ---- */

/* number of leaves of a member (member = -1: all members) */
icarus_status icarus_n_leaves(icarus_ctx *ctx, int member, int *n);

/* leaves of a member as rows (level, i, j, k), Morton order; host int32 [n][4] */
icarus_status icarus_get_tree(icarus_ctx *ctx, int member, int32_t *rows, int capacity, int *n);

/* Copy a member's state between host FP64 arrays and the device.
 * is_prim = 1 takes primitive variables (converted on the device).  n = number
 * of doubles in the host array (must equal leaves * 8 * cells per block). */
icarus_status icarus_set_state(icarus_ctx *ctx, int member, const double *host, size_t n, int is_prim);
icarus_status icarus_get_state(icarus_ctx *ctx, int member, double *host, size_t n);

/* One leaf block of a member (leaf = index within the member, Morton order)
 * with its two ghost layers as they were last filled (by icarus_flag_refine,
 * icarus_probe or icarus_ghost_fill; a step leaves them stale): host FP64
 * [8][n0+4][n1+4][n2+4] of conserved variables, n = that count.  Lets a test
 * evaluate a block-local operator on exactly the data the device saw.
 * ICARUS_ERR_ARG for a bad member, leaf or n.  Synchronises. */
icarus_status icarus_get_padded(icarus_ctx *ctx, int member, int leaf, double *host, size_t n);

/* The CME tracer rho X (Sect. 3.1) of a member's leaves, host FP64
 * [leaf][i][j][k] over interior cells (n = leaves * cells per block), leaves
 * in Morton order.  The tracer is the CME's mass fraction X stored as rho X;
 * it enters with X = 1 through the inner-boundary cells the cone CME covers
 * (X = 0 elsewhere) and is carried by each face's mass flux with X from the
 * face's upwind cell, in both stages; it is prolonged and restricted like the
 * other variables (not refluxed).  ICARUS_ERR_STATE if the descriptor has no
 * tracer, ICARUS_ERR_ARG for a bad member or n.  Synchronise. */
icarus_status icarus_get_tracer(icarus_ctx *ctx, int member, double *host, size_t n);
icarus_status icarus_set_tracer(icarus_ctx *ctx, int member, const double *host, size_t n);

/* member time (host write / read) */
icarus_status icarus_set_time(icarus_ctx *ctx, int member, double t);

/* Earth's direction for the windows of the shock criterion (Sect. 3.2) of
 * one member: colatitude colat and longitude lon0 - rate (t - t0) in the
 * co-rotating frame, t the member's time (rate is the synodic rotation rate:
 * Earth drifts against the rotation).  Windows that need Earth pass no cell
 * until it is set.  Not stored in checkpoints.  ICARUS_ERR_ARG for a bad
 * member or a non-finite value. */
icarus_status icarus_set_earth(icarus_ctx *ctx, int member, double colat, double lon0, double t0, double rate);

/* Per-member finest level (<= descriptor max_level). */
icarus_status icarus_set_member_max_level(icarus_ctx *ctx, int member, int max_level);

/* Fill ghost cells of the current state at the member times (the state the
 * estimator and the probe see). */
icarus_status icarus_ghost_fill(icarus_ctx *ctx);

/* Deterministic FP64 sums over a member's leaves of V * U (8 doubles, host). */
icarus_status icarus_conservation_sums(icarus_ctx *ctx, int member, double *out8);

/* Same result as icarus_conservation_sums, for callers that may not allocate
 * device memory while they run (a host framework that hands the whole GPU to
 * its own pool at start-up, a service that must never stall on an
 * allocation).  This call allocates nothing: its scratch is a fixed array of
 * the library's own device memory (room for 16384 leaves per member, 1 MiB),
 * held on every GPU that loads the library until the process exits.  The
 * paper has no counterpart; it is a service of this library.
 *   member   member whose leaves are summed; out8: 8 doubles, host.
 *   errors   ICARUS_ERR_CAPACITY (and a message on stderr) if the member has
 *            more than 16384 leaves; ICARUS_ERR_ARG on bad arguments;
 *            ICARUS_ERR_CUDA if a CUDA call fails.
 * The array and this call's kernels are put in place on a device when the
 * first context is created there (icarus_init_grid looks up the array's
 * address with that device current and caches it), so create contexts before
 * handing the rest of the GPU to another pool and before any stream capture.
 * All calls share the one array; calls that overlap on the GPU race.
 * Synchronises. */
icarus_status icarus_conservation_sums_static(icarus_ctx *ctx, int member, double *out8);

/* Current CFL time step of every member (host, n_members doubles). */
icarus_status icarus_get_dt(icarus_ctx *ctx, double *dt_out);

/* Cumulative leaf-cell updates of every member (a cell advanced by one full
 * step counts once; members past their stop time do not count).  Host,
 * n_members doubles.  Synchronises. */
icarus_status icarus_cell_updates(icarus_ctx *ctx, double *out);

/* Sticky device status word: bit 0 NaN seen, bit 1 floor budget exceeded,
 * bit 2 bounded wait gave up, bit 3 a ghost cell's neighbour was missing
 * from the tree (balance broken; reported as ICARUS_ERR_NONPHYSICAL);
 * *floor_hits receives the floor counter. */
icarus_status icarus_status_word(icarus_ctx *ctx, uint32_t *word, uint64_t *floor_hits);

/* Stage-kernel tile shape (theta x phi cells per CTA) and radial segment
 * length; 0 = library default.  Used by the autotuner. */
icarus_status icarus_set_tile(icarus_ctx *ctx, int tile_theta, int tile_phi, int r_segment);

/* Floor budget.  Density and pressure floors (rho_floor, p_floor) are applied
 * after every stage and counted (icarus_status_word).  A step whose floor hits
 * exceed max_fraction times the leaf cells it advanced (all members) sets bit 1
 * of the status word: the next call that reads the word (every synchronising
 * call, and icarus_step itself, see there) returns ICARUS_ERR_NONPHYSICAL and
 * the context is poisoned.  0 disables the budget.  Default
 * ICARUS_DEFAULT_FLOOR_BUDGET.  Not stored in checkpoints.  ICARUS_ERR_ARG for
 * a negative or NaN fraction. */
#define ICARUS_DEFAULT_FLOOR_BUDGET 0.1
icarus_status icarus_set_floor_budget(icarus_ctx *ctx, double max_fraction);

/* FP32 mode: the pressure of a cell is recomputed in FP64 (from the stored
 * FP32 variables) where p < p_over_e * e or p < beta * B^2/2.  Defaults 0.002
 * and 0.1 (low-beta cells, and cells where FP32 cancellation would cost more
 * than ~1e-4 of p); 0, 0 disables the islands.  No effect in FP64 mode. */
icarus_status icarus_set_fp64_islands(icarus_ctx *ctx, double p_over_e, double beta);

/* How the stage kernels get halo cells that a same-level leaf holds: 1 (the
 * default) reads them from that leaf's interior, and the step's ghost fills
 * cover only the regions around each leaf that coarser or finer leaves hold
 * (plus the physical boundaries); 0 fills every ghost cell before each stage
 * and reads the ghost layer.  Both give the same bits; the switch exists for
 * tests and measurements. */
icarus_status icarus_set_direct_halo(icarus_ctx *ctx, int enable);

/* Capture one step of the launch sequence in a CUDA graph and replay it in
 * icarus_step (1) or launch kernels directly (0).  Default 1. */
icarus_status icarus_use_graph(icarus_ctx *ctx, int enable);

/* Number of kernels launched per step with the current tree (for launch
 * accounting). */
icarus_status icarus_kernels_per_step(icarus_ctx *ctx, int *n);

/* ---- learned refinement pre-flagger ----
 * The paper refines from criteria on the solution (Sect. 3); this predictor
 * (no counterpart in the paper) anticipates the estimator's decision one
 * regrid ahead.  Per block: the index-space gradient magnitude of density,
 * radial speed and pressure, each divided by the cell's magnitude, averaged
 * over the three variables and over 4x4x4 sub-cubes (block sizes must be
 * multiples of 4) -> 64 inputs; MLP 64 -> 128 (ReLU) -> 128 (ReLU) -> 1
 * (sigmoid); binary cross-entropy; Adam (beta 0.9/0.999, eps 1e-8).  FP32.
 * Parameters: W1[128][64], b1[128], W2[128][128], b2[128], w3[128], b3
 * (24961 floats).  All calls synchronise. */

/* Load parameters (host FP32, n = 24961); resets the Adam moments. */
icarus_status icarus_mlp_set_params(icarus_ctx *ctx, const float *host, size_t n);
icarus_status icarus_mlp_get_params(icarus_ctx *ctx, float *host, size_t n);

/* Features of every leaf (global leaf order) after a ghost fill; host_out
 * (optional) receives n_leaves x 64 floats.  The 4 x 4 x 4 sub-cubes need
 * block sizes that are multiples of 4 (else ICARUS_ERR_ARG); each sub-cube
 * mean is summed in a fixed order, so the features are the same bits on
 * every call. */
icarus_status icarus_mlp_features(icarus_ctx *ctx, float *host_out);

/* Refinement probability of every leaf (features + forward), host n_leaves. */
icarus_status icarus_mlp_predict_leaves(icarus_ctx *ctx, float *prob_host);

/* Forward on n <= 4096 host samples x[n][64] -> y[n]. */
icarus_status icarus_mlp_predict(icarus_ctx *ctx, const float *x_host, int n, float *y_host);

/* Gradient of the mean cross-entropy over n <= 4096 host samples (targets
 * 0/1) -> grad_host[24961]; loss_out (optional) receives the mean loss. */
icarus_status icarus_mlp_grad(icarus_ctx *ctx, const float *x_host, const float *t_host, int n, float *grad_host,
                              float *loss_out);

/* Device training set (at most 65536 samples): clear, append host samples. */
icarus_status icarus_mlp_dataset_clear(icarus_ctx *ctx);
icarus_status icarus_mlp_dataset_add(icarus_ctx *ctx, const float *x_host, const float *t_host, int n, int *total);

/* Adam on the first n_train samples of the training set: `epochs` passes in
 * seeded shuffled minibatches of `batch` (<= 4096) at learning rate lr;
 * loss_per_epoch (optional, epochs floats) receives the summed loss. */
icarus_status icarus_mlp_train(icarus_ctx *ctx, int n_train, int epochs, int batch, double lr, uint64_t seed,
                               float *loss_per_epoch);

/* Measured arithmetic peak of the current device on `stream` (cudaStream_t,
 * NULL = legacy default): kind 0 FP64 FMA, 1 FP32 FMA, 2 FP32 FMA on packed
 * pairs; *flops_per_s counts two flops per FMA.  The rooflines of the FP64
 * and FP32 stage kernels are taken against these figures.  Synchronises;
 * allocates nothing.  (A measurement helper; the paper has no counterpart.) */
icarus_status icarus_alu_peak(int kind, void *stream, double *flops_per_s);

/* Per-launch timing with CUDA events (enable = 1).  While enabled,
 * icarus_step launches the kernels directly instead of replaying the graph
 * and records an event pair around every launch on the context's stream. */
icarus_status icarus_profile(icarus_ctx *ctx, int enable);

/* Device time (ms) and number of launches per kernel kind accumulated since
 * the previous read, then reset.  Kinds: 0 dt begin, 1 ghost fill from
 * neighbours, 2 physical-boundary ghosts, 3 predictor stage, 4 corrector
 * stage, 5 reflux, 6 dt finalize, 7 refinement estimator (flagging), 8 regrid
 * data movement, 9 CFL time step of the whole state (after a regrid or a
 * state upload).  Kinds 7-9 are recorded by icarus_flag_refine and
 * icarus_regrid while profiling is enabled.  ms and count hold nkinds
 * entries (<= 10).  Synchronises the stream. */
icarus_status icarus_profile_read(icarus_ctx *ctx, double *ms, int *count, int nkinds);

/* Checkpoint and resume (the paper runs for days of simulated time; it has no
 * passage on checkpoints).  icarus_save writes to the host file `path`
 * everything a step reads: the descriptor fields that fix grid and physics,
 * per member its finest level, cone CME, leaf tree, time, CFL time step and
 * cell-update count, the inner-boundary maps and background speeds, the
 * leaves' state in the working precision, the FP64-island thresholds, the
 * floor-hit count and the pre-flagger's parameters if set (not its Adam
 * moments).  Binary, host byte order.  Synchronises the stream.
 * icarus_load reads such a file into a context created with the same
 * descriptor (n_cells, block, max_level, stretch, geometry, extents, gamma,
 * omega, cfl, divb_cd, floors, precision, n_members, boundaries; max_blocks
 * and the arena may differ): stepping then continues bit for bit as the
 * saved context would have.  Errors: ICARUS_ERR_ARG if the file cannot be
 * opened, is not a checkpoint of this version or does not match the
 * descriptor (the context is then unchanged); ICARUS_ERR_CAPACITY if its
 * leaves exceed max_blocks (unchanged).  A successful load clears a
 * poisoned context's status word. */
icarus_status icarus_save(icarus_ctx *ctx, const char *path);
icarus_status icarus_load(icarus_ctx *ctx, const char *path);

void icarus_destroy(icarus_ctx *ctx);
const char *icarus_status_string(icarus_status s);

#ifdef __cplusplus
}
#endif
#endif
