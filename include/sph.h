/*
 * sph.h -- C-ABI of the GB300 multi-resolution SPH density/force library (libsph).
 *
 * The library computes the two SPH interaction passes of Gonnet, Schaller,
 * Theuns & Chalk, "SWIFT: Fast algorithms for multi-resolution SPH on
 * multi-core architectures" (arXiv:1309.3783):
 *
 *   density  -- every particle i gathers the particles j within its own
 *               smoothing length (Section II, first stage);
 *   force    -- every particle i interacts with the particles j within
 *               max(h_i, h_j) (Section II, second stage);
 *
 * with the neighbours found through the hierarchical cell decomposition of
 * Section II-B (top grid with cell edge >= h_max, recursive splitting of cells,
 * of self-interactions and of pair-interactions) and the sorted, axis-projected
 * cell-pair interactions of Section II-C (Fig. 3).  Every step runs in CUDA
 * kernels for sm_103a on one GPU.
 *
 * Physics (the paper prints no equations; the library uses the textbook
 * formulation of Gadget-2, the code the paper compares against):
 *   support radius  H = gamma_K * h, gamma_K = 1.825742 (FP32), "within h" = r < H;
 *   kernel          cubic spline with compact support H;
 *   density         rho_i = sum_{r_ij < H_i} m_j W(r_ij, H_i), j = i included;
 *   h update        Newton on (4 pi/3) H^3 sum_j W = N_ngb (Section III-B: 48);
 *   ghost           P = (gamma-1) rho u, c = sqrt(gamma P / rho), grad-h factor f;
 *   force           pressure with grad-h terms + Monaghan viscosity (alpha = 2.0).
 *
 * Conventions
 *   - Every call returns sph_status; on error it fills no output and
 *     sph_last_error() describes the failure.
 *   - The caller owns every pointer it passes.  The library owns the device
 *     state of a box until sph_box_destroy().
 *   - Pointers are host pointers unless the call takes a `mem` argument equal
 *     to SPH_MEM_DEVICE, in which case they are device pointers on the
 *     context's device.
 *   - Work is ordered on the context's CUDA stream.  Calls that return host
 *     data (sph_get with host memory, sph_h_update's counters, sph_get_stats)
 *     synchronise that stream.
 *   - Per-particle outputs come back in the caller's particle order.
 *   - Neighbour counts and interacting pair sets are exact: the decision
 *     r_ij < H is taken in FP32 with a guard band and re-taken in FP64 from the
 *     caller's positions (d = x_i - x_j per component, wrapped by +-L when
 *     |d| > L/2, r2 = (d0 d0 + d1 d1) + d2 d2, no fused multiply-add,
 *     compared with H*H) for every pair inside the band.
 */
#ifndef SPH_H
#define SPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPH_OK = 0,
    SPH_E_INVALID = -1,        /* bad argument or input value (NaN, h <= 0, x outside [0, L)) */
    SPH_E_OOM = -2,            /* device allocation failed or budget exceeded                 */
    SPH_E_H_TOO_LARGE = -3,    /* H_max does not fit the box (periodic: H_max >= L/4)         */
    SPH_E_NOT_BUILT = -4,      /* pass called before sph_build / sph_density                 */
    SPH_E_NOT_CONVERGED = -5,  /* h iteration stopped with unconverged particles              */
    SPH_E_TIMEOUT = -6,        /* a bounded device-side wait gave up                          */
    SPH_E_CUDA = -7,           /* CUDA runtime error                                          */
    SPH_E_BUSY = -8            /* server queue full / request not finished                    */
} sph_status;

typedef enum { SPH_MEM_HOST = 0, SPH_MEM_DEVICE = 1 } sph_mem;

/* Method parameters.  sph_params_default() fills the paper's values
 * (Section III-B: N_ngb = 48, gamma = 5/3, alpha = 2.0, C_CFL = 0.3; cells are
 * split above 400 particles when more than 87.5 % have H below half the edge). */
typedef struct sph_params {
    float gamma_kernel;   /* H / h of the cubic spline (1.825742)                    */
    float n_ngb;          /* target weighted neighbour number (48)                   */
    float gamma_gas;      /* adiabatic index (5/3)                                   */
    float alpha_visc;     /* viscosity alpha (2.0)                                   */
    float c_cfl;          /* Courant factor for sph_cfl_dt (0.3)                     */
    float h_tol;          /* relative tolerance on the neighbour number (1e-4)      */
    int32_t h_max_iter;   /* h iterations before giving up (30)                      */
    int32_t leaf_max;     /* split a cell when it holds more particles (400)         */
    float split_frac;     /* ... and more than this fraction has H < edge/2 (0.875)  */
    int32_t max_depth;    /* deepest cell level, <= 20 (20)                          */
    float split_headroom; /* pairs split, and the top grid is chosen, only when
                             H (1 + split_headroom) clears the limit, so that h
                             may grow by that much before the interactions must be
                             rebuilt; 0 = the paper's rule exactly (0.1)        */
    int32_t reuse;        /* 1: sph_step keeps the cell decomposition, its lists and
                             sorted indices over steps while they stay valid
                             (Section II-C: sorted indices re-used until the
                             decomposition must be re-computed): every particle keeps
                             its cell, and H + 2 * (largest displacement since the
                             build) must stay below the limit its interactions
                             assumed, else the step rebuilds.  0: rebuild every
                             step (0)                                            */
    int32_t sort_merge;   /* 1: a cell's sorted cluster lists (cells of 33-2048
                             clusters) are built by merging its leaves' sorted
                             runs pairwise up to the cell (Section II-C: a cell's
                             sort follows from its children's by a linear merge);
                             0: every list is sorted directly (a bitonic sort in
                             shared memory, faster on GB300 at these sizes).
                             Both give the same lists (0)                        */
    int32_t cluster_max;  /* particles per cluster, the unit a warp loads and the
                             interaction kernels cull by box (1..32; 32)          */
    int32_t compensated;  /* density sums with compensated (Kahan-Neumaier)
                             summation: 1 on, 0 off, -1 on from n_ngb >= 100,
                             where the neighbour sums have many terms (-1)       */
    int32_t precision;    /* position precision of the pair arithmetic: 0 = each
                             particle's offset from its cell's centre, rounded once
                             to FP32 from the FP64 position (the error scales with
                             the cell); 1 = plain FP32: positions held as x / L
                             rounded to FP32 in the box frame (error up to 2^-25 L
                             whatever the cell), the offsets taken from them.  In
                             both, counts and pair sets stay exact: the guard band
                             of the FP32 decision covers the rounding and pairs
                             inside it are decided in FP64 (0)                   */
    int32_t graphs;       /* 1: a kick-drift-kick step of sph_step is launched as
                             one CUDA graph with conditional nodes (captured after
                             a host-driven build and launched again while the boxes
                             keep their top levels and the capacities hold; one
                             synchronisation per step); 0: every launch from the
                             host, with the synchronisations of a build (1)      */
    int32_t pair_cache;   /* 1: the first density pass of an h iteration keeps its
                             interacting pairs (per batch of staged partners: their
                             indices and each own particle's exact pair mask), and
                             the force pass replays them for every task whose
                             particles kept their h since then instead of culling
                             and testing the candidates again; about 256 bytes
                             per batch, about one batch per particle (the pool
                             starts at 1.5 and grows to what a recording took;
                             tasks a full pool could not keep cull again).  The pair
                             set is the same.  On GB300 the force pass then takes
                             a quarter less time and the recording first density
                             pass about as much more; 0: the force pass culls on
                             its own (0)                                           */
    int32_t h_gather;     /* 1: a later pass of the h iteration (Section II-D, the
                             density loop again for the particles whose h has not
                             converged) in which at most an eighth of the
                             particles iterate gathers: each leaf's iterating
                             particles are packed into clusters of up to 32 and
                             every interaction runs for the packed clusters of its
                             cells, the own side only, instead of the symmetric
                             tasks of every cluster near an iterating particle.
                             The sums are the same up to rounding order; counts
                             stay exact.  0: the symmetric tasks in every pass;
                             passes with pair counting (sph_box_count_pairs) also
                             take them (1)                                          */
} sph_params;

typedef struct sph_ctx sph_ctx;
typedef struct sph_box sph_box;

/* Output fields of sph_get.  Element type and count per particle in brackets. */
typedef enum {
    SPH_FIELD_RHO = 0,        /* density                              [f32 x1] */
    SPH_FIELD_DRHO_DH = 1,    /* d rho / d h                          [f32 x1] */
    SPH_FIELD_NW = 2,         /* number density sum_j W               [f32 x1] */
    SPH_FIELD_NNGB = 3,       /* weighted neighbour number (4pi/3)H^3 nw [f32] */
    SPH_FIELD_COUNT = 4,      /* neighbours j != i with r < H_i       [i32 x1] */
    SPH_FIELD_H = 5,          /* smoothing length                     [f32 x1] */
    SPH_FIELD_P = 6,          /* pressure                             [f32 x1] */
    SPH_FIELD_C = 7,          /* sound speed                          [f32 x1] */
    SPH_FIELD_F = 8,          /* grad-h factor f                      [f32 x1] */
    SPH_FIELD_A = 9,          /* acceleration                         [f32 x3] */
    SPH_FIELD_DUDT = 10,      /* du/dt                                [f32 x1] */
    SPH_FIELD_VSIG = 11,      /* max signal velocity over force pairs [f32 x1] */
    SPH_FIELD_CONVERGED = 12, /* 1 when h converged                   [i32 x1] */
    SPH_FIELD_X = 13,         /* position                             [f64 x3] */
    SPH_FIELD_V = 14,         /* velocity                             [f32 x3] */
    SPH_FIELD_U = 15,         /* internal energy                      [f32 x1] */
    SPH_FIELD_REDUCTIONS = 16, /* 8 doubles: sum m a (3), sum m (v.a + du/dt),
                                 sum m v (3), sum m (v^2/2 + u); n must be 8 */
    SPH_FIELD_FORCE_COUNT = 17 /* force partners j != i with r < max(H_i, H_j)
                                 [i32 x1]; only after a force pass run with pair
                                 counting on (sph_box_count_pairs) */
} sph_field;

/* Counters of the last build and passes. */
typedef struct sph_stats {
    int64_t n_particles;
    int64_t n_cells;            /* cells of the tree (all levels)                     */
    int64_t n_leaves;
    int64_t n_selfs;            /* final self-interactions                            */
    int64_t n_pairs;            /* final pair-interactions                            */
    int64_t n_sort_segments;    /* (cell, axis) sorted lists                          */
    int64_t n_sorted_entries;
    int32_t top_level;          /* level of the top grid (edge L / 2^top_level)       */
    int32_t depth;              /* deepest level holding a cell                       */
    int32_t h_iterations;       /* density passes of the last sph_h_update            */
    int32_t rebuilds;           /* tree rebuilds during the last sph_h_update         */
    int64_t n_unconverged;
    /* filled only when pair counting is on (sph_box_count_pairs); summed over
       the density passes of the last sph_density / sph_h_update and the force
       passes since then */
    int64_t density_pairs;      /* unordered pairs with r < max(H_i, H_j)             */
    int64_t density_sides;      /* sum over those pairs of [r < H_i] + [r < H_j]      */
    int64_t density_candidates; /* unordered pairs whose distance was evaluated       */
    int64_t density_pairs_cellpair;      /* ... of which in cell-pair interactions     */
    int64_t density_sides_cellpair;
    int64_t density_candidates_cellpair;
    int64_t force_pairs;        /* unordered pairs with r < max(H_i,H_j), r > 0       */
    int64_t force_candidates;
    int64_t force_pairs_cellpair;
    int64_t force_candidates_cellpair;
    int64_t guard_rechecks;     /* predicate decisions re-taken in FP64               */
    int64_t builds;             /* full decompositions built since the box was set    */
    int64_t reuses;             /* steps that kept the decomposition (params.reuse)   */
    int64_t h_active_after_first; /* particles the first density pass of the last h
                                     iteration left unconverged (the quality of the
                                     starting h: the previous step's roots, extrapolated) */
    int64_t leaf_max;           /* the box's split threshold (set or autotuned)      */
    int64_t cluster_max;        /* the box's particles per cluster (set or autotuned) */
    int64_t graph_steps;        /* steps of sph_step run as one captured graph (params.graphs) */
    int64_t host_steps;         /* steps whose passes were launched from the host       */
    int64_t host_syncs;         /* synchronisations of the host with the box's stream   */
    /* filled only when pair counting is on: force tasks since the last density
       or h update replayed from the pairs the first density pass kept
       (params.pair_cache), and those that culled their candidates again (a
       particle near them took a new h, or the records ran out of room)      */
    int64_t force_tasks_replayed;
    int64_t force_tasks_culled;
    int64_t h_gathered_passes;  /* later density passes of the last h iteration
                                   launched from the host (sph_h_update, or a step
                                   not run as a graph) that gathered (params.h_gather) */
} sph_stats;

/* Device time of one phase of the path (CUDA events on the stream the phase runs
 * on: the context stream, except `shift` -- the particle-side part of the build --
 * which runs on the box's own side stream while `lists` runs on the context
 * stream; the two overlap, so phase times can add up to more than the step). */
typedef struct sph_profile_entry {
    char name[32];              /* ingest, keys_sort, tree, lists, shift, axis_sort,
                                   density (pair and self interactions),
                                   density_tasks (the pass's live task list), ghost,
                                   force, force_tasks, reduce, kick_drift, output,
                                   reuse (keeping the decomposition, params.reuse) */
    int64_t calls;              /* times the phase ran while recording                */
    int64_t launches;           /* kernel launches inside it                          */
    double ms;                  /* summed device time                                 */
} sph_profile_entry;

/* ---- parameters and context ------------------------------------------------ */

/* Fill *p with the paper's values.  Never fails. */
void sph_params_default(sph_params* p);

/* Create a context on CUDA device `device` with its own non-blocking stream.
 * params may be NULL (defaults).  *out receives the handle.
 * Errors: SPH_E_INVALID (bad params or device), SPH_E_CUDA. */
sph_status sph_ctx_create(const sph_params* params, int device, sph_ctx** out);

/* Replace the context's stream with a caller-owned cudaStream_t (passed as
 * void*; NULL restores the context's own stream).  The caller keeps the stream
 * alive while the context uses it.  All work of a call is ordered on that stream:
 * the part of a build that a box runs on its own side stream is forked from it
 * and joined back into it with events. */
sph_status sph_ctx_set_stream(sph_ctx* ctx, void* cuda_stream);

/* The stream the context launches on, as a cudaStream_t cast to void*. */
void* sph_ctx_stream(sph_ctx* ctx);

/* Destroy a context.  Errors: SPH_E_BUSY while boxes or servers created on it
 * are alive (destroy them first). */
sph_status sph_ctx_destroy(sph_ctx* ctx);

/* Text of the last error on this context (never NULL; "" when none). */
const char* sph_last_error(sph_ctx* ctx);

/* ---- boxes ------------------------------------------------------------------ */

/* Create a box for n particles in the cube [0, L)^3, periodic or open.
 * Allocates the box's device memory for n particles.
 * Errors: SPH_E_INVALID (n < 1, L <= 0), SPH_E_OOM, SPH_E_CUDA. */
sph_status sph_box_create(sph_ctx* ctx, int64_t n, double box_len, int periodic, sph_box** out);

/* Copy the particle state into the box (host or device pointers, see `mem`).
 * x: n*3 doubles (x0 y0 z0 x1 ...), each in [0, L); v: n*3 floats; m, u, h:
 * n floats each (m > 0, u >= 0, h > 0, all finite).  Values are checked on the
 * device during the next sph_build (SPH_E_INVALID then).  Clears built state. */
sph_status sph_box_set(sph_box* box, const double* x, const float* v, const float* m,
                       const float* u, const float* h, int mem);

/* Set one state field of the box from caller-order data (host or device, see
 * `mem`): SPH_FIELD_A (n*3 floats) and SPH_FIELD_DUDT (n floats) restore the
 * forces of the last step, so that sph_step with dt > 0 continues a run from a
 * saved state (a checkpoint) without recomputing them; SPH_FIELD_H (n floats)
 * replaces h.  Call after sph_box_set.  Errors: SPH_E_INVALID (other fields,
 * n mismatch). */
sph_status sph_box_set_field(sph_box* box, int field, const void* src, int64_t n, int mem);

/* Mark the box's first n_owned particles (caller order) as its own and the
 * others as a halo: copies of particles that another rank owns in a spatial
 * decomposition of one box over several GPUs (the distributed-memory version
 * the paper names as future work, Section IV).  Halo particles take part in
 * every pass, so that the owned particles find all their neighbours, but only
 * owned particles enter the conservation sums (SPH_FIELD_REDUCTIONS), which the
 * ranks then add.  Default: every particle (n_owned = n).  Kept until the next
 * call; the reductions of an earlier force pass are invalidated.
 * Errors: SPH_E_INVALID (n_owned outside 0..n). */
sph_status sph_box_set_owned(sph_box* box, int64_t n_owned);

/* Turn exact pair counting on (1) or off (0) for the following passes; the
 * counts appear in sph_stats.  Counting adds atomics to the pair kernels. */
sph_status sph_box_count_pairs(sph_box* box, int on);

sph_status sph_box_destroy(sph_box* box);

/* ---- the hot path (Section II) --------------------------------------------- */

/* Build the decomposition from the current positions and h: support radii,
 * keys, sort, cell tree with the split rule, particle offsets relative to
 * their cell, self/pair interaction lists with recursive splitting, and the
 * per-cell sorted projections along every needed cell-pair axis (Sections
 * II-B, II-C).  Errors: SPH_E_INVALID, SPH_E_H_TOO_LARGE, SPH_E_OOM, SPH_E_CUDA. */
sph_status sph_build(sph_box* box);

/* One density pass at the current h over every particle (builds first when
 * needed).  Fills rho, d rho/dh, nw, N~, count. */
sph_status sph_density(sph_box* box);

/* Iterate h to N~ = n_ngb within h_tol (params), with density passes over the
 * still unconverged particles, rebuilding the decomposition when an h grows
 * past what the cell splits assumed; then computes the ghost quantities.
 * *n_unconverged and *iterations (either may be NULL) receive the outcome.
 * Returns SPH_E_NOT_CONVERGED when particles remain unconverged after
 * h_max_iter passes (their h is left at the last value evaluated). */
sph_status sph_h_update(sph_box* box, int64_t* n_unconverged, int32_t* iterations);

/* Force pass over pairs with r < max(H_i, H_j) using the ghost quantities of
 * the last density pass, then the FP64 conservation reductions.
 * Errors: SPH_E_NOT_BUILT when no density pass preceded it. */
sph_status sph_force(sph_box* box);

/* One full step: build, density with h iteration, force, reductions; when
 * dt > 0 it is a kick-drift-kick step: v += a dt/2, u += du/dt dt/2 with the
 * forces of the previous step (computed first when absent), x += v dt in FP64
 * (wrapped into [0, L) for periodic boxes), then the passes at the new
 * positions and the closing half kick. */
sph_status sph_step(sph_box* box, double dt);

/* Courant time step C_CFL * min_i H_i / max_i vsig_i of the last force pass. */
sph_status sph_cfl_dt(sph_box* box, double* dt);

/* Copy a field (see sph_field) into dst, in the caller's particle order.
 * n is the particle count (8 for SPH_FIELD_REDUCTIONS).  With mem ==
 * SPH_MEM_HOST the call synchronises the stream.
 * Errors: SPH_E_INVALID (n mismatch), SPH_E_NOT_BUILT (field not computed). */
sph_status sph_get(sph_box* box, int field, void* dst, int64_t n, int mem);

/* Copy n_fields fields (at most 64) at once: field fields[k] into dst[k] with
 * n[k] elements as in sph_get, all to memory of kind mem, with one
 * synchronisation at the end (host destinations in page-locked memory are
 * filled asynchronously until then).  Errors as sph_get; fields before a
 * failing one may have been copied. */
sph_status sph_get_fields(sph_box* box, int32_t n_fields, const int32_t* fields, void* const* dst,
                          const int64_t* n, int mem);

/* Counters of the last build and passes (synchronises). */
sph_status sph_get_stats(sph_box* box, sph_stats* out);

/* Start (on = 1, clearing earlier records) or stop recording the device time of
 * every phase of this box with CUDA events on the context stream. */
sph_status sph_box_profile(sph_box* box, int on);

/* Per-phase totals recorded since sph_box_profile(box, 1): fills up to cap
 * entries (14 phases), *n_out receives the number of phases.  Synchronises. */
sph_status sph_get_profile(sph_box* box, int32_t cap, sph_profile_entry* out, int32_t* n_out);

/* Kernel launches made by the library in this process so far. */
int64_t sph_launch_count(void);

/* FP32 throughput of the device, measured: a kernel of independent fused
 * multiply-add chains (8 per thread, no memory traffic) over every SM, timed
 * with CUDA events on the context's stream after a warm-up launch.  *tflops
 * receives the rate (2 flops per FMA); the roofline's measured FP32 ceiling.
 * Synchronises. */
sph_status sph_measure_fp32_peak(sph_ctx* ctx, double* tflops);

/* Autotune the cell split threshold leaf_max (Section II-B splits cells above
 * it; the paper uses 400 on its CPUs) and the particles per cluster for this
 * box's current particles: times build + density + force for leaf_max in {24,
 * 32, 48, 64, 96, 128, 192, 256, 400, 600, 800, 1200, 1600, 2400, 3200, 4800}
 * with clusters of 32,
 * then clusters of 16 and 24 at the best leaf_max, and keeps the fastest pair for
 * the box.
 * *leaf_max (may be NULL) receives the leaf size; sph_get_stats reports both.
 * Results of the passes run while tuning are discarded (the box is unbuilt). */
sph_status sph_box_tune(sph_box* box, int32_t* leaf_max);

/* Set the box's particles per cluster (1..32); clears built state. */
sph_status sph_box_set_cluster_max(sph_box* box, int32_t cluster_max);

/* Set the box's split threshold leaf_max (>= 1); clears built state. */
sph_status sph_box_set_leaf_max(sph_box* box, int32_t leaf_max);

/* ---- introspection of the decomposition (Section II-B) -------------------- */

/* Cells of the current tree.  For cell c < min(cap, count): level[c], the
 * integer coordinates ijk[3c..3c+2] at that level (cell edge L / 2^level),
 * count[c] particles, split[c] = 1 when the cell was split.  *n_out receives
 * the number of cells.  Synchronises. */
sph_status sph_get_cells(sph_box* box, int64_t cap, int32_t* level, int32_t* ijk,
                         int32_t* count, int32_t* split, int64_t* n_out);

/* Final interactions: kind[k] = 0 (self of cell a[k]) or 1 (pair a[k], b[k]
 * along axis[k] in 0..12, from a towards b).  Cell numbers index the
 * sph_get_cells arrays.  Selfs come first.  Synchronises.
 * Axis numbering: the offset of b from a in cell units (periodic image
 * included) is, for axis 0..12: (1,0,0) (-1,1,0) (0,1,0) (1,1,0) (-1,-1,1)
 * (0,-1,1) (1,-1,1) (-1,0,1) (0,0,1) (1,0,1) (-1,1,1) (0,1,1) (1,1,1). */
sph_status sph_get_interactions(sph_box* box, int64_t cap, int32_t* kind, int32_t* a,
                                int32_t* b, int32_t* axis, int64_t* n_out);

/* ---- batched and served boxes ---------------------------------------------- */

typedef struct sph_server sph_server;

/* A server keeps many boxes resident on the device and advances all admitted
 * boxes by one step per tick with one batched pipeline (one launch per kernel
 * for all boxes).  Boxes are admitted while their device footprint fits in
 * budget_bytes (0 = 80 % of free device memory) and at most max_boxes are
 * resident; the rest wait in submission order. */
sph_status sph_server_create(sph_ctx* ctx, int64_t budget_bytes, int32_t max_boxes, sph_server** out);

/* Queue a box of n particles (host arrays as in sph_box_set) to advance
 * n_steps steps of size dt (dt = 0: passes only, no kick/drift).  *id receives
 * the request id.  Inputs are copied at submission.
 * Errors: SPH_E_INVALID, SPH_E_OOM (box can never fit the budget). */
sph_status sph_server_submit(sph_server* s, int64_t n, double box_len, int periodic,
                             const double* x, const float* v, const float* m, const float* u,
                             const float* h, int32_t n_steps, double dt, int64_t* id);

/* Bound the work of one tick: boxes are admitted only while the resident
 * particles stay within max_particles (a box larger than that is admitted
 * when nothing else is resident), so that the time of a batched step stays
 * bounded while bursts of requests wait in the queue.  0 (the default): no
 * bound beyond the memory budget.  Errors: SPH_E_INVALID (max_particles < 0). */
sph_status sph_server_set_tick_budget(sph_server* s, int64_t max_particles);

/* Run one tick: admit waiting boxes that fit (their intake pass: h iterated
 * from the submitted h, starting forces), advance every admitted box by one
 * step in one batched pipeline, retire finished boxes.  *n_active receives the
 * number of boxes advanced (0 when idle). */
sph_status sph_server_tick(sph_server* s, int32_t* n_active);

/* State of request id: *done = 1 when all its steps ran.  step_ms (may be
 * NULL, capacity max_steps) receives the device time of each of its steps. */
sph_status sph_server_poll(sph_server* s, int64_t id, int32_t* done, float* step_ms, int32_t max_steps);

/* Device time of the intake pass request id went through in its admission
 * tick (its h iteration from the initial h and its starting forces, batched
 * with the other boxes admitted in that tick); -1 when it had none (waiting,
 * or a request of n_steps = 0, which runs as passes of the batched step). */
sph_status sph_server_intake_ms(sph_server* s, int64_t id, float* ms);

/* Copy a field of a finished request (as sph_get, host memory). */
sph_status sph_server_get(sph_server* s, int64_t id, int field, void* dst, int64_t n);

/* Forget a finished request and its results. */
sph_status sph_server_release(sph_server* s, int64_t id);

sph_status sph_server_destroy(sph_server* s);

/* ---- density without allocation ---------------------------------------------
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory (an allocator-free embedding, code that must
 * not reach the driver's allocator after start-up, or a pre-sized arena owned
 * by someone else).  It computes the density pass of a small box with no
 * context, no box and no allocation: its working memory (a uniform cell list
 * and the particles sorted by cell, about 0.4 MB) is one static device array
 * that every device holds from the moment the library is loaded until the
 * process exits.
 *
 * x (n*3 doubles in [0, L)), m, h (n floats), rho (n floats, out) and count
 * (n int32, out) are device pointers on the current device; stream is a
 * cudaStream_t (NULL: the legacy default stream).  Results: rho_i including the
 * self term and the neighbour count j != i with r_ij < H_i, H = 1.825742 h,
 * decided exactly like sph_density.  Returns SPH_E_INVALID for n < 1 or
 * n > SPH_STATIC_MAX_N, for a non-finite L <= 0, and for any particle with a
 * coordinate outside [0, L) or an h or m that is not finite and positive (the
 * checks of sph_build); SPH_E_H_TOO_LARGE when a periodic box is narrower than
 * three H_max; SPH_E_CUDA on a runtime error.  Synchronises the stream.
 * The first call on a device looks up the array's address: make it before any
 * stream capture.  All calls share the one array (each call clears what it
 * needs), so calls that overlap on the GPU, from any stream or thread, race:
 * serialise them. */
#define SPH_STATIC_MAX_N 16384
#define SPH_STATIC_GAMMA_K 1.825742f
sph_status sph_density_static(const double* x, const float* m, const float* h, int64_t n, double box_len,
                              int periodic, float* rho, int32_t* count, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SPH_H */
