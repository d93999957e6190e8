/*
 * gamma.h -- C ABI of the GB300 gamma-index library (libgamma_gb300.so).
 *
 * Computes, for every reference voxel r_r, the gamma index of Eq. (1)
 * (Section 2.1): the minimum Euclidean distance in the normalised
 * dose-distance space (r / DTA, D / DD) from (r_r, D_r(r_r)) to the
 * continuous evaluation surface spanned by the evaluation dose points (the
 * geometric method of Ju et al. that the paper adopts, Section 2.1), using the
 * radially sorted cell table and early exit of Algorithm A1 (steps 2-4) and a
 * GPU kernel that evaluates every simplex face rather than recursing
 * (Section 2.2, Algorithm A2 step 6).
 *
 * Conventions shared by every call:
 *  - Dose grids are float32, C-ordered (z, y, x), contiguous.  A 2D problem
 *    has ndim = 2 and shape[0] = 1; spacing[0] is then ignored.  Every axis of
 *    the problem needs at least two voxels.  Reference and evaluation grids
 *    coincide (same shape, spacing and origin).
 *  - The evaluation surface is the graph of the piecewise-linear interpolant
 *    of the evaluation dose over the Freudenthal triangulation of the grid
 *    (each cube with lower corner p is split into the simplices
 *    p -> p+e_s1 -> p+e_s1+e_s2 -> ... over the axis permutations s).
 *    Simplices with a vertex outside the grid do not exist.
 *  - Pointers named *_dev are device pointers on the handle's device; *_host
 *    are host pointers (pinned memory recommended).  Device pointers passed to
 *    gamma_create are borrowed: the caller keeps them alive and unchanged in
 *    shape for the handle's lifetime; their contents may change between runs.
 *  - Calls on one handle must not overlap: a handle owns one set of scratch
 *    buffers, and two runs in flight at once race on them.
 *  - Every call that takes a handle makes the handle's device current for the
 *    duration of the call and restores the caller's device before returning.
 *  - Return value: GAMMA_OK (0) or a negative gamma_status.  No call throws,
 *    aborts or prints.
 */
#ifndef GAMMA_GB300_H
#define GAMMA_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gamma_ctx *gamma_handle;

typedef enum {
    GAMMA_OK = 0,
    GAMMA_ERR_INVALID_ARG = -1,     /* null pointer, bad criteria, bad option */
    GAMMA_ERR_SHAPE = -2,           /* ndim not 2/3, an axis with < 2 voxels, too many voxels */
    GAMMA_ERR_NAN_INPUT = -3,       /* a NaN or Inf dose was seen by the last run */
    GAMMA_ERR_OOM = -4,             /* device or host allocation failed */
    GAMMA_ERR_TABLE_TOO_LARGE = -5, /* the requested cell table cannot be built */
    GAMMA_ERR_TIMEOUT = -6,         /* a bounded device wait gave up */
    GAMMA_ERR_CUDA = -7,            /* a CUDA runtime call failed (see gamma_last_cuda_error) */
    GAMMA_ERR_NOT_RUN = -8,         /* results requested before any run */
    GAMMA_ERR_MODEL = -9,           /* model file missing, malformed or of the wrong shape */
    GAMMA_ERR_QUEUE_FULL = -10,     /* internal work queue overflowed (results incomplete) */
    GAMMA_ERR_TOO_LARGE = -11,      /* grid larger than gamma_run_noalloc's fixed scratch */
    GAMMA_ERR_DOSE_NORM = -12       /* global criteria without a positive dose norm (see below) */
} gamma_status;

typedef enum { GAMMA_GLOBAL = 0, GAMMA_LOCAL = 1 } gamma_mode;

/* Gamma criteria (Eq. 1: Delta D and Delta d; Section 3.6).
 *  dd_frac     DD criterion as a fraction (0.03 = 3 %), > 0.
 *  dta_mm      DTA criterion in mm, > 0.
 *  mode        GAMMA_GLOBAL: Delta D = dd_frac * D_norm for every voxel.
 *              GAMMA_LOCAL:  Delta D(v) = dd_frac * D_r(v).
 *  cutoff_frac a reference voxel is evaluated iff D_r(v) >= cutoff_frac *
 *              D_norm (and, in local mode, D_r(v) > 0); the comparison is
 *              taken in float32.  Others get NaN and are not counted.
 *  dose_norm   D_norm; <= 0 means the maximum of the reference dose,
 *              computed on the device at every run.  Global criteria need
 *              D_norm > 0: a run whose reference has no positive dose (and
 *              no dose_norm given) evaluates no voxel (every gamma NaN) and
 *              its pass rate reports GAMMA_ERR_DOSE_NORM. */
typedef struct {
    float dd_frac;
    float dta_mm;
    int mode;
    float cutoff_frac;
    float dose_norm;
} gamma_criteria;

/* Counters of the last run (gamma_get_stats). */
typedef struct {
    int64_t n_voxels;        /* grid voxels */
    int64_t n_eval;          /* evaluated voxels (passed the cutoff) */
    int64_t n_pass;          /* evaluated voxels with gamma <= 1 */
    int64_t tail_voxels;     /* voxels that searched past the key-0 cells */
    int64_t overflow_voxels; /* voxels that ran past the table and scanned their box */
    int64_t fp64_cells;      /* cells recomputed in FP64 (near-singular Gram matrix) */
    int64_t seeded;          /* queued voxels seeded by an attached model */
    int64_t seed_improved;   /* ... whose upper bound the seed lowered */
    int64_t cells_keyed;     /* stats mode: tail cells reached before the early exit */
    int64_t cells_visited;   /* stats mode: tail cells whose faces were evaluated */
    int64_t cells_pruned;    /* stats mode: tail cells skipped by the dose lower bound */
    double d_norm;           /* dose norm used */
    double r_max;            /* max over evaluated voxels of DD/Delta D (Algorithm A1 step 1) */
    int64_t table_entries;   /* cell table length */
    double table_radius;     /* every cell with key < table_radius is in the table */
    uint32_t flags;          /* internal flags (non-finite input, queue overflow) */
    int64_t lane_slot_steps; /* stats mode, default walk: 32 x the warps' loop steps of the
                                queue walk, idle lanes included (0 for the other walks) */
} gamma_stats;

/* Per-phase device times of the last run, in ms, measured with CUDA events
 * recorded on the run's stream (option "timing" = 1), in the split of
 * Section 3.1: transfer (T_t: h2d + d2h, host-buffer runs only), processing
 * (T_p: prepare + order) and search (T_gamma: shell + tail). */
typedef struct {
    float h2d_ms;       /* host-to-device copies (gamma_run_host) */
    float prepare_ms;   /* dose norm and finite check */
    float shell_ms;     /* gamma0 and the key-0 cells, every voxel */
    float order_ms;     /* cost ordering of the queued voxels */
    float tail_ms;      /* table walk of the queued voxels */
    float d2h_ms;       /* device-to-host copy of the gamma map (gamma_run_host) */
    float total_ms;     /* first to last event */
    int overlapped;     /* 1: an overlapped gamma_run_host run, whose phases run
                         * concurrently: every field is then the time from the
                         * start of the run to the END of that phase (h2d: the
                         * last input copy; prepare: the reference reduction;
                         * shell: the last z slab; d2h: the map copy-out;
                         * total: the final patch of the queued voxels);
                         * 2: the same, with the shell gated per z slab */
} gamma_timings;

/* Create a handle for one dose-pair geometry (Algorithm A1 steps 2-3: builds
 * the radially sorted cell table on the host and uploads it).
 *  out          receives the handle.
 *  ref_dev,     reference / evaluation doses, device, float32, shape below,
 *  eval_dev     borrowed.  Both NULL: the handle allocates its own device
 *               buffers, to be filled by gamma_run_host.  One NULL: error.
 *  ndim         2 or 3.
 *  shape        (nz, ny, nx); nz = 1 for 2D.  nz*ny*nx < 2^31.
 *  spacing_mm   (hz, hy, hx) voxel size in mm, > 0 (hz ignored for 2D).
 *  crit         criteria (copied).
 * Errors: INVALID_ARG, SHAPE, OOM, TABLE_TOO_LARGE, CUDA.  Synchronous. */
int gamma_create(gamma_handle *out, const float *ref_dev, const float *eval_dev, int ndim,
                 const int64_t shape[3], const float spacing_mm[3], const gamma_criteria *crit);

/* Create a handle for reference and evaluation doses on different grids
 * (the paper interpolates doses to other resolutions, Section 3).  Each grid
 * has its own shape (nz, ny, nx), spacing (hz, hy, hx) and origin (z, y, x) of
 * its first node, in mm, on the same axes; nz = 1 for 2D.  The evaluation
 * surface is the Freudenthal interpolant of the evaluation grid (at least 2
 * nodes per axis); gamma is computed for every reference voxel from its own
 * position, wherever it falls (inside the evaluation grid or not).  The
 * dose norm (global mode) and the cutoff use the reference doses.  Both
 * buffers are borrowed device float32 arrays; gamma_run writes nz*ny*nx
 * reference-grid values.  Identical geometries give an ordinary handle (the
 * coincident-grid search).  Options: "timing", "fp64_tau_exp10", "walk", "table_cap",
 * "lanes_per_voxel" (lanes that walk one reference voxel's cells together,
 * default 8).
 * Errors: INVALID_ARG, SHAPE, OOM, CUDA.  Synchronous. */
int gamma_create_grids(gamma_handle *out, const float *ref_dev, const float *eval_dev, int ndim,
                       const int64_t ref_shape[3], const float ref_spacing_mm[3],
                       const float ref_origin_mm[3], const int64_t eval_shape[3],
                       const float eval_spacing_mm[3], const float eval_origin_mm[3],
                       const gamma_criteria *crit);

/* Point an existing handle at a new dose pair of the same geometry (device,
 * borrowed).  Errors: INVALID_ARG. */
int gamma_set_inputs(gamma_handle h, const float *ref_dev, const float *eval_dev);

/* Compute the gamma map (Algorithm A1 step 4 / A2 steps 2-7) on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  gamma_out_dev: device,
 * float32, nz*ny*nx, written in full (NaN where not evaluated); the caller
 * owns it.  Stream-ordered: returns once the work is queued, without
 * synchronising and without allocating.  Errors: INVALID_ARG, CUDA. */
int gamma_run(gamma_handle h, float *gamma_out_dev, void *cuda_stream);

/* gamma_run on host buffers: copies ref_host and eval_host (float32, nz*ny*nx
 * each) to the handle's own device buffers, runs, and copies the gamma map
 * back into gamma_out_host.  Only for handles created with NULL device inputs.
 * Stream-ordered like gamma_run: the host buffers must stay valid until
 * `cuda_stream` reaches the end of the run (for example until gamma_pass_rate
 * returns).
 * When all three buffers are page-locked and mapped (cudaHostAlloc /
 * cudaMallocHost / pinned tensors) and option "pipeline" is not 0, the
 * copies overlap the search: the reference dose is copied first and reduced
 * while the evaluation dose follows in z slabs; the shell starts as soon as
 * the dose norm is known, each of its tiles waiting (bounded) for the slabs
 * that hold the slices it reads, which a stream write after each slab's copy
 * announces; the map is copied out while the queued voxels are
 * searched, and a kernel then writes their final values into gamma_out_host
 * through its mapped address.  That work runs on two streams the handle
 * owns, ordered after all earlier work on `cuda_stream`, which in turn waits
 * for it.  Otherwise (pageable buffers, option "design"
 * or an attached model) every step runs in order on `cuda_stream`.
 * Errors: INVALID_ARG, CUDA. */
int gamma_run_host(gamma_handle h, const float *ref_host, const float *eval_host,
                   float *gamma_out_host, void *cuda_stream);

/* Pass rate of the last run: rate = n_pass / n_eval (0 when n_eval = 0),
 * pass iff gamma <= 1.  Synchronises the last run's stream.  Any output
 * pointer may be NULL.  Errors: NOT_RUN, NAN_INPUT (the last run saw a
 * non-finite dose; its results are meaningless), QUEUE_FULL, DOSE_NORM
 * (global criteria, no positive dose norm: no voxel evaluated; on a batch
 * handle, any pair), CUDA. */
int gamma_pass_rate(gamma_handle h, double *rate, int64_t *n_eval, int64_t *n_pass);

/* Counters of the last run (synchronises its stream).  Errors: NOT_RUN, CUDA. */
int gamma_get_stats(gamma_handle h, gamma_stats *out);

/* Phase times of the last run (needs option "timing" = 1 before the run;
 * synchronises its stream).  Errors: NOT_RUN, INVALID_ARG (timing was off),
 * CUDA. */
int gamma_get_timings(gamma_handle h, gamma_timings *out);

/* Tuning and diagnostic options (take effect at the next run):
 *  "walk"             3 (default): voxel by voxel
 *                     from a queue ordered by cost; a cell that passes the
 *                     dose-gap test joins a per-warp buffer, and the warp
 *                     evaluates 32 such cells at a time, one per lane; the
 *                     most expensive voxels walk 4 lanes each (options
 *                     "group_bucket", "group8_bucket"; "lanes_per_voxel" does
 *                     not apply).  0: voxel by voxel, "lanes_per_voxel" lanes
 *                     each, every lane evaluating its own cells
 *                     (gamma_run_noalloc always walks this way; batch handles
 *                     take 0 or 3 only); 1: tile by
 *                     tile: each block stages the evaluation doses around one
 *                     256-voxel tile in shared memory (one TMA copy) and walks
 *                     the table for that tile's queued voxels, the lanes per
 *                     voxel chosen per tile; 2: row by row: each warp
 *                     independently takes one 32-voxel row of a shell tile
 *                     with queued voxels, stages the doses around it in shared
 *                     memory (one TMA copy) and walks the table for the row's
 *                     queued voxels.  Every walk gives the same map.  Handles
 *                     of gamma_create_grids take 0 (default: lanes_per_voxel
 *                     lanes per reference voxel, each lane evaluating its own
 *                     cells) or 3 (cells evaluated 32 at a time by the warp,
 *                     8 lanes per voxel; same map, slower on the measured
 *                     two-grid workloads).
 *  "group_bucket"     "walk" 3: queued voxels whose cost bucket (1 + floor(2
 *                     log2 of the cells below their starting bound)) is at
 *                     least this value walk 4 lanes each, the rest one lane
 *                     each (default 9; 32: every voxel one lane).  -1: the
 *                     walk chooses this and the next two thresholds from the
 *                     queue: with c(b) = 2^((2b - 1)/4) cells per voxel of
 *                     bucket b and T = (sum of c over the queue) / (the
 *                     walk's lanes), a voxel walks 4 lanes above s T cells,
 *                     8 above 4 s T and 32 above 8 s T (s = group_auto_pct
 *                     / 100, default 100).  gamma_autotune keeps whichever of
 *                     the two runs faster.
 *  "group8_bucket"    "walk" 3, group_bucket >= 0: ... and those of this
 *                     bucket and above 8 lanes each (default 32: none)
 *  "group32_bucket"   "walk" 3, group_bucket >= 0: ... and those of this
 *                     bucket and above 32 lanes, a whole warp, each (default
 *                     32: none)
 *  "group_auto_pct"   the slack s of the automatic choice, in percent
 *  "lanes_per_voxel"  2, 4, 8, 16 or 32 lanes search one queued voxel together
 *                     (the voxel-by-voxel walk, "walk" 0)
 *  "table_cap"        maximum cell-table length (rebuilds the table)
 *  "fp64_tau_exp10"   FP64 redo when the normalised Gram determinant
 *                     det(G)/prod(G_ii) < 10^-value; value <= 0 disables it
 *  "stats"            1: count cells in the tail search (slower)
 *  "sort_tail"        0: process queued voxels in discovery order instead
 *                     of most-expensive-first (ablation)
 *  "timing"           1: record per-phase CUDA events (gamma_get_timings)
 *  "pipeline"         gamma_run_host on page-locked buffers: 1 to 8 overlaps
 *                     the copies with the search, the evaluation dose in that
 *                     many z slabs (default 8; 1: the shell waits for the
 *                     whole dose); 0 runs in order
 *  "graph"            0 launches directly instead of capturing and replaying
 *                     a CUDA graph (default 1).  Batch handles capture at
 *                     their first run (not with "timing"); single-pair
 *                     handles once gamma_run has run twice on the same
 *                     output with no option or input change between (not
 *                     with "timing", a model or "design")
 *  "shell_blocks_per_sm"  1 to 4: resident blocks per SM the key-0 cell
 *                     kernel's register budget is sized for (default 2)
 *  "tail_blocks_per_sm"   1 to 4: the same for the table-walk kernels
 *                     (default 2; lanes_per_voxel defaults to 8; 4 applies
 *                     to "walk" 3 only, the other walks take 3)
 *  "design"           ablation of the paper's GPU design (Algorithm A2;
 *                     single-pair handles): 0 this library's two-phase search
 *                     (default); 1 one thread per voxel in the order of a
 *                     radix sort by DD, walking the whole cell table with
 *                     every simplex of every cell; 2 the same without the
 *                     sort.  Same results; allocates 16 bytes per voxel.
 *  "seed_min_bucket"  with a model attached: only queued voxels whose cost
 *                     bucket (1 + floor(2 log2 cells with key < gamma0)) is
 *                     at least this get a proposal (default 13: >= 64 cells);
 *                     0 seeds every queued voxel
 *  "drop_slab_flag"   failure test: k + 1 leaves slab k's readiness flag
 *                     unwritten in overlapped runs, so that the gated shell's
 *                     bounded wait gives up (GAMMA_ERR_TIMEOUT); 0 (default)
 *  "face_eval"        design 1 / 2 only: 0 every face in closed form (the
 *                     paper's choice, Section 2.2); 1 the full simplices by
 *                     Ju's recursion (Section 2.1)
 * Errors: INVALID_ARG (unknown key or value), TABLE_TOO_LARGE, OOM. */
int gamma_set_option(gamma_handle h, const char *key, int64_t value);

/* Current value of a launch option (the ones gamma_autotune chooses and the
 * walk's queue parts): "lanes_per_voxel", "shell_blocks_per_sm",
 * "tail_blocks_per_sm", "walk", "group_bucket", "group8_bucket",
 * "group32_bucket", "group_auto_pct".  No counterpart in the paper.
 * Errors: INVALID_ARG (null pointer or unknown key). */
int gamma_get_option(gamma_handle h, const char *key, int64_t *value);

/* Release the handle and everything it owns (synchronises its last stream).
 * NULL is allowed. */
void gamma_destroy(gamma_handle h);

/* ---------------------------------------------------------------------------
 * Batched runs: many dose pairs of uneven size, geometry and criteria in one
 * sequence of persistent launches (prepare, key-0 cells, cost ordering,
 * table walk), grouped by dimension, with one queue of expensive voxels
 * ordered by (cost bucket, pair) across all pairs of a group, captured once
 * into a CUDA graph and replayed.  This scales the per-voxel independence of
 * the gamma search (Section 1) from one pair to many; the paper itself runs
 * one pair at a time (Algorithm A2).
 */
typedef struct {
    const float *ref_dev;      /* device, float32, (nz, ny, nx), borrowed */
    const float *eval_dev;     /* device, float32, same shape, borrowed */
    float *gamma_out_dev;      /* device, float32, nz*ny*nx, caller-owned */
    int ndim;                  /* 2 or 3 */
    int64_t shape[3];          /* (nz, ny, nx), nz = 1 for 2D */
    float spacing_mm[3];       /* (hz, hy, hx) */
    gamma_criteria crit;
} gamma_pair_desc;

/* Create a batch handle over 1 <= n_pairs <= 65535 descriptors (copied;
 * device buffers borrowed).  Each pair gets its own cell table and scratch;
 * the handle adds 6 bytes per voxel of all pairs for the shared work order.
 * Errors: INVALID_ARG, SHAPE, OOM, TABLE_TOO_LARGE, CUDA.  Synchronous. */
int gamma_batch_create(gamma_handle *out, int n_pairs, const gamma_pair_desc *pairs);

/* Compute every pair's gamma map on `cuda_stream`.  The first call (and the
 * first after an option change) captures the launch sequence into a CUDA
 * graph on a private stream; later calls replay it on `cuda_stream`.
 * Stream-ordered, no allocation after the first call.  Errors: INVALID_ARG,
 * CUDA.  gamma_pass_rate / gamma_get_stats on a batch handle report the
 * totals over all pairs. */
int gamma_batch_run(gamma_handle h, void *cuda_stream);

/* Pass rate and counts of one pair of the last batched run (synchronises).
 * Errors: INVALID_ARG (pair out of range or not a batch), NOT_RUN, NAN_INPUT,
 * QUEUE_FULL, DOSE_NORM, CUDA. */
int gamma_batch_pass_rate(gamma_handle h, int pair, double *rate, int64_t *n_eval,
                          int64_t *n_pass);

/* Counters of one pair of the last batched run (synchronises). */
int gamma_batch_get_stats(gamma_handle h, int pair, gamma_stats *out);

/* Autotuner: times the full run (single or batch handle) for every
 * combination of lanes_per_voxel in {2, 4, 8, 16, 32} (not varied for the
 * staged and the warp-evaluated walks, which take none), shell_blocks_per_sm
 * in {1, 2, 3, 4} and tail_blocks_per_sm in {1, 2, 3} ({1, 2, 3, 4} for the
 * warp-evaluated walk) (two warm-ups and `reps` timed
 * runs each, CUDA events on `cuda_stream`), keeps the fastest as the handle's
 * options and returns it (any output pointer may be NULL).  For the
 * warp-evaluated walk it then times the other choice of queue parts
 * ("group_bucket" fixed or -1, chosen from the queue) at those shapes and
 * keeps the faster.  gamma_out_dev receives the
 * gamma map of a single-pair handle (device, nz*ny*nx floats) and is ignored
 * for a batch handle.  Errors as for the runs. */
int gamma_autotune(gamma_handle h, float *gamma_out_dev, void *cuda_stream, int reps,
                   int64_t *lanes_per_voxel, int64_t *shell_blocks_per_sm,
                   int64_t *tail_blocks_per_sm, float *best_ms);

/* ---------------------------------------------------------------------------
 * Learned proposal (no counterpart in the paper).  A 375-128-128-4 network
 * (ReLU; BF16 weights on the tensor cores, FP32 accumulation) reads a
 * 5x5x5 patch of three normalised channels around a reference voxel --
 * (D_e - D_r(v))/dD, |grad D_e| dta/dD, |grad D_r| dta/dD -- and proposes the
 * offset of the nearest surface point (normalised units x/dta, y/dta, z/dta)
 * and log(gamma + 1e-3).  When a model is attached to a handle, every voxel
 * queued for the table walk gets an exact upper bound from the faces of the
 * cells around the proposed point before the walk; the walk itself is
 * unchanged, so results stay exact.
 */
typedef struct gamma_model_s *gamma_model;

/* New model with He-normal weights drawn from `seed`.  Errors: OOM, CUDA. */
int gamma_model_create(gamma_model *out, uint64_t seed);
void gamma_model_destroy(gamma_model m);
/* Number of FP32 parameters (fixed layout: W1[128][384], b1[128], W2[128][128],
 * b2[128], W3[8][128], b3[8]; padding entries stay zero). */
int64_t gamma_model_num_params(void);
/* Copy parameters (which = 0), gradients of the last backward (1) or the Adam
 * moments (2, 3) to host memory of n = gamma_model_num_params() floats. */
int gamma_model_get_params(gamma_model m, float *host, int64_t n, int which);
int gamma_model_set_params(gamma_model m, const float *host, int64_t n);
/* Forward a batch: X_bf16_dev is M x 384 bfloat16 (device), Y_dev M x 4 float. */
int gamma_model_forward(gamma_model m, const void *X_bf16_dev, int64_t M, float *Y_dev,
                        void *cuda_stream);
/* Inference with the kernel the search uses: the three layers on the
 * fifth-generation tensor cores (tcgen05.mma, BF16 operands, FP32
 * accumulation in tensor memory), 128 rows per tile.  X_bf16_dev is M x 384
 * bfloat16 (device, 16-byte aligned, row-major), Y_dev M x 4 float (device).
 * Synchronises the stream.  Errors: INVALID_ARG, CUDA, TIMEOUT (a bounded
 * wait for the tensor cores gave up). */
int gamma_model_infer(gamma_model m, const void *X_bf16_dev, int64_t M, float *Y_dev,
                      void *cuda_stream);
/* Gradients of the mean Huber loss (delta 1) against targets T_dev (M x 4
 * float, rows with a NaN last column are ignored); loss_out optional (host). */
int gamma_model_backward(gamma_model m, const void *X_bf16_dev, const float *T_dev, int64_t M,
                         float *loss_out, void *cuda_stream);
/* backward + one Adam step (beta 0.9 / 0.999, eps 1e-8) with learning rate lr. */
int gamma_model_train_step(gamma_model m, const void *X_bf16_dev, const float *T_dev, int64_t M,
                           float lr, float *loss_out, void *cuda_stream);
/* Binary weights file (magic "GAMMAMLP", version 1, shapes, Adam state). */
int gamma_model_save(gamma_model m, const char *path);
int gamma_model_load(gamma_model m, const char *path);

/* Features of the listed voxels of a handle's dose pair: X_bf16_dev gets
 * n x 384 bfloat16.  Global criteria with dose_norm <= 0 use the dose norm of
 * the handle's last run (run it first). */
int gamma_features(gamma_handle h, const uint32_t *voxels_dev, int64_t n, void *X_bf16_dev,
                   void *cuda_stream);
/* Training targets of the listed voxels from a finished gamma map of the same
 * handle: targets_dev gets n x 4 floats (nearest-point offset in normalised
 * units, log(gamma + 1e-3)); NaN rows for voxels not evaluated or beyond the
 * table. */
int gamma_labels(gamma_handle h, const float *gamma_map_dev, const uint32_t *voxels_dev,
                 int64_t n, float *targets_dev, void *cuda_stream);
/* Attach a model to a single-pair handle (borrowed; NULL detaches) or load one
 * from a file that the handle then owns. */
int gamma_set_model(gamma_handle h, gamma_model m);
int gamma_load_model(gamma_handle h, const char *path);

/* Measured FP32 fused multiply-add throughput of the current device, the
 * confirmation of the FP32 peak the search's roofline is quoted against
 * (SMs x 128 FP32 lanes x 2 FLOP x SM clock).  Every SM runs 2048 threads of
 * eight independent multiply-add chains; one launch of about a millisecond is
 * timed with CUDA events on `cuda_stream` after a warm-up launch, best of three.
 * tflops gets 2 FLOP per FMA over that time, ms (may be NULL) the time of the
 * best launch.  Allocates nothing; syncs the stream.  Returns
 * GAMMA_ERR_INVALID_ARG for a NULL tflops, GAMMA_ERR_CUDA on a CUDA failure. */
int gamma_measure_fp32_peak(double *tflops, double *ms, void *cuda_stream);

/* Static description of a status code. */
const char *gamma_strerror(int code);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char *gamma_last_cuda_error(void);

/* Library version string. */
const char *gamma_version(void);

/* ---------------------------------------------------------------------------
 * Allocation-free variant.  The paper has no counterpart: this entry point
 * exists for callers that must not have a library allocate device memory --
 * applications whose device memory is owned by their own pool allocator (a
 * treatment-planning or QA system, a deep-learning framework operator), for
 * which a hidden cudaMalloc/cudaFree would break their memory budget and may
 * implicitly synchronise the whole device.
 *
 * gamma_run_noalloc computes the same gamma map as gamma_create + gamma_run
 * (global or local criteria, cutoff, NaN outside it) without allocating any
 * memory: no cudaMalloc, cudaFree, or heap allocation.  Its scratch (counters,
 * cell table, queue) is one fixed device array inside the library, which every
 * GPU that loads the library holds (about 20.3 MB) until the process exits.
 *  ref_dev, eval_dev  device, float32, (nz, ny, nx) C-order, borrowed.
 *  gamma_out_dev      device, float32, nz*ny*nx, written in full; caller-owned.
 *  ndim, shape,       as in gamma_create; at most GAMMA_NOALLOC_MAX_VOXELS
 *  spacing_mm, crit   voxels (else GAMMA_ERR_TOO_LARGE).
 *  cuda_stream        cudaStream_t of the work (NULL = legacy default stream).
 *  n_eval, n_pass     optional (may be NULL); when either is given the call
 *                     synchronises the stream and returns the counts.
 * Every call shares the one scratch array and leaves its contents there:
 * calls whose GPU work overlaps (different streams, several host threads)
 * race on it and give wrong results, so serialise them.  The first call on
 * each device looks up the array's device address with that device current;
 * make it before any stream capture begins.  The cell table is built on the
 * host during the call and reaches the device inside the parameters of the
 * call's own launches, so nothing the call enqueues reads host memory after
 * it returns.  Voxels whose search runs past the GAMMA_NOALLOC_MAX_TABLE-entry
 * table finish with the exact box scan.  The launch shapes are the defaults
 * of a new handle.
 * Errors: INVALID_ARG, SHAPE, TOO_LARGE, NAN_INPUT and DOSE_NORM (only when
 * counts are requested), CUDA. */
#define GAMMA_NOALLOC_MAX_VOXELS 4194304
#define GAMMA_NOALLOC_MAX_TABLE 32768
int gamma_run_noalloc(const float *ref_dev, const float *eval_dev, float *gamma_out_dev, int ndim,
                      const int64_t shape[3], const float spacing_mm[3],
                      const gamma_criteria *crit, void *cuda_stream, int64_t *n_eval,
                      int64_t *n_pass);

#ifdef __cplusplus
}
#endif

#endif /* GAMMA_GB300_H */
