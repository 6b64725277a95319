/*
 * tfdp.h -- C ABI of the GB300 (sm_103a) t-FDP force-evaluation library.
 *
 * t-FDP is the force-directed graph layout of "Force-directed graph layouts
 * revisited: a new force based on the t-Distribution" (Zhong et al., arXiv
 * 2303.03964). One iteration computes, for every node i of an undirected graph
 * with n nodes and m edges:
 *
 *   frep(i) = sum_{j != i} (x_i - x_j) / (1 + |x_i - x_j|^2)^gamma
 *             repulsive t-force, Sec. 3.3 Eq. (replusive), Sec. 3.4 Eq. (repfK);
 *             exact O(n^2) sum, or the interpolation-based FFT ("ibFFT") of Sec. 3.4
 *   fatt(i) = alpha * sum_{j <-> i} (1 + beta / (1 + |x_i - x_j|^2)) (x_j - x_i)
 *             attractive force, Sec. 3.3 Eq. (newforce), weighted by alpha as in
 *             the resultant force of Sec. 3.3
 *   x_i    += D(i) * min(1, s_t / |D(i)|),   D(i) = frep(i) + fatt(i)
 *             position update (Sec. 3.1: the resultant force moves each node until
 *             convergence). The step s_t = s0 (s_min / s0)^(t / (T - 1)) is a reading:
 *             the paper gives no schedule.
 *
 * Conventions for every entry point:
 *   - Every call returns a tfdp_status; no C++ exception crosses the ABI.
 *   - Arrays of positions or forces are n x 2 row-major FP32 (x0, y0, x1, y1, ...),
 *     in the caller's node order.
 *   - Pointers flagged `on_device` are CUDA device pointers on the graph's device,
 *     otherwise host pointers. Input buffers are copied; the caller keeps ownership
 *     of every buffer it passes and may free it when the call returns (for async
 *     calls: once the call returns, host inputs have been consumed).
 *   - A graph owns its device memory; tfdp_destroy_graph frees it.
 *   - Calls on one graph are not thread-safe; different graphs are independent.
 *   - Work is enqueued on the CUDA stream given at creation (0 = legacy default).
 */
#ifndef TFDP_H
#define TFDP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TFDP_OK = 0,
    TFDP_ERR_INVALID_ARG = 1,   /* null pointer, negative size, unknown enum value */
    TFDP_ERR_BAD_GRAPH = 2,     /* edge id out of range, self-loop or duplicate edge */
    TFDP_ERR_PARAM_RANGE = 3,   /* gamma <= 1, alpha < 0, beta < 0, bad k or grid cap */
    TFDP_ERR_OUT_OF_MEMORY = 4, /* device or host allocation refused */
    TFDP_ERR_CUDA = 5,          /* a CUDA runtime call failed (see tfdp_last_cuda_error) */
    TFDP_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    TFDP_ERR_BUSY = 7,          /* the object is in use by another request */
    TFDP_ERR_DEVICE_CHECK = 8   /* a device-side consistency check failed */
} tfdp_status;

/* How the repulsive sum is evaluated. */
typedef enum {
    TFDP_REP_EXACT = 0, /* tiled all-pairs sum of Eq. (repfK), Sec. 3.4 "exact method" */
    TFDP_REP_FFT = 1,   /* interpolation-based FFT of Sec. 3.4 */
    TFDP_REP_AUTO = 2   /* whichever of the two has the shorter estimated iteration for the
                         * graph's n (Sec. 4.1 "Runtime Performance" finds the exact method
                         * faster than ibFFT below about 500 nodes on its hardware):
                         * the exact sum while 9 us + n^2 / 3.0e12 s <= 40 us + 15 us per doubling
                         * of the FFT size P above 512 (measured on GB300: the exact sum up to
                         * n ~ 9,600 at P = 512 and ~13,500 at P = 2048). Resolved when the graph
                         * is created and at each tfdp_set_params; tfdp_get_params reports the
                         * resolved mode, tfdp_graph_footprint sizes for it. tfdp_params_check
                         * checks AUTO parameters as for TFDP_REP_FFT. */
} tfdp_rep_mode;

/* Arithmetic of the grid convolution (the FFT step of Sec. 3.4). */
typedef enum {
    TFDP_PREC_FP32 = 0,  /* FP32 spread, FFT and interpolation */
    TFDP_PREC_BF16X3 = 1 /* the transforms along y and the spectral product as BF16
                            split-precision tensor-core products (hi x hi + hi x lo +
                            lo x hi, FP32 accumulation); FFT size 2048 only (grid_max
                            513..1024) and a fixed k, else TFDP_ERR_PARAM_RANGE */
} tfdp_precision;

/* Box side of the interpolation grid, Sec. 3.4 ("Choices of k"). Both policies take
 * the layout square [x_min, x_max]^2 (x_min / x_max = min / max over both
 * coordinates), N_int = min(max(n_int_min, ceil(L)), floor(grid_max / k)) with
 * L = x_max - x_min, and G = N_int * k grid nodes per axis.                       */
typedef enum {
    TFDP_GRID_PAPER = 0, /* h = L / N_int: recomputed, and the spectrum rebuilt, every iteration */
    TFDP_GRID_SNAP_H = 1 /* h = smallest 2^e (16 + j) / 16 >= L / N_int: the spectrum is
                            rebuilt only when h crosses a 1/16-octave step */
} tfdp_grid_policy;

#define TFDP_K_DYNAMIC 0

typedef struct {
    double alpha;        /* attraction weight (Sec. 3.3), default 0.1, >= 0 */
    double beta;         /* short-range attraction weight (Sec. 3.3), default 8, >= 0 */
    double gamma;        /* repulsion exponent (Sec. 3.3), default 2, > 1 (Eq. exponentcondiction) */
    int32_t k_interp;    /* interpolation nodes per box and axis, 1..3, default 3 (Sec. 3.4);
                          * TFDP_K_DYNAMIC (0): the paper's dynamic strategy (Sec. 3.4 "Choices
                          * of k"): k = 1 while t < floor(0.9 T), 2 while t < floor(0.95 T),
                          * then 3, with T = total_iters (FFT path; the boundaries are a
                          * reading). Buffers are sized for the largest need over k = 1..3. */
    int32_t n_int_min;   /* lower bound of N_int, default 50 (Sec. 3.4) */
    int32_t grid_max;    /* cap on G = N_int * k, default 1023; sizes the FFT: P = nextpow2(2 grid_max - 1) */
    int32_t grid_policy; /* tfdp_grid_policy, default TFDP_GRID_SNAP_H */
    int32_t rep_mode;    /* tfdp_rep_mode, default TFDP_REP_FFT (a graph holds EXACT or FFT) */
    int32_t precision;   /* tfdp_precision, default TFDP_PREC_FP32 */
    double step0;        /* s0, default 1.0 (layout units) */
    double step_min;     /* s_min, default 0.01 */
    int32_t total_iters; /* T of the step schedule, default 300 (Sec. 4.1 implies 300) */
    int32_t reserved[7]; /* must be zero */
} tfdp_params;

/* Per-graph diagnostics of the last completed iteration (synchronises the stream). */
typedef struct {
    int64_t iteration;        /* number of iterations done (next t) */
    double net_frep[2];       /* FP64 sum over nodes of frep(i); ~0 by antisymmetry */
    double grid_lo;           /* origin of the grid square */
    double grid_h;            /* box side */
    int32_t grid_n_int;       /* boxes per axis */
    int32_t grid_G;           /* grid nodes per axis */
    int32_t fft_P;            /* FFT size per axis */
    int32_t spectrum_builds;  /* how many times the kernel spectrum was (re)built */
    int32_t device_flags;     /* nonzero: a device-side check failed (bit field) */
    int32_t kernels_per_iteration; /* kernel launches of one iteration in the current mode */
    int32_t grid_k;           /* interpolation nodes per box and axis of that iteration */
    int32_t reserved[5];
} tfdp_stats;

/* Stages of one iteration, in launch order, for tfdp_get_stage_times. */
enum {
    TFDP_STAGE_SORT = 0,          /* FFT path: grid policy, box of each node, counting sort (4 kernels) */
    TFDP_STAGE_SPREAD = 1,        /* FFT path: Lagrange projection onto the grid */
    TFDP_STAGE_SPECTRUM = 2,      /* FFT path: kernel spectrum (returns at once when cached) */
    TFDP_STAGE_ROWS_FWD = 3,      /* FFT path: forward transform along x */
    TFDP_STAGE_COLS = 4,          /* FFT path: transform along y, spectral product, inverse */
    TFDP_STAGE_ROWS_INV = 5,      /* FFT path: inverse transform along x */
    TFDP_STAGE_GATHER_UPDATE = 6, /* FFT path: back-projection + update */
    TFDP_STAGE_EXACT = 7,         /* exact path: all-pairs repulsion */
    TFDP_STAGE_EDGE_UPDATE = 8,   /* exact path: attraction + update */
    TFDP_STAGE_ATTRACT = 9,       /* FFT path: attraction, on a second stream concurrent with stages 0-5 */
    TFDP_NUM_STAGES = 10
};

typedef struct tfdp_graph tfdp_graph;

/* Human-readable name of a status code (static storage). */
const char* tfdp_status_str(tfdp_status s);

/* Message of the last CUDA error seen by this thread's calls ("" if none). */
const char* tfdp_last_cuda_error(void);

/* Fill *out with the defaults: alpha 0.1, beta 8, gamma 2 (Sec. 3.3), k 3,
 * n_int_min 50 (Sec. 3.4), grid_max 1023, SNAP_H, FFT repulsion, FP32, s0 1,
 * s_min 0.01, T 300. */
tfdp_status tfdp_params_default(tfdp_params* out);

/* Check a parameter set against Sec. 3.3: gamma > 1 (Eq. exponentcondiction),
 * alpha >= 0, beta >= 0, 1 <= k <= 3, grid_max >= k, step0 >= step_min > 0,
 * total_iters >= 1. *weight_ok (may be NULL) is set to 1 iff alpha (1 + beta) < 1
 * (Eq. limitweight); a set that breaks only that soft condition is accepted. */
tfdp_status tfdp_params_check(const tfdp_params* p, int* weight_ok);

/*
 * Create a graph: n nodes, m undirected edges.
 *   edges   host, 2m int32 node ids (i0, j0, i1, j1, ...); copied. An id outside
 *           [0, n), a self-loop or a duplicate pair (in either order) gives
 *           TFDP_ERR_BAD_GRAPH. m = 0 is allowed (edges may then be NULL).
 *   xy0     host, n x 2 FP32 initial positions; copied. NULL: positions uniform in
 *           [-sqrt(n)/2, sqrt(n)/2]^2 from `seed` (SplitMix64 counter generator).
 *   params  NULL = defaults. grid_max and k_interp size the device buffers.
 *   stream  cudaStream_t to enqueue on (NULL = legacy default stream).
 *   out     receives the handle; untouched on error.
 * Allocates all device memory of the graph (positions, CSR, sort buffers, grids,
 * spectra) on the current device. n = 0 is allowed.
 */
tfdp_status tfdp_create_graph(int64_t n, int64_t m, const int32_t* edges, const float* xy0,
                              uint64_t seed, const tfdp_params* params, void* stream,
                              tfdp_graph** out);

/* Replace the parameters. Changing gamma, k_interp, grid policy or grid_max marks
 * the kernel spectrum stale (alpha and beta only enter the edge term, Sec. 3.3, and
 * never need it). A larger grid_max or k reallocates the grid buffers. Does not
 * reset the iteration counter. */
tfdp_status tfdp_set_params(tfdp_graph* g, const tfdp_params* p);
tfdp_status tfdp_get_params(const tfdp_graph* g, tfdp_params* out);

/* Overwrite all positions (n x 2 FP32, caller order). Asynchronous on the stream. */
tfdp_status tfdp_set_positions(tfdp_graph* g, const float* xy, int on_device);

/* Device-side checks. The synchronising calls tfdp_synchronize, tfdp_get_positions,
 * tfdp_eval_forces and tfdp_run report the device flags raised since their last report:
 * TFDP_ERR_TIMEOUT when a bounded device-side wait gave up, TFDP_ERR_DEVICE_CHECK for
 * any other failed check (a position that became NaN or infinite, a box or sorted slot
 * out of range). Outputs are written all the same; the flags are then cleared, the
 * visit order of the next iteration restarts from the caller order, and
 * tfdp_stats.device_flags keeps every flag seen. */

/* Copy positions (n x 2 FP32, caller order) out. Synchronises the stream. */
tfdp_status tfdp_get_positions(tfdp_graph* g, float* xy, int on_device);

/* Run `iters` >= 0 iterations, starting at the graph's iteration counter t (which
 * selects s_t); advances t by iters. Asynchronous: launches one captured CUDA graph
 * per iteration on the stream. Errors of earlier asynchronous work surface here or
 * in the next synchronising call. */
tfdp_status tfdp_iterate(tfdp_graph* g, int32_t iters);

/* Set / read the iteration counter t (warm restart, Sec. 5 "Global Refinement"). */
tfdp_status tfdp_set_iteration(tfdp_graph* g, int64_t t);

/* Evaluate frep and fatt (n x 2 FP32 each, caller order; either may be NULL) at
 * the current positions without moving any node. Synchronises the stream. */
tfdp_status tfdp_eval_forces(tfdp_graph* g, float* frep, float* fatt, int on_device);

/* Diagnostics of the last iteration or force evaluation. Synchronises the stream. */
tfdp_status tfdp_get_stats(tfdp_graph* g, tfdp_stats* out);

/* Bracket the stages whose bit (1 << TFDP_STAGE_*) is set in `mask` with CUDA events
 * in every iteration; 0 turns timing off. The events are recorded on a side branch
 * forked at each stage border (no kernel waits for them), so a stage's time runs from
 * the completion of the work before it to its own completion, and timing costs the
 * iteration well under 1 us. Changing the mask recaptures the iteration graphs at the
 * next tfdp_iterate. */
tfdp_status tfdp_set_stage_timing_mask(tfdp_graph* g, uint32_t mask);

/* tfdp_set_stage_timing_mask with every stage (enable != 0) or none (enable = 0). */
tfdp_status tfdp_set_stage_timing(tfdp_graph* g, int enable);

/* Device time in ms of each stage of the most recent iteration or force evaluation
 * run with stage timing on; ms has nstages entries indexed by TFDP_STAGE_*; stages not
 * timed or not run in the current mode are 0. Synchronises the stream.
 * TFDP_ERR_INVALID_ARG if timing is off. */
tfdp_status tfdp_get_stage_times(tfdp_graph* g, float* ms, int nstages);

/* Upload positions, run `iters` iterations and download the result in one call (the
 * end-to-end form of tfdp_set_positions + tfdp_iterate + tfdp_get_positions, with one
 * host synchronisation at the end).
 *   xy_in   2n floats, caller order, host memory; NULL keeps the current positions
 *   iters   >= 0 iterations (Sec. 3.1 loop with the step schedule of the parameters)
 *   xy_out  2n floats, host memory, receives the positions after the iterations; may
 *           equal xy_in. Page-locked (pinned) buffers make both copies DMA transfers.
 * TFDP_ERR_INVALID_ARG for a NULL graph or xy_out, iters < 0. */
tfdp_status tfdp_run(tfdp_graph* g, const float* xy_in, int32_t iters, float* xy_out);

/* Local refinement (Sec. 5 "Local Refinement", fisheye views): per-node weights. The
 * repulsion between nodes i and j is scaled by w_rep[i] * w_rep[j] and the attraction
 * along edge (i, j) by w_att[i] * w_att[j]. The paper describes the effect (stronger
 * attraction between focal nodes and their neighbours, stronger repulsion elsewhere),
 * not a formula; the products are a reading that keeps the forces the negative gradient
 * of one energy. Both paths (exact and ibFFT) apply them; the ibFFT spreads r_j as the
 * charge of node j.
 *   w_rep, w_att  n floats each in caller order, in host memory (on_device = 0) or device
 *                 memory (on_device = 1), finite and in [0, TFDP_WEIGHT_MAX]; NULL resets
 *                 that kind to 1 (the plain method). Copied; the caller keeps ownership.
 * Takes effect from the next iteration or force evaluation (synchronises the stream and
 * recaptures the iteration graphs). The library keeps up to 12 n bytes for the weights,
 * which tfdp_graph_footprint does not count. TFDP_ERR_PARAM_RANGE if a weight is out of
 * range (nothing changes). Batches and served jobs take no weights. */
#define TFDP_WEIGHT_MAX 64.0f
tfdp_status tfdp_set_node_weights(tfdp_graph* g, const float* w_rep, const float* w_att, int on_device);

/* Wait for all work queued on the graph's stream. */
tfdp_status tfdp_synchronize(tfdp_graph* g);

/* Move the graph to another CUDA stream (waits for the work queued on the old one). */
tfdp_status tfdp_graph_set_stream(tfdp_graph* g, void* stream);

/* Device bytes tfdp_create_graph would allocate for n nodes, m edges and `params`
 * (NULL = defaults): an upper bound, above the allocation by at most a few KB plus
 * 4 bytes per node of degree <= 32 counted in the bound 2m/33 on the hubs (the degrees
 * are not known here); used for admission by memory footprint. */
tfdp_status tfdp_graph_footprint(int64_t n, int64_t m, const tfdp_params* params, size_t* bytes);

/* Free the graph and its device memory (synchronises first). NULL is a no-op. */
tfdp_status tfdp_destroy_graph(tfdp_graph* g);

/*
 * Batches: many independent graphs advanced together (Sec. 3.4 ibFFT path for every
 * graph; the batching itself has no counterpart in the paper). Graphs keep their own
 * parameters, grids, spectra, state and iteration counters; the arithmetic per graph is
 * that of a single graph, so each graph's result equals its solo run. Graphs are grouped
 * into parts by (k_interp, FFT size); each call runs the parts one after another on the
 * stream, each as nine launches per iteration (one per phase, every launch spanning all
 * graphs of the part) or as one cooperative persistent launch for all its iterations
 * (tfdp_batch_set_phase_launches, tfdp_batch_autotune).
 */
typedef struct tfdp_batch tfdp_batch;

/*
 * Create a batch of num_graphs >= 1 graphs on the current device.
 *   n, m       per graph node and edge counts (n >= 1)
 *   edges      per graph host pointer to 2 m int32 ids (NULL allowed when m = 0)
 *   xy0        per graph host pointer to n x 2 FP32 initial positions
 *   params     NULL (defaults for all) or num_graphs parameter sets; rep_mode is forced
 *              to TFDP_REP_FFT; each graph has a fixed k_interp (1..3; TFDP_K_DYNAMIC
 *              gives TFDP_ERR_PARAM_RANGE) and FP32 precision; a graph's FFT size
 *              follows from its grid_max and k and must be <= 2048 (grid_max <= 1024),
 *              else TFDP_ERR_PARAM_RANGE. Graphs of the same (k, FFT size) share a part.
 *   stream     cudaStream_t for all work of the batch
 * Inputs are copied. Errors as for tfdp_create_graph.
 */
tfdp_status tfdp_batch_create(int32_t num_graphs, const int64_t* n, const int64_t* m,
                              const int32_t* const* edges, const float* const* xy0,
                              const tfdp_params* params, void* stream, tfdp_batch** out);

/* Run `iters` iterations of every graph (per part: 9 iters launches or one persistent
 * launch, replayed from a captured CUDA graph). Asynchronous on the batch's stream. */
tfdp_status tfdp_batch_iterate(tfdp_batch* b, int32_t iters);

/* Forces of graph `graph` at the current positions (the whole batch is evaluated
 * once, no node moves); frep / fatt n x 2 FP32, either may be NULL. Synchronises. */
tfdp_status tfdp_batch_eval_forces(tfdp_batch* b, int32_t graph, float* frep, float* fatt,
                                   int on_device);

/* Positions of graph `graph` (n x 2 FP32, caller order). Synchronises. */
tfdp_status tfdp_batch_get_positions(tfdp_batch* b, int32_t graph, float* xy, int on_device);

/* Diagnostics of graph `graph` (as tfdp_get_stats). Synchronises. */
tfdp_status tfdp_batch_get_stats(tfdp_batch* b, int32_t graph, tfdp_stats* out);

tfdp_status tfdp_batch_synchronize(tfdp_batch* b);
tfdp_status tfdp_batch_destroy(tfdp_batch* b);

/* CTAs of the cooperative launch of the largest part (all co-resident on the device),
 * 0 for NULL. */
int32_t tfdp_batch_grid_blocks(const tfdp_batch* b);

/* Number of parts (distinct (k_interp, FFT size) groups) of the batch, 0 for NULL. */
int32_t tfdp_batch_num_parts(const tfdp_batch* b);

/*
 * Grid autotuner for batches (points per cell and grid size of Sec. 3.4, per graph; the
 * tuning itself has no counterpart in the paper). For every graph it picks the
 * interpolation order k and the grid cap with the cheapest FFT (size first, then k) whose
 * repulsion error against the exact all-pairs sum of the same positions is at most
 * max(max_error_ratio x the error of the reference parameters `base` (NULL: defaults),
 * min_error_bound), measured on the GPU with the single-graph API (one exact and a few
 * FFT force evaluations per measured graph, O(n^2) for the exact one). The candidates are
 * every k = 1..3 at each FFT size below the reference's (grid cap P / 2), then the
 * reference itself. Graphs are grouped by size (half octaves of n); up to `probes` graphs
 * of each group are measured and the group takes the cheapest candidate that meets the
 * bound on every measured graph.
 *   out_params  num_graphs sets: `base` with k_interp and grid_max chosen per graph
 *   out_error   NULL or num_graphs values: the largest measured error of the chosen
 *               setting in the graph's group
 * Synchronises the current device's work it launches; allocates and frees temporary
 * graphs. TFDP_ERR_INVALID_ARG for bad pointers, probes < 1, max_error_ratio < 1 or
 * min_error_bound < 0.
 */
tfdp_status tfdp_batch_plan(int32_t num_graphs, const int64_t* n, const int64_t* m, const int32_t* const* edges,
                            const float* const* xy0, const tfdp_params* base, double max_error_ratio,
                            double min_error_bound, int32_t probes, tfdp_params* out_params,
                            double* out_error);

/* Launch-shape autotuner, per part: times `trials` force evaluations of the whole batch
 * as one cooperative persistent launch at each number of co-resident CTAs per SM the
 * kernel allows, and as nine ordinary launches per iteration (one per phase, one CTA per
 * work item, each kernel at its own occupancy), and keeps the fastest. *chosen_blocks
 * (may be NULL) receives the largest cooperative CTA count kept, 0 when every part runs
 * per-phase launches. Before the first call every part runs per-phase launches.
 * Synchronises; no node moves. */
tfdp_status tfdp_batch_autotune(tfdp_batch* b, int32_t trials, int32_t* chosen_blocks);

/* Launch shape of every part: on = 1 one launch per phase, on = 0 the cooperative
 * persistent launch (at the last CTA count the autotuner kept, else the occupancy
 * limit). The results do not depend on it. TFDP_ERR_INVALID_ARG unless on is 0 or 1.
 * Synchronises the batch's stream when the shape changes. */
tfdp_status tfdp_batch_set_phase_launches(tfdp_batch* b, int32_t on);

/* Number of parts that run one launch per phase, 0 for NULL. */
int32_t tfdp_batch_phase_parts(const tfdp_batch* b);

/*
 * Serving: interactive layout jobs with continuous batching. A job is a graph and a
 * queue of requests: its initial layout, then updates (new alpha, beta, gamma applied
 * to the current layout, with the step schedule restarted over the update's
 * iterations: the warm-started re-layout of Sec. 5 "Global Refinement"). Jobs are
 * admitted in arrival order as soon as a slot is free and their device footprint
 * (tfdp_graph_footprint) fits the budget; admitted jobs keep positions and kernel
 * spectra resident, each on its own stream, and a worker thread advances all of them
 * by up to chunk_iters iterations per tick, so their kernels overlap on the device.
 * A job's result does not depend on the other jobs (the iteration is bitwise
 * reproducible). The batching has no counterpart in the paper.
 */
typedef struct tfdp_server tfdp_server;

typedef struct {
    int64_t request_id;
    int64_t job_id;
    int32_t kind;      /* 0: initial layout, 1: update */
    int32_t iters;
    double t_submit;   /* seconds since the server was created */
    double t_start;    /* first iteration queued */
    double t_done;     /* last iteration completed */
    int32_t status;    /* tfdp_status of the request */
    int32_t reserved;
} tfdp_done;

typedef struct {
    int32_t active;          /* admitted jobs */
    int32_t peak_active;
    int32_t waiting;         /* submitted, not admitted yet */
    int32_t jobs;            /* known jobs (admitted, waiting or finishing) */
    size_t used_bytes;       /* footprint of the admitted jobs */
    size_t budget_bytes;
    int64_t node_iterations; /* sum over completed iterations of the job's node count */
    int32_t reserved[8];
} tfdp_server_stats;

/* Start a server on the current device: admission budget in bytes, at most
 * max_active admitted jobs, chunk_iters iterations per job per scheduling tick. */
tfdp_status tfdp_server_create(size_t hbm_budget_bytes, int32_t max_active, int32_t chunk_iters,
                               tfdp_server** out);

/* Submit a job (inputs copied) whose first request lays it out for `iters` iterations
 * with `params` (NULL = defaults). TFDP_ERR_OUT_OF_MEMORY if its footprint exceeds the
 * whole budget. Returns its job id and the request id. Thread-safe. */
tfdp_status tfdp_server_submit(tfdp_server* s, int64_t n, int64_t m, const int32_t* edges,
                               const float* xy0, const tfdp_params* params, int32_t iters,
                               int64_t* job_id, int64_t* request_id);

/* Queue an update of a job: `params` (same k_interp, grid_max and rep_mode as the job)
 * with the step schedule restarted over `iters` iterations. Thread-safe. */
tfdp_status tfdp_server_update(tfdp_server* s, int64_t job_id, const tfdp_params* params,
                               int32_t iters, int64_t* request_id);

/* Take up to `max` completed requests (oldest first); waits up to wait_ms for one. */
tfdp_status tfdp_server_poll(tfdp_server* s, tfdp_done* out, int32_t max, int32_t* count,
                             int32_t wait_ms);

/* Positions of an admitted job with no request pending (n x 2 FP32, caller order);
 * TFDP_ERR_BUSY while it has work queued. */
tfdp_status tfdp_server_get_positions(tfdp_server* s, int64_t job_id, float* xy);

/* Free the job's slot and memory once its queued requests are done. */
tfdp_status tfdp_server_release(tfdp_server* s, int64_t job_id);

tfdp_status tfdp_server_get_stats(tfdp_server* s, tfdp_server_stats* out);

/* Stop the worker threads and free every job. */
tfdp_status tfdp_server_destroy(tfdp_server* s);

/*
 * Exact repulsion without any device allocation, for callers that cannot allocate:
 * code running under a framework whose caching allocator owns the device memory pool
 * and forbids side allocations, and latency-critical loops where cudaMalloc / cudaFree
 * could synchronise the device. The paper has no counterpart of this entry point. It
 * computes the exact all-pairs repulsion
 *     frep(i) = sum_{j != i} (x_i - x_j) / (1 + |x_i - x_j|^2)^gamma.
 *   xy      device pointer on the current device, n x 2 FP32 positions, 8-byte aligned
 *           (caller-owned, read only)
 *   n       0 <= n <= TFDP_NOALLOC_MAX_N, else TFDP_ERR_PARAM_RANGE
 *   gamma   > 1, else TFDP_ERR_PARAM_RANGE
 *   frep    device pointer on the current device, n x 2 FP32 output, 8-byte aligned
 *           (caller-owned)
 *   A NULL, misaligned, host or other-device pointer gives TFDP_ERR_INVALID_ARG before
 *   anything is launched.
 *   stream  cudaStream_t the two kernels are enqueued on (NULL = legacy default);
 *           the call returns once they are enqueued
 * Its only scratch is a fixed 2 MiB array of partial sums inside the library; every
 * GPU that loads the library holds it until the process exits. The call makes no
 * cudaMalloc, cudaFree or other allocating call. The first call on a device does a
 * one-time set-up (it looks up the device address of that array with the device
 * current); make that first call before any stream capture on the device. All calls
 * share the array: calls that can overlap on the GPU (other streams, other host
 * threads) race and corrupt each other's results, so order them (one stream, or
 * events). Each call overwrites every entry it reads, so no clearing is needed.
 */
#define TFDP_NOALLOC_MAX_N 16384
tfdp_status tfdp_exact_repulsion_noalloc(const float* xy, int64_t n, double gamma, float* frep,
                                         void* stream);

/*
 * Test hooks for failure detection (the paper has no counterpart). They make a failure
 * happen on the host, or as a bounded device-side wait that runs out; neither faults
 * the GPU.
 *   TFDP_INJECT_FFT_ALLOC   refuse the graph's next `value` FFT-buffer allocations as if
 *                           the device had no memory left (host side: nothing reaches
 *                           the device). The call that needed the buffers returns
 *                           TFDP_ERR_OUT_OF_MEMORY; an FFT-mode graph left without them
 *                           retries the allocation in its next tfdp_iterate or
 *                           tfdp_eval_forces and launches nothing until it succeeds.
 *   TFDP_INJECT_SCAN_STALL  value > 0: from the next iteration on, the first tile of the
 *                           box-count scan (the counting sort of Sec. 3.4's projection)
 *                           withholds its status word and every look-back wait gives up
 *                           after `value` polls, so the waits of the later tiles run out;
 *                           the kernel records this in the device flags and returns, and
 *                           the next synchronising call (tfdp_synchronize,
 *                           tfdp_get_positions, tfdp_eval_forces, tfdp_run) returns
 *                           TFDP_ERR_TIMEOUT. value = 0 restores normal operation.
 *                           Synchronises the stream.
 * TFDP_ERR_INVALID_ARG for an unknown `what` or value < 0.
 */
enum { TFDP_INJECT_FFT_ALLOC = 1, TFDP_INJECT_SCAN_STALL = 2 };
tfdp_status tfdp_debug_inject(tfdp_graph* g, int what, int value);

/*
 * Test hook: copy an internal buffer of the last FFT-mode force evaluation to host
 * memory `dst` of `bytes` bytes (TFDP_ERR_INVALID_ARG if too small or unknown).
 *   TFDP_DEBUG_GRID_CHARGES  3 x G x G FP32: rho, m_x, m_y (the spread, Sec. 3.4 step 1)
 *   TFDP_DEBUG_GRID_OUTPUT   G x G x 4 FP32: A, O_x, O_y, 0 (the grid interaction, step 2)
 *   TFDP_DEBUG_SORT_PERM     n int32: node id at each cell-sorted slot
 *   TFDP_DEBUG_CELL_START    N_int^2 + 1 int32: first sorted slot of each box
 * Synchronises the stream.
 */
enum {
    TFDP_DEBUG_GRID_CHARGES = 1,
    TFDP_DEBUG_GRID_OUTPUT = 2,
    TFDP_DEBUG_SORT_PERM = 3,
    TFDP_DEBUG_CELL_START = 4
};
tfdp_status tfdp_debug_fetch(tfdp_graph* g, int what, void* dst, size_t bytes);

#ifdef __cplusplus
}
#endif

#endif /* TFDP_H */
