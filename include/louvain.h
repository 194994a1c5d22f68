/*
 * louvain.h -- C ABI of the GB300 synchronous parallel Louvain library.
 *
 * Method: Forster, "Parallel Louvain Community Detection Optimized for GPUs"
 * (arXiv 1805.10904): the local-moving phase of Algorithm 1 (Eq. 1-5 with the
 * Sec. 3.1 minimum-label rules) repeated inside the multi-level driver of
 * Algorithm 2, with renumbering and graph induction after each level (Sec. 5.1.2).
 * Degree-one vertex following (a heuristic of Lu et al. that Sec. 7 refers to) is
 * applied before the first sweep of level 0.
 *
 * Arithmetic is exact: weights are integers >= 1, sums are int64, gains and
 * modularity are compared as int64 or int128 integers (Qn = (2W)^2 * Q), so the
 * labels returned are one deterministic function of the input.
 *
 * Conventions for every call:
 *   - Return value: LOUVAIN_OK (0) or one of the LOUVAIN_ERR_* codes below.  No call
 *     aborts, exits or traps; after an error the handle stays usable and
 *     louvain_last_error() describes the failure.
 *   - Streams are CUstream / cudaStream_t values passed as void*; NULL means the
 *     legacy default stream.  Every call returns only after its GPU work on that stream
 *     has completed.
 *   - Input arrays are borrowed for the duration of the call and never retained.
 *   - Results are owned by the library until louvain_result_free().
 */
#ifndef GB300_LOUVAIN_H
#define GB300_LOUVAIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define LOUVAIN_OK 0
#define LOUVAIN_ERR_INVALID_ARG 1  /* NULL pointer, negative size, bad config field        */
#define LOUVAIN_ERR_NOT_SYMMETRIC 2/* A_ij != A_ji (full checks only)                      */
#define LOUVAIN_ERR_DUPLICATE_EDGE 3 /* a row lists a column twice or unsorted (full checks) */
#define LOUVAIN_ERR_BAD_WEIGHT 4   /* a weight < 1 (Sec. 2: weights are positive)           */
#define LOUVAIN_ERR_INDEX_RANGE 5  /* row_ptr not monotone from 0, or a column outside [0,n) */
#define LOUVAIN_ERR_OOM 6          /* device or host allocation failed                      */
#define LOUVAIN_ERR_CUDA 7         /* a CUDA runtime call failed (message has the CUDA text) */
#define LOUVAIN_ERR_TIMEOUT 8      /* reserved: no call returns it (no device wait spins)    */
#define LOUVAIN_ERR_INTERNAL 9     /* a device-side consistency check failed                */
#define LOUVAIN_PENDING 10         /* serving: the ticket has not finished                   */
#define LOUVAIN_ERR_REJECTED 11    /* serving: request larger than the memory budget         */
#define LOUVAIN_ERR_TOO_LARGE 12   /* sum of weights above 2^62, or n above 2^31 - 1         */

/* pointer kinds of input arrays */
#define LOUVAIN_PTR_HOST 0   /* host memory: copied to the device inside the call (timed as e2e) */
#define LOUVAIN_PTR_DEVICE 1 /* device memory on the handle's device, read in place             */

/* ---------------------------------------------------------------- configuration */
typedef void *(*louvain_alloc_fn)(size_t bytes, void *ctx, void *stream);
typedef void (*louvain_free_fn)(void *ptr, void *ctx, void *stream);

typedef struct {
    uint32_t struct_size;      /* sizeof(louvain_config), set by louvain_config_init       */
    /* phase threshold theta as an exact rational (Algorithm 1 / Algorithm 2 threshold);
     * a sweep ends the level when (Qn_new - Qn_prev) * den < num * (2W)^2.              */
    int64_t theta_num;         /* default 1                                              */
    int64_t theta_den;         /* default 1000000                                        */
    int32_t max_iters;         /* sweeps per level cap, default 1000                     */
    int32_t max_levels;        /* default 64                                             */
    int32_t vertex_following;  /* 1 (default): degree-one following before level 0       */
    int32_t vf_all_levels;     /* 1: also before every later level; default 0            */
    int32_t checks;            /* 1 (default): index and weight checks; 2: also symmetry,
                                  sortedness and duplicates; 0 is treated as 1             */
    /* Widths, chosen per level from its largest weighted degree d_max and 2W: sweep gains
     * are int64 when d_max * 2W <= 2^62 (|gain of i| <= 2W * delta_i), else int128; sweep
     * table sums are 32-bit when d_max < 2^32 (e_{i->c} <= delta_i), induction sums when
     * 2W < 2^32 (a community's sum <= 2W); all exact.  The flags force the wide forms. */
    int32_t force_int128;      /* 1: int128 gains even when int64 is exact               */
    int32_t wide_sums;         /* 1: 64-bit table sums even when 32 bits are exact        */
    /* degree-bin thresholds on the row length d (entries stored in the row):
     *   d <= bin_small -> one thread per vertex            (0 <= bin_small <= 8)
     *   d <= bin_mid1  -> 8 lanes per vertex               (bin_mid1 <= 32)
     *   d <= bin_mid2  -> one warp per vertex              (bin_mid2 <= 128)
     *   d <= bin_cta1 / bin_cta2 / bin_cta3 -> one CTA of 128 / 256 / 1024 threads per
     *                     vertex with a shared-memory table of at least 4/3 d slots
     *                     (bin_cta3 <= 12288; lowered to 6144 when sums are 64-bit)
     *   d <= 2/4/8/16 * bin_cta3 -> a thread-block cluster of 2/4/8/16 such CTAs per
     *                     vertex, the table spread over the cluster's shared memory
     *                     (sizes the device cannot host are skipped)
     *   larger         -> CTA chunks of chunk_entries entries, merged by hash partition
     *                     of the neighbouring communities (graph induction: one global
     *                     table per long community).
     * Thresholds must not decrease.  All zero selects the defaults 8, 32, 128, 512, 2048,
     * 12288.  The same thresholds bin the communities (by entries) when coarsening. */
    int32_t bin_small;
    int32_t bin_mid1;
    int32_t bin_mid2;
    int32_t bin_cta1;
    int32_t bin_cta2;
    int32_t bin_cta3;
    int32_t chunk_entries;     /* power of two in [32, 4096]; 0 = default 4096           */
    int32_t profile;           /* 1: time kernel groups with CUDA events (louvain_result_counters) */
    int32_t cuda_graphs;       /* 1 (default): each phase's sweeps run as a CUDA graph whose  */
                               /* while node repeats sweep, controller and apply on the      */
                               /* device until the controllers stop (no host round trip per  */
                               /* sweep); 0, or profile = 1: one host round trip per sweep   */
    int32_t autotune;          /* 1: louvain_run picks the bin thresholds and chunk length  */
                               /* by measurement (louvain_autotune) on the first graph of   */
                               /* each (n, nnz) and reuses them; the results do not change */
    int32_t threshold_mode;    /* 0 (default): absolute phase test (Qn_new - Qn_prev) < theta */
                               /* * (2W)^2; 1: the relative test printed in Algorithm 1,    */
                               /* |Q_new - Q_prev| / |Q_prev| < theta (Q_prev = 0 stops only */
                               /* when Q is unchanged); the outer test of Algorithm 2 is    */
                               /* absolute in both modes                                    */
    int32_t post_merge;        /* 1: after every phase, a vertex whose non-loop neighbours  */
                               /* all lie in one other community joins it if that move's    */
                               /* Eq. 4 gain is positive (Sec. 5.1.2); the level then       */
                               /* records the merged state and its modularity; 0 (default) */
    int32_t keep_coarse;       /* 1: a one-graph run keeps the graph induced after every    */
                               /* recorded level (louvain_result_coarse_graph), so a run   */
                               /* can be resumed from it (louvain_resume)                   */
    int32_t sweep_streams;     /* streams the degree bins of one sweep run on side by side */
                               /* (0..4; default 4; 0 or 1: one after another)             */
    int32_t part_keys;         /* rows spanning several chunks are merged by partition: the */
                               /* expected distinct keys per partition (64 .. 2^30; 0 or */
                               /* the default 2048); larger means fewer partitions      */
    int32_t coloring;          /* 1: Lu et al.'s colouring heuristic, which Sec. 7 names    */
                               /* among the parallel heuristics it builds on: each level's */
                               /* graph gets a distance-1 colouring (Jones-Plassmann      */
                               /* rounds, priorities from SplitMix64's output function of */
                               /* the vertex id, smallest free colour) and a sweep takes  */
                               /* the colour classes in increasing colour, each deciding  */
                               /* on the state its predecessors left (louvain_run and     */
                               /* louvain_resume only); 0 (default): synchronous sweeps   */
    int32_t host_labels;       /* 1: each recorded level's labels are copied to pinned host */
                               /* memory on a copy stream while the later levels run (the */
                               /* pinned blocks are kept by the handle for its next runs, */
                               /* and outlive it while a result uses them); the run returns */
                               /* with every copy done, louvain_result_labels returns that */
                               /* memory and louvain_result_labels_into copies from it on  */
                               /* the host; 0 (default): labels stay on the device until  */
                               /* first asked for                                          */
    /* device memory: both NULL means stream-ordered cudaMallocAsync/cudaFreeAsync */
    louvain_alloc_fn alloc;
    louvain_free_fn free;
    void *alloc_ctx;
} louvain_config;

/* Fill *cfg with the defaults above.  Returns LOUVAIN_ERR_INVALID_ARG for NULL. */
int louvain_config_init(louvain_config *cfg);

/* ---------------------------------------------------------------- handle */
typedef struct louvain_handle louvain_handle;
typedef struct louvain_result louvain_result;

/* Create a handle bound to CUDA device `device`.  cfg may be NULL (defaults); it is
 * copied.  On success *out owns the handle (free with louvain_destroy). */
int louvain_create(const louvain_config *cfg, int device, louvain_handle **out);

/* Release the handle; NULL is ignored.  Results created from it must be freed first. */
void louvain_destroy(louvain_handle *h);

/* Text of the last error on this handle ("" if none).  Valid until the next call. */
const char *louvain_last_error(const louvain_handle *h);

/* ---------------------------------------------------------------- single graph */
/* Run multi-level Louvain (Algorithm 2 around Algorithm 1) on one undirected graph
 * G(V, E, w) given as symmetric CSR (Sec. 2):
 *   n        number of vertices (0 <= n <= 2^31 - 1)
 *   row_ptr  int64[n + 1], row_ptr[0] = 0, non-decreasing; nnz = row_ptr[n]
 *   col_idx  int32[nnz], column ids in [0, n); both directions of every non-loop edge
 *            are stored, a loop (i, i) once; no column twice in a row
 *   weights  int32[nnz] >= 1, A_ij = A_ji; NULL means every weight is 1
 *   ptr_kind LOUVAIN_PTR_HOST or LOUVAIN_PTR_DEVICE for all three arrays
 *   stream   stream the work is ordered on
 * On success *out receives the result: one entry per recorded level, a level being
 * recorded when it merged at least two communities.  A graph that is not symmetric is
 * detected only with checks = 2; with checks = 1 its result is unspecified (every access
 * still stays in bounds).  A column repeated in a row is merged as one neighbour.
 * Errors: INVALID_ARG, INDEX_RANGE, BAD_WEIGHT, NOT_SYMMETRIC / DUPLICATE_EDGE
 * (checks = 2), TOO_LARGE, OOM, CUDA, INTERNAL. */
int louvain_run(louvain_handle *h, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                const int32_t *weights, int ptr_kind, void *stream, louvain_result **out);

/* Choose the degree-bin thresholds and chunk length for a graph by measurement (this
 * library's addition; the thresholds only decide which kernel handles a row, never a
 * result).  Each trial is a whole run with a candidate set in the handle's configuration,
 * timed with CUDA events around the run (best of two); a coordinate search over
 * {bin_small, bin_mid1, bin_mid2, bin_cta1, bin_cta2, bin_cta3, chunk_entries} keeps a
 * change when it is at least 2% faster.  The choice is cached on the handle per (n, nnz)
 * and used by louvain_run when autotune = 1.  Arguments as in louvain_run; bins_out gets
 * the seven values in that order, *best_ms the trial time of the choice (-1 on a cache
 * hit), *trials the trial runs made (0 on a cache hit); either may be NULL. */
int louvain_autotune(louvain_handle *h, int64_t n, const int64_t *row_ptr,
                     const int32_t *col_idx, const int32_t *weights, int ptr_kind, void *stream,
                     int32_t bins_out[7], double *best_ms, int32_t *trials);

/* ---------------------------------------------------------------- batch of graphs */
/* Largest number of graphs in one louvain_run_batch call. */
#define LOUVAIN_MAX_BATCH_GRAPHS 1048576

/* Run louvain_run on each of num_graphs independent graphs in one pass over the device:
 * every phase step (degree bins, sweeps, controller, renumbering, coarsening) is launched
 * once for all graphs that still have a phase at that level, and each graph's controller
 * (Algorithm 1 stopping rule) and outer test (Algorithm 2) run independently, so graph g's
 * result is identical -- labels, Qn, iterations, trace -- to louvain_run on graph g alone.
 * The method itself is defined for one graph; batching is this library's addition.
 *   graph_vptr  HOST int64[num_graphs + 1]: graph g owns vertices [graph_vptr[g],
 *               graph_vptr[g+1]) of the stacked CSR; graph_vptr[0] = 0, non-decreasing
 *               (empty graphs allowed), n = graph_vptr[num_graphs] <= 2^31 - 1
 *   graph_eptr  HOST int64[num_graphs + 1] or NULL: if given, must equal
 *               row_ptr[graph_vptr[g]] for every g (checked)
 *   row_ptr, col_idx, weights, ptr_kind, stream: one CSR over all n vertices exactly as in
 *               louvain_run (block-diagonal: column ids are global and must lie in the
 *               row's own graph range, else INDEX_RANGE)
 *   out         array of num_graphs result pointers; out[g] gets graph g's result, its
 *               labels numbered for graph g's own vertices 0..n_g-1.  Each result is
 *               freed with louvain_result_free (in any order).  Per-graph counters: [0]
 *               edge visits of that graph; the other counters and times describe the
 *               whole batch.
 * Device memory: as louvain_run for the stacked graph, plus (max_iters + 1) * num_graphs
 * * 24 bytes of trace and O(num_graphs) controller state.  Errors as louvain_run, plus
 * TOO_LARGE for num_graphs > LOUVAIN_MAX_BATCH_GRAPHS.  On error no result is returned. */
int louvain_run_batch(louvain_handle *h, int32_t num_graphs, const int64_t *graph_vptr,
                      const int64_t *graph_eptr, const int64_t *row_ptr, const int32_t *col_idx,
                      const int32_t *weights, int ptr_kind, void *stream, louvain_result **out);

/* ---------------------------------------------------------------- serving */
/* A request loop on the handle for graphs that arrive over time (this library's addition;
 * the method itself is defined for one graph).  Submitted graphs wait in a FIFO queue and
 * are admitted while fewer than max_slots graphs are in flight and the sum of their
 * estimated device footprints (below) stays within hbm_budget_bytes.  An admitted graph is
 * copied to the device and checked on a stream of its own, then joins the graphs already
 * running at their next level boundary: every level step runs one set of launches for all
 * resident graphs (as louvain_run_batch does), and each graph keeps its own 2W, controllers
 * and outer test, so its result is identical to louvain_run on it alone.  When its run ends
 * its result is ready for louvain_poll and its slot and budget go back to the queue.
 * Footprint estimate: 8 (n + 1) + 8 nnz + 160 n + 40 nnz bytes.  Two native threads (upload
 * and engine) serve the handle; device memory comes from the handle's allocator on the
 * serving streams.  While serving is open, louvain_run and louvain_run_batch on this handle
 * return INVALID_ARG.  Errors: INVALID_ARG (already open, max_slots < 1, budget 0), CUDA,
 * OOM. */
int louvain_serve_open(louvain_handle *h, uint64_t hbm_budget_bytes, int max_slots);

/* Queue one graph (arrays as in louvain_run, HOST pointers only; they are copied before
 * the call returns).  *ticket identifies it for louvain_poll.  Errors: INVALID_ARG (not
 * serving, device pointers, closing), INDEX_RANGE (row_ptr[0] != 0 or row_ptr[n] < 0),
 * TOO_LARGE, OOM.  Graphs failing the checks of louvain_run (INDEX_RANGE, BAD_WEIGHT,
 * NOT_SYMMETRIC / DUPLICATE_EDGE with checks = 2, TOO_LARGE) and graphs whose footprint
 * exceeds the whole budget (REJECTED) report their error through louvain_poll. */
int louvain_submit(louvain_handle *h, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                   const int32_t *weights, int ptr_kind, uint64_t *ticket);

/* Wait up to wait_ms (0: do not wait, < 0: wait until done) for the graph of `ticket`.
 * Returns OK with *out = its result (freed with louvain_result_free; times_ms[3] of
 * louvain_result_counters is its submit-to-finish latency and times_ms[2] its wait for
 * admission), PENDING if it is not done yet (poll again), or the graph's error; a ticket is
 * consumed by the call that returns its outcome.  INVALID_ARG for an unknown ticket. */
int louvain_poll(louvain_handle *h, uint64_t ticket, int wait_ms, louvain_result **out);

/* status[0] = bytes admitted (footprints in flight), [1] slots in use, [2] graphs queued for
 * admission, [3] finished graphs not yet polled. */
int louvain_serve_status(const louvain_handle *h, int64_t status[4]);

/* Stop accepting graphs, finish every graph already submitted, free the results that were
 * never polled and end the request loop.  louvain_destroy closes an open loop itself. */
int louvain_serve_close(louvain_handle *h);

/* ---------------------------------------------------------------- checkpoint / resume */
/* With keep_coarse = 1 a one-graph run keeps, for every recorded level l that the run went
 * on from, the graph induced after it (the input of level l + 1; Sec. 5.1.2).  Its sizes:
 * louvain_result_coarse_graph (INVALID_ARG when level l has none); its arrays, copied into
 * caller buffers on the host or the device: louvain_result_coarse_copy (int64 row offsets
 * [n + 1], int32 columns [nnz], weights of weight_bytes 4 or 8 each [nnz]; NULL skips one). */
int louvain_result_coarse_graph(const louvain_result *r, int level, int64_t *n, int64_t *nnz,
                                int32_t *weight_bytes);
int louvain_result_coarse_copy(const louvain_result *r, int level, int64_t *row_ptr,
                               int32_t *col_idx, void *weights, int ptr_kind);

/* Continue a run from a saved level: the graph induced after level start_level - 1 (as
 * louvain_result_coarse_copy gives it; weights int32 or int64 by weight_bytes) and that
 * level's Qn (qn_prev, {high, low}) for the outer test of Algorithm 2.  The run computes
 * levels start_level, start_level + 1, ... exactly as the uninterrupted run did (vertex
 * following only with vf_all_levels, max_levels counted from level 0); the result's level
 * k is level start_level + k, its labels number the given graph's vertices, and its trace
 * carries the true level numbers.  Errors as louvain_run, plus INVALID_ARG for start_level
 * < 1 or >= max_levels. */
int louvain_resume(louvain_handle *h, int32_t start_level, const int64_t qn_prev[2], int64_t n,
                   const int64_t *row_ptr, const int32_t *col_idx, const void *weights,
                   int32_t weight_bytes, int ptr_kind, void *stream, louvain_result **out);

/* ---------------------------------------------------------------- edge-list input */
/* Symmetric CSR for louvain_run from an undirected edge list in any order (the neighbour
 * computation of Sec. 5.1.2: source-target pairs plus their reverses, sorted by source and
 * target, counted per source and prefix-summed into row offsets).  Reading of this
 * library: a pair (u, v, w) with u != v gives the entries (u, v) and (v, u); a loop (u, u)
 * gives one entry (u, u); entries with the same (row, column) are merged by adding their
 * weights; rows come out sorted by column.
 *   n          vertices (0 <= n <= 2^31 - 1; n = 0 needs m = 0)
 *   m          edges (0 <= m <= 2^40)
 *   src, dst   int32[m] endpoints in [0, n); weights int32[m] >= 1 or NULL (all 1);
 *              ptr_kind LOUVAIN_PTR_HOST (copied inside the call) or LOUVAIN_PTR_DEVICE
 *   row_ptr    DEVICE int64[n + 1], written
 *   col_idx, w_out  DEVICE int32, room for 2m entries; the first *nnz are the CSR, the rest
 *              is scratch of the call
 *   nnz        HOST int64 out
 * Work is ordered on `stream` and finished when the call returns.  Scratch is about 48
 * bytes per edge from the handle's allocator.  Errors: INVALID_ARG, INDEX_RANGE (an
 * endpoint outside [0, n)), BAD_WEIGHT, TOO_LARGE (a merged weight above 2^31 - 1, or the
 * size limits), OOM, CUDA. */
int louvain_csr_from_edges(louvain_handle *h, int64_t n, int64_t m, const int32_t *src,
                           const int32_t *dst, const int32_t *weights, int ptr_kind, void *stream,
                           int64_t *row_ptr, int32_t *col_idx, int32_t *w_out, int64_t *nnz);

/* ---------------------------------------------------------------- results */
/* Number of recorded levels (0 when nothing merged, e.g. no edges). */
int louvain_result_num_levels(const louvain_result *r);

/* Number of vertices of the input graph. */
int64_t louvain_result_num_vertices(const louvain_result *r);

/* Labels of the original vertices after level `level`, compacted to 0..ncomm-1 in the
 * order of the level's community labels (Sec. 5.1.2 renumbering).  *labels points to
 * n int32 values in host memory owned by r (copied from the device on first access, or
 * during the run with config.host_labels = 1), valid until r is destroyed.  ncomm may be
 * NULL. */
int louvain_result_labels(const louvain_result *r, int level, const int32_t **labels,
                          int64_t *ncomm);

/* Same labels copied into the caller's host buffer dst (n int32 values, any host memory;
 * the copy goes through a pinned staging buffer of the library, two 8 MB halves so the
 * transfer of one overlaps the host copy of the other).  Returns when dst is filled.
 * Errors: INVALID_ARG (bad level, dst NULL with n > 0), CUDA. */
int louvain_result_labels_into(const louvain_result *r, int level, int32_t *dst);

/* Same labels in device memory owned by r (no copy). */
int louvain_result_labels_device(const louvain_result *r, int level, const int32_t **labels);

/* Modularity of level `level` (Eq. 3): q = (double)Qn / (double)TW^2 with TW = 2W; the
 * exact values as int128 limbs {high (signed), low (bit pattern)}.  Any out pointer may be
 * NULL.  qn_init is Qn of the level's state before its first sweep. */
int louvain_result_modularity(const louvain_result *r, int level, double *q, int64_t qn[2],
                              int64_t qn_init[2], int64_t *tw);

/* Per-level counters: sweeps applied, vertices and stored entries of the graph the level
 * ran on, communities after it, and whether the sweep cap stopped it.  Any out pointer may
 * be NULL. */
int louvain_result_level_info(const louvain_result *r, int level, int32_t *iters,
                              int64_t *n_level, int64_t *nnz_level, int64_t *ncomm,
                              int32_t *hit_iter_cap);

/* Sweep trace in execution order over all phases run (recorded levels first, then the
 * final phase that merged nothing): for entry t, the level, the 1-based sweep index, the
 * vertices moved and Qn after the sweep (two int64 limbs per entry).  With all arrays NULL
 * it only returns the entry count through *len. */
int louvain_result_trace(const louvain_result *r, int64_t *len, int32_t *level, int32_t *iter,
                         int64_t *moved, int64_t *qn);

/* Work and time counters of the run:
 *   counters[0] edge visits: sum over phases of (sweeps applied) * nnz of the phase's graph
 *   counters[1] sweep kernels launched (including the one speculative sweep per phase
 *               whose moves are discarded, see louvain_run)
 *   counters[2] algorithmic bytes of all local-move sweeps: per sweep
 *               nnz * (4 column + s_w weight + 4 gathered label)
 *               + cand * 8 (deg of each distinct neighbouring community)
 *               + n * (8 row offset + 8 deg_i read for sum deg^2 + 4 label + 8 delta
 *                      + 8 deg of the own community + 4 proposed label)
 *               + (8 row offset + 4 list entry) per vertex of the list-driven kernels,
 *               s_w = 4 for int32 weights and 8 for int64
 *   counters[3] distinct neighbour communities summed over vertices and sweeps
 *   counters[4] kernels launched by the run
 * times_ms[0] local-move kernels (device time), [1] graph induction from its first to its
 * last kernel, [2] reserved, [3] wall time of louvain_run; [4] the dominant local-move kernel alone,
 * [5] the thread-per-vertex kernel, [6] the lane-group kernels, [7] the CTA, cluster and
 * chunk kernels; counters[5] launches of the dominant kernel, counters[6] its algorithmic
 * bytes, counters[7] the bin slot it serves (louvain_result_bin_stats numbering).
 * Arrays of 8; unused slots are zero.  Device times are filled only when the config had
 * profile = 1. */
int louvain_result_counters(const louvain_result *r, int64_t counters[8], double times_ms[8]);

/* Number of degree bins of the local-move sweep (see louvain_config's bin thresholds). */
int louvain_num_bins(void);

/* Statistics of degree bin `bin` summed over the sweeps of the run: device time of its
 * kernel (profile = 1 only, else 0), kernel launches, algorithmic bytes (formula of
 * louvain_result_counters), rows handled and stored entries of those rows.  Slots
 * 0 .. louvain_num_bins() - 1 cover every sweep but the first of each phase; slot
 * louvain_num_bins() + b covers bin b in the first sweep of each phase, which (when every
 * row of the phase's graph lists each column at most once: always after the first level,
 * and at the first level when every input row has strictly increasing columns) scores row
 * entries directly instead of aggregating them in tables, its candidates other than the
 * vertex's own community being distinct then.  Any out pointer may be NULL. */
int louvain_result_bin_stats(const louvain_result *r, int bin, double *time_ms,
                             int64_t *launches, int64_t *alg_bytes, int64_t *rows,
                             int64_t *entries);

/* Graph induction (Sec. 5.1.2 "Inducing new graph": the coarse graph of the communities,
 * A'_ab = sum of A_uv over C(u) = a, C(v) = b) summed over the run's levels:
 *   *inductions  coarse graphs built
 *   *alg_bytes   algorithmic bytes: per induction
 *                nnz * (4 column + s_w weight + 4 label of the target)
 *                + n * (8 row offset + 4 label of the member)
 *                + nnz' * (4 column + s_w' weight) + (n' + 1) * 8 new row offsets,
 *                for a fine graph of n vertices and nnz entries (s_w = 4 or 8) and a coarse
 *                graph of n' vertices and nnz' entries (s_w' = 4 when 2W < 2^31, else 8);
 *                the library's own temporaries are not counted.  In a batch these are the
 *                totals of every level step the graph took part in.
 *   *time_ms     device time from the first to the last induction kernel (profile = 1
 *                only, else 0)
 * Any out pointer may be NULL.  Errors: INVALID_ARG (r NULL). */
int louvain_result_coarsen_stats(const louvain_result *r, int64_t *inductions,
                                 int64_t *alg_bytes, double *time_ms);

/* How the result's level steps ran: info[0] sweeps run inside CUDA graphs (device-side
 * loop, cuda_graphs = 1), [1] sweeps run with one host round trip each (with cuda_graphs = 1
 * only the table-free first sweeps, see louvain_result_bin_stats), [2] engine level
 * steps, [3] sweep graphs captured, [4] autotuning trial runs made by this call, [5] 1 when
 * the bins came from the handle's autotuning cache.  For a batch or served graph the
 * numbers cover the steps it took part in. */
int louvain_result_exec_info(const louvain_result *r, int64_t info[6]);

/* Free a result and its host and device memory; NULL is ignored. */
void louvain_result_free(louvain_result *r);

/* ---------------------------------------------------------------- without allocation */
/* The paper has no counterpart to this entry point; it serves callers of this library
 * that cannot allocate device memory while they run -- for example a service whose GPU
 * memory is entirely reserved at start-up by another framework's allocator, or code that
 * must not trigger the device-wide synchronisation that cudaMalloc and cudaFree imply.
 *
 * louvain_modularity_noalloc computes the exact modularity (Eq. 3) of a caller-given
 * partition, like louvain_result_modularity reports it for the levels of a run, without
 * allocating anything: its scratch (one degree per community plus a few accumulators) is a
 * static device array of LOUVAIN_NOALLOC_MAX_VERTICES + 8 64-bit words (32 MiB + 64 bytes),
 * reserved on a GPU by the first call there (see below) and held until the process exits.
 *   n         vertices, 0 <= n <= LOUVAIN_NOALLOC_MAX_VERTICES, else LOUVAIN_ERR_TOO_LARGE
 *             (checked before any device work)
 *   row_ptr, col_idx, weights
 *             device CSR as for louvain_run (weights NULL = all 1), on the current device
 *   labels    device int32[n], community label of every vertex, each in [0, n)
 *   stream    stream the work is ordered on; the call returns after it completes
 *   qn, tw, q host outputs: Qn = (2W)^2 Q as int128 limbs {high, low}, 2W, and
 *             Q = (double)Qn / (double)(2W)^2 (0 when 2W = 0); any may be NULL
 * Errors: INVALID_ARG, TOO_LARGE (also 2^33 or more weighted entries, whose 64-bit sums
 * could wrap), INDEX_RANGE (row offsets, a column or a label out of range), BAD_WEIGHT,
 * CUDA (also when an error of the caller's earlier work is still pending on entry; it is
 * left pending).
 * First call on each device: it is the set-up.  CUDA loads this library's GPU code lazily,
 * so that call loads the code that holds the array -- which reserves the array's 32 MiB on
 * the device -- and looks up the array's device address with cudaGetSymbolAddress (the
 * current device must be the one the graph lives on).  A caller that reserves all of its
 * device memory up front must make this first call before doing so, and the first call
 * should come before any stream capture; every later call allocates nothing.  The call
 * synchronises its stream before it returns.  Every call on a device uses the same array
 * and clears the part it needs at its start, so calls whose GPU work overlaps (on
 * different streams or from different host threads) race and give wrong results. */
#define LOUVAIN_NOALLOC_MAX_VERTICES 4194304
int louvain_modularity_noalloc(int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                               const int32_t *weights, const int32_t *labels, void *stream,
                               int64_t qn[2], int64_t *tw, double *q);

/* ---------------------------------------------------------------- version */
/* ABI version of this header: 1. */
int louvain_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GB300_LOUVAIN_H */
