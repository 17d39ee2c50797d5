/*
 * blest.h -- C ABI of a GB300 (sm_103a) breadth-first search built on Binarised
 * Virtual Slice Sets (BVSS), after "BLEST: Blazingly Efficient BFS using Tensor
 * Cores" (Elbek and Kaya).
 *
 * Problem (Section 2, Background and Notation): for a graph G = (V, E) and a
 * source s, compute level[v] = length of a shortest s -> v path.  The search is
 * pull-only: with A the adjacency matrix of the transposed graph and x the
 * current frontier bit-vector, the next frontier is the Boolean SpMSpV
 * y = A (AND, OR) x, repeated until y = 0.  Several sources stack their frontiers
 * into a bit-matrix and the step becomes a Boolean SpMM.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns a blest_status; nothing aborts the process and no kernel
 *   traps.  blest_last_error() gives a human-readable message for the calling
 *   thread's last failure.
 * - Vertex ids are int32 in [0, n).  Levels are int32: 0 for a source, -1 for a
 *   vertex that no source reaches.  All outputs use the caller's ORIGINAL vertex
 *   ids; the internal reordering is undone on the device.
 * - Host pointers stay owned by the caller; the library copies what it keeps.
 *   Device pointers (the *_device calls) must be CUDA device memory of the
 *   current device, also caller-owned.
 * - A handle owns its device memory and one CUDA stream.  A handle is not
 *   re-entrant: calls on the same handle must not overlap in time.  Distinct
 *   handles may be used from distinct threads.
 * - The graph must be symmetric (u in N(v) iff v in N(u)).  Self-loops and
 *   duplicate entries are accepted and ignored; they do not change levels.
 *   Rows need not be sorted.
 */
#ifndef BLEST_H
#define BLEST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct blest_graph* blest_handle;

typedef enum {
    BLEST_OK = 0,
    BLEST_ERR_INVALID_ARG = 1,   /* bad pointer, size, id or option */
    BLEST_ERR_NOT_SYMMETRIC = 2, /* some edge (u, v) has no (v, u) */
    BLEST_ERR_TOO_LARGE = 3,     /* nnz >= 2^31, or more virtual slice sets than int32 holds */
    BLEST_ERR_OOM = 4,           /* device or host allocation failed */
    BLEST_ERR_CUDA = 5,          /* a CUDA runtime call failed (message in blest_last_error) */
    BLEST_ERR_TIMEOUT = 6,       /* a grid barrier gave up after the configured limit */
    BLEST_ERR_INTERNAL = 7       /* a device-side consistency check failed (e.g. queue overflow) */
} blest_status;

/* Vertex reordering applied before the BVSS build (Section 3.2). */
typedef enum {
    BLEST_ORDER_NONE = 0,       /* keep the input order */
    BLEST_ORDER_COMPRESS = 1,   /* pre-pass + JaccardWithWindows (Algorithm 1), for social-like graphs */
    BLEST_ORDER_BANDWIDTH = 2,  /* Reverse Cuthill-McKee, for non-social graphs (Section 3.2.1) */
    BLEST_ORDER_AUTO = 3        /* COMPRESS if social-like, else BANDWIDTH (Section 3.2.1 classifier) */
} blest_order;

/* Level-update scheme (Section 4.2). */
typedef enum {
    BLEST_UPDATE_AUTO = 0,      /* lazy iff the update divergence exceeds 25,000 (Section 5) */
    BLEST_UPDATE_EAGER = 1,     /* Algorithm 2: level write + returning atomicOr at each hit */
    BLEST_UPDATE_LAZY = 2       /* Algorithm 3: returnless mark, then a coalesced finalisation sweep */
} blest_update;

/* How a virtual slice set is pulled against its frontier word (Section 4.1). */
typedef enum {
    BLEST_PULL_POPC = 0,        /* CUDA cores: AND of each 8-bit mask with the frontier byte */
    BLEST_PULL_MMA = 1          /* two m8n8k128 b1 AND+POPC tensor-core MMAs per VSS (Figure 2c) */
} blest_pull;

/* Keys for blest_set_option.  Options apply to later traversals. */
typedef enum {
    BLEST_OPT_UPDATE = 0,            /* blest_update value */
    BLEST_OPT_PULL = 1,              /* blest_pull value */
    BLEST_OPT_BLOCKS_PER_SM = 2,     /* persistent-grid blocks per SM; 0 = as many as fit */
    BLEST_OPT_BARRIER_TIMEOUT_US = 3,/* grid-barrier wait limit in microseconds (default 2,000,000) */
    BLEST_OPT_RECORD_LEVELS = 4,     /* 1 = record the per-level queue sizes (blest_get_run_info) */
    BLEST_OPT_UNROLL = 5,            /* virtual slice sets a warp handles at once: 1, 2 (default) or 4
                                        (4 only with the 8-stage TMA ring) */
    BLEST_OPT_TEST_PHANTOM_BLOCK = 6,/* testing: 1 = every barrier waits for one block that does not
                                        exist, so the next traversal must end in BLEST_ERR_TIMEOUT */
    BLEST_OPT_VISITED_FILTER = 7,    /* 1 = test V_curr before marking a row; 2 = lazy update also skips
                                        rows already marked at this level: it tests V_next (which contains
                                        V_curr), read at L2, on levels where fewer than n/4 rows have a
                                        level, V_curr after; 3 = as 2 with V_next read through L1 (staler,
                                        cheaper); 4 (default) = V_next through L1 at every level; 0 = off;
                                        the eager update uses 1 for 2, 3 and 4 */
    BLEST_OPT_MIN_BLOCKS = 8,        /* kernel variant compiled for 2 (default) or 3 blocks per SM */
    BLEST_OPT_STAGE_DEPTH = 9,       /* lazy stage 1 prefetch: 0 = none; 2 (default) = the next group's
                                        tiles in registers while the current group's hits are handled; 3 =
                                        the next two groups' tiles; 4 or 8 = a per-warp TMA ring of that
                                        many stages in shared memory; used with BLEST_OPT_MIN_BLOCKS = 2 */
    BLEST_OPT_LAYOUT = 10,           /* BVSS layout read by the lazy register paths (stage depth 0 or 2,
                                        2 blocks/SM): 0 = every VSS padded to tau = 128 slices (Section
                                        3.1.2, default); 1 = compact groups of 4 slices, only the last
                                        group of a slice set padded (built from the padded layout on
                                        first use: about 5 B per slice more device memory) */
    BLEST_OPT_SCHEDULE = 11,         /* stage-1 work split of the register pipelines (stage depth 2, 3):
                                        0 = static, warp w takes queue entries w, w + W, ...;
                                        1 = on levels with at least 16 queue entries per warp, static
                                        for the first 7/8 of the queue, then warps take chunks of the
                                        rest from a per-level counter, sized (entries left) /
                                        (2 x warps) within [2 x unroll, 64] (guided); else as 0 (default) */
    BLEST_OPT_MS_PULL = 12,          /* multi-source pull: BLEST_PULL_POPC (default) ORs the frontier words
                                        the masks select on the CUDA cores; BLEST_PULL_MMA computes the
                                        same Boolean product with m16n8k128 b1 AND+POPC tensor-core MMAs */
    BLEST_OPT_MS_CHUNK = 13,         /* sources per multi-source launch (the k-tile): 64, 128 or 256
                                        (default); a call with more sources runs several launches */
    BLEST_OPT_MS_BLOCKS_PER_SM = 14, /* multi-source persistent-grid blocks per SM; 0 (default) = the
                                        value of BLEST_OPT_BLOCKS_PER_SM (0 = as many as fit) */
    BLEST_OPT_MS_LEVELS = 15,        /* how the multi-source traversal keeps levels until its output pass:
                                        1 = vertex-major (one entry per reached (vertex, source)), 2 = bit
                                        planes (plane p = bit p of every level; updated once per plane
                                        and distinct level at which a vertex gains bits), 0 (default) =
                                        planes on graphs the Section 5 rule updates lazily, else
                                        vertex-major */
    BLEST_OPT_MS_VISITED_FILTER = 16 /* multi-source marks: 1 = read the row's V_curr word and mark only
                                        sources that have not reached it; 2 (default) = read its V_next
                                        word instead (V_next contains V_curr: also skips sources marked
                                        at this level); 0 = mark every hit word (no dependent read; V_next
                                        still contains V_curr, so the levels are the same) */
} blest_option;

/* Creation parameters; pass NULL to blest_graph_create_ex for the defaults. */
typedef struct {
    int32_t window;          /* JaccardWithWindows window w, a multiple of 8 (default 65536, Section 5) */
    int32_t threads;         /* host threads for cleaning, the symmetry check, every ordering
                                (windows of JaccardWithWindows, large BFS levels of the pre-pass
                                and of RCM) and relabelling; 0 = all cores.  The result does
                                not depend on it. */
    int32_t skip_symmetry_check; /* 1 = trust the caller that the input is symmetric */
    int32_t prepass;         /* BLEST_ORDER_COMPRESS pre-pass before Algorithm 1: 0 = BFS from the
                                highest-degree vertices (default), 1 = Gorder (window 5, common
                                neighbours of degree <= 64 counted), slower, host only */
} blest_create_params;

/* Table 3 columns plus timings of the preprocessing, filled by blest_get_stats. */
typedef struct {
    int64_t n;                   /* vertices */
    int64_t nnz;                 /* directed entries after dropping self-loops and duplicates */
    int64_t num_slice_sets;      /* ceil(n / 8) */
    int64_t num_vss;             /* virtual slice sets */
    int64_t num_slices;          /* padded slices = 128 * num_vss */
    int64_t unpadded_slices;     /* non-empty slices */
    int64_t connectivity_bits;   /* 8 * unpadded_slices */
    double  update_divergence;   /* U_div (Section 3.2.1) */
    double  compression_ratio;   /* nnz / connectivity_bits (Section 3.2) */
    int64_t bvss_bytes;          /* device bytes of the four static arrays */
    int64_t state_bytes;         /* device bytes of queues, bitmaps and levels */
    int32_t order;               /* blest_order actually used */
    int32_t update;              /* blest_update the AUTO rule picks for this graph */
    double  order_seconds;       /* host reordering time (batch handles: the per-graph cleaning,
                                    checks, reordering and relabelling, graphs run concurrently) */
    double  build_seconds;       /* everything else in create (cleaning, upload, device BVSS build) */
} blest_stats;

/* What the last traversal on a handle did, filled by blest_get_run_info. */
typedef struct {
    int32_t levels;              /* BFS levels processed (the last one finds nothing new) */
    int32_t update;              /* blest_update used */
    int32_t pull;                /* blest_pull used */
    int32_t grid_blocks;         /* persistent-grid blocks */
    int32_t threads_per_block;
    int32_t recorded;            /* entries of the queue-size record below that are valid */
    int32_t output_path;         /* how levels reached the output: 0 written in place (no
                                    reordering), 1 written by the sweeps straight to their
                                    original ids (lazy with a reordering), 2 kept in BVSS ids
                                    and gathered by an unpermute pass */
} blest_run_info;

/* ---------------------------------------------------------------- graphs */

/* Build a handle for the symmetric CSR graph (row_ptr[n+1], col_idx[row_ptr[n]],
 * host memory, int32, row_ptr[0] = 0, non-decreasing).  Steps: clean (sort rows,
 * drop self-loops and duplicates), check symmetry, reorder (Section 3.2),
 * upload, build BVSS on the device (Section 3.1: slice sets of sigma = 8 columns,
 * virtual slice sets of tau = 128 slices, slices sorted by row and placed
 * lane-major, the last VSS of a slice set padded with zero masks), compute the
 * Table 3 statistics.  On failure *out is NULL.  n = 0 gives an empty handle.
 * Errors: INVALID_ARG (NULL pointer, n < 0, malformed row_ptr, id out of range),
 * NOT_SYMMETRIC, TOO_LARGE, OOM, CUDA. */
blest_status blest_graph_create(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                blest_order order, blest_handle* out);

/* Same, with explicit parameters (NULL = defaults). */
blest_status blest_graph_create_ex(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                   blest_order order, const blest_create_params* params,
                                   blest_handle* out);

/* Build one handle over the disjoint union of num_graphs graphs, for batched
 * traversal of many graphs in one persistent launch.  Graph g has n_each[g]
 * vertices and CSR (row_ptrs[g], col_idxs[g]) in its own local ids, and is
 * reordered with orders[g] inside its own id range; in the union, graph g's
 * vertices follow those of graphs 0..g-1.  The graphs are cleaned, checked and
 * reordered concurrently on the host threads of params (the handle does not
 * depend on their number).  Errors as blest_graph_create; the message names
 * the lowest-numbered graph that failed. */
blest_status blest_batch_create(int32_t num_graphs, const int32_t* n_each,
                                const int32_t* const* row_ptrs, const int32_t* const* col_idxs,
                                const int32_t* orders, const blest_create_params* params,
                                blest_handle* out);

/* Release the handle and all its device memory.  NULL is ignored. */
void blest_destroy(blest_handle h);

/* Set one option (blest_option key) for the handle's later traversals.
 * INVALID_ARG for an unknown key or a value outside the key's range; setting
 * BLEST_OPT_LAYOUT = 1 builds the compact layout first (OOM/CUDA on failure). */
blest_status blest_set_option(blest_handle h, int32_t key, int64_t value);

/* Copy the handle's statistics (Table 3 columns, timings) to *out (host,
 * caller-owned).  INVALID_ARG for NULL arguments. */
blest_status blest_get_stats(blest_handle h, blest_stats* out);

/* --------------------------------------------------------------- traversal */

/* Single-source BFS (Algorithms 2 and 3, fused into one persistent kernel per
 * traversal, Section 4.3).  levels: host memory of n int32, caller-owned,
 * written in original ids.  Blocks until done.
 * Errors: INVALID_ARG (NULL handle/levels, src outside [0, n)), TIMEOUT, INTERNAL, CUDA. */
blest_status blest_bfs(blest_handle h, int32_t src, int32_t* levels);

/* BFS tree (the parent-array form of Section 2) of the traversal from src:
 * levels as blest_bfs, and parents (host, n int32): parents[v] = the smallest
 * original id among the neighbours of v one level closer to src (a unique
 * choice), parents[src] = src, -1 for unreached vertices.  Computed by one
 * extra pass over the BVSS after the traversal.  Errors: as blest_bfs. */
blest_status blest_bfs_parents(blest_handle h, int32_t src, int32_t* levels, int32_t* parents);

/* k independent BFS runs from srcs[0..k) (host array), as one Boolean SpMM per
 * level over an n x k frontier bit-matrix (Section 2, multi-source form).
 * levels: host memory of k*n int32, row-major by source: levels[i*n + v] is the
 * level of v from srcs[i].  Duplicate sources are allowed.  k = 0 does nothing.
 * Sources run in launches of at most 256.  The handle keeps the device state of
 * the largest launch so far until blest_destroy: three bit matrices of n x W
 * 64-bit words (W = 1, 2 or 4 for up to 64, 128 or 256 sources), an n x k8 int32
 * level buffer (k8 = the launch's source count rounded up to 8), and 3 queues of
 * numVSS entries.  Errors: as blest_bfs. */
blest_status blest_msbfs(blest_handle h, const int32_t* srcs, int32_t k, int32_t* levels);

/* One BFS whose level-0 frontier is the whole set srcs[0..k) (host array):
 * levels[v] = distance from v to the nearest source.  On a batch handle, with
 * one source per graph, this is an independent BFS in every graph.
 * levels: host memory of n int32. */
blest_status blest_bfs_multiroot(blest_handle h, const int32_t* srcs, int32_t k, int32_t* levels);

/* Batch handle: one source per graph, srcs_local[g] in graph g's local ids;
 * levels: host memory of sum(n_each) int32, graph g's levels at the offset of g. */
blest_status blest_batch_bfs(blest_handle h, const int32_t* srcs_local, int32_t* levels);

/* Batch handle, CUDA-graph form: blest_batch_graph_capture records one batched
 * traversal (source upload from a pinned list, clears, the persistent kernel)
 * into a CUDA graph bound to d_levels (device, sum(n_each) int32, caller-owned,
 * must stay valid while the capture is used); blest_batch_graph_launch writes
 * new sources (srcs_local[g] in graph g's local ids) into the pinned list and
 * replays the graph on `stream` (NULL = the handle's stream) without waiting
 * for it.  A launch first waits until the previous replay has finished.
 * Completion and device status: blest_sync.  Errors: INVALID_ARG, CUDA. */
blest_status blest_batch_graph_capture(blest_handle h, int32_t* d_levels);
blest_status blest_batch_graph_launch(blest_handle h, const int32_t* srcs_local, void* stream);

/* Device-memory forms.  They enqueue the traversal on `stream` (a cudaStream_t;
 * NULL = the handle's own stream; pass cudaStreamLegacy for the legacy default
 * stream) and return without waiting; sources are host
 * arrays read before the call returns.  d_levels is device memory of n (or k*n)
 * int32.  The status of the traversal (TIMEOUT, INTERNAL) is reported by the
 * next blest_sync on the handle; a launch failure is reported at once. */
blest_status blest_bfs_device(blest_handle h, int32_t src, int32_t* d_levels, void* stream);
blest_status blest_msbfs_device(blest_handle h, const int32_t* srcs, int32_t k, int32_t* d_levels,
                                void* stream);
blest_status blest_bfs_multiroot_device(blest_handle h, const int32_t* srcs, int32_t k,
                                        int32_t* d_levels, void* stream);

/* Wait for every traversal enqueued on the handle and return the first device
 * status they reported (BLEST_OK if none failed). */
blest_status blest_sync(blest_handle h);

/* Checkpoint of a handle's preprocessed graph: the vertex order, the BVSS
 * arrays of Section 3.1, the batch boundaries and the statistics, so that
 * blest_graph_load skips the reordering and the build.  Binary file in this
 * library's format version 1 (magic "BLESTG1", native little-endian layout of
 * blest_stats); options, the compact layout and traversal state are not
 * saved.  blest_graph_save returns INVALID_ARG if the file cannot be written. */
blest_status blest_graph_save(blest_handle h, const char* path);

/* Reads a file written by blest_graph_save.  Every index in it (vertex order,
 * realPtrs, virtualToReal, VSS counts, row ids, mask bits against the columns
 * that exist) is checked against the header's sizes on the host before any
 * device memory is allocated; the first inconsistency returns INVALID_ARG with
 * a message.  *out is NULL on failure. */
blest_status blest_graph_load(const char* path, blest_handle* out);

/* Distance statistics of k single-source traversals, run as batched
 * multi-source traversals (the multi-source applications of Section 6:
 * closeness centrality and diameter).  For source srcs[i] (original id):
 * reached[i] = vertices at finite distance, the source included; sum_dist[i] =
 * the sum of those distances; ecc[i] = the largest (the source's eccentricity
 * within its component).  Closeness = (reached - 1) / sum_dist (0 for an
 * isolated source) and the diameter lower bound max_i ecc[i] follow from them.
 * All three outputs are host arrays of k entries, caller-owned.  Sources are
 * processed in batches of up to 256 whose level rows fit in 4 GiB of device
 * scratch allocated for the call; returns INVALID_ARG for a source out of
 * range (before any work), OOM if the scratch cannot be allocated. */
blest_status blest_distance_stats(blest_handle h, const int32_t* srcs, int32_t k, int64_t* reached,
                                  int64_t* sum_dist, int32_t* ecc);

/* Per-level queue sizes of the last traversal (recorded when
 * BLEST_OPT_RECORD_LEVELS = 1): queue_sizes[l-1] = virtual slice sets processed
 * at level l, up to cap entries.  Waits for the handle's work first. */
blest_status blest_get_run_info(blest_handle h, blest_run_info* info, int32_t* queue_sizes, int32_t cap);

/* Device timeline of the last single-frontier traversal (recorded when
 * BLEST_OPT_RECORD_LEVELS = 1), in globaltimer nanoseconds: times_ns[1] =
 * kernel entry, times_ns[0] = start of level 0's sweep; for level l >= 1,
 * times_ns[2l] = start of its stage 1 and times_ns[2l+1] = start of its
 * finalisation sweep (lazy only); for the last level L, times_ns[2L+2] = end
 * of the traversal and times_ns[2L+3] = end of block 0's share of the
 * unpermute epilogue.  Up to cap entries. */
blest_status blest_get_level_times(blest_handle h, uint64_t* times_ns, int32_t cap);

/* Load balance of the last single-frontier traversal (recorded with
 * BLEST_OPT_RECORD_LEVELS = 1): for level l >= 1, first_ns[l-1] and
 * last_ns[l-1] are the globaltimer stamps (ns) at which the first and the last
 * block of the persistent grid finished the level's stage 1 (phase 0) or its
 * finalisation sweep (phase 1, lazy levels only; entries of eager levels are
 * left at UINT64_MAX / 0); their gap is the time blocks wait at the level's
 * barrier for the slowest one.  Up to cap entries each; both arrays host,
 * caller-owned.  INVALID_ARG for another phase.  Waits for the handle's work. */
blest_status blest_get_level_arrivals(blest_handle h, int32_t phase, uint64_t* first_ns, uint64_t* last_ns,
                                      int32_t cap);

/* ---------------------------------------------------------------- autotune */

/* Result of blest_autotune: the options it kept and what they measured. */
typedef struct {
    int32_t update;              /* blest_update kept (EAGER or LAZY) */
    int32_t pull;                /* blest_pull kept */
    int32_t unroll;
    int32_t min_blocks;
    int32_t visited_filter;
    int32_t blocks_per_sm;       /* 0 = as many as fit */
    int32_t stage_depth;         /* BLEST_OPT_STAGE_DEPTH kept */
    int32_t layout;              /* BLEST_OPT_LAYOUT kept */
    int32_t schedule;            /* BLEST_OPT_SCHEDULE kept */
    int32_t candidates;          /* variants timed */
    double  best_ms;             /* mean device time per traversal of the kept variant */
    double  rule_ms;             /* same for the Section 5 rule (lazy iff U_div > 25,000), CUDA-core pull */
} blest_tune_result;

/* Time single-source traversal variants on the k host sources srcs[0..k)
 * with CUDA events, each variant after one untimed pass, and keep the fastest
 * as the handle's options.  Two stages: a few representative variants of the
 * eager and the lazy update (plus the Section 5 rule's plain kernel, reported
 * as rule_ms) pick the update scheme; then every variant of that scheme is
 * timed (pull back-end, unroll, occupancy variant, visited filter, blocks per
 * SM, prefetch depth, layout, schedule).  out may be NULL.
 * Errors: INVALID_ARG (k < 1, bad source), TIMEOUT, INTERNAL, CUDA. */
blest_status blest_autotune(blest_handle h, const int32_t* srcs, int32_t k, blest_tune_result* out);

/* As blest_autotune, but every timing is ONE traversal from all k roots at once
 * (the multi-root form: level = distance to the nearest root), which is the
 * launch a batch handle runs for its graphs (blest_batch_bfs and the captured
 * blest_batch_graph_launch; srcs are then union ids, one per graph).  best_ms
 * and rule_ms are per multi-root traversal.  A batch handle captured before the
 * call keeps the variant it was captured with: capture again afterwards. */
blest_status blest_autotune_multiroot(blest_handle h, const int32_t* srcs, int32_t k, blest_tune_result* out);

/* Result of blest_autotune_msbfs. */
typedef struct {
    int32_t pull;                /* BLEST_OPT_MS_PULL kept */
    int32_t chunk;               /* BLEST_OPT_MS_CHUNK kept (sources per launch) */
    int32_t blocks_per_sm;       /* BLEST_OPT_MS_BLOCKS_PER_SM kept (0 = as many as fit) */
    int32_t levels;              /* BLEST_OPT_MS_LEVELS kept (1 vertex-major, 2 bit planes) */
    int32_t visited_filter;      /* BLEST_OPT_MS_VISITED_FILTER kept */
    int32_t candidates;          /* variants timed */
    double  best_ms;             /* device time of one call over all k sources, kept variant */
    double  popc_ms;             /* best time with the CUDA-core pull */
    double  mma_ms;              /* best time with the tensor-core pull */
} blest_ms_tune_result;

/* Time multi-source traversal variants on one call over the k host sources
 * srcs[0..k) (Section 2's multi-source form) with CUDA events, each variant
 * after one untimed pass, and keep the fastest as the handle's options: pull
 * back-end (CUDA-core OR or b1 tensor-core MMA), sources per launch (64, 128,
 * 256; only sizes that change the launches of k sources), blocks per SM, level
 * layout and the visited test before the marks (the MMA back-end is timed with
 * bit planes and the test only).
 * Allocates a k x n device level buffer for the duration of the call.  out may
 * be NULL.  Errors: INVALID_ARG (k < 1, bad source), OOM, TIMEOUT, INTERNAL, CUDA. */
blest_status blest_autotune_msbfs(blest_handle h, const int32_t* srcs, int32_t k, blest_ms_tune_result* out);

/* ----------------------------------------------------------------- export */

/* Copy an internal array to host memory (bytes must equal the array's size,
 * which blest_export_size reports).  For tests and statistics. */
typedef enum {
    BLEST_ARRAY_REAL_PTRS = 0,       /* int32[num_slice_sets + 1] */
    BLEST_ARRAY_VIRTUAL_TO_REAL = 1, /* int32[num_vss] */
    BLEST_ARRAY_ROW_IDS = 2,         /* int32[128 * num_vss] */
    BLEST_ARRAY_MASKS = 3,           /* uint32[32 * num_vss] */
    BLEST_ARRAY_NEW_ID = 4,          /* int32[n]: new_id[original id] */
    BLEST_ARRAY_VSS_COUNT = 5,       /* int32[num_vss]: unpadded slices per VSS */
    /* compact layout (BLEST_OPT_LAYOUT = 1; exporting builds it): slice k of
       slice set s, in row order, is sub-slot k % 4 of group goff[s] + k / 4;
       the last group of a slice set is padded with its last row id, mask 0 */
    BLEST_ARRAY_COMPACT_OFFSETS = 6, /* int32[num_slice_sets + 1]: goff, goff[num_slice_sets] = groups */
    BLEST_ARRAY_COMPACT_ROWS = 7,    /* int32[4 * groups] */
    BLEST_ARRAY_COMPACT_MASKS = 8    /* uint32[groups]: byte q = mask of sub-slot q */
} blest_array;

int64_t blest_export_size(blest_handle h, int32_t which);
blest_status blest_export(blest_handle h, int32_t which, void* host_out, int64_t bytes);

/* ---------------------------------------------------------- host-only calls */

/* The vertex order blest_graph_create would use, without any GPU: new_id[v] =
 * position of v in the new order (the pi^-1 of Algorithm 1).  Same input rules
 * as blest_graph_create; new_id is host memory of n int32. */
blest_status blest_compute_order(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                 blest_order order, const blest_create_params* params,
                                 int32_t* new_id);

/* 1 if the Section 3.2.1 classifier calls the graph social-like, else 0;
 * negative blest_status on bad input. */
int32_t blest_is_social(int32_t n, const int32_t* row_ptr, const int32_t* col_idx);

/* ------------------------------------------------------ sharded traversal */

/* One rank's share of a single-source BFS whose pull is split over `world` ranks
 * (one GPU each) by slice set: rank r pulls only the queued VSSs of the slice
 * sets s with s mod world = r.  Between the pull and the finalisation sweep of
 * every level, the ranks combine their V_next words (the lazy marks of
 * Algorithm 3) with a bitwise OR; every rank then runs the same sweep on the
 * combined words, so all of them end with the full level array.  The paper
 * names multi-GPU BFS as future work (Section 6); this is that exchange step,
 * one n/32-word OR per level.  The caller owns the collective: an all-gather of
 * every rank's words followed by blest_shard_merge, or any all-reduce with
 * bitwise OR.  Every rank's handle holds the same graph in the same order.
 *
 * A traversal is: blest_shard_begin, then per level blest_shard_pull, the
 * exchange, and blest_shard_finish, until finish reports *more == 0.  Steps are
 * enqueued on `stream` (NULL = the handle's stream); finish waits for it.  The
 * steps use the lazy update on the padded layout whatever the handle's
 * options, and the handle runs no other traversal until finish reports the end.
 *
 * blest_shard_begin: src is an original id; d_levels (device int32[n]) receives
 * the levels in original ids (-1 unreached) as the levels are finished, complete
 * once *more == 0.  Runs level 0 (the root).  Errors: INVALID_ARG (rank outside
 * [0, world), bad source, batch handle, empty graph), CUDA. */
blest_status blest_shard_begin(blest_handle h, int32_t rank, int32_t world, int32_t src, int32_t* d_levels,
                               void* stream);

/* Stage 1 of the current level over this rank's queue; d_words (device
 * uint32[ceil(n/32)]) receives the rank's V_next words (bit u % 32 of word u / 32
 * = row u, in BVSS order, marked at this or an earlier level). */
blest_status blest_shard_pull(blest_handle h, uint32_t* d_words, void* stream);

/* d_dst[i] = OR over j < count of d_src[j * words + i] (device arrays): merges
 * all-gathered word arrays.  Errors: INVALID_ARG, CUDA. */
blest_status blest_shard_merge(uint32_t* d_dst, const uint32_t* d_src, int64_t words, int32_t count, void* stream);

/* The level's finalisation sweep on d_merged (the OR of every rank's words):
 * newly reached rows get the level, and the rank's own slice sets holding them
 * are queued for the next level.  Waits for the stream; *more = 1 if the level
 * reached a row (the traversal goes on), 0 when it is over.
 * Errors: INVALID_ARG, TIMEOUT, INTERNAL, CUDA. */
blest_status blest_shard_finish(blest_handle h, const uint32_t* d_merged, int32_t* more, void* stream);

/* blest_shard_finish in two calls, for callers that overlap or time the steps:
 * blest_shard_sweep only enqueues the sweep on the stream; blest_shard_more then
 * waits for the handle's work and sets *more as finish does.  Each sweep must be
 * followed by one blest_shard_more before the next pull. */
blest_status blest_shard_sweep(blest_handle h, const uint32_t* d_merged, void* stream);
blest_status blest_shard_more(blest_handle h, int32_t* more);

/* ---------------------------------------------------------------- testing */

/* The stage-1 pull of one virtual slice set, on the device, for every tile:
 * hits[i] bit q (q = 0..3) is set iff sub-slot q of masks[i] (bits 8q..8q+7)
 * ANDed with alpha[i / 32] is nonzero -- Eq. 1's threshold of the AND/POPC
 * product.  masks: device uint32[32 * tiles]; alpha: device uint8[tiles];
 * hits: device uint8[32 * tiles].  pull selects the CUDA-core or the tensor-core
 * path.  Synchronous. */
blest_status blest_debug_pull(const uint32_t* d_masks, const uint8_t* d_alpha, int32_t tiles,
                              int32_t pull, uint8_t* d_hits);

/* ------------------------------------------------------------ query server */

/* A server keeps graph handles resident and answers multi-source queries with
 * continuous batching: a scheduler thread packs the waiting queries of a graph
 * (in arrival order, up to max_batch_sources sources) into one multi-source
 * launch whenever a launch slot is free and the launch's device memory fits
 * under memory_cap_bytes next to the launches in flight; queries that arrive
 * meanwhile join a later launch, and launches run concurrently on their own
 * streams.  Each query's levels are those blest_msbfs gives for it alone.  The
 * graph handles must outlive the server and must not be used by other calls
 * while it runs. */
typedef struct blest_server* blest_server_handle;

typedef struct {
    int64_t memory_cap_bytes;    /* device bytes launches in flight may hold (default 40 GiB) */
    int32_t max_batch_sources;   /* sources per launch, 1..256 (default 64) */
    int32_t max_inflight;        /* launches in flight at once (default 4, at most 64) */
    int32_t blocks_per_sm;       /* persistent-grid blocks per SM of each launch (default 1) */
    int32_t max_queries_per_launch; /* 0 = no limit (default); 1 = one query per launch (no coalescing) */
    int32_t narrow_sms;          /* SMs of the persistent grid of a launch on a graph whose previous
                                    launch ran more than narrow_levels levels (0 = every launch uses all
                                    SMs, default): high-diameter graphs have small levels, and a narrow
                                    grid crosses each level barrier faster and leaves the other SMs to
                                    the launches of other graphs */
    int32_t narrow_levels;       /* level count above which a graph counts as long: its launches turn
                                    narrow (narrow_sms) and count against long_slots (default 256) */
    int32_t long_slots;          /* launches of long graphs (the previous launch of the graph ran more
                                    than narrow_levels levels) in flight at once; the other slots stay
                                    free for the other graphs' launches, so that a short query does not
                                    wait behind thousand-level traversals.  0 = max_inflight - 1, at
                                    least 1 (default); a value >= max_inflight sets no limit */
} blest_server_params;

typedef struct {
    int64_t launches;            /* multi-source launches issued */
    int64_t sources_launched;    /* sources over all launches */
    int64_t queries_done;
    int64_t queries_waiting;
    int64_t memory_in_use;       /* device bytes held by launches in flight */
    int64_t memory_peak;
} blest_server_stats;

/* graphs: num_graphs handles; params may be NULL.  Errors: INVALID_ARG, OOM, CUDA. */
blest_status blest_server_create(const blest_handle* graphs, int32_t num_graphs, const blest_server_params* params,
                                 blest_server_handle* out);

/* Queue a query: k sources (host array, original ids of graph `graph`); levels
 * receives k * n int32 (source-major) and may be host or device memory, or NULL
 * to discard the result; use page-locked host memory or device memory for
 * fully asynchronous completion.  *ticket identifies the query.  Returns at
 * once.  Errors: INVALID_ARG, TOO_LARGE (k > max_batch_sources, or one query
 * alone exceeds the memory cap). */
blest_status blest_server_submit(blest_server_handle s, int32_t graph, const int32_t* srcs, int32_t k,
                                 int32_t* levels, uint64_t* ticket);

/* Wait up to timeout_s seconds (negative = no limit) for the query, return its
 * status and (optionally) its latency from submission to completion, and
 * release the ticket.  Errors: INVALID_ARG (unknown ticket), TIMEOUT (not done
 * yet; the ticket stays valid), or the query's own status. */
blest_status blest_server_wait(blest_server_handle s, uint64_t ticket, double timeout_s, double* latency_s);

/* paused = 1: start no new launch (launches in flight finish, queries keep
 * queueing); paused = 0: resume.  Lets a caller drain the GPU or build up a
 * backlog that the next launches coalesce. */
blest_status blest_server_pause(blest_server_handle s, int32_t paused);

blest_status blest_server_get_stats(blest_server_handle s, blest_server_stats* out);

/* Stop the scheduler after the launches in flight; queries still waiting are
 * dropped.  NULL is ignored. */
void blest_server_destroy(blest_server_handle s);

/* ------------------------------------------------- allocation-free traversal */

/* Single-source BFS that allocates nothing, for callers that may not call
 * cudaMalloc: plugins and embedded runtimes whose host application owns every
 * device allocation and lends them only their input and output buffers, and
 * services whose device memory is budgeted up front so that no request can
 * fail or stall on an allocation.  The paper has no counterpart; this is a
 * deployment variant of blest_bfs_device.
 *
 * Inputs are the BVSS arrays of a graph in device memory, as blest_export gives
 * them: d_real_ptrs (int32[ceil(n/8)+1]), d_row_ids (int32[128*num_vss]),
 * d_masks (uint32[32*num_vss]) and d_new_id (int32[n], original id -> BVSS id;
 * NULL if the BVSS uses the original order).  src_bvss is the source in BVSS
 * ids (new_id[src]).  d_levels (int32[n], device) receives the levels in
 * ORIGINAL ids.  update is BLEST_UPDATE_EAGER or BLEST_UPDATE_LAZY.  stream is a
 * cudaStream_t (NULL = the legacy default stream).  The call is blocking: it
 * enqueues the clears and the traversal on the stream, then waits for the
 * stream to finish them before it reads the traversal's status and returns.
 *
 * Working memory comes from one fixed device array inside the library (about
 * 21 MiB), which every GPU that loads the library keeps until the process
 * exits.  Limits: n <= 2,097,152 vertices and num_vss <= 524,288 virtual slice
 * sets; larger graphs get BLEST_ERR_TOO_LARGE.  The first call on a device looks
 * up the array's device address (once per device, with that device current);
 * make that first call before any stream capture.  All calls share the one
 * array and each clears what it needs, so calls that overlap on the GPU (from
 * several host threads or streams) race and must be serialised by the caller.
 * Errors: INVALID_ARG, TOO_LARGE, TIMEOUT, INTERNAL, CUDA. */
blest_status blest_bfs_static_scratch(int32_t n, int64_t num_vss, const int32_t* d_real_ptrs,
                                      const int32_t* d_row_ids, const uint32_t* d_masks,
                                      const int32_t* d_new_id, int32_t src_bvss, int32_t* d_levels,
                                      int32_t update, void* stream);

/* Static name of a status code ("BLEST_OK", ...); never NULL. */
const char* blest_status_string(blest_status s);

/* Message of the last failure on the calling thread (thread-local, valid until
 * the thread's next failing call); "" if none. */
const char* blest_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BLEST_H */
