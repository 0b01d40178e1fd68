/*
 * acc_motif.h — C ABI of a GB300 (sm_103a) library that counts the connected
 * induced k-vertex subgraphs of a directed graph, k = 3, 4, 5, grouped by
 * isomorphism class.
 *
 * The operation is the one the paper states as Problems Motifs-3, Motifs-4
 * and Motifs-5 (Background section, "Problem statement"): given a directed
 * graph G(V,E), count the connected induced subgraphs of size k, grouped by
 * the 13, 199 or 9364 isomorphism classes of connected k-vertex digraphs.
 * "Connected" is taken in the undirected version G* of G (Notation section:
 * {u,v} is an edge of G* iff (u,v) or (v,u) is an arc of G), i.e. weak
 * connectivity.  Counts are exact int64.
 *
 * Class numbering (the paper's histogram positions are arbitrary): the
 * adjacency code of an ordered vertex tuple (w_0..w_{k-1}) sets bit
 * i*(k-1) + (j - [j > i]) iff the arc w_i -> w_j exists; the canonical code
 * of a digraph is the minimum code over its k! vertex orders; class c is the
 * c-th smallest canonical code among connected k-vertex digraphs.
 * acc_motif_class_code() returns that code so callers can name classes.
 *
 * Conventions for every entry point:
 *  - Return value: ACC_OK (0) or a negative ACC_ERR_* code.  No C++
 *    exception crosses this interface.
 *  - "device" pointers are CUDA device (or managed) memory of the context's
 *    device; "host" pointers are ordinary (preferably pinned) host memory.
 *    The caller owns every pointer it passes; the library never frees one,
 *    and reads or writes one only inside a call that passes it (a prepared
 *    batch's graphs: until its last run).  Pointers remembered to recognise
 *    a repeated call are compared, never dereferenced.
 *  - stream is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is stream-ordered: results are valid once the caller
 *    synchronises the stream, unless the entry point says it synchronises.
 *  - A context is not thread-safe: use one per host thread, or lock around it.
 *    Calls on one context must not overlap on the GPU (they share its
 *    workspace); issue them on one stream or synchronise in between.
 */
#ifndef ACC_MOTIF_H
#define ACC_MOTIF_H

#include <stdint.h>

#if defined(__GNUC__)
#define ACC_API __attribute__((visibility("default")))
#else
#define ACC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define ACC_OK 0
#define ACC_ERR_K (-1)        /* k is not 3, 4 or 5 */
#define ACC_ERR_INPUT (-2)    /* malformed graph: bad rowptr, column out of range, self-loop, bad size */
#define ACC_ERR_NOMEM (-3)    /* a device or pinned-host allocation failed */
#define ACC_ERR_TIMEOUT (-4)  /* a bounded device wait gave up */
#define ACC_ERR_OVERFLOW (-5) /* a count or an index would not fit its type */
#define ACC_ERR_CUDA (-6)     /* a CUDA runtime call failed */
#define ACC_ERR_ARG (-7)      /* null pointer, bad handle or bad option */
#define ACC_ERR_TOO_LARGE (-8) /* n above ACC_MAX_N (dense pair-state matrix limit) */
#define ACC_ERR_INTERNAL (-9)  /* an internal consistency check failed (a library bug) */

/* Largest vertex count the dense n x n pair-state matrix is built for
 * (n^2/4 bytes: 64 GiB at this limit, within one GB300's memory; the
 * per-warp overflow lists add 8(n + 64) bytes per resident warp).  Larger
 * graphs, up to ACC_MAX_N_SPARSE vertices, are counted in ACC_MODE_COUNT
 * only, built without the dense matrix (ACC_ADJ_SPARSE below). */
#define ACC_MAX_N 524288
#define ACC_MAX_N_SPARSE 67108864

typedef struct acc_ctx acc_ctx;

/* Message for an error code (static string, never NULL). */
ACC_API const char *acc_strerror(int code);

/* 13, 199 or 9364 for k = 3, 4, 5 (Problems Motifs-3/4/5); ACC_ERR_K otherwise. */
ACC_API int acc_motif_num_classes(int k);

/*
 * Create a context on CUDA device `device` (the device is made current for
 * the calling thread).  The context owns a grow-only workspace.  The code ->
 * class tables are shared by every context on the device: built on the
 * device at the first use of each k by any of them, freed with the last
 * context that used them.  *out receives the handle.  Errors: ACC_ERR_ARG
 * (out NULL), ACC_ERR_CUDA.
 */
ACC_API int acc_ctx_create(acc_ctx **out, int device);

/* Release a context and all its device memory (NULL is a no-op; the shared
 * class tables are released with the last context on the device).  Waits
 * for the context's outstanding work. */
ACC_API void acc_ctx_destroy(acc_ctx *ctx);

/*
 * Build (once per device) and cache the code -> class table for k on the
 * context's device, stream-ordered on `stream`, then wait for it.  Counting calls do
 * this themselves on first use; call it ahead to keep the one-time cost
 * (largest for k = 5: 2^20 codes x 120 relabellings) out of a timed region.
 * Errors: ACC_ERR_ARG, ACC_ERR_K, ACC_ERR_NOMEM, ACC_ERR_CUDA.
 */
ACC_API int acc_motif_prepare(acc_ctx *ctx, int k, void *stream);

/*
 * Count the connected induced k-subgraphs of one directed graph by class
 * (Problems Motifs-3/4/5).
 *
 *  d_rowptr  device int64[n+1]: out-CSR row offsets, d_rowptr[0] = 0,
 *            non-decreasing, d_rowptr[n] = m.
 *  d_col     device int32[m]: arc targets; row v lists the heads of arcs
 *            v -> u.  Any order within a row; repeated arcs count once
 *            (E is a set).  A self-loop or a target outside [0, n) is an
 *            input error.
 *  n, m      vertex and arc counts, 0 <= n <= ACC_MAX_N (ACC_MAX_N_SPARSE in
 *            ACC_MODE_COUNT), 0 <= m < 2^31.
 *  k         3, 4 or 5.
 *  stream    cudaStream_t (void*), see above.
 *  d_counts  device int64[acc_motif_num_classes(k)], overwritten.
 *  d_status  device int32[1] or NULL.  When non-NULL the call is fully
 *            asynchronous: it returns after enqueueing, and *d_status
 *            receives ACC_OK or the error the device found (ACC_ERR_INPUT for
 *            a malformed graph, in which case d_counts is unspecified).  When
 *            NULL the call waits for its own work and returns that status.
 *
 * Overflow guard (the paper keeps its counts in "integer" variables; here
 * they are int64): before enumerating, the device bounds N_k from the G*
 * degrees (every connected k-set has a spanning tree; each tree shape is
 * counted from its centre, every further neighbour taken at the largest
 * degree D: k = 3 sum C(d,2); k = 4 sum C(d,3) + (D-1) sum d(d-1)/2;
 * k = 5 sum C(d,4) + (D-1) sum d(d-1)(d-2)/2 + (D-1)^2 sum d^2/2; and never
 * above C(n,k)).  If the bound exceeds 2^62 the status becomes
 * ACC_ERR_OVERFLOW, nothing is enumerated and d_counts is unspecified.  The
 * bound is loose for hubs with many low-degree neighbours, so such a graph
 * can be refused although its exact counts would fit: for example an out-star
 * with 50000 leaves at k = 5 (bound 6.5e18, exact N_5 = C(50000, 4) = 2.6e17).
 *
 * Device-found errors: ACC_ERR_INPUT, ACC_ERR_OVERFLOW (above),
 * ACC_ERR_INTERNAL.  Host-checked errors (returned before anything is
 * enqueued): ACC_ERR_ARG, ACC_ERR_K, ACC_ERR_INPUT (negative sizes),
 * ACC_ERR_TOO_LARGE, ACC_ERR_NOMEM, ACC_ERR_CUDA.
 */
ACC_API int acc_motif_count(acc_ctx *ctx, const int64_t *d_rowptr, const int32_t *d_col, int32_t n,
                    int64_t m, int k, void *stream, int64_t *d_counts, int32_t *d_status);

/*
 * The same count with host arrays: copies h_rowptr (int64[n+1]) and h_col
 * (int32[m]) to the device on the context's own stream, counts, copies the
 * int64[num_classes(k)] result to h_counts and waits.  Pinned host memory
 * gives the fastest copies.  Returns the status of the whole call.
 */
ACC_API int acc_motif_count_host(acc_ctx *ctx, const int64_t *h_rowptr, const int32_t *h_col, int32_t n,
                         int64_t m, int k, int64_t *h_counts);

/*
 * Batched form: many graphs counted by one sequence of launches (the
 * significance step of the motif pipeline counts a real graph and an ensemble
 * of randomised copies, Implementation section, steps i-iii; the paper counts
 * each graph separately).
 *
 * acc_graph_desc describes one graph in device memory, with the same layout
 * and rules as acc_motif_count's arguments.
 */
typedef struct {
    const int64_t *rowptr; /* device int64[n+1] */
    const int32_t *col;    /* device int32[m] */
    int32_t n;
    int64_t m;
} acc_graph_desc;

/*
 * Prepare a batch of B graphs (h_graphs: host array of B descriptors) for
 * k: first waits for `stream` (an earlier run on it may still read the
 * previous batch's descriptors), then validates sizes, lays out every graph's
 * buffers in the context's workspace, uploads the descriptors and builds the
 * table for k; waits.  The graphs' device arrays must stay valid and
 * unchanged until the batch's last acc_motif_batch_run.  Preparing replaces
 * the previous batch; a run of the previous batch still in flight on another
 * stream must be waited for by the caller first.  Errors:
 * ACC_ERR_ARG, ACC_ERR_K, ACC_ERR_INPUT, ACC_ERR_TOO_LARGE (some n above
 * ACC_MAX_N), ACC_ERR_OVERFLOW (more than 2^31-1 vertices or arcs in total),
 * ACC_ERR_NOMEM, ACC_ERR_CUDA.
 */
ACC_API int acc_motif_batch_prepare(acc_ctx *ctx, const acc_graph_desc *h_graphs, int32_t B, int k, void *stream);

/*
 * Count every graph of the prepared batch: d_counts is device
 * int64[B * num_classes(k)], row g = graph g, overwritten.  d_status as in
 * acc_motif_count (the overflow guard bounds every graph of the batch by
 * the degree sums of all of them, and by C(largest n, k)).  With d_status non-NULL the call only enqueues kernels
 * (no allocation, no copy, no wait), so it can be captured into a CUDA graph
 * and replayed; only a run after acc_ctx_set_mode or acc_ctx_set_adjacency
 * changed the context since the prepare may first grow the workspace for
 * the new path (ACC_ERR_TOO_LARGE if the new mode cannot take the batch's
 * largest graph).  A captured run stays valid until the next
 * acc_motif_batch_prepare on the context (which rewrites the descriptors the
 * capture reads; the batch's sizes are baked into the captured launches) or
 * until a later call on the context grows its workspace; capture again after
 * either.
 */
ACC_API int acc_motif_batch_run(acc_ctx *ctx, void *stream, int64_t *d_counts, int32_t *d_status);

/* acc_motif_batch_prepare followed by acc_motif_batch_run. */
ACC_API int acc_motif_count_batch(acc_ctx *ctx, const acc_graph_desc *h_graphs, int32_t B, int k, void *stream,
                                  int64_t *d_counts, int32_t *d_status);

/*
 * Tune the schedule for the prepared batch: runs the batch once for each of
 * a fixed set of candidate (light, target) pairs, timed with CUDA events on
 * `stream`, and keeps the fastest in the context (acc_ctx_set_schedule).
 * Waits for the device.  h_light, h_target, h_ms (nullable) receive the
 * chosen pair and its time.  Errors: ACC_ERR_ARG (no prepared batch), any
 * error a batch run returns (the previous schedule is then kept).
 */
ACC_API int acc_motif_batch_autotune(acc_ctx *ctx, void *stream, int64_t *h_light, int64_t *h_target,
                                     float *h_ms);

/*
 * Z-scores of class counts against randomised copies (significance step of
 * the motif pipeline; the paper gives no formula).  d_counts is device
 * int64[groups][group_size][num_classes(k)]: entry 0 of each group is the
 * real graph, entries 1..R (R = group_size - 1 >= 1) its randomisations.
 * d_z is device double[groups][num_classes(k)]:
 *   Z_c = (N_c - mu_c) / sigma_c,  mu_c = (sum_i N_ic) / R,
 *   sigma_c = sqrt(sum_i (N_ic - mu_c)^2 / R) (population deviation,
 *   accumulated in increasing i), NaN when sigma_c = 0,
 * every step an IEEE round-to-nearest double operation (no fused
 * multiply-add).  Stream-ordered; no context needed.
 */
ACC_API int acc_motif_zscores(const int64_t *d_counts, int32_t groups, int32_t group_size, int k, void *stream,
                              double *d_z);

/*
 * Randomised copies for the random ensemble of the significance step
 * (Implementation section, steps i and iii: the real graph and a set of
 * random graphs are counted; the paper fixes no generator).
 *
 * Each of the G graphs (h_graphs, host array; same layout and rules as
 * acc_motif_count's arguments, and simple: no repeated arc) gets R copies.
 * Arc e of a graph is (row holding position e) -> col[e].  A copy keeps
 * rowptr and starts as col; it then makes attempts_per_arc * m attempts,
 * each drawing positions e1 then e2 uniformly below m from SplitMix64
 * (Steele, Lea and Flood, 2014; a draw x maps to the high 64 bits of x * m),
 * the stream of copy r of graph g seeded h_seeds[g] + r (mod 2^64).  With
 * a -> b = arc e1 and c -> d = arc e2 of the copy:
 *   ACC_RAND_SWAP    rejected if e1 == e2, a == d, c == b, or a -> d or
 *                    c -> b is already an arc; otherwise a -> d and c -> b.
 *                    Every in- and out-degree is kept.
 *   ACC_RAND_MUTUAL  an arc is mutual when its reverse is an arc.  Rejected
 *                    if e1 == e2, a == d, c == b, exactly one of the two
 *                    arcs is mutual, or a and d or c and b are adjacent;
 *                    otherwise two single arcs become a -> d and c -> b, and
 *                    two mutual pairs a <-> b and c <-> d become a <-> d and
 *                    c <-> b.  Every vertex keeps its single in- and
 *                    out-degree and its number of mutual neighbours.
 * A repeated arc in the input is not an error, but the copies are then only
 * defined by the procedure above (a row entry counts as an arc).
 *
 *  d_out       device int32[R * sum of m]: graph g's copies start at element
 *              R * (m_0 + ... + m_{g-1}), copy r at that start + r * m_g,
 *              each m_g targets in the positions of the graph's col (so copy
 *              r is the out-CSR (rowptr_g, that slice)).
 *  d_accepted  device int64[G * R] or NULL: accepted swaps of copy r of
 *              graph g at g * R + r.
 *  d_status    as in acc_motif_count (ACC_ERR_INPUT for a malformed graph;
 *              d_out is then unspecified).
 * The call waits for `stream` and uploads the descriptors (graphs, R,
 * attempts and seeds) unless they equal the previous call's on this context;
 * then, with d_status non-NULL, it only enqueues its kernels, so a repeated
 * call can be captured into a CUDA graph and replayed.  Host-checked
 * errors: ACC_ERR_ARG (null pointers, G or R negative, unknown mode,
 * attempts_per_arc negative), ACC_ERR_INPUT (negative sizes, m >= 2^31, m > 0
 * with n = 0), ACC_ERR_OVERFLOW (attempts_per_arc * m above 2^62),
 * ACC_ERR_NOMEM, ACC_ERR_CUDA.
 */
#define ACC_RAND_SWAP 0
#define ACC_RAND_MUTUAL 1
ACC_API int acc_swap_randomise(acc_ctx *ctx, const acc_graph_desc *h_graphs, int32_t G, int32_t R,
                               int64_t attempts_per_arc, const uint64_t *h_seeds, int mode, void *stream,
                               int32_t *d_out, int64_t *d_accepted, int32_t *d_status);

/*
 * Device memory acc_swap_randomise may keep for the copies' adjacency
 * bitmaps (R * sum over graphs of n * ceil(n / 128) * 16 bytes; default
 * 16 GiB), plus, for ACC_RAND_MUTUAL, 4 (R + 1) bytes per arc of reverse
 * positions.  Within the limit, and when growing to it leaves half of the
 * free memory, both modes decide 16 attempts per step speculatively; else
 * they decide them one by one by scanning rows.  The copies are the same
 * either way.  0 always scans rows.  Errors: ACC_ERR_ARG.
 */
ACC_API int acc_ctx_set_randomise_memory(acc_ctx *ctx, int64_t bytes);

/*
 * Serving form: a request server with continuous batching on one GPU.
 *
 * Requests (resident graph, k) are submitted at any time.  A request is
 * admitted as soon as one of the server's slots is free and the slot's device
 * workspace for it fits the memory budget, in the order of the admission
 * policy (acc_server_set_policy; a request that cannot fit even with every
 * slot idle fails with ACC_ERR_NOMEM).  Each slot has its own
 * context and CUDA stream, so admitted requests overlap on the device; a
 * request on a graph of at most 4096 vertices takes 1/8 of the GPU's
 * enumeration grid (its few work units cannot fill more) and so runs beside
 * the others, a larger one takes the whole grid.
 * Results are the same as acc_motif_count's for the same graph and k.  The
 * server does its host work only inside these calls (no threads), so call
 * acc_server_progress or acc_server_poll regularly.  A server is not
 * thread-safe.
 */
typedef struct acc_server acc_server;
#define ACC_REQ_QUEUED 0
#define ACC_REQ_RUNNING 1
#define ACC_REQ_DONE 2

/* Server on `device` with `slots` (1..64) concurrent requests and a device
 * memory budget for the slots' workspaces in bytes. */
ACC_API int acc_server_create(acc_server **out, int device, int32_t slots, int64_t mem_budget_bytes);
/* Admission order of queued requests.
 *  ACC_SERVE_SHORTEST (default): the request with the smallest
 *   est * exp(-wait / aging_s) goes first, where est is the graph's work
 *   estimate for its k (sum over vertices of d^(k-1), d = out- plus
 *   in-degree, taken when the graph is registered) and wait the seconds it
 *   has queued; small requests overtake large ones, and a large request's
 *   key halves every aging_s * ln 2 seconds, so none waits forever.
 *  ACC_SERVE_FIFO: submission order.
 * If the chosen request does not fit the budget, admission waits for a
 * running request to finish.  Errors: ACC_ERR_ARG (unknown policy,
 * aging_s <= 0). */
#define ACC_SERVE_FIFO 0
#define ACC_SERVE_SHORTEST 1
ACC_API int acc_server_set_policy(acc_server *srv, int policy, double aging_s);
/* Waits for running requests, releases everything (NULL is a no-op). */
ACC_API void acc_server_destroy(acc_server *srv);
/* Register a resident graph (device arrays as in acc_motif_count; they must
 * hold the graph when this is called and stay valid while the server may
 * count it).  Reads the arrays once to estimate the graph's work per k (a
 * synchronous copy to the host for graphs of at most 2^26 arcs; larger
 * graphs are estimated from n and m).  *graph_id receives its id. */
ACC_API int acc_server_add_graph(acc_server *srv, const int64_t *d_rowptr, const int32_t *d_col, int32_t n,
                                 int64_t m, int32_t *graph_id);
/* Pre-size every slot (within the budget) for the largest registered graph
 * and build the class tables of every k, so serving allocates nothing; waits. */
ACC_API int acc_server_reserve(acc_server *srv);
/* Queue a request; *request_id receives its id.  Admits what fits. */
ACC_API int acc_server_submit(acc_server *srv, int32_t graph_id, int k, int64_t *request_id);
/* Retire finished requests and admit queued ones; *running / *queued
 * (nullable) receive the current numbers. */
ACC_API int acc_server_progress(acc_server *srv, int32_t *running, int32_t *queued);
/* Progress, then report request_id: *state = ACC_REQ_QUEUED, _RUNNING,
 * _DONE or a negative error code; when done, h_counts (nullable, host
 * int64[num_classes(k)]) receives the counts and *latency_s (nullable) the
 * seconds from submission to completion (-1 while not finished). */
ACC_API int acc_server_poll(acc_server *srv, int64_t request_id, int32_t *state, int64_t *h_counts,
                            double *latency_s);
/* Run until no request is queued or running. */
ACC_API int acc_server_drain(acc_server *srv);

/* Canonical adjacency code of class cls (0 <= cls < num_classes(k)). */
ACC_API int acc_motif_class_code(acc_ctx *ctx, int k, int32_t cls, uint32_t *code);

/* Class of an adjacency code (< 2^(k(k-1))); *cls = -1 for a code whose
 * digraph is not weakly connected. */
ACC_API int acc_motif_classify_code(acc_ctx *ctx, int k, uint32_t code, int32_t *cls);

/* Copy the whole code -> class table for k to host int16[2^(k(k-1))]
 * (-1 = disconnected). */
ACC_API int acc_motif_copy_table(acc_ctx *ctx, int k, int16_t *h_table);

/*
 * Copy the launch and workload statistics of the context's last
 * acc_motif_count call to host int64[ACC_STATS_LEN]; waits for the device
 * (call it after that count has completed):
 *   [0] kernels the call launched, [1] base work units (vertices for k = 3,
 *   neighbour-list positions for k = 4, 5), [2] chunks heavy units were split
 *   into, [3] undirected edges |E*|, [4] largest degree in G*, [5] blocks of
 *   each enumeration launch, [6] neighbour entries the last two levels
 *   scanned (ACC_MODE_COUNT; 0 in ACC_MODE_ENUMERATE).
 */
#define ACC_STATS_LEN 7
ACC_API int acc_motif_last_stats(acc_ctx *ctx, int64_t *h_stats);

/*
 * How the last two levels of the enumeration are counted.
 *  ACC_MODE_COUNT (default): per extension list, the pairs of members that
 *   are not adjacent are counted per pair of state-vector groups (their class
 *   depends only on the two members' states to the prefix), the adjacent
 *   pairs are corrected one by one from the members' neighbour lists, as the
 *   paper's Table starb counts patterns from set sizes minus edges.  For a
 *   set of at least 8192 arcs the build also stores, per neighbour entry
 *   v -> x, where x's list passes v (8 bytes per entry), so the scans of
 *   the root's neighbours' lists start without a search.
 *  ACC_MODE_ENUMERATE: every k-subset is visited and classified on its own.
 *  ACC_MODE_FORMULA: for k = 3, the paper's per-vertex formulas (Thm teo3,
 *   Algorithm s3, Table starb): open triples from the sizes of each vertex's
 *   out-only / in-only / bidirected neighbour sets, triangles listed once and
 *   the open triples they were counted as moved out; no subset is visited.
 *   For k = 4, the paper's per-edge formulas (Thm lema4d, Cor coro:a,
 *   Algorithm mine, Fact correction): for each edge {u, v} of G*, pairs of
 *   vertices adjacent to u or v counted per pair of its 15 neighbour sets
 *   (Fig. edgesets), linked pairs moved to their own class, each class then
 *   divided by the number of edges that reach its pattern.  For k = 5, the
 *   paper's per-triple formulas (Lemma lema5d, Algorithm fived, Algorithm
 *   partfive): for each connected 3-set of G*, pairs of vertices adjacent to
 *   it counted per pair of its 63 neighbour sets, linked pairs moved to their
 *   own class, each class divided by the number of connected 3-sets that
 *   reach its pattern.
 *  ACC_MODE_AUTO: ACC_MODE_FORMULA for k = 3 on graphs of at most 16384
 *   vertices (where the per-vertex formulas measured faster than the count
 *   mode; above, hubs make their triangle listing the longer scan),
 *   ACC_MODE_COUNT otherwise (for k = 4, 5 the count mode scans fewer
 *   neighbour entries than the per-edge and per-triple formulas on every
 *   graph measured, dense ones included).
 * All modes give identical counts.  Errors: ACC_ERR_ARG.
 */
#define ACC_MODE_COUNT 0
#define ACC_MODE_ENUMERATE 1
#define ACC_MODE_FORMULA 2
#define ACC_MODE_AUTO 3
ACC_API int acc_ctx_set_mode(acc_ctx *ctx, int mode);

/*
 * Adjacency structure the count mode probes (ACC_MODE_COUNT; the other modes
 * always read the dense pair-state block).  The paper tests adjacency "in
 * O(1)" by hashing (its k=4 and k=5 complexity discussion).
 *  ACC_ADJ_DENSE: the dense n x n pair-state block (2 bits per ordered pair),
 *   one load per probe; n^2/4 bytes, so its probes leave L2 for large n.
 *  ACC_ADJ_HASH: per-vertex open-addressing tables of the neighbour entries
 *   (32 bytes per entry of the G* neighbour lists, built on the device after
 *   the lists), one 16-byte load per probe in the common case.
 *  ACC_ADJ_SPARSE: the same hashed tables, and the neighbour lists built
 *   without the dense block: every arc puts a raw entry in both endpoints'
 *   rows, each row is sorted (one warp in shared memory up to 2048 raw
 *   entries, one block in global memory above) and its repeated neighbours
 *   merged.  Memory O(n + m); the call waits once for the build (the
 *   per-warp overflow lists are sized by the largest degree it finds), so it
 *   is never replayed from a launch graph.
 *  ACC_ADJ_AUTO (default): sparse above ACC_MAX_N vertices; hashed when the
 *   largest graph of the count or batch has at least 49152 vertices for
 *   k = 5, 131072 for k = 3, 4 (where the dense probes, out of L2, get slower
 *   than the hashed ones); dense otherwise.
 * Except for ACC_ADJ_SPARSE the dense block is built in every case (it also
 * deduplicates the arcs).  All choices give identical counts.  Errors:
 * ACC_ERR_ARG.
 */
#define ACC_ADJ_AUTO 0
#define ACC_ADJ_DENSE 1
#define ACC_ADJ_HASH 2
#define ACC_ADJ_SPARSE 3
ACC_API int acc_ctx_set_adjacency(acc_ctx *ctx, int adjacency);

/*
 * Work schedule of the enumeration (not in the paper: how the ESU units are
 * spread over the GPU).  A unit (a root, or a root and one neighbour) whose
 * estimated work is at most `light` runs whole on one warp; a heavier one is
 * cut into row tiles of about `target` work that any warp may take.  Work is
 * counted in scanned neighbour entries (count mode) or leaves (enumerate
 * mode).  0 selects the built-in default: light 2048 and target 4096, except
 * in the count mode light 6144 for k = 4 and target 16384 for k = 5 (whose
 * tiles share one scan of the level-2 rows, so longer tiles save work).
 * Values above 2^40 or negative are ACC_ERR_ARG.  The schedule changes speed
 * only, never the counts.  acc_ctx_get_schedule reports the values in effect
 * for k = 3.
 */
ACC_API int acc_ctx_set_schedule(acc_ctx *ctx, int64_t light, int64_t target);
ACC_API int acc_ctx_get_schedule(acc_ctx *ctx, int64_t *light, int64_t *target);

/*
 * Stage timing.  With timing on (on != 0), every acc_motif_count records CUDA
 * events on its stream around its stages.  acc_motif_last_timing waits for
 * the last call's end event and writes float h_ms[4], in milliseconds:
 * [0] graph build, [1] enumeration (both launches), [2] enumeration phase 1
 * (light units run, heavy units queued), [3] phase 2 (queue drained).
 * Errors: ACC_ERR_ARG (timing off or no count yet), ACC_ERR_CUDA.
 */
ACC_API int acc_ctx_set_timing(acc_ctx *ctx, int on);

/*
 * Launch graphs for repeated counts (on = 1, the default): a count that
 * repeats the previous one on this context (same device buffers, n, m, k,
 * mode, schedule and workspace) replays one CUDA graph of its whole launch
 * sequence instead of launching the kernels one by one; the graph is
 * captured at the first repeat (a one-off count launches one by one and
 * captures nothing).  The kernels, and so the results,
 * are the same either way; the contents of the buffers may change between
 * repeats.  Stage timing (acc_ctx_set_timing) always launches one by one.
 * Errors: ACC_ERR_ARG.
 */
ACC_API int acc_ctx_set_launch_graphs(acc_ctx *ctx, int on);
ACC_API int acc_motif_last_timing(acc_ctx *ctx, float *h_ms);

/*
 * Build the code -> class table for k without allocating anything.
 *
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory where they need the table -- code under a fixed
 * memory budget handed out up front, a framework that owns the device
 * allocator, or work being captured into a CUDA graph.  It needs no context
 * and calls no cudaMalloc, cudaFree or other allocating routine.
 *
 *  k             3, 4 or 5 (ACC_ERR_K otherwise).
 *  stream        cudaStream_t (void*); the call only enqueues work.
 *  d_table       device int16[2^(k(k-1))]: receives the same table as
 *                acc_motif_copy_table (-1 = not weakly connected).  An entry
 *                of -2 would mark a canonical code ranked past the last class
 *                (a library bug; the context entry points check for it and
 *                fail with ACC_ERR_INTERNAL, this one leaves the check to the
 *                caller: every entry is >= -1 in a correct table).
 *  d_class_code  device uint32[num_classes(k)]: canonical code of each class,
 *                as acc_motif_class_code.
 *
 * Working memory: a fixed array of 8 MiB and 8 KiB inside the library (room
 * for the 2^20 codes of k = 5; anything larger is rejected with
 * ACC_ERR_TOO_LARGE).  Every GPU that loads the library holds it until the
 * process exits.  A call looks up the array's device address (cudaGetSymbolAddress)
 * on the current device, except while `stream` is being captured: then it
 * reuses the address an earlier call on that device found, and fails with
 * ACC_ERR_CUDA if there was none.  So make one call on each device before any
 * stream capture, and one more after a cudaDeviceReset (which reloads the
 * library's device image, possibly elsewhere).  All calls share the array: each call writes
 * every word of it that it reads, so no state carries over, but calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.
 */
ACC_API int acc_motif_build_table_static(int k, void *stream, int16_t *d_table, uint32_t *d_class_code);

#ifdef __cplusplus
}
#endif

#endif /* ACC_MOTIF_H */
