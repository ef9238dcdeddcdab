/*
 * lpa.h -- C ABI of the GB300 (sm_103a) label-propagation library liblpa.so.
 *
 * The library implements the community-detection method of "nu-LPA: Fast GPU-based
 * Label Propagation Algorithm (LPA) for Community Detection" (Sahu, arXiv 2411.11468):
 * every unprocessed vertex i takes the label with the largest total edge weight among
 * its neighbours' labels (Eq. 3), ties going to the smallest label (Section 4,
 * item 5); Pick-Less (Section 4.1) restricts moves to smaller labels every
 * pl_period-th iteration; a vertex that changes label marks its neighbours for the
 * next sweep (Section 4, item 4); the loop stops when the changed fraction falls
 * below the tolerance on a non-Pick-Less iteration or after max_iters sweeps
 * (Algorithm 1).  Neighbour-label weights are accumulated in per-vertex open-addressing
 * hashtables with the hybrid quadratic-double probe of Algorithm 2 (Section 4.2).
 *
 * Input graphs are undirected CSR graphs as in the paper's Preliminaries: every
 * edge {i, j} is stored in row i and in row j with the same weight w_ij >= 0.
 * Vertex ids and labels are int32; weights and label sums are float32 (the
 * paper's Configuration paragraph); when every weight is an integer and every weighted
 * degree is below 2^24 the label sums are kept as uint32, which gives the same sums and
 * the same winners (lpa_tuning.float_values selects float32 or float64 sums instead;
 * weights that are all exactly 1 are taken as unit weights).  Modularity (Eq. 1) is exact
 * for integer weights, else float64.
 *
 * Conventions for every call:
 *  - Status: every call returns LPA_OK (0) or a negative LPA_E* code; lpa_strerror()
 *    names the code and lpa_last_error() returns a message for the calling thread's
 *    last failure.  No call traps or asserts on the device.
 *  - Ownership: the library copies its inputs into device memory it owns; callers
 *    keep their arrays.  Handles are freed with the matching *_destroy call.
 *  - Streams: `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).
 *    All device work of a handle is ordered on that stream.  Calls that return
 *    host-visible results synchronise that stream before returning.
 *  - Threads: one handle must not be used by two threads at once; distinct handles
 *    are independent.
 *  - Pointers marked "host or device" are host pointers unless the call's flags say
 *    LPA_DEVICE_PTRS (or its on_device argument is non-zero), in which case they are
 *    device pointers valid on the current CUDA device.
 */
#ifndef LPA_H
#define LPA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define LPA_OK        0
#define LPA_EINVAL   (-1)   /* invalid argument or invalid graph                      */
#define LPA_ENOMEM   (-2)   /* device or pinned host allocation failed                */
#define LPA_ECUDA    (-3)   /* a CUDA runtime call or kernel launch failed            */
#define LPA_ETIMEOUT (-4)   /* a bounded device wait gave up (reserved: no kernel of
                               this version waits on another, so no call returns it)   */
#define LPA_ESTATE   (-5)   /* call not valid in the handle's current state           */
#define LPA_ECANCELED (-6)  /* server request cancelled (lpa_server_cancel)           */

/* ---- lpa_run modes (Section 4 item 1 is the asynchronous mode) -------------------- */
#define LPA_SYNC    0       /* deterministic: every sweep reads the previous sweep's labels */
#define LPA_ASYNC   1       /* the paper's mode: labels updated in place while others read */
#define LPA_RESUME  16      /* or-ed into mode: continue from the handle's current state    */

/* ---- lpa_create / lpa_batch_create flags ------------------------------------------ */
#define LPA_OFFSETS_I32      0   /* offsets are int32_t[n+1]                           */
#define LPA_OFFSETS_I64      1   /* offsets are int64_t[n+1]                           */
#define LPA_HOST_PTRS        0   /* input arrays are host pointers                     */
#define LPA_DEVICE_PTRS      2   /* input arrays are device pointers                   */
#define LPA_CHECK_SYMMETRIC  4   /* also verify that the graph is undirected           */
#define LPA_BORROW_INPUTS    8   /* lpa_server_submit: read the host arrays at admission  */

/* ---- statistics ------------------------------------------------------------------- */
#define LPA_STATS_MAX_ITERS 64   /* per-iteration arrays hold the first 64 iterations  */
#define LPA_NUM_KERNELS     12   /* kernel slots of the per-kernel arrays              */

/* Kernel slots, in launch order within one sweep. */
#define LPA_K_THREAD      0   /* thread per vertex, private table (lowest degrees)     */
#define LPA_K_GROUP       1   /* small lane group per vertex, shared table in smem     */
#define LPA_K_WARP        2   /* warp per vertex, table in smem                        */
#define LPA_K_CTA         3   /* thread block per vertex, table in smem (tier 1)       */
#define LPA_K_CTA_LARGE   4   /* thread block per vertex, table in smem (tier 2)       */
#define LPA_K_CTA_XL      5   /* thread block per vertex, table in smem (tier 3)       */
#define LPA_K_HUB_BEGIN   6   /* hubs: take the processed flags                        */
#define LPA_K_HUB_ACC     7   /* hubs: several blocks accumulate into an HBM table     */
#define LPA_K_HUB_CLEAR   8   /* hubs: clear the table slots used in this sweep        */
#define LPA_K_HUB_MOVE    9   /* hubs: move decision                                   */
#define LPA_K_HUB_MARK   10   /* hubs: mark the neighbours of hubs that moved          */
#define LPA_K_APPLY      11   /* synchronous mode: publish the sweep's new labels      */

typedef struct lpa_stats {
    /* input */
    int32_t time_kernels;     /* non-zero: time every kernel with CUDA events          */
    /* output */
    int32_t iterations;       /* sweeps run (absolute index of the next sweep)         */
    int32_t converged;        /* 1 when the tolerance test ended the run               */
    int32_t first_iter;       /* absolute index of the first sweep of this call        */
    int64_t changed[LPA_STATS_MAX_ITERS];   /* dN: vertices that changed label        */
    int64_t active[LPA_STATS_MAX_ITERS];    /* vertices processed (unprocessed at start) */
    int64_t edges[LPA_STATS_MAX_ITERS];     /* CSR entries scanned                    */
    int64_t marks[LPA_STATS_MAX_ITERS];     /* CSR entries of the vertices that moved */
    float   iter_ms[LPA_STATS_MAX_ITERS];   /* device time of each sweep              */
    float   total_ms;                       /* device time of the whole call          */
    int32_t launches;                       /* kernels launched by this call          */
    int64_t probe_fallbacks;                /* linear-probe fallbacks (Algorithm 2 budget spent) */
    /* per kernel slot (filled when time_kernels != 0), indexed [iteration][slot]
       for the first LPA_STATS_MAX_ITERS iterations of this call                    */
    float   kernel_ms[LPA_STATS_MAX_ITERS][LPA_NUM_KERNELS];
    int64_t kernel_edges[LPA_STATS_MAX_ITERS][LPA_NUM_KERNELS];
    int64_t kernel_active[LPA_STATS_MAX_ITERS][LPA_NUM_KERNELS];
} lpa_stats;

/* Degree-bucket configuration.  A vertex of degree D is handled by the first bucket
 * whose limit is >= D; vertices above cta_xl_max are hubs.  Limits must not decrease.
 * Shared-memory tables have capacity nextPow2(D << smem_table_shift) - 1 (shift 0 is the
 * paper's nextPow2(D) - 1, shift 1 keeps the load factor at or below one half); each
 * bucket's table, sized for its largest degree, must fit in shared memory, else
 * lpa_set_tuning returns LPA_EINVAL.  Hub tables have capacity
 * nextPow2(D << hub_table_shift) - 1 and live in HBM, or, with hub_cluster = 1 and integer
 * sums, in the distributed shared memory of a 2..16-block thread-block cluster when they
 * fit there (up to 2^18 slots; larger ones stay in HBM). */
typedef struct lpa_tuning {
    int32_t thread_max;       /* thread per vertex for 1 <= D <= thread_max               */
    int32_t group_max;        /* group of group_lanes lanes per vertex                   */
    int32_t group_lanes;      /* 2, 4, 8 or 16                                           */
    int32_t warp_max;         /* warp per vertex                                         */
    int32_t cta_max;          /* block of cta_threads per vertex, smem table             */
    int32_t cta_threads;      /* 64, 128, 256, 512 or 1024 (also for the other tiers)    */
    int32_t cta_large_max;    /* block of cta_large_threads per vertex                   */
    int32_t cta_large_threads;
    int32_t hub_chunk;        /* CSR entries per block in the hub accumulate kernel     */
    int32_t hub_table_shift;  /* 0..3                                                    */
    int32_t smem_table_shift; /* 0..2                                                    */
    int32_t cta_xl_max;       /* block of cta_xl_threads per vertex; above: hubs         */
    int32_t cta_xl_threads;
    int32_t item_vertices;    /* vertices per work item of the thread/group/warp kernels (0 = default) */
    int32_t float_values;     /* label sums: 0 uint32 when exact, else float32; 1 float32;
                                 2 float64 (Section 4.4's 64-bit hashtable values)       */
    int32_t hub_cluster;      /* 1: hub tables in cluster shared memory where they fit   */
    int32_t probe;            /* table probe scheme (Section 4.2): 0 quadratic-double
                                 (Algorithm 2: Mersenne moduli p1, p2), 1 linear,
                                 2 quadratic, 3 double hashing, 4 (the default)
                                 Algorithm 2's quadratic-double recurrence over the
                                 whole power-of-two table with multiplicative hashes;
                                 the table contents, hence the labels, do not depend on it */
    int32_t flat_buckets;     /* bit b (b = 0 thread, 1 group, 2 warp): that bucket runs
                                 the flattened kernel (a warp per batch of vertices whose
                                 rows it scans as one run) instead of one thread / lane
                                 group / warp per vertex                                   */
    int32_t hub_two_pass;     /* hubs with integer sums and HBM tables accumulate in two
                                 passes through shared memory (entries or per-chunk sums sent
                                 to label partitions, then each partition summed) instead of
                                 global atomics on the HBM tables: 0 never, 1 in the first
                                 sweep of a run from fresh labels, 2 in every sweep        */
    int32_t reserved[1];      /* zero                                                    */
} lpa_tuning;

typedef struct lpa_graph lpa_graph;

/* Copies an undirected CSR graph to the device and prepares the degree buckets.
 *  offsets   host or device; int32_t or int64_t [n_vertices + 1] (flags), offsets[0] = 0,
 *            non-decreasing, offsets[n_vertices] = n_entries.
 *  indices   host or device; int32_t [n_entries], each in [0, n_vertices).  Self-loops are
 *            allowed and skipped by the sweep (Algorithm 1 skips j = i).
 *  weights   host or device; float [n_entries], finite and >= 0; NULL = unit weights.
 *            Weights that are all exactly 1 are taken as unit weights (the same sums; the
 *            kernels skip the weight reads and the device copy is released).
 *  n_vertices in [0, 2^31 - 1); n_entries >= 0.
 *  flags     LPA_OFFSETS_I32 / LPA_OFFSETS_I64, LPA_HOST_PTRS / LPA_DEVICE_PTRS,
 *            optionally LPA_CHECK_SYMMETRIC.
 *  cuda_stream the stream all work of the handle is ordered on.
 *  out       receives the handle; NULL on failure.
 * Errors: LPA_EINVAL for a violated precondition (checked on the device), LPA_ENOMEM,
 * LPA_ECUDA.  Labels start as vertex ids (Algorithm 1). */
int lpa_create(const void *offsets, const int32_t *indices, const float *weights,
               int64_t n_vertices, int64_t n_entries, int flags, void *cuda_stream,
               lpa_graph **out);

/* Runs label propagation (Algorithm 1).
 *  tolerance  stop after a non-Pick-Less sweep l with dN / n < tolerance (double compare).
 *  max_iters  absolute cap on the sweep index (the paper uses 20); sweeps run while l < max_iters.
 *  pl_period  Pick-Less on sweeps with l % pl_period == 0 (the paper: 4); 0 disables it.
 *  mode       LPA_SYNC or LPA_ASYNC, optionally | LPA_RESUME.  Without LPA_RESUME the
 *             labels restart at vertex ids, every vertex is unprocessed and l starts at 0;
 *             with it the run continues from the handle's labels, flags and next l.
 *  stats      optional (NULL allowed); see lpa_stats.
 * LPA_SYNC is deterministic: with integer-valued weights and weighted degrees below 2^24
 * every label sum is exact and the labels equal the synchronous definition bit for bit.
 * LPA_ASYNC lets sweeps read labels written in the same sweep (nondeterministic). */
int lpa_run(lpa_graph *g, double tolerance, int max_iters, int pl_period, int mode,
            lpa_stats *stats);

/* lpa_run with the Cross-Check of Section 4.1 after every cc_period-th sweep (sweeps l with
 * l % cc_period == 0; 0 = never, which is lpa_run): each vertex that moved in that sweep keeps
 * its new label c* only when vertex c* is in community c*, else it returns to its label
 * before the sweep.  The paper reverts atomically so that both vertices of a swap do not
 * revert; here the moved vertices are checked in increasing id order against the labels as
 * they stand, earlier reverts included (resolved on the device by pointer jumping over the
 * forest of moves that depend on an earlier mover).  dN counts the moves that remain; marks
 * made during the sweep stay.  pl_period = cc_period > 0 is the paper's Hybrid.  Synchronous
 * mode only (LPA_EINVAL for LPA_ASYNC); the first call with cc_period > 0 allocates 20 bytes per
 * vertex for the check.  LPA_ESTATE if the resolution did not finish (not expected). */
int lpa_run_cc(lpa_graph *g, double tolerance, int max_iters, int pl_period, int cc_period, int mode,
               lpa_stats *stats);

/* Copies the n = n_vertices labels to `out` (host or device per out_on_device). */
int lpa_labels(const lpa_graph *g, int32_t *out, int64_t n, int out_on_device);

/* Modularity of the current labels, Eq. 1 in its community form
 * Q = sum_c [sigma_c / 2m - (Sigma_c / 2m)^2].  With integer weights (and weighted degrees
 * below 2^24) every sum is an exact integer on the device and Q = (2m sigma - sum Sigma_c^2)
 * / (2m)^2 is rounded once; otherwise the sums are accumulated in float64.  The graph is
 * undirected with symmetric weights (lpa_create's precondition): sigma_c counts each edge
 * {i, j} from its entry with j > i at twice its weight.
 * A graph with no edge weight (2m = 0) has Q = 0. */
int lpa_modularity(const lpa_graph *g, double *q);

/* Sets the labels (each in [0, n)), marks every vertex unprocessed and resets the
 * next sweep index to 0 (host or device per on_device). */
int lpa_set_labels(lpa_graph *g, const int32_t *labels, int64_t n, int on_device);

/* Checkpoint of the loop state of Algorithm 1: labels [n], unprocessed flags [n]
 * (0/1) and the next sweep index.  Either array may be NULL. */
int lpa_get_state(const lpa_graph *g, int32_t *labels, uint8_t *unprocessed, int32_t *next_iter,
                  int64_t n, int on_device);
int lpa_set_state(lpa_graph *g, const int32_t *labels, const uint8_t *unprocessed, int32_t next_iter,
                  int64_t n, int on_device);

/* Replaces the stream of the handle (the caller orders any pending work). */
int lpa_set_stream(lpa_graph *g, void *cuda_stream);

/* Degree-bucket configuration of a handle (defaults set by lpa_create). */
int lpa_get_tuning(const lpa_graph *g, lpa_tuning *t);
int lpa_set_tuning(lpa_graph *g, const lpa_tuning *t);

/* Sizes of a handle. */
int64_t lpa_num_vertices(const lpa_graph *g);
int64_t lpa_num_entries(const lpa_graph *g);
/* Device bytes held by a handle. */
int64_t lpa_device_bytes(const lpa_graph *g);

void lpa_destroy(lpa_graph *g);

const char *lpa_strerror(int status);
const char *lpa_last_error(void);

/* Fault injection for tests (host side only, process-wide): after `after` further device
 * allocations by the library succeed, every later one fails with LPA_ENOMEM as if the device
 * were full; a negative value turns it off.  Every entry point must then fail cleanly
 * (no partial handle, nothing leaked).  The paper has no counterpart. */
void lpa_debug_fail_allocations(long long after);

/* Returns the device memory that destroyed single-graph handles left in the library's memory
 * pools to the driver.  Handles take their device memory from one stream-ordered pool per
 * device that keeps freed blocks, so that creating a handle after destroying another does not
 * allocate and free gigabytes again; call this when the memory is wanted elsewhere (another
 * library, a larger allocation).  Synchronises every device that has a pool.  The paper has no
 * counterpart.  LPA_ECUDA if a CUDA call fails. */
int lpa_trim_memory(void);
const char *lpa_kernel_name(int slot);

/* ---- batches: many independent graphs solved together -------------------------------- */

/* One input graph of a batch or a server request: same conventions as lpa_create. */
typedef struct lpa_graph_desc {
    const void *offsets;       /* int32_t or int64_t [n_vertices + 1] (per flags)          */
    const int32_t *indices;    /* [n_entries]                                               */
    const float *weights;      /* [n_entries] or NULL (unit weights)                        */
    int64_t n_vertices;
    int64_t n_entries;
} lpa_graph_desc;

/* Outcome of one graph's run in a batch or a server request. */
typedef struct lpa_result {
    int32_t iterations;        /* sweeps run                                                */
    int32_t converged;         /* 1 when the tolerance test ended the run                   */
    int64_t last_changed;      /* dN of the last sweep                                      */
} lpa_result;

typedef struct lpa_batch lpa_batch;

/* Copies n_graphs independent graphs to the device (one memory arena for all of them) and
 * prepares one combined launch plan: every sweep kernel covers the vertices of every graph,
 * so thousands of small graphs cost the launches of one.  Each graph keeps its own run state
 * (sweep index, Pick-Less phase, changed count, stop decision), so results are the same as
 * running each graph alone with lpa_run.  1 <= n_graphs <= 65535; flags as lpa_create
 * (offset width and host/device pointers apply to every graph).  Errors as lpa_create. */
int lpa_batch_create(int n_graphs, const lpa_graph_desc *descs, int flags, void *cuda_stream, lpa_batch **out);

/* Runs every graph of the batch from fresh labels (Algorithm 1 for each graph, same
 * tolerance, cap, Pick-Less period and mode).  The max_iters sweeps are recorded once into a
 * CUDA graph and replayed; graphs that stop early do no further work.
 *  results   optional, [n_graphs]; device_ms optional (device time of the run). */
int lpa_batch_run(lpa_batch *b, double tolerance, int max_iters, int pl_period, int mode, lpa_result *results,
                  float *device_ms);

/* Labels of graph `graph` (its own vertex ids), n = its n_vertices; host or device out. */
int lpa_batch_labels(const lpa_batch *b, int graph, int32_t *out, int64_t n, int out_on_device);

/* Modularity of every graph, q [n_graphs]. */
int lpa_batch_modularity(lpa_batch *b, double *q);

/* A borrowed handle of graph `graph` (valid until lpa_batch_destroy; do not destroy it): its
 * lpa_run solves that graph alone on the same device data. */
int lpa_batch_graph(lpa_batch *b, int graph, lpa_graph **out);

/* Degree-bucket configuration shared by every graph of the batch (lpa_tuning above); setting
 * it rebuilds every graph's buckets (labels untouched).  LPA_EINVAL as lpa_set_tuning. */
int lpa_batch_get_tuning(const lpa_batch *b, lpa_tuning *t);
int lpa_batch_set_tuning(lpa_batch *b, const lpa_tuning *t);

int lpa_batch_size(const lpa_batch *b);
int64_t lpa_batch_device_bytes(const lpa_batch *b);
void lpa_batch_destroy(lpa_batch *b);

/* ---- server: continuous batching of label-propagation requests ----------------------- */

typedef struct lpa_server lpa_server;

/* A request server on the current device.  Resident requests live in one device arena of
 * hbm_budget_bytes; a request is admitted when its graph fits in the arena (and fewer than
 * max_resident requests are running), in arrival order, later requests passing one that does
 * not fit yet.  Each lpa_server_step admits what fits, runs one sweep of every running request
 * in the same kernel launches (each request at its own sweep index), and retires the requests
 * whose run stopped. */
int lpa_server_create(size_t hbm_budget_bytes, int max_resident, void *cuda_stream, lpa_server **out);

/* Queues a request: the graph (host arrays; flags: offset width) and its run parameters (as
 * lpa_run; mode LPA_SYNC or LPA_ASYNC).  *request_id receives its id.  The arrays are copied at
 * submission, unless flags has LPA_BORROW_INPUTS: then they are read when the request is
 * admitted, and the caller keeps them alive and unchanged until lpa_server_poll lists the
 * request (pinned host memory makes admission's copy fastest).
 * LPA_EINVAL when the graph alone can never fit the budget. */
int lpa_server_submit(lpa_server *s, const lpa_graph_desc *graph, int flags, double tolerance, int max_iters,
                      int pl_period, int mode, int64_t *request_id);

/* One scheduling step (admission, one sweep of every running request, retirement).
 * *n_running and *n_queued (optional) report the state after the step; *n_completed (optional)
 * the requests that finished in this step. */
int lpa_server_step(lpa_server *s, int *n_completed, int *n_running, int *n_queued);

/* Cancels a request: a queued one leaves the queue, a running one is retired (its memory goes
 * back to the arena); either is then listed by lpa_server_poll with status LPA_ECANCELED.
 * LPA_ESTATE when it has already finished, LPA_EINVAL for an unknown id. */
int lpa_server_cancel(lpa_server *s, int64_t request_id);

/* Ids of finished requests not yet collected (at most max_ids); *n receives how many. */
int lpa_server_poll(lpa_server *s, int64_t *ids, int max_ids, int *n);

/* Collects a finished request: labels [n] (host), its result, and its timeline in seconds
 * on the server's clock (submitted, admitted, finished; each may be NULL).  The request is
 * forgotten afterwards.  LPA_ESTATE when the request has not finished. */
int lpa_server_result(lpa_server *s, int64_t request_id, int32_t *labels, int64_t n, lpa_result *result,
                      double *t_submit, double *t_admit, double *t_finish);

/* Seconds on the server's clock (the clock of the timelines above). */
double lpa_server_clock(const lpa_server *s);
int64_t lpa_server_device_bytes(const lpa_server *s);
void lpa_server_destroy(lpa_server *s);

/* ---- autotuning of the degree buckets ---------------------------------------------- */

/* Picks the handle's degree-bucket configuration by timing: a coordinate descent over fixed
 * candidates for each lpa_tuning field (hub chunk, block sizes and thresholds of the three
 * block tiers, warp and group thresholds, lanes per group, thread threshold), starting from
 * the current configuration; hub tables in HBM or in cluster shared memory (hub_cluster) are
 * one more axis.  Every candidate is applied (lpa_set_tuning) and timed on the
 * run given by tolerance / max_iters / pl_period / mode (as lpa_run, from fresh labels; best
 * of reps CUDA-event timings); a candidate is kept when it is at least 2% faster.  Section 4.3
 * chooses its one switch degree (thread vs block per vertex) by timing a range of thresholds
 * offline; this makes that choice per graph, for every bucket boundary and block size.
 * On return the best configuration is installed and copied to *best (optional), its time to
 * *best_ms (optional), the number of timed configurations to *evaluated (optional); the
 * labels are those of the last timed run.  Tuning changes only which kernel handles a vertex
 * and launch shapes: synchronous labels do not depend on it.  LPA_EINVAL for bad arguments
 * (max_iters >= 1, 1 <= reps <= 16). */
int lpa_autotune(lpa_graph *g, double tolerance, int max_iters, int pl_period, int mode, int reps,
                 lpa_tuning *best, float *best_ms, int *evaluated);

/* The same search for a batch: every candidate is applied to all graphs
 * (lpa_batch_set_tuning) and timed by lpa_batch_run's device time. */
int lpa_batch_autotune(lpa_batch *b, double tolerance, int max_iters, int pl_period, int mode, int reps,
                       lpa_tuning *best, float *best_ms, int *evaluated);

/* ---- modularity without device allocation ------------------------------------------ */

/* Largest n_vertices accepted by lpa_modularity_noalloc. */
#define LPA_NOALLOC_MAX_VERTICES (1 << 20)

/* Modularity (Eq. 1) of a labelled CSR graph that the caller holds on the device, computed
 * without allocating any device memory.  The paper has no counterpart: this entry point is
 * for callers that cannot call cudaMalloc, such as code running under another framework's
 * device memory pool, services that have reserved all device memory up front, or paths that
 * must avoid the allocator's implicit synchronisation.
 *  offsets  device, int64_t [n_vertices + 1]; indices device, int32_t [n_entries];
 *  weights  device, float [n_entries] (finite, >= 0) or NULL for unit weights;
 *  labels   device, int32_t [n_vertices], each in [0, n_vertices);
 *  q        host, receives Q (float64 accumulation).
 * Scratch: one fixed array of LPA_NOALLOC_MAX_VERTICES + 8 doubles (8 MiB) compiled into the
 * library; every GPU that loads the library holds it until the process exits, and every call
 * on that GPU uses it.  Calls that overlap on the GPU (other streams or host threads) race on
 * it; order them.  Each call clears the part it reads first.  Every call looks up the array's
 * address on the current device (cudaGetSymbolAddress); cuda_stream must belong to that
 * device.  The call works on cuda_stream and synchronises it before returning, so it must not
 * be made on a stream that is being captured into a CUDA graph.
 * Errors: LPA_EINVAL for n_vertices > LPA_NOALLOC_MAX_VERTICES, NULL arrays, or a graph /
 * labels that fail the device-side checks; LPA_ECUDA for a failed CUDA call. */
int lpa_modularity_noalloc(const int64_t *offsets, const int32_t *indices, const float *weights,
                           const int32_t *labels, int64_t n_vertices, int64_t n_entries,
                           void *cuda_stream, double *q);

/* sizeof(lpa_stats) for which = 0, sizeof(lpa_tuning) for which = 1 (binding checks). */
size_t lpa_struct_size(int which);

#ifdef __cplusplus
}
#endif
#endif /* LPA_H */
