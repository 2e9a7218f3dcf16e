/*
 * wcc.h -- C ABI of the GB300 Well-Connected Clusters (WCC) refinement library.
 *
 * WCC (paper Section 2.3, Algorithms 2 and 3, with the connected component
 * refinement CCR of Section 2.2, Algorithm 1) takes a graph G and a
 * clustering C and returns the clusters of C refined until each one is well
 * connected: every input cluster is split into connected components, low
 * degree vertices are peeled, an exact minimum edge cut is computed, and a
 * cluster whose cut is at or below the criterion f(n) (Section 2; log10 n in
 * Section 3) is bisected on that cut and both sides are refined again, until
 * every part is accepted or is smaller than the size threshold.
 *
 * Every step runs in this library's CUDA kernels on one GPU.  There is no CPU
 * fallback: without a usable GPU every call returns WCC_ERR_CUDA.
 *
 * Conventions for every function:
 *   - Status codes are returned; nothing throws across the ABI.  On any
 *     status other than WCC_OK / WCC_PENDING, wcc_last_error() returns a
 *     thread-local message describing the failure, and output buffers are
 *     left unspecified.
 *   - The caller owns every input and output buffer and keeps it valid for
 *     the duration of the call.  Handles returned by the library are owned by
 *     the caller until the matching destroy call.
 *   - on_device = 1: pointer arguments marked "host or device" are CUDA
 *     device pointers (e.g. torch.Tensor.data_ptr() of a CUDA tensor) and
 *     `stream` (a cudaStream_t, NULL = the legacy default stream) orders the
 *     library's work after the caller's prior work on that stream.
 *     on_device = 0: they are host pointers; the library copies them.
 *   - All calls are synchronous with respect to the host unless stated.
 *   - Vertex ids are int32 in [0, n); edge offsets are int64.
 */
#ifndef WCC_H
#define WCC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wcc_graph wcc_graph;
typedef struct wcc_server wcc_server;

typedef enum {
  WCC_OK = 0,
  WCC_PENDING = 1,        /* request not finished yet (wcc_poll) */
  WCC_ERR_INVALID = -1,   /* malformed argument or graph */
  WCC_ERR_OOM = -2,       /* device memory (or a configured budget) exhausted */
  WCC_ERR_CUDA = -3,      /* CUDA runtime / launch failure, or no GPU */
  WCC_ERR_TIMEOUT = -4,   /* a bounded device-side wait ran out */
  WCC_ERR_BUSY = -5,      /* request can never fit the server's budget */
  WCC_ERR_INTERNAL = -6   /* a consistency check inside the library failed */
} wcc_status;

/* Criterion f(n) of Section 2 in exact integer form: a cluster of n vertices
 * whose minimum cut is c fails iff c <= T(n), where T(n) is
 *   LOG10:  largest t with 10^t <= n   (floor(log10 n); the rule of Section 3)
 *   LOG2:   largest t with 2^t <= n
 *   SQRT:   largest t with t*t <= n
 *   LINEAR: floor(num * n / den)       (f(n) = k n with k = num/den) */
typedef enum {
  WCC_RULE_LOG10 = 0,
  WCC_RULE_LOG2 = 1,
  WCC_RULE_SQRT = 2,
  WCC_RULE_LINEAR = 3
} wcc_rule_kind;

typedef struct {
  int32_t kind;  /* wcc_rule_kind */
  int32_t reserved;
  int64_t num;   /* LINEAR only: 0 <= num < 2^31 */
  int64_t den;   /* LINEAR only: 0 < den < 2^31 */
} wcc_threshold_rule;

/* Execution schedule of wcc_run.  Both give bit-identical results.
 *   BATCHED: one persistent cooperative kernel drains a device-side work
 *            queue holding every work item (input clusters and the parts
 *            produced by splits), many items in flight at once.
 *   PLAIN:   one kernel launch per work item, driven by a host loop. */
typedef enum { WCC_MODE_BATCHED = 0, WCC_MODE_PLAIN = 1 } wcc_mode;

typedef struct {
  int64_t in_clusters;   /* distinct input labels >= 0 */
  int64_t out_clusters;  /* accepted clusters */
  int64_t items;         /* work items processed */
  int64_t splits;        /* items bisected on their min cut */
  int64_t peeled;        /* vertices removed by peeling */
  int64_t ni_passes;     /* contraction passes (maximum-adjacency orderings) */
  int64_t sw_phases;     /* Stoer-Wagner phases */
  int64_t max_item;      /* largest input cluster refined (vertices) */
  int64_t alg_bytes;     /* algorithmic HBM bytes of the refinement's extractions: 8 B per
                          * member of an input cluster (row offsets) plus 8 B per adjacency
                          * entry of every extracted item (neighbour id and its label) */
  double ms_membership;  /* device time: grouping vertices by input label */
  double ms_refine;      /* device time: the refinement kernel(s) */
  double ms_output;      /* device time: numbering the accepted clusters */
  double ms_total;       /* host wall time of the call */
} wcc_stats;

/* Create a graph from a CSR.  row_off[n+1] (int64, row_off[0] = 0,
 * non-decreasing, row_off[n] = nnz) and cols[nnz] (int32) describe a simple
 * undirected graph: each row strictly ascending (no repeated neighbours), no
 * self-loop, and v in row u iff u in row v.  The whole CSR is checked on the
 * device; a violation returns WCC_ERR_INVALID.  The graph keeps its own
 * device copy; the input buffers (host or device) may be freed on return.
 * Graph data structure: the CSR part of the double-index format of
 * Section 2.1. */
int wcc_create_graph(const int64_t *row_off, const int32_t *cols, int64_t n, int64_t nnz,
                     int on_device, void *stream, wcc_graph **out);

/* Create a graph from an edge list src[m], dst[m] (host or device, int32 ids
 * in [0, n)), built on the device: both directions, self-loops and repeated
 * edges dropped, rows sorted.  An id outside [0, n) returns
 * WCC_ERR_INVALID. */
int wcc_create_graph_from_edges(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                                int on_device, void *stream, wcc_graph **out);

/* Number of vertices / directed CSR entries (2 x undirected edges). */
int64_t wcc_graph_num_vertices(const wcc_graph *g);
int64_t wcc_graph_nnz(const wcc_graph *g);

/* Copy the graph's CSR out (host or device buffers of n+1 and nnz
 * entries). */
int wcc_graph_export_csr(const wcc_graph *g, int64_t *row_off, int32_t *cols, int on_device,
                         void *stream);

/* Refine a clustering (Algorithm 2 with CCR first).
 *   clustering_in[n]  (host or device) int32: input cluster of each vertex,
 *                     any value >= 0; -1 = vertex in no cluster.
 *   rule              criterion (NULL = LOG10).
 *   min_size          smallest part kept: the paper's s_pre = s_post = s is
 *                     min_size = s + 1 (Section 3 uses s = 1, min_size 2);
 *                     values below 2 act as 2.
 *   mode              wcc_mode.
 *   clustering_out[n] (host or device) int32: accepted clusters numbered
 *                     0..K-1 in ascending order of their smallest vertex id,
 *                     -1 for every vertex in no accepted cluster.  Written
 *                     only on WCC_OK.  May not alias clustering_in.
 *   stats             optional (NULL to skip).
 * Returns WCC_OK, WCC_ERR_INVALID (bad rule or sizes), WCC_ERR_OOM,
 * WCC_ERR_CUDA, WCC_ERR_TIMEOUT (a device-side queue wait exceeded its
 * limit) or WCC_ERR_INTERNAL. */
int wcc_run(const wcc_graph *g, const int32_t *clustering_in, const wcc_threshold_rule *rule,
            int32_t min_size, int32_t mode, int32_t *clustering_out, int on_device, void *stream,
            wcc_stats *stats);

/* CM refinement (Section 2.4, Algorithms 4-5): wcc_run in BATCHED mode,
 * except that each part of a cut split with at least min_size vertices first
 * goes through the community step (GetCommunities of Algorithm 5), and every
 * community of at least min_size vertices is checked again (peel,
 * connectivity, cut) like any other part.  The community step is CPM local
 * moving at resolution cpm_num / cpm_den on the part's induced subgraph:
 * sweeps over the part's vertices in ascending id, from singletons, at most
 * 64 sweeps or until one moves nothing; a vertex taken out of its community
 * c0 joins the neighbouring community c of largest gain
 * k(v,c) * cpm_den - cpm_num * |c| (|c| without v; or, when c0 keeps other
 * members, an empty community with gain 0: the id n + v while no vertex holds
 * it, else the smallest id no vertex holds, with community ids 0..2n-1 over
 * the part's n vertices and vertex v starting in v), ties to the smallest
 * community id, and only when that gain beats staying in c0; then every
 * community is split into its connected parts.  Arguments,
 * layouts and results as wcc_run.  WCC_ERR_INVALID unless
 * 0 <= cpm_num <= 2^31 and 1 <= cpm_den <= 2^31. */
int wcc_run_cm(const wcc_graph *g, const int32_t *clustering_in, const wcc_threshold_rule *rule,
               int32_t min_size, int64_t cpm_num, int64_t cpm_den, int32_t *clustering_out,
               int on_device, void *stream, wcc_stats *stats);

/* Release a graph (NULL is ignored). */
void wcc_destroy_graph(wcc_graph *g);

/* ---- serving: continuous batching of refinement requests ----------------
 * A server refines many requests at once in one persistent kernel: requests
 * are admitted in arrival order whenever a request slot is free and their
 * estimated device memory fits the budget, and a request admitted while
 * others are on the GPU joins the running kernel at once (its work overlaps
 * theirs).  Every result equals what wcc_run returns for the same input.
 * The server takes the device current at wcc_server_create; every graph
 * submitted with wcc_submit must live on that device and stay alive (not
 * destroyed) until its request has been collected by wcc_poll / wcc_wait.
 * wcc_submit_edges hands the server an edge list instead: the server then
 * builds, keeps and releases the request's graph itself. */

/* Create a server using at most mem_budget_bytes of device memory for its
 * queue, slabs and admitted requests.  WCC_ERR_INVALID if the budget cannot
 * hold the fixed structures and one small request. */
int wcc_server_create(int64_t mem_budget_bytes, wcc_server **out);

/* Queue a refinement of graph g with the host clustering clustering_in[n]
 * (copied before the call returns), rule (NULL = LOG10) and min_size as in
 * wcc_run.  *ticket identifies the request.  WCC_ERR_BUSY when the request
 * can never fit the server's budget or queue. */
int wcc_submit(wcc_server *s, const wcc_graph *g, const int32_t *clustering_in,
               const wcc_threshold_rule *rule, int32_t min_size, uint64_t *ticket);

/* Queue a refinement of a graph given as an edge list: src[m], dst[m] (host,
 * int32 ids in [0, n)) on n vertices, with clustering_in[n] (host), rule and
 * min_size as in wcc_run.  clustering_in is copied before the call returns;
 * src and dst are not: the server reads them when it admits the request, so
 * they must stay valid and unchanged until the request's result has been
 * collected (or the server destroyed).  Pinned host memory makes that upload
 * a direct DMA.  The server builds the graph on the device on admission
 * (both directions, self-loops and repeated edges dropped, as
 * wcc_create_graph_from_edges) and releases it when the request finishes;
 * the graph's CSR counts against the budget for the request's lifetime, the
 * builder's transient memory during the admission.  An id outside [0, n)
 * fails the request (WCC_ERR_INVALID from wcc_poll / wcc_wait).
 * WCC_ERR_BUSY when the request can never fit the budget or queue. */
int wcc_submit_edges(wcc_server *s, const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                     const int32_t *clustering_in, const wcc_threshold_rule *rule,
                     int32_t min_size, uint64_t *ticket);

/* Admission counters of a server (instrumentation). */
typedef struct {
  int64_t budget_bytes;     /* budget left for requests after the fixed structures */
  int64_t used_bytes;       /* held by the requests admitted now */
  int64_t peak_used_bytes;  /* most ever held at once (with a build's transient memory) */
  int64_t admitted;         /* requests admitted so far */
  int64_t budget_waits;     /* requests that had to wait for budget before admission */
  int64_t slot_waits;       /* admission attempts that found every request slot taken */
  int64_t peak_active;      /* most requests admitted at once */
  int64_t max_active;       /* request slots */
} wcc_server_counters;
int wcc_server_info(wcc_server *s, wcc_server_counters *out);

/* Non-blocking: WCC_PENDING while the request runs; WCC_OK once finished,
 * with the result written to the host buffer clustering_out[n] (numbered as
 * in wcc_run) and stats filled (nullable; ms_total = submit to finish,
 * ms_refine = admission to finish, ms_membership = grouping); or the
 * request's error.  A ticket is collected once; afterwards it is unknown
 * (WCC_ERR_INVALID). */
int wcc_poll(wcc_server *s, uint64_t ticket, int32_t *clustering_out, wcc_stats *stats);

/* As wcc_poll, but waits up to timeout_ms for the request to finish;
 * returns WCC_PENDING if it is still running then. */
int wcc_wait(wcc_server *s, uint64_t ticket, int64_t timeout_ms, int32_t *clustering_out,
             wcc_stats *stats);

/* Finish every submitted request, stop the server and release it (NULL is
 * ignored).  Results not collected by then are discarded. */
void wcc_server_destroy(wcc_server *s);

/* Build a CSR without allocating any memory.  The paper has no counterpart:
 * this is a service for callers that cannot allocate device memory, for
 * example code running under an allocator that owns the whole device, a
 * host framework that forbids allocation after start-up, or a caller that
 * must not add allocations to a carefully sized memory budget.  It computes
 * the same CSR as wcc_create_graph_from_edges + wcc_graph_export_csr (both
 * directions, self-loops and repeated edges dropped, rows sorted) but writes
 * it straight into the caller's device buffers.
 *   src[m], dst[m]  device int32 edge endpoints in [0, n).
 *   row_off[n+1]    device int64 output; cols: device int32 output with room
 *                   for 2*m entries (the first *nnz are written).
 *   nnz             host int64 output: number of directed entries.
 *   stream          cudaStream_t the work is ordered on (NULL = legacy
 *                   default stream); the call returns after it finishes.
 * Limits: m <= 131072 (2^17) and n <= 4194304 (2^22); larger inputs return
 * WCC_ERR_INVALID with a message naming the limit, as does an endpoint
 * outside [0, n).
 * Its working memory is one fixed array of about 6.5 MB in the library's
 * static device memory, present on every GPU that loads the library until
 * the process exits; the call itself performs no device allocation (see
 * wcc_device_allocations).  The array's address is looked up on every call
 * with the current device; `stream` must belong to that device, else
 * WCC_ERR_INVALID.  The array is shared by all calls and keeps the last
 * call's contents (each call clears what it needs), so calls that may
 * overlap on the GPU -- different streams, or several host threads -- race
 * and must be serialised by the caller.  The call reads values back and
 * synchronises `stream` before it returns, so it cannot be recorded into a
 * CUDA graph (stream capture). */
int wcc_build_csr_no_alloc(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                           int64_t *row_off, int32_t *cols, int64_t *nnz, void *stream);

/* ---- tuning ------------------------------------------------------------
 * The refinement kernel schedules work items by size: items of at most
 * tiny_max vertices run one per warp (up to 8 per CTA) unless their members'
 * degree sum exceeds tiny_max_deg; larger items run on a whole CTA in shared
 * memory (smem_kb per CTA) or, when they do not fit, in a global slab; after
 * the first contraction pass, at most dense_max super-vertices finish on a
 * dense weight matrix; items of at least forest_min_n vertices first try the
 * forest acceptance test.  None of these changes a result, only the time.
 * The setting is process-wide; the environment variables WCC_TINY_N,
 * WCC_TINY_DEG, WCC_DENSE_NSV, WCC_FOREST_MIN_N and WCC_SMEM_KB, when set,
 * take precedence over it. */
typedef struct wcc_tuning {
  int32_t tiny_max;      /* 0..64 (0: no item runs on a single warp) */
  int32_t tiny_max_deg;  /* >= 0 */
  int32_t dense_max;     /* 0..128 (0: always the sparse passes) */
  int32_t forest_min_n;  /* >= 0 (0: never) */
  int32_t smem_kb;       /* >= 0 (0: the largest a CTA can opt into) */
  int32_t reserved[3];   /* zero */
} wcc_tuning;

/* Current process-wide tuning (before environment overrides).  Needs no GPU. */
int wcc_get_tuning(wcc_tuning *out);

/* Sets the process-wide tuning; values outside the ranges above return
 * WCC_ERR_INVALID and change nothing.  Needs no GPU. */
int wcc_set_tuning(const wcc_tuning *t);

/* Autotuner: times wcc_run (BATCHED) of this graph and clustering under a
 * small set of candidate tunings (one knob at a time from the current one,
 * keeping each improvement), checks that every candidate gives the same
 * refined clustering (else WCC_ERR_INTERNAL), sets the fastest as the
 * process-wide tuning and returns it in *best (time of one run in *best_ms,
 * either may be NULL).  clustering_in as for wcc_run (host or device, per
 * on_device); stream as for wcc_run.  When cache_path is not NULL the result
 * is written there as a small JSON object naming the device (see
 * wcc_load_tuning).  Takes about 2 x (number of candidates) runs. */
int wcc_autotune(const wcc_graph *g, const int32_t *clustering_in, const wcc_threshold_rule *rule,
                 int32_t min_size, int on_device, void *stream, const char *cache_path,
                 wcc_tuning *best, double *best_ms);

/* Reads a tuning written by wcc_autotune and sets it process-wide (and
 * returns it in *out, which may be NULL).  When a GPU is present and the
 * file names another device model, nothing is set and WCC_ERR_INVALID is
 * returned; a missing or malformed file also returns WCC_ERR_INVALID. */
int wcc_load_tuning(const char *cache_path, wcc_tuning *out);

/* ---- resumable runs (checkpoint / resume) ----------------------------------
 * A job is wcc_run in steps.  wcc_job_start groups the clustering and queues
 * the input clusters (Algorithm 1's loop) without refining anything;
 * wcc_job_step runs the refinement until the queue is empty (WCC_OK) or
 * time_budget_ms has passed (WCC_PENDING: the kernel stopped at an item
 * boundary, every queued item is kept; time_budget_ms < 0: no limit).
 * Every CTA of a step takes one queued item before it looks at the time, so
 * each step that returns WCC_PENDING has made progress, even with budget 0.
 * wcc_job_save writes the queue -- the queued items' vertex lists, the
 * clusters accepted so far, the statistics -- to a file; wcc_job_load
 * rebuilds a job from it on a graph with the same vertex and edge counts
 * (the graph itself is not stored: load it onto the same graph).
 * wcc_job_finish, once a step has returned WCC_OK (else WCC_ERR_BUSY),
 * writes the refined clustering exactly as wcc_run would, with the same
 * conventions for clustering_out / on_device / stream / stats.  The result
 * does not depend on where the steps stopped or on a save/load in between.
 * A job uses its graph until wcc_job_destroy; destroy jobs before their
 * graph.  Loading checks a checksum and returns WCC_ERR_INVALID on a
 * corrupt, truncated or foreign file. */
typedef struct wcc_job wcc_job;
int wcc_job_start(const wcc_graph *g, const int32_t *clustering_in, const wcc_threshold_rule *rule,
                  int32_t min_size, int on_device, void *stream, wcc_job **out);
int wcc_job_step(wcc_job *job, int64_t time_budget_ms, void *stream);
int wcc_job_save(wcc_job *job, const char *path, void *stream);
int wcc_job_load(const wcc_graph *g, const char *path, void *stream, wcc_job **out);
int wcc_job_finish(wcc_job *job, int32_t *clustering_out, int on_device, void *stream,
                   wcc_stats *stats);
void wcc_job_destroy(wcc_job *job);

/* ---- one graph's input clusters refined on several GPUs -----------------
 * Algorithms 1-2 refine every input cluster on its own (Section 2.2-2.3), so
 * the input clusters of one graph can be split into disjoint shards, one
 * per GPU, each refined with wcc_run on a full copy of the graph (labels of
 * other shards set to -1).  The shard results are merged through cluster
 * minima: per vertex, the smallest vertex id of its output cluster.  The
 * shards' minima arrays are disjoint (-1 outside the shard), so their
 * element-wise maximum (one all-reduce) is the minima of the whole run, and
 * wcc_number_by_minima numbers it exactly as a single wcc_run would. */

/* Per vertex v, the smallest vertex id of v's cluster: labels[n] (host or
 * device per on_device, int32 in [-1, n), -1 = no cluster, e.g. the output
 * of wcc_run) -> minima[n] (-1 where labels is -1).  A label outside
 * [-1, n) returns WCC_ERR_INVALID. */
int wcc_cluster_minima(const int32_t *labels, int64_t n, int32_t *minima, int on_device,
                       void *stream);

/* Canonical numbering from cluster minima (as wcc_cluster_minima writes
 * them): labels_out[n] gets 0..K-1 in ascending order of each cluster's
 * smallest vertex and -1 where minima is -1, the numbering of wcc_run; *k
 * (nullable) receives K.  Every entry must be -1 or a vertex r <= v with
 * minima[r] == r, else WCC_ERR_INVALID. */
int wcc_number_by_minima(const int32_t *minima, int64_t n, int32_t *labels_out, int64_t *k,
                         int on_device, void *stream);

/* Number of CUDA kernels this library has launched in this process so far
 * (instrumentation: lets a caller count the kernels of a timed region). */
int64_t wcc_kernel_launches(void);

/* Number of device allocations (cudaMalloc calls) this library has made in
 * this process so far.  Freed blocks are cached and reused, so repeated
 * calls of the same sizes usually add none; instrumentation only. */
int64_t wcc_device_allocations(void);

/* Message of the last failure on the calling thread ("" if none). */
const char *wcc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* WCC_H */
