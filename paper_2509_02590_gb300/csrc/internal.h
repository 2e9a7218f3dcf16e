// internal.h -- host-side declarations shared by the library's translation
// units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace wccg {

// A growable device allocation owned by the library.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  int dev = -1;  // device the block belongs to
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf();
  void *ensure(size_t b);  // grows (discarding contents) when b > bytes
  void release();
  template <typename T>
  T *as() const { return static_cast<T *>(p); }
};

// Process-wide count of kernels launched by the library (wcc_kernel_launches).
void note_launch(int64_t k = 1);
int64_t launches_so_far();

// ---- primitives.cu -------------------------------------------------------
// Device-wide exclusive prefix sum out[i] = sum(in[0..i)); `total` (device,
// nullable) receives sum(in[0..n)).  `temp` must hold scan_temp_bytes(n).
size_t scan_temp_bytes(int64_t n);
void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total, void *temp,
                        cudaStream_t s);
void exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total, void *temp,
                        cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on key bits [0, bits), one
// kernel per 8-bit digit.  Uses keys/vals and keys_alt/vals_alt as ping-pong
// buffers; returns true when the sorted result ended in the *_alt buffers.
// `temp`: radix_temp_bytes(n).  A bounded wait that runs out sets
// DERR_TIMEOUT in the device word *err (the caller reads it back).
size_t radix_temp_bytes(int64_t n);
bool radix_sort_pairs_u32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                          int64_t n, int bits, void *temp, unsigned *err, cudaStream_t s);
// Same for 64-bit keys without values, on key bits [0, bits).
bool radix_sort_keys_u64(uint64_t *keys, uint64_t *keys_alt, int64_t n, int bits, void *temp,
                         unsigned *err, cudaStream_t s);

// Per-request workspace of the pipeline stages: grown on demand, kept
// between runs; sk/sv remember where group_by_label() left its sort.
struct Workspace {
  DevBuf b[24];
  uint32_t *sk = nullptr, *sv = nullptr;
};

// ---- csr.cu ----------------------------------------------------------------
// CSR of an edge list by rows (count, scatter, sort every row on chip, pack),
// for graphs whose longest row fits one CTA's shared memory.  Fills off[0..n]
// and adj_buf (room for 2m entries) and returns true; returns false when a
// row is too long, leaving off and adj_buf with unspecified contents (the
// caller then sorts all entries).  An endpoint outside [0, n) fails with
// WCC_ERR_INVALID.  `b`: its temporaries, grown on demand.
constexpr int CSR_ROW_BUFS = 7;
bool csr_by_rows(const int32_t *src, const int32_t *dst, int64_t m, int64_t n, int64_t *off,
                 DevBuf &adj_buf, int64_t *nnz_out, DevBuf (&b)[CSR_ROW_BUFS], cudaStream_t s);

// ---- graph ----------------------------------------------------------------
struct Graph {
  int64_t n = 0;
  int64_t nnz = 0;
  int device = 0;
  DevBuf off;  // int64 [n+1]
  DevBuf adj;  // int32 [nnz]
  std::mutex run_mutex;  // wcc_run calls on one graph are serialised
  // per-run buffers, kept between runs
  Workspace ws;
  DevBuf rb[16];
};

// ---- refine.cu -------------------------------------------------------------
// Work item of the device queue.
struct Item {
  int64_t vbeg;   // start of the item's vertex list in its request's vertex pool
  int32_t n;      // vertices
  uint16_t flags; // ITEM_TOP: an input cluster (CCR first, Algorithm 1);
                  // ITEM_INH: a side of a cut split whose parent left first-pass records
  uint16_t req;   // request it belongs to (index into the request table)
};
enum : uint16_t { ITEM_TOP = 1u, ITEM_INH = 2u };

// One refinement request: its graph, its per-vertex state and its counters.
// wcc_run uses one; a server keeps a table of them for the requests it has
// admitted, and the refinement kernel reads the entry an item names.
struct ReqCtx {
  const int64_t *off;          // graph CSR
  const int32_t *adj;
  int64_t n_vertices;
  int32_t *pool;               // vertex lists of all the request's items
  unsigned long long *slot;    // per vertex: (queue index << 32) | local id, ~0 = none
  int32_t *label_min;          // per vertex: smallest vertex id of its accepted cluster, or -1
  unsigned long long *inh;     // per vertex: record of the last first contraction pass over it
                               // (kcap << 56 | position << 32 | root vertex id); NULL = unused
  int32_t rule_kind, min_size;
  int64_t rule_num, rule_den;
  long long pending;           // published but unfinished items of this request
  long long items, splits, peeled, ni_passes, sw_phases, accepted, alg_bytes;
  unsigned long long seed_end; // end of the queue range of its input clusters (largest first)
};

// A ring slot: the item plus the queue sequence number it was published
// under (seq == index means "ready").
struct QSlot {
  Item item;
  uint64_t seq;
};

// Device counters of one refinement run.
struct RunCounters {
  unsigned long long head;     // next queue index to claim
  unsigned long long tail;     // next queue index to reserve (published once its seq is set)
  long long pending;           // reserved but unfinished items, all requests
  unsigned int error;          // DERR_* bits
  unsigned int err_info;       // first failing detail (debug aid)
  int open;                    // 1 while a server may still add work (kernel idles instead of exiting)
  int closing;                 // set by the first CTA of an open kernel that idled out: all leave
};

// Optional per-item profile record (phase durations in SM cycles: load,
// extraction, CCR, peel, CC, contraction, Stoer-Wagner, output).
struct ItemProf {
  unsigned seq;
  int n, E, nalive, passes, nsv, outcome, smid, slab, top;
  unsigned dt[8];
  long long t_begin, t_end;  // %globaltimer (ns) when the item started and ended
  long long dbg[4];  // first contraction pass: loop cycles, pick cycles, steps, scan cycles
  int forest;        // forest test: rounds it took (negative: gave up after that many)
  int nsv1;          // super-vertices after the first contraction pass
  long long forest_cycles;
  long long fdbg[6];  // forest test: BFS cycles, BFS levels, tree checks, extra trees, degree+contraction, relabel
};

// Per-CTA time split of one profiled run (clock64 cycles of thread 0).
struct CtaProf {
  long long claim;     // claiming and waiting for items
  long long tiny;      // batches of items on single warps
  long long cta;       // items on the whole CTA
  int batches, tiny_items, cta_items, pad;
};

struct RefineParams {
  ReqCtx *reqs;               // request table (device)
  int *done_flags;            // optional, host-mapped: set to 1 when a request's last item ends
  QSlot *ring;
  uint64_t ring_cap;
  RunCounters *ctr;
  uint64_t wait_limit_ns;     // longest wait for a published item while work is pending
  uint64_t idle_limit_ns;     // open kernels leave after this long with nothing pending
  // per-CTA global working memory for items that do not fit in shared memory
  char *slab;
  size_t slab_bytes;          // per CTA
  size_t smem_bytes;          // dynamic shared memory per CTA
  int forest_min_n;           // smallest item that tries the forest acceptance test (0 = never)
  int dense_max;              // most super-vertices the dense finish takes (0 = never)
  int tiny_max;               // items of at most this many vertices run one per warp (0 = never)
  int tiny_max_deg;           // ... when their members' degree sum is at most this
  const volatile int *stop_flag;  // optional, host-mapped: when nonzero, CTAs claim nothing more
  int tickets;                // closed run: claims are tickets (see k_refine)
  int single_item;            // PLAIN mode: process only queue index `single_index`
  unsigned long long single_index;
  ItemProf *prof;             // optional per-item profile (NULL = off)
  CtaProf *prof_cta;          // with prof: one entry per CTA
  unsigned prof_cap;
  unsigned *prof_count;
  // CM (Algorithm 5): the sides of a cut split are written to the pool and
  // listed here for the community step instead of being published
  int cm;
  Item *cda;
  unsigned long long *cda_count;
  unsigned long long cda_cap;
};

// Bytes of working memory an item of n vertices and at most e local
// directed edges needs.
size_t item_workspace_bytes(int64_t n, int64_t e);
int refine_block_threads();
size_t refine_smem_max_bytes(int device);
// CTAs of the refinement kernel resident on the whole device with
// smem_bytes of dynamic shared memory each.
int refine_max_ctas(int device, size_t smem_bytes);
void launch_refine(const RefineParams &p, int grid, bool cooperative, cudaStream_t s);

// ---- pipeline.cu: the stages around the refinement kernel ------------------
// Result of grouping one request's vertices by input label.
struct GroupInfo {
  int64_t clusters;   // distinct labels >= 0
  int64_t skip;       // unclustered vertices
  int64_t kept;       // clusters with >= min_size vertices (they become items)
  int64_t max_n;      // largest kept cluster
  int64_t max_dsum;   // largest degree sum of a kept cluster
};

// a2: groups the vertices of labels (device) by input label (stable radix
// sort), computes the kept clusters, their sizes and degree sums, and orders
// them largest first.  Leaves its arrays in ws for seed_items().  One
// read-back inside (the sort width) plus one at the end (the result).
GroupInfo group_by_label(const int64_t *off, int64_t n, const int32_t *labels, int min_size,
                         Workspace &ws, cudaStream_t s);

// Publishes the kept clusters of the last group_by_label() on ws as ITEM_TOP
// items of request `req` (context at reqs_dev + req): reserves their queue
// indices, fills pool and slot (which must hold ~0 for every vertex), writes
// the descriptors and publishes them.  Asynchronous on s.
void seed_items(const GroupInfo &gi, int64_t n, Workspace &ws, uint16_t req, ReqCtx *ctx_dev,
                int32_t *pool, unsigned long long *slot, QSlot *ring, uint64_t cap,
                RunCounters *ctr, cudaStream_t s);

// a9: out[v] = rank of the accepted cluster whose smallest vertex is
// label_min[v] (ascending), -1 where label_min is -1.  Asynchronous on s.
// Per vertex, the smallest vertex of its cluster (labels in [-1, n)).
void cluster_minima(const int32_t *labels, int64_t n, int32_t *minima, Workspace &ws,
                    cudaStream_t s);
// *out = max(*out, largest entry of a[0..n)).
void k_max_i32_launch(const int32_t *a, int64_t n, int32_t *out, cudaStream_t s);
// WCC_ERR_INVALID unless every entry is -1 or a representative r <= v with
// minima[r] == r.
void check_minima(const int32_t *minima, int64_t n, Workspace &ws, cudaStream_t s);
void number_clusters(const int32_t *label_min, int64_t n, int32_t *out, Workspace &ws,
                     cudaStream_t s);

int64_t bitlen_u64(uint64_t x);
unsigned grid_for(int64_t n, int per = 256);
void check_device_error(unsigned err, const char *what);

// ---- api.cu helpers shared with the server ------------------------------------
int current_device();                       // fails with WCC_ERR_CUDA without a GPU
uint64_t wait_limit_ns();                   // WCC_WAIT_LIMIT_MS (default 30 s)
size_t refine_smem_bytes_config(int device);  // WCC_SMEM_KB (default: opt-in maximum)
int forest_min_n_config();                    // WCC_FOREST_MIN_N
int dense_max_config();                       // WCC_DENSE_NSV
int tiny_max_config();                        // WCC_TINY_N
int tiny_max_deg_config();                    // WCC_TINY_DEG

// ---- job.cu: a refinement in resumable steps --------------------------------
struct Job;
Job *job_start(Graph *g, const int32_t *lab_in, const wcc_threshold_rule *rule, int32_t min_size,
               int on_device, cudaStream_t s);
bool job_step(Job *j, int64_t budget_ms, cudaStream_t s);  // true: the queue is empty
void job_finish(Job *j, int32_t *out, int on_device, cudaStream_t s, wcc_stats *stats);
void job_save(Job *j, const char *path, cudaStream_t s);
Job *job_load(Graph *g, const char *path, cudaStream_t s);
void job_destroy(Job *j);
// The process-wide tuning the *_config() functions fall back to.
wcc_tuning current_tuning();
void store_tuning(const wcc_tuning &t);
bool tuning_valid(const wcc_tuning &t);

wcc_threshold_rule checked_rule(const wcc_threshold_rule *rule);
// A graph from an edge list, built on the device (the CSR builder of
// wcc_create_graph_from_edges); host edges are copied first (on_device 0).
Graph *create_from_edges(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                         int on_device, cudaStream_t s);

template <typename T>
T read_back(const T *dev, cudaStream_t s) {
  T h;
  WCC_CUDA(cudaMemcpyAsync(&h, dev, sizeof(T), cudaMemcpyDeviceToHost, s));
  WCC_CUDA(cudaStreamSynchronize(s));
  return h;
}

// ---- cm.cu ----------------------------------------------------------------
// The community step of CM over the parts a refinement run parked
// (RefineParams::cda, nparts of them): CPM local moving at gnum/gden and the
// connected parts of every community, written back to the pool; the
// communities of at least min_size members are reserved at the queue's tail
// (head reset to it), their slots set and published.  partof / loc: int32
// [n_vertices], -1 on entry and on return.  max_n / max_dsum bound a part's
// size and degree sum (those of the largest input cluster).  Returns the
// number of items published.
unsigned long long cm_round(const Item *parts, unsigned long long nparts, ReqCtx *reqs,
                            int64_t gnum, int64_t gden, int32_t *partof, int32_t *loc,
                            int64_t n_vertices, int64_t max_n, int64_t max_dsum, RunCounters *ctr,
                            QSlot *ring, uint64_t cap, int grid_max, DevBuf &scratch,
                            DevBuf &items, DevBuf &misc, cudaStream_t s);

}  // namespace wccg

// The opaque handle of the C ABI.
struct wcc_graph {
  wccg::Graph *g;
};
