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

// Stable LSD radix sort of (key, value) pairs on key bits [0, bits).  Uses
// keys/vals and keys_alt/vals_alt as ping-pong buffers; returns true when the
// sorted result ended in the *_alt buffers.  `temp`: radix_temp_bytes(n).
size_t radix_temp_bytes(int64_t n);
bool radix_sort_pairs_u32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                          int64_t n, int bits, void *temp, cudaStream_t s);
// Same for 64-bit keys without values, on key bits [0, bits).
bool radix_sort_keys_u64(uint64_t *keys, uint64_t *keys_alt, int64_t n, int bits, void *temp,
                         cudaStream_t s);

// ---- graph ----------------------------------------------------------------
struct Graph {
  int64_t n = 0;
  int64_t nnz = 0;
  int device = 0;
  DevBuf off;  // int64 [n+1]
  DevBuf adj;  // int32 [nnz]
  std::mutex run_mutex;  // wcc_run calls on one graph are serialised
  // per-run workspace, kept between runs
  DevBuf ws[32];
};

// ---- refine.cu -------------------------------------------------------------
// Work item of the device queue.
struct Item {
  int64_t vbeg;   // start of the item's vertex list in the vertex pool
  int32_t n;      // vertices
  uint32_t flags; // ITEM_TOP: an input cluster (CCR first, Algorithm 1)
};
enum : uint32_t { ITEM_TOP = 1u };

// A ring slot: the item plus the queue sequence number it was published
// under (seq == index means "ready").
struct QSlot {
  Item item;
  uint64_t seq;
};

// Device counters of one refinement run.
struct RunCounters {
  unsigned long long head;     // next queue index to claim
  unsigned long long tail;     // next queue index to publish
  long long pending;           // published but unfinished items
  unsigned int error;          // DERR_* bits
  unsigned int err_info;       // first failing detail (debug aid)
  long long items, splits, peeled, ni_passes, sw_phases, accepted;
  long long alg_bytes;         // bytes of adjacency + slot gathers actually read
};

// Optional per-item profile record (phase durations in SM cycles: load,
// extraction, CCR, peel, CC, contraction, Stoer-Wagner, output).
struct ItemProf {
  unsigned seq;
  int n, E, nalive, passes, nsv, outcome, smid, slab, top;
  unsigned dt[8];
  long long t_begin;
  long long dbg[4];  // first contraction pass: loop cycles, pick cycles, steps, scan cycles
};

struct RefineParams {
  const int64_t *off;
  const int32_t *adj;
  int64_t n_vertices;
  int32_t *pool;              // vertex lists of all items (length = clustered vertices)
  unsigned long long *slot;   // per vertex: (item seq << 32) | local id, ~0 = none
  int32_t *label_min;         // per vertex: smallest vertex id of its accepted cluster, or -1
  QSlot *ring;
  uint64_t ring_cap;
  RunCounters *ctr;
  int32_t rule_kind;
  int64_t rule_num, rule_den;
  int32_t min_size;
  uint64_t wait_limit_ns;
  // per-CTA global working memory for items that do not fit in shared memory
  char *slab;
  size_t slab_bytes;          // per CTA
  size_t smem_bytes;          // dynamic shared memory per CTA
  int single_item;            // PLAIN mode: process only queue index `single_index`
  unsigned long long single_index;
  ItemProf *prof;             // optional per-item profile (NULL = off)
  unsigned prof_cap;
  unsigned *prof_count;
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

}  // namespace wccg
