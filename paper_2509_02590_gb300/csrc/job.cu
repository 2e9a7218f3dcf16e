// job.cu -- a refinement in resumable steps, with the device queue as its
// checkpoint.
//
// wcc_run grows the queue from the input clusters and drains it in one
// kernel.  A job does the same in steps: each step runs the persistent
// kernel until the queue is empty or a time budget is over; then a
// host-mapped stop flag makes every CTA stop claiming, so the kernel ends at
// an item boundary with the queue intact: the items in [head, tail) (each a
// vertex list in the pool, a size and its flags), the accepted clusters so
// far (label_min) and the counters.  That state is all a later step needs,
// so it can be written to a file and loaded again onto the same graph --
// in another process, after a restart -- and the result is the one wcc_run
// gives.  A loaded queue is renumbered from 0 and its vertices' slots are
// rebuilt from the item lists.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#include "internal.h"

namespace wccg {

struct Job {
  Graph *g = nullptr;
  int device = 0;
  wcc_threshold_rule rule{};
  int32_t min_size = 2;
  int64_t n = 0, in_clusters = 0, max_n = 0, max_dsum = 0, pool_len = 0;
  uint64_t cap = 0;
  int grid = 0;
  size_t smem_bytes = 0, slab_bytes = 0;
  DevBuf pool, slot, lmin, inh, ring, ctr, req, slab, out;
  int *stop_host = nullptr, *stop_dev = nullptr;
  bool done = false;
  ~Job() {
    if (stop_host) cudaFreeHost(stop_host);
  }
};

namespace {

constexpr char MAGIC[8] = {'W', 'C', 'C', 'J', 'O', 'B', '1', 0};

// slot[v] = (queue tag << 32) | position of v in its item, for every member
// of the queued items [0, count).  One CTA per item.
__global__ void k_job_slots(const QSlot *__restrict__ ring, const int32_t *__restrict__ pool,
                            unsigned long long count, unsigned long long *slot) {
  const unsigned long long q = blockIdx.x;
  if (q >= count) return;
  const Item it = ring[q].item;
  const unsigned long long tag = (unsigned long long)queue_tag(q) << 32;
  for (int p = threadIdx.x; p < it.n; p += blockDim.x) slot[pool[it.vbeg + p]] = tag | (unsigned)p;
}

// *maxd = the largest member degree sum over the queued items [0, count).
// One CTA per item.
__global__ void k_job_dsum(const QSlot *__restrict__ items, const int32_t *__restrict__ pool,
                           const int64_t *__restrict__ off, unsigned long long count,
                           unsigned long long *maxd) {
  __shared__ long long part[32];
  const unsigned long long q = blockIdx.x;
  if (q >= count) return;
  const Item it = items[q].item;
  long long d = 0;
  for (int p = threadIdx.x; p < it.n; p += blockDim.x) {
    const int32_t v = pool[it.vbeg + p];
    d += off[v + 1] - off[v];
  }
  d = warp_sum(d);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x < 32) {
    long long t = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0;
    t = warp_sum(t);
    if (threadIdx.x == 0) atomicMax(maxd, (unsigned long long)t);
  }
}

void sizes_for(Job &j) {
  j.smem_bytes = refine_smem_bytes_config(j.device);
  j.grid = refine_max_ctas(j.device, j.smem_bytes);
  j.cap = (uint64_t)j.n + 2ull * j.grid + 1024;
  const size_t need = item_workspace_bytes(j.max_n, j.max_dsum);
  j.slab_bytes = need > j.smem_bytes ? ((need + 255) & ~(size_t)255) : 256;
}

void alloc_common(Job &j) {
  j.slot.ensure(8 * (size_t)std::max<int64_t>(j.n, 1));
  j.lmin.ensure(4 * (size_t)std::max<int64_t>(j.n, 1));
  j.inh.ensure(8 * (size_t)std::max<int64_t>(j.n, 1));
  j.ring.ensure(sizeof(QSlot) * j.cap);
  j.ctr.ensure(sizeof(RunCounters));
  j.req.ensure(sizeof(ReqCtx));
  j.slab.ensure(j.slab_bytes * (size_t)j.grid);
  WCC_CUDA(cudaHostAlloc((void **)&j.stop_host, sizeof(int), cudaHostAllocMapped));
  *j.stop_host = 0;
  WCC_CUDA(cudaHostGetDevicePointer((void **)&j.stop_dev, j.stop_host, 0));
}

ReqCtx request_of(const Job &j) {
  ReqCtx h{};
  h.off = j.g->off.as<int64_t>();
  h.adj = j.g->adj.as<int32_t>();
  h.n_vertices = j.n;
  h.pool = j.pool.as<int32_t>();
  h.slot = j.slot.as<unsigned long long>();
  h.label_min = j.lmin.as<int32_t>();
  h.inh = j.inh.as<unsigned long long>();
  h.rule_kind = j.rule.kind;
  h.min_size = j.min_size;
  h.rule_num = j.rule.num;
  h.rule_den = j.rule.den;
  return h;
}

}  // namespace

Job *job_start(Graph *g, const int32_t *lab_in, const wcc_threshold_rule *rule, int32_t min_size,
               int on_device, cudaStream_t s) {
  std::unique_ptr<Job> j(new Job());
  j->g = g;
  j->device = g->device;
  j->rule = checked_rule(rule);
  j->min_size = min_size < 2 ? 2 : min_size;
  j->n = g->n;
  const int64_t n = j->n;
  if (n > 0 && lab_in == nullptr) fail(WCC_ERR_INVALID, "clustering_in is NULL");
  DevBuf in;
  const int32_t *d_in = lab_in;
  if (n > 0 && !on_device) {
    int32_t *p = static_cast<int32_t *>(in.ensure(4 * (size_t)n));
    WCC_CUDA(cudaMemcpyAsync(p, lab_in, 4 * (size_t)n, cudaMemcpyHostToDevice, s));
    d_in = p;
  }
  GroupInfo gi{};
  if (n > 0) gi = group_by_label(g->off.as<int64_t>(), n, d_in, j->min_size, g->ws, s);
  j->in_clusters = gi.clusters;
  j->max_n = gi.max_n;
  j->max_dsum = gi.max_dsum;
  j->pool_len = std::max<int64_t>(n - gi.skip, 1);
  sizes_for(*j);
  j->pool.ensure(4 * (size_t)j->pool_len);
  alloc_common(*j);
  if (n > 0) {
    WCC_CUDA(cudaMemsetAsync(j->slot.p, 0xff, 8 * (size_t)n, s));
    WCC_CUDA(cudaMemsetAsync(j->lmin.p, 0xff, 4 * (size_t)n, s));
  }
  WCC_CUDA(cudaMemsetAsync(j->ctr.p, 0, sizeof(RunCounters), s));
  const ReqCtx h = request_of(*j);
  WCC_CUDA(cudaMemcpyAsync(j->req.p, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  if (gi.kept > 0) {
    WCC_CUDA(cudaMemsetAsync(j->ring.p, 0xff, sizeof(QSlot) * j->cap, s));
    seed_items(gi, n, g->ws, 0, j->req.as<ReqCtx>(), j->pool.as<int32_t>(),
               j->slot.as<unsigned long long>(), j->ring.as<QSlot>(), j->cap,
               j->ctr.as<RunCounters>(), s);
  } else {
    j->done = true;
  }
  WCC_CUDA(cudaStreamSynchronize(s));
  return j.release();
}

// Runs the kernel until the queue is empty (returns true) or budget_ms has
// passed (false; budget_ms < 0: no limit).
bool job_step(Job *j, int64_t budget_ms, cudaStream_t s) {
  if (j->done) return true;
  *(volatile int *)j->stop_host = 0;
  RefineParams p{};
  p.reqs = j->req.as<ReqCtx>();
  p.ring = j->ring.as<QSlot>();
  p.ring_cap = j->cap;
  p.ctr = j->ctr.as<RunCounters>();
  p.wait_limit_ns = wait_limit_ns();
  p.idle_limit_ns = 0;
  p.smem_bytes = j->smem_bytes;
  p.slab = j->slab.as<char>();
  p.slab_bytes = j->slab_bytes;
  p.forest_min_n = forest_min_n_config();
  p.dense_max = dense_max_config();
  p.tiny_max = tiny_max_config();
  p.tiny_max_deg = tiny_max_deg_config();
  p.stop_flag = j->stop_dev;
  cudaEvent_t ev;
  WCC_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  try {
    launch_refine(p, j->grid, true, s);
    WCC_CUDA(cudaEventRecord(ev, s));
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      const cudaError_t q = cudaEventQuery(ev);
      if (q == cudaSuccess) break;
      if (q != cudaErrorNotReady) WCC_CUDA(q);
      if (budget_ms >= 0 &&
          std::chrono::steady_clock::now() - t0 >= std::chrono::milliseconds(budget_ms)) {
        // every CTA finishes its current item and leaves
        *(volatile int *)j->stop_host = 1;
        WCC_CUDA(cudaEventSynchronize(ev));
        break;
      }
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
  } catch (...) {
    cudaEventDestroy(ev);
    throw;
  }
  cudaEventDestroy(ev);
  const RunCounters c = read_back(j->ctr.as<RunCounters>(), s);
  if (c.error) {
    fail((c.error & DERR_TIMEOUT) ? WCC_ERR_TIMEOUT : WCC_ERR_INTERNAL,
         "refinement failed on the device (error bits " + std::to_string(c.error) + ")");
  }
  j->done = c.pending <= 0;
  return j->done;
}

void job_finish(Job *j, int32_t *out, int on_device, cudaStream_t s, wcc_stats *stats) {
  if (!j->done) fail(WCC_ERR_BUSY, "the job still has queued work: step it to completion first");
  if (!out && j->n > 0) fail(WCC_ERR_INVALID, "clustering_out is NULL");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (j->n == 0) return;
  int32_t *d_out = out;
  if (!on_device) d_out = static_cast<int32_t *>(j->out.ensure(4 * (size_t)j->n));
  number_clusters(j->lmin.as<int32_t>(), j->n, d_out, j->g->ws, s);
  if (!on_device)
    WCC_CUDA(cudaMemcpyAsync(out, d_out, 4 * (size_t)j->n, cudaMemcpyDeviceToHost, s));
  const ReqCtx h = read_back(j->req.as<ReqCtx>(), s);
  if (stats) {
    stats->in_clusters = j->in_clusters;
    stats->out_clusters = h.accepted;
    stats->items = h.items;
    stats->splits = h.splits;
    stats->peeled = h.peeled;
    stats->ni_passes = h.ni_passes;
    stats->sw_phases = h.sw_phases;
    stats->max_item = j->max_n;
    stats->alg_bytes = h.alg_bytes;
  }
}

// File layout (little-endian): magic[8]; int64 n, nnz, in_clusters, max_n,
// max_dsum; int32 rule kind, min_size; int64 rule num, den; int64 items,
// splits, peeled, ni_passes, sw_phases, accepted, alg_bytes; int64 queued
// items P, their members M; P x {int32 size, int32 flags}; M x int32 member
// ids (item after item); n x int32 label_min; uint64 FNV-1a of everything
// before it.
namespace {
struct Writer {
  FILE *f;
  uint64_t h = 1469598103934665603ull;
  void put(const void *p, size_t b) {
    const unsigned char *c = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < b; ++i) h = (h ^ c[i]) * 1099511628211ull;
    if (fwrite(p, 1, b, f) != b) fail(WCC_ERR_INVALID, "short write");
  }
  template <typename T>
  void put(const T &v) { put(&v, sizeof(v)); }
};
struct Reader {
  FILE *f;
  uint64_t h = 1469598103934665603ull;
  void get(void *p, size_t b) {
    if (fread(p, 1, b, f) != b) fail(WCC_ERR_INVALID, "truncated job file");
    const unsigned char *c = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < b; ++i) h = (h ^ c[i]) * 1099511628211ull;
  }
  template <typename T>
  T get() {
    T v;
    get(&v, sizeof(v));
    return v;
  }
};
}  // namespace

void job_save(Job *j, const char *path, cudaStream_t s) {
  if (!path) fail(WCC_ERR_INVALID, "path is NULL");
  const RunCounters c = read_back(j->ctr.as<RunCounters>(), s);
  if (c.error) fail(WCC_ERR_INTERNAL, "the job failed on the device; nothing to save");
  const ReqCtx h = read_back(j->req.as<ReqCtx>(), s);
  const uint64_t P = c.tail - c.head;
  std::vector<QSlot> q(P);
  if (P) {
    // the ring slots [head, tail), in at most two pieces
    const uint64_t a = c.head % j->cap, first = std::min<uint64_t>(P, j->cap - a);
    WCC_CUDA(cudaMemcpyAsync(q.data(), j->ring.as<QSlot>() + a, sizeof(QSlot) * first,
                             cudaMemcpyDeviceToHost, s));
    if (first < P)
      WCC_CUDA(cudaMemcpyAsync(q.data() + first, j->ring.as<QSlot>(), sizeof(QSlot) * (P - first),
                               cudaMemcpyDeviceToHost, s));
  }
  std::vector<int32_t> pool((size_t)j->pool_len), lmin((size_t)j->n);
  WCC_CUDA(cudaMemcpyAsync(pool.data(), j->pool.p, 4 * (size_t)j->pool_len, cudaMemcpyDeviceToHost, s));
  if (j->n)
    WCC_CUDA(cudaMemcpyAsync(lmin.data(), j->lmin.p, 4 * (size_t)j->n, cudaMemcpyDeviceToHost, s));
  WCC_CUDA(cudaStreamSynchronize(s));
  int64_t M = 0;
  for (uint64_t i = 0; i < P; ++i) {
    if (q[i].seq != c.head + i) fail(WCC_ERR_INTERNAL, "a queued item is not published");
    M += q[i].item.n;
  }
  FILE *f = fopen(path, "wb");
  if (!f) fail(WCC_ERR_INVALID, std::string("cannot write ") + path);
  Writer w{f};
  try {
    w.put(MAGIC, sizeof(MAGIC));
    for (int64_t v : {j->n, j->g->nnz, j->in_clusters, j->max_n, j->max_dsum}) w.put(v);
    w.put((int32_t)j->rule.kind);
    w.put((int32_t)j->min_size);
    w.put((int64_t)j->rule.num);
    w.put((int64_t)j->rule.den);
    for (long long v : {h.items, h.splits, h.peeled, h.ni_passes, h.sw_phases, h.accepted, h.alg_bytes})
      w.put((int64_t)v);
    w.put((int64_t)P);
    w.put(M);
    for (uint64_t i = 0; i < P; ++i) {
      w.put((int32_t)q[i].item.n);
      // first-pass records are not saved: a resumed item computes its own
      w.put((int32_t)(q[i].item.flags & ITEM_TOP));
    }
    for (uint64_t i = 0; i < P; ++i) w.put(pool.data() + q[i].item.vbeg, 4 * (size_t)q[i].item.n);
    if (j->n) w.put(lmin.data(), 4 * (size_t)j->n);
    const uint64_t sum = w.h;
    w.put(sum);
  } catch (...) {
    fclose(f);
    throw;
  }
  if (fclose(f) != 0) fail(WCC_ERR_INVALID, std::string("cannot write ") + path);
}

Job *job_load(Graph *g, const char *path, cudaStream_t s) {
  if (!path) fail(WCC_ERR_INVALID, "path is NULL");
  FILE *f = fopen(path, "rb");
  if (!f) fail(WCC_ERR_INVALID, std::string("cannot read ") + path);
  std::unique_ptr<Job> j(new Job());
  std::vector<int32_t> sizes, flags, members, lmin;
  int64_t P = 0;
  try {
    Reader r{f};
    char magic[8];
    r.get(magic, sizeof(magic));
    if (std::memcmp(magic, MAGIC, sizeof(MAGIC)) != 0) fail(WCC_ERR_INVALID, "not a job file");
    const int64_t n = r.get<int64_t>(), nnz = r.get<int64_t>();
    if (n != g->n || nnz != g->nnz)
      fail(WCC_ERR_INVALID, "the job file belongs to another graph (vertex or edge count differs)");
    j->in_clusters = r.get<int64_t>();
    // the stored largest item and degree sum are informational: the working
    // memory is sized from the loaded items themselves below
    (void)r.get<int64_t>();
    (void)r.get<int64_t>();
    j->rule.kind = r.get<int32_t>();
    j->min_size = std::max<int32_t>(2, r.get<int32_t>());
    j->rule.num = r.get<int64_t>();
    j->rule.den = r.get<int64_t>();
    j->rule = checked_rule(&j->rule);
    int64_t st[7];
    for (int64_t &v : st) v = r.get<int64_t>();
    P = r.get<int64_t>();
    const int64_t M = r.get<int64_t>();
    if (P < 0 || M < 0 || M > n || P > n) fail(WCC_ERR_INVALID, "corrupt job file (counts)");
    sizes.resize((size_t)P);
    flags.resize((size_t)P);
    int64_t sum_m = 0;
    for (int64_t i = 0; i < P; ++i) {
      sizes[i] = r.get<int32_t>();
      flags[i] = r.get<int32_t>();
      if (sizes[i] < 1) fail(WCC_ERR_INVALID, "corrupt job file (item size)");
      sum_m += sizes[i];
    }
    if (sum_m != M) fail(WCC_ERR_INVALID, "corrupt job file (member count)");
    members.resize((size_t)M);
    if (M) r.get(members.data(), 4 * (size_t)M);
    {
      std::vector<uint8_t> seen((size_t)n, 0);
      for (int32_t v : members) {
        if (v < 0 || v >= n) fail(WCC_ERR_INVALID, "corrupt job file (vertex id)");
        if (seen[v]++) fail(WCC_ERR_INVALID, "corrupt job file (a vertex listed twice)");
      }
    }
    lmin.resize((size_t)n);
    if (n) r.get(lmin.data(), 4 * (size_t)n);
    for (int32_t x : lmin)
      if (x < -1 || x >= n) fail(WCC_ERR_INVALID, "corrupt job file (cluster minimum)");
    const uint64_t want = r.h;
    uint64_t got = 0;
    if (fread(&got, 1, sizeof(got), f) != sizeof(got) || got != want)
      fail(WCC_ERR_INVALID, "corrupt job file (checksum)");
    fclose(f);
    f = nullptr;
    j->g = g;
    j->device = g->device;
    j->n = n;
    j->pool_len = std::max<int64_t>(M, 1);
    // the queue renumbered from 0, item lists packed in order
    std::vector<QSlot> q((size_t)P);
    int64_t at = 0;
    j->max_n = 0;
    for (int64_t i = 0; i < P; ++i) {
      q[i].item.vbeg = at;
      q[i].item.n = sizes[i];
      q[i].item.flags = (uint16_t)(flags[i] & ITEM_TOP);
      q[i].item.req = 0;
      q[i].seq = (uint64_t)i;
      at += sizes[i];
      j->max_n = std::max<int64_t>(j->max_n, sizes[i]);
    }
    j->pool.ensure(4 * (size_t)j->pool_len);
    if (M)
      WCC_CUDA(cudaMemcpyAsync(j->pool.p, members.data(), 4 * (size_t)M, cudaMemcpyHostToDevice, s));
    j->max_dsum = 0;
    if (P) {
      DevBuf tq, td;
      auto *dq = static_cast<QSlot *>(tq.ensure(sizeof(QSlot) * (size_t)P));
      auto *dmax = static_cast<unsigned long long *>(td.ensure(8));
      WCC_CUDA(cudaMemcpyAsync(dq, q.data(), sizeof(QSlot) * (size_t)P, cudaMemcpyHostToDevice, s));
      WCC_CUDA(cudaMemsetAsync(dmax, 0, 8, s));
      k_job_dsum<<<(unsigned)P, 256, 0, s>>>(dq, j->pool.as<int32_t>(), g->off.as<int64_t>(),
                                             (unsigned long long)P, dmax);
      note_launch();
      WCC_CUDA(cudaGetLastError());
      j->max_dsum = (int64_t)read_back(dmax, s);
    }
    sizes_for(*j);
    alloc_common(*j);
    if (n) {
      WCC_CUDA(cudaMemcpyAsync(j->lmin.p, lmin.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, s));
      WCC_CUDA(cudaMemsetAsync(j->slot.p, 0xff, 8 * (size_t)n, s));
    }
    WCC_CUDA(cudaMemsetAsync(j->ring.p, 0xff, sizeof(QSlot) * j->cap, s));
    if (P)
      WCC_CUDA(cudaMemcpyAsync(j->ring.p, q.data(), sizeof(QSlot) * (size_t)P, cudaMemcpyHostToDevice, s));
    RunCounters c{};
    c.head = 0;
    c.tail = (unsigned long long)P;
    c.pending = P;
    WCC_CUDA(cudaMemcpyAsync(j->ctr.p, &c, sizeof(c), cudaMemcpyHostToDevice, s));
    ReqCtx h = request_of(*j);
    h.pending = P;
    h.items = st[0];
    h.splits = st[1];
    h.peeled = st[2];
    h.ni_passes = st[3];
    h.sw_phases = st[4];
    h.accepted = st[5];
    h.alg_bytes = st[6];
    h.seed_end = 0;  // no block claims over the loaded items: one per claim, same results
    WCC_CUDA(cudaMemcpyAsync(j->req.p, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    if (P) {
      k_job_slots<<<(unsigned)P, 256, 0, s>>>(j->ring.as<QSlot>(), j->pool.as<int32_t>(),
                                              (unsigned long long)P, j->slot.as<unsigned long long>());
      note_launch();
      WCC_CUDA(cudaGetLastError());
    }
    WCC_CUDA(cudaStreamSynchronize(s));
    j->done = P == 0;
  } catch (...) {
    if (f) fclose(f);
    throw;
  }
  return j.release();
}

void job_destroy(Job *j) { delete j; }

}  // namespace wccg
