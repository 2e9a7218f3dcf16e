// server.cu -- continuous-batching refinement service (wcc_server_*,
// wcc_submit, wcc_poll, wcc_wait).
//
// One persistent refinement kernel serves every admitted request at once:
// the device queue holds items of different requests (each item names its
// request's context in a device table), so a request that arrives while
// others are being refined is grouped, seeded and picked up by the running
// kernel without waiting for them.  A host worker thread
//   - admits waiting requests in arrival order when a request slot is free,
//     their estimated device memory fits the budget and the queue has room;
//   - groups each admitted request's vertices by label and publishes its
//     input clusters on a side stream (the kernel leaves RESERVED_SMS
//     streaming multiprocessors free for that work);
//   - watches per-request completion flags the kernel sets in host-mapped
//     memory, numbers the finished request's clusters, copies them out and
//     releases its memory;
//   - relaunches the kernel whenever it has gone idle and work is pending.
// The kernel runs with its queue "open": with nothing pending it waits
// (bounded by an idle limit) instead of exiting, and when it does leave, it
// leaves as a whole (no CTA keeps running alone on work admitted late).
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace wccg {

namespace {

constexpr int MAX_SLOTS = 256;        // requests refined at the same time
constexpr int RESERVED_SMS = 8;       // left free for grouping / seeding / numbering
constexpr uint64_t IDLE_LIMIT_NS = 5ull * 1000 * 1000;

using clock_t_ = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  Graph *g = nullptr;
  int64_t n = 0;
  // the input labels' copy and the result, in pageable host memory: pinning
  // or unpinning memory per request (cudaHostAlloc / cudaFreeHost) waits for
  // the device, and the device runs the open refinement kernel until it
  // idles, so each submission or collection would stall on the whole load
  std::vector<int32_t> h_in, h_out;
  // a request that brings its graph as an edge list: the caller's edge
  // buffers (valid until the request is collected), then the graph the
  // server builds from them on admission and owns
  const int32_t *h_src = nullptr, *h_dst = nullptr;
  int64_t m = 0;
  std::unique_ptr<Graph> own;
  size_t build_bytes = 0;    // transient device memory of building that graph
  bool waited_budget = false;
  wcc_threshold_rule rule{};
  int min_size = 2;
  size_t est_bytes = 0;
  int64_t ring_need = 0;
  int status = WCC_PENDING;
  std::string error;
  wcc_stats stats{};
  clock_t_::time_point t_submit, t_admit;
  // device state while admitted
  int slot = -1;
  Workspace ws;
  DevBuf d_in, d_out, pool, vslot, lmin, inh;
  GroupInfo gi{};
  void release_device() {
    for (auto &b : ws.b) b.release();
    d_in.release();
    d_out.release();
    pool.release();
    vslot.release();
    lmin.release();
    inh.release();
    if (own) {
      own.reset();
      g = nullptr;
    }
  }
};

// Device bytes one request of n vertices may hold at once: its state (input
// and output labels, vertex pool, slots, cluster minima, first-pass records)
// and the grouping workspace, about 120 bytes per vertex, doubled for the
// power-of-two block rounding of the allocator, plus 1 MB.
size_t estimate_bytes(int64_t n) { return (size_t)n * 240 + (1u << 20); }

// A graph the server builds from an edge list: its CSR (int64 offsets,
// int32 columns for both directions), rounded up like every block, held
// until the request finishes.
size_t graph_bytes(int64_t n, int64_t m) { return 2 * (8 * (size_t)(n + 1) + 8 * (size_t)m); }

// The builder's transient memory while one such graph is built (the edge
// copies, two 64-bit key arrays and two 32-bit flag arrays over the 2m
// directed entries, scan and sort temporaries), rounded up: needed only
// during the admission that builds it.
size_t build_bytes(int64_t n, int64_t m) { return 2 * (56 * (size_t)m + 8 * (size_t)n) + (1u << 20); }

struct Server {
  int device = 0;
  int64_t budget = 0, used = 0;
  int grid = 0;
  size_t smem_bytes = 0, slab_bytes = 0;
  uint64_t ring_cap = 0;
  int64_t ring_reserved = 0;
  DevBuf ring, ctr, slab, reqtab;
  int *done_host = nullptr;  // host-mapped completion flags, one per slot
  int *done_dev = nullptr;
  cudaStream_t kstream = nullptr, astream = nullptr;
  cudaEvent_t kdone = nullptr;
  bool kernel_running = false;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> waiting;
  std::unordered_map<uint64_t, Request *> tickets;
  Request *active[MAX_SLOTS] = {};
  int n_active = 0;
  bool stop = false;
  uint64_t next_ticket = 1;
  // counters (wcc_server_info)
  int64_t admitted = 0, budget_waits = 0, slot_waits = 0, peak_used = 0, peak_active = 0;
};

void finish(Server *S, Request *R, int status, const std::string &err) {
  std::lock_guard<std::mutex> lk(S->mu);
  R->status = status;
  R->error = err;
  R->stats.ms_total =
      std::chrono::duration<double, std::milli>(clock_t_::now() - R->t_submit).count();
  S->cv_done.notify_all();
}

void free_slot(Server *S, Request *R) {
  if (R->slot >= 0) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->active[R->slot] = nullptr;
    ((volatile int *)S->done_host)[R->slot] = 0;
    R->slot = -1;
    --S->n_active;
    S->used -= (int64_t)R->est_bytes;
    S->ring_reserved -= R->ring_need;
  }
  R->release_device();
}

// Numbers the finished request's clusters, copies them to the host and
// releases its device memory.
void finalize(Server *S, Request *R) {
  try {
    ReqCtx *ctx = S->reqtab.as<ReqCtx>() + R->slot;
    number_clusters(R->lmin.as<int32_t>(), R->n, R->d_out.as<int32_t>(), R->ws, S->astream);
    WCC_CUDA(cudaMemcpyAsync(R->h_out.data(), R->d_out.p, 4 * R->n, cudaMemcpyDeviceToHost,
                             S->astream));
    ReqCtx h = read_back(ctx, S->astream);
    R->stats.in_clusters = R->gi.clusters;
    R->stats.out_clusters = h.accepted;
    R->stats.items = h.items;
    R->stats.splits = h.splits;
    R->stats.peeled = h.peeled;
    R->stats.ni_passes = h.ni_passes;
    R->stats.sw_phases = h.sw_phases;
    R->stats.max_item = R->gi.max_n;
    R->stats.alg_bytes = h.alg_bytes;
    R->stats.ms_refine =
        std::chrono::duration<double, std::milli>(clock_t_::now() - R->t_admit).count();
    free_slot(S, R);
    finish(S, R, WCC_OK, "");
  } catch (const Error &e) {
    free_slot(S, R);
    finish(S, R, e.code, e.msg);
  }
}

bool can_admit(Server *S, Request *R) {
  if (S->n_active >= MAX_SLOTS) {
    ++S->slot_waits;
    return false;
  }
  if (S->used + (int64_t)(R->est_bytes + R->build_bytes) > S->budget) {
    if (!R->waited_budget) ++S->budget_waits;
    R->waited_budget = true;
    return false;
  }
  if ((uint64_t)(S->ring_reserved + R->ring_need) + (uint64_t)S->grid + 1024 > S->ring_cap)
    return false;
  return true;
}

// Groups the request, fills its context and publishes its input clusters.
void admit(Server *S, Request *R) {
  int slot = 0;
  while (S->active[slot]) ++slot;
  R->slot = slot;
  S->active[slot] = R;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    ++S->n_active;
    S->used += (int64_t)R->est_bytes;
    S->ring_reserved += R->ring_need;
    ++S->admitted;
    S->peak_used = std::max<int64_t>(S->peak_used, S->used + (int64_t)R->build_bytes);
    S->peak_active = std::max<int64_t>(S->peak_active, S->n_active);
  }
  R->t_admit = clock_t_::now();
  try {
    const int64_t n = R->n;
    cudaStream_t s = S->astream;
    if (!R->g) {
      // the request's own graph, built on the device from its edge list
      R->own.reset(create_from_edges(R->h_src, R->h_dst, R->m, n, 0, s));
      R->g = R->own.get();
      R->h_src = R->h_dst = nullptr;
    }
    int32_t *d_in = static_cast<int32_t *>(R->d_in.ensure(4 * n));
    WCC_CUDA(cudaMemcpyAsync(d_in, R->h_in.data(), 4 * n, cudaMemcpyHostToDevice, s));
    auto t0 = clock_t_::now();
    R->gi = group_by_label(R->g->off.as<int64_t>(), n, d_in, R->min_size, R->ws, s);
    R->stats.ms_membership =
        std::chrono::duration<double, std::milli>(clock_t_::now() - t0).count();
    const size_t need = item_workspace_bytes(R->gi.max_n, R->gi.max_dsum);
    if (R->gi.kept > 0 && need > S->smem_bytes && need > S->slab_bytes)
      fail(WCC_ERR_BUSY, "the largest input cluster (" + std::to_string(R->gi.max_n) +
                             " vertices) needs more working memory than this server's " +
                             std::to_string(S->slab_bytes) + "-byte per-CTA slab");
    int32_t *pool = static_cast<int32_t *>(R->pool.ensure(4 * std::max<int64_t>(n - R->gi.skip, 1)));
    auto *vslot = static_cast<unsigned long long *>(R->vslot.ensure(8 * n));
    auto *lmin = static_cast<int32_t *>(R->lmin.ensure(4 * n));
    auto *inh = static_cast<unsigned long long *>(R->inh.ensure(8 * n));
    R->d_out.ensure(4 * n);
    WCC_CUDA(cudaMemsetAsync(vslot, 0xff, 8 * n, s));
    WCC_CUDA(cudaMemsetAsync(lmin, 0xff, 4 * n, s));
    ReqCtx h{};
    h.off = R->g->off.as<int64_t>();
    h.adj = R->g->adj.as<int32_t>();
    h.n_vertices = n;
    h.pool = pool;
    h.slot = vslot;
    h.label_min = lmin;
    h.inh = inh;
    h.rule_kind = R->rule.kind;
    h.min_size = R->min_size;
    h.rule_num = R->rule.num;
    h.rule_den = R->rule.den;
    ReqCtx *ctx = S->reqtab.as<ReqCtx>() + slot;
    WCC_CUDA(cudaMemcpyAsync(ctx, &h, sizeof(h), cudaMemcpyHostToDevice, s));
    ((volatile int *)S->done_host)[slot] = 0;
    if (R->gi.kept > 0)
      seed_items(R->gi, n, R->ws, (uint16_t)slot, ctx, pool, vslot, S->ring.as<QSlot>(),
                 S->ring_cap, S->ctr.as<RunCounters>(), s);
    WCC_CUDA(cudaStreamSynchronize(s));
    if (R->gi.kept == 0) finalize(S, R);
  } catch (const Error &e) {
    free_slot(S, R);
    finish(S, R, e.code, e.msg);
  }
}

void launch_kernel(Server *S) {
  RefineParams p{};
  p.reqs = S->reqtab.as<ReqCtx>();
  p.done_flags = S->done_dev;
  p.ring = S->ring.as<QSlot>();
  p.ring_cap = S->ring_cap;
  p.ctr = S->ctr.as<RunCounters>();
  p.wait_limit_ns = wait_limit_ns();
  p.idle_limit_ns = IDLE_LIMIT_NS;
  p.smem_bytes = S->smem_bytes;
  p.forest_min_n = forest_min_n_config();
  p.dense_max = dense_max_config();
  p.tiny_max = tiny_max_config();
  p.tiny_max_deg = tiny_max_deg_config();
  p.slab = S->slab.as<char>();
  p.slab_bytes = S->slab_bytes;
  // a previous instance may have closed on idling out; the launch reopens
  WCC_CUDA(cudaMemsetAsync(&S->ctr.as<RunCounters>()->closing, 0, sizeof(int), S->kstream));
  launch_refine(p, S->grid, true, S->kstream);
  WCC_CUDA(cudaEventRecord(S->kdone, S->kstream));
  S->kernel_running = true;
}

// After a kernel reported an error: fail every admitted request and reset
// the queue.
void reset_after_error(Server *S, unsigned err) {
  std::string msg;
  try {
    check_device_error(err, "refinement");
  } catch (const Error &e) {
    msg = e.msg;
  }
  for (int k = 0; k < MAX_SLOTS; ++k) {
    Request *R = S->active[k];
    if (!R) continue;
    free_slot(S, R);
    finish(S, R, (err & DERR_TIMEOUT) ? WCC_ERR_TIMEOUT : WCC_ERR_INTERNAL, msg);
  }
  RunCounters c{};
  c.open = 1;
  WCC_CUDA(cudaMemcpyAsync(S->ctr.p, &c, sizeof(c), cudaMemcpyHostToDevice, S->astream));
  WCC_CUDA(cudaMemsetAsync(S->ring.p, 0xff, sizeof(QSlot) * S->ring_cap, S->astream));
  WCC_CUDA(cudaStreamSynchronize(S->astream));
}

void worker_loop(Server *S) {
  cudaSetDevice(S->device);
  for (;;) {
    bool busy = false;
    try {
      for (int k = 0; k < MAX_SLOTS; ++k) {
        Request *R = S->active[k];
        if (R && ((volatile int *)S->done_host)[k]) {
          finalize(S, R);
          busy = true;
        }
      }
      if (S->kernel_running && cudaEventQuery(S->kdone) == cudaSuccess) {
        S->kernel_running = false;
        RunCounters c = read_back(S->ctr.as<RunCounters>(), S->astream);
        if (c.error) reset_after_error(S, c.error);
      }
      for (;;) {
        Request *R = nullptr;
        {
          std::lock_guard<std::mutex> lk(S->mu);
          if (!S->waiting.empty() && can_admit(S, S->waiting.front())) {
            R = S->waiting.front();
            S->waiting.pop_front();
          }
        }
        if (!R) break;
        admit(S, R);
        busy = true;
      }
      if (!S->kernel_running && S->n_active > 0) {
        launch_kernel(S);
        busy = true;
      }
    } catch (const Error &e) {
      // a CUDA failure outside a request: fail what is admitted
      for (int k = 0; k < MAX_SLOTS; ++k)
        if (S->active[k]) {
          Request *R = S->active[k];
          free_slot(S, R);
          finish(S, R, e.code, e.msg);
        }
    }
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->stop && S->waiting.empty() && S->n_active == 0) break;
    if (!busy) S->cv_work.wait_for(lk, std::chrono::microseconds(50));
  }
  // close the queue so that the kernel leaves, then wait for it
  RunCounters c{};
  cudaMemcpyAsync(&S->ctr.as<RunCounters>()->open, &c.open, sizeof(int), cudaMemcpyHostToDevice,
                  S->astream);
  cudaStreamSynchronize(S->astream);
  cudaStreamSynchronize(S->kstream);
}

Server *create_server(int64_t budget) {
  std::unique_ptr<Server> S(new Server());
  S->device = current_device();
  S->budget = budget;
  S->smem_bytes = refine_smem_max_bytes(S->device);
  const int sms_total = refine_max_ctas(S->device, S->smem_bytes);
  int sms = 0;
  WCC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device));
  S->grid = std::max(1, std::min(sms_total, sms) - RESERVED_SMS);
  S->ring_cap = (uint64_t)std::min<int64_t>(std::max<int64_t>(budget / 2048, 1 << 16), 1 << 26);
  S->slab_bytes = (size_t)std::min<int64_t>(std::max<int64_t>(budget / (8 * S->grid), 1 << 20),
                                            64ll << 20);
  S->slab_bytes = (S->slab_bytes + 255) & ~(size_t)255;
  const int64_t fixed = (int64_t)(sizeof(QSlot) * S->ring_cap + S->slab_bytes * S->grid +
                                  sizeof(ReqCtx) * MAX_SLOTS + 4096);
  if (budget < fixed + (int64_t)estimate_bytes(1024))
    fail(WCC_ERR_INVALID, "memory budget " + std::to_string(budget) +
                              " is below the server's fixed structures (" +
                              std::to_string(fixed) + " bytes) plus one small request");
  S->budget -= fixed;
  S->ring.ensure(sizeof(QSlot) * S->ring_cap);
  S->ctr.ensure(sizeof(RunCounters));
  S->slab.ensure(S->slab_bytes * (size_t)S->grid);
  S->reqtab.ensure(sizeof(ReqCtx) * MAX_SLOTS);
  WCC_CUDA(cudaHostAlloc((void **)&S->done_host, sizeof(int) * MAX_SLOTS, cudaHostAllocMapped));
  std::memset(S->done_host, 0, sizeof(int) * MAX_SLOTS);
  WCC_CUDA(cudaHostGetDevicePointer((void **)&S->done_dev, S->done_host, 0));
  WCC_CUDA(cudaStreamCreateWithFlags(&S->kstream, cudaStreamNonBlocking));
  WCC_CUDA(cudaStreamCreateWithFlags(&S->astream, cudaStreamNonBlocking));
  WCC_CUDA(cudaEventCreateWithFlags(&S->kdone, cudaEventDisableTiming));
  RunCounters c{};
  c.open = 1;
  WCC_CUDA(cudaMemcpyAsync(S->ctr.p, &c, sizeof(c), cudaMemcpyHostToDevice, S->astream));
  WCC_CUDA(cudaMemsetAsync(S->ring.p, 0xff, sizeof(QSlot) * S->ring_cap, S->astream));
  WCC_CUDA(cudaMemsetAsync(S->reqtab.p, 0, sizeof(ReqCtx) * MAX_SLOTS, S->astream));
  WCC_CUDA(cudaStreamSynchronize(S->astream));
  Server *raw = S.get();
  S->worker = std::thread(worker_loop, raw);
  return S.release();
}

void destroy_server(Server *S) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto &kv : S->tickets) delete kv.second;
  if (S->kdone) cudaEventDestroy(S->kdone);
  if (S->kstream) cudaStreamDestroy(S->kstream);
  if (S->astream) cudaStreamDestroy(S->astream);
  if (S->done_host) cudaFreeHost(S->done_host);
  delete S;
}

// Queues a request: of graph g, or (g == NULL) of the graph of the edge list
// src[m], dst[m] on n vertices, which the server builds when it admits the
// request and releases when the request finishes.
uint64_t submit(Server *S, Graph *g, const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                const int32_t *labels, const wcc_threshold_rule *rule, int32_t min_size) {
  std::unique_ptr<Request> R(new Request());
  if (g) {
    if (g->device != S->device) fail(WCC_ERR_INVALID, "graph and server are on different devices");
    n = g->n;
    R->g = g;
    R->est_bytes = estimate_bytes(n);
  } else {
    if (n < 0 || n >= (1ll << 31) - 1) fail(WCC_ERR_INVALID, "n must be in [0, 2^31-1)");
    if (m < 0 || 2 * m >= (1ll << 32)) fail(WCC_ERR_INVALID, "m must be in [0, 2^31)");
    if (m > 0 && (!src || !dst)) fail(WCC_ERR_INVALID, "src/dst is NULL");
    R->m = m;
    R->est_bytes = estimate_bytes(n) + graph_bytes(n, m);
    R->build_bytes = build_bytes(n, m);
  }
  if (!labels && n > 0) fail(WCC_ERR_INVALID, "clustering_in is NULL");
  R->n = n;
  R->rule = checked_rule(rule);
  R->min_size = min_size < 2 ? 2 : min_size;
  R->ring_need = n / 2 + 2;
  if ((int64_t)(R->est_bytes + R->build_bytes) > S->budget)
    fail(WCC_ERR_BUSY, "a graph of " + std::to_string(n) + " vertices and " + std::to_string(m) +
                           " edges needs about " + std::to_string(R->est_bytes + R->build_bytes) +
                           " bytes, more than the server's budget");
  if ((uint64_t)R->ring_need + (uint64_t)S->grid + 1024 > S->ring_cap)
    fail(WCC_ERR_BUSY, "the graph is too large for the server's queue");
  R->t_submit = clock_t_::now();
  if (R->n > 0) {
    R->h_in.assign(labels, labels + R->n);
    R->h_out.resize((size_t)R->n);
  }
  if (!g) {
    R->h_src = src;
    R->h_dst = dst;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  const uint64_t t = S->next_ticket++;
  R->ticket = t;
  Request *raw = R.release();
  S->tickets[t] = raw;
  if (raw->n == 0) {
    raw->status = WCC_OK;
  } else {
    S->waiting.push_back(raw);
    S->cv_work.notify_all();
  }
  return t;
}

// Hands a finished request's result out and forgets it; WCC_PENDING if it
// is not finished.
int collect(Server *S, std::unique_lock<std::mutex> &lk, uint64_t ticket, int32_t *out,
            wcc_stats *stats) {
  auto it = S->tickets.find(ticket);
  if (it == S->tickets.end()) fail(WCC_ERR_INVALID, "unknown ticket " + std::to_string(ticket));
  Request *R = it->second;
  if (R->status == WCC_PENDING) return WCC_PENDING;
  S->tickets.erase(it);
  lk.unlock();
  std::unique_ptr<Request> own(R);
  if (R->status != WCC_OK) fail(R->status, R->error);
  if (R->n > 0) {
    if (!out) fail(WCC_ERR_INVALID, "clustering_out is NULL");
    std::memcpy(out, R->h_out.data(), 4 * R->n);
  }
  if (stats) *stats = R->stats;
  return WCC_OK;
}

}  // namespace

}  // namespace wccg

struct wcc_server {
  wccg::Server *s;
};

using namespace wccg;

namespace {
template <typename F>
int guarded_s(F &&f) {
  try {
    return f();
  } catch (const Error &e) {
    set_last_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return WCC_ERR_OOM;
  } catch (const std::exception &e) {
    set_last_error(e.what());
    return WCC_ERR_INTERNAL;
  }
}
}  // namespace

extern "C" {

int wcc_server_create(int64_t mem_budget_bytes, wcc_server **out) {
  return guarded_s([&] {
    if (!out) fail(WCC_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (mem_budget_bytes <= 0) fail(WCC_ERR_INVALID, "mem_budget_bytes must be > 0");
    Server *S = create_server(mem_budget_bytes);
    *out = new wcc_server{S};
    set_last_error("");
    return (int)WCC_OK;
  });
}

int wcc_submit(wcc_server *s, const wcc_graph *g, const int32_t *clustering_in,
               const wcc_threshold_rule *rule, int32_t min_size, uint64_t *ticket) {
  return guarded_s([&] {
    if (!s || !ticket) fail(WCC_ERR_INVALID, "NULL argument");
    if (!g) fail(WCC_ERR_INVALID, "graph is NULL");
    *ticket = submit(s->s, g->g, nullptr, nullptr, 0, 0, clustering_in, rule, min_size);
    set_last_error("");
    return (int)WCC_OK;
  });
}

int wcc_submit_edges(wcc_server *s, const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                     const int32_t *clustering_in, const wcc_threshold_rule *rule,
                     int32_t min_size, uint64_t *ticket) {
  return guarded_s([&] {
    if (!s || !ticket) fail(WCC_ERR_INVALID, "NULL argument");
    *ticket = submit(s->s, nullptr, src, dst, m, n, clustering_in, rule, min_size);
    set_last_error("");
    return (int)WCC_OK;
  });
}

int wcc_server_info(wcc_server *s, wcc_server_counters *out) {
  return guarded_s([&] {
    if (!s || !out) fail(WCC_ERR_INVALID, "NULL argument");
    Server *S = s->s;
    std::lock_guard<std::mutex> lk(S->mu);
    out->budget_bytes = S->budget;
    out->used_bytes = S->used;
    out->peak_used_bytes = S->peak_used;
    out->admitted = S->admitted;
    out->budget_waits = S->budget_waits;
    out->slot_waits = S->slot_waits;
    out->peak_active = S->peak_active;
    out->max_active = MAX_SLOTS;
    return (int)WCC_OK;
  });
}

int wcc_poll(wcc_server *s, uint64_t ticket, int32_t *clustering_out, wcc_stats *stats) {
  return guarded_s([&] {
    if (!s) fail(WCC_ERR_INVALID, "server is NULL");
    std::unique_lock<std::mutex> lk(s->s->mu);
    int r = collect(s->s, lk, ticket, clustering_out, stats);
    if (r == WCC_OK) set_last_error("");
    return r;
  });
}

int wcc_wait(wcc_server *s, uint64_t ticket, int64_t timeout_ms, int32_t *clustering_out,
             wcc_stats *stats) {
  return guarded_s([&] {
    if (!s) fail(WCC_ERR_INVALID, "server is NULL");
    Server *S = s->s;
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = clock_t_::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    for (;;) {
      auto it = S->tickets.find(ticket);
      if (it == S->tickets.end()) fail(WCC_ERR_INVALID, "unknown ticket " + std::to_string(ticket));
      if (it->second->status != WCC_PENDING) break;
      if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
        auto it2 = S->tickets.find(ticket);
        if (it2 != S->tickets.end() && it2->second->status == WCC_PENDING) return (int)WCC_PENDING;
      }
    }
    int r = collect(S, lk, ticket, clustering_out, stats);
    if (r == WCC_OK) set_last_error("");
    return r;
  });
}

void wcc_server_destroy(wcc_server *s) {
  if (!s) return;
  destroy_server(s->s);
  delete s;
}

}  // extern "C"
