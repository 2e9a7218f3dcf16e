// api.cu -- the C ABI (include/wcc.h): graph handles, the refinement run
// (membership grouping, queue seeding, the refinement kernel, output
// numbering) and error reporting.
#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <memory>
#include <unordered_map>

#include <mutex>

#include "internal.h"

namespace wccg {

static thread_local std::string g_last_error;

void fail(int code, const std::string &msg) { throw Error{code, msg}; }

void set_last_error(const std::string &msg) { g_last_error = msg; }

static std::atomic<int64_t> g_launches{0};
void note_launch(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// Device allocations (cudaMalloc calls that succeeded) made by the library.
static std::atomic<int64_t> g_allocs{0};

// Process-wide cache of device blocks, per device and power-of-two size
// class.  Every API call ends with a stream synchronisation, so a block that
// a finished call released can be handed to the next call at once; a graph
// created and destroyed per request then costs no cudaMalloc / cudaFree (and
// no device-wide synchronisation of cudaFree) after the first one.  When an
// allocation fails, the cached blocks of that device are returned to the
// driver and the allocation retried once.
namespace {
struct BlockCache {
  std::mutex mu;
  std::unordered_map<uint64_t, std::vector<void *>> free_blocks;  // (device << 8 | class)
};
BlockCache &block_cache() {
  static BlockCache *c = new BlockCache();  // never destroyed: blocks live until exit
  return *c;
}
int size_class(size_t b) {
  int k = 8;  // 256 bytes
  while (((size_t)1 << k) < b) ++k;
  return k;
}
void trim_cache(int dev) {
  BlockCache &c = block_cache();
  std::lock_guard<std::mutex> lk(c.mu);
  for (auto &kv : c.free_blocks) {
    if ((int)(kv.first >> 8) != dev) continue;
    for (void *q : kv.second) cudaFree(q);
    kv.second.clear();
  }
}
}  // namespace

DevBuf::~DevBuf() { release(); }

void DevBuf::release() {
  if (p) {
    BlockCache &c = block_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    c.free_blocks[((uint64_t)dev << 8) | (uint64_t)size_class(bytes)].push_back(p);
  }
  p = nullptr;
  bytes = 0;
  dev = -1;
}

void *DevBuf::ensure(size_t b) {
  if (b <= bytes && p) return p;
  release();
  const int k = size_class(b);
  const size_t want = (size_t)1 << k;
  WCC_CUDA(cudaGetDevice(&dev));
  {
    BlockCache &c = block_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.free_blocks.find(((uint64_t)dev << 8) | (uint64_t)k);
    if (it != c.free_blocks.end() && !it->second.empty()) {
      p = it->second.back();
      it->second.pop_back();
      bytes = want;
      return p;
    }
  }
  cudaError_t e = cudaMalloc(&p, want);
  if (e == cudaErrorMemoryAllocation) {
    (void)cudaGetLastError();
    trim_cache(dev);
    e = cudaMalloc(&p, want);
  }
  if (e != cudaSuccess) {
    p = nullptr;
    (void)cudaGetLastError();
    fail(e == cudaErrorMemoryAllocation ? WCC_ERR_OOM : WCC_ERR_CUDA,
         "device allocation of " + std::to_string(want) + " bytes failed: " +
             cudaGetErrorString(e));
  }
  g_allocs.fetch_add(1, std::memory_order_relaxed);
  bytes = want;
  return p;
}

int current_device() {
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) {
    (void)cudaGetLastError();
    fail(WCC_ERR_CUDA, std::string("no usable CUDA device: ") +
                           (e != cudaSuccess ? cudaGetErrorString(e) : "device count is 0"));
  }
  int dev = 0;
  WCC_CUDA(cudaGetDevice(&dev));
  return dev;
}

// Limit of every device-side queue wait (WCC_WAIT_LIMIT_MS, default 30 s):
// a CTA that waits longer sets DERR_TIMEOUT and leaves, so a fault in the
// queue protocol ends the kernel instead of hanging the GPU.
uint64_t wait_limit_ns() {
  const char *e = getenv("WCC_WAIT_LIMIT_MS");
  long long ms = e ? atoll(e) : 30000;
  if (ms < 1) ms = 1;
  return (uint64_t)ms * 1000000ull;
}

// Items of at least this many vertices first try the forest acceptance test
// (WCC_FOREST_MIN_N; 0, the default, turns it off: on the measured workloads
// the maximum-adjacency pass decides faster).
// The process-wide tuning (wcc_set_tuning / wcc_autotune / wcc_load_tuning);
// an environment variable, when set, overrides its field.
static std::mutex g_tune_mu;
static wcc_tuning g_tune = {64, 4096, 128, 0, 0, {0, 0, 0}};

wcc_tuning current_tuning() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tune;
}
void store_tuning(const wcc_tuning &t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune = t;
}
bool tuning_valid(const wcc_tuning &t) {
  return t.tiny_max >= 0 && t.tiny_max <= 64 && t.tiny_max_deg >= 0 && t.dense_max >= 0 &&
         t.dense_max <= 128 && t.forest_min_n >= 0 && t.smem_kb >= 0 && t.reserved[0] == 0 &&
         t.reserved[1] == 0 && t.reserved[2] == 0;
}
static long long env_or(const char *name, long long fallback) {
  const char *e = getenv(name);
  return e ? atoll(e) : fallback;
}

int forest_min_n_config() {
  long long v = env_or("WCC_FOREST_MIN_N", current_tuning().forest_min_n);
  if (v < 0) v = 0;
  if (v > (1ll << 30)) v = 1ll << 30;
  return (int)v;
}

// Most super-vertices left after the first contraction pass that the dense
// finish takes (WCC_DENSE_NSV, at most 128; 0 keeps every item on the sparse
// passes).
int dense_max_config() {
  const long long v = env_or("WCC_DENSE_NSV", current_tuning().dense_max);
  return (int)(v < 0 ? 0 : v > 128 ? 128 : v);
}

// Items of at most this many vertices (WCC_TINY_N, at most 64; 0 keeps every
// item on a whole CTA) are refined one per warp, up to 8 at once per CTA.
int tiny_max_config() {
  const long long v = env_or("WCC_TINY_N", current_tuning().tiny_max);
  return (int)(v < 0 ? 0 : v > 64 ? 64 : v);
}

// ... unless their members' degree sum exceeds WCC_TINY_DEG (a hub's row would
// keep one warp busy while its CTA waits).
int tiny_max_deg_config() {
  const long long v = env_or("WCC_TINY_DEG", current_tuning().tiny_max_deg);
  return (int)(v < 0 ? 0 : v > (1ll << 30) ? (1ll << 30) : v);
}

// CSR builder of wcc_create_graph_from_edges (WCC_CSR_BUILDER): "rows" sorts
// every row on chip (and sorts all entries at once when a row is too long
// for that); "radix" always sorts all entries at once; "auto" (the default)
// takes the rows for edge lists of up to CSR_ROWS_AUTO_MAX_EDGES edges.  Both
// give the same CSR.
constexpr int64_t CSR_ROWS_AUTO_MAX_EDGES = 1ll << 24;
bool csr_rows_config(int64_t m) {
  const char *e = getenv("WCC_CSR_BUILDER");
  if (e && strcmp(e, "rows") == 0) return true;
  if (e && strcmp(e, "radix") == 0) return false;
  return m <= CSR_ROWS_AUTO_MAX_EDGES;
}

// Dynamic shared memory per refinement CTA (WCC_SMEM_KB, default: the
// largest a CTA can opt into, one CTA per SM).  Items whose working set is
// larger use a global slab.
size_t refine_smem_bytes_config(int device) {
  const int tk = current_tuning().smem_kb;
  long long kb = env_or("WCC_SMEM_KB", tk > 0 ? tk : (1ll << 30));
  long long mx = (long long)(refine_smem_max_bytes(device) / 1024);
  if (kb < 16) kb = 16;
  if (kb > mx) kb = mx;
  return (size_t)kb * 1024;
}

// Validates a threshold rule and min_size; returns the rule to use.
wcc_threshold_rule checked_rule(const wcc_threshold_rule *rule) {
  wcc_threshold_rule r = rule ? *rule : wcc_threshold_rule{WCC_RULE_LOG10, 0, 0, 1};
  if (r.kind < WCC_RULE_LOG10 || r.kind > WCC_RULE_LINEAR)
    fail(WCC_ERR_INVALID, "unknown threshold rule kind " + std::to_string(r.kind));
  if (r.kind == WCC_RULE_LINEAR &&
      (r.den <= 0 || r.num < 0 || r.den >= (1ll << 31) || r.num >= (1ll << 31)))
    fail(WCC_ERR_INVALID, "LINEAR rule needs 0 <= num < 2^31 and 0 < den < 2^31");
  return r;
}

namespace {

constexpr int TB = 256;

inline unsigned blocks_for(int64_t n, int per = TB) { return grid_for(n, per); }

// ---------------------------------------------------------------- CSR checks
// Warp per vertex: offsets in range and non-decreasing, ids in [0, n), no
// self-loop, rows strictly ascending, and symmetry (v found in row u by
// binary search).
__global__ void k_validate_csr(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                               int64_t n, int64_t nnz, unsigned *err) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const int64_t v = w;
  const int64_t b = off[v], e = off[v + 1];
  if (b < 0 || e < b || e > nnz) {
    if (lane == 0) atomicOr(err, DERR_INVALID);
    return;
  }
  for (int64_t q = b + lane; q < e; q += 32) {
    int32_t u = adj[q];
    bool bad = u < 0 || u >= n || u == v || (q > b && adj[q - 1] >= u);
    if (!bad) {
      int64_t lo = off[u], hi = off[u + 1];
      if (lo < 0 || hi < lo || hi > nnz) {
        bad = true;
      } else {
        while (lo < hi) {
          int64_t mid = (lo + hi) >> 1;
          if (adj[mid] < v) lo = mid + 1; else hi = mid;
        }
        bad = !(lo < off[u + 1] && adj[lo] == v);
      }
    }
    if (bad) atomicOr(err, DERR_INVALID);
  }
}

// ---------------------------------------------------------------- CSR build
__global__ void k_edge_keys(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                            int64_t m, int64_t n, int b, uint64_t *keys, unsigned *err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  int32_t u = src[i], v = dst[i];
  if (u < 0 || u >= n || v < 0 || v >= n) {
    atomicOr(err, DERR_INVALID);
    keys[2 * i] = keys[2 * i + 1] = ~0ull;
    return;
  }
  if (u == v) {
    keys[2 * i] = keys[2 * i + 1] = ~0ull;
    return;
  }
  keys[2 * i] = ((uint64_t)u << b) | (uint64_t)v;
  keys[2 * i + 1] = ((uint64_t)v << b) | (uint64_t)u;
}

// keep[i] = 1 for the first copy of each valid key (sorted input)
__global__ void k_unique_flags(const uint64_t *__restrict__ keys, int64_t n2, uint32_t *keep,
                               uint64_t invalid) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n2) return;
  uint64_t k = keys[i];
  keep[i] = (k != invalid && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
}

// The kept entries in order, and the degree of every row.  Keys are sorted,
// so a warp's entries mostly share a row: one atomic per row and warp.
__global__ void k_compact_edges(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ keep,
                                const uint32_t *__restrict__ pos, int64_t n2, int b,
                                int32_t *cols, int64_t *deg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool kept = i < n2 && keep[i];
  const uint64_t k = kept ? keys[i] : 0ull;
  const unsigned long long u = kept ? (unsigned long long)(k >> b) : ~0ull;
  if (kept) cols[pos[i]] = (int32_t)(k & ((1ull << b) - 1));
  const unsigned peers = __match_any_sync(FULL, u);
  if (kept && (peers & lanemask_lt()) == 0)
    atomicAdd((unsigned long long *)&deg[u], (unsigned long long)__popc(peers));
}

// ---------------------------------------------------------------- helpers
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) WCC_CUDA(cudaSetDevice(dev));
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};


void check_derr(unsigned err, const char *what) { check_device_error(err, what); }




// Writes the per-item profile of the last refinement as CSV (appending).
void dump_item_profile(const RefineParams &p, const char *path, int ctas, cudaStream_t s) {
  unsigned cnt = read_back(p.prof_count, s);
  if (cnt > p.prof_cap) cnt = p.prof_cap;
  std::vector<ItemProf> h(cnt);
  if (cnt) {
    WCC_CUDA(cudaMemcpyAsync(h.data(), p.prof, sizeof(ItemProf) * cnt, cudaMemcpyDeviceToHost, s));
    WCC_CUDA(cudaStreamSynchronize(s));
  }
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "seq,n,E,nalive,passes,nsv,outcome,smid,slab,top,load,extract,ccr,peel,cc,contract,"
             "sw,out,t_begin,t_end,p1_cycles,p1_marks,p1_steps,later_passes,forest,nsv1,forest_cycles,f_bfs,f_levels,f_check,"
             "f_trees,f_contract,f_relabel\n");
  for (const ItemProf &q : h)
    fprintf(f, "%u,%d,%d,%d,%d,%d,%d,%d,%d,%d,%u,%u,%u,%u,%u,%u,%u,%u,%lld,%lld,%lld,%lld,%lld,%lld,%d,%d,"
               "%lld,%lld,%lld,%lld,%lld,%lld,%lld\n",
            q.seq, q.n, q.E, q.nalive, q.passes, q.nsv, q.outcome, q.smid, q.slab, q.top,
            q.dt[0], q.dt[1], q.dt[2], q.dt[3], q.dt[4], q.dt[5], q.dt[6], q.dt[7], q.t_begin, q.t_end,
            q.dbg[0], q.dbg[1], q.dbg[2], q.dbg[3], q.forest, q.nsv1, q.forest_cycles, q.fdbg[0],
            q.fdbg[1], q.fdbg[2], q.fdbg[3], q.fdbg[4], q.fdbg[5]);
  fclose(f);
  if (ctas <= 0 || p.prof_cta == nullptr) return;
  std::vector<CtaProf> c((size_t)ctas);
  WCC_CUDA(cudaMemcpyAsync(c.data(), p.prof_cta, sizeof(CtaProf) * (size_t)ctas,
                           cudaMemcpyDeviceToHost, s));
  WCC_CUDA(cudaStreamSynchronize(s));
  f = fopen((std::string(path) + ".cta").c_str(), "a");
  if (!f) return;
  fprintf(f, "cta,claim,tiny,cta_time,batches,tiny_items,cta_items\n");
  for (int i = 0; i < ctas; ++i)
    fprintf(f, "%d,%lld,%lld,%lld,%d,%d,%d\n", i, c[i].claim, c[i].tiny, c[i].cta, c[i].batches,
            c[i].tiny_items, c[i].cta_items);
  fclose(f);
}



struct Timer {
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  bool on;
  explicit Timer(bool enable) : on(enable) {
    if (on)
      for (auto &e : ev) WCC_CUDA(cudaEventCreate(&e));
  }
  ~Timer() {
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
  }
  void mark(int i, cudaStream_t s) {
    if (on) WCC_CUDA(cudaEventRecord(ev[i], s));
  }
  double ms(int a, int b) {
    if (!on) return 0;
    float f = 0;
    WCC_CUDA(cudaEventElapsedTime(&f, ev[a], ev[b]));
    return f;
  }
};


enum RunBuf { R_IN, R_OUT, R_POOL, R_SLOT, R_LMIN, R_RING, R_CTR, R_SLAB, R_REQ, R_INH,
              R_CM_PARTS, R_CM_PARTOF, R_CM_SCRATCH, R_CM_ITEMS, R_CM_MISC, R_COUNT };
static_assert(R_COUNT <= 16, "Graph::rb holds 16 buffers");

// CM (Section 2.4, Algorithms 4-5): the resolution of its CPM community step.
struct CmOpts {
  int64_t gnum, gden;
};
static_assert(R_COUNT <= 16, "run buffers");

void run_impl(Graph *g, const int32_t *lab_in, const wcc_threshold_rule *rule, int32_t min_size,
              int32_t mode, int32_t *lab_out, int on_device, cudaStream_t s, wcc_stats *stats,
              const CmOpts *cm = nullptr) {
  auto t_start = std::chrono::steady_clock::now();
  const int64_t n = g->n;
  const wcc_threshold_rule r = checked_rule(rule);
  if (mode != WCC_MODE_BATCHED && mode != WCC_MODE_PLAIN)
    fail(WCC_ERR_INVALID, "unknown mode " + std::to_string(mode));
  if (min_size < 2) min_size = 2;
  if (lab_in == nullptr || lab_out == nullptr)
    fail(WCC_ERR_INVALID, "clustering_in and clustering_out must not be NULL");
  if (lab_in == lab_out) fail(WCC_ERR_INVALID, "clustering_out may not alias clustering_in");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n == 0) return;
  Timer tm(stats != nullptr);
  DevBuf *rb = g->rb;

  // input labels on the device
  const int32_t *d_in = lab_in;
  if (!on_device) {
    int32_t *p = static_cast<int32_t *>(rb[R_IN].ensure(4 * n));
    WCC_CUDA(cudaMemcpyAsync(p, lab_in, 4 * n, cudaMemcpyHostToDevice, s));
    d_in = p;
  }
  tm.mark(0, s);

  // ---- a2: group vertices by input label
  const GroupInfo gi = group_by_label(g->off.as<int64_t>(), n, d_in, min_size, g->ws, s);

  // ---- queue, pool, slots, the one-entry request table
  const int dev = g->device;
  const size_t smem_bytes = refine_smem_bytes_config(dev);
  const int grid = refine_max_ctas(dev, smem_bytes);
  const uint64_t cap = (uint64_t)n + 2ull * grid + 1024;
  int32_t *pool = static_cast<int32_t *>(rb[R_POOL].ensure(4 * std::max<int64_t>(n - gi.skip, 1)));
  auto *slot = static_cast<unsigned long long *>(rb[R_SLOT].ensure(8 * n));
  auto *lmin = static_cast<int32_t *>(rb[R_LMIN].ensure(4 * n));
  auto *inh = static_cast<unsigned long long *>(rb[R_INH].ensure(8 * n));
  auto *ring = static_cast<QSlot *>(rb[R_RING].ensure(sizeof(QSlot) * cap));
  auto *ctr = static_cast<RunCounters *>(rb[R_CTR].ensure(sizeof(RunCounters)));
  auto *req = static_cast<ReqCtx *>(rb[R_REQ].ensure(sizeof(ReqCtx)));
  WCC_CUDA(cudaMemsetAsync(slot, 0xff, 8 * n, s));
  WCC_CUDA(cudaMemsetAsync(lmin, 0xff, 4 * n, s));
  WCC_CUDA(cudaMemsetAsync(ctr, 0, sizeof(RunCounters), s));
  ReqCtx hreq{};
  hreq.off = g->off.as<int64_t>();
  hreq.adj = g->adj.as<int32_t>();
  hreq.n_vertices = n;
  hreq.pool = pool;
  hreq.slot = slot;
  hreq.label_min = lmin;
  hreq.inh = inh;
  hreq.rule_kind = r.kind;
  hreq.min_size = min_size;
  hreq.rule_num = r.num;
  hreq.rule_den = r.den;
  WCC_CUDA(cudaMemcpyAsync(req, &hreq, sizeof(hreq), cudaMemcpyHostToDevice, s));
  if (gi.kept > 0) {
    WCC_CUDA(cudaMemsetAsync(ring, 0xff, sizeof(QSlot) * cap, s));
    seed_items(gi, n, g->ws, 0, req, pool, slot, ring, cap, ctr, s);
  }
  tm.mark(1, s);

  // ---- refinement
  if (gi.kept > 0) {
    size_t need = item_workspace_bytes(gi.max_n, gi.max_dsum);
    size_t slab_bytes = need > smem_bytes ? ((need + 255) & ~(size_t)255) : 256;
    RefineParams p{};
    p.reqs = req;
    p.ring = ring;
    p.ring_cap = cap;
    p.ctr = ctr;
    p.wait_limit_ns = wait_limit_ns();
    p.idle_limit_ns = 0;
    p.smem_bytes = smem_bytes;
    p.slab_bytes = slab_bytes;
    p.forest_min_n = forest_min_n_config();
    p.dense_max = dense_max_config();
    // with no more input clusters than CTAs, every item gets a whole CTA:
    // one warp per small item only pays off when items outnumber the CTAs
    // (a 50-vertex item's subtree takes about 2.5 times longer on one warp);
    // WCC_TINY_N, when set, decides regardless
    p.tiny_max = (gi.kept <= (int64_t)grid && getenv("WCC_TINY_N") == nullptr) ? 0
                                                                              : tiny_max_config();
    p.tiny_max_deg = tiny_max_deg_config();
    // optional per-item profile (WCC_PROFILE_ITEMS=<csv path>)
    const char *prof_path = getenv("WCC_PROFILE_ITEMS");
    DevBuf prof_buf;
    const unsigned prof_cap = 1u << 20;
    DevBuf prof_cta_buf;
    if (prof_path && *prof_path) {
      char *pb = static_cast<char *>(prof_buf.ensure(sizeof(ItemProf) * prof_cap + 64));
      p.prof = reinterpret_cast<ItemProf *>(pb + 64);
      p.prof_count = reinterpret_cast<unsigned *>(pb);
      p.prof_cap = prof_cap;
      WCC_CUDA(cudaMemsetAsync(pb, 0, 64, s));
      p.prof_cta = static_cast<CtaProf *>(prof_cta_buf.ensure(sizeof(CtaProf) * (size_t)grid));
      WCC_CUDA(cudaMemsetAsync(p.prof_cta, 0, sizeof(CtaProf) * (size_t)grid, s));
    }
    if (mode == WCC_MODE_BATCHED && cm) {
      // CM: the sides of every cut split are parked; after each run the
      // community step publishes their communities and the kernel runs again
      p.slab = static_cast<char *>(rb[R_SLAB].ensure(slab_bytes * (size_t)grid));
      p.single_item = 0;
      p.tickets = 1;
      p.tiny_max = 0;  // every item on a whole CTA, where the split is parked
      p.cm = 1;
      p.cda_cap = (unsigned long long)n + 1024;
      p.cda = static_cast<Item *>(rb[R_CM_PARTS].ensure(sizeof(Item) * p.cda_cap + 64));
      p.cda_count = reinterpret_cast<unsigned long long *>(
          static_cast<char *>(rb[R_CM_PARTS].p) + sizeof(Item) * p.cda_cap);
      int32_t *partof = static_cast<int32_t *>(rb[R_CM_PARTOF].ensure(8 * (size_t)n));
      WCC_CUDA(cudaMemsetAsync(partof, 0xff, 8 * (size_t)n, s));
      for (;;) {
        WCC_CUDA(cudaMemsetAsync(p.cda_count, 0, sizeof(unsigned long long), s));
        launch_refine(p, grid, true, s);
        const RunCounters c = read_back(ctr, s);
        if (c.error) break;  // reported below
        const unsigned long long parked = read_back(p.cda_count, s);
        if (parked == 0) break;
        const unsigned long long added =
            cm_round(p.cda, parked, req, cm->gnum, cm->gden, partof, partof + n, n, gi.max_n,
                     gi.max_dsum, ctr, ring, cap, grid, rb[R_CM_SCRATCH], rb[R_CM_ITEMS],
                     rb[R_CM_MISC], s);
        if (added == 0) break;
      }
    } else if (mode == WCC_MODE_BATCHED) {
      p.slab = static_cast<char *>(rb[R_SLAB].ensure(slab_bytes * (size_t)grid));
      p.single_item = 0;
      p.tickets = 1;  // nothing is added while the run lasts
      launch_refine(p, grid, true, s);
    } else {
      p.slab = static_cast<char *>(rb[R_SLAB].ensure(slab_bytes));
      p.single_item = 1;
      unsigned long long tail = (unsigned long long)gi.kept;
      for (unsigned long long j = 0; j < tail; ++j) {
        p.single_index = j;
        launch_refine(p, 1, false, s);
        if (j + 1 == tail) {
          RunCounters c = read_back(ctr, s);
          if (c.error) break;
          tail = c.tail;
        }
      }
    }
    if (p.prof) dump_item_profile(p, prof_path, mode == WCC_MODE_BATCHED ? grid : 0, s);
  }
  tm.mark(2, s);
  // ---- a9: ids = rank of each accepted cluster's smallest vertex, numbered
  // into the staging buffer right behind the kernel; the run's counters are
  // read after it (one wait for both), and the result reaches clustering_out
  // only once they show no error
  int32_t *d_out = static_cast<int32_t *>(rb[R_OUT].ensure(4 * n));
  number_clusters(lmin, n, d_out, g->ws, s);
  tm.mark(3, s);
  RunCounters hc{};
  ReqCtx hr{};
  if (gi.kept > 0) {
    WCC_CUDA(cudaMemcpyAsync(&hc, ctr, sizeof(hc), cudaMemcpyDeviceToHost, s));
    WCC_CUDA(cudaMemcpyAsync(&hr, req, sizeof(hr), cudaMemcpyDeviceToHost, s));
    WCC_CUDA(cudaStreamSynchronize(s));
    check_derr(hc.error, "refinement");
  }
  WCC_CUDA(cudaMemcpyAsync(lab_out, d_out, 4 * n,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  WCC_CUDA(cudaStreamSynchronize(s));

  if (stats) {
    stats->in_clusters = gi.clusters;
    stats->out_clusters = hr.accepted;
    stats->items = hr.items;
    stats->splits = hr.splits;
    stats->peeled = hr.peeled;
    stats->ni_passes = hr.ni_passes;
    stats->sw_phases = hr.sw_phases;
    stats->max_item = gi.max_n;
    stats->alg_bytes = hr.alg_bytes;
    stats->ms_membership = tm.ms(0, 1);
    stats->ms_refine = tm.ms(1, 2);
    stats->ms_output = tm.ms(2, 3);
    stats->ms_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start)
            .count();
  }
}

Graph *create_from_csr(const int64_t *off, const int32_t *adj, int64_t n, int64_t nnz,
                       int on_device, cudaStream_t s) {
  if (n < 0 || n >= (1ll << 31) - 1) fail(WCC_ERR_INVALID, "n must be in [0, 2^31-1)");
  if (nnz < 0) fail(WCC_ERR_INVALID, "nnz must be >= 0");
  if (n > 0 && off == nullptr) fail(WCC_ERR_INVALID, "row_off is NULL");
  if (nnz > 0 && adj == nullptr) fail(WCC_ERR_INVALID, "cols is NULL");
  std::unique_ptr<Graph> g(new Graph());
  g->device = current_device();
  g->n = n;
  g->nnz = nnz;
  int64_t *d_off = static_cast<int64_t *>(g->off.ensure(8 * (n + 1)));
  int32_t *d_adj = static_cast<int32_t *>(g->adj.ensure(4 * std::max<int64_t>(nnz, 1)));
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (n > 0) {
    WCC_CUDA(cudaMemcpyAsync(d_off, off, 8 * (n + 1), kind, s));
  } else {
    WCC_CUDA(cudaMemsetAsync(d_off, 0, 8, s));
  }
  if (nnz > 0) WCC_CUDA(cudaMemcpyAsync(d_adj, adj, 4 * nnz, kind, s));
  // first and last offsets
  int64_t ends[2] = {0, 0};
  WCC_CUDA(cudaMemcpyAsync(&ends[0], d_off, 8, cudaMemcpyDeviceToHost, s));
  WCC_CUDA(cudaMemcpyAsync(&ends[1], d_off + n, 8, cudaMemcpyDeviceToHost, s));
  WCC_CUDA(cudaStreamSynchronize(s));
  if (ends[0] != 0 || ends[1] != nnz) fail(WCC_ERR_INVALID, "row_off[0] != 0 or row_off[n] != nnz");
  if (n > 0) {
    DevBuf e;
    unsigned *d_err = static_cast<unsigned *>(e.ensure(4));
    WCC_CUDA(cudaMemsetAsync(d_err, 0, 4, s));
    k_validate_csr<<<blocks_for(n * 32), TB, 0, s>>>(d_off, d_adj, n, nnz, d_err); note_launch();
    WCC_CUDA(cudaGetLastError());
    unsigned err = read_back(d_err, s);
    if (err) fail(WCC_ERR_INVALID, "CSR is not a simple symmetric graph with sorted rows");
  }
  return g.release();
}

Graph *build_from_edges(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                        int on_device, cudaStream_t s) {
  if (n < 0 || n >= (1ll << 31) - 1) fail(WCC_ERR_INVALID, "n must be in [0, 2^31-1)");
  if (m < 0 || 2 * m >= (1ll << 32)) fail(WCC_ERR_INVALID, "m must be in [0, 2^31)");
  if (m > 0 && (src == nullptr || dst == nullptr)) fail(WCC_ERR_INVALID, "src/dst is NULL");
  std::unique_ptr<Graph> g(new Graph());
  g->device = current_device();
  g->n = n;
  DevBuf bsrc, bdst, bk, bk2, btemp, bkeep, bpos;
  const int32_t *d_src = src, *d_dst = dst;
  if (!on_device && m > 0) {
    int32_t *a = static_cast<int32_t *>(bsrc.ensure(4 * m));
    int32_t *b = static_cast<int32_t *>(bdst.ensure(4 * m));
    WCC_CUDA(cudaMemcpyAsync(a, src, 4 * m, cudaMemcpyHostToDevice, s));
    WCC_CUDA(cudaMemcpyAsync(b, dst, 4 * m, cudaMemcpyHostToDevice, s));
    d_src = a;
    d_dst = b;
  }
  const int b = (int)std::max<int64_t>(1, bitlen_u64(n > 0 ? (uint64_t)(n - 1) : 0));
  const int64_t n2 = 2 * m;
  int64_t *d_off = static_cast<int64_t *>(g->off.ensure(8 * (n + 1)));
  WCC_CUDA(cudaMemsetAsync(d_off, 0, 8 * (n + 1), s));
  int64_t nnz = 0;
  if (m > 0 && csr_rows_config(m)) {
    DevBuf rbufs[CSR_ROW_BUFS];
    if (csr_by_rows(d_src, d_dst, m, n, d_off, g->adj, &nnz, rbufs, s)) {
      g->nnz = nnz;
      return g.release();
    }
    WCC_CUDA(cudaMemsetAsync(d_off, 0, 8 * (n + 1), s));  // the degree counts start at zero
  }
  if (m > 0) {
    // the columns get room for every directed entry, so nothing has to be
    // read back before the end: one read of {error, nnz} closes the build
    uint64_t *k1 = static_cast<uint64_t *>(bk.ensure(8 * n2));
    uint64_t *k2 = static_cast<uint64_t *>(bk2.ensure(8 * n2));
    void *temp = btemp.ensure(std::max(radix_temp_bytes(n2), scan_temp_bytes(n + 1)) + 64);
    uint32_t *keep = static_cast<uint32_t *>(bkeep.ensure(4 * (n2 + 2)));
    uint32_t *pos = static_cast<uint32_t *>(bpos.ensure(4 * (n2 + 1)));
    unsigned *d_err = keep + n2 + 1;
    WCC_CUDA(cudaMemsetAsync(d_err, 0, 4, s));
    k_edge_keys<<<blocks_for(m), TB, 0, s>>>(d_src, d_dst, m, n, b, k1, d_err); note_launch();
    WCC_CUDA(cudaGetLastError());
    uint64_t *sorted = k1;
    // valid keys are (u << b) | v < 2^(2b) - 1 (u != v); dropped self-loops
    // carry all ones, so sorting on the low 2b bits puts them last
    if (radix_sort_keys_u64(k1, k2, n2, 2 * b, temp, d_err, s)) sorted = k2;
    k_unique_flags<<<blocks_for(n2), TB, 0, s>>>(sorted, n2, keep, ~0ull); note_launch();
    exclusive_scan_u32(keep, pos, n2, pos + n2, temp, s);
    int32_t *d_adj = static_cast<int32_t *>(g->adj.ensure(4 * n2));
    k_compact_edges<<<blocks_for(n2), TB, 0, s>>>(sorted, keep, pos, n2, b, d_adj, d_off);
    note_launch();
    exclusive_scan_i64(d_off, d_off, n + 1, nullptr, temp, s);
    WCC_CUDA(cudaGetLastError());
    uint32_t tail[2] = {0, 0};
    WCC_CUDA(cudaMemcpyAsync(&tail[0], d_err, 4, cudaMemcpyDeviceToHost, s));
    WCC_CUDA(cudaMemcpyAsync(&tail[1], pos + n2, 4, cudaMemcpyDeviceToHost, s));
    WCC_CUDA(cudaStreamSynchronize(s));
    if (tail[0] & DERR_INVALID) fail(WCC_ERR_INVALID, "edge endpoint outside [0, n)");
    if (tail[0]) fail(WCC_ERR_TIMEOUT, "CSR build: a bounded wait of the sort ran out");
    nnz = tail[1];
  } else {
    g->adj.ensure(4);
  }
  WCC_CUDA(cudaStreamSynchronize(s));
  g->nnz = nnz;
  return g.release();
}

// ---------------------------------------------------------------- CSR build without allocation
// Scratch of wcc_build_csr_no_alloc: one array in the module's static device
// memory, so a caller that must not allocate device memory can still build a
// CSR.  Every GPU that loads this library holds it until the process exits.
// Layout (256-byte aligned pieces): two 64-bit key buffers and two 32-bit
// flag/position buffers of 2*NOALLOC_MAX_EDGES (+1) entries, the sort/scan
// temporaries, and a small result word.
constexpr int64_t NOALLOC_MAX_EDGES = 1 << 17;
constexpr int64_t NOALLOC_MAX_VERTICES = 1 << 22;
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)6656 * 1024;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch on the current device.  It is looked
// up on every call (a cheap driver query), so the address always belongs to
// the context the work runs in, also after a cudaDeviceReset.
void *noalloc_scratch() {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    (void)cudaGetLastError();
    fail(WCC_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch) failed: ") +
                           cudaGetErrorString(e));
  }
  return p;
}

void build_csr_no_alloc(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                        int64_t *row_off, int32_t *cols, int64_t *nnz_out, cudaStream_t s) {
  if (m < 0 || m > NOALLOC_MAX_EDGES)
    fail(WCC_ERR_INVALID, "wcc_build_csr_no_alloc: m must be in [0, " +
                              std::to_string(NOALLOC_MAX_EDGES) + "], got " + std::to_string(m));
  if (n < 0 || n > NOALLOC_MAX_VERTICES)
    fail(WCC_ERR_INVALID, "wcc_build_csr_no_alloc: n must be in [0, " +
                              std::to_string(NOALLOC_MAX_VERTICES) + "], got " +
                              std::to_string(n));
  if (row_off == nullptr || nnz_out == nullptr || (m > 0 && (src == nullptr || dst == nullptr || cols == nullptr)))
    fail(WCC_ERR_INVALID, "wcc_build_csr_no_alloc: NULL buffer");
  const int dev = current_device();
  if (s != nullptr) {
    // the scratch address is the current device's: the stream must be too
    int sdev = -1;
    WCC_CUDA(cudaStreamGetDevice(s, &sdev));
    if (sdev != dev)
      fail(WCC_ERR_INVALID, "wcc_build_csr_no_alloc: the stream belongs to device " +
                                std::to_string(sdev) + ", the current device is " +
                                std::to_string(dev));
  }
  char *base = static_cast<char *>(noalloc_scratch());
  const int64_t n2 = 2 * m;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t cap2 = (size_t)(2 * NOALLOC_MAX_EDGES);
  size_t o = 0;
  uint64_t *k1 = reinterpret_cast<uint64_t *>(base + o); o += al(8 * cap2);
  uint64_t *k2 = reinterpret_cast<uint64_t *>(base + o); o += al(8 * cap2);
  uint32_t *keep = reinterpret_cast<uint32_t *>(base + o); o += al(4 * (cap2 + 1));
  uint32_t *pos = reinterpret_cast<uint32_t *>(base + o); o += al(4 * (cap2 + 1));
  unsigned *err = reinterpret_cast<unsigned *>(base + o); o += al(16);
  void *temp = base + o;
  o += al(std::max(radix_temp_bytes((int64_t)cap2), scan_temp_bytes(NOALLOC_MAX_VERTICES + 1)));
  if (o > NOALLOC_SCRATCH_BYTES) fail(WCC_ERR_INTERNAL, "no-alloc scratch layout exceeds its array");
  // the degree counts accumulate in row_off, and the error word must start clear
  WCC_CUDA(cudaMemsetAsync(row_off, 0, 8 * (size_t)(n + 1), s));
  WCC_CUDA(cudaMemsetAsync(err, 0, 16, s));
  int64_t nnz = 0;
  if (m > 0) {
    const int b = (int)std::max<int64_t>(1, bitlen_u64(n > 0 ? (uint64_t)(n - 1) : 0));
    k_edge_keys<<<blocks_for(m), TB, 0, s>>>(src, dst, m, n, b, k1, err); note_launch();
    WCC_CUDA(cudaGetLastError());
    if (read_back(err, s)) fail(WCC_ERR_INVALID, "edge endpoint outside [0, n)");
    uint64_t *sorted = radix_sort_keys_u64(k1, k2, n2, 2 * b, temp, err, s) ? k2 : k1;
    k_unique_flags<<<blocks_for(n2), TB, 0, s>>>(sorted, n2, keep, ~0ull); note_launch();
    exclusive_scan_u32(keep, pos, n2, pos + n2, temp, s);
    k_compact_edges<<<blocks_for(n2), TB, 0, s>>>(sorted, keep, pos, n2, b, cols, row_off);
    note_launch();
    exclusive_scan_i64(row_off, row_off, n + 1, nullptr, temp, s);
    WCC_CUDA(cudaGetLastError());
    nnz = (int64_t)read_back(pos + n2, s);
    if (read_back(err, s)) fail(WCC_ERR_TIMEOUT, "wcc_build_csr_no_alloc: a bounded wait of the sort ran out");
  }
  WCC_CUDA(cudaStreamSynchronize(s));
  *nnz_out = nnz;
}

// ---- autotuner ---------------------------------------------------------------
// Coordinate search from the current tuning: each knob in turn tries its
// other candidate values with the rest fixed, and an improvement of more
// than 2% is kept.  Every candidate's result must equal the first (the knobs
// change only the schedule).  A run is timed as the best of two after one
// warm-up, through the host-buffer path.
void autotune_impl(Graph *g, const int32_t *lab_in, const wcc_threshold_rule *rule,
                   int32_t min_size, int on_device, cudaStream_t s, const char *cache_path,
                   wcc_tuning *best_out, double *best_ms) {
  const int64_t n = g->n;
  if (n > 0 && lab_in == nullptr) fail(WCC_ERR_INVALID, "clustering_in is NULL");
  std::vector<int32_t> lab((size_t)n), ref((size_t)n), out((size_t)n);
  if (n > 0) {
    WCC_CUDA(cudaMemcpyAsync(lab.data(), lab_in, 4 * (size_t)n,
                             on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
    WCC_CUDA(cudaStreamSynchronize(s));
  }
  const wcc_tuning start = current_tuning();
  auto measure = [&](const wcc_tuning &t, std::vector<int32_t> &o) {
    store_tuning(t);
    wcc_stats st{};
    run_impl(g, lab.data(), rule, min_size, WCC_MODE_BATCHED, o.data(), 0, s, &st);
    double best = 1e300;
    for (int r = 0; r < 2; ++r) {
      run_impl(g, lab.data(), rule, min_size, WCC_MODE_BATCHED, o.data(), 0, s, &st);
      best = std::min(best, st.ms_total);
    }
    return best;
  };
  wcc_tuning cur = start;
  double cur_ms = 0.0;
  try {
    cur_ms = measure(cur, ref);
    struct Knob {
      int32_t wcc_tuning::*field;
      std::vector<int32_t> values;
    };
    const Knob knobs[] = {{&wcc_tuning::tiny_max, {0, 32, 64}},
                          {&wcc_tuning::tiny_max_deg, {1024, 4096, 16384}},
                          {&wcc_tuning::dense_max, {32, 64, 128}},
                          {&wcc_tuning::smem_kb, {0, 160}},
                          {&wcc_tuning::forest_min_n, {0, 48}}};
    for (const Knob &k : knobs) {
      const int32_t base = cur.*k.field;
      for (int32_t v : k.values) {
        if (v == base) continue;
        wcc_tuning t = cur;
        t.*k.field = v;
        const double ms = measure(t, out);
        if (out != ref) fail(WCC_ERR_INTERNAL, "a candidate tuning changed the refined clustering");
        if (ms < 0.98 * cur_ms) {
          cur = t;
          cur_ms = ms;
        }
      }
    }
  } catch (...) {
    store_tuning(start);
    throw;
  }
  store_tuning(cur);
  if (cache_path) {
    cudaDeviceProp prop{};
    WCC_CUDA(cudaGetDeviceProperties(&prop, g->device));
    FILE *f = fopen(cache_path, "w");
    if (!f) fail(WCC_ERR_INVALID, std::string("cannot write ") + cache_path);
    fprintf(f,
            "{\"device\": \"%s\", \"sms\": %d, \"n\": %lld, \"nnz\": %lld, \"ms\": %.4f, "
            "\"tiny_max\": %d, \"tiny_max_deg\": %d, \"dense_max\": %d, \"forest_min_n\": %d, "
            "\"smem_kb\": %d}\n",
            prop.name, prop.multiProcessorCount, (long long)g->n, (long long)g->nnz, cur_ms,
            cur.tiny_max, cur.tiny_max_deg, cur.dense_max, cur.forest_min_n, cur.smem_kb);
    fclose(f);
  }
  if (best_out) *best_out = cur;
  if (best_ms) *best_ms = cur_ms;
}

// The value of "key" in the small JSON object written above.
bool json_int(const std::string &js, const char *key, long long *v) {
  const std::string k = std::string("\"") + key + "\":";
  const size_t p = js.find(k);
  if (p == std::string::npos) return false;
  char *end = nullptr;
  *v = strtoll(js.c_str() + p + k.size(), &end, 10);
  return end != js.c_str() + p + k.size();
}

void load_tuning_impl(const char *path, wcc_tuning *out) {
  if (!path) fail(WCC_ERR_INVALID, "cache_path is NULL");
  FILE *f = fopen(path, "r");
  if (!f) fail(WCC_ERR_INVALID, std::string("cannot read ") + path);
  std::string js;
  char buf[512];
  size_t r;
  while ((r = fread(buf, 1, sizeof(buf), f)) > 0 && js.size() < 65536) js.append(buf, r);
  fclose(f);
  wcc_tuning t{};
  long long v;
  int32_t wcc_tuning::*fields[] = {&wcc_tuning::tiny_max, &wcc_tuning::tiny_max_deg,
                                   &wcc_tuning::dense_max, &wcc_tuning::forest_min_n,
                                   &wcc_tuning::smem_kb};
  const char *names[] = {"tiny_max", "tiny_max_deg", "dense_max", "forest_min_n", "smem_kb"};
  for (int i = 0; i < 5; ++i) {
    if (!json_int(js, names[i], &v) || v < INT32_MIN || v > INT32_MAX)
      fail(WCC_ERR_INVALID, std::string(path) + ": missing or malformed \"" + names[i] + "\"");
    t.*fields[i] = (int32_t)v;
  }
  if (!tuning_valid(t)) fail(WCC_ERR_INVALID, std::string(path) + ": tuning out of range");
  // the device it was tuned on, when a GPU is there to compare with
  int count = 0;
  if (cudaGetDeviceCount(&count) == cudaSuccess && count > 0) {
    cudaDeviceProp prop{};
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
      const std::string want = std::string("\"device\": \"") + prop.name + "\"";
      if (js.find(want) == std::string::npos)
        fail(WCC_ERR_INVALID, std::string(path) + " was tuned on another device model");
    }
  } else {
    cudaGetLastError();  // no GPU: nothing to compare with
  }
  store_tuning(t);
  if (out) *out = t;
}

template <typename F>
int guarded(F &&f) {
  try {
    f();
    g_last_error.clear();
    return WCC_OK;
  } catch (const Error &e) {
    g_last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc &) {
    g_last_error = "host allocation failed";
    return WCC_ERR_OOM;
  } catch (const std::exception &e) {
    g_last_error = e.what();
    return WCC_ERR_INTERNAL;
  }
}

}  // namespace

Graph *create_from_edges(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                         int on_device, cudaStream_t s) {
  return build_from_edges(src, dst, m, n, on_device, s);
}

}  // namespace wccg


using namespace wccg;

extern "C" {

int wcc_create_graph(const int64_t *row_off, const int32_t *cols, int64_t n, int64_t nnz,
                     int on_device, void *stream, wcc_graph **out) {
  return guarded([&] {
    if (!out) fail(WCC_ERR_INVALID, "out is NULL");
    *out = nullptr;
    Graph *g = create_from_csr(row_off, cols, n, nnz, on_device, (cudaStream_t)stream);
    *out = new wcc_graph{g};
  });
}

int wcc_create_graph_from_edges(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                                int on_device, void *stream, wcc_graph **out) {
  return guarded([&] {
    if (!out) fail(WCC_ERR_INVALID, "out is NULL");
    *out = nullptr;
    Graph *g = create_from_edges(src, dst, m, n, on_device, (cudaStream_t)stream);
    *out = new wcc_graph{g};
  });
}

int64_t wcc_graph_num_vertices(const wcc_graph *g) { return g ? g->g->n : -1; }

int64_t wcc_graph_nnz(const wcc_graph *g) { return g ? g->g->nnz : -1; }

int wcc_graph_export_csr(const wcc_graph *g, int64_t *row_off, int32_t *cols, int on_device,
                         void *stream) {
  return guarded([&] {
    if (!g || !row_off || (!cols && g->g->nnz > 0)) fail(WCC_ERR_INVALID, "NULL argument");
    DeviceGuard dg(g->g->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    WCC_CUDA(cudaMemcpyAsync(row_off, g->g->off.p, 8 * (g->g->n + 1), k, s));
    if (g->g->nnz > 0) WCC_CUDA(cudaMemcpyAsync(cols, g->g->adj.p, 4 * g->g->nnz, k, s));
    WCC_CUDA(cudaStreamSynchronize(s));
  });
}

int wcc_run(const wcc_graph *g, const int32_t *clustering_in, const wcc_threshold_rule *rule,
            int32_t min_size, int32_t mode, int32_t *clustering_out, int on_device, void *stream,
            wcc_stats *stats) {
  return guarded([&] {
    if (!g) fail(WCC_ERR_INVALID, "graph is NULL");
    std::lock_guard<std::mutex> lk(g->g->run_mutex);
    DeviceGuard dg(g->g->device);
    run_impl(g->g, clustering_in, rule, min_size, mode, clustering_out, on_device,
             (cudaStream_t)stream, stats);
  });
}

int wcc_run_cm(const wcc_graph *g, const int32_t *clustering_in, const wcc_threshold_rule *rule,
               int32_t min_size, int64_t cpm_num, int64_t cpm_den, int32_t *clustering_out,
               int on_device, void *stream, wcc_stats *stats) {
  return guarded([&] {
    if (!g) fail(WCC_ERR_INVALID, "graph is NULL");
    if (cpm_num < 0 || cpm_den < 1 || cpm_num > (1ll << 31) || cpm_den > (1ll << 31))
      fail(WCC_ERR_INVALID, "the resolution must be cpm_num / cpm_den with 0 <= cpm_num <= 2^31 "
                            "and 1 <= cpm_den <= 2^31");
    std::lock_guard<std::mutex> lk(g->g->run_mutex);
    DeviceGuard dg(g->g->device);
    const CmOpts o{cpm_num, cpm_den};
    run_impl(g->g, clustering_in, rule, min_size, WCC_MODE_BATCHED, clustering_out, on_device,
             (cudaStream_t)stream, stats, &o);
  });
}

void wcc_destroy_graph(wcc_graph *g) {
  if (!g) return;
  {
    DeviceGuard *dg = nullptr;
    try {
      dg = new DeviceGuard(g->g->device);
    } catch (...) {
    }
    delete g->g;
    delete dg;
  }
  delete g;
}

int wcc_build_csr_no_alloc(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                           int64_t *row_off, int32_t *cols, int64_t *nnz, void *stream) {
  return guarded([&] {
    build_csr_no_alloc(src, dst, m, n, row_off, cols, nnz, (cudaStream_t)stream);
  });
}

int wcc_cluster_minima(const int32_t *labels, int64_t n, int32_t *minima, int on_device,
                       void *stream) {
  return guarded([&] {
    if (n < 0 || n >= (1ll << 31) - 1) fail(WCC_ERR_INVALID, "n must be in [0, 2^31-1)");
    if (n > 0 && (labels == nullptr || minima == nullptr)) fail(WCC_ERR_INVALID, "NULL buffer");
    current_device();
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws;
    DevBuf din, dout;
    const int32_t *l = labels;
    int32_t *o = minima;
    if (!on_device && n > 0) {
      int32_t *t = static_cast<int32_t *>(din.ensure(4 * n));
      WCC_CUDA(cudaMemcpyAsync(t, labels, 4 * n, cudaMemcpyHostToDevice, s));
      l = t;
      o = static_cast<int32_t *>(dout.ensure(4 * n));
    }
    cluster_minima(l, n, o, ws, s);
    if (!on_device && n > 0) {
      WCC_CUDA(cudaMemcpyAsync(minima, o, 4 * n, cudaMemcpyDeviceToHost, s));
      WCC_CUDA(cudaStreamSynchronize(s));
    }
  });
}

int wcc_number_by_minima(const int32_t *minima, int64_t n, int32_t *labels_out, int64_t *k,
                         int on_device, void *stream) {
  return guarded([&] {
    if (n < 0 || n >= (1ll << 31) - 1) fail(WCC_ERR_INVALID, "n must be in [0, 2^31-1)");
    if (n > 0 && (minima == nullptr || labels_out == nullptr)) fail(WCC_ERR_INVALID, "NULL buffer");
    current_device();
    cudaStream_t s = (cudaStream_t)stream;
    Workspace ws;
    DevBuf din, dout;
    const int32_t *mn = minima;
    int32_t *o = labels_out;
    if (!on_device && n > 0) {
      int32_t *t = static_cast<int32_t *>(din.ensure(4 * n));
      WCC_CUDA(cudaMemcpyAsync(t, minima, 4 * n, cudaMemcpyHostToDevice, s));
      mn = t;
      o = static_cast<int32_t *>(dout.ensure(4 * n));
    }
    check_minima(mn, n, ws, s);
    if (n > 0) number_clusters(mn, n, o, ws, s);
    int32_t top = -1;
    if (n > 0) {
      // ids are dense and ascending by smallest vertex: K = 1 + the largest id
      int32_t *mx = static_cast<int32_t *>(ws.b[23].ensure(4));
      WCC_CUDA(cudaMemsetAsync(mx, 0xff, 4, s));
      k_max_i32_launch(o, n, mx, s);
      WCC_CUDA(cudaMemcpyAsync(&top, mx, 4, cudaMemcpyDeviceToHost, s));
    }
    if (!on_device && n > 0) WCC_CUDA(cudaMemcpyAsync(labels_out, o, 4 * n, cudaMemcpyDeviceToHost, s));
    WCC_CUDA(cudaStreamSynchronize(s));
    if (k) *k = (int64_t)top + 1;
  });
}

int64_t wcc_kernel_launches(void) { return launches_so_far(); }

int64_t wcc_device_allocations(void) { return g_allocs.load(std::memory_order_relaxed); }

const char *wcc_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

extern "C" {

int wcc_get_tuning(wcc_tuning *out) {
  return wccg::guarded([&] {
    if (!out) wccg::fail(WCC_ERR_INVALID, "out is NULL");
    *out = wccg::current_tuning();
  });
}

int wcc_set_tuning(const wcc_tuning *t) {
  return wccg::guarded([&] {
    if (!t) wccg::fail(WCC_ERR_INVALID, "tuning is NULL");
    if (!wccg::tuning_valid(*t)) wccg::fail(WCC_ERR_INVALID, "tuning out of range");
    wccg::store_tuning(*t);
  });
}

int wcc_autotune(const wcc_graph *g, const int32_t *clustering_in, const wcc_threshold_rule *rule,
                 int32_t min_size, int on_device, void *stream, const char *cache_path,
                 wcc_tuning *best, double *best_ms) {
  return wccg::guarded([&] {
    if (!g || !g->g) wccg::fail(WCC_ERR_INVALID, "graph is NULL");
    std::lock_guard<std::mutex> lk(g->g->run_mutex);
    wccg::DeviceGuard dg(g->g->device);
    wccg::autotune_impl(g->g, clustering_in, rule, min_size, on_device, (cudaStream_t)stream,
                        cache_path, best, best_ms);
  });
}

int wcc_load_tuning(const char *cache_path, wcc_tuning *out) {
  return wccg::guarded([&] { wccg::load_tuning_impl(cache_path, out); });
}

}  // extern "C"

struct wcc_job {
  wccg::Job *j;
  const wcc_graph *g;
};

extern "C" {

int wcc_job_start(const wcc_graph *g, const int32_t *clustering_in, const wcc_threshold_rule *rule,
                  int32_t min_size, int on_device, void *stream, wcc_job **out) {
  return wccg::guarded([&] {
    if (!g || !g->g || !out) wccg::fail(WCC_ERR_INVALID, "graph and out must not be NULL");
    std::lock_guard<std::mutex> lk(g->g->run_mutex);
    wccg::DeviceGuard dg(g->g->device);
    wccg::Job *j = wccg::job_start(g->g, clustering_in, rule, min_size, on_device,
                                   (cudaStream_t)stream);
    *out = new wcc_job{j, g};
  });
}

int wcc_job_step(wcc_job *job, int64_t time_budget_ms, void *stream) {
  int st = WCC_OK;
  const int r = wccg::guarded([&] {
    if (!job) wccg::fail(WCC_ERR_INVALID, "job is NULL");
    wccg::DeviceGuard dg(job->g->g->device);
    st = wccg::job_step(job->j, time_budget_ms, (cudaStream_t)stream) ? WCC_OK : WCC_PENDING;
  });
  return r == WCC_OK ? st : r;
}

int wcc_job_save(wcc_job *job, const char *path, void *stream) {
  return wccg::guarded([&] {
    if (!job) wccg::fail(WCC_ERR_INVALID, "job is NULL");
    wccg::DeviceGuard dg(job->g->g->device);
    wccg::job_save(job->j, path, (cudaStream_t)stream);
  });
}

int wcc_job_load(const wcc_graph *g, const char *path, void *stream, wcc_job **out) {
  return wccg::guarded([&] {
    if (!g || !g->g || !out) wccg::fail(WCC_ERR_INVALID, "graph and out must not be NULL");
    wccg::DeviceGuard dg(g->g->device);
    wccg::Job *j = wccg::job_load(g->g, path, (cudaStream_t)stream);
    *out = new wcc_job{j, g};
  });
}

int wcc_job_finish(wcc_job *job, int32_t *clustering_out, int on_device, void *stream,
                   wcc_stats *stats) {
  return wccg::guarded([&] {
    if (!job) wccg::fail(WCC_ERR_INVALID, "job is NULL");
    std::lock_guard<std::mutex> lk(job->g->g->run_mutex);
    wccg::DeviceGuard dg(job->g->g->device);
    wccg::job_finish(job->j, clustering_out, on_device, (cudaStream_t)stream, stats);
  });
}

void wcc_job_destroy(wcc_job *job) {
  if (!job) return;
  wccg::guarded([&] {
    wccg::DeviceGuard dg(job->g->g->device);
    wccg::job_destroy(job->j);
  });
  delete job;
}

}  // extern "C"
