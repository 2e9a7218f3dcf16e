// pipeline.cu -- the stages around the refinement kernel, shared by wcc_run
// and the serving loop: grouping the vertices of a request by input label
// (a2), publishing its input clusters as work items (a8 seeding), and
// numbering the accepted clusters (a9).
#include "internal.h"

namespace wccg {

namespace {

constexpr int TB = 256;

// Workspace slots.
enum {
  B_KEYS, B_VALS, B_KEYS2, B_VALS2, B_TEMP, B_HEAD, B_HIDX, B_CSTART, B_PDEG, B_KEEP, B_QIDX,
  B_DG, B_OK1, B_OV1, B_OK2, B_OV2, B_INFO, B_FLAG, B_RANK, B_BASE, B_COUNT
};
static_assert(B_COUNT <= 24, "workspace slots");

struct SeedInfo {
  unsigned long long max_n;     // largest kept cluster
  unsigned long long max_dsum;  // largest degree sum of a kept cluster
  long long clusters;           // K: distinct labels
  long long skip;               // unclustered vertices (they sort first)
  unsigned err;                 // DERR_* bits
  unsigned maxkey;              // largest label + 1
  unsigned kept;                // clusters with >= min_size members
  unsigned pad;
};

// keys[v] = label + 1 (0 for unclustered), vals[v] = v; largest key; labels
// below -1 are malformed.
__global__ void k_make_keys(const int32_t *__restrict__ lab, int64_t n, uint32_t *keys,
                            uint32_t *vals, unsigned *maxkey, unsigned *err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned k = 0;
  if (i < n) {
    int32_t c = lab[i];
    if (c < -1) atomicOr(err, DERR_INVALID);
    k = c < 0 ? 0u : (unsigned)c + 1u;
    keys[i] = k;
    vals[i] = (uint32_t)i;
  }
  k = warp_max(k);
  if ((threadIdx.x & 31) == 0 && k) atomicMax(maxkey, k);
}

__global__ void k_heads(const uint32_t *__restrict__ sk, int64_t n, uint32_t *head) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  head[i] = (sk[i] != 0 && (i == 0 || sk[i - 1] != sk[i])) ? 1u : 0u;
}

// cstart[c] = first sorted position of cluster c, cstart[K] = n; also
// records K and the number of unclustered vertices (they sort first).
__global__ void k_starts(const uint32_t *__restrict__ head, const uint32_t *__restrict__ hidx,
                         int64_t n, int64_t *cstart, SeedInfo *info) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t K = hidx[n];
  if (i < n && head[i]) {
    cstart[hidx[i]] = i;
    if (hidx[i] == 0) info->skip = i;
  }
  if (i == 0) {
    cstart[K] = n;
    info->clusters = K;
    if (K == 0) info->skip = n;
  }
}

// degree of each vertex in sorted order (for the per-cluster degree sums)
__global__ void k_sorted_deg(const uint32_t *__restrict__ sv, const int64_t *__restrict__ off,
                             int64_t n, int64_t *dg) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t v = sv[i];
  dg[i] = off[v + 1] - off[v];
}

__global__ void k_keep(const int64_t *__restrict__ cstart, const uint32_t *__restrict__ Kp,
                       int64_t cap, int min_size, uint32_t *keep,
                       const int64_t *__restrict__ pdeg, SeedInfo *info) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t K = *Kp;
  unsigned long long sz = 0, ds = 0;
  if (c < cap && c >= K) keep[c] = 0u;
  if (c < K) {
    sz = (unsigned long long)(cstart[c + 1] - cstart[c]);
    bool k = (int64_t)sz >= min_size;
    keep[c] = k ? 1u : 0u;
    if (k) ds = (unsigned long long)(pdeg[cstart[c + 1]] - pdeg[cstart[c]]);
    else sz = 0;
  }
  sz = warp_max(sz);
  ds = warp_max(ds);
  if ((threadIdx.x & 31) == 0) {
    if (sz) atomicMax(&info->max_n, sz);
    if (ds) atomicMax(&info->max_dsum, ds);
  }
}

// Sort keys putting kept clusters first, larger ones earlier (longest work
// first); unkept clusters get the largest key.
__global__ void k_size_keys(const int64_t *__restrict__ cstart, const uint32_t *__restrict__ keep,
                            int64_t K, uint32_t max_n, uint32_t *keys, uint32_t *vals) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= K) return;
  uint32_t sz = (uint32_t)(cstart[c + 1] - cstart[c]);
  keys[c] = keep[c] ? max_n - sz : max_n + 1;
  vals[c] = (uint32_t)c;
}

// The same order for at most ORDER_SMALL clusters in one block: the keys of
// k_size_keys paired with the cluster index (which breaks ties as the
// stable sort does), sorted by a bitonic network in shared memory, and the
// kept clusters' ranks written as k_invert does.
constexpr int ORDER_SMALL = 4096;
__global__ void __launch_bounds__(1024) k_order_small(const int64_t *__restrict__ cstart,
                                                      const uint32_t *__restrict__ keep, int64_t K,
                                                      uint32_t max_n, int64_t nkept,
                                                      uint32_t *qidx) {
  __shared__ unsigned long long a[ORDER_SMALL];
  int P = 2;
  while (P < K) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    unsigned long long v = ~0ull;
    if (i < K) {
      const uint32_t sz = (uint32_t)(cstart[i + 1] - cstart[i]);
      const uint32_t key = keep[i] ? max_n - sz : max_n + 1;
      v = ((unsigned long long)key << 32) | (unsigned)i;
    }
    a[i] = v;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long x = a[i], y = a[l];
          if ((x > y) == ((i & k) == 0)) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < nkept; i += blockDim.x) qidx[(uint32_t)a[i]] = (uint32_t)i;
}

__global__ void k_invert(const uint32_t *__restrict__ order, int64_t nkept, uint32_t *qidx) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nkept) qidx[order[i]] = (uint32_t)i;
}

// Reserves queue indices [base, base + nkept) for the items of one request
// and counts them as pending (globally and for the request) before any of
// them is published.
__global__ void k_reserve(RunCounters *ctr, ReqCtx *ctx, long long nkept,
                          unsigned long long *base) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    atomicAdd(reinterpret_cast<unsigned long long *>(&ctx->pending),
              static_cast<unsigned long long>(nkept));
    atomicAdd(reinterpret_cast<unsigned long long *>(&ctr->pending),
              static_cast<unsigned long long>(nkept));
    __threadfence();
    const unsigned long long b = atomicAdd(&ctr->tail, (unsigned long long)nkept);
    *base = b;
    ctx->seed_end = b + (unsigned long long)nkept;
  }
}

// pool[i - skip] = sorted vertex; slot[v] = (queue index << 32) | rank
__global__ void k_pool_slots(const uint32_t *__restrict__ sv, const uint32_t *__restrict__ head,
                             const uint32_t *__restrict__ hidx, const int64_t *__restrict__ cstart,
                             const uint32_t *__restrict__ keep, const uint32_t *__restrict__ qidx,
                             const unsigned long long *__restrict__ base, int64_t n, int64_t skip,
                             int32_t *pool, unsigned long long *slot) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || i < skip) return;
  uint32_t v = sv[i];
  pool[i - skip] = (int32_t)v;
  int64_t c = (int64_t)hidx[i] + head[i] - 1;  // inclusive head count - 1
  if (keep[c])
    slot[v] = ((unsigned long long)queue_tag(*base + qidx[c]) << 32) | (unsigned)(i - cstart[c]);
}

// Descriptors of the kept clusters, then their publication.
__global__ void k_seed(const int64_t *__restrict__ cstart, const uint32_t *__restrict__ keep,
                       const uint32_t *__restrict__ qidx, const unsigned long long *__restrict__ base,
                       int64_t K, int64_t skip, uint16_t req, QSlot *ring, uint64_t cap) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= K || !keep[c]) return;
  uint64_t q = *base + qidx[c];
  QSlot *s = &ring[q % cap];
  s->item.vbeg = cstart[c] - skip;
  s->item.n = (int32_t)(cstart[c + 1] - cstart[c]);
  s->item.flags = ITEM_TOP;
  s->item.req = req;
  __threadfence();
  atomicExch((unsigned long long *)&s->seq, (unsigned long long)q);
}

__global__ void k_out_flags(const int32_t *__restrict__ lmin, int64_t n, uint32_t *flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = lmin[i] == (int32_t)i ? 1u : 0u;
}

__global__ void k_out_final(const int32_t *__restrict__ lmin, const uint32_t *__restrict__ rank,
                            int64_t n, int32_t *out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t r = lmin[i];
  out[i] = r >= 0 ? (int32_t)rank[r] : -1;
}

template <typename T>
T *buf(Workspace &ws, int k, size_t count) {
  return static_cast<T *>(ws.b[k].ensure(sizeof(T) * (count > 0 ? count : 1)));
}

}  // namespace

int64_t bitlen_u64(uint64_t x) {
  int64_t b = 0;
  while (x) { ++b; x >>= 1; }
  return b;
}

unsigned grid_for(int64_t n, int per) {
  int64_t b = (n + per - 1) / per;
  if (b < 1) b = 1;
  if (b > 0x7fffffff) b = 0x7fffffff;
  return (unsigned)b;
}

void check_device_error(unsigned err, const char *what) {
  if (!err) return;
  if (err & DERR_INVALID) fail(WCC_ERR_INVALID, std::string(what) + ": malformed input");
  if (err & DERR_TIMEOUT)
    fail(WCC_ERR_TIMEOUT, std::string(what) + ": a device-side queue wait exceeded its limit");
  if (err & DERR_CAPACITY)
    fail(WCC_ERR_INTERNAL, std::string(what) + ": an internal capacity bound was exceeded");
  fail(WCC_ERR_INTERNAL, std::string(what) + ": internal consistency check failed");
}

GroupInfo group_by_label(const int64_t *off, int64_t n, const int32_t *labels, int min_size,
                         Workspace &ws, cudaStream_t s) {
  GroupInfo gi{};
  uint32_t *keys = buf<uint32_t>(ws, B_KEYS, n);
  uint32_t *vals = buf<uint32_t>(ws, B_VALS, n);
  uint32_t *keys2 = buf<uint32_t>(ws, B_KEYS2, n);
  uint32_t *vals2 = buf<uint32_t>(ws, B_VALS2, n);
  void *temp = ws.b[B_TEMP].ensure(std::max(radix_temp_bytes(n), scan_temp_bytes(n + 1)));
  SeedInfo *info = buf<SeedInfo>(ws, B_INFO, 1);
  WCC_CUDA(cudaMemsetAsync(info, 0, sizeof(SeedInfo), s));
  k_make_keys<<<grid_for(n), TB, 0, s>>>(labels, n, keys, vals, &info->maxkey, &info->err);
  note_launch();
  WCC_CUDA(cudaGetLastError());
  SeedInfo h0 = read_back(info, s);
  if (h0.err) check_device_error(h0.err, "clustering_in");
  uint32_t *sk = keys, *sv = vals;
  if (radix_sort_pairs_u32(keys, vals, keys2, vals2, n, (int)bitlen_u64(h0.maxkey), temp,
                           &info->err, s)) {
    sk = keys2;
    sv = vals2;
  }
  ws.sk = sk;
  ws.sv = sv;
  uint32_t *head = buf<uint32_t>(ws, B_HEAD, n + 1);
  uint32_t *hidx = buf<uint32_t>(ws, B_HIDX, n + 1);
  k_heads<<<grid_for(n), TB, 0, s>>>(sk, n, head); note_launch();
  WCC_CUDA(cudaGetLastError());
  // hidx[n] receives the number of distinct labels K; arrays indexed by
  // cluster are sized by n so that K need not be read back here
  exclusive_scan_u32(head, hidx, n, hidx + n, temp, s);
  int64_t *cstart = buf<int64_t>(ws, B_CSTART, n + 1);
  k_starts<<<grid_for(n), TB, 0, s>>>(head, hidx, n, cstart, info); note_launch();
  // per-cluster degree sums (prefix sums of degrees in sorted order)
  int64_t *dg = buf<int64_t>(ws, B_DG, n + 1);
  int64_t *pdeg = buf<int64_t>(ws, B_PDEG, n + 1);
  uint32_t *keep = buf<uint32_t>(ws, B_KEEP, n + 1);
  uint32_t *qidx = buf<uint32_t>(ws, B_QIDX, n + 1);
  k_sorted_deg<<<grid_for(n), TB, 0, s>>>(sv, off, n, dg); note_launch();
  WCC_CUDA(cudaMemsetAsync(dg + n, 0, 8, s));
  exclusive_scan_i64(dg, pdeg, n + 1, nullptr, temp, s);
  k_keep<<<grid_for(n), TB, 0, s>>>(cstart, hidx + n, n, min_size, keep, pdeg, info);
  note_launch();
  exclusive_scan_u32(keep, qidx, n, &info->kept, temp, s);
  WCC_CUDA(cudaGetLastError());
  SeedInfo hi = read_back(info, s);
  if (hi.err) check_device_error(hi.err, "grouping");
  gi.clusters = hi.clusters;
  gi.skip = hi.skip;
  gi.kept = (int64_t)hi.kept;
  gi.max_n = (int64_t)hi.max_n;
  gi.max_dsum = (int64_t)hi.max_dsum;
  const int64_t K = gi.clusters;
  if (gi.kept > 1 && K <= ORDER_SMALL) {
    // queue order: largest input clusters first (qidx = rank by size), in one block
    k_order_small<<<1, 1024, 0, s>>>(cstart, keep, K, (uint32_t)gi.max_n, gi.kept, qidx);
    note_launch();
    WCC_CUDA(cudaGetLastError());
  } else if (gi.kept > 1) {
    // queue order: largest input clusters first (qidx = rank by size)
    uint32_t *ok1 = buf<uint32_t>(ws, B_OK1, K);
    uint32_t *ov1 = buf<uint32_t>(ws, B_OV1, K);
    uint32_t *ok2 = buf<uint32_t>(ws, B_OK2, K);
    uint32_t *ov2 = buf<uint32_t>(ws, B_OV2, K);
    k_size_keys<<<grid_for(K), TB, 0, s>>>(cstart, keep, K, (uint32_t)gi.max_n, ok1, ov1);
    note_launch();
    uint32_t *ov = ov1;
    if (radix_sort_pairs_u32(ok1, ov1, ok2, ov2, K, (int)bitlen_u64(gi.max_n + 1), temp,
                             &info->err, s))
      ov = ov2;
    k_invert<<<grid_for(gi.kept), TB, 0, s>>>(ov, gi.kept, qidx); note_launch();
    WCC_CUDA(cudaGetLastError());
    const unsigned e = read_back(&info->err, s);
    if (e) check_device_error(e, "grouping");
  }
  return gi;
}

void seed_items(const GroupInfo &gi, int64_t n, Workspace &ws, uint16_t req, ReqCtx *ctx_dev,
                int32_t *pool, unsigned long long *slot, QSlot *ring, uint64_t cap,
                RunCounters *ctr, cudaStream_t s) {
  if (gi.kept <= 0) return;
  unsigned long long *base = buf<unsigned long long>(ws, B_BASE, 1);
  k_reserve<<<1, 32, 0, s>>>(ctr, ctx_dev, gi.kept, base); note_launch();
  k_pool_slots<<<grid_for(n), TB, 0, s>>>(ws.sv, static_cast<uint32_t *>(ws.b[B_HEAD].p),
                                          static_cast<uint32_t *>(ws.b[B_HIDX].p),
                                          static_cast<int64_t *>(ws.b[B_CSTART].p),
                                          static_cast<uint32_t *>(ws.b[B_KEEP].p),
                                          static_cast<uint32_t *>(ws.b[B_QIDX].p), base, n,
                                          gi.skip, pool, slot);
  note_launch();
  k_seed<<<grid_for(gi.clusters), TB, 0, s>>>(static_cast<int64_t *>(ws.b[B_CSTART].p),
                                              static_cast<uint32_t *>(ws.b[B_KEEP].p),
                                              static_cast<uint32_t *>(ws.b[B_QIDX].p), base,
                                              gi.clusters, gi.skip, req, ring, cap);
  note_launch();
  WCC_CUDA(cudaGetLastError());
}

// ---- merging refinements of disjoint sets of input clusters ------------------
__global__ void k_fill_i32(int32_t *a, int64_t n, int32_t v) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

// Per vertex, the smallest vertex of its cluster, from labels in [-1, n):
// every vertex lowers its label's entry of mins (initially n) to its id.
__global__ void k_label_mins(const int32_t *__restrict__ lab, int64_t n, int32_t *mins,
                             unsigned *err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t l = lab[i];
  if (l < -1 || l >= n) {
    atomicOr(err, DERR_INVALID);
    return;
  }
  if (l >= 0) atomicMin(&mins[l], (int32_t)i);
}

__global__ void k_vertex_mins(const int32_t *__restrict__ lab, const int32_t *__restrict__ mins,
                              int64_t n, int32_t *out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t l = lab[i];
  out[i] = (l >= 0 && l < n) ? mins[l] : -1;
}

// Minima must name a vertex of the same cluster whose own minimum is
// itself (a representative), and never exceed the vertex.
__global__ void k_check_minima(const int32_t *__restrict__ mn, int64_t n, unsigned *err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t r = mn[i];
  if (r == -1) return;
  if (r < 0 || r > i || mn[r] != r) atomicOr(err, DERR_INVALID);
}

__global__ void k_max_i32(const int32_t *__restrict__ a, int64_t n, int32_t *out) {
  int32_t m = -1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = a[i] > m ? a[i] : m;
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

void k_max_i32_launch(const int32_t *a, int64_t n, int32_t *out, cudaStream_t s) {
  const unsigned g = grid_for(n) < 1024u ? grid_for(n) : 1024u;
  k_max_i32<<<g, TB, 0, s>>>(a, n, out); note_launch();
  WCC_CUDA(cudaGetLastError());
}

void cluster_minima(const int32_t *labels, int64_t n, int32_t *minima, Workspace &ws,
                    cudaStream_t s) {
  int32_t *mins = buf<int32_t>(ws, B_RANK, n);
  unsigned *err = buf<unsigned>(ws, B_FLAG, 1);
  WCC_CUDA(cudaMemsetAsync(err, 0, 4, s));
  if (n > 0) {
    k_fill_i32<<<grid_for(n), TB, 0, s>>>(mins, n, (int32_t)n); note_launch();
    k_label_mins<<<grid_for(n), TB, 0, s>>>(labels, n, mins, err); note_launch();
    k_vertex_mins<<<grid_for(n), TB, 0, s>>>(labels, mins, n, minima); note_launch();
    WCC_CUDA(cudaGetLastError());
  }
  unsigned h = 0;
  WCC_CUDA(cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, s));
  WCC_CUDA(cudaStreamSynchronize(s));
  if (h) fail(WCC_ERR_INVALID, "a label outside [-1, n)");
}

void check_minima(const int32_t *minima, int64_t n, Workspace &ws, cudaStream_t s) {
  unsigned *err = buf<unsigned>(ws, B_TEMP, 1);
  WCC_CUDA(cudaMemsetAsync(err, 0, 4, s));
  if (n > 0) {
    k_check_minima<<<grid_for(n), TB, 0, s>>>(minima, n, err); note_launch();
    WCC_CUDA(cudaGetLastError());
  }
  unsigned h = 0;
  WCC_CUDA(cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, s));
  WCC_CUDA(cudaStreamSynchronize(s));
  if (h) fail(WCC_ERR_INVALID, "minima: an entry is not the smallest vertex of a cluster");
}

void number_clusters(const int32_t *label_min, int64_t n, int32_t *out, Workspace &ws,
                     cudaStream_t s) {
  uint32_t *flag = buf<uint32_t>(ws, B_FLAG, n);
  uint32_t *rank = buf<uint32_t>(ws, B_RANK, n);
  void *temp = ws.b[B_TEMP].ensure(std::max(radix_temp_bytes(n), scan_temp_bytes(n + 1)));
  k_out_flags<<<grid_for(n), TB, 0, s>>>(label_min, n, flag); note_launch();
  exclusive_scan_u32(flag, rank, n, nullptr, temp, s);
  k_out_final<<<grid_for(n), TB, 0, s>>>(label_min, rank, n, out); note_launch();
  WCC_CUDA(cudaGetLastError());
}

}  // namespace wccg
