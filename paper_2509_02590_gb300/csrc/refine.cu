// refine.cu -- the refinement kernel: one CTA processes one work item at a
// time (an input cluster, or a part produced by an earlier split), entirely
// in on-chip shared memory when the item fits, else in a per-CTA slab of
// global memory.
//
// Per item (paper: Algorithm 1 for input clusters, then Algorithm 3 with a
// peel and a connectivity check in front of the cut):
//   1. extraction of the induced subgraph G[S] (Algorithm 1 / 3: E_c = edges
//      with both ends in V_c) into a local CSR, local id = rank of the global
//      id in S: one flat, load-balanced pass over all adjacency entries of
//      the members with an 8-byte gather of slot[u] = (item << 32 | local id)
//      per entry; local ids are 16-bit when the item has < 65535 vertices;
//   2. input clusters only: connected components (CCR); each component with
//      at least min_size vertices is queued, or refinement continues in place
//      when the cluster is one component;
//   3. round-synchronous peel of vertices with degree <= T(n);
//   4. if the peel removed anything: connected components; more than one ->
//      queue each large component (an item arrives connected, so without a
//      peel the check is skipped);
//   5. Nagamochi-Ibaraki contraction with k = T+1: maximum-adjacency passes
//      (keys capped at k, ties to the smallest id) merging every edge whose
//      key reaches k, until one super-vertex (accept: min cut > T) or a pass
//      merges nothing;
//   6. otherwise canonical Stoer-Wagner on the contracted graph (ties to the
//      smallest id, earliest minimum phase, side = last-added super-vertex)
//      and both sides with at least min_size vertices are queued
//      (MinCutPartition and the recursion of Algorithm 3).
// Children are written in place into the parent's range of the vertex pool
// and published to a device-side ring queue; CTAs claim queue indices with
// an atomic counter and wait (bounded by %globaltimer) for publication.
#include "internal.h"

namespace wccg {

namespace {

constexpr int RB = 256;        // threads per CTA
constexpr int RW = RB / 32;    // warps per CTA
constexpr size_t SMEM_MAX_BYTES = 227 * 1024;  // opt-in limit per CTA

// Dynamic shared memory of a refinement CTA.  Item code instantiated for
// shared memory derives every pointer from this symbol, so the compiler
// knows their address space and uses shared-memory instructions instead of
// generic ones.
extern __shared__ __align__(16) char wcc_dyn_smem[];

// Contraction passes keep every not-yet-added super-vertex in the bucket of
// its (capped) key: KB_LEVELS bitmaps over local ids plus one summary bit per
// bitmap word, so "largest key, then smallest id" is the highest non-empty
// bucket's lowest set bit.  Caps above KB_LEVELS-1 use the linear argmax.
constexpr int KB_LEVELS = 16;
// Items whose first contraction pass covers at least this many vertices
// record it for the sides of a later cut.
constexpr int INH_MIN_N = 64;

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline int bm_words(int64_t n) { return (int)((n + 31) / 32); }
__host__ __device__ inline int bm_sum_words(int64_t n) { return (bm_words(n) + 31) / 32; }
__host__ __device__ inline size_t bucket_bitmap_bytes(int64_t n) {
  return align16(4 * (size_t)KB_LEVELS * (size_t)(bm_words(n) + bm_sum_words(n)));
}

// Working memory of one item of n vertices and at most d local adjacency
// entries (d = sum of the members' global degrees); see carve().
template <typename IT>
__host__ __device__ inline size_t ws_bytes(int64_t n, int64_t d) {
  size_t b = 0;
  b += align16(4 * (size_t)n);              // gid
  b += align16(4 * (size_t)(n + 1));        // off
  b += 6 * align16(4 * (size_t)(n + 1));    // A, B, C, D, G, H
  b += align16(8 * (size_t)(n + 1));        // E and F (one int64 array during extraction)
  b += 4 * align16((size_t)n);              // alive, flag, side, kst
  b += bucket_bitmap_bytes(n);              // key buckets
  b += align16(4 * (size_t)((d + 31) / 32 + 1));  // contraction marks, one bit per entry
  b += align16(sizeof(IT) * (size_t)d);     // local adjacency
  return b + 64;
}

template <typename IT>
struct Mem {
  int32_t *gid, *off, *A, *B, *C, *D, *E, *F, *G, *H;
  int64_t *wide;       // E..F viewed as int64[n+1]
  uint8_t *alive, *flag, *side;
  uint8_t *kst;        // first contraction pass: capped key, or 255 once added / dead
  uint32_t *bm, *bms;  // bucket bitmaps [levels][W], summaries [levels][S]
  uint32_t *vis;       // first contraction pass: added vertices, one bit each (W words)
  int W, S;
  uint32_t *ebits;     // one bit per local adjacency entry
  IT *adj;
  size_t smem_used;    // bytes of dynamic shared memory the item occupies
  bool off_in_smem;    // a global-slab item keeps its row offsets in shared memory
};

template <typename IT>
__device__ __forceinline__ Mem<IT> carve(char *base, int n, int64_t d) {
  Mem<IT> m;
  char *p = base;
  auto take = [&](size_t b) { char *r = p; p += align16(b); return r; };
  m.gid = (int32_t *)take(4 * (size_t)n);
  m.off = (int32_t *)take(4 * (size_t)(n + 1));
  m.A = (int32_t *)take(4 * (size_t)(n + 1));
  m.B = (int32_t *)take(4 * (size_t)(n + 1));
  m.C = (int32_t *)take(4 * (size_t)(n + 1));
  m.D = (int32_t *)take(4 * (size_t)(n + 1));
  m.G = (int32_t *)take(4 * (size_t)(n + 1));
  m.H = (int32_t *)take(4 * (size_t)(n + 1));
  m.wide = (int64_t *)take(8 * (size_t)(n + 1));
  m.E = (int32_t *)m.wide;
  m.F = m.E + (n + 1);
  m.alive = (uint8_t *)take((size_t)n);
  m.flag = (uint8_t *)take((size_t)n);
  m.side = (uint8_t *)take((size_t)n);
  m.kst = (uint8_t *)take((size_t)n);
  m.W = bm_words(n);
  m.S = bm_sum_words(n);
  m.bm = (uint32_t *)take(bucket_bitmap_bytes(n));
  m.bms = m.bm + (size_t)KB_LEVELS * m.W;
  m.ebits = (uint32_t *)take(4 * (size_t)((d + 31) / 32 + 1));
  m.adj = (IT *)take(sizeof(IT) * (size_t)d);
  m.vis = reinterpret_cast<uint32_t *>(m.E);
  m.smem_used = 0;
  m.off_in_smem = false;
  return m;
}

// An item in the global slab keeps the first contraction pass's hot state --
// keys (n bytes), the key levels it can use with their summaries, the added
// bits -- in shared memory when that fits: the pass's dependent chain then
// never waits on L2.  levels = T(n)+2 bounds kcap+1, since the peel only
// lowers n.
__host__ __device__ inline size_t hot_bytes(int64_t n, int levels) {
  return align16((size_t)n) + align16(4 * (size_t)levels * (size_t)(bm_words(n) + bm_sum_words(n))) +
         align16(4 * (size_t)bm_words(n));
}
// Also the local row offsets (read on every step's dependent chain) when
// they fit beside the rest.
template <typename IT>
__device__ __forceinline__ bool carve_hot(Mem<IT> &m, int n, int levels, size_t smem_bytes) {
  const size_t hb = hot_bytes(n, levels);
  if (hb > smem_bytes) return false;
  char *h = wcc_dyn_smem;
  m.kst = reinterpret_cast<uint8_t *>(h);
  h += align16((size_t)n);
  m.bm = reinterpret_cast<uint32_t *>(h);
  m.bms = m.bm + (size_t)levels * m.W;
  h += align16(4 * (size_t)levels * (size_t)(m.W + m.S));
  m.vis = reinterpret_cast<uint32_t *>(h);
  h += align16(4 * (size_t)m.W);
  m.smem_used = hb;
  if (hb + align16(4 * (size_t)(n + 1)) <= smem_bytes) {
    m.off = reinterpret_cast<int32_t *>(h);
    m.smem_used = hb + align16(4 * (size_t)(n + 1));
    m.off_in_smem = true;
  }
  return true;
}

// Block-level scalars.
struct Sh {
  int32_t scan[RW + 1];
  long long lscan[RW + 1];
  int go;
  int32_t i0;
  unsigned long long u0, u1;
  int32_t ntouched;
  int32_t contracted;
  int32_t changed;
  int32_t sw_s, sw_t, sw_cut, sw_x, sw_key;
  // per-item profile (only when RefineParams::prof is set)
  long long ts[9];
  long long dbg[4];
  int32_t used_slab, pf_E, pf_nalive, pf_passes, pf_nsv, pf_forest, pf_nsv1;
  long long pf_forest_cycles, pf_t0;
  long long fdbg[6];
  uint32_t sink[32];  // per-lane dummy targets of branch-free warp code
  Item batch[RW];     // claimed items: the first one, then more when it is small
  unsigned long long bseq[RW];
  int32_t nb;
  unsigned long long claim_h;  // first index of the block claimed after the first item
  int32_t claim_k;             // its length
  int32_t duf[32];    // dense finish: merges of one pass (union-find over indices)
  uint32_t dside;     // dense finish: side of the minimum cut (mask of indices)
  int32_t wduf[128], wgrp[128];  // wide dense finish: union-find, sets of initial indices
  uint32_t wside[4];             // wide dense finish: side of the minimum cut
  int32_t dcut, dpasses, dphases;
};

// Outcome of one item.
enum : int { OUT_ERROR = -1, OUT_DROPPED = 0, OUT_CCR_SPLIT = 1, OUT_CC_SPLIT = 2,
             OUT_ACCEPT = 3, OUT_CUT_SPLIT = 4 };

// Cycle stamp k of the per-item profile (thread 0; no-op unless enabled).
__device__ __forceinline__ void prof_stamp(const RefineParams &P, Sh &sh, int k) {
  if (P.prof && threadIdx.x == 0) sh.ts[k] = clock64();
}

// ---- small device helpers ----------------------------------------------------

// A request's context as this CTA sees it: loaded through L2 (not L1), since
// a server reuses a table entry for a later request while the kernel runs.
__device__ __forceinline__ ReqCtx load_ctx(const ReqCtx *g) {
  ReqCtx r;
  r.off = reinterpret_cast<const int64_t *>(__ldcg(reinterpret_cast<const unsigned long long *>(&g->off)));
  r.adj = reinterpret_cast<const int32_t *>(__ldcg(reinterpret_cast<const unsigned long long *>(&g->adj)));
  r.n_vertices = __ldcg(reinterpret_cast<const long long *>(&g->n_vertices));
  r.pool = reinterpret_cast<int32_t *>(__ldcg(reinterpret_cast<const unsigned long long *>(&g->pool)));
  r.slot = reinterpret_cast<unsigned long long *>(
      __ldcg(reinterpret_cast<const unsigned long long *>(&g->slot)));
  r.label_min =
      reinterpret_cast<int32_t *>(__ldcg(reinterpret_cast<const unsigned long long *>(&g->label_min)));
  r.inh = reinterpret_cast<unsigned long long *>(
      __ldcg(reinterpret_cast<const unsigned long long *>(&g->inh)));
  r.rule_kind = __ldcg(&g->rule_kind);
  r.min_size = __ldcg(&g->min_size);
  r.rule_num = __ldcg(reinterpret_cast<const long long *>(&g->rule_num));
  r.rule_den = __ldcg(reinterpret_cast<const long long *>(&g->rule_den));
  return r;
}

// Signed 64-bit atomic add (two's complement through the unsigned overload).
__device__ __forceinline__ void add_ll(long long *p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
}

// Criterion threshold T(n) (Section 2, criterion f(n)): the largest integer
// with cut <= T(n) <=> cut <= f(n) for integer cuts.
__device__ int64_t threshold_of(int kind, int64_t num, int64_t den, int64_t n) {
  if (n < 1) return -1;
  int64_t t = 0, p = 1;
  switch (kind) {
    case WCC_RULE_LOG10:
      while (p <= n / 10) { p *= 10; ++t; }
      return t;
    case WCC_RULE_LOG2:
      return 63 - __clzll((unsigned long long)n);
    case WCC_RULE_SQRT: {
      t = (int64_t)sqrt((double)n);
      while (t > 0 && t * t > n) --t;
      while ((t + 1) * (t + 1) <= n) ++t;
      return t;
    }
    case WCC_RULE_LINEAR:
      return den > 0 ? (num * n) / den : -1;
    default:
      return -1;
  }
}

// Lock-free union-find over ids whose links always point to a smaller id, so
// the root of a set is its smallest member.
__device__ __forceinline__ int uf_find(int32_t *p, int x) {
  volatile int32_t *vp = p;
  int y = vp[x];
  while (y != x) {
    int z = vp[y];
    if (z != y) vp[x] = z;  // path halving: z is an ancestor of x
    x = y;
    y = z;
  }
  return x;
}

__device__ __forceinline__ void uf_union(int32_t *p, int a, int b) {
  for (;;) {
    a = uf_find(p, a);
    b = uf_find(p, b);
    if (a == b) return;
    if (a > b) { int t = a; a = b; b = t; }
    int old = atomicCAS(&p[b], b, a);
    if (old == b) return;
    b = old;
  }
}

// Like uf_union, but reports whether the call joined two different sets.
// Concurrent calls are linearisable, so the edges whose call returned true
// form a spanning forest of all the edges tried.
__device__ __forceinline__ bool uf_link(int32_t *p, int a, int b) {
  for (;;) {
    a = uf_find(p, a);
    b = uf_find(p, b);
    if (a == b) return false;
    if (a > b) { int t = a; a = b; b = t; }
    if (atomicCAS(&p[b], b, a) == b) return true;
  }
}

// In-place exclusive scan of a[0..n) by the whole block; returns the total.
__device__ int block_scan_array(int32_t *a, int n, Sh &sh) {
  int carry = 0;
  for (int base = 0; base < n; base += RB) {
    int i = base + threadIdx.x;
    int v = i < n ? a[i] : 0;
    int tot;
    int ex = block_exclusive_scan<RB>(v, &tot, sh.scan);
    if (i < n) a[i] = carry + ex;
    carry += tot;
  }
  return carry;
}

__device__ int block_sum_int(int v, Sh &sh) {
  int tot;
  block_exclusive_scan<RB>(v, &tot, sh.scan);
  return tot;
}

__device__ long long block_sum_ll(long long v, Sh &sh) {
  long long tot;
  block_exclusive_scan<RB>(v, &tot, sh.lscan);
  return tot;
}

// ---- connected components of the alive vertices ----------------------------
// Hook-and-shortcut rounds: every alive edge (i, j) lowers the label of the
// larger of f[i], f[j] to the smaller one (atomicMin), then every label is
// shortcut to its label's label until stable; rounds repeat until neither
// step changes anything.  Labels only decrease and stay ids of the same
// component, so the fixpoint labels each component with its smallest id.
// f[i] = that id (-1 for dead vertices; f defaults to B); returns the number
// of components.  With emask, only the adjacency entries whose bit is set
// count as edges (an undirected edge may be marked on either of its two
// entries).
template <typename IT>
__device__ __forceinline__ int components(const Mem<IT> &m, int n, Sh &sh, int32_t *f = nullptr,
                          const uint32_t *emask = nullptr) {
  if (f == nullptr) f = m.B;
  volatile int32_t *vf = f;
  for (int i = threadIdx.x; i < n; i += RB) f[i] = m.alive[i] ? i : -1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int round = 0; round <= n; ++round) {
    if (threadIdx.x == 0) sh.changed = 0;
    __syncthreads();
    int changed = 0;
    for (int i = threadIdx.x; i < n; i += RB) {
      if (!m.alive[i]) continue;
      const int b = m.off[i], e = m.off[i + 1];
      if (e - b > 32) continue;
      for (int q = b; q < e; ++q) {
        const int j = m.adj[q];
        if (emask) {
          if (!(emask[q >> 5] & (1u << (q & 31)))) continue;
        } else if (j <= i || !m.alive[j]) {
          continue;
        }
        const int a = vf[i], c = vf[j];
        if (a != c) {
          const int hi = a > c ? a : c, lo = a > c ? c : a;
          if (atomicMin(&f[hi], lo) > lo) changed = 1;
        }
      }
    }
    for (int i = warp; i < n; i += RW) {
      const int b = m.off[i], e = m.off[i + 1];
      if (!m.alive[i] || e - b <= 32) continue;
      for (int q = b + lane; q < e; q += 32) {
        const int j = m.adj[q];
        if (emask) {
          if (!(emask[q >> 5] & (1u << (q & 31)))) continue;
        } else if (j <= i || !m.alive[j]) {
          continue;
        }
        const int a = vf[i], c = vf[j];
        if (a != c) {
          const int hi = a > c ? a : c, lo = a > c ? c : a;
          if (atomicMin(&f[hi], lo) > lo) changed = 1;
        }
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += RB) {
      if (!m.alive[i]) continue;
      int x = vf[i];
      int y = vf[x];
      while (y != x) {
        x = y;
        y = vf[x];
      }
      if (vf[i] != x) {
        vf[i] = x;
        changed = 1;
      }
    }
    if (changed) sh.changed = 1;
    __syncthreads();
    if (!sh.changed) break;
  }
  int roots = 0;
  for (int i = threadIdx.x; i < n; i += RB) roots += (m.alive[i] && f[i] == i);
  return block_sum_int(roots, sh);
}

// ---- connected components (Afforest-style) ---------------------------------
// Union-find over the alive vertices (uf, root = smallest id): every vertex
// first links along its first two alive neighbours, the sets are
// compressed, and then only vertices outside the set of the smallest alive
// vertex process the rest of their rows (an edge with one end in that set is
// seen from its other end; an edge with both ends in it is already inside
// one set).  The result is exactly the connected components, with far fewer
// unions than hooking every edge.  cur is per-vertex scratch.
template <typename IT>
__device__ __forceinline__ void afforest(const Mem<IT> &m, int n, int32_t *uf, int32_t *cur,
                                         Sh &sh) {
  for (int i = threadIdx.x; i < n; i += RB) {
    uf[i] = i;
    cur[i] = m.off[i];
  }
  if (threadIdx.x == 0) sh.i0 = n;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += RB)
    if (m.alive[i]) { atomicMin(&sh.i0, i); break; }
  // sampling: two alive neighbours per vertex
  for (int r = 0; r < 2; ++r) {
    for (int i = threadIdx.x; i < n; i += RB) {
      if (!m.alive[i]) continue;
      const int e = m.off[i + 1];
      int q = cur[i];
      for (; q < e; ++q) {
        const int j = m.adj[q];
        if (m.alive[j]) {
          uf_union(uf, i, j);
          ++q;
          break;
        }
      }
      cur[i] = q;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += RB)
    if (m.alive[i]) uf[i] = uf_find(uf, i);
  __syncthreads();
  const int i0 = sh.i0;
  const int giant = i0 < n ? uf_find(uf, i0) : -1;
  // every vertex outside the giant set processes the rest of its row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < n; i += RB) {
    if (!m.alive[i]) continue;
    const int e = m.off[i + 1];
    if (e - cur[i] > 64 || uf_find(uf, i) == giant) continue;
    for (int q = cur[i]; q < e; ++q) {
      const int j = m.adj[q];
      if (m.alive[j]) uf_union(uf, i, j);
    }
  }
  for (int i = warp; i < n; i += RW) {
    if (!m.alive[i]) continue;
    const int e = m.off[i + 1];
    if (e - cur[i] <= 64 || uf_find(uf, i) == giant) continue;
    for (int q = cur[i] + lane; q < e; q += 32) {
      const int j = m.adj[q];
      if (m.alive[j]) uf_union(uf, i, j);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += RB)
    if (m.alive[i]) uf[i] = uf_find(uf, i);
  __syncthreads();
}

// Connected components of the alive vertices by afforest(): f[i] = smallest
// alive id of i's component (-1 if dead); returns the number of components.
template <typename IT>
__device__ __forceinline__ int components_af(const Mem<IT> &m, int n, int32_t *f, int32_t *cur,
                                             Sh &sh) {
  afforest(m, n, f, cur, sh);
  int roots = 0;
  for (int i = threadIdx.x; i < n; i += RB) {
    if (!m.alive[i]) {
      f[i] = -1;
      continue;
    }
    roots += f[i] == i;
  }
  __syncthreads();
  return block_sum_int(roots, sh);
}

// ---- publishing children -------------------------------------------------
// tag[i] in [0, n) names the child of local vertex i (-1: none).  Every tag
// with at least min_size members becomes a new queue item whose vertex list
// (ascending) is written into the parent's pool range.  Uses C, D, E, F.
// With keep_largest, the kept child with the most members (ties: smallest
// tag) is not published: the caller refines it in place, and the children
// that are published fill the front of the range.  Returns that child's tag
// (-1: none) and, in *emitted, the members published ahead of it.
template <typename IT>
__device__ __forceinline__ int emit_children(const RefineParams &P, const ReqCtx &R,
                                             ReqCtx *Rg, uint16_t req, const Mem<IT> &m,
                                             const int32_t *tag, int n, int64_t vbeg, Sh &sh,
                                             uint16_t cflags = 0, bool keep_largest = false,
                                             int *emitted = nullptr) {
  int32_t *cnt = m.C, *cidx = m.D, *cbase = m.E, *run = m.F;
  for (int t = threadIdx.x; t < n; t += RB) cnt[t] = 0;
  if (threadIdx.x == 0) sh.u1 = 0ull;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += RB)
    if (tag[i] >= 0) atomicAdd(&cnt[tag[i]], 1);
  __syncthreads();
  if (keep_largest) {
    unsigned long long best = 0ull;
    for (int t = threadIdx.x; t < n; t += RB)
      if (cnt[t] >= R.min_size) {
        const unsigned long long pk = ((unsigned long long)cnt[t] << 32) | (unsigned)(0x7fffffff - t);
        best = pk > best ? pk : best;
      }
    if (best) atomicMax(&sh.u1, best);
    __syncthreads();
  }
  const int L = sh.u1 ? 0x7fffffff - (int)(unsigned)(sh.u1 & 0xffffffffull) : -1;
  for (int t = threadIdx.x; t < n; t += RB) {
    bool keep = cnt[t] >= R.min_size && t != L;
    cidx[t] = keep ? 1 : 0;
    cbase[t] = keep ? cnt[t] : 0;
    run[t] = 0;
  }
  __syncthreads();
  int nchild = block_scan_array(cidx, n, sh);
  const int total = block_scan_array(cbase, n, sh);
  if (emitted) *emitted = total;
  if (nchild == 0) return L;
  if (threadIdx.x == 0) {
    add_ll(&Rg->pending, (long long)nchild);
    add_ll(&P.ctr->pending, (long long)nchild);
    __threadfence();
    sh.u0 = atomicAdd(&P.ctr->tail, (unsigned long long)nchild);
  }
  __syncthreads();
  const unsigned long long s0 = sh.u0;
  // members in ascending local order, one warp, 32 at a time
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int b = 0; b < n; b += 32) {
      int i = b + lane;
      int t = i < n ? tag[i] : -1;
      bool kept = t >= 0 && t != L && cnt[t] >= R.min_size;
      int key = kept ? t : -1;
      unsigned peers = __match_any_sync(FULL, key);
      int rank = __popc(peers & lanemask_lt());
      int before = kept ? run[t] : 0;
      __syncwarp();
      if (kept) {
        int pos = before + rank;
        int32_t v = m.gid[i];
        R.pool[vbeg + cbase[t] + pos] = v;
        R.slot[v] = ((unsigned long long)queue_tag(s0 + cidx[t]) << 32) | (unsigned)pos;
        if (rank == 0) run[t] = before + __popc(peers);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  __threadfence();
  // descriptors, then publication
  for (int t = threadIdx.x; t < n; t += RB) {
    if (cnt[t] < R.min_size || t == L) continue;
    unsigned long long q = s0 + cidx[t];
    QSlot *sl = &P.ring[q % P.ring_cap];
    sl->item.vbeg = vbeg + cbase[t];
    sl->item.n = cnt[t];
    sl->item.flags = cflags;
    sl->item.req = req;
  }
  __threadfence();
  __syncthreads();
  for (int t = threadIdx.x; t < n; t += RB) {
    if (cnt[t] < R.min_size || t == L) continue;
    unsigned long long q = s0 + cidx[t];
    atomicExch((unsigned long long *)&P.ring[q % P.ring_cap].seq, q);
  }
  __syncthreads();
  return L;
}

// CM (Algorithm 5): the two sides of a cut split (tag 0 / 1, -1 = not a
// member) with at least min_size members are written to the item's pool
// range in ascending local order, side 0 first, and listed in P.cda for the
// community step, which runs after the kernel; nothing is published.
template <typename IT>
__device__ __forceinline__ void park_sides(const RefineParams &P, const ReqCtx &R, uint16_t req,
                                           const Mem<IT> &m, const int32_t *tag, int n,
                                           int64_t vbeg, Sh &sh) {
  int a0 = 0, a1 = 0;
  for (int i = threadIdx.x; i < n; i += RB) {
    a0 += tag[i] == 0;
    a1 += tag[i] == 1;
  }
  const int c0 = block_sum_int(a0, sh);
  const int c1 = block_sum_int(a1, sh);
  const bool k0 = c0 >= R.min_size, k1 = c1 >= R.min_size;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const unsigned lt = lanemask_lt();
    int r0 = 0, r1 = 0;
    for (int b = 0; b < n; b += 32) {
      const int i = b + lane;
      const int t = i < n ? tag[i] : -1;
      const bool w0 = k0 && t == 0, w1 = k1 && t == 1;
      const unsigned m0 = __ballot_sync(FULL, w0), m1 = __ballot_sync(FULL, w1);
      if (w0) R.pool[vbeg + r0 + __popc(m0 & lt)] = m.gid[i];
      if (w1) R.pool[vbeg + (k0 ? c0 : 0) + r1 + __popc(m1 & lt)] = m.gid[i];
      r0 += __popc(m0);
      r1 += __popc(m1);
    }
  }
  if (threadIdx.x == 0 && (k0 || k1)) {
    const unsigned long long k = (k0 ? 1ull : 0ull) + (k1 ? 1ull : 0ull);
    unsigned long long at = atomicAdd(P.cda_count, k);
    if (at + k > P.cda_cap) {
      atomicOr(&P.ctr->error, DERR_CAPACITY);
    } else {
      if (k0) P.cda[at++] = Item{vbeg, c0, (uint16_t)0, req};
      if (k1) P.cda[at] = Item{vbeg + (k0 ? c0 : 0), c1, (uint16_t)0, req};
    }
  }
  __syncthreads();
}

// Continues an item in place as its child L (the component labelled L in
// tag): every other vertex becomes dead.  Returns the child's size.
template <typename IT>
__device__ __forceinline__ int restrict_alive(const Mem<IT> &m, const int32_t *tag, int L, int n,
                                              Sh &sh) {
  int c = 0;
  for (int i = threadIdx.x; i < n; i += RB) {
    const bool a = m.alive[i] && tag[i] == L;
    m.alive[i] = a;
    c += a;
  }
  return block_sum_int(c, sh);
}

// ---- maximum-adjacency machinery -----------------------------------------
// The current super-vertices are the ids X with grp[X] == X among alive
// vertices.  group_members() counts and lists their members: members of X
// are D[C[X] .. C[X+1]) (C indexed by id), and G[0..nsv) lists the
// super-vertices in ascending order.  Uses C, D, G, H; returns nsv.
template <typename IT>
__device__ __forceinline__ int group_members(const Mem<IT> &m, const int32_t *grp, int n, Sh &sh) {
  int32_t *gof = m.C, *mem = m.D, *svl = m.G, *tmp = m.H;
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i <= n; i += RB) gof[i] = 0;
  __syncthreads();
  // counts and slots are taken once per group present in a warp (large
  // super-vertices would otherwise serialise on one counter)
  for (int base = 0; base < n; base += RB) {
    const int i = base + threadIdx.x;
    const int g = (i < n && m.alive[i]) ? grp[i] : -1;
    const unsigned peers = __match_any_sync(FULL, g);
    if (g >= 0 && lane == __ffs(peers) - 1) atomicAdd(&gof[g], __popc(peers));
  }
  __syncthreads();
  block_scan_array(gof, n + 1, sh);
  for (int i = threadIdx.x; i < n; i += RB) tmp[i] = gof[i];
  __syncthreads();
  for (int base = 0; base < n; base += RB) {
    const int i = base + threadIdx.x;
    const int g = (i < n && m.alive[i]) ? grp[i] : -1;
    const unsigned peers = __match_any_sync(FULL, g);
    const int leader = __ffs(peers) - 1;
    int at = 0;
    if (g >= 0 && lane == leader) at = atomicAdd(&tmp[g], __popc(peers));
    at = __shfl_sync(FULL, at, leader);
    if (g >= 0) mem[at + __popc(peers & lanemask_lt())] = i;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += RB) tmp[i] = (m.alive[i] && grp[i] == i) ? 1 : 0;
  __syncthreads();
  const int nsv = block_scan_array(tmp, n, sh);
  for (int i = threadIdx.x; i < n; i += RB)
    if (m.alive[i] && grp[i] == i) svl[tmp[i]] = i;
  __syncthreads();
  return nsv;
}

__device__ __forceinline__ unsigned long long pack_key(int key, int id) {
  return ((unsigned long long)(unsigned)key << 32) | (unsigned)(~(unsigned)id);
}

// Adds the weights of super-vertex X's edges to every not-yet-added
// neighbour Y: acc[Y] += w(X, Y); each Y reached is listed once in touched.
// Warp 0 only.
template <typename IT>
__device__ __forceinline__ void scan_super_vertex(const Mem<IT> &m, const int32_t *grp, int X,
                                                  Sh &sh) {
  const int lane = threadIdx.x & 31;
  int32_t *acc = m.E, *touched = m.H;
  const int mb = m.C[X], me = m.C[X + 1];
  if (me - mb == 1) {
    const int i = m.D[mb];
    for (int e = m.off[i] + lane; e < m.off[i + 1]; e += 32) {
      const int j = m.adj[e];
      if (!m.alive[j]) continue;
      const int Y = grp[j];
      if (Y == X || m.flag[Y]) continue;
      if (atomicAdd(&acc[Y], 1) == 0) touched[atomicAdd(&sh.ntouched, 1)] = Y;
    }
  } else {
    for (int q = mb + lane; q < me; q += 32) {
      const int i = m.D[q];
      for (int e = m.off[i]; e < m.off[i + 1]; ++e) {
        const int j = m.adj[e];
        if (!m.alive[j]) continue;
        const int Y = grp[j];
        if (Y == X || m.flag[Y]) continue;
        if (atomicAdd(&acc[Y], 1) == 0) touched[atomicAdd(&sh.ntouched, 1)] = Y;
      }
    }
  }
}

// One maximum-adjacency ordering over the current super-vertices with a
// linear argmax, run by warp 0.  kcap > 0: keys capped at kcap and every
// edge X-Y whose key reaches kcap is merged into nrep (a contraction pass);
// kcap == 0: exact keys (a Stoer-Wagner phase), reporting the last two
// super-vertices s, t and the cut of the phase.  Needs group_members() and
// zeroed E (acc), F (key), flag (in A).  touched (H) is reused: the
// grouping's temporaries are dead by then.
template <typename IT>
__device__ __forceinline__ void ma_ordering(const Mem<IT> &m, const int32_t *grp, int32_t *nrep, int nsv,
                            int kcap, Sh &sh) {
  int32_t *acc = m.E, *key = m.F, *touched = m.H, *svl = m.G;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int contracted = 0;
    int s = -1, t = -1, cut = 0;
    if (lane == 0) sh.ntouched = 0;
    __syncwarp();
    for (int step = 0; step < nsv; ++step) {
      unsigned long long best = 0;
      for (int j = lane; j < nsv; j += 32) {
        const int Y = svl[j];
        if (!m.flag[Y]) {
          const unsigned long long v = pack_key(key[Y], Y);
          best = v > best ? v : best;
        }
      }
      best = warp_max(best);
      const int X = (int)(~(unsigned)(best & 0xffffffffu));
      s = t;
      t = X;
      cut = (int)(best >> 32);
      if (lane == 0) m.flag[X] = 1;
      __syncwarp();
      if (step == nsv - 1) break;  // the last super-vertex has no unadded neighbour
      scan_super_vertex(m, grp, X, sh);
      __syncwarp();
      const int nt = sh.ntouched;
      for (int q = lane; q < nt; q += 32) {
        const int Y = touched[q];
        const int a = acc[Y];
        acc[Y] = 0;
        int nk = key[Y] + a;
        if (kcap > 0 && nk >= kcap) {
          nk = kcap;
          uf_union(nrep, X, Y);
          contracted = 1;
        }
        key[Y] = nk;
      }
      __syncwarp();
      if (lane == 0) sh.ntouched = 0;
      __syncwarp();
    }
    contracted = __any_sync(FULL, contracted);
    if (lane == 0) {
      sh.contracted = contracted;
      sh.sw_s = s;
      sh.sw_t = t;
      sh.sw_cut = cut;
    }
  }
  __syncthreads();
}

// Bucket structure: clear levels 0..kcap, put every super-vertex (alive and,
// when grp is given, grp[i] == i) in level 0.  Whole block.
template <typename IT>
__device__ __forceinline__ void buckets_init(const Mem<IT> &m, const int32_t *grp, int n, int kcap) {
  const int W = m.W, S = m.S;
  for (int q = threadIdx.x; q < (kcap + 1) * W; q += RB) m.bm[q] = 0u;
  for (int q = threadIdx.x; q < (kcap + 1) * S; q += RB) m.bms[q] = 0u;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += RB)
    if (m.alive[i] && (grp == nullptr || grp[i] == i)) atomicOr(&m.bm[i >> 5], 1u << (i & 31));
  __syncthreads();
  for (int w = threadIdx.x; w < W; w += RB)
    if (m.bm[w]) atomicOr(&m.bms[w >> 5], 1u << (w & 31));
  __syncthreads();
}

// Warp 0: the not-yet-added super-vertex with the largest key, ties to the
// smallest id = the lowest set bit of the highest non-empty bucket.  Returns
// (level << 24) | id, or -1 if every bucket is empty (a broken invariant).
template <typename IT>
__device__ __forceinline__ int bucket_pick(const Mem<IT> &m, int kcap) {
  const int lane = threadIdx.x & 31;
  const int W = m.W, S = m.S;
  volatile uint32_t *bm = m.bm, *bms = m.bms;
  for (int L = kcap; L >= 0; --L) {
    for (int s0 = 0; s0 < S; s0 += 32) {
      const uint32_t sw = (s0 + lane < S) ? bms[L * S + s0 + lane] : 0u;
      const unsigned b = __ballot_sync(FULL, sw != 0u);
      if (b) {
        const int fl = __ffs(b) - 1;
        const uint32_t swv = __shfl_sync(FULL, sw, fl);
        const int w = (s0 + fl) * 32 + __ffs(swv) - 1;
        const uint32_t word = bm[L * W + w];
        return (L << 24) | (w * 32 + __ffs(word) - 1);
      }
    }
  }
  return -1;
}

// Lane 0: take X out of bucket L.
template <typename IT>
__device__ __forceinline__ void bucket_remove_single(const Mem<IT> &m, int L, int X) {
  const int w = X >> 5;
  const uint32_t nw = m.bm[L * m.W + w] & ~(1u << (X & 31));
  m.bm[L * m.W + w] = nw;
  if (nw == 0u) m.bms[L * m.S + (w >> 5)] &= ~(1u << (w & 31));
}

// Concurrent moves by warp lanes: every lane clears first, then (after
// __syncwarp) sets, so a summary bit is never cleared under a new member.
template <typename IT>
__device__ __forceinline__ void bucket_clear(const Mem<IT> &m, int L, int Y) {
  const uint32_t bit = 1u << (Y & 31);
  const uint32_t r = atomicAnd(&m.bm[L * m.W + (Y >> 5)], ~bit);
  if ((r & ~bit) == 0u) atomicAnd(&m.bms[L * m.S + (Y >> 10)], ~(1u << ((Y >> 5) & 31)));
}
template <typename IT>
__device__ __forceinline__ void bucket_set(const Mem<IT> &m, int L, int Y) {
  atomicOr(&m.bm[L * m.W + (Y >> 5)], 1u << (Y & 31));
  atomicOr(&m.bms[L * m.S + (Y >> 10)], 1u << ((Y >> 5) & 31));
}

// Smallest id > p in level L of the cumulative key bitmaps that is not yet
// added (vis), or -1; warp 0, all lanes.  Levels of more than 64 words are
// searched through their summary bits; with clear set, summary bits whose
// words hold no unadded member are cleared on the way (only when no key
// update can run concurrently).
__device__ __forceinline__ int next_member(volatile uint32_t *bm, volatile uint32_t *bms,
                                           volatile uint32_t *vis, int W, int S, int L, int p,
                                           bool clear) {
  const int lane = threadIdx.x & 31;
  const int p1 = p + 1, w1 = p1 >> 5;
  const uint32_t first_mask = FULL << (p1 & 31);
  if (W <= 64) {
    uint32_t a = 0u, b = 0u;
    if (lane < W && lane >= w1) a = bm[L * W + lane] & ~vis[lane];
    if (lane + 32 < W && lane + 32 >= w1) b = bm[L * W + 32 + lane] & ~vis[32 + lane];
    if (lane == w1) a &= first_mask;
    if (lane + 32 == w1) b &= first_mask;
    const unsigned ba = __ballot_sync(FULL, a != 0u), bb = __ballot_sync(FULL, b != 0u);
    if (!(ba | bb)) return -1;
    const int fl = ba ? __ffs(ba) - 1 : 32 + __ffs(bb) - 1;
    const uint32_t word = __shfl_sync(FULL, fl < 32 ? a : b, fl & 31);
    return fl * 32 + __ffs(word) - 1;
  }
  const int sfirst = w1 >> 5;
  for (int sbase = sfirst & ~31; sbase < S; sbase += 32) {
    const int sidx = sbase + lane;
    uint32_t sw = (sidx < S && sidx >= sfirst) ? bms[L * S + sidx] : 0u;
    if (sidx == sfirst) sw &= FULL << (w1 & 31);
    unsigned bal = __ballot_sync(FULL, sw != 0u);
    while (bal) {
      const int fl = __ffs(bal) - 1;
      const uint32_t swv = __shfl_sync(FULL, sw, fl);
      const int widx = (sbase + fl) * 32 + lane;
      uint32_t wv = ((swv >> lane) & 1u) ? bm[L * W + widx] & ~vis[widx] : 0u;
      if (clear && ((swv >> lane) & 1u) && wv == 0u)
        atomicAnd((uint32_t *)&bms[L * S + sbase + fl], ~(1u << lane));  // no unadded member
      if (widx == w1) wv &= first_mask;
      const unsigned bw = __ballot_sync(FULL, wv != 0u);
      if (bw) {
        const int ll = __ffs(bw) - 1;
        const uint32_t word = __shfl_sync(FULL, wv, ll);
        return ((sbase + fl) * 32 + ll) * 32 + __ffs(word) - 1;
      }
      bal &= bal - 1;
    }
  }
  return -1;
}

// First contraction pass, on the item's own vertices (every super-vertex a
// single vertex, every edge weight 1): the maximum-adjacency ordering with
// keys capped at kcap, ties to the smallest id, run by warp 0.
//
// A key grows by exactly one per step, so the key levels are cumulative
// bitmaps (bit v of level L is set once v's key reaches L) and added
// vertices are masked out by the vis bitmap (in registers, lane l holding
// words l and l+32, when a level has at most 64 words).  With top = the
// largest key of an unadded vertex, the added vertex X is always the
// smallest unadded member of level top, so the next pick is one of: the
// smallest neighbour whose key just rose above top (it alone has the new
// largest key), the smaller of X's successor in level top and the smallest
// neighbour that just reached top, or X's successor -- and only when level
// top runs out is a level searched from scratch.  The successor search
// does not depend on the key updates, so it overlaps them, and one packed
// reduction gives the largest new key with its smallest holder.
//
// The step records only when each vertex was added (pos, F) and when each
// key reached kcap (sat, H); the entry X -> j is contracted iff j was still
// unadded when X was added and its key had reached kcap by then, which the
// whole block evaluates afterwards, merging the ends by union-find.  The
// step is written without lane-divergent branches: lanes without work write
// to per-lane dummy words or store the value every lane stores.  Returns
// whether anything merged; nrep receives the merged sets labelled by their
// smallest id.
template <typename IT>
__device__ __forceinline__ bool ma_pass_first(const RefineParams &P, const Mem<IT> &m, int32_t *nrep,
                                              int n, int nsv, int kcap, int E, unsigned *err,
                                              Sh &sh) {
  const int W = m.W, S = m.S;
  const bool summaries = W > 64;
  uint32_t *vis_w = m.vis;
  int32_t *pos = m.F, *sat = m.H, *ord = m.D;
  uint32_t *sink = sh.sink;  // per-lane dummy targets
  for (int i = threadIdx.x; i < n; i += RB) {
    m.kst[i] = m.alive[i] ? 0 : 255;
    sat[i] = 0x7fffffff;
  }
  for (int q = threadIdx.x; q < (kcap + 1) * W; q += RB) m.bm[q] = q < W ? FULL : 0u;
  for (int q = threadIdx.x; q < (kcap + 1) * S; q += RB) {
    const int nw = W - q * 32;  // level 0: every word has members
    m.bms[q] = q < S ? (nw >= 32 ? FULL : (1u << nw) - 1u) : 0u;
  }
  for (int w = threadIdx.x; w < W; w += RB) {
    uint32_t dead = 0u;  // dead vertices and the padding past n count as added
    for (int b = 0; b < 32; ++b) {
      const int v = w * 32 + b;
      if (v >= n || !m.alive[v]) dead |= 1u << b;
    }
    vis_w[w] = dead;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    volatile uint32_t *bm = m.bm, *bms = m.bms, *vis = vis_w;
    volatile uint8_t *kst = m.kst;
    int top = 0;
    const long long tp0 = P.prof ? clock64() : 0;
    uint32_t va = 0u, vb = 0u;
    if (!summaries) {
      va = lane < W ? (uint32_t)vis[lane] : 0xffffffffu;
      vb = lane + 32 < W ? (uint32_t)vis[32 + lane] : 0xffffffffu;
    }
    int X = next_member(bm, bms, vis, W, S, 0, -1, true);
    if (!summaries) {
      // levels of at most 64 words: lane l reads words l and l+32 (clamped
      // to the last word; the masks drop the clamped copies)
      const int la = lane < W ? lane : W - 1, lb = lane + 32 < W ? lane + 32 : W - 1;
      for (int step = 0; step < nsv; ++step) {
        if (X < 0) {
          if (lane == 0) atomicOr(err, DERR_INTERNAL);
          break;
        }
        pos[X] = step;
        ord[step] = X;
        kst[X] = 255;
        const int xw = X >> 5;
        const uint32_t xb = 1u << (X & 31);
        va |= xw == lane ? xb : 0u;
        vb |= xw == lane + 32 ? xb : 0u;
        if (step == nsv - 1) break;
        const int b = m.off[X], e = m.off[X + 1];
        const uint32_t sa = bm[top * W + la], sb = bm[top * W + lb];
        const int q = b + lane;
        const int jr = (int)m.adj[q < e ? q : b];
        const int j = q < e ? jr : X;
        // successor of X in level top, packed like a key update
        const int p1 = X + 1, w1 = p1 >> 5;
        const uint32_t fm = 0xffffffffu << (p1 & 31);
        uint32_t wa = (lane < W && lane >= w1) ? sa & ~va : 0u;
        uint32_t wb = (lane + 32 < W && lane + 32 >= w1) ? sb & ~vb : 0u;
        wa &= lane == w1 ? fm : 0xffffffffu;
        wb &= lane + 32 == w1 ? fm : 0xffffffffu;
        const int ok = kst[j];
        const unsigned ba = __ballot_sync(FULL, wa != 0u), bb = __ballot_sync(FULL, wb != 0u);
        const int fl = ba ? __ffs(ba) - 1 : 32 + __ffs(bb) - 1;
        const uint32_t word = __shfl_sync(FULL, fl < 32 ? wa : wb, fl & 31);
        const int succ = fl * 32 + __ffs(word) - 1;
        const unsigned ks = (ba | bb) ? ((unsigned)top << 24) | (0xffffffu - (unsigned)succ) : 0u;
        // key update of the first 32 neighbours (ok < kcap: unadded, not capped)
        const bool moved = ok < kcap;
        const int nk = ok + 1;
        kst[moved ? j : X] = moved ? (uint8_t)nk : (uint8_t)255;
        atomicOr(moved ? &m.bm[nk * W + (j >> 5)] : &sink[lane], moved ? 1u << (j & 31) : 0u);
        sat[moved && nk == kcap ? j : n] = step;  // H[n] is spare
        unsigned pk = moved ? ((unsigned)nk << 24) | (0xffffffu - (unsigned)j) : 0u;
        pk = pk > ks ? pk : ks;
        for (int q0 = b + 32; q0 < e; q0 += 32) {  // rows longer than 32 entries
          const int qq = q0 + lane;
          const int jj = qq < e ? (int)m.adj[qq] : X;
          const int o2 = kst[jj];
          const bool mv2 = o2 < kcap;
          const int n2 = o2 + 1;
          kst[mv2 ? jj : X] = mv2 ? (uint8_t)n2 : (uint8_t)255;
          atomicOr(mv2 ? &m.bm[n2 * W + (jj >> 5)] : &sink[lane], mv2 ? 1u << (jj & 31) : 0u);
          sat[mv2 && n2 == kcap ? jj : n] = step;
          const unsigned p2 = mv2 ? ((unsigned)n2 << 24) | (0xffffffu - (unsigned)jj) : 0u;
          pk = p2 > pk ? p2 : pk;
        }
        // the largest key, then the smallest id: the next vertex to add
        pk = __reduce_max_sync(FULL, pk);
        if (pk != 0u && (int)(pk >> 24) >= top) {
          top = (int)(pk >> 24);
          X = (int)(0xffffffu - (pk & 0xffffffu));
        } else {
          // level top has no unadded member left: the highest level that has
          if (lane < W) vis[lane] = va;
          if (lane + 32 < W) vis[32 + lane] = vb;
          __syncwarp();
          X = -1;
          while (top > 0 && X < 0) {
            --top;
            X = next_member(bm, bms, vis, W, S, top, -1, true);
          }
        }
        __syncwarp();
      }
    } else {
      // levels of more than 64 words: the successor is looked for in the 64
      // words from X's on (nearly always there in a dense level), else
      // through the summary bits; added bits are in vis.  The successor is
      // the next vertex about two times in three, so its row bounds and
      // first adjacency chunk are loaded speculatively during the step
      // (rows may sit in the global slab, where each dependent load costs
      // an L2 round trip).
      int pf_x = -1, pf_b = 0, pf_e = 0, pf_j = 0;
      const bool adj_global = __isGlobal(m.adj);
      for (int step = 0; step < nsv; ++step) {
        if (X < 0) {
          if (lane == 0) atomicOr(err, DERR_INTERNAL);
          break;
        }
        pos[X] = step;
        ord[step] = X;
        kst[X] = 255;
        atomicOr(lane == 0 ? &vis_w[X >> 5] : &sink[lane], lane == 0 ? 1u << (X & 31) : 0u);
        {
          // keep the summaries exact: lane L drops X's word from level L's
          // summary when X was its last unadded member there (before this
          // step's key updates, which set any bit they need again)
          const int xw = X >> 5;
          const uint32_t left = lane <= top ? (uint32_t)bm[lane * W + xw] & ~((uint32_t)vis[xw] | (1u << (X & 31))) : 1u;
          atomicAnd(left == 0u ? (uint32_t *)&bms[lane * S + (xw >> 5)] : &sink[lane],
                    left == 0u ? ~(1u << (xw & 31)) : 0xffffffffu);
        }
        if (step == nsv - 1) break;
        const bool hit = X == pf_x;
        const int b = hit ? pf_b : m.off[X], e = hit ? pf_e : m.off[X + 1];
        if (adj_global) {
          // rows of the next ids follow this one in memory, and the next
          // vertex is most often the next id of its level: ask L1 for the
          // lines ahead
          constexpr int PER_LINE = 128 / (int)sizeof(IT);
          const long long qa = (long long)b + (long long)PER_LINE * (lane + 1);
          const IT *pa = m.adj + (qa < E ? qa : E - 1);
          asm volatile("prefetch.global.L1 [%0];" ::"l"(pa));
        }
        const int p1 = X + 1, w1 = p1 >> 5;
        const int ia = w1 + lane, ib = w1 + 32 + lane;
        const uint32_t sa = ia < W ? bm[top * W + ia] : 0u, sb = ib < W ? bm[top * W + ib] : 0u;
        const uint32_t va = ia < W ? (uint32_t)vis[ia] : 0xffffffffu;
        const uint32_t vb = ib < W ? (uint32_t)vis[ib] : 0xffffffffu;
        const int q = b + lane;
        const int jr = hit ? pf_j : (int)m.adj[q < e ? q : b];
        const int j = q < e ? jr : X;
        uint32_t wa = sa & ~va;
        const uint32_t wb = sb & ~vb;
        wa &= lane == 0 ? 0xffffffffu << (p1 & 31) : 0xffffffffu;
        const int ok = kst[j];
        const unsigned ba = __ballot_sync(FULL, wa != 0u), bb = __ballot_sync(FULL, wb != 0u);
        int succ;
        if (ba | bb) {
          const int fl = ba ? __ffs(ba) - 1 : 32 + __ffs(bb) - 1;
          const uint32_t word = __shfl_sync(FULL, fl < 32 ? wa : wb, fl & 31);
          succ = (w1 + fl) * 32 + __ffs(word) - 1;
        } else {
          succ = w1 + 64 < W ? next_member(bm, bms, vis, W, S, top, 32 * (w1 + 64) - 1, false) : -1;
        }
        const unsigned ks = succ >= 0 ? ((unsigned)top << 24) | (0xffffffu - (unsigned)succ) : 0u;
        // speculative row bounds of the successor (used next step if it is picked)
        const int nb = succ >= 0 ? m.off[succ] : 0, ne = succ >= 0 ? m.off[succ + 1] : 0;
        const bool moved = ok < kcap;
        const int nk = ok + 1;
        kst[moved ? j : X] = moved ? (uint8_t)nk : (uint8_t)255;
        atomicOr(moved ? &m.bm[nk * W + (j >> 5)] : &sink[lane], moved ? 1u << (j & 31) : 0u);
        atomicOr(moved ? &m.bms[nk * S + (j >> 10)] : &sink[lane], moved ? 1u << ((j >> 5) & 31) : 0u);
        sat[moved && nk == kcap ? j : n] = step;
        unsigned pk = moved ? ((unsigned)nk << 24) | (0xffffffu - (unsigned)j) : 0u;
        pk = pk > ks ? pk : ks;
        for (int q0 = b + 32; q0 < e; q0 += 32) {  // rows longer than 32 entries
          const int qq = q0 + lane;
          const int jj = qq < e ? (int)m.adj[qq] : X;
          const int o2 = kst[jj];
          const bool mv2 = o2 < kcap;
          const int n2 = o2 + 1;
          kst[mv2 ? jj : X] = mv2 ? (uint8_t)n2 : (uint8_t)255;
          atomicOr(mv2 ? &m.bm[n2 * W + (jj >> 5)] : &sink[lane], mv2 ? 1u << (jj & 31) : 0u);
          atomicOr(mv2 ? &m.bms[n2 * S + (jj >> 10)] : &sink[lane], mv2 ? 1u << ((jj >> 5) & 31) : 0u);
          sat[mv2 && n2 == kcap ? jj : n] = step;
          const unsigned p2 = mv2 ? ((unsigned)n2 << 24) | (0xffffffu - (unsigned)jj) : 0u;
          pk = p2 > pk ? p2 : pk;
        }
        // the successor's first adjacency chunk, issued after this step's own
        // loads so that waiting for its row bounds stalls nothing
        pf_x = succ;
        pf_b = nb;
        pf_e = ne;
        pf_j = succ >= 0 ? (int)m.adj[nb + lane < ne ? nb + lane : nb] : 0;
        pk = __reduce_max_sync(FULL, pk);
        if (pk != 0u && (int)(pk >> 24) >= top) {
          top = (int)(pk >> 24);
          X = (int)(0xffffffu - (pk & 0xffffffu));
        } else {
          // level top has no unadded member left: the highest level that has
          __syncwarp();
          X = -1;
          while (top > 0 && X < 0) {
            --top;
            X = next_member(bm, bms, vis, W, S, top, -1, true);
          }
        }
        __syncwarp();
      }
    }
    if (lane == 0) {
      sh.dbg[0] = P.prof ? clock64() - tp0 : 0;
      sh.dbg[2] = nsv;
    }
  }
  __syncthreads();
  const long long tm0 = P.prof ? clock64() : 0;
  // Merge the ends of every entry a -> j whose key reached kcap while j was
  // still unadded (union-find, root = smallest id), Afforest-style: a vertex
  // whose key reached kcap did so when the vertex added at that step
  // (ord[sat]) scanned it, and that pair is one such entry, so one union per
  // vertex builds most of the structure; then only vertices outside the
  // largest set so formed scan their rows (an edge with both ends inside it
  // adds nothing, and an edge with one end outside is seen from that end).
  // Rows longer than 32 entries are listed for whole warps.
  int32_t *lr = m.C;
  uint8_t *out_g = m.flag;
  for (int i = threadIdx.x; i < n; i += RB) nrep[i] = i;
  if (threadIdx.x == 0) sh.ntouched = 0;
  __syncthreads();
  int any = 0;
  for (int i = threadIdx.x; i < n; i += RB) {
    const int si = sat[i];
    if (si < nsv && m.alive[i]) {
      uf_union(nrep, i, ord[si]);
      any = 1;
    }
  }
  if (!__syncthreads_or(any)) return false;  // no key reached kcap: nothing merges
  for (int i = threadIdx.x; i < n; i += RB)
    if (m.alive[i]) nrep[i] = uf_find(nrep, i);
  __syncthreads();
  if (threadIdx.x < 32) {
    // the root held by most of 32 spread vertices
    const int lane = threadIdx.x;
    const int v = (int)(((long long)lane * n) / 32);
    const int r = m.alive[v] ? nrep[v] : -1;
    const unsigned peers = __match_any_sync(FULL, r);
    const unsigned long long key =
        r >= 0 ? ((unsigned long long)__popc(peers) << 32) | (unsigned)r : 0ull;
    const unsigned long long best = warp_max(key);
    if (lane == 0) sh.i0 = best ? (int)(best & 0xffffffffu) : -1;
  }
  __syncthreads();
  const int giant = sh.i0;
  for (int i = threadIdx.x; i < n; i += RB) out_g[i] = m.alive[i] && nrep[i] != giant;
  __syncthreads();
  auto marked = [&](int v, int u) {  // the edge {v, u} is contracted
    const int pv = pos[v], pu = pos[u];
    return pv < pu ? sat[u] <= pv : sat[v] <= pu;
  };
  for (int v = threadIdx.x; v < n; v += RB) {
    if (!out_g[v]) continue;
    const int b0 = m.off[v], e0 = m.off[v + 1];
    if (e0 - b0 > 32) {
      lr[atomicAdd(&sh.ntouched, 1)] = v;
      continue;
    }
    for (int q = b0; q < e0; ++q) {
      const int u = m.adj[q];
      if (m.alive[u] && marked(v, u)) uf_union(nrep, v, u);
    }
  }
  __syncthreads();
  {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nlr = sh.ntouched;
    for (int k = warp; k < nlr; k += RW) {
      const int v = lr[k];
      for (int q = m.off[v] + lane; q < m.off[v + 1]; q += 32) {
        const int u = m.adj[q];
        if (m.alive[u] && marked(v, u)) uf_union(nrep, v, u);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += RB)
    if (m.alive[i]) nrep[i] = uf_find(nrep, i);
  __syncthreads();
  if (P.prof && threadIdx.x == 0) sh.dbg[1] = clock64() - tm0;
  return true;
}

// The ordering of ma_ordering() with the whole block scanning each added
// super-vertex: for a few large super-vertices (later contraction passes
// and Stoer-Wagner phases after the first pass contracted most edges), where
// one warp walking thousands of member rows would dominate.  Warp 0 picks
// (linear argmax, ties to the smallest id); same contract as ma_ordering().
constexpr int BLOCK_NSV = 64;  // at most this many super-vertices

template <typename IT>
__device__ __forceinline__ void ma_ordering_block(const Mem<IT> &m, const int32_t *grp, int32_t *nrep,
                                                  int nsv, int kcap, Sh &sh) {
  int32_t *acc = m.E, *key = m.F, *touched = m.H, *svl = m.G;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int contracted = 0;
  int s = -1, t = -1, cut = 0;
  if (threadIdx.x == 0) sh.ntouched = 0;
  for (int step = 0; step < nsv; ++step) {
    if (warp == 0) {
      unsigned long long best = 0;
      for (int j = lane; j < nsv; j += 32) {
        const int Y = svl[j];
        if (!m.flag[Y]) {
          const unsigned long long v = pack_key(key[Y], Y);
          best = v > best ? v : best;
        }
      }
      best = warp_max(best);
      if (lane == 0) {
        const int X = (int)(~(unsigned)(best & 0xffffffffu));
        m.flag[X] = 1;
        sh.sw_x = X;
        sh.sw_key = (int)(best >> 32);
      }
    }
    __syncthreads();
    const int X = sh.sw_x;
    s = t;
    t = X;
    cut = sh.sw_key;
    if (step == nsv - 1) break;  // the last super-vertex has no unadded neighbour
    const int mb = m.C[X], me = m.C[X + 1];
    auto visit = [&](int e) {
      const int j = m.adj[e];
      if (!m.alive[j]) return;
      const int Y = grp[j];
      if (Y == X || m.flag[Y]) return;
      if (atomicAdd(&acc[Y], 1) == 0) touched[atomicAdd(&sh.ntouched, 1)] = Y;
    };
    if (me - mb <= RW) {
      // few members: a warp per member, lanes along its row
      for (int q = mb + warp; q < me; q += RW) {
        const int i = m.D[q];
        for (int e = m.off[i] + lane; e < m.off[i + 1]; e += 32) visit(e);
      }
    } else {
      for (int q = mb + threadIdx.x; q < me; q += RB) {
        const int i = m.D[q];
        for (int e = m.off[i]; e < m.off[i + 1]; ++e) visit(e);
      }
    }
    __syncthreads();
    const int nt = sh.ntouched;
    for (int q = threadIdx.x; q < nt; q += RB) {
      const int Y = touched[q];
      const int a = acc[Y];
      acc[Y] = 0;
      int nk = key[Y] + a;
      if (kcap > 0 && nk >= kcap) {
        nk = kcap;
        uf_union(nrep, X, Y);
        contracted = 1;
      }
      key[Y] = nk;
    }
    __syncthreads();
    if (threadIdx.x == 0) sh.ntouched = 0;  // ordered before the next scan by the pick's barrier
  }
  contracted = __syncthreads_or(contracted);
  if (threadIdx.x == 0) {
    sh.contracted = contracted;
    sh.sw_s = s;
    sh.sw_t = t;
    sh.sw_cut = cut;
  }
  __syncthreads();
}

// A later contraction pass (super-vertices with several members, integer
// edge multiplicities) with the key buckets; merges every X-Y whose key
// reaches kcap into nrep.  Same order and result as ma_ordering(kcap).
// Needs group_members() and zeroed E (acc), F (key), flag.
template <typename IT>
__device__ __forceinline__ void ma_pass_bucketed(const Mem<IT> &m, const int32_t *grp, int32_t *nrep, int n,
                                 int nsv, int kcap, unsigned *err, Sh &sh) {
  int32_t *acc = m.E, *key = m.F, *touched = m.H;
  buckets_init(m, grp, n, kcap);
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int contracted = 0;
    if (lane == 0) sh.ntouched = 0;
    __syncwarp();
    for (int step = 0; step < nsv; ++step) {
      const int pk = bucket_pick(m, kcap);
      if (pk < 0) {
        if (lane == 0) atomicOr(err, DERR_INTERNAL);
        break;
      }
      const int L = pk >> 24, X = pk & 0xffffff;
      if (lane == 0) {
        bucket_remove_single(m, L, X);
        m.flag[X] = 1;
      }
      __syncwarp();
      if (step == nsv - 1) break;
      scan_super_vertex(m, grp, X, sh);
      __syncwarp();
      const int nt = sh.ntouched;
      for (int q = lane; q < nt; q += 32) {
        const int Y = touched[q];
        const int a = acc[Y];
        acc[Y] = 0;
        const int ok = key[Y];
        int nk = ok + a;
        if (nk >= kcap) {
          nk = kcap;
          uf_union(nrep, X, Y);
          contracted = 1;
        }
        if (nk != ok) {
          bucket_clear(m, ok, Y);
          key[Y] = nk;
        } else {
          touched[q] = -1 - Y;  // no move needed
        }
      }
      __syncwarp();
      for (int q = lane; q < nt; q += 32) {
        const int Y = touched[q];
        if (Y >= 0) bucket_set(m, key[Y], Y);
      }
      __syncwarp();
      if (lane == 0) sh.ntouched = 0;
      __syncwarp();
    }
    contracted = __any_sync(FULL, contracted);
    if (lane == 0) sh.contracted = contracted;
  }
  __syncthreads();
}

// ---- few super-vertices: a dense finish ---------------------------------------
// With at most 32 super-vertices left (indexed in ascending order of their
// smallest member, so index order is id order), their integer edge weights
// fit a small matrix w[nsv][nsv] and one warp runs the remaining capped
// contraction passes and the Stoer-Wagner phases on it, lane l holding
// super-vertex l, with exactly the rules of the sparse passes: largest key,
// ties to the smallest id; in a capped pass every X-Y whose key reaches kcap
// when X is added merges (survivor: the smaller id); a phase's cut is the key
// of the last super-vertex t, the earliest minimum is kept, its side is t's
// members, and t merges into the one added before it.
constexpr int DENSE_NSV = 32;  // one lane per super-vertex
static_assert(DENSE_NSV <= 32, "the dense finish keeps one super-vertex per lane");

// Adds row and column l of w into r (r < l), zeroes r's diagonal.  Warp 0.
__device__ __forceinline__ void dense_fold(int32_t *w, int nsv, int r, int l) {
  const int c = threadIdx.x & 31;
  if (c < nsv) w[r * nsv + c] += w[l * nsv + c];
  __syncwarp();
  if (c < nsv) w[c * nsv + r] += w[c * nsv + l];
  __syncwarp();
  if (c == 0) w[r * nsv + r] = 0;
  __syncwarp();
}

// One maximum-adjacency ordering over the live indices (mask live); kcap > 0
// caps keys and records merges in duf; kcap == 0 reports s, t and the cut.
__device__ __forceinline__ void dense_order(const int32_t *w, int nsv, uint32_t live, int kcap,
                                            int32_t *duf, int &s, int &t, int &cut, bool &merged) {
  const int l = threadIdx.x & 31;
  long long key = 0;
  bool added = !((live >> l) & 1u);
  const int cnt = __popc(live);
  s = t = -1;
  cut = 0;
  merged = false;
  for (int step = 0; step < cnt; ++step) {
    // largest key, ties to the smallest index
    const unsigned long long pk =
        added ? 0ull : (((unsigned long long)key << 6) | (unsigned long long)(63 - l)) + 1ull;
    unsigned long long best = pk;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long x = __shfl_xor_sync(FULL, best, o);
      best = x > best ? x : best;
    }
    const int X = 63 - (int)((best - 1ull) & 63ull);
    s = t;
    t = X;
    cut = (int)((best - 1ull) >> 6);
    added |= l == X;
    const int wx = l < nsv ? w[X * nsv + l] : 0;
    if (!added && wx > 0) {
      long long nk = key + wx;
      if (kcap > 0 && nk >= kcap) {
        nk = kcap;
        // merge l into X's set (duf links point to smaller indices)
        volatile int32_t *vd = duf;
        int a = X, b = l;
        for (;;) {
          while (vd[a] != a) a = vd[a];
          while (vd[b] != b) b = vd[b];
          if (a == b) break;
          if (a > b) { const int tt = a; a = b; b = tt; }
          if (atomicCAS(&duf[b], b, a) == b) break;
        }
        merged = true;
      }
      key = nk;
    }
    __syncwarp();
  }
  merged = __any_sync(FULL, merged);
}

struct DenseResult {
  int cut;        // minimum cut, or -1 when the contraction left one super-vertex
  uint32_t side;  // the minimum cut's side (mask of initial indices)
  int passes, phases;
};

// Runs the dense finish on w (nsv <= 32 indices; the super-vertices are the
// indices in live0) with one warp (any warp; all its lanes call).  duf: 32
// ints of scratch.  Every lane returns the result.
__device__ DenseResult dense_finish(int32_t *w, int nsv, uint32_t live0, int kcap, int32_t *duf) {
  const int l = threadIdx.x & 31;
  uint32_t live = live0;
  uint32_t mem = 1u << l;  // lane l: the initial indices it holds
  int passes = 0, phases = 0;
  bool more = true;
  while (more && __popc(live) > 1) {
    duf[l] = l;
    __syncwarp();
    int s, t, cut;
    bool merged;
    dense_order(w, nsv, live, kcap, duf, s, t, cut, merged);
    ++passes;
    more = merged;
    if (!merged) break;
    // fold every merged index into its root, in ascending order
    volatile int32_t *vd = duf;
    for (int x = 0; x < nsv; ++x) {
      if (!((live >> x) & 1u)) continue;
      int r = x;
      while (vd[r] != r) r = vd[r];
      if (r == x) continue;
      dense_fold(w, nsv, r, x);
      const uint32_t mx = __shfl_sync(FULL, mem, x);
      if (l == r) mem |= mx;
      live &= ~(1u << x);
    }
  }
  DenseResult res{-1, 0u, passes, 0};
  while (__popc(live) > 1) {
    int s, t, cut;
    bool merged;
    dense_order(w, nsv, live, 0, duf, s, t, cut, merged);
    ++phases;
    if (res.cut < 0 || cut < res.cut) {
      res.cut = cut;
      res.side = __shfl_sync(FULL, mem, t);
    }
    const int lo = s < t ? s : t, hi = s < t ? t : s;
    dense_fold(w, nsv, lo, hi);
    const uint32_t mh = __shfl_sync(FULL, mem, hi);
    if (l == lo) mem |= mh;
    live &= ~(1u << hi);
  }
  res.phases = phases;
  __syncwarp();
  return res;
}

// The same dense finish for up to DENSE_WIDE_NSV super-vertices: lane l
// holds indices l, l+32, ... (K per lane); the merged sets are tracked in
// grp[initial index] = the index that holds it now, and the minimum cut's
// side is returned as a mask of initial indices (side[j], bit l = index
// l + 32 j).  Same rules, same results, as dense_finish.
constexpr int DENSE_WIDE_NSV = 128;

template <int K>
__device__ __forceinline__ bool dw_live(const uint32_t (&live)[K], int x) {
  bool r = false;
#pragma unroll
  for (int j = 0; j < K; ++j) r = (x >> 5) == j ? ((live[j] >> (x & 31)) & 1u) != 0u : r;
  return r;
}

template <int K>
__device__ __forceinline__ void dw_kill(uint32_t (&live)[K], int x) {
#pragma unroll
  for (int j = 0; j < K; ++j)
    if ((x >> 5) == j) live[j] &= ~(1u << (x & 31));
}

// Adds row and column x of w into r (r < x), zeroes r's diagonal, moves
// x's members to r.  One warp.
template <int K>
__device__ __forceinline__ void dense_fold_w(int32_t *w, int nsv, int r, int x, int32_t *grp) {
  const int c = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int cc = c + 32 * j;
    if (cc < nsv) w[r * nsv + cc] += w[x * nsv + cc];
  }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int cc = c + 32 * j;
    if (cc < nsv) {
      w[cc * nsv + r] += w[cc * nsv + x];
      if (grp[cc] == x) grp[cc] = r;
    }
  }
  __syncwarp();
  if (c == 0) w[r * nsv + r] = 0;
  __syncwarp();
}

template <int K>
__device__ __forceinline__ void dense_order_w(const int32_t *w, int nsv, const uint32_t (&live)[K],
                                              int kcap, int32_t *duf, int &s, int &t, int &cut,
                                              bool &merged) {
  const int l = threadIdx.x & 31;
  long long key[K];
  bool added[K];
  int cnt = 0;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    key[j] = 0;
    added[j] = !((live[j] >> l) & 1u);
    cnt += __popc(live[j]);
  }
  s = t = -1;
  cut = 0;
  merged = false;
  for (int step = 0; step < cnt; ++step) {
    // largest key, ties to the smallest index
    unsigned long long best = 0ull;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const unsigned long long pk =
          added[j] ? 0ull
                   : (((unsigned long long)key[j] << 7) | (unsigned long long)(127 - (l + 32 * j))) + 1ull;
      best = pk > best ? pk : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long x = __shfl_xor_sync(FULL, best, o);
      best = x > best ? x : best;
    }
    const int X = 127 - (int)((best - 1ull) & 127ull);
    s = t;
    t = X;
    cut = (int)((best - 1ull) >> 7);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int idx = l + 32 * j;
      added[j] |= idx == X;
      const int wx = idx < nsv ? w[X * nsv + idx] : 0;
      if (!added[j] && wx > 0) {
        long long nk = key[j] + wx;
        if (kcap > 0 && nk >= kcap) {
          nk = kcap;
          volatile int32_t *vd = duf;
          int a = X, b = idx;
          for (;;) {
            while (vd[a] != a) a = vd[a];
            while (vd[b] != b) b = vd[b];
            if (a == b) break;
            if (a > b) { const int tt = a; a = b; b = tt; }
            if (atomicCAS(&duf[b], b, a) == b) break;
          }
          merged = true;
        }
        key[j] = nk;
      }
    }
    __syncwarp();
  }
  merged = __any_sync(FULL, merged);
}

// The live indices are live0[j] (bit l = index l + 32 j) or, with live0
// NULL, all of 0..nsv-1; a dead index has zero weights.  duf, grp: nsv ints
// each; side: K words.
template <int K>
__device__ DenseResult dense_finish_w(int32_t *w, int nsv, int kcap, int32_t *duf, int32_t *grp,
                                      uint32_t *side, const uint32_t *live0 = nullptr) {
  const int l = threadIdx.x & 31;
  uint32_t live[K];
  int nlive = 0;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int b = 32 * j;
    live[j] = nsv >= b + 32 ? FULL : (nsv > b ? (1u << (nsv - b)) - 1u : 0u);
    if (live0) live[j] &= live0[j];
    nlive += __popc(live[j]);
    if (l + b < nsv) grp[l + b] = l + b;
  }
  __syncwarp();
  int passes = 0, phases = 0;
  while (nlive > 1) {
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (l + 32 * j < nsv) duf[l + 32 * j] = l + 32 * j;
    __syncwarp();
    int s, t, cut;
    bool merged;
    dense_order_w<K>(w, nsv, live, kcap, duf, s, t, cut, merged);
    ++passes;
    if (!merged) break;
    // fold every merged index into its root, in ascending order
    volatile int32_t *vd = duf;
    for (int x = 0; x < nsv; ++x) {
      if (!dw_live<K>(live, x)) continue;
      int r = x;
      while (vd[r] != r) r = vd[r];
      if (r == x) continue;
      dense_fold_w<K>(w, nsv, r, x, grp);
      dw_kill<K>(live, x);
      --nlive;
    }
  }
  DenseResult res{-1, 0u, passes, 0};
  while (nlive > 1) {
    int s, t, cut;
    bool merged;
    dense_order_w<K>(w, nsv, live, 0, duf, s, t, cut, merged);
    ++phases;
    if (res.cut < 0 || cut < res.cut) {
      res.cut = cut;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const unsigned b = __ballot_sync(FULL, l + 32 * j < nsv && grp[l + 32 * j] == t);
        if (l == 0) side[j] = b;
      }
    }
    const int lo = s < t ? s : t, hi = s < t ? t : s;
    dense_fold_w<K>(w, nsv, lo, hi, grp);
    dw_kill<K>(live, hi);
    --nlive;
  }
  res.phases = phases;
  __syncwarp();
  return res;
}

// Exact acceptance test for lambda >= kcap by forest certificates.  Take
// kcap-1 edge-disjoint spanning forests, each maximal in the edges the earlier
// ones left.  An edge (u, v) in none of them has u and v joined by a path in
// every forest (else that forest could have taken it) and by itself: kcap
// edge-disjoint paths, so lambda(u, v) >= kcap and contracting u, v keeps
// every cut below kcap (the sparse-certificate argument of Nagamochi and
// Ibaraki).  Rounds repeat on the contracted multigraph (a super-vertex is
// labelled by its smallest member; parallel edges stay separate copies).  One
// super-vertex left certifies lambda >= kcap; that is exactly the item's
// acceptance, whichever contraction reached it, so the result is the one the
// canonical passes give.  When few super-vertices are left, the dense
// finish's capped passes decide on their weight matrix (they keep every cut
// below kcap as well).  A super-vertex of degree below kcap (lambda < kcap),
// a round that contracts nothing, too many super-vertices after the last
// round, or a failing dense check gives up and the canonical passes decide.
//
// Each forest is one pass of union-find links over the unused edges (each
// undirected edge once, from its smaller end): the edges whose link joined
// two sets form a spanning forest of them, and it is maximal.  The
// union-find array lives in shared memory when the item leaves room.
// Returns the rounds taken (> 0: certified) or minus the rounds tried.
// Uses C, D, E, G, H, ebits (and wide for the dense check).
constexpr int FOREST_MAX_K = 16;       // at most 15 forests a round
constexpr int FOREST_ROUNDS = 4;
constexpr int FOREST_LONG_ROW = 32;    // rows longer than this go to a whole warp

// Calls f(a, q, b) for every adjacency entry q = (a -> b) of every alive
// vertex a with sel(a): rows up to FOREST_LONG_ROW entries by one thread,
// longer rows (listed in lr[0..nlr)) by a whole warp.
template <typename IT, typename Sel, typename F>
__device__ __forceinline__ void rows_pass(const Mem<IT> &m, int n, const int32_t *lr, int nlr,
                                          Sel sel, F f) {
  for (int a = threadIdx.x; a < n; a += RB) {
    if (!m.alive[a]) continue;
    const int b0 = m.off[a], e0 = m.off[a + 1];
    if (e0 - b0 > FOREST_LONG_ROW || !sel(a)) continue;
    for (int q = b0; q < e0; ++q) f(a, q, (int)m.adj[q]);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = warp; k < nlr; k += RW) {
    const int a = lr[k];
    if (!sel(a)) continue;
    for (int q = m.off[a] + lane; q < m.off[a + 1]; q += 32) f(a, q, (int)m.adj[q]);
  }
}

template <typename IT>
__device__ __forceinline__ int forest_accept(const Mem<IT> &m, int n, int kcap, int32_t *cf, Sh &sh,
                                             bool prof) {
  long long tc = prof ? clock64() : 0;
  auto lap = [&](int k) {  // profile: cycles since the last lap into fdbg[k]
    if (prof) {
      const long long t = clock64();
      if (threadIdx.x == 0) sh.fdbg[k] += t - tc;
      tc = t;
    }
  };
  int32_t *lr = m.D, *rep = m.G, *deg = m.H;
  uint32_t *used = m.ebits;
  volatile uint32_t *vu = used;
  const int E = m.off[n];
  if (threadIdx.x == 0) sh.ntouched = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += RB) {
    rep[i] = m.alive[i] ? i : -1;
    if (m.alive[i] && m.off[i + 1] - m.off[i] > FOREST_LONG_ROW) lr[atomicAdd(&sh.ntouched, 1)] = i;
  }
  __syncthreads();
  const int nlr = sh.ntouched;
  auto all = [](int) { return true; };
  auto is_used = [&](int q) { return (vu[q >> 5] >> (q & 31)) & 1u; };
  int nroots = 0;
  for (int round = 1; round <= FOREST_ROUNDS; ++round) {
    if (round > 1) {
      // a super-vertex with fewer than kcap edges to the others is a cut
      // below kcap: the item fails, the canonical passes find its cut
      for (int i = threadIdx.x; i < n; i += RB) deg[i] = 0;
      __syncthreads();
      rows_pass(m, n, lr, nlr, all, [&](int a, int q, int b) {
        const int A = rep[a], B = rep[b];
        if (B >= 0 && B != A) atomicAdd(&deg[A], 1);
      });
      __syncthreads();
      int low = 0;
      for (int i = threadIdx.x; i < n; i += RB) low |= rep[i] == i && deg[i] < kcap;
      if (__syncthreads_or(low)) return -round;
      lap(4);
    }
    for (int q = threadIdx.x; q < (E + 31) / 32; q += RB) used[q] = 0u;
    for (int f = 1; f < kcap; ++f) {
      for (int i = threadIdx.x; i < n; i += RB) cf[i] = i;
      __syncthreads();
      rows_pass(m, n, lr, nlr, all, [&](int a, int q, int b) {
        if (b < a) return;  // each undirected edge once
        const int A = rep[a], B = rep[b];
        if (B < 0 || B == A || is_used(q)) return;
        if (uf_link(cf, A, B)) atomicOr(&used[q >> 5], 1u << (q & 31));
      });
      __syncthreads();
      if (prof && threadIdx.x == 0) sh.fdbg[1] += 1;
      lap(0);
    }
    for (int i = threadIdx.x; i < n; i += RB) cf[i] = i;
    __syncthreads();
    int merged = 0;
    rows_pass(m, n, lr, nlr, all, [&](int a, int q, int b) {
      if (b < a) return;
      const int A = rep[a], B = rep[b];
      if (B < 0 || B == A || is_used(q)) return;
      merged |= uf_link(cf, A, B);
    });
    if (!__syncthreads_or(merged)) return -round;
    lap(2);
    int roots = 0;
    for (int i = threadIdx.x; i < n; i += RB) {
      const int r = rep[i];
      if (r >= 0) {
        const int nr = uf_find(cf, r);
        rep[i] = nr;
        roots += nr == i;
      }
    }
    nroots = block_sum_int(roots, sh);
    lap(5);
    if (nroots == 1) return round;
    if (nroots <= DENSE_WIDE_NSV && nroots * nroots <= 2 * (n + 1)) {
      // few super-vertices: the dense finish's capped passes decide
      int32_t *idx = m.C, *rank = m.H;
      int32_t *w = reinterpret_cast<int32_t *>(m.wide);
      for (int i = threadIdx.x; i < n; i += RB) rank[i] = (rep[i] == i) ? 1 : 0;
      for (int q = threadIdx.x; q < nroots * nroots; q += RB) w[q] = 0;
      __syncthreads();
      block_scan_array(rank, n, sh);
      for (int i = threadIdx.x; i < n; i += RB)
        if (rep[i] == i) idx[i] = rank[i];
      __syncthreads();
      rows_pass(m, n, lr, nlr, all, [&](int a, int q, int b) {
        const int A = rep[a], B = rep[b];
        if (B >= 0 && B != A) atomicAdd(&w[idx[A] * nroots + idx[B]], 1);
      });
      __syncthreads();
      if (threadIdx.x < 32) {
        DenseResult dr;
        if (nroots <= DENSE_NSV)
          dr = dense_finish(w, nroots, nroots >= 32 ? 0xffffffffu : (1u << nroots) - 1u, kcap,
                            sh.duf);
        else if (nroots <= 64)
          dr = dense_finish_w<2>(w, nroots, kcap, sh.wduf, sh.wgrp, sh.wside);
        else
          dr = dense_finish_w<4>(w, nroots, kcap, sh.wduf, sh.wgrp, sh.wside);
        if (threadIdx.x == 0) sh.dcut = dr.cut;
      }
      __syncthreads();
      lap(3);
      return sh.dcut < 0 ? round : -round;
    }
  }
  return -FOREST_ROUNDS;
}

template <typename IT>
__device__ __forceinline__ void reset_ma_state(const Mem<IT> &m, int n) {
  for (int i = threadIdx.x; i < n; i += RB) {
    m.E[i] = 0;
    m.F[i] = 0;
    m.flag[i] = 0;
  }
  __syncthreads();
}

// ---- items of at most 64 vertices: one warp each ---------------------------------
// A CTA that claims such an item claims up to RW-1 more at once and gives
// every small one to a warp of its own (larger ones run on the whole CTA
// afterwards).  With n <= 32 R (R = 1 or 2 rows per lane) the induced
// subgraph is a bit matrix: lane l holds the rows of members l and l + 32 as
// bitmasks over local ids, components grow by OR-reductions of rows, the
// peel is a popcount, and the contraction passes and Stoer-Wagner phases are
// the dense finish on the same matrix -- the same steps and rules as the CTA
// path, in registers.  The parts an item splits into (components, the two
// sides of its cut) are subsets of the same matrix, so the warp refines
// them itself, one after the other, instead of queueing them: each part is
// the same child item (its vertex set alone decides its outcome, and the
// local ids keep their order), only without its own claim and extraction.
constexpr int TINY_MAX = 64;

template <int R>
struct TinyMask;
template <>
struct TinyMask<1> { using T = uint32_t; };
template <>
struct TinyMask<2> { using T = unsigned long long; };

// Scratch of one warp, in ints: weights (32R)^2, union-find and merged sets
// (2 x 32R), the part stack (32 masks of R words), row bits (32R masks),
// the degree prefix (32R) and the cut side (4).
template <int R>
__host__ __device__ constexpr size_t tiny_scratch_ints() {
  return (size_t)(32 * R) * (32 * R) + 2 * (32 * R) + 32 * R + (32 * R) * R + 32 * R + 4;
}
constexpr size_t TINY_SCRATCH = 4 * tiny_scratch_ints<2>();     // items of up to 64 vertices
constexpr size_t TINY_SCRATCH_32 = 4 * tiny_scratch_ints<1>();  // up to 32
static_assert(TINY_SCRATCH % 8 == 0 && TINY_SCRATCH_32 % 8 == 0, "mask arrays stay aligned");

__device__ __forceinline__ uint32_t warp_or(uint32_t x) { return __reduce_or_sync(FULL, x); }
__device__ __forceinline__ unsigned long long warp_or(unsigned long long x) {
  const uint32_t lo = __reduce_or_sync(FULL, (uint32_t)x);
  const uint32_t hi = __reduce_or_sync(FULL, (uint32_t)(x >> 32));
  return ((unsigned long long)hi << 32) | lo;
}
__device__ __forceinline__ int popc_m(uint32_t x) { return __popc(x); }
__device__ __forceinline__ int popc_m(unsigned long long x) { return __popcll(x); }
__device__ __forceinline__ int ffs_m(uint32_t x) { return __ffs(x); }
__device__ __forceinline__ int ffs_m(unsigned long long x) { return __ffsll((long long)x); }

template <int R, typename M>
__device__ __forceinline__ M tiny_component(const M (&row)[R], M set, int start) {
  const int l = threadIdx.x & 31;
  M V = (M)1 << start, F = V;
  for (;;) {
    M acc = 0;
#pragma unroll
    for (int j = 0; j < R; ++j)
      if ((F >> (l + 32 * j)) & 1u) acc |= row[j];
    const M nx = warp_or(acc) & set & ~V;
    if (!nx) return V;
    V |= nx;
    F = nx;
  }
}

// Pushes every component of set (with at least min_size members) onto the
// part stack stk[0..*sp).  Returns the number of components.
template <int R, typename M>
__device__ __forceinline__ int tiny_push_components(const M (&row)[R], M set, int min_size, M *stk,
                                                    int &sp) {
  int k = 0;
  M rem = set;
  while (rem) {
    const M c = tiny_component<R, M>(row, set, ffs_m(rem) - 1);
    if ((threadIdx.x & 31) == 0 && popc_m(c) >= min_size) stk[sp] = c;
    sp += popc_m(c) >= min_size ? 1 : 0;
    ++k;
    rem &= ~c;
  }
  __syncwarp();
  return k;
}

// Returns false, having done nothing, when the members' degree sum exceeds
// P.tiny_max_deg (a hub's row would keep one warp busy while its CTA waits).
template <int R>
__device__ bool tiny_item_body(const RefineParams &P, unsigned long long seq, const Item &it,
                               int32_t *scratch) {
  using M = typename TinyMask<R>::T;
  constexpr int NV = 32 * R;  // vertices a warp holds
  const int l = threadIdx.x & 31;
  const int n = it.n;
  ReqCtx *Rg = &P.reqs[it.req];
  const ReqCtx Rc = load_ctx(Rg);
  int32_t *w = scratch, *duf = scratch + NV * NV, *grp = duf + NV;
  M *stk = reinterpret_cast<M *>(grp + NV);
  M *rbits = stk + 32;
  int32_t *pre = reinterpret_cast<int32_t *>(rbits + NV);
  uint32_t *wside = reinterpret_cast<uint32_t *>(pre + NV);
  int32_t v[R];
  int64_t rb[R];
  int len[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int i = l + 32 * j;
    v[j] = i < n ? __ldcg(&Rc.pool[it.vbeg + i]) : -1;
    rb[j] = i < n ? Rc.off[v[j]] : 0;
    len[j] = i < n ? (int)(Rc.off[v[j] + 1] - rb[j]) : 0;
  }
  int D = 0;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int inc = warp_inclusive_scan(len[j]) + D;
    pre[l + 32 * j] = inc;
    D = __shfl_sync(FULL, inc, 31);
  }
  if (D > P.tiny_max_deg) return false;
  const uint32_t tag = queue_tag(seq);
  // 1. extraction, flat over the D adjacency entries of the members: lane l
  // takes entries l, l+32, ..., eight at a time (eight neighbour loads, then
  // eight slot gathers in flight); entry f belongs to the row whose degree
  // prefix first exceeds f, and a hit sets that row's bit in shared memory
#pragma unroll
  for (int j = 0; j < R; ++j) rbits[l + 32 * j] = 0;
  __syncwarp();
  constexpr int Q = 8;
  for (int f0 = 0; f0 < D; f0 += 32 * Q) {
    int32_t u[Q];
    int rr[Q];
#pragma unroll
    for (int z = 0; z < Q; ++z) {
      const int f = f0 + 32 * z + l;
      int lo = 0, hi = NV - 1;  // smallest r with pre[r] > f
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] > f) hi = mid; else lo = mid + 1;
      }
      rr[z] = f < D ? lo : -1;
    }
#pragma unroll
    for (int z = 0; z < Q; ++z) {
      const int r = rr[z] < 0 ? 0 : rr[z];
      int64_t br = __shfl_sync(FULL, rb[0], r & 31);
      int lr = __shfl_sync(FULL, len[0], r & 31);
      if (R == 2) {
        const int64_t b1 = __shfl_sync(FULL, rb[R - 1], r & 31);
        const int l1 = __shfl_sync(FULL, len[R - 1], r & 31);
        if (r >= 32) { br = b1; lr = l1; }
      }
      const int sr = pre[r] - lr;
      u[z] = rr[z] >= 0 ? Rc.adj[br + (f0 + 32 * z + l - sr)] : -1;
    }
    unsigned long long sl[Q];
#pragma unroll
    for (int z = 0; z < Q; ++z) sl[z] = u[z] >= 0 ? __ldcg(&Rc.slot[u[z]]) : 0ull;
#pragma unroll
    for (int z = 0; z < Q; ++z)
      if (u[z] >= 0 && (unsigned)(sl[z] >> 32) == tag)
        atomicOr(&rbits[rr[z]], (M)1 << (unsigned)(sl[z] & 0xffffffffu));
  }
  __syncwarp();
  M row[R];
#pragma unroll
  for (int j = 0; j < R; ++j) row[j] = l + 32 * j < n ? rbits[l + 32 * j] : (M)0;
  // statistics of the whole subtree, added once at the end (lane 0)
  long long st_items = 1, st_peeled = 0, st_passes = 0, st_phases = 0, st_acc = 0, st_splits = 0;
  bool failed = false;
  const M all = n >= NV ? ~(M)0 : (((M)1 << n) - 1);
  int sp = 0;
  bool whole = true;  // the item itself is refined as it is
  // 2. input cluster: CCR (Algorithm 1); when it splits, its components are
  // the parts
  if (it.flags & ITEM_TOP) {
    const int k = tiny_push_components<R, M>(row, all, Rc.min_size, stk, sp);
    if (k == 1) sp = 0;
    else whole = false;
  }
  M set = all;
  for (;;) {
    if (!whole) {
      if (sp == 0) break;
      set = stk[--sp];
      st_items += 1;
    }
    whole = false;
    __syncwarp();
    const int nset = popc_m(set);
    // 3. peel, round-synchronous, T from the alive count
    M cur = set;
    for (;;) {
      const int64_t T = threshold_of(Rc.rule_kind, Rc.rule_num, Rc.rule_den, popc_m(cur));
      M rm = 0;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const bool r = ((cur >> (l + 32 * j)) & 1u) && popc_m(row[j] & cur) <= T;
        rm |= (M)__ballot_sync(FULL, r) << (32 * j);
      }
      if (!rm) break;
      cur &= ~rm;
    }
    const int nal = popc_m(cur);
    st_peeled += nset - nal;
    if (nal < Rc.min_size) continue;
    // 4. connectivity of what is left (only a peel can disconnect it)
    if (nal < nset) {
      const int sp0 = sp;
      const int k = tiny_push_components<R, M>(row, cur, Rc.min_size, stk, sp);
      if (k > 1) continue;
      sp = sp0;  // one component: refine it as it is
    }
    // 5-6. contraction with k = T+1, then canonical Stoer-Wagner: the dense
    // finish on the part's own vertices (index = local id)
    const int64_t T = threshold_of(Rc.rule_kind, Rc.rule_num, Rc.rule_den, nal);
    const int kcap = (int)(T + 1 < (1ll << 30) ? T + 1 : (1ll << 30));
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int i = l + 32 * j;
      const M rw = ((cur >> i) & 1u) ? row[j] & cur : (M)0;
#pragma unroll 8
      for (int b = 0; b < NV; ++b) w[i * NV + b] = (int32_t)((rw >> b) & 1u);
    }
    __syncwarp();
    DenseResult dr;
    M side;
    if (R == 1) {
      dr = dense_finish(w, 32, (uint32_t)cur, kcap, duf);
      side = (M)dr.side;
    } else {
      uint32_t live0[2] = {(uint32_t)cur, (uint32_t)((unsigned long long)cur >> 32)};
      dr = dense_finish_w<2>(w, NV, kcap, duf, grp, wside, live0);
      __syncwarp();
      side = (M)wside[0] | ((M)wside[R - 1] << (32 * (R - 1)));
    }
    st_passes += dr.passes;
    st_phases += dr.phases;
    if (dr.cut < 0) {
      // accept (Algorithm 3: save V_c); output id resolved after the run
      const int i0 = ffs_m(cur) - 1;
      int32_t minv = __shfl_sync(FULL, v[0], i0 & 31);
      if (R == 2) {
        const int32_t m1 = __shfl_sync(FULL, v[R - 1], i0 & 31);
        if (i0 >= 32) minv = m1;
      }
#pragma unroll
      for (int j = 0; j < R; ++j)
        if ((cur >> (l + 32 * j)) & 1u) Rc.label_min[v[j]] = minv;
      st_acc += 1;
      continue;
    }
    if (dr.cut > T) {
      failed = true;
      break;
    }
    // Algorithm 3: bisect on the minimum cut; both sides are parts
    st_splits += 1;
    const M s0 = cur & ~side, s1 = cur & side;
    if (l == 0) {
      int q = sp;
      if (popc_m(s0) >= Rc.min_size) stk[q++] = s0;
      if (popc_m(s1) >= Rc.min_size) stk[q++] = s1;
    }
    sp += (popc_m(s0) >= Rc.min_size ? 1 : 0) + (popc_m(s1) >= Rc.min_size ? 1 : 0);
    __syncwarp();
  }
  if (l == 0) {
    if (failed) atomicOr(&P.ctr->error, DERR_INTERNAL);
    add_ll(&Rg->items, st_items);
    add_ll(&Rg->alg_bytes, ((it.flags & ITEM_TOP) ? 8ll * n : 0ll) + 8ll * D);
    if (st_peeled) add_ll(&Rg->peeled, st_peeled);
    if (st_passes) add_ll(&Rg->ni_passes, st_passes);
    if (st_phases) add_ll(&Rg->sw_phases, st_phases);
    if (st_acc) add_ll(&Rg->accepted, st_acc);
    if (st_splits) add_ll(&Rg->splits, st_splits);
  }
  return true;
}

// tiny_item_body, recorded in the per-item profile when it is enabled
// (outcome 100, no phase split).
__device__ __forceinline__ bool tiny_item_any(const RefineParams &P, unsigned long long seq,
                                              const Item &it, int32_t *scratch) {
  return it.n <= 32 ? tiny_item_body<1>(P, seq, it, scratch)
                    : tiny_item_body<2>(P, seq, it, scratch);
}

__device__ __forceinline__ bool tiny_item(const RefineParams &P, unsigned long long seq,
                                          const Item &it, int32_t *scratch) {
  if (!P.prof) return tiny_item_any(P, seq, it, scratch);
  const long long t0 = (long long)globaltimer_ns();
  const bool done = tiny_item_any(P, seq, it, scratch);
  __syncwarp();
  if ((threadIdx.x & 31) == 0 && done) {
    const unsigned r = atomicAdd(P.prof_count, 1u);
    if (r < P.prof_cap) {
      ItemProf *q = &P.prof[r];
      q->seq = (unsigned)seq;
      q->n = it.n;
      q->E = q->nalive = q->passes = q->nsv = -1;
      q->outcome = 100;
      unsigned smid;
      asm("mov.u32 %0, %%smid;" : "=r"(smid));
      q->smid = (int)smid;
      q->slab = 0;
      q->top = (int)(it.flags & ITEM_TOP);
      for (int z = 0; z < 8; ++z) q->dt[z] = 0;
      q->t_begin = t0;
      q->t_end = (long long)globaltimer_ns();
      for (int z = 0; z < 4; ++z) q->dbg[z] = 0;
      q->forest = q->nsv1 = 0;
      q->forest_cycles = 0;
      for (int z = 0; z < 6; ++z) q->fdbg[z] = 0;
    }
  }
  return done;
}

// The end of an item: the request's and the run's pending counts drop (the
// request's last item raises its host-mapped done flag).  One thread.
__device__ __forceinline__ void finish_item(const RefineParams &P, uint16_t req) {
  __threadfence();
  ReqCtx &R = P.reqs[req];
  const unsigned long long left =
      atomicAdd(reinterpret_cast<unsigned long long *>(&R.pending), ~0ull);  // -1
  if (left == 1ull && P.done_flags) {
    // the request's last item: everything it wrote is visible first
    __threadfence_system();
    ((volatile int *)P.done_flags)[req] = 1;
  }
  add_ll(&P.ctr->pending, -1ll);
}

// ---- one work item ---------------------------------------------------------
template <typename IT, bool SM>
__device__ __noinline__ int process_item(const RefineParams &P, unsigned long long seq,
                                         const Item &it, char *slab, int64_t dbound, Sh &sh) {
  char *base = SM ? wcc_dyn_smem : slab;
  const int n = it.n;
  const int64_t vbeg = it.vbeg;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  ReqCtx *Rg = &P.reqs[it.req];
  const ReqCtx R = load_ctx(Rg);
  ReqCtx *ctr = Rg;  // per-request statistics (atomics)
  Mem<IT> m = carve<IT>(base, n, dbound);
  if (SM) m.smem_used = ws_bytes<IT>(n, dbound);
  if (!SM) {
    const int64_t T0 = threshold_of(R.rule_kind, R.rule_num, R.rule_den, n);
    carve_hot(m, n, (int)(T0 + 2 < KB_LEVELS ? T0 + 2 : KB_LEVELS), P.smem_bytes);
  }

  // global row start and degree of every member
  int64_t *gbeg = m.wide;
  int32_t *pdeg = m.C, *cnt = m.D;
  for (int i = threadIdx.x; i < n; i += RB) {
    const int32_t v = __ldcg(&R.pool[vbeg + i]);
    m.gid[i] = v;
    const int64_t b = R.off[v];
    gbeg[i] = b;
    pdeg[i] = (int32_t)(R.off[v + 1] - b);
    cnt[i] = 0;
  }
  __syncthreads();
  const int D = block_scan_array(pdeg, n, sh);
  if (threadIdx.x == 0) pdeg[n] = D;
  __syncthreads();
  prof_stamp(P, sh, 1);

  // 1. extraction, flat over all D adjacency entries of the members so that
  // every thread keeps independent loads in flight: entry f of row i keeps
  // its neighbour u iff slot[u] names this item; tmp[f] = local id or ~0
  IT *tmp = m.adj;
  const IT NONE = (IT)~(IT)0;
  if (!SM) {
    // items in the global slab: their row bounds are global too, so a
    // per-entry row cursor would put a dependent global load on every
    // entry; instead each warp takes two rows at a time, reads their bounds
    // once, and its lanes walk the rows together (64 neighbour loads and 64
    // slot gathers in flight per warp)
    for (int r0 = 2 * warp; r0 < n; r0 += 2 * RW) {
      const int r1 = r0 + 1 < n ? r0 + 1 : r0;
      const int o0 = pdeg[r0], d0 = pdeg[r0 + 1] - o0;
      const int o1 = pdeg[r1], d1 = r1 != r0 ? pdeg[r1 + 1] - o1 : 0;
      const int64_t g0 = gbeg[r0], g1 = gbeg[r1];
      int c0 = 0, c1 = 0;
      const int dm = d0 > d1 ? d0 : d1;
      for (int k = lane; k - lane < dm; k += 32) {
        const bool a0 = k < d0, a1 = k < d1;
        const int32_t u0 = a0 ? R.adj[g0 + k] : 0;
        const int32_t u1 = a1 ? R.adj[g1 + k] : 0;
        const unsigned long long s0 = a0 ? __ldcg(&R.slot[u0]) : 0ull;
        const unsigned long long s1 = a1 ? __ldcg(&R.slot[u1]) : 0ull;
        const bool h0 = a0 && (unsigned)(s0 >> 32) == queue_tag(seq);
        const bool h1 = a1 && (unsigned)(s1 >> 32) == queue_tag(seq);
        if (a0) tmp[o0 + k] = h0 ? (IT)(unsigned)(s0 & 0xffffffffu) : NONE;
        if (a1) tmp[o1 + k] = h1 ? (IT)(unsigned)(s1 & 0xffffffffu) : NONE;
        c0 += __popc(__ballot_sync(FULL, h0));
        c1 += __popc(__ballot_sync(FULL, h1));
      }
      if (lane == 0) {
        cnt[r0] = c0;
        if (r1 != r0) cnt[r1] = c1;
      }
    }
  } else {
    // warp w owns entries [w*chunk, (w+1)*chunk); lane l takes every 32nd
    // entry of it, four at a time, following its row with a cursor
    const int chunk = (D + RW - 1) / RW;
    const int f0 = warp * chunk, f1 = min(D, f0 + chunk);
    int row = 0;
    if (f0 + lane < f1) {
      int lo = 0, hi = n;  // largest i with pdeg[i] <= f0 + lane
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pdeg[mid] <= f0 + lane) lo = mid; else hi = mid;
      }
      row = lo;
    }
    for (int fb = f0 + lane; fb < f1; fb += 128) {
      int fs[4], rs[4];
      int32_t us[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int f = fb + 32 * k;
        fs[k] = f;
        if (f < f1) {
          while (pdeg[row + 1] <= f) ++row;
          rs[k] = row;
          us[k] = R.adj[gbeg[row] + (f - pdeg[row])];
        }
      }
      unsigned long long sl[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) sl[k] = fs[k] < f1 ? __ldcg(&R.slot[us[k]]) : 0ull;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (fs[k] >= f1) continue;
        const bool hit = (unsigned)(sl[k] >> 32) == queue_tag(seq);
        tmp[fs[k]] = hit ? (IT)(unsigned)(sl[k] & 0xffffffffu) : NONE;
        if (hit) atomicAdd(&cnt[rs[k]], 1);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += RB) m.off[i] = cnt[i];
  __syncthreads();
  const int E = block_scan_array(m.off, n, sh);
  if (threadIdx.x == 0) m.off[n] = E;
  // order-preserving compaction of tmp into the local adjacency, in chunks
  // read fully into registers before any write (destinations never pass the
  // chunk's own sources)
  {
    constexpr int CI = 4;
    int carry = 0;
    for (int c0 = 0; c0 < D; c0 += RB * CI) {
      IT v[CI];
      int k = 0;
#pragma unroll
      for (int q = 0; q < CI; ++q) {
        const int f = c0 + threadIdx.x * CI + q;
        v[q] = f < D ? tmp[f] : NONE;
        k += v[q] != NONE;
      }
      int tot;
      int ex = block_exclusive_scan<RB>(k, &tot, sh.scan);
      int w = carry + ex;
#pragma unroll
      for (int q = 0; q < CI; ++q)
        if (v[q] != NONE) m.adj[w++] = v[q];
      carry += tot;
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += RB) m.alive[i] = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    add_ll(&ctr->items, 1ll);
    // algorithmic bytes of the extraction: an input cluster reads its
    // members' row offsets (8 B) and, per adjacency entry, the neighbour id
    // and its label (4 + 4 B); re-inducing a part after a split reads the
    // entries again (8 B each)
    add_ll(&ctr->alg_bytes, (long long)((it.flags & ITEM_TOP) ? 8 * n : 0) + 8 * (long long)D);
    sh.pf_E = E;
  }
  prof_stamp(P, sh, 2);

  // The item's vertices are the alive ones.  When it splits into components,
  // the largest one with at least min_size vertices is not queued: this CTA
  // continues with it in place (its induced subgraph is already here; it is
  // the same child item, only without waiting behind the queue), and its
  // later children go to the pool range vb behind the published ones.
  int nalive = n;
  int64_t vb = vbeg;

  // 2. input cluster: CCR (Algorithm 1)
  if (it.flags & ITEM_TOP) {
    int nc = components_af(m, n, m.B, m.H, sh);
    if (nc != 1) {
      int emitted = 0;
      const int L = emit_children(P, R, Rg, it.req, m, m.B, n, vb, sh, 0, true, &emitted);
      if (L < 0) return OUT_CCR_SPLIT;
      nalive = restrict_alive(m, m.B, L, n, sh);
      vb += emitted;
      if (threadIdx.x == 0) add_ll(&ctr->items, 1ll);
    }
  }
  prof_stamp(P, sh, 3);

  // 3. peel (round-synchronous, T recomputed from the alive count)
  int32_t *deg = m.A;
  for (int i = threadIdx.x; i < n; i += RB) deg[i] = m.off[i + 1] - m.off[i];
  __syncthreads();
  const int n_item = nalive;
  for (;;) {
    const int64_t T = threshold_of(R.rule_kind, R.rule_num, R.rule_den, nalive);
    int rem = 0;
    for (int i = threadIdx.x; i < n; i += RB) {
      bool r = m.alive[i] && deg[i] <= T;
      m.flag[i] = r;
      rem += r;
    }
    rem = block_sum_int(rem, sh);
    if (rem == 0) break;
    for (int i = warp; i < n; i += RW) {
      if (!m.flag[i]) continue;
      for (int e = m.off[i] + lane; e < m.off[i + 1]; e += 32) atomicSub(&deg[m.adj[e]], 1);
      if (lane == 0) m.alive[i] = 0;
    }
    __syncthreads();
    nalive -= rem;
  }
  if (threadIdx.x == 0) {
    if (nalive < n_item) add_ll(&ctr->peeled, (long long)(n_item - nalive));
    sh.pf_nalive = nalive;
  }
  prof_stamp(P, sh, 4);
  if (nalive < R.min_size) return OUT_DROPPED;

  // 4. connectivity of what is left (an item arrives connected: input
  // clusters passed CCR above, children are components or sides of a
  // minimum cut, which are connected; only a peel can disconnect it).  The
  // component continued in place needs no peel of its own: T only grows
  // with n, so every vertex left already has degree > T of its smaller size.
  if (nalive < n_item) {
    int nc = components_af(m, n, m.B, m.H, sh);
    if (nc > 1) {
      int emitted = 0;
      const int L = emit_children(P, R, Rg, it.req, m, m.B, n, vb, sh, 0, true, &emitted);
      if (L < 0) return OUT_CC_SPLIT;
      nalive = restrict_alive(m, m.B, L, n, sh);
      vb += emitted;
      if (threadIdx.x == 0) add_ll(&ctr->items, 1ll);
    }
  }
  prof_stamp(P, sh, 5);

  // 5. contraction with k = T+1
  const int64_t T = threshold_of(R.rule_kind, R.rule_num, R.rule_den, nalive);
  const int kcap = (int)(T + 1 < (1ll << 30) ? T + 1 : (1ll << 30));
  int32_t *rep = m.A, *nrep = m.B;
  int nsv = 1, passes = 0;
  int dense_cut = -1;  // >= 0: the dense finish found the cut (side in m.side)
  bool certified = false;
  bool inh_valid = false;  // R.inh holds this item's first-pass records
  if (kcap <= FOREST_MAX_K && P.forest_min_n > 0 && nalive >= P.forest_min_n) {
    const long long f0 = P.prof ? clock64() : 0;
    // the forests' union-find: in shared memory for an item in the global
    // slab when its row offsets did not move there (the first pass's state
    // there is set up only later)
    int32_t *cf = m.B;
    if (!SM && !m.off_in_smem && 4 * (size_t)n <= P.smem_bytes)
      cf = reinterpret_cast<int32_t *>(wcc_dyn_smem);
    const int fr = forest_accept(m, n, kcap, cf, sh, P.prof != nullptr);
    certified = fr > 0;
    if (P.prof && threadIdx.x == 0) {
      sh.pf_forest = fr;
      sh.pf_forest_cycles = clock64() - f0;
    }
  }
  if (!certified) {
    nsv = nalive;
    bool more = true;
    const bool bucketed = kcap < KB_LEVELS && n < (1 << 24);  // pick packs the id in 24 bits
    if (bucketed) {
      if (threadIdx.x == 0) add_ll(&ctr->ni_passes, 1ll);
      ++passes;
      // A side S of a parent's cut (value <= T) whose members are the first
      // |S| vertices of the parent's first-pass order, with the same kcap
      // and nothing peeled here, would run exactly that order's prefix: at
      // every step of it the parent took the unvisited vertex of largest
      // capped key, smallest id, and before the order left S no vertex
      // outside S had been added, so S's keys and saturation steps are the
      // same in the induced subgraph.  No entry between S and the other
      // side is contracted (its far end would have kcap > T neighbours in
      // S, across a cut of at most T), so the parent's first-pass sets on S
      // are this item's.  Their roots are taken from the records instead of
      // repeating the pass; any record that does not fit falls back to it.
      bool inherited = false;
      if ((it.flags & ITEM_INH) && R.inh != nullptr && nalive == n) {
        int bad = 0;
        for (int i = threadIdx.x; i < n; i += RB) {
          const unsigned long long rec = __ldcg(&R.inh[m.gid[i]]);
          const int kc = (int)(rec >> 56), p = (int)((rec >> 32) & 0xffffffu);
          const long long r = (long long)(uint32_t)rec;
          int loc = -1;
          if (kc == kcap && p < n && r < R.n_vertices) {
            const unsigned long long sr = __ldcg(&R.slot[r]);
            if ((unsigned)(sr >> 32) == queue_tag(seq)) loc = (int)(unsigned)(sr & 0xffffffffu);
          }
          if (loc < 0 || loc > i) bad = 1;  // a root is the smallest member of its set
          rep[i] = loc;
        }
        if (!__syncthreads_or(bad)) {
          for (int i = threadIdx.x; i < n; i += RB)
            if (rep[rep[i]] != rep[i]) bad = 1;
          inherited = !__syncthreads_or(bad);
        }
      }
      int r1 = 0;
      if (inherited) {
        for (int i = threadIdx.x; i < n; i += RB) r1 += rep[i] == i;
        nsv = block_sum_int(r1, sh);
        more = nsv < nalive;  // the pass contracted something
        inh_valid = true;
      } else {
        const bool any = ma_pass_first(P, m, nrep, n, nalive, kcap, E, &P.ctr->error, sh);
        // this pass's records, for the sides of a later cut (position in
        // m.F, root as a vertex id)
        const bool rec = R.inh != nullptr && nalive >= INH_MIN_N;
        const int32_t *pos = m.F;
        for (int i = threadIdx.x; i < n; i += RB) {
          const int r = m.alive[i] ? (any ? nrep[i] : i) : -1;
          rep[i] = r;
          r1 += r == i;
          if (rec && r >= 0)
            R.inh[m.gid[i]] = ((unsigned long long)kcap << 56) |
                              ((unsigned long long)(unsigned)pos[i] << 32) | (unsigned)m.gid[r];
        }
        nsv = block_sum_int(r1, sh);
        more = any;
        inh_valid = rec;
      }
      if (P.prof && threadIdx.x == 0) sh.pf_nsv1 = nsv;
    } else {
      for (int i = threadIdx.x; i < n; i += RB) rep[i] = m.alive[i] ? i : -1;
      __syncthreads();
    }
    const long long tl0 = P.prof ? clock64() : 0;
    // the weight matrix of the dense finish: in E..F when it fits, else in
    // the dynamic shared memory past what the item occupies
    int32_t *wmat = nullptr;
    if (nsv * nsv <= 2 * (n + 1)) {
      wmat = reinterpret_cast<int32_t *>(m.wide);
    } else {
      const size_t at = align16(m.smem_used);
      if (at + 4 * (size_t)nsv * (size_t)nsv <= P.smem_bytes)
        wmat = reinterpret_cast<int32_t *>(wcc_dyn_smem + at);
    }
    if (bucketed && more && nsv > 1 && nsv <= P.dense_max && nsv <= DENSE_WIDE_NSV &&
        wmat != nullptr) {
      // few super-vertices left: their weight matrix, then the dense finish
      int32_t *idx = m.C, *lr = m.D, *rank = m.H;
      int32_t *w = wmat;
      for (int i = threadIdx.x; i < n; i += RB) rank[i] = (m.alive[i] && rep[i] == i) ? 1 : 0;
      for (int q = threadIdx.x; q < nsv * nsv; q += RB) w[q] = 0;
      if (threadIdx.x == 0) sh.ntouched = 0;
      __syncthreads();
      block_scan_array(rank, n, sh);
      for (int i = threadIdx.x; i < n; i += RB)
        if (m.alive[i] && rep[i] == i) idx[i] = rank[i];
      __syncthreads();
      // every entry between two super-vertices (each edge from both ends)
      for (int a = threadIdx.x; a < n; a += RB) {
        if (!m.alive[a]) continue;
        const int b0 = m.off[a], e0 = m.off[a + 1];
        if (e0 - b0 > 32) {
          lr[atomicAdd(&sh.ntouched, 1)] = a;
          continue;
        }
        const int A = idx[rep[a]];
        for (int q = b0; q < e0; ++q) {
          const int r = rep[m.adj[q]];
          if (r < 0) continue;
          const int B = idx[r];
          if (B != A) atomicAdd(&w[A * nsv + B], 1);
        }
      }
      __syncthreads();
      {
        const int nl = sh.ntouched;
        for (int k = warp; k < nl; k += RW) {
          const int a = lr[k], A = idx[rep[a]];
          for (int q = m.off[a] + lane; q < m.off[a + 1]; q += 32) {
            const int r = rep[m.adj[q]];
            if (r < 0) continue;
            const int B = idx[r];
            if (B != A) atomicAdd(&w[A * nsv + B], 1);
          }
        }
      }
      __syncthreads();
      if (threadIdx.x < 32) {
        DenseResult dr;
        if (nsv <= DENSE_NSV) {
          dr = dense_finish(w, nsv, nsv >= 32 ? 0xffffffffu : (1u << nsv) - 1u, kcap, sh.duf);
          if (threadIdx.x == 0) sh.wside[0] = dr.side;
        } else if (nsv <= 64) {
          dr = dense_finish_w<2>(w, nsv, kcap, sh.wduf, sh.wgrp, sh.wside);
        } else {
          dr = dense_finish_w<4>(w, nsv, kcap, sh.wduf, sh.wgrp, sh.wside);
        }
        if (threadIdx.x == 0) {
          sh.dcut = dr.cut;
          sh.dside = dr.side;
          sh.dpasses = dr.passes;
          sh.dphases = dr.phases;
        }
      }
      __syncthreads();
      passes += sh.dpasses;
      if (threadIdx.x == 0) {
        add_ll(&ctr->ni_passes, (long long)sh.dpasses);
        add_ll(&ctr->sw_phases, (long long)sh.dphases);
      }
      if (sh.dcut < 0) {
        nsv = 1;
      } else {
        dense_cut = sh.dcut;
        for (int i = threadIdx.x; i < n; i += RB) {
          const int k = m.alive[i] ? idx[rep[i]] : 0;
          m.side[i] = m.alive[i] && ((sh.wside[k >> 5] >> (k & 31)) & 1u);
        }
        __syncthreads();
      }
      more = false;
    }
    while (more && nsv > 1) {
      nsv = group_members(m, rep, n, sh);
      reset_ma_state(m, n);
      for (int i = threadIdx.x; i < n; i += RB) nrep[i] = i;
      __syncthreads();
      if (threadIdx.x == 0) add_ll(&ctr->ni_passes, 1ll);
      ++passes;
      if (nsv <= BLOCK_NSV)
        ma_ordering_block(m, rep, nrep, nsv, kcap, sh);
      else if (bucketed)
        ma_pass_bucketed(m, rep, nrep, n, nsv, kcap, &P.ctr->error, sh);
      else
        ma_ordering(m, rep, nrep, nsv, kcap, sh);
      if (!sh.contracted) break;
      int roots = 0;
      for (int i = threadIdx.x; i < n; i += RB) {
        if (!m.alive[i]) continue;
        const int r = uf_find(nrep, rep[i]);
        rep[i] = r;
        roots += r == i;
      }
      nsv = block_sum_int(roots, sh);
    }
    if (P.prof && threadIdx.x == 0) sh.dbg[3] = clock64() - tl0;
  }
  if (threadIdx.x == 0) {
    sh.pf_passes = passes;
    sh.pf_nsv = nsv;
  }
  prof_stamp(P, sh, 6);
  if (nsv <= 1) {
    // accept (Algorithm 3: save V_c); output id resolved after the run
    if (threadIdx.x == 0) sh.i0 = n;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += RB)
      if (m.alive[i]) { atomicMin(&sh.i0, i); break; }
    __syncthreads();
    const int32_t minv = m.gid[sh.i0];
    for (int i = threadIdx.x; i < n; i += RB)
      if (m.alive[i]) R.label_min[m.gid[i]] = minv;
    if (threadIdx.x == 0) add_ll(&ctr->accepted, 1ll);
    __syncthreads();
    return OUT_ACCEPT;
  }

  // 6. canonical Stoer-Wagner on the contracted graph; grp = A (starts as rep)
  if (dense_cut >= 0) {
    if (dense_cut > T) {
      if (threadIdx.x == 0) atomicOr(&P.ctr->error, DERR_INTERNAL);
      return OUT_ERROR;
    }
  } else {
    int32_t *grp = m.A;
    int best = 0x7fffffff;
    while (nsv > 1) {
      group_members(m, grp, n, sh);
      reset_ma_state(m, n);
      if (threadIdx.x == 0) add_ll(&ctr->sw_phases, 1ll);
      if (nsv <= BLOCK_NSV)
        ma_ordering_block(m, grp, (int32_t *)nullptr, nsv, 0, sh);
      else
        ma_ordering(m, grp, (int32_t *)nullptr, nsv, 0, sh);
      const int s = sh.sw_s, t = sh.sw_t, cut = sh.sw_cut;
      if (cut < best) {
        best = cut;
        for (int i = threadIdx.x; i < n; i += RB) m.side[i] = m.alive[i] && grp[i] == t;
      }
      __syncthreads();
      const int lo = s < t ? s : t, hi = s < t ? t : s;
      for (int i = threadIdx.x; i < n; i += RB)
        if (m.alive[i] && grp[i] == hi) grp[i] = lo;
      __syncthreads();
      --nsv;
    }
    prof_stamp(P, sh, 7);
    if (best > T) {
      if (threadIdx.x == 0) atomicOr(&P.ctr->error, DERR_INTERNAL);
      return OUT_ERROR;
    }
  }
  if (threadIdx.x == 0) add_ll(&ctr->splits, 1ll);
  for (int i = threadIdx.x; i < n; i += RB) m.B[i] = m.alive[i] ? (m.side[i] ? 1 : 0) : -1;
  __syncthreads();
  if (P.cm)
    park_sides(P, R, it.req, m, m.B, n, vb, sh);
  else
    emit_children(P, R, Rg, it.req, m, m.B, n, vb, sh, inh_valid ? ITEM_INH : (uint16_t)0);
  return OUT_CUT_SPLIT;
}

// Chooses the local id width and the memory (shared or the CTA's slab) for
// an item, then processes it.
__device__ int run_item(const RefineParams &P, unsigned long long seq, const Item &it, char *slab,
                        Sh &sh) {
  const int n = it.n;
  const ReqCtx R = load_ctx(&P.reqs[it.req]);
  long long dsum = 0;
  for (int i = threadIdx.x; i < n; i += RB) {
    const int32_t v = __ldcg(&R.pool[it.vbeg + i]);
    dsum += R.off[v + 1] - R.off[v];
  }
  dsum = block_sum_ll(dsum, sh);
  const bool narrow = n < 65535;
  const size_t need = narrow ? ws_bytes<uint16_t>(n, dsum) : ws_bytes<int32_t>(n, dsum);
  const bool in_smem = need <= P.smem_bytes;
  if (!in_smem && (need > P.slab_bytes || dsum >= (1ll << 31))) {
    if (threadIdx.x == 0) {
      atomicOr(&P.ctr->error, DERR_CAPACITY);
      atomicExch(&P.ctr->err_info, (unsigned)n);
    }
    return OUT_ERROR;
  }
  if (threadIdx.x == 0) sh.used_slab = !in_smem;
  if (in_smem)
    return narrow ? process_item<uint16_t, true>(P, seq, it, slab, dsum, sh)
                  : process_item<int32_t, true>(P, seq, it, slab, dsum, sh);
  return narrow ? process_item<uint16_t, false>(P, seq, it, slab, dsum, sh)
                : process_item<int32_t, false>(P, seq, it, slab, dsum, sh);
}

// Waits (bounded) for queue index q to be published and reads its item
// with two 8-byte loads.  False, with DERR_TIMEOUT set, when the wait runs
// out or the run has failed meanwhile.
static_assert(offsetof(Item, vbeg) == 0 && offsetof(Item, n) == 8 && offsetof(Item, flags) == 12 &&
                  offsetof(Item, req) == 14 && sizeof(Item) == 16,
              "an item is read as two 8-byte words");
__device__ __forceinline__ bool fetch_item(const RefineParams &P, unsigned long long q, Item &out) {
  QSlot *sl = &P.ring[q % P.ring_cap];
  volatile RunCounters *vctr = P.ctr;
  const uint64_t t1 = globaltimer_ns();
  unsigned ns2 = 32;
  for (;;) {
    if (*(volatile unsigned long long *)&sl->seq == q) break;
    if (vctr->error != 0 || globaltimer_ns() - t1 > P.wait_limit_ns) {
      atomicOr(&P.ctr->error, DERR_TIMEOUT);
      return false;
    }
    __nanosleep(ns2);
    ns2 = ns2 < 1024 ? ns2 * 2 : ns2;
  }
  __threadfence();
  const volatile unsigned long long *w = reinterpret_cast<const volatile unsigned long long *>(&sl->item);
  const unsigned long long a = w[0], b = w[1];
  out.vbeg = (int64_t)a;
  out.n = (int32_t)(uint32_t)b;
  out.flags = (uint16_t)(b >> 32);
  out.req = (uint16_t)(b >> 48);
  return true;
}

// ---- the persistent kernel ---------------------------------------------------
// Thread 0 claims a queue index only when one has been reserved (head <
// tail), by compare-and-swap, and then waits -- bounded by wait_limit_ns --
// for its publication.  With nothing reserved it waits for more: the kernel
// ends when nothing is pending and the queue is closed, or (open, serving)
// once one CTA has found nothing pending for idle_limit_ns and set closing;
// a wait for work that is pending but never published ends at wait_limit_ns
// with DERR_TIMEOUT.
__global__ void __launch_bounds__(RB, 1) k_refine(RefineParams P) {
  __shared__ Sh sh;
  char *slab = P.slab + (size_t)blockIdx.x * P.slab_bytes;
  RunCounters *ctr = P.ctr;
  volatile RunCounters *vctr = ctr;
  // items of up to 64 vertices on single warps when the scratch of eight
  // warps fits the shared memory, else up to 32, else none
  int tiny_lim = P.tiny_max;
  if (tiny_lim > 32 && P.smem_bytes < (size_t)RW * TINY_SCRATCH) tiny_lim = 32;
  if (tiny_lim > 0 && P.smem_bytes < (size_t)RW * TINY_SCRATCH_32) tiny_lim = 0;
  const size_t tiny_scr = tiny_lim > 32 ? TINY_SCRATCH : TINY_SCRATCH_32;
  const bool tiny_ok = tiny_lim > 0;
  bool took = false;  // thread 0: this CTA has claimed an item in this launch
  CtaProf cp{0, 0, 0, 0, 0, 0, 0};  // thread 0, profile only
  long long pc = P.prof ? clock64() : 0;
  for (;;) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      if (lane == 0 && P.tickets) {
        // A closed run (nothing is added from outside while it runs) claims
        // its first item by ticket: a fetch-and-add on the head never fails,
        // so the CTAs do not contend on a compare-and-swap.  Ticket j is an
        // item once it is reserved (j < tail); while it is not, the CTA
        // waits for it, holding no other work, and leaves once nothing is
        // pending (no item in flight could reserve it any more: an
        // unfinished reserved index keeps pending above zero).
        int go = 0;
        const unsigned long long j = atomicAdd(&ctr->head, 1ull);
        const uint64_t t0 = globaltimer_ns();
        unsigned ns = 32;
        for (;;) {
          if (vctr->error != 0) break;
          if (j < vctr->tail) {
            go = 1;
            break;
          }
          if (vctr->pending <= 0) break;
          if (globaltimer_ns() - t0 > P.wait_limit_ns) {
            atomicOr(&ctr->error, DERR_TIMEOUT);
            break;
          }
          __nanosleep(ns);
          ns = ns < 4096 ? ns * 2 : ns;
        }
        if (go && !fetch_item(P, j, sh.batch[0])) go = 0;
        sh.bseq[0] = j;
        // a small input cluster: the block after it (see below)
        int k = 0;
        unsigned long long hb = 0;
        if (go && tiny_ok && sh.batch[0].n <= tiny_lim && (sh.batch[0].flags & ITEM_TOP)) {
          const unsigned long long send = __ldcg(&P.reqs[sh.batch[0].req].seed_end);
          for (int tries = 0; tries < 4; ++tries) {
            const unsigned long long h = vctr->head, t = vctr->tail;
            const unsigned long long lim = t < send ? t : send;
            if (h >= lim) break;
            const int kk = (int)min((unsigned long long)(RW - 1), lim - h);
            if (atomicCAS(&ctr->head, h, h + kk) == h) {
              k = kk;
              hb = h;
              break;
            }
          }
        }
        sh.claim_h = hb;
        sh.claim_k = k;
        sh.go = go;
      } else if (lane == 0) {
        int go = 0;
        unsigned long long j = 0;
        const uint64_t t0 = globaltimer_ns();
        unsigned ns = 32;
        for (;;) {
          if (vctr->error != 0) break;
          if (P.single_item) {
            j = P.single_index;
            go = 1;
            break;
          }
          // a job step whose time is up: leave at this item boundary (the
          // queue keeps everything not yet claimed).  A CTA takes one item
          // before it looks, so that every step makes progress.
          if (P.stop_flag && took && *P.stop_flag) break;
          const unsigned long long h = vctr->head, t = vctr->tail;
          if (h < t) {
            if (atomicCAS(&ctr->head, h, h + 1) == h) {
              j = h;
              go = 1;
              took = true;
              break;
            }
            continue;
          }
          if (P.stop_flag && *P.stop_flag) break;
          // an open (serving) kernel leaves as a whole: the first CTA that
          // idled out closes it for all, so that work admitted meanwhile
          // never runs on a few stragglers; the host relaunches it for that
          // work
          if (vctr->closing) break;
          const long long pend = vctr->pending;
          const uint64_t waited = globaltimer_ns() - t0;
          if (pend <= 0) {
            if (!vctr->open) break;
            if (waited > P.idle_limit_ns) {
              atomicExch(&ctr->closing, 1);
              break;
            }
          } else if (waited > P.wait_limit_ns) {
            atomicOr(&ctr->error, DERR_TIMEOUT);
            break;
          }
          __nanosleep(ns);
          ns = ns < 4096 ? ns * 2 : ns;
        }
        if (go && !fetch_item(P, j, sh.batch[0])) go = 0;
        sh.bseq[0] = j;
        // a small input cluster: claim up to RW-1 more at once, one per
        // warp.  A request's input clusters are queued largest first in one
        // range, so the ones after a small one up to the range's end are
        // small too; taking them as a block costs one compare-and-swap and
        // never holds a larger item back behind them
        int k = 0;
        unsigned long long hb = 0;
        if (go && tiny_ok && !P.single_item && sh.batch[0].n <= tiny_lim &&
            (sh.batch[0].flags & ITEM_TOP) && !(P.stop_flag && *P.stop_flag)) {
          const unsigned long long send = __ldcg(&P.reqs[sh.batch[0].req].seed_end);
          for (int tries = 0; tries < 8; ++tries) {
            if (vctr->error != 0) break;
            const unsigned long long h = vctr->head, t = vctr->tail;
            const unsigned long long lim = t < send ? t : send;
            if (h >= lim) break;
            const int kk = (int)min((unsigned long long)(RW - 1), lim - h);
            if (atomicCAS(&ctr->head, h, h + kk) == h) {
              k = kk;
              hb = h;
              break;
            }
          }
        }
        sh.claim_h = hb;
        sh.claim_k = k;
        sh.go = go;
      }
      __syncwarp();
      // the block's items: waited for and read by lanes 1..k at once
      const int k = sh.claim_k;
      bool ok = true;
      if (lane >= 1 && lane <= k) {
        const unsigned long long q = sh.claim_h + (unsigned long long)(lane - 1);
        ok = fetch_item(P, q, sh.batch[lane]);
        sh.bseq[lane] = q;
      }
      const unsigned bad = __ballot_sync(FULL, !ok);
      if (lane == 0) {
        // a failed wait has set the error: the items after it stay unprocessed
        const int fetched = bad ? __ffs(bad) - 2 : k;
        sh.nb = sh.go ? 1 + fetched : 0;
      }
    }
    __syncthreads();
    if (P.prof && threadIdx.x == 0) {
      const long long t = clock64();
      cp.claim += t - pc;
      pc = t;
    }
    if (!sh.go) break;
    const int nb = sh.nb;
    if (threadIdx.x == 0) sh.ntouched = 0;  // bit k: batch item k runs on the CTA
    __syncthreads();
    if (tiny_ok) {
      const int warp = threadIdx.x >> 5;
      if (warp < nb && sh.batch[warp].n <= tiny_lim) {
        const Item ti = sh.batch[warp];
        const bool done = tiny_item(P, sh.bseq[warp], ti,
                                    reinterpret_cast<int32_t *>(wcc_dyn_smem + (size_t)warp * tiny_scr));
        __syncwarp();
        if ((threadIdx.x & 31) == 0) {
          if (done) finish_item(P, ti.req);
          else atomicOr(&sh.ntouched, 1 << warp);
        }
      }
      __syncthreads();
      if (P.prof && threadIdx.x == 0) {
        const long long t = clock64();
        cp.tiny += t - pc;
        pc = t;
        ++cp.batches;
        for (int k = 0; k < nb; ++k)
          cp.tiny_items += (sh.batch[k].n <= tiny_lim && !((sh.ntouched >> k) & 1)) ? 1 : 0;
      }
    }
    const int cta_mask = sh.ntouched;
    for (int k = 0; k < nb; ++k) {
      const Item it = sh.batch[k];
      if (tiny_ok && it.n <= tiny_lim && !((cta_mask >> k) & 1)) continue;
      const unsigned long long iseq = sh.bseq[k];
      if (P.prof && threadIdx.x == 0) {
        const long long t = clock64();
        for (int z = 0; z < 9; ++z) sh.ts[z] = t;
        sh.used_slab = 0;
        sh.pf_E = sh.pf_nalive = sh.pf_passes = sh.pf_nsv = -1;
        sh.pf_forest = sh.pf_nsv1 = 0;
        sh.pf_forest_cycles = 0;
        sh.pf_t0 = (long long)globaltimer_ns();
        for (int z = 0; z < 6; ++z) sh.fdbg[z] = 0;
        for (int z = 0; z < 4; ++z) sh.dbg[z] = 0;
      }
      __syncthreads();
      const int outcome = run_item(P, iseq, it, slab, sh);
      __syncthreads();
      if (P.prof && threadIdx.x == 0) {
        // fill skipped stamps forward, then record
        sh.ts[8] = clock64();
        for (int z = 1; z < 8; ++z)
          if (sh.ts[z] < sh.ts[z - 1]) sh.ts[z] = sh.ts[z - 1];
        const unsigned r = atomicAdd(P.prof_count, 1u);
        if (r < P.prof_cap) {
          ItemProf *q = &P.prof[r];
          q->seq = (unsigned)iseq;
          q->n = it.n;
          q->E = sh.pf_E;
          q->nalive = sh.pf_nalive;
          q->passes = sh.pf_passes;
          q->nsv = sh.pf_nsv;
          q->outcome = outcome;
          unsigned smid;
          asm("mov.u32 %0, %%smid;" : "=r"(smid));
          q->smid = (int)smid;
          q->slab = sh.used_slab;
          q->top = (int)(it.flags & ITEM_TOP);
          for (int z = 0; z < 8; ++z) q->dt[z] = (unsigned)(sh.ts[z + 1] - sh.ts[z]);
          q->t_begin = sh.pf_t0;
          q->t_end = (long long)globaltimer_ns();
          for (int z = 0; z < 4; ++z) q->dbg[z] = sh.dbg[z];
          q->forest = sh.pf_forest;
          q->nsv1 = sh.pf_nsv1;
          q->forest_cycles = sh.pf_forest_cycles;
          for (int z = 0; z < 6; ++z) q->fdbg[z] = sh.fdbg[z];
        }
      }
      if (threadIdx.x == 0) finish_item(P, it.req);
      __syncthreads();
      if (P.prof && threadIdx.x == 0) {
        const long long t = clock64();
        cp.cta += t - pc;
        pc = t;
        ++cp.cta_items;
      }
    }
    if (P.single_item) break;
  }
  if (P.prof && P.prof_cta && threadIdx.x == 0) P.prof_cta[blockIdx.x] = cp;
}

}  // namespace

size_t item_workspace_bytes(int64_t n, int64_t d) {
  return n < 65535 ? ws_bytes<uint16_t>(n, d) : ws_bytes<int32_t>(n, d);
}

int refine_block_threads() { return RB; }

// Largest dynamic shared memory a refinement CTA can opt into on this
// device: the per-block opt-in limit minus the kernel's static shared memory.
size_t refine_smem_max_bytes(int device) {
  int optin = 0;
  WCC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  cudaFuncAttributes fa;
  WCC_CUDA(cudaFuncGetAttributes(&fa, k_refine));
  size_t mx = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
  mx &= ~(size_t)1023;
  return mx < SMEM_MAX_BYTES ? mx : SMEM_MAX_BYTES;
}

static void set_smem_attr(int device) {
  WCC_CUDA(cudaFuncSetAttribute(k_refine, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)refine_smem_max_bytes(device)));
}

int refine_max_ctas(int device, size_t smem_bytes) {
  set_smem_attr(device);
  int per_sm = 0;
  WCC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_refine, RB, smem_bytes));
  int sms = 0;
  WCC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  int r = per_sm * sms;
  if (r < 1) fail(WCC_ERR_CUDA, "refinement kernel cannot be resident on this device");
  return r;
}

void launch_refine(const RefineParams &p, int grid, bool cooperative, cudaStream_t s) {
  int device = 0;
  WCC_CUDA(cudaGetDevice(&device));
  set_smem_attr(device);
  RefineParams pc = p;
  if (cooperative) {
    void *args[] = {&pc};
    WCC_CUDA(cudaLaunchCooperativeKernel((const void *)k_refine, dim3(grid), dim3(RB), args,
                                         p.smem_bytes, s));
    note_launch();
  } else {
    k_refine<<<grid, RB, p.smem_bytes, s>>>(pc); note_launch();
    WCC_CUDA(cudaGetLastError());
  }
}

}  // namespace wccg
