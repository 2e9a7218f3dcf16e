// refine.cu -- the refinement kernel: one CTA processes one work item at a
// time (an input cluster, or a part produced by an earlier split), entirely
// in on-chip shared memory when the item fits, else in a per-CTA slab of
// global memory (L2-resident for the sizes that need it).
//
// Per item (paper: Algorithm 1 for input clusters, then Algorithm 3 with a
// peel and a connectivity check in front of the cut):
//   1. extraction of the induced subgraph G[S] (Algorithm 1 / 3: E_c = edges
//      with both ends in V_c) into a local CSR, local id = rank of the global
//      id in S, by warp-per-vertex scans of the global adjacency with one
//      8-byte gather of slot[u] = (item << 32 | local id) per neighbour;
//   2. input clusters only: connected components (CCR); each component with
//      at least min_size vertices is queued, or refinement continues in place
//      when the cluster is one component;
//   3. round-synchronous peel of vertices with degree <= T(n);
//   4. connected components; more than one -> queue each large component;
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
constexpr size_t SMEM_BYTES = 56 * 1024;
constexpr uint32_t SLOT_NONE_HI = 0xffffffffu;

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Working memory of one item: see carve().
__host__ __device__ inline size_t ws_fixed_bytes(int64_t n) {
  size_t b = 0;
  b += align16(4 * (size_t)n);        // gid
  b += align16(4 * (size_t)(n + 1));  // off
  b += 8 * align16(4 * (size_t)(n + 1));  // A..H
  b += align16(8 * (size_t)n);        // pk
  b += 3 * align16((size_t)n);        // alive, flag, side
  return b;
}

struct Mem {
  int32_t *gid, *off, *A, *B, *C, *D, *E, *F, *G, *H;
  unsigned long long *pk;
  uint8_t *alive, *flag, *side;
  int32_t *adj;
  int64_t adj_cap;
};

__device__ inline Mem carve(char *base, size_t bytes, int n) {
  Mem m;
  char *p = base;
  auto take = [&](size_t b) { char *r = p; p += align16(b); return r; };
  m.gid = (int32_t *)take(4 * (size_t)n);
  m.off = (int32_t *)take(4 * (size_t)(n + 1));
  m.A = (int32_t *)take(4 * (size_t)(n + 1));
  m.B = (int32_t *)take(4 * (size_t)(n + 1));
  m.C = (int32_t *)take(4 * (size_t)(n + 1));
  m.D = (int32_t *)take(4 * (size_t)(n + 1));
  m.E = (int32_t *)take(4 * (size_t)(n + 1));
  m.F = (int32_t *)take(4 * (size_t)(n + 1));
  m.G = (int32_t *)take(4 * (size_t)(n + 1));
  m.H = (int32_t *)take(4 * (size_t)(n + 1));
  m.pk = (unsigned long long *)take(8 * (size_t)n);
  m.alive = (uint8_t *)take((size_t)n);
  m.flag = (uint8_t *)take((size_t)n);
  m.side = (uint8_t *)take((size_t)n);
  m.adj = (int32_t *)p;
  m.adj_cap = (int64_t)((base + bytes - p) / 4);
  return m;
}

// Block-level scalars.
struct Sh {
  int32_t scan[RW + 1];
  long long lscan[RW + 1];
  unsigned long long seq;
  Item item;
  int go;
  int32_t i0, i1, i2, i3;
  long long l0;
  unsigned long long u0;
  int32_t ntouched;
  int32_t contracted;
  int32_t sw_s, sw_t, sw_cut;
};

// ---- small device helpers ----------------------------------------------------

// Signed 64-bit atomic add (two's complement through the unsigned overload).
__device__ __forceinline__ void add_ll(long long *p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
}

// Criterion threshold T(n) (Section 2, criterion f(n)): the largest integer
// with cut <= T(n) <=> cut <= f(n) for integer cuts.  Written here
// independently of any host code.
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
// parent = B; returns the number of components; B[i] = smallest alive local
// id of i's component (or -1 for dead vertices).
__device__ int components(const Mem &m, int n, Sh &sh) {
  for (int i = threadIdx.x; i < n; i += RB) m.B[i] = m.alive[i] ? i : -1;
  __syncthreads();
  // warp per vertex: hook every alive edge (i, j), i < j
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < n; i += RW) {
    if (!m.alive[i]) continue;
    for (int e = m.off[i] + lane; e < m.off[i + 1]; e += 32) {
      int j = m.adj[e];
      if (j > i && m.alive[j]) uf_union(m.B, i, j);
    }
  }
  __syncthreads();
  int roots = 0;
  for (int i = threadIdx.x; i < n; i += RB) {
    if (!m.alive[i]) continue;
    int r = uf_find(m.B, i);
    roots += (r == i);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += RB)
    if (m.alive[i]) m.B[i] = uf_find(m.B, i);
  __syncthreads();
  return block_sum_int(roots, sh);
}

// ---- publishing children -------------------------------------------------
// tag[i] in [0, n) names the child of local vertex i (-1: none).  Every tag
// with at least min_size members becomes a new queue item whose vertex list
// (ascending) is written into the parent's pool range.  Uses C, D, E, F.
__device__ void emit_children(const RefineParams &P, const Mem &m, const int32_t *tag, int n,
                              int64_t vbeg, Sh &sh) {
  int32_t *cnt = m.C, *cidx = m.D, *cbase = m.E, *run = m.F;
  for (int t = threadIdx.x; t < n; t += RB) cnt[t] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += RB)
    if (tag[i] >= 0) atomicAdd(&cnt[tag[i]], 1);
  __syncthreads();
  for (int t = threadIdx.x; t < n; t += RB) {
    bool keep = cnt[t] >= P.min_size;
    cidx[t] = keep ? 1 : 0;
    cbase[t] = keep ? cnt[t] : 0;
    run[t] = 0;
  }
  __syncthreads();
  int nchild = block_scan_array(cidx, n, sh);
  block_scan_array(cbase, n, sh);
  if (nchild == 0) return;
  if (threadIdx.x == 0) {
    sh.u0 = atomicAdd(&P.ctr->tail, (unsigned long long)nchild);
    add_ll(&P.ctr->pending, (long long)nchild);
  }
  __syncthreads();
  const unsigned long long s0 = sh.u0;
  // members in ascending local order, one warp, 32 at a time
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int b = 0; b < n; b += 32) {
      int i = b + lane;
      int t = i < n ? tag[i] : -1;
      bool kept = t >= 0 && cnt[t] >= P.min_size;
      int key = kept ? t : -1;
      unsigned peers = __match_any_sync(FULL, key);
      int rank = __popc(peers & lanemask_lt());
      int before = kept ? run[t] : 0;
      __syncwarp();
      if (kept) {
        int pos = before + rank;
        int32_t v = m.gid[i];
        P.pool[vbeg + cbase[t] + pos] = v;
        P.slot[v] = ((unsigned long long)(s0 + cidx[t]) << 32) | (unsigned)pos;
        if (rank == 0) run[t] = before + __popc(peers);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  __threadfence();
  // descriptors, then publication
  for (int t = threadIdx.x; t < n; t += RB) {
    if (cnt[t] < P.min_size) continue;
    unsigned long long q = s0 + cidx[t];
    QSlot *sl = &P.ring[q % P.ring_cap];
    sl->item.vbeg = vbeg + cbase[t];
    sl->item.n = cnt[t];
    sl->item.flags = 0;
  }
  __threadfence();
  __syncthreads();
  for (int t = threadIdx.x; t < n; t += RB) {
    if (cnt[t] < P.min_size) continue;
    unsigned long long q = s0 + cidx[t];
    atomicExch((unsigned long long *)&P.ring[q % P.ring_cap].seq, q);
  }
  __syncthreads();
}

// ---- maximum-adjacency machinery -----------------------------------------
// The current super-vertices are the ids X with grp[X] == X among alive
// vertices.  group_members() lists them (pos[X] = list index, ascending) and
// groups their members: members of the super-vertex at list index j are
// D[C[j] .. C[j+1]).  Returns the count.  Uses C, D, G (pos), H (temp).
__device__ int group_members(const Mem &m, const int32_t *grp, int n, Sh &sh) {
  int32_t *pos = m.G, *gof = m.C, *mem = m.D, *fill = m.H;
  for (int i = threadIdx.x; i < n; i += RB) pos[i] = (m.alive[i] && grp[i] == i) ? 1 : 0;
  __syncthreads();
  int nsv = block_scan_array(pos, n, sh);
  for (int j = threadIdx.x; j <= nsv; j += RB) gof[j] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += RB)
    if (m.alive[i]) atomicAdd(&gof[pos[grp[i]]], 1);
  __syncthreads();
  block_scan_array(gof, nsv + 1, sh);
  for (int j = threadIdx.x; j < nsv; j += RB) fill[j] = gof[j];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += RB)
    if (m.alive[i]) mem[atomicAdd(&fill[pos[grp[i]]], 1)] = i;
  __syncthreads();
  return nsv;
}

__device__ __forceinline__ unsigned long long pack_key(int key, int id) {
  return ((unsigned long long)(unsigned)key << 32) | (unsigned)(~(unsigned)id);
}

// One maximum-adjacency ordering over the current super-vertices, run by
// warp 0 (the other warps wait at the closing barrier).  kcap > 0: keys
// capped at kcap and every edge X-Y whose key reaches kcap is merged into
// nrep (the contraction pass); kcap == 0: exact keys (a Stoer-Wagner phase),
// reporting the last two super-vertices s, t and the cut of the phase.
// Uses E (acc), F (key), H (touched), pk, flag (in A).
__device__ void ma_ordering(const Mem &m, const int32_t *grp, int32_t *nrep, int nsv, int kcap,
                            Sh &sh) {
  int32_t *acc = m.E, *key = m.F, *touched = m.H, *pos = m.G;
  for (int j = threadIdx.x; j < nsv; j += RB) {
    int X = m.D[m.C[j]];  // any member; its group id
    X = grp[X];
    m.pk[j] = pack_key(0, X);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int contracted = 0;
    int s = -1, t = -1, cut = 0;
    if (lane == 0) sh.ntouched = 0;
    __syncwarp();
    for (int step = 0; step < nsv; ++step) {
      unsigned long long best = 0;
      for (int j = lane; j < nsv; j += 32) {
        unsigned long long v = m.pk[j];
        best = v > best ? v : best;
      }
      best = warp_max(best);
      const int X = (int)(~(unsigned)(best & 0xffffffffu));
      const int kX = (int)(best >> 32);
      s = t;
      t = X;
      cut = kX;
      if (lane == 0) {
        m.pk[pos[X]] = 0ull;
        m.flag[X] = 1;
      }
      __syncwarp();
      if (step == nsv - 1) break;  // the last super-vertex has no unadded neighbour
      const int g = pos[X];
      const int mb = m.C[g], me = m.C[g + 1];
      if (me - mb == 1) {
        const int i = m.D[mb];
        for (int e = m.off[i] + lane; e < m.off[i + 1]; e += 32) {
          int j = m.adj[e];
          if (!m.alive[j]) continue;
          int Y = grp[j];
          if (Y == X || m.flag[Y]) continue;
          if (atomicAdd(&acc[Y], 1) == 0) touched[atomicAdd(&sh.ntouched, 1)] = Y;
        }
      } else {
        for (int q = mb + lane; q < me; q += 32) {
          const int i = m.D[q];
          for (int e = m.off[i]; e < m.off[i + 1]; ++e) {
            int j = m.adj[e];
            if (!m.alive[j]) continue;
            int Y = grp[j];
            if (Y == X || m.flag[Y]) continue;
            if (atomicAdd(&acc[Y], 1) == 0) touched[atomicAdd(&sh.ntouched, 1)] = Y;
          }
        }
      }
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
        m.pk[pos[Y]] = pack_key(nk, Y);
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

__device__ void reset_ma_state(const Mem &m, int n) {
  for (int i = threadIdx.x; i < n; i += RB) {
    m.E[i] = 0;
    m.F[i] = 0;
    m.flag[i] = 0;
  }
  __syncthreads();
}

// ---- one work item ---------------------------------------------------------
__device__ void process_item(const RefineParams &P, unsigned long long seq, const Item &it,
                             char *smem, char *slab, Sh &sh) {
  const int n = it.n;
  const int64_t vbeg = it.vbeg;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  RunCounters *ctr = P.ctr;

  // upper bound on local edges: sum of global degrees of the members
  long long dsum = 0;
  for (int i = threadIdx.x; i < n; i += RB) {
    int32_t v = P.pool[vbeg + i];
    dsum += P.off[v + 1] - P.off[v];
  }
  dsum = block_sum_ll(dsum, sh);
  const size_t need = ws_fixed_bytes(n) + 4 * (size_t)dsum + 64;
  char *base;
  size_t bytes;
  if (need <= P.smem_bytes) {
    base = smem;
    bytes = P.smem_bytes;
  } else {
    base = slab;
    bytes = P.slab_bytes;
    if (need > bytes) {
      if (threadIdx.x == 0) {
        atomicOr(&ctr->error, DERR_CAPACITY);
        atomicExch(&ctr->err_info, (unsigned)n);
      }
      return;
    }
  }
  Mem m = carve(base, bytes, n);
  for (int i = threadIdx.x; i < n; i += RB) m.gid[i] = P.pool[vbeg + i];
  __syncthreads();

  // 1. extraction: count, scan, fill
  for (int i = warp; i < n; i += RW) {
    const int32_t v = m.gid[i];
    const int64_t b = P.off[v], e = P.off[v + 1];
    int c = 0;
    for (int64_t q = b + lane; q < e; q += 32) {
      unsigned long long s = P.slot[P.adj[q]];
      c += (unsigned)(s >> 32) == (unsigned)seq;
    }
    c = warp_sum(c);
    if (lane == 0) m.off[i] = c;
  }
  __syncthreads();
  const int E = block_scan_array(m.off, n, sh);
  if (threadIdx.x == 0) m.off[n] = E;
  if (E > m.adj_cap) {
    if (threadIdx.x == 0) atomicOr(&ctr->error, DERR_CAPACITY);
    return;
  }
  for (int i = warp; i < n; i += RW) {
    const int32_t v = m.gid[i];
    const int64_t b = P.off[v], e = P.off[v + 1];
    int w = m.off[i];
    for (int64_t q0 = b; q0 < e; q0 += 32) {
      int64_t q = q0 + lane;
      bool hit = false;
      int loc = 0;
      if (q < e) {
        unsigned long long s = P.slot[P.adj[q]];
        hit = (unsigned)(s >> 32) == (unsigned)seq;
        loc = (int)(unsigned)(s & 0xffffffffu);
      }
      unsigned mask = __ballot_sync(FULL, hit);
      if (hit) m.adj[w + __popc(mask & lanemask_lt())] = loc;
      w += __popc(mask);
    }
  }
  for (int i = threadIdx.x; i < n; i += RB) m.alive[i] = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    add_ll(&ctr->items, 1ll);
    add_ll(&ctr->alg_bytes, (long long)(4 * n + 16 * n + 12 * dsum));
  }

  // 2. input cluster: CCR (Algorithm 1)
  if (it.flags & ITEM_TOP) {
    int nc = components(m, n, sh);
    if (nc != 1) {
      emit_children(P, m, m.B, n, vbeg, sh);
      return;
    }
  }

  // 3. peel (round-synchronous, T recomputed from the alive count)
  int32_t *deg = m.A;
  for (int i = threadIdx.x; i < n; i += RB) deg[i] = m.off[i + 1] - m.off[i];
  __syncthreads();
  int nalive = n;
  for (;;) {
    const int64_t T = threshold_of(P.rule_kind, P.rule_num, P.rule_den, nalive);
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
  if (threadIdx.x == 0 && nalive < n) add_ll(&ctr->peeled, (long long)(n - nalive));
  if (nalive < P.min_size) return;

  // 4. connectivity of what is left
  {
    int nc = components(m, n, sh);
    if (nc > 1) {
      emit_children(P, m, m.B, n, vbeg, sh);
      return;
    }
  }

  // 5. contraction with k = T+1
  const int64_t T = threshold_of(P.rule_kind, P.rule_num, P.rule_den, nalive);
  const int kcap = (int)(T + 1 < (1ll << 30) ? T + 1 : (1ll << 30));
  int32_t *rep = m.A, *nrep = m.B;
  for (int i = threadIdx.x; i < n; i += RB) rep[i] = m.alive[i] ? i : -1;
  __syncthreads();
  int nsv;
  for (;;) {
    nsv = group_members(m, rep, n, sh);
    if (nsv <= 1) break;
    reset_ma_state(m, n);
    for (int i = threadIdx.x; i < n; i += RB) nrep[i] = i;
    __syncthreads();
    if (threadIdx.x == 0) add_ll(&ctr->ni_passes, 1ll);
    ma_ordering(m, rep, nrep, nsv, kcap, sh);
    if (!sh.contracted) break;
    for (int i = threadIdx.x; i < n; i += RB)
      if (m.alive[i]) rep[i] = uf_find(nrep, rep[i]);
    __syncthreads();
  }

  if (nsv <= 1) {
    // accept (Algorithm 3: save V_c); output id resolved after the run
    if (threadIdx.x == 0) sh.i0 = n;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += RB)
      if (m.alive[i]) { atomicMin(&sh.i0, i); break; }
    __syncthreads();
    const int32_t minv = m.gid[sh.i0];
    for (int i = threadIdx.x; i < n; i += RB)
      if (m.alive[i]) P.label_min[m.gid[i]] = minv;
    if (threadIdx.x == 0) add_ll(&ctr->accepted, 1ll);
    __syncthreads();
    return;
  }

  // 6. canonical Stoer-Wagner on the contracted graph; grp = A (starts as rep)
  int32_t *grp = m.A;
  int best = 0x7fffffff;
  while (nsv > 1) {
    group_members(m, grp, n, sh);
    reset_ma_state(m, n);
    if (threadIdx.x == 0) add_ll(&ctr->sw_phases, 1ll);
    ma_ordering(m, grp, nullptr, nsv, 0, sh);
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
  if (best > T) {
    if (threadIdx.x == 0) atomicOr(&ctr->error, DERR_INTERNAL);
    return;
  }
  if (threadIdx.x == 0) add_ll(&ctr->splits, 1ll);
  for (int i = threadIdx.x; i < n; i += RB) m.B[i] = m.alive[i] ? (m.side[i] ? 1 : 0) : -1;
  __syncthreads();
  emit_children(P, m, m.B, n, vbeg, sh);
}

// ---- the persistent kernel ---------------------------------------------------
__global__ void __launch_bounds__(RB) k_refine(RefineParams P) {
  extern __shared__ __align__(16) char smem[];
  __shared__ Sh sh;
  char *slab = P.slab + (size_t)blockIdx.x * P.slab_bytes;
  RunCounters *ctr = P.ctr;
  for (;;) {
    if (threadIdx.x == 0) {
      int go = 1;
      unsigned long long j;
      if (P.single_item) {
        j = P.single_index;
      } else {
        j = atomicAdd(&ctr->head, 1ull);
      }
      QSlot *sl = &P.ring[j % P.ring_cap];
      const uint64_t t0 = globaltimer_ns();
      unsigned ns = 32;
      for (;;) {
        unsigned long long s = *(volatile unsigned long long *)&sl->seq;
        if (s == j) break;
        if (*(volatile unsigned *)&ctr->error != 0) { go = 0; break; }
        if (*(volatile long long *)&ctr->pending <= 0) { go = 0; break; }
        if (globaltimer_ns() - t0 > P.wait_limit_ns) {
          atomicOr(&ctr->error, DERR_TIMEOUT);
          go = 0;
          break;
        }
        __nanosleep(ns);
        ns = ns < 4096 ? ns * 2 : ns;
      }
      __threadfence();
      if (go) {
        volatile Item *vi = &sl->item;
        sh.item.vbeg = vi->vbeg;
        sh.item.n = vi->n;
        sh.item.flags = vi->flags;
        sh.seq = j;
      }
      sh.go = go;
    }
    __syncthreads();
    if (!sh.go) break;
    const Item it = sh.item;
    process_item(P, sh.seq, it, smem, slab, sh);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      add_ll(&ctr->pending, -1ll);
    }
    if (P.single_item) break;
  }
}

}  // namespace

size_t item_workspace_bytes(int64_t n, int64_t e) { return ws_fixed_bytes(n) + 4 * (size_t)e + 64; }

int refine_block_threads() { return RB; }

size_t refine_smem_bytes() { return SMEM_BYTES; }

int refine_max_ctas(int device) {
  static int cached[64] = {0};
  if (device >= 0 && device < 64 && cached[device]) return cached[device];
  WCC_CUDA(cudaFuncSetAttribute(k_refine, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SMEM_BYTES));
  int per_sm = 0;
  WCC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_refine, RB, SMEM_BYTES));
  int sms = 0;
  WCC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  int r = per_sm * sms;
  if (r < 1) fail(WCC_ERR_CUDA, "refinement kernel cannot be resident on this device");
  if (device >= 0 && device < 64) cached[device] = r;
  return r;
}

void launch_refine(const RefineParams &p, int grid, bool cooperative, cudaStream_t s) {
  WCC_CUDA(cudaFuncSetAttribute(k_refine, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)SMEM_BYTES));
  RefineParams pc = p;
  if (cooperative) {
    void *args[] = {&pc};
    WCC_CUDA(cudaLaunchCooperativeKernel((const void *)k_refine, dim3(grid), dim3(RB), args,
                                         SMEM_BYTES, s));
    note_launch();
  } else {
    k_refine<<<grid, RB, SMEM_BYTES, s>>>(pc); note_launch();
    WCC_CUDA(cudaGetLastError());
  }
}

}  // namespace wccg
