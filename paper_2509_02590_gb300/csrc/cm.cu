// cm.cu -- the community step of CM (Section 2.4, Algorithm 5: each side of a
// cut split goes through GetCommunities before it is checked again).
//
// The refinement kernel, in CM mode, writes the two sides of every cut split
// to the pool and lists them (RefineParams::cda) instead of publishing them.
// After the kernel has drained the queue, cm_round() runs:
//   k_cda      one CTA per listed part: the part's induced subgraph on local
//              ids (rank of the global id in the part's ascending list), CPM
//              local moving by one warp, the connected parts of every
//              community, and the communities of at least min_size members
//              written back to the part's pool range (ascending root, members
//              ascending) and listed as new items;
//   k_cda_reserve / k_cda_publish   the new items reserved at the queue's
//              tail, their members' slots set, and published;
// and the refinement kernel is launched again on them, until a round parks
// nothing.
//
// CPM local moving (Constant Potts Model at resolution gamma = gnum/gden):
// sweeps over the part's vertices in ascending local id, at most
// CPM_MAX_SWEEPS of them, until a sweep moves nothing.  Vertex v, taken out
// of its community c0, would gain g(c) = k(v, c) * gden - gnum * n_c by
// joining community c (k = edges from v into c, n_c its size without v); an
// empty community gains 0.  Candidates: the communities of v's neighbours
// other than c0, and, when c0 holds more than v, an empty community: n + v
// when nobody holds it, else the smallest id nobody holds (community ids run
// over 0..2n-1, v starting in v).  The largest gain wins,
// ties to the smallest id, and v moves only when it beats g(c0).
#include <algorithm>
#include <climits>

#include "internal.h"

namespace wccg {

namespace {

constexpr int CB = 256;
constexpr int CPM_MAX_SWEEPS = 64;

// Words of per-part state: gid[n], off[n+1], comm[n], size[2n], kc[2n],
// adj[d] (d local entries).  After the local moving, size holds the
// union-find and the community sizes, kc the output offsets and indices.
__host__ __device__ inline size_t cda_words(int64_t n, int64_t d) {
  return (size_t)(7 * n + 1 + d);
}

__device__ __forceinline__ int uf_root(int32_t *uf, int x) {
  while (true) {
    const int p = uf[x];
    if (p == x) return x;
    const int g = uf[p];
    if (g != p) uf[x] = g;  // halving; any value written is an ancestor
    x = p;
  }
}

// Links the sets of a and b, the larger root under the smaller, so that
// every root is the smallest member of its set.
__device__ __forceinline__ void uf_link_min(int32_t *uf, int a, int b) {
  while (true) {
    a = uf_root(uf, a);
    b = uf_root(uf, b);
    if (a == b) return;
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    if (atomicCAS(&uf[hi], hi, lo) == hi) return;
  }
}

// Exclusive prefix sum of a[0..n) in place, by the whole block; returns the
// total.
__device__ int block_scan_inplace(int32_t *a, int n, int32_t *tmp) {
  int carry = 0;
  for (int b = 0; b < n; b += CB) {
    const int i = b + threadIdx.x;
    const int v = i < n ? a[i] : 0;
    int tot;
    const int ex = block_exclusive_scan<CB>(v, &tot, tmp);
    if (i < n) a[i] = carry + ex;
    carry += tot;
  }
  return carry;
}

// CPM local moving by one warp over a part's state at ws (the layout of
// cda_words).  Instantiated once with ws derived from the block's shared
// array and once for the global scratch, so that each loop addresses its
// own space directly rather than through generic loads.
__device__ __forceinline__ void cpm_local_moving(int32_t *ws, int n, long long gnum,
                                                 long long gden) {
  const int lane = threadIdx.x & 31;
  int32_t *off = ws + n, *comm = off + n + 1, *size = comm + n, *kc = size + 2 * n;
  const int32_t *adj = kc + 2 * n;
  for (int sweep = 0; sweep < CPM_MAX_SWEEPS; ++sweep) {
    int moved = 0;
    for (int v = 0; v < n; ++v) {
      // n + v's size is read with the row (sizes change only at a move,
      // after the step's last use of it)
      const int c0 = comm[v], b = off[v], e = off[v + 1], szn = size[n + v];
      // the first 32 neighbours' communities stay in a register for the
      // three passes below (most rows are that short)
      const int cu0 = b + lane < e ? comm[adj[b + lane]] : -1;
      // neighbours' communities counted, one shared atomic a neighbour
      // (grouping equal communities by a warp match first took longer than
      // the atomics' address conflicts it saves)
      for (int q0 = b; q0 < e; q0 += 32) {
        const int q = q0 + lane;
        const int cu = q0 == b ? cu0 : (q < e ? comm[adj[q]] : -1);
        if (cu >= 0) atomicAdd(&kc[cu], 1);
      }
      __syncwarp();
      const long long s0 = size[c0] - 1;  // c0 without v
      const long long g0 = (long long)kc[c0] * gden - gnum * s0;
      long long bg = LLONG_MIN;
      int bc = INT_MAX;
      for (int q = b + lane; q < e; q += 32) {
        const int cu = q < b + 32 ? cu0 : comm[adj[q]];
        if (cu == c0) continue;
        const long long g = (long long)kc[cu] * gden - gnum * (long long)size[cu];
        if (g > bg || (g == bg && cu < bc)) {
          bg = g;
          bc = cu;
        }
      }
      // an empty community: n + v when nobody holds it, else the smallest id
      // nobody holds (size[c0] still counts v here, so c0 never looks empty;
      // at most n of the 2n ids are held)
      int ce = n + v;
      if (s0 > 0 && szn != 0) {
        ce = -1;
        for (int b0 = 0; ce < 0 && b0 < 2 * n; b0 += 32) {
          const int i = b0 + lane;
          const unsigned z = __ballot_sync(FULL, i < 2 * n && size[i] == 0);
          if (z) ce = b0 + __ffs(z) - 1;
        }
      }
      if (lane == 0 && s0 > 0 && ce >= 0) {
        if (0 > bg || (0 == bg && ce < bc)) {
          bg = 0;
          bc = ce;
        }
      }
      // the warp's best: largest gain (its order-preserving unsigned image
      // reduced high word, then low word), then the smallest id
      {
        const bool has = bc != INT_MAX;
        const unsigned long long ug = (unsigned long long)bg ^ 0x8000000000000000ull;
        const unsigned hi = has ? (unsigned)(ug >> 32) : 0u;
        const unsigned mhi = __reduce_max_sync(FULL, hi);
        const bool h1 = has && hi == mhi;
        const unsigned mlo = __reduce_max_sync(FULL, h1 ? (unsigned)ug : 0u);
        const bool h2 = h1 && (unsigned)ug == mlo;
        const unsigned mid = __reduce_max_sync(FULL, h2 ? ~(unsigned)bc : 0u);
        if (__ballot_sync(FULL, has)) {
          bc = (int)~mid;
          bg = (long long)((((unsigned long long)mhi << 32) | mlo) ^ 0x8000000000000000ull);
        } else {
          bc = INT_MAX;
          bg = LLONG_MIN;
        }
      }
      __syncwarp();
      for (int q = b + lane; q < e; q += 32) kc[q < b + 32 ? cu0 : comm[adj[q]]] = 0;
      __syncwarp();
      if (bc != INT_MAX && bg > g0) {
        if (lane == 0) {
          comm[v] = bc;
          size[c0] -= 1;
          size[bc] += 1;
        }
        ++moved;
      }
      __syncwarp();
    }
    if (moved == 0) break;
  }
}

__global__ void __launch_bounds__(CB, 1) k_cda(const Item *__restrict__ parts, unsigned long long nparts,
                                            const ReqCtx *__restrict__ reqs, long long gnum,
                                            long long gden, int32_t *partof, int32_t *loc,
                                            int32_t *gscratch, size_t gwords, size_t swords,
                                            Item *out, unsigned long long *nout,
                                            unsigned long long out_cap, unsigned *err) {
  extern __shared__ int32_t smem_ws[];
  __shared__ int32_t tmp[CB / 32 + 1];
  __shared__ unsigned long long s_ds, s_at;
  const int lane = threadIdx.x & 31;
  for (unsigned long long p = blockIdx.x; p < nparts; p += gridDim.x) {
    const Item it = parts[p];
    const ReqCtx &R = reqs[it.req];
    const int n = it.n;
    const int64_t vbeg = it.vbeg;
    const int min_size = R.min_size;
    // the part's members marked, and its local entries counted: the state
    // lives in shared memory when it fits
    for (int i = threadIdx.x; i < n; i += CB) {
      const int32_t v = R.pool[vbeg + i];
      partof[v] = (int32_t)p;
      loc[v] = i;
    }
    if (threadIdx.x == 0) s_ds = 0;
    __syncthreads();
    long long ds = 0;
    for (int i = threadIdx.x; i < n; i += CB) {
      const int32_t v = R.pool[vbeg + i];
      for (int64_t q = R.off[v]; q < R.off[v + 1]; ++q) ds += partof[R.adj[q]] == (int32_t)p;
    }
    atomicAdd(&s_ds, (unsigned long long)ds);
    __syncthreads();
    const size_t need = cda_words(n, (int64_t)s_ds);
    int32_t *ws;
    if (need <= swords) {
      ws = smem_ws;
    } else if (need <= gwords) {
      ws = gscratch + (size_t)blockIdx.x * gwords;
    } else {
      for (int i = threadIdx.x; i < n; i += CB) partof[R.pool[vbeg + i]] = -1;
      if (threadIdx.x == 0) atomicOr(err, DERR_CAPACITY);
      __syncthreads();
      continue;
    }
    int32_t *gid = ws, *off = gid + n, *comm = off + n + 1, *size = comm + n, *kc = size + 2 * n;
    int32_t *adj = kc + 2 * n;
    // after the local moving: union-find and sizes in size[], output
    // offsets and indices in kc[]
    int32_t *uf = size, *cnt = size + n, *base = kc, *kidx = kc + n;
    // the induced subgraph on local ids
    for (int i = threadIdx.x; i < n; i += CB) {
      const int32_t v = R.pool[vbeg + i];
      gid[i] = v;
      int d = 0;
      for (int64_t q = R.off[v]; q < R.off[v + 1]; ++q) d += partof[R.adj[q]] == (int32_t)p;
      off[i] = d;
    }
    __syncthreads();
    const int E = block_scan_inplace(off, n, tmp);
    if (threadIdx.x == 0) off[n] = E;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += CB) {
      const int32_t v = gid[i];
      int w = off[i];
      for (int64_t q = R.off[v]; q < R.off[v + 1]; ++q) {
        const int32_t u = R.adj[q];
        if (partof[u] == (int32_t)p) adj[w++] = loc[u];
      }
      comm[i] = i;
      size[i] = 1;
      size[n + i] = 0;
      kc[i] = 0;
      kc[n + i] = 0;
    }
    __syncthreads();
    // CPM local moving, one warp, on the state in shared memory or in the
    // global scratch
    if (threadIdx.x < 32) {
      if (ws == smem_ws)
        cpm_local_moving(smem_ws, n, gnum, gden);
      else
        cpm_local_moving(ws, n, gnum, gden);
    }
    __syncthreads();
    // the connected parts of every community
    for (int i = threadIdx.x; i < n; i += CB) {
      uf[i] = i;
      cnt[i] = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += CB)
      for (int q = off[i]; q < off[i + 1]; ++q) {
        const int u = adj[q];
        if (u > i && comm[u] == comm[i]) uf_link_min(uf, i, u);
      }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += CB) {
      const int r = uf_root(uf, i);
      comm[i] = r;  // comm now holds the root
      atomicAdd(&cnt[r], 1);
    }
    __syncthreads();
    // kept communities, in ascending root order; uf becomes the running
    // fill per root
    for (int i = threadIdx.x; i < n; i += CB) {
      const bool keep = comm[i] == i && cnt[i] >= min_size;
      base[i] = keep ? cnt[i] : 0;
      kidx[i] = keep ? 1 : 0;
      uf[i] = 0;
    }
    __syncthreads();
    block_scan_inplace(base, n, tmp);
    const int nkeep = block_scan_inplace(kidx, n, tmp);
    if (threadIdx.x == 0) {
      s_at = atomicAdd(nout, (unsigned long long)nkeep);
      if (s_at + nkeep > out_cap) atomicOr(err, DERR_CAPACITY);
    }
    __syncthreads();
    const unsigned long long at = s_at;
    const bool room = at + nkeep <= out_cap;
    // members in ascending local order, one warp
    if (threadIdx.x < 32 && room) {
      for (int b = 0; b < n; b += 32) {
        const int i = b + lane;
        const int r = i < n ? comm[i] : -1;
        const bool kept = r >= 0 && cnt[r] >= min_size;
        const int key = kept ? r : -1;
        const unsigned peers = __match_any_sync(FULL, key);
        const int rank = __popc(peers & lanemask_lt());
        const int before = kept ? uf[r] : 0;
        __syncwarp();
        if (kept) {
          R.pool[vbeg + base[r] + before + rank] = gid[i];
          if (rank == 0) uf[r] = before + __popc(peers);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (room)
      for (int i = threadIdx.x; i < n; i += CB)
        if (comm[i] == i && cnt[i] >= min_size)
          out[at + kidx[i]] = Item{vbeg + base[i], cnt[i], (uint16_t)0, it.req};
    for (int i = threadIdx.x; i < n; i += CB) partof[gid[i]] = -1;
    __syncthreads();
  }
}

// Head back to the tail (a closed run's tickets may have passed it), the new
// items reserved there, and the pending counts raised.
__global__ void k_cda_reserve(RunCounters *ctr, const unsigned long long *nout,
                              unsigned long long *base) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned long long k = *nout;
  const unsigned long long t = ctr->tail;
  ctr->head = t;
  ctr->tail = t + k;
  ctr->pending += (long long)k;
  *base = t;
}

// One warp per new item: its members' slots, the descriptor, then the
// publication.
__global__ void k_cda_publish(const Item *__restrict__ items, const unsigned long long *nout,
                              const unsigned long long *base, ReqCtx *reqs, QSlot *ring,
                              uint64_t cap) {
  const unsigned long long k = *nout;
  const int lane = threadIdx.x & 31;
  const unsigned long long w0 = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long w = w0; w < k; w += nw) {
    const Item it = items[w];
    const unsigned long long q = *base + w;
    ReqCtx &R = reqs[it.req];
    for (int j = lane; j < it.n; j += 32) {
      const int32_t v = R.pool[it.vbeg + j];
      R.slot[v] = ((unsigned long long)queue_tag(q) << 32) | (unsigned)j;
    }
    __syncwarp();
    if (lane == 0) {
      atomicAdd(reinterpret_cast<unsigned long long *>(&R.pending), 1ull);
      QSlot *sl = &ring[q % cap];
      sl->item = it;
      __threadfence();
      atomicExch(reinterpret_cast<unsigned long long *>(&sl->seq), q);
    }
  }
}

}  // namespace

size_t cda_scratch_words(int64_t max_n, int64_t max_dsum) { return cda_words(max_n, max_dsum); }

unsigned long long cm_round(const Item *parts, unsigned long long nparts, ReqCtx *reqs,
                            int64_t gnum, int64_t gden, int32_t *partof, int32_t *loc,
                            int64_t n_vertices, int64_t max_n, int64_t max_dsum, RunCounters *ctr,
                            QSlot *ring, uint64_t cap, int grid_max, DevBuf &scratch,
                            DevBuf &items, DevBuf &misc, cudaStream_t s) {
  if (nparts == 0) return 0;
  int dev = 0;
  WCC_CUDA(cudaGetDevice(&dev));
  int smax = 0;
  WCC_CUDA(cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t smem = (size_t)smax - 2048;  // the kernel's static shared memory beside it
  WCC_CUDA(cudaFuncSetAttribute(k_cda, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = (int)std::min<unsigned long long>(nparts, (unsigned long long)grid_max);
  const size_t gwords = cda_words(max_n, max_dsum);
  int32_t *gs = static_cast<int32_t *>(scratch.ensure(4 * gwords * (size_t)grid));
  // every new item has at least two members
  const unsigned long long out_cap = (unsigned long long)n_vertices / 2 + 1;
  Item *out = static_cast<Item *>(items.ensure(sizeof(Item) * out_cap));
  auto *m = static_cast<unsigned long long *>(misc.ensure(64));  // nout, base, err
  WCC_CUDA(cudaMemsetAsync(m, 0, 64, s));
  k_cda<<<grid, CB, smem, s>>>(parts, nparts, reqs, gnum, gden, partof, loc, gs, gwords, smem / 4,
                               out, m, out_cap, reinterpret_cast<unsigned *>(m + 2));
  note_launch();
  WCC_CUDA(cudaGetLastError());
  k_cda_reserve<<<1, 32, 0, s>>>(ctr, m, m + 1); note_launch();
  unsigned long long h[3];
  WCC_CUDA(cudaMemcpyAsync(h, m, 24, cudaMemcpyDeviceToHost, s));
  WCC_CUDA(cudaStreamSynchronize(s));
  const unsigned err = (unsigned)h[2];
  if (err & DERR_CAPACITY) fail(WCC_ERR_INTERNAL, "community step: a part or its output did not fit");
  if (h[0] > 0) {
    const unsigned blocks = (unsigned)std::min<unsigned long long>((h[0] + 7) / 8, 4096ull);
    k_cda_publish<<<blocks, CB, 0, s>>>(out, m, m + 1, reqs, ring, cap); note_launch();
    WCC_CUDA(cudaGetLastError());
  }
  return h[0];
}

}  // namespace wccg
