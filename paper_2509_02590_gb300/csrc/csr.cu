// csr.cu -- the device CSR builder behind wcc_create_graph_from_edges.
//
// An undirected edge list becomes a symmetric CSR with ascending,
// duplicate-free rows and no self-loops.  Rows first, then the order inside
// each row:
//   1. a degree count (atomics) and its scan give every row's start;
//   2. every edge is scattered into both of its rows through a per-row
//      cursor (the order inside a row is arbitrary at this point);
//   3. every row is sorted and freed of duplicates in place: by a warp in
//      registers (at most 32 entries), by a CTA in shared memory (at most
//      MID_MAX entries), or -- for the few longer rows -- by one radix sort of
//      (row rank, column) keys over just those rows' entries;
//   4. the unique counts are scanned into the row offsets, and only when
//      some row lost duplicates are the rows packed into a fresh array.
// Each directed entry is read and written a handful of times, against the
// log-many passes of a radix sort of 64-bit (row, column) keys over all of
// them, and the transient memory is a few bytes per vertex (plus the keys of
// the long rows) instead of about 24 bytes per directed entry.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace wccg {
namespace {

constexpr int CB = 256;
constexpr int SMALL_MAX = 32;     // longest row a warp sorts in registers
constexpr int MID_MAX = 16384;    // longest row a CTA sorts in shared memory

__global__ void k_csr_count(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                            int64_t m, int64_t n, uint32_t *cnt, unsigned *err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int32_t u = src[i], v = dst[i];
  if (u < 0 || u >= n || v < 0 || v >= n) {
    atomicOr(err, DERR_INVALID);
    return;
  }
  if (u == v) return;
  atomicAdd(&cnt[u], 1u);
  atomicAdd(&cnt[v], 1u);
}

// cnt counts down from each row's length: an entry's slot is its row start
// plus the count its decrement left.
__global__ void k_csr_scatter(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                              int64_t m, int64_t n, const uint32_t *__restrict__ start,
                              uint32_t *cnt, int32_t *raw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int32_t u = src[i], v = dst[i];
  if (u < 0 || u >= n || v < 0 || v >= n || u == v) return;
  raw[start[u] + atomicSub(&cnt[u], 1u) - 1u] = v;
  raw[start[v] + atomicSub(&cnt[v], 1u) - 1u] = u;
}

// Warp per row.  Rows of at most SMALL_MAX entries: bitonic sort across the
// lanes, then the first copy of each value is kept, packed to the row's
// front, and ucnt[row] = how many.  Longer rows are listed for the other
// kernels: ctr[0] rows in mid, ctr[1] rows in big, ctr[2] entries of big rows.
__global__ void k_csr_rows_small(const uint32_t *__restrict__ start, int64_t n, int32_t *raw,
                                 int64_t *ucnt, uint32_t *mid, uint32_t *big, uint32_t *ctr) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const uint32_t s = start[w];
  const uint32_t L = start[w + 1] - s;
  if (L > (uint32_t)SMALL_MAX) {
    if (lane == 0) {
      if (L <= (uint32_t)MID_MAX) {
        mid[atomicAdd(&ctr[0], 1u)] = (uint32_t)w;
      } else {
        big[atomicAdd(&ctr[1], 1u)] = (uint32_t)w;
        atomicAdd(&ctr[2], L);
      }
    }
    return;
  }
  int32_t x = (uint32_t)lane < L ? raw[s + lane] : INT32_MAX;  // pads sort last
  for (int k = 2; k <= 32; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int32_t y = __shfl_xor_sync(FULL, x, j);
      const bool up = (lane & k) == 0, low = (lane & j) == 0;
      x = (low == up) ? min(x, y) : max(x, y);
    }
  }
  const int32_t prev = __shfl_up_sync(FULL, x, 1);
  const bool keep = (uint32_t)lane < L && (lane == 0 || x != prev);
  const unsigned b = __ballot_sync(FULL, keep);
  if (keep) raw[s + __popc(b & lanemask_lt())] = x;
  if (lane == 0) ucnt[w] = __popc(b);
}

// Appends the kept values of sorted v[0, L) (first copies) to out, in
// order, in chunks of CB; returns how many.  v may be out itself (global,
// in place): a chunk reads all of its values before any write, writes land
// at or before their sources, and the value before a chunk is carried.
__device__ int dedup_sorted(const int32_t *v, int L, int32_t *out, int32_t *scan_tmp,
                            int32_t *carry) {
  int base = 0;
  int32_t before = -1;  // no vertex id is negative
  for (int c = 0; c < L; c += CB) {
    const int i = c + (int)threadIdx.x;
    const int32_t x = i < L ? v[i] : 0;
    const int32_t prev = threadIdx.x == 0 ? before : (i < L ? v[i - 1] : 0);
    const int keep = (i < L && (i == 0 || x != prev)) ? 1 : 0;
    int tot;
    const int ex = block_exclusive_scan<CB>(keep, &tot, scan_tmp);
    if (keep) out[base + ex] = x;
    if (i == min(c + CB, L) - 1) *carry = x;
    base += tot;
    __syncthreads();
    before = *carry;
  }
  return base;
}

// CTA per listed row of (SMALL_MAX, MID_MAX] entries: bitonic sort in
// shared memory (padded to a power of two), then the duplicate-free row back
// to the row's front.  Rows are taken in turn by a grid of any size.
__global__ void __launch_bounds__(CB) k_csr_rows_mid(const uint32_t *__restrict__ start,
                                                     const uint32_t *__restrict__ mid,
                                                     const uint32_t *__restrict__ ctr,
                                                     int32_t *raw, int64_t *ucnt) {
  extern __shared__ int32_t sv[];  // MID_MAX values
  __shared__ int32_t scan_tmp[CB / 32 + 1];
  __shared__ int32_t carry;
  const uint32_t nmid = ctr[0];
  for (uint32_t q = blockIdx.x; q < nmid; q += gridDim.x) {
    const uint32_t row = mid[q];
    const uint32_t s = start[row];
    const int L = (int)(start[row + 1] - s);
    int P = 2 * SMALL_MAX;
    while (P < L) P <<= 1;
    for (int i = threadIdx.x; i < P; i += CB) sv[i] = i < L ? raw[s + i] : INT32_MAX;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = threadIdx.x; t < P / 2; t += CB) {
          const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));  // pair (i, i + j)
          const int l = i | j;
          const int32_t a = sv[i], b = sv[l];
          if ((a > b) == ((i & k) == 0)) {
            sv[i] = b;
            sv[l] = a;
          }
        }
        __syncthreads();
      }
    }
    const int u = dedup_sorted(sv, L, raw + s, scan_tmp, &carry);
    if (threadIdx.x == 0) ucnt[row] = u;
    __syncthreads();  // sv is refilled for the next row
  }
}

__global__ void k_csr_big_len(const uint32_t *__restrict__ start, const uint32_t *__restrict__ big,
                              uint32_t nbig, uint32_t *len) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nbig) len[r] = start[big[r] + 1] - start[big[r]];
}

// keys[koff[r] + j] = (r << b) | j-th entry of listed long row r.
__global__ void k_csr_big_keys(const uint32_t *__restrict__ start, const uint32_t *__restrict__ big,
                               const uint32_t *__restrict__ koff, uint32_t nbig,
                               const int32_t *__restrict__ raw, int b, uint64_t *keys) {
  for (uint32_t r = blockIdx.x; r < nbig; r += gridDim.x) {
    const uint32_t s = start[big[r]], L = start[big[r] + 1] - s, o = koff[r];
    for (uint32_t j = threadIdx.x; j < L; j += blockDim.x)
      keys[o + j] = ((uint64_t)r << b) | (uint32_t)raw[s + j];
  }
}

// Sorted keys back into their rows: key i of rank r is entry i - koff[r].
__global__ void k_csr_big_back(const uint64_t *__restrict__ keys, uint32_t ne,
                               const uint32_t *__restrict__ start, const uint32_t *__restrict__ big,
                               const uint32_t *__restrict__ koff, int b, int32_t *raw) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ne) return;
  const uint64_t k = keys[i];
  const uint32_t r = (uint32_t)(k >> b);
  raw[start[big[r]] + (i - koff[r])] = (int32_t)(k & ((1ull << b) - 1));
}

// CTA per listed long row (now sorted): duplicates out, in place.
__global__ void __launch_bounds__(CB) k_csr_big_dedup(const uint32_t *__restrict__ start,
                                                      const uint32_t *__restrict__ big,
                                                      uint32_t nbig, int32_t *raw, int64_t *ucnt) {
  __shared__ int32_t scan_tmp[CB / 32 + 1];
  __shared__ int32_t carry;
  for (uint32_t r = blockIdx.x; r < nbig; r += gridDim.x) {
    const uint32_t row = big[r], s = start[row];
    const int L = (int)(start[row + 1] - s);
    const int u = dedup_sorted(raw + s, L, raw + s, scan_tmp, &carry);
    if (threadIdx.x == 0) ucnt[row] = u;
  }
}

// Warp per row: the row's kept prefix to its final place.
__global__ void k_csr_pack(const uint32_t *__restrict__ start, const int64_t *__restrict__ off,
                           int64_t n, const int32_t *__restrict__ raw, int32_t *cols) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const int64_t o = off[w], L = off[w + 1] - o;
  const uint32_t s = start[w];
  for (int64_t j = lane; j < L; j += 32) cols[o + j] = raw[s + j];
}

}  // namespace

int64_t build_csr_rows(const int32_t *src, const int32_t *dst, int64_t m, int64_t n, Graph &g,
                       cudaStream_t s) {
  const int64_t n2 = 2 * m;
  int64_t *d_off = g.off.as<int64_t>();  // zeroed by the caller, n + 1 entries
  if (n == 0) fail(WCC_ERR_INVALID, "edge endpoint outside [0, n)");
  int sms = 0;
  WCC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g.device));
  DevBuf bcnt, bstart, blist, bmisc, btemp;
  uint32_t *cnt = static_cast<uint32_t *>(bcnt.ensure(4 * (size_t)n));
  uint32_t *start = static_cast<uint32_t *>(bstart.ensure(4 * (size_t)(n + 1)));
  uint32_t *mid = static_cast<uint32_t *>(blist.ensure(8 * (size_t)n));
  uint32_t *big = mid + n;
  uint32_t *misc = static_cast<uint32_t *>(bmisc.ensure(64));  // err, ctr[3]
  unsigned *d_err = misc;
  uint32_t *ctr = misc + 1;
  void *temp = btemp.ensure(scan_temp_bytes(n + 1) + 64);
  int32_t *raw = static_cast<int32_t *>(g.adj.ensure(4 * (size_t)n2));
  WCC_CUDA(cudaMemsetAsync(cnt, 0, 4 * (size_t)n, s));
  WCC_CUDA(cudaMemsetAsync(misc, 0, 64, s));

  // 1-2: row starts, then every entry into its row
  k_csr_count<<<grid_for(m, CB), CB, 0, s>>>(src, dst, m, n, cnt, d_err);
  note_launch();
  exclusive_scan_u32(cnt, start, n, start + n, temp, s);
  k_csr_scatter<<<grid_for(m, CB), CB, 0, s>>>(src, dst, m, n, start, cnt, raw);
  note_launch();
  // 3a: short rows sorted, the others listed
  k_csr_rows_small<<<grid_for(n * 32, CB), CB, 0, s>>>(start, n, raw, d_off, mid, big, ctr);
  note_launch();
  WCC_CUDA(cudaGetLastError());
  uint32_t hb[5];
  WCC_CUDA(cudaMemcpyAsync(hb, misc, 16, cudaMemcpyDeviceToHost, s));
  WCC_CUDA(cudaMemcpyAsync(hb + 4, start + n, 4, cudaMemcpyDeviceToHost, s));
  WCC_CUDA(cudaStreamSynchronize(s));
  if (hb[0]) fail(WCC_ERR_INVALID, "edge endpoint outside [0, n)");
  const uint32_t nmid = hb[1], nbig = hb[2], nbig_entries = hb[3], nraw = hb[4];

  // 3b: rows of up to MID_MAX entries, in shared memory
  if (nmid > 0) {
    const size_t smem = 4 * (size_t)MID_MAX;
    WCC_CUDA(cudaFuncSetAttribute(k_csr_rows_mid, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    const unsigned grid = (unsigned)std::min<int64_t>(nmid, 3ll * sms);
    k_csr_rows_mid<<<grid, CB, smem, s>>>(start, mid, ctr, raw, d_off);
    note_launch();
    WCC_CUDA(cudaGetLastError());
  }
  // 3c: the longest rows, one radix sort of (rank, column) over their entries
  DevBuf bk1, bk2, bkoff, brtemp;
  if (nbig > 0) {
    const int b = (int)std::max<int64_t>(1, bitlen_u64((uint64_t)(n - 1)));
    const int rb = (int)std::max<int64_t>(1, bitlen_u64((uint64_t)(nbig - 1)));
    uint32_t *koff = static_cast<uint32_t *>(bkoff.ensure(8 * ((size_t)nbig + 1)));
    uint32_t *len = koff + nbig + 1;
    uint64_t *k1 = static_cast<uint64_t *>(bk1.ensure(8 * (size_t)nbig_entries));
    uint64_t *k2 = static_cast<uint64_t *>(bk2.ensure(8 * (size_t)nbig_entries));
    void *rtemp = brtemp.ensure(std::max(radix_temp_bytes(nbig_entries), scan_temp_bytes(nbig + 1)) + 64);
    k_csr_big_len<<<grid_for(nbig, CB), CB, 0, s>>>(start, big, nbig, len);
    note_launch();
    exclusive_scan_u32(len, koff, nbig, koff + nbig, rtemp, s);
    const unsigned grid = (unsigned)std::min<int64_t>(nbig, 4ll * sms);
    k_csr_big_keys<<<grid, CB, 0, s>>>(start, big, koff, nbig, raw, b, k1);
    note_launch();
    const uint64_t *sorted = radix_sort_keys_u64(k1, k2, nbig_entries, rb + b, rtemp, s) ? k2 : k1;
    k_csr_big_back<<<grid_for(nbig_entries, CB), CB, 0, s>>>(sorted, nbig_entries, start, big,
                                                             koff, b, raw);
    note_launch();
    k_csr_big_dedup<<<grid, CB, 0, s>>>(start, big, nbig, raw, d_off);
    note_launch();
    WCC_CUDA(cudaGetLastError());
  }
  // 4: offsets from the unique counts; pack only if something was dropped
  exclusive_scan_i64(d_off, d_off, n + 1, nullptr, temp, s);
  WCC_CUDA(cudaGetLastError());
  int64_t nnz = 0;
  WCC_CUDA(cudaMemcpyAsync(&nnz, d_off + n, 8, cudaMemcpyDeviceToHost, s));
  WCC_CUDA(cudaStreamSynchronize(s));
  if (nnz != (int64_t)nraw) {
    DevBuf packed;
    int32_t *cols = static_cast<int32_t *>(packed.ensure(4 * (size_t)std::max<int64_t>(nnz, 1)));
    k_csr_pack<<<grid_for(n * 32, CB), CB, 0, s>>>(start, d_off, n, raw, cols);
    note_launch();
    WCC_CUDA(cudaGetLastError());
    WCC_CUDA(cudaStreamSynchronize(s));
    std::swap(g.adj.p, packed.p);
    std::swap(g.adj.bytes, packed.bytes);
    std::swap(g.adj.dev, packed.dev);
  }
  return nnz;
}

}  // namespace wccg
