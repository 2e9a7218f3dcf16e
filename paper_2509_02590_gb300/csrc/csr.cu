// csr.cu -- the CSR builder by rows.
//
// The CSR of Section 2.1's graph store (both directions, self-loops and
// repeated edges dropped, every row ascending) built as a counting sort by
// row followed by a sort of every row on chip:
//   1. the entries of every row are counted (both directions of every edge
//      that is not a self-loop; an endpoint outside [0, n) is an error);
//   2. an exclusive scan of the counts gives each row's range;
//   3. every entry is written into its row's range through a per-row
//      cursor (the count, counted back down to zero);
//   4. every row is sorted and its repeats dropped, the unique entries
//      written back to the front of the row: rows of up to 256 entries by
//      one warp in registers (a bitonic network over 1, 2, 4 or 8 values a
//      lane), longer ones by a whole CTA in shared memory;
//   5. a scan of the unique counts gives the final offsets, and one copy
//      packs the rows.
// Nothing is read back before the end: one read of {error, longest row}
// closes the build.  A row longer than ROW_MAX is left unsorted, and the
// caller then builds the graph with the full sort instead.
#include <algorithm>

#include "internal.h"

namespace wccg {

namespace {

constexpr int CB = 256;        // threads per block
constexpr int ROW_WARP = 256;  // rows up to this long: one warp, in registers
constexpr int ROW_MAX = 16384; // rows up to this long: one CTA, in shared memory
constexpr int CTA_SORT_CTAS = 152 * 3;

__global__ void k_row_count(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                            int64_t m, int64_t n, uint32_t *cnt, unsigned *err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = src[i], v = dst[i];
    if (u < 0 || u >= n || v < 0 || v >= n) {
      atomicOr(err, DERR_INVALID);
      continue;
    }
    if (u == v) continue;
    atomicAdd(&cnt[u], 1u);
    atomicAdd(&cnt[v], 1u);
  }
}

// Entry positions within a row are taken by counting the row's count back
// down, so the counts end at zero.
__global__ void k_row_scatter(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                              int64_t m, int64_t n, const uint32_t *__restrict__ start,
                              uint32_t *cnt, int32_t *tmp) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = src[i], v = dst[i];
    if (u < 0 || u >= n || v < 0 || v >= n || u == v) continue;
    tmp[start[u] + atomicSub(&cnt[u], 1u) - 1u] = v;
    tmp[start[v] + atomicSub(&cnt[v], 1u) - 1u] = u;
  }
}

// Bitonic sort of 32 * R values held R to a lane: value i = r * 32 + lane
// sits in x[r] of lane `lane`; ascending in i at the end.  Partners closer
// than 32 apart are exchanged across lanes, farther ones within a lane.
template <int R>
__device__ __forceinline__ void warp_bitonic(int32_t (&x)[R], int lane) {
#pragma unroll
  for (int k = 2; k <= 32 * R; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int p = r ^ (j >> 5);
          if (p > r) {
            const bool up = ((r * 32 + lane) & k) == 0;
            const int32_t lo = min(x[r], x[p]), hi = max(x[r], x[p]);
            x[r] = up ? lo : hi;
            x[p] = up ? hi : lo;
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int32_t y = __shfl_xor_sync(FULL, x[r], j);
          const bool up = ((r * 32 + lane) & k) == 0, lower = (lane & j) == 0;
          x[r] = (lower == up) ? min(x[r], y) : max(x[r], y);
        }
      }
    }
  }
}

// One row of len <= 32 * R entries at tmp[s..): sorted, first copies
// written back to the front in order; returns their number.
template <int R>
__device__ __forceinline__ int warp_sort_row(int32_t *tmp, uint32_t s, int len, int lane) {
  int32_t x[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = r * 32 + lane;
    x[r] = i < len ? tmp[s + i] : 0x7fffffff;
  }
  warp_bitonic<R>(x, lane);
  int base = 0;
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int32_t up = __shfl_up_sync(FULL, x[r], 1);
    const int32_t last = __shfl_sync(FULL, r > 0 ? x[r > 0 ? r - 1 : 0] : 0, 31);
    const int32_t prev = lane > 0 ? up : last;
    const int i = r * 32 + lane;
    const bool keep = i < len && (i == 0 || x[r] != prev);
    const unsigned mask = __ballot_sync(FULL, keep);
    if (keep) tmp[s + base + __popc(mask & lt)] = x[r];
    base += __popc(mask);
  }
  return base;
}

// Every row, one warp each: rows of at most ROW_WARP entries are sorted
// here; longer ones are listed for k_row_sort_cta, with the longest length.
__global__ void k_row_sort_warp(int32_t *tmp, const uint32_t *__restrict__ start, int64_t n,
                                uint32_t *ndeg, int32_t *rows, unsigned *nrows,
                                unsigned *maxlen) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
    const uint32_t s = start[u];
    const int len = (int)(start[u + 1] - s);
    int d;
    if (len <= 32) {
      d = warp_sort_row<1>(tmp, s, len, lane);
    } else if (len <= 64) {
      d = warp_sort_row<2>(tmp, s, len, lane);
    } else if (len <= 128) {
      d = warp_sort_row<4>(tmp, s, len, lane);
    } else if (len <= ROW_WARP) {
      d = warp_sort_row<8>(tmp, s, len, lane);
    } else {
      if (lane == 0) {
        rows[atomicAdd(nrows, 1u)] = (int32_t)u;
        atomicMax(maxlen, (unsigned)len);
      }
      continue;
    }
    if (lane == 0) ndeg[u] = (uint32_t)d;
  }
}

// The listed rows (more than ROW_WARP entries), one CTA each: a bitonic
// network in shared memory over the next power of two, then the first
// copies written back in order.  Rows longer than ROW_MAX are skipped (the
// caller sees the longest length and builds with the full sort).
__global__ void __launch_bounds__(CB) k_row_sort_cta(int32_t *tmp, const uint32_t *__restrict__ start,
                                                    const int32_t *__restrict__ rows,
                                                    const unsigned *__restrict__ nrows,
                                                    uint32_t *ndeg) {
  extern __shared__ int32_t a[];
  __shared__ int32_t scan[CB / 32 + 1];
  const unsigned total = *nrows;
  for (unsigned r = blockIdx.x; r < total; r += gridDim.x) {
    const int32_t u = rows[r];
    const uint32_t s = start[u];
    const int len = (int)(start[u + 1] - s);
    if (len > ROW_MAX) {
      if (threadIdx.x == 0) ndeg[u] = 0;  // nothing of it is packed
      continue;
    }
    int P = 512;
    while (P < len) P <<= 1;
    for (int i = threadIdx.x; i < P; i += CB) a[i] = i < len ? tmp[s + i] : 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < P; i += CB) {
          const int l = i ^ j;
          if (l > i) {
            const int32_t x = a[i], y = a[l];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              a[i] = y;
              a[l] = x;
            }
          }
        }
        __syncthreads();
      }
    int carry = 0;
    for (int base = 0; base < len; base += CB) {
      const int i = base + threadIdx.x;
      const bool keep = i < len && (i == 0 || a[i] != a[i - 1]);
      int tot;
      const int ex = block_exclusive_scan<CB>(keep ? 1 : 0, &tot, scan);
      if (keep) tmp[s + carry + ex] = a[i];
      carry += tot;
    }
    if (threadIdx.x == 0) ndeg[u] = (uint32_t)carry;
    __syncthreads();
  }
}

// Final offsets (the scanned unique counts, widened) and the rows packed,
// one warp per row.
__global__ void k_row_pack(const int32_t *__restrict__ tmp, const uint32_t *__restrict__ start,
                           const uint32_t *__restrict__ pos, int64_t n, int64_t *off,
                           int32_t *adj) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u <= n; u += nw) {
    const int64_t o = pos[u];
    if (lane == 0) off[u] = o;
    if (u == n) continue;
    const uint32_t s = start[u];
    const int64_t len = (int64_t)pos[u + 1] - o;
    for (int64_t i = lane; i < len; i += 32) adj[o + i] = tmp[s + i];
  }
}

unsigned grid_of(int64_t threads) {
  const int64_t b = (threads + CB - 1) / CB;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 20));
}

}  // namespace

bool csr_by_rows(const int32_t *src, const int32_t *dst, int64_t m, int64_t n, int64_t *off,
                 DevBuf &adj_buf, int64_t *nnz_out, DevBuf (&b)[CSR_ROW_BUFS], cudaStream_t s) {
  const int64_t n2 = 2 * m;
  uint32_t *cnt = static_cast<uint32_t *>(b[0].ensure(4 * (size_t)(n + 1)));
  uint32_t *start = static_cast<uint32_t *>(b[1].ensure(4 * (size_t)(n + 1)));
  uint32_t *ndeg = static_cast<uint32_t *>(b[2].ensure(4 * (size_t)(n + 1)));
  int32_t *rows = static_cast<int32_t *>(b[3].ensure(4 * (size_t)std::max<int64_t>(n, 1)));
  int32_t *tmp = static_cast<int32_t *>(b[4].ensure(4 * (size_t)std::max<int64_t>(n2, 1)));
  unsigned *misc = static_cast<unsigned *>(b[5].ensure(64));  // err, nrows, maxlen, total
  void *temp = b[6].ensure(scan_temp_bytes(n + 1) + 64);
  int32_t *adj = static_cast<int32_t *>(adj_buf.ensure(4 * (size_t)std::max<int64_t>(n2, 1)));
  WCC_CUDA(cudaMemsetAsync(cnt, 0, 4 * (size_t)(n + 1), s));
  WCC_CUDA(cudaMemsetAsync(misc, 0, 64, s));
  const unsigned gm = grid_of(m);
  k_row_count<<<gm, CB, 0, s>>>(src, dst, m, n, cnt, misc); note_launch();
  exclusive_scan_u32(cnt, start, n + 1, misc + 3, temp, s);
  k_row_scatter<<<gm, CB, 0, s>>>(src, dst, m, n, start, cnt, tmp); note_launch();
  k_row_sort_warp<<<grid_of(32 * n), CB, 0, s>>>(tmp, start, n, ndeg, rows, misc + 1, misc + 2);
  note_launch();
  const size_t smem = 4 * (size_t)ROW_MAX;
  static_assert(4 * ROW_MAX > 48 * 1024, "the CTA sort opts into more than 48 KB");
  WCC_CUDA(cudaFuncSetAttribute(k_row_sort_cta, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  k_row_sort_cta<<<CTA_SORT_CTAS, CB, smem, s>>>(tmp, start, rows, misc + 1, ndeg); note_launch();
  WCC_CUDA(cudaMemsetAsync(ndeg + n, 0, 4, s));
  exclusive_scan_u32(ndeg, cnt, n + 1, nullptr, temp, s);  // cnt is all zero again: reuse it
  k_row_pack<<<grid_of(32 * (n + 1)), CB, 0, s>>>(tmp, start, cnt, n, off, adj); note_launch();
  WCC_CUDA(cudaGetLastError());
  unsigned h[4];
  int64_t nnz = 0;
  WCC_CUDA(cudaMemcpyAsync(h, misc, 16, cudaMemcpyDeviceToHost, s));
  WCC_CUDA(cudaMemcpyAsync(&nnz, off + n, 8, cudaMemcpyDeviceToHost, s));
  WCC_CUDA(cudaStreamSynchronize(s));
  if (h[0] & DERR_INVALID) fail(WCC_ERR_INVALID, "edge endpoint outside [0, n)");
  if (h[2] > (unsigned)ROW_MAX) return false;
  *nnz_out = nnz;
  return true;
}

}  // namespace wccg
