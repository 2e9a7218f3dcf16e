// primitives.cu -- device-wide prefix sums and stable LSD radix sorts used by
// the membership grouping and the CSR builder.  HBM-bound; tiles of
// SCAN_BLOCK x SCAN_ITEMS elements.
#include "internal.h"

namespace wccg {

namespace {

constexpr int SB = 256;          // threads per scan / sort block
constexpr int SI = 8;            // elements per thread
constexpr int TILE = SB * SI;    // elements per tile

int64_t ntiles_of(int64_t n) { return (n + TILE - 1) / TILE; }

// ---- scan -----------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(SB) k_tile_reduce(const T *__restrict__ in, int64_t n,
                                                   T *__restrict__ partial) {
  __shared__ T red[SB / 32];
  const int64_t base = (int64_t)blockIdx.x * TILE;
  T s = 0;
#pragma unroll
  for (int k = 0; k < SI; k++) {
    int64_t i = base + (int64_t)k * SB + threadIdx.x;
    if (i < n) s += in[i];
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    T w = threadIdx.x < SB / 32 ? red[threadIdx.x] : T(0);
    w = warp_sum(w);
    if (threadIdx.x == 0) partial[blockIdx.x] = w;
  }
}

// Single block: in-place exclusive scan of partial[0..nt), total to *total.
template <typename T>
__global__ void __launch_bounds__(SB) k_scan_partials(T *partial, int64_t nt, T *total) {
  __shared__ T sm[SB / 32 + 1];
  T carry = 0;
  for (int64_t b = 0; b < nt; b += SB) {
    int64_t i = b + threadIdx.x;
    T v = i < nt ? partial[i] : T(0);
    T tot;
    T ex = block_exclusive_scan<SB>(v, &tot, sm);
    if (i < nt) partial[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// Per-tile exclusive scan plus the tile's offset.  Elements are taken in the
// blocked order (thread t owns SI consecutive elements) so that loads of a
// warp stay within a few cache lines.
template <typename T>
__global__ void __launch_bounds__(SB) k_tile_scan(const T *__restrict__ in, T *__restrict__ out,
                                                 int64_t n, const T *__restrict__ partial,
                                                 T *total_single) {
  __shared__ T sm[SB / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * TILE + (int64_t)threadIdx.x * SI;
  T v[SI];
  T s = 0;
#pragma unroll
  for (int k = 0; k < SI; k++) {
    int64_t i = base + k;
    v[k] = i < n ? in[i] : T(0);
    s += v[k];
  }
  T tot;
  T ex = block_exclusive_scan<SB>(s, &tot, sm);
  T run = (partial ? partial[blockIdx.x] : T(0)) + ex;
#pragma unroll
  for (int k = 0; k < SI; k++) {
    int64_t i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
  if (total_single && threadIdx.x == 0) *total_single = tot;
}

template <typename T>
void exclusive_scan_impl(const T *in, T *out, int64_t n, T *total, void *temp, cudaStream_t s) {
  if (n <= 0) {
    if (total) WCC_CUDA(cudaMemsetAsync(total, 0, sizeof(T), s));
    return;
  }
  int64_t nt = ntiles_of(n);
  if (nt == 1) {
    k_tile_scan<T><<<1, SB, 0, s>>>(in, out, n, nullptr, total); note_launch();
    WCC_CUDA(cudaGetLastError());
    return;
  }
  T *partial = static_cast<T *>(temp);
  k_tile_reduce<T><<<(unsigned)nt, SB, 0, s>>>(in, n, partial); note_launch();
  k_scan_partials<T><<<1, SB, 0, s>>>(partial, nt, total); note_launch();
  k_tile_scan<T><<<(unsigned)nt, SB, 0, s>>>(in, out, n, partial, nullptr); note_launch();
  WCC_CUDA(cudaGetLastError());
}

// ---- radix sort -------------------------------------------------------------
// One pass = digit histogram per tile, scan of the digit-major histogram
// table, then a stable scatter.  Stability inside a tile: elements are ranked
// in index order, with __match_any_sync giving each element its rank among
// equal digits of its warp and a per-warp count table giving the warps
// before it.

template <typename K>
__device__ __forceinline__ unsigned digit_of(K k, int shift) {
  return (unsigned)((k >> shift) & (K)0xff);
}

template <typename K>
__global__ void __launch_bounds__(SB) k_radix_hist(const K *__restrict__ keys, int64_t n,
                                                  int shift, uint32_t *__restrict__ hist,
                                                  int64_t nt) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * TILE;
#pragma unroll
  for (int k = 0; k < SI; k++) {
    int64_t i = base + (int64_t)k * SB + threadIdx.x;
    if (i < n) atomicAdd(&h[digit_of(keys[i], shift)], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nt + blockIdx.x] = h[threadIdx.x];
}

template <typename K, bool HAS_VAL>
__global__ void __launch_bounds__(SB) k_radix_scatter(const K *__restrict__ kin,
                                                     const uint32_t *__restrict__ vin,
                                                     K *__restrict__ kout,
                                                     uint32_t *__restrict__ vout, int64_t n,
                                                     int shift,
                                                     const uint32_t *__restrict__ offs,
                                                     int64_t nt) {
  constexpr int NW = SB / 32;
  __shared__ uint32_t base_d[256];
  __shared__ uint32_t wcnt[NW][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  base_d[threadIdx.x] = offs[(int64_t)threadIdx.x * nt + blockIdx.x];
  const int64_t tbase = (int64_t)blockIdx.x * TILE;
  for (int k = 0; k < SI; k++) {
    int64_t i = tbase + (int64_t)k * SB + threadIdx.x;
    bool valid = i < n;
    K key = valid ? kin[i] : K(0);
    uint32_t val = (HAS_VAL && valid) ? vin[i] : 0u;
    unsigned d = valid ? digit_of(key, shift) : 256u;
    unsigned peers = __match_any_sync(FULL, d);
    unsigned rank = __popc(peers & lanemask_lt());
#pragma unroll
    for (int w = 0; w < NW; w++) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    if (valid && rank == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < NW; w++) {
      uint32_t c = wcnt[w][threadIdx.x];
      wcnt[w][threadIdx.x] = run;
      run += c;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = base_d[d] + wcnt[warp][d] + rank;
      kout[pos] = key;
      if (HAS_VAL) vout[pos] = val;
    }
    __syncthreads();
    base_d[threadIdx.x] += run;
    (void)lane;
  }
}

template <typename K, bool HAS_VAL>
bool radix_sort_impl(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt, int64_t n,
                     int bits, void *temp, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return false;
  if (n >= (int64_t)1 << 32) fail(WCC_ERR_INVALID, "radix sort: more than 2^32-1 elements");
  int64_t nt = ntiles_of(n);
  uint32_t *hist = static_cast<uint32_t *>(temp);
  void *scan_tmp = hist + 256 * nt;
  K *ka = keys, *kb = keys_alt;
  uint32_t *va = vals, *vb = vals_alt;
  bool in_alt = false;
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<K><<<(unsigned)nt, SB, 0, s>>>(ka, n, shift, hist, nt); note_launch();
    exclusive_scan_impl<uint32_t>(hist, hist, 256 * nt, nullptr, scan_tmp, s);
    k_radix_scatter<K, HAS_VAL><<<(unsigned)nt, SB, 0, s>>>(ka, va, kb, vb, n, shift, hist, nt); note_launch();
    WCC_CUDA(cudaGetLastError());
    std::swap(ka, kb);
    std::swap(va, vb);
    in_alt = !in_alt;
  }
  return in_alt;
}

}  // namespace

size_t scan_temp_bytes(int64_t n) { return (size_t)(ntiles_of(n) + 1) * sizeof(int64_t); }

void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total, void *temp,
                        cudaStream_t s) {
  exclusive_scan_impl<uint32_t>(in, out, n, total, temp, s);
}

void exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *total, void *temp,
                        cudaStream_t s) {
  exclusive_scan_impl<int64_t>(in, out, n, total, temp, s);
}

size_t radix_temp_bytes(int64_t n) {
  int64_t nt = ntiles_of(n);
  return (size_t)256 * nt * sizeof(uint32_t) + scan_temp_bytes(256 * nt) + 256;
}

bool radix_sort_pairs_u32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                          int64_t n, int bits, void *temp, cudaStream_t s) {
  return radix_sort_impl<uint32_t, true>(keys, vals, keys_alt, vals_alt, n, bits, temp, s);
}

bool radix_sort_keys_u64(uint64_t *keys, uint64_t *keys_alt, int64_t n, int bits, void *temp,
                         cudaStream_t s) {
  return radix_sort_impl<uint64_t, false>(keys, nullptr, keys_alt, nullptr, n, bits, temp, s);
}

}  // namespace wccg
