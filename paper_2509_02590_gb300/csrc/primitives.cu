// primitives.cu -- device-wide prefix sums and stable LSD radix sorts used by
// the membership grouping and the CSR builder.  HBM-bound; tiles of
// SCAN_BLOCK x SCAN_ITEMS elements.
#include <algorithm>

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
// Stable LSD radix sort, 8-bit digits, one kernel per pass ("one sweep"):
//   - one read of all keys first counts the digits of every pass (a digit's
//     global count does not depend on the order), and their exclusive
//     prefix gives each digit's start in the output of every pass;
//   - in a pass, each CTA takes the next tile (a counter hands tiles out in
//     order), ranks its keys among equal digits in index order (per warp by
//     __match_any_sync and a count table, then across warps), publishes its
//     per-digit counts, and finds the number of keys of each digit in all
//     earlier tiles by looking back over their published words (decoupled
//     look-back: a tile that has its inclusive prefix ends the walk); the
//     tile is then staged in shared memory in sorted order and each digit's
//     run written out contiguously.
// A status word holds a state (2 bits: aggregate or inclusive prefix), the
// pass it belongs to (8 bits) and a count; the status array is cleared once
// per sort.  Every wait on a predecessor is bounded: past the limit the
// sort sets DERR_TIMEOUT in *err and leaves its result unspecified.

constexpr int OS_SI = 16;                 // keys per thread (16: 5% faster than 8 or 12 on 400M keys)
constexpr int OS_TILE = SB * OS_SI;       // keys per tile
constexpr int OS_MAXPASS = 8;             // 64-bit keys
constexpr unsigned long long ST_AGG = 1ull << 62, ST_PRE = 2ull << 62;
constexpr unsigned long long ST_VAL = (1ull << 54) - 1;

int64_t os_tiles(int64_t n) { return (n + OS_TILE - 1) / OS_TILE; }

template <typename K>
__device__ __forceinline__ unsigned digit_of(K k, int shift) {
  return (unsigned)((k >> shift) & (K)0xff);
}

// hist[p][d] += count of keys whose digit p is d (all passes, one read)
template <typename K>
__global__ void __launch_bounds__(SB) k_digit_counts(const K *__restrict__ keys, int64_t n,
                                                    int npass, uint32_t *__restrict__ hist) {
  __shared__ uint32_t h[OS_MAXPASS][256];
#pragma unroll
  for (int p = 0; p < OS_MAXPASS; ++p) h[p][threadIdx.x] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * SB + threadIdx.x; i < n; i += (int64_t)gridDim.x * SB) {
    const K k = keys[i];
    for (int p = 0; p < npass; ++p) atomicAdd(&h[p][digit_of(k, 8 * p)], 1u);
  }
  __syncthreads();
  for (int p = 0; p < npass; ++p)
    if (h[p][threadIdx.x]) atomicAdd(&hist[p * 256 + threadIdx.x], h[p][threadIdx.x]);
}

// In place: hist[p][d] -> exclusive prefix over d (one block, thread = digit).
__global__ void __launch_bounds__(SB) k_digit_starts(uint32_t *hist, int npass) {
  __shared__ uint32_t sm[SB / 32 + 1];
  for (int p = 0; p < npass; ++p) {
    const uint32_t v = hist[p * 256 + threadIdx.x];
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan<SB>(v, &tot, sm);
    hist[p * 256 + threadIdx.x] = ex;
  }
}

template <typename K, bool HAS_VAL>
__global__ void __launch_bounds__(SB, 3) k_onesweep(const K *__restrict__ kin,
                                                const uint32_t *__restrict__ vin,
                                                K *__restrict__ kout, uint32_t *__restrict__ vout,
                                                int64_t n, int shift, unsigned tag,
                                                const uint32_t *__restrict__ gbase,
                                                unsigned long long *status, unsigned *tile_ctr,
                                                unsigned *err, unsigned long long wait_ns) {
  constexpr int NW = SB / 32;
  __shared__ uint32_t wcnt[NW][256];  // per-warp digit counts, then per-warp offsets
  __shared__ uint32_t dstart[256];    // tile-local start of each digit
  __shared__ unsigned long long gpos[256];  // where each digit's run of this tile goes
  __shared__ uint32_t scan_sm[NW + 1];
  __shared__ unsigned tile_sh;
  __shared__ K stage[OS_TILE];
  __shared__ uint32_t vstage[HAS_VAL ? OS_TILE : 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) tile_sh = atomicAdd(tile_ctr, 1u);
#pragma unroll
  for (int w = 0; w < NW; ++w) wcnt[w][threadIdx.x] = 0;
  __syncthreads();
  const unsigned tile = tile_sh;
  const int64_t tbase = (int64_t)tile * OS_TILE;
  const int tn = (int)min((int64_t)OS_TILE, n - tbase);
  K key[OS_SI];
  uint32_t val[OS_SI];
  uint32_t lrank[OS_SI];
  unsigned dig[OS_SI];
#pragma unroll
  for (int k = 0; k < OS_SI; ++k) {
    const int li = warp * (32 * OS_SI) + k * 32 + lane;  // tile-local index
    const bool valid = li < tn;
    key[k] = valid ? kin[tbase + li] : K(0);
    val[k] = (HAS_VAL && valid) ? vin[tbase + li] : 0u;
    dig[k] = valid ? digit_of(key[k], shift) : 256u;
  }
#pragma unroll
  for (int k = 0; k < OS_SI; ++k) {
    const unsigned d = dig[k];
    const unsigned peers = __match_any_sync(FULL, d);
    const unsigned before = __popc(peers & lanemask_lt());
    const uint32_t base = d < 256u ? wcnt[warp][d] : 0u;
    __syncwarp();
    if (d < 256u && before == 0) wcnt[warp][d] = base + __popc(peers);
    __syncwarp();
    lrank[k] = base + before;
  }
  __syncthreads();
  // thread t owns digit t: offsets of each warp within the digit, the tile's
  // count of the digit, the tile-local starts
  uint32_t c = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const uint32_t x = wcnt[w][threadIdx.x];
    wcnt[w][threadIdx.x] = c;
    c += x;
  }
  uint32_t tot;
  dstart[threadIdx.x] = block_exclusive_scan<SB>(c, &tot, scan_sm);
  // publish this tile's count of digit t, then add up the earlier tiles'
  const unsigned long long tg = (unsigned long long)(tag & 0xffu) << 54;
  unsigned long long *my = status + (size_t)tile * 256 + threadIdx.x;
  unsigned long long excl = 0;
  if (tile == 0) {
    atomicExch(my, ST_PRE | tg | (unsigned long long)c);
  } else {
    atomicExch(my, ST_AGG | tg | (unsigned long long)c);
    // eight predecessors' words are loaded at once per step: the walk passes
    // aggregates until it meets an inclusive prefix (tile 0 always has one)
    constexpr int LB = 8;
    int64_t p = (int64_t)tile - 1;
    const uint64_t t0 = globaltimer_ns();
    bool done = false;
    while (!done) {
      unsigned long long w[LB];
#pragma unroll
      for (int z = 0; z < LB; ++z)
        w[z] = p - z >= 0 ? *(volatile unsigned long long *)(status + (size_t)(p - z) * 256 +
                                                             threadIdx.x)
                          : 0ull;
      int used = 0;
#pragma unroll
      for (int z = 0; z < LB; ++z) {
        if (done || used < z) continue;  // stopped earlier in this window
        const unsigned long long x = w[z];
        if ((x >> 62) == 0 || ((x >> 54) & 0xffull) != (tag & 0xffu)) continue;  // not yet
        excl += x & ST_VAL;
        used = z + 1;
        if ((x >> 62) == 2ull || p - z == 0) done = true;
      }
      p -= used;
      if (done) break;
      if (used == 0 && globaltimer_ns() - t0 > wait_ns) {  // a predecessor never published
        atomicOr(err, DERR_TIMEOUT);
        __threadfence();
        break;
      }
    }
    // published even after a timeout, so that no successor waits in turn
    atomicExch(my, ST_PRE | tg | (excl + c));
  }
  gpos[threadIdx.x] = (unsigned long long)gbase[threadIdx.x] + excl;
  __threadfence();
  // after a timeout anywhere the counts may be wrong: write nothing
  const bool failed = *(volatile unsigned *)err & DERR_TIMEOUT;
  if (__syncthreads_or(failed)) return;
#pragma unroll
  for (int k = 0; k < OS_SI; ++k) {
    const unsigned d = dig[k];
    if (d < 256u) {
      const uint32_t pos = dstart[d] + wcnt[warp][d] + lrank[k];
      stage[pos] = key[k];
      if (HAS_VAL) vstage[pos] = val[k];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < tn; i += SB) {
    const K kk = stage[i];
    const unsigned d = digit_of(kk, shift);
    const unsigned long long op = gpos[d] + (unsigned long long)(i - (int)dstart[d]);
    if (op >= (unsigned long long)n) continue;  // cannot happen with consistent counts
    kout[op] = kk;
    if (HAS_VAL) vout[op] = vstage[i];
  }
}

// Layout of the sort's temporary memory: digit starts of every pass, the
// tile counters of every pass, the status words of every tile.
struct SortTemp {
  uint32_t *hist;
  unsigned *tile_ctr;
  unsigned long long *status;
};
SortTemp sort_temp(void *temp) {
  SortTemp t;
  char *p = static_cast<char *>(temp);
  t.hist = reinterpret_cast<uint32_t *>(p);
  t.tile_ctr = reinterpret_cast<unsigned *>(p + 4 * 256 * OS_MAXPASS);
  t.status = reinterpret_cast<unsigned long long *>(p + 4 * 256 * OS_MAXPASS + 256);
  return t;
}

template <typename K, bool HAS_VAL>
bool radix_sort_impl(K *keys, uint32_t *vals, K *keys_alt, uint32_t *vals_alt, int64_t n,
                     int bits, void *temp, unsigned *err, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return false;
  if (n >= (int64_t)1 << 32) fail(WCC_ERR_INVALID, "radix sort: more than 2^32-1 elements");
  const int npass = (bits + 7) / 8;
  if (npass > OS_MAXPASS) fail(WCC_ERR_INTERNAL, "radix sort: key too wide");
  const int64_t nt = os_tiles(n);
  SortTemp t = sort_temp(temp);
  WCC_CUDA(cudaMemsetAsync(t.hist, 0, 4 * 256 * OS_MAXPASS + 256, s));
  WCC_CUDA(cudaMemsetAsync(t.status, 0, sizeof(unsigned long long) * 256 * (size_t)nt, s));
  {
    const int64_t blocks = std::min<int64_t>((n + SB - 1) / SB, 1184);
    k_digit_counts<K><<<(unsigned)blocks, SB, 0, s>>>(keys, n, npass, t.hist); note_launch();
    k_digit_starts<<<1, SB, 0, s>>>(t.hist, npass); note_launch();
  }
  const unsigned long long wait_ns = 1000ull * 1000 * 1000;  // 1 s
  K *ka = keys, *kb = keys_alt;
  uint32_t *va = vals, *vb = vals_alt;
  bool in_alt = false;
  for (int p = 0; p < npass; ++p) {
    k_onesweep<K, HAS_VAL><<<(unsigned)nt, SB, 0, s>>>(ka, va, kb, vb, n, 8 * p, (unsigned)(p + 1),
                                                       t.hist + 256 * p, t.status, t.tile_ctr + p,
                                                       err, wait_ns);
    note_launch();
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
  return 4 * 256 * OS_MAXPASS + 256 + sizeof(unsigned long long) * 256 * (size_t)os_tiles(n) + 256;
}

bool radix_sort_pairs_u32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                          int64_t n, int bits, void *temp, unsigned *err, cudaStream_t s) {
  return radix_sort_impl<uint32_t, true>(keys, vals, keys_alt, vals_alt, n, bits, temp, err, s);
}

bool radix_sort_keys_u64(uint64_t *keys, uint64_t *keys_alt, int64_t n, int bits, void *temp,
                         unsigned *err, cudaStream_t s) {
  return radix_sort_impl<uint64_t, false>(keys, nullptr, keys_alt, nullptr, n, bits, temp, err, s);
}

}  // namespace wccg
