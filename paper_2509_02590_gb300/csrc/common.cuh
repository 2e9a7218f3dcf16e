// common.cuh -- error handling and small device helpers shared by the
// library's translation units (CUDA path only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/wcc.h"

namespace wccg {

// Host-side failure carried to the C ABI boundary, where it becomes a status
// code plus the thread-local message of wcc_last_error().
struct Error {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string &msg);
void set_last_error(const std::string &msg);  // the thread-local message of wcc_last_error()

#define WCC_CUDA(call)                                                               \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      ::wccg::fail(e_ == cudaErrorMemoryAllocation ? WCC_ERR_OOM : WCC_ERR_CUDA,     \
                   std::string(#call) + " failed: " + cudaGetErrorString(e_));       \
  } while (0)

// Device-side error word bits (written by kernels with atomicOr, read by the
// host after the run).
enum : uint32_t {
  DERR_TIMEOUT = 1u,    // a bounded spin-wait ran out
  DERR_CAPACITY = 2u,   // an internal buffer bound was exceeded
  DERR_INTERNAL = 4u,   // a consistency check failed
  DERR_INVALID = 8u,    // malformed input found on the device
};

constexpr unsigned FULL = 0xffffffffu;

// The 32-bit tag a vertex's slot holds for the queue index of its current
// item.  Never all ones (the "no item" value), and unique among any 2^32-1
// consecutive indices, which outlive every request.
__host__ __device__ __forceinline__ uint32_t queue_tag(unsigned long long q) {
  return (uint32_t)(q % 0xffffffffull);
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T x = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += x;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T x = __shfl_xor_sync(FULL, v, o);
    v = x > v ? x : v;
  }
  return v;
}

// Exclusive scan across a thread block of BLOCK threads (all must call).
// smem: at least BLOCK/32 + 1 elements.  Returns the exclusive prefix of v;
// *total receives the block sum.
template <int BLOCK, typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *total, T *smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = BLOCK / 32;
  T inc = warp_inclusive_scan(v);
  if (lane == 31) smem[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < NW ? smem[lane] : T(0);
    T wi = warp_inclusive_scan(w);
    if (lane < NW) smem[lane] = wi - w;
    if (lane == NW - 1) smem[NW] = wi;
  }
  __syncthreads();
  T r = smem[warp] + inc - v;
  *total = smem[NW];
  __syncthreads();
  return r;
}

}  // namespace wccg
