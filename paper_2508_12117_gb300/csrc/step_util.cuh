// Device helpers shared by the step kernels: error flag, deterministic warp /
// block reductions and scans, the bounded grid-wide barrier of the cooperative
// kernels and the early-exit test after a recorded error.
#pragma once
#include <cuda_runtime.h>

#include "spider.h"
#include "view.h"

namespace spider {
namespace {

__device__ __forceinline__ void set_error(int32_t* counters, int code) {
  atomicCAS(&counters[kCntError], 0, code);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum with a fixed reduction tree (deterministic). All threads get it.
template <typename T>
__device__ T block_sum(T v, T* sm /* >= 32 */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sm[wid] = v;
  __syncthreads();
  T t = lane < nw ? sm[lane] : T(0);
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sm[0] = t;
  __syncthreads();
  T r = sm[0];
  __syncthreads();
  return r;
}

// Exclusive block scan of small integers; returns the prefix, *total = sum.
__device__ int block_exscan(int v, int* sm /* >= 33 */, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) sm[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = lane < nw ? sm[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) sm[lane] = s;  // inclusive per-warp totals
  }
  __syncthreads();
  int warp_base = wid ? sm[wid - 1] : 0;
  *total = sm[nw - 1];
  __syncthreads();
  return warp_base + x - v;
}

// Software grid barrier for a cooperative launch, with a bounded wait
// (globaltimer, 2 s): on timeout the error flag is set and the caller returns.
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// The limit comes from the step parameters (spider_set_wait_limit_ns); a limit
// of 0 gives up at once whenever the barrier is not complete on arrival.  The
// error flag is checked on the first spin and every 1024 spins after it, so a
// CTA that finds another CTA's error leaves without waiting out its limit.
__device__ bool grid_barrier(int32_t* counters, uint64_t limit_ns) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    volatile int32_t* gen = counters + kCntBarGen;
    const int32_t g0 = *gen;
    __threadfence();
    const int32_t arrived = atomicAdd(&counters[kCntBarArrive], 1);
    ok = 1;
    if (arrived == (int)gridDim.x - 1) {
      counters[kCntBarArrive] = 0;
      __threadfence();
      atomicAdd(&counters[kCntBarGen], 1);
    } else {
      const uint64_t t0 = gtimer();
      for (uint32_t n = 0; *gen == g0; ++n) {
        if ((n & 1023u) == 0) {
          if (((volatile int32_t*)counters)[kCntError] != 0) { ok = 0; break; }
          if (gtimer() - t0 >= limit_ns) {
            set_error(counters, SPIDER_E_TIMEOUT);
            ok = 0;
            break;
          }
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// A kernel that runs after a bounded wait returns at once when an earlier
// kernel of the step recorded an error: the tables it would read (component
// labels, work lists) may be incomplete.
__device__ __forceinline__ bool aborted(const StepView& v) {
  return *((volatile const int32_t*)v.counters + kCntError) != 0;
}

// In a step solved through the piece inverses, the general component solver
// runs only when a unit exceeded the limits of that path (v.gate set).
__device__ __forceinline__ bool gated_off(const StepView& v) {
  return v.gate && *((volatile const int32_t*)v.gate) == 0;
}

// the same test taken once per CTA, for kernels with block-wide barriers
__device__ __forceinline__ bool aborted_cta(const StepView& v) {
  __shared__ int a;
  __syncthreads();
  if (threadIdx.x == 0) a = aborted(v) ? 1 : 0;
  __syncthreads();
  return a != 0;
}

}  // namespace
}  // namespace spider
