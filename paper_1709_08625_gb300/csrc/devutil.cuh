// devutil.cuh -- small device helpers shared by the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hlc_internal.h"

namespace hlc {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int dimv(const Dim& d, const int* ranks) {
  if (d.slot < 0) return d.n;
  const int r = ranks[d.slot];
  return r < d.n ? r : d.n;
}

__device__ __forceinline__ double* vptr(const Bases& B, const Mv& v) { return B.buf[v.buf] + v.off; }

__device__ __forceinline__ void record_error(int* status, int code, int detail) {
  if (atomicCAS(status, 0, code) == 0) status[1] = detail;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; all threads get the result.  `red` needs 33 entries.
template <class T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    T t = lane < nw ? red[lane] : T(0);
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// Block-wide argmax of |value| with ties to the smaller index; returns the
// index (or -1 when every candidate is excluded) and the value in *best.
__device__ __forceinline__ int block_argmax(double v, int idx, double* redv, int* redi, double* best) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi >= 0 && (idx < 0 || oi < idx))) {
      v = ov;
      idx = oi;
    }
  }
  __syncthreads();
  if (lane == 0) {
    redv[w] = v;
    redi[w] = idx;
  }
  __syncthreads();
  if (w == 0) {
    v = lane < nw ? redv[lane] : -1.0;
    idx = lane < nw ? redi[lane] : -1;
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ov > v || (ov == v && oi >= 0 && (idx < 0 || oi < idx))) {
        v = ov;
        idx = oi;
      }
    }
    if (lane == 0) {
      redv[32] = v;
      redi[32] = idx;
    }
  }
  __syncthreads();
  *best = redv[32];
  return redi[32];
}

// Bounded waits: a CTA gives up after kBarrierNs (or once another CTA has
// given up), records DEV_TIMEOUT, raises the abort flag and leaves.
constexpr unsigned long long kBarrierNs = 2000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier of `expected` CTAs in global memory.  Thread 0 of each CTA
// arrives on *count; the last to arrive resets it and advances *gen, which
// the others wait on.  Returns false when the wait gave up (time limit, or
// the abort flag raised by another CTA); the caller then leaves.
__device__ __forceinline__ bool bounded_barrier(unsigned int* count, unsigned int* gen_p, unsigned int expected,
                                                unsigned int* abort_p, int* status) {
  __shared__ int bb_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = gen_p;
    volatile unsigned int* abort = abort_p;
    int good = *abort == 0;
    if (good) {
      const unsigned int g = *gen;
      __threadfence();
      if (atomicAdd(count, 1u) == expected - 1) {
        atomicExch(count, 0u);
        __threadfence();
        atomicAdd(gen_p, 1u);
      } else {
        const unsigned long long t0 = global_ns();
        while (*gen == g) {
          if (*abort || global_ns() - t0 > kBarrierNs) {
            atomicExch(abort_p, 1u);
            record_error(status, DEV_TIMEOUT, 0);
            good = 0;
            break;
          }
          __nanosleep(32);
        }
      }
      __threadfence();
    }
    bb_ok = good;
  }
  __syncthreads();
  return bb_ok != 0;
}

}  // namespace hlc
