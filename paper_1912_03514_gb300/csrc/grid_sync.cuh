// Grid-wide barrier for kernels whose blocks are all resident (cooperative
// launches), with a bounded wait.
//
// The barrier word lives in global memory and is zero before the first
// launch that uses it.  Block 0 adds 2³¹ − (G − 1), every other block adds 1,
// so the word's top bit flips exactly when the last of the G blocks arrives
// and the low bits return to their value before the barrier.  Each block
// reads the top bit before its first arrival (no flip can have happened yet,
// since a flip needs this block's arrival) and toggles its expectation per
// barrier; arrival is a release reduction (nothing to wait for), the wait an
// acquire load.  A wait that runs out (2 s by default) returns false so that the kernel
// can stop with an error instead of hanging; the word is then inconsistent
// and must be zeroed before the next launch.
#pragma once

#include "internal.h"

namespace mihs {

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct GridBarrier {
  unsigned int* word;
  unsigned int expect;  // top bit after the next barrier (thread 0 only)
};

// Call from thread 0 before this block's first arrival.
__device__ __forceinline__ void grid_barrier_init(GridBarrier& gb, unsigned int* word) {
  gb.word = word;
  gb.expect = ld_acquire_gpu(word) >> 31;
}

// Every thread of every block calls it; returns false in every thread of the
// block if the wait ran out (after limit_ns).
__device__ __forceinline__ bool grid_barrier(GridBarrier& gb, int* s_ok, uint64_t limit_ns = kWaitLimitNs) {
  __syncthreads();  // this block's writes precede thread 0's release
  if (threadIdx.x == 0) {
    const unsigned int add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
    gb.expect ^= 1u;
    red_release_add(gb.word, add);
    int ok = 1;
    if ((ld_acquire_gpu(gb.word) >> 31) != gb.expect) {
      const uint64_t t0 = global_timer_ns();
      for (uint32_t i = 1;; ++i) {
        if ((ld_acquire_gpu(gb.word) >> 31) == gb.expect) break;
        if ((i & 63u) == 0 && global_timer_ns() - t0 > limit_ns) {
          ok = 0;
          break;
        }
      }
    }
    *s_ok = ok;
  }
  __syncthreads();  // the other blocks' writes are visible to this block
  return *s_ok != 0;
}

}  // namespace mihs
