// grid_sync.cuh -- the bounded two-level grid barrier of the persistent
// (cooperative) kernels.
//
// Blocks arrive on one of kBarGroups group counters (each on its own
// 128-byte line); the last arrival of a group adds one to the global
// counter, which every block polls.  The wait is bounded: at most
// kBarrierSpins polls and kBarrierTimeoutNs of %globaltimer, and it gives up
// at once when another block has recorded an error; a block that gives up
// records error code 4 and the caller stops stepping, so a broken grid ends
// with a status the host reads instead of hanging.
#pragma once
#include <cstdint>

namespace sbqa {

constexpr unsigned kBarrierSpins = 1u << 24;     // polls per grid barrier at most
constexpr uint64_t kBarrierTimeoutNs = 1000000000;  // and at most 1 s of waiting (%globaltimer)
// Two-level grid barrier: blocks arrive on one of kBarGroups group counters
// (each on its own 128-byte line); the last arrival of a group adds one to
// the global counter, which every block polls.  Counter words: global at 0,
// group g at kBarStride * (g + 1).
constexpr unsigned kBarGroups = 32, kBarStride = 32;
inline int grid_barrier_words() { return int(kBarStride * (kBarGroups + 1)); }

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// skip: this block does not arrive (the test hook), so every block's wait
// runs out and the launch ends with error code 4.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned k, int *err, bool skip = false) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    // barrier number k (1, 2, ...): a block's fence + group atomic releases its
    // writes, the group's last arrival (atomic, fence) acquires them and
    // releases them again with its fence + global atomic, the poll acquires
    const unsigned G = gridDim.x < kBarGroups ? gridDim.x : kBarGroups;
    const unsigned g = blockIdx.x % G;
    const unsigned size_g = (gridDim.x - g + G - 1) / G;  // blocks b with b % G == g
    __threadfence();
    if (!skip) {
      const unsigned old = atomicAdd(bar + kBarStride * (g + 1), 1u);
      if (old + 1 == size_g * k) {  // last arrival of the group
        __threadfence();
        atomicAdd(bar, 1u);
      }
    }
    const unsigned target = G * k;
    const uint64_t t0 = globaltimer_ns();
    unsigned v = 0;
    unsigned it = 0;
    bool ok = false;
    for (; it < kBarrierSpins; ++it) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) {
        ok = true;
        break;
      }
      if ((it & 15) == 15 && (globaltimer_ns() - t0 > kBarrierTimeoutNs || *(volatile int *)err != 0)) break;
      __nanosleep(it < 64 ? 32 : 128);
    }
    s_ok = ok;
    if (!s_ok) atomicCAS(err, 0, 4);
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace sbqa
