// Device helpers shared by the persistent kernels (sparse / matrix-free and dense): a grid-wide
// barrier whose waits are bounded, deterministic warp reductions and coherent vector loads.
#pragma once

#include "magnus_internal.cuh"

namespace mg {

constexpr unsigned kFull = 0xffffffffu;

static __device__ __forceinline__ long long globaltimer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
static __device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Coherent load of a vector entry that other blocks may have written before the last barrier.
static __device__ __forceinline__ double2 ldv(const double2 *p) { return __ldca(p); }

// Grid-wide barrier with a bounded wait.  Returns false (in every thread of the block) if the
// wait gave up or another block reported an error; the caller then leaves the kernel.  Every block
// adds 1 to one counter, block 0 adds 2^31 - (nblocks - 1): the counter's top bit flips exactly at
// the last arrival (its low 31 bits, zero at launch, return to zero for the next barrier), so the
// waiters only watch that bit and the last block does no extra atomic.
static __device__ __noinline__ bool grid_barrier(GridBar *bar, unsigned nblocks, long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned add = (blockIdx.x == 0) ? 0x80000000u - (nblocks - 1u) : 1u;
    __threadfence();
    const unsigned old = atomicAdd(&bar->count, add);
    if (!(((old + add) ^ old) & 0x80000000u)) {  // not the last arrival: wait for the flip
      const long long t0 = globaltimer_ns();
      for (unsigned spin = 0;; spin++) {
        if ((ld_acquire_gpu(&bar->count) ^ old) & 0x80000000u) break;
        if ((spin & 31u) == 31u) {
          if (*(volatile int *)&bar->error) { ok = 0; break; }
          if (globaltimer_ns() - t0 > limit_ns || spin > (1u << 28)) {
            atomicExch(&bar->error, 1);
            ok = 0;
            break;
          }
        }
        __nanosleep(20);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

static __device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

}  // namespace mg
