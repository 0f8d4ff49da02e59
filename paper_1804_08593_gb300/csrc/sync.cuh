// Barrier among the CTAs of a cooperative launch (or a fixed subset of them), with a bounded
// wait: no CTA ever spins forever on a peer.
#pragma once

#include "tc_m5.cuh"

namespace dwf {

// The counter counts arrivals; `target` is the number of arrivals that completes this
// barrier (barrier k of a group of C CTAs: (k + 1) C, counter zero at launch).  Gives up
// after the wait limit (the default when wait_ns is 0), records the error and returns false
// in every thread of the CTA, which then leaves the kernel; its peers then give up at their
// next barrier, so the launch always ends.  Writes before the barrier are visible to every
// CTA after it (release by a fence and the arrival, acquire by the waiting thread, then the
// CTA barrier); data written during the launch must not be read through the non-coherent
// cache.
__device__ __forceinline__ bool slot_barrier(unsigned* ctr, unsigned target,
                                             unsigned long long wait_ns, int* err) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    int ok = 1;
    const unsigned long long lim = wait_ns ? wait_ns : tc::DEFAULT_WAIT_NS;
    const unsigned long long t0 = tc::globaltimer_ns();
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
      if (v >= target) break;
      if (tc::globaltimer_ns() - t0 > lim) {
        ok = 0;
        if (err) atomicExch(err, 1);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

}  // namespace dwf
