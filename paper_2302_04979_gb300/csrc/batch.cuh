// Grid barrier of the persistent batched-step kernels (kernels.cu: FP64 step,
// kernels_f32.cu: refined mixed step).
#pragma once

#include <cuda_runtime.h>

namespace smx {

__device__ __forceinline__ unsigned long long batch_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// All CTAs are co-resident (cooperative launch).  The wait is bounded (wait_ns,
// one second by default); a CTA that gives up sets bit 1 of the status word and
// the whole launch returns after the barrier.
__device__ inline bool batch_barrier(unsigned* bar, unsigned* status, unsigned nblocks, unsigned long long wait_ns) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            bar[0] = 0;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = batch_ns();
            while (*gen == g) {
                if (batch_ns() - t0 > wait_ns) {
                    ok = 0;
                    atomicOr(status, 2u);
                    break;
                }
            }
        }
        __threadfence();
        ok_s = ok && !(*(volatile unsigned*)status & 2u);
    }
    __syncthreads();
    return ok_s != 0;
}

}  // namespace smx
