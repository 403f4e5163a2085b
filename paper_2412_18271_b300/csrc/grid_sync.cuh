// Grid-wide barrier of the persistent (cooperative) kernels: a 64-bit
// arrival counter with an acq_rel add and an acquire poll, every wait bounded.
// The add returns the count before it, so the last block to arrive knows the
// barrier is complete (its acq_rel add has synchronised with every earlier
// release) and does not poll.
#pragma once

#include "mdpf_internal.cuh"

namespace mdpf {

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long atom_add_acq_rel(unsigned long long *p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.acq_rel.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier number `epoch` (1, 2, ...).  Returns false in every
// thread of the block if this block gave up waiting.
__device__ __forceinline__ bool grid_barrier(unsigned long long *bar, unsigned long long epoch, uint32_t *status,
                                             long long limit_ns, int *s_fail) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int fail = 0;
        if (gridDim.x > 1) {
            const unsigned long long target = epoch * gridDim.x;
            const unsigned long long old = atom_add_acq_rel(bar, 1ull);
            const unsigned long long t0 = globaltimer();
            unsigned int spins = 0;
            while (old + 1 < target && ld_acquire(bar) < target) {
                if ((++spins & 31u) == 0u && (long long)(globaltimer() - t0) > limit_ns) {
                    atomicOr(status, MDPF_STATUS_TIMEOUT);
                    fail = 1;
                    break;
                }
            }
        }
        *s_fail = fail;
    }
    __syncthreads();
    return *s_fail == 0;
}

}  // namespace mdpf
