// Grid-wide barrier of the persistent (cooperative) kernels: a 64-bit
// arrival counter with a release add and an acquire poll, every wait bounded.
#pragma once

#include "mdpf_internal.cuh"

namespace mdpf {

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long atom_add_release(unsigned long long *p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
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
            atom_add_release(bar, 1ull);
            const unsigned long long t0 = globaltimer();
            unsigned int spins = 0;
            while (ld_acquire(bar) < target) {
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
