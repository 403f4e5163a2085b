// Small device helpers: fixed-point accumulation and warp reductions.
#pragma once

#include "mdpf_internal.cuh"

namespace mdpf {

// value * 2^32 rounded to int64, added atomically (two's complement wrap-around
// makes the unsigned add an exact signed add).
__device__ __forceinline__ void fx_add(unsigned long long *p, float v) {
    atomicAdd(p, (unsigned long long)__float2ll_rn(v * 4294967296.0f));
}
__device__ __forceinline__ void fx_add_d(unsigned long long *p, double v) {
    atomicAdd(p, (unsigned long long)__double2ll_rn(v * 4294967296.0));
}
__device__ __forceinline__ double fx_val(unsigned long long u) { return (double)(long long)u * kFxInv; }

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace mdpf
