// Small device helpers: fixed-point accumulation and warp reductions.
#pragma once

#include "mdpf_internal.cuh"

namespace mdpf {

// v * 2^32 truncated toward zero to int64, from the bit pattern of v with
// integer operations only (the 64-bit float-to-integer conversion instruction
// runs on the FP64 pipe, which is narrow on this GPU).  |v| >= 2^31 saturates
// (a non-finite value too; callers flag those separately).
__device__ __forceinline__ long long fx_from_float(float v) {
    const unsigned int b = __float_as_uint(v);
    const int e = (int)((b >> 23) & 0xFFu);
    const unsigned long long m = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u);
    const int sh = e - 118;  // v * 2^32 = m * 2^(e - 127 - 23 + 32)
    unsigned long long r;
    if (e == 0 || sh <= -24) r = 0ull;
    else if (sh < 0) r = m >> (-sh);
    else if (sh <= 38) r = m << sh;
    else r = 0x7FFFFFFFFFFFFFFFull;
    return (b >> 31) ? -(long long)r : (long long)r;
}

// v * 2^32 as int64 fixed point, added atomically (two's complement wrap-around
// makes the unsigned add an exact signed add).
__device__ __forceinline__ void fx_add(unsigned long long *p, float v) {
    atomicAdd(p, (unsigned long long)fx_from_float(v));
}
__device__ __forceinline__ void fx_add_d(unsigned long long *p, double v) {
    atomicAdd(p, (unsigned long long)__double2ll_rn(v * 4294967296.0));
}
__device__ __forceinline__ double fx_val(unsigned long long u) { return (double)(long long)u * kFxInv; }

// Per-lane values of a warp, each rounded to fixed point and then summed as
// integers (exact, so the total does not depend on how values are grouped
// into warps), added by lane 0.
__device__ __forceinline__ void fx_warp_add_d(unsigned long long *p, double v) {
    long long q = __double2ll_rn(v * 4294967296.0);
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if ((threadIdx.x & 31) == 0 && q != 0) atomicAdd(p, (unsigned long long)q);
}

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace mdpf
