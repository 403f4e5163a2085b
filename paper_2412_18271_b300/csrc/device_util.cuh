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
// An int64 as the exact double.  For |i| < 2^51 by the exponent-bias
// method: adding i to the bit pattern of 1.5 * 2^52 places it in the mantissa
// of a double in [2^52, 2^53), and one exact subtraction removes the bias
// (one FP64 addition instead of the 64-bit integer-to-float conversion; FP64
// work is scarce on this GPU).  Larger values take the conversion instruction.
__device__ __forceinline__ double fx_exact(long long i) {
    if (i > -(1ll << 51) && i < (1ll << 51))
        return __longlong_as_double(i + 0x4338000000000000ll) - 6755399441055744.0;
    return (double)i;
}

// x * 2^32 rounded to the nearest int64 by the same exponent-bias method
// (|x| < 2^19), else the conversion instruction.
__device__ __forceinline__ long long fx_from_double(double x) {
    const double y = x * kFxScale;
    if (y > -2251799813685248.0 && y < 2251799813685248.0)
        return __double_as_longlong(y + 6755399441055744.0) - 0x4338000000000000ll;
    return __double2ll_rn(y);
}

// Finite test of a double on its bits (integer instructions only).
__device__ __forceinline__ bool finite_bits(double v) {
    return (__double_as_longlong(v) & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}

__device__ __forceinline__ double fx_val(unsigned long long u) {
    return fx_exact((long long)u) * kFxInv;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-lane values of a warp, each rounded to fixed point and then summed as
// integers (exact, so the total does not depend on how values are grouped
// into warps), added by lane 0.
__device__ __forceinline__ void fx_warp_add_d(unsigned long long *p, double v) {
    long long q = __double2ll_rn(v * 4294967296.0);
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if ((threadIdx.x & 31) == 0 && q != 0) atomicAdd(p, (unsigned long long)q);
}

// Butterfly sum over a warp: every lane ends with the same value (IEEE addition commutes), in a fixed order.
__device__ __forceinline__ float warp_sum_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace mdpf
