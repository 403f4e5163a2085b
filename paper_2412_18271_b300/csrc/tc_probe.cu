// Check of the tensor-core operand path that the MLP kernels share (tests
// only): one CTA stores A [128 x 64] and B [n x 64] (BF16) into its shared
// memory with the swizzled K-major store the MLP epilogues use for the
// operands they write (st_operand32), at chosen byte offsets, issues the four
// tcgen05 MMAs of one 64-wide K chunk with the descriptors the MLP kernels
// use (sdesc, idesc_bf16, mma_bf16), and reads D = A B^T back from tensor
// memory with tcgen05.ld (tmem_ld32).  Run over every operand placement, it
// pins those helpers against a host product wherever an operand can sit in
// the 227 KB of a CTA.
//
// Warps 0-3, thread t owns row t of A and rows t, t + 128 of B, and TMEM
// lane t of D.  The completion wait is bounded (kTcWaitNs); on expiry the
// kernel records MDPF_STATUS_TIMEOUT, waits (bounded) once more for the MMAs
// before freeing its tensor memory, and writes no D.
#include <cuda.h>
#include <cuda_bf16.h>

#include "mdpf_internal.cuh"
#include "tc_util.cuh"

namespace mdpf {
namespace {

constexpr int kProbeThreads = 128;
constexpr int kProbeDynSmem = 232448 - 256;   // the opt-in maximum less this kernel's static shared memory
constexpr int kProbeCap = 225 * 1024;         // operand bytes addressable after the 1024-byte alignment

__global__ void __launch_bounds__(kProbeThreads, 1)
k_tc_probe(const __nv_bfloat16 *A, const __nv_bfloat16 *B, float *D, int n, int a_off, int b_off, uint32_t *status) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long s_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = smem_u32(sm);
    const uint32_t bar = smem_u32(&s_bar);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;

    if (t == 0) {
        mbar_init(bar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // the operands, as the epilogues write theirs: 32 values at a time, rounded to BF16, swizzled
    float v[32];
    for (int r = t; r < 128 + n; r += kProbeThreads) {
        const bool isA = r < 128;
        const int row = isA ? r : r - 128;
        const __nv_bfloat16 *src = (isA ? A : B) + (size_t)row * 64;
        unsigned char *dst = sm + (isA ? a_off : b_off);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = __bfloat162float(src[32 * h + j]);
            st_operand32(dst, row, 32 * h, v);
        }
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (t == 0) {
        const uint32_t idesc = idesc_bf16(n);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            mma_bf16(tmem, sdesc(sbase + a_off + 32u * k), sdesc(sbase + b_off + 32u * k), idesc, k > 0 ? 1u : 0u);
        mma_commit(bar);
    }
    const bool ok = warp_wait(bar, 0, &s_abort);
    if (ok) {
        tc_fence_after();
        const int row = 32 * warp + lane;
        for (int c0 = 0; c0 < n; c0 += 32) {
            tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) D[(size_t)row * n + c0 + j] = v[j];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (s_abort) {
        if (t == 0) {
            atomicOr(status, MDPF_STATUS_TIMEOUT);
            mbar_drain(bar, 0);
        }
        __syncthreads();
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
    }
}

}  // namespace
}  // namespace mdpf

using namespace mdpf;

extern "C" int mdpf_debug_tc_probe(const void *d_a, const void *d_b, float *d_d, int32_t n, int32_t a_off,
                                   int32_t b_off, uint32_t *d_status, void *cuda_stream) {
    if (!d_a || !d_b || !d_d || !d_status) return fail(nullptr, MDPF_ERR_INVALID_ARG, "mdpf_debug_tc_probe: NULL pointer");
    if (n != 128 && n != 256) return fail(nullptr, MDPF_ERR_INVALID_ARG, "mdpf_debug_tc_probe: n must be 128 or 256");
    const long long a0 = a_off, a1 = a0 + 128 * 128, b0 = b_off, b1 = b0 + (long long)n * 128;
    if (a0 < 0 || b0 < 0 || a0 % 1024 != 0 || b0 % 1024 != 0 || a1 > kProbeCap || b1 > kProbeCap)
        return fail(nullptr, MDPF_ERR_INVALID_ARG,
                    "mdpf_debug_tc_probe: offsets must be multiples of 1024 with both operands inside 225 KB");
    if (a0 < b1 && b0 < a1) return fail(nullptr, MDPF_ERR_INVALID_ARG, "mdpf_debug_tc_probe: the operands overlap");
    cudaError_t e = cudaFuncSetAttribute(k_tc_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeDynSmem);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaFuncSetAttribute(k_tc_probe)");
    k_tc_probe<<<1, kProbeThreads, kProbeDynSmem, (cudaStream_t)cuda_stream>>>(
        static_cast<const __nv_bfloat16 *>(d_a), static_cast<const __nv_bfloat16 *>(d_b), d_d, n, a_off, b_off,
        d_status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "mdpf_debug_tc_probe launch");
    return MDPF_OK;
}
