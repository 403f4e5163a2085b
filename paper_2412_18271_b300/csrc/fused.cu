// Fused learned force evaluation: features -> per-element MLP (tcgen05) ->
// force adjoint, one CTA per tile of up to 128 atoms of one element.  The
// features G and the input gradient dE/dG stay in shared and tensor memory;
// only positions, neighbour rows and weights are read, and only the per-atom
// energies and fixed-point forces are written.
//
//   phase A  the 16 compute warps take the tile's atoms one at a time (shared
//            counter): neighbours, features and range check (learned_terms.cuh);
//            each row goes to the GEMM operand in shared memory as BF16, in
//            the 128-byte-swizzled K-major layout TMA would have produced; rows
//            past the tile's atoms are zero
//   phase B  the GEMMs and their epilogues of the tensor-core MLP (as in
//            mlp_tc.cu, GEMM1's A operand now resident; layer 1's CELU output
//            enters GEMM2 as a BF16 pair hi + lo): energy per atom into E_row
//            and the energy slot, dE/dG into TMEM columns 0..383
//   phase C  per quarter tile: the 32 rows of dE/dG from TMEM into shared memory
//            (FP32, the adjoint's padded row layout), then the compute warps
//            take those atoms one at a time: neighbours again, chain rule to
//            fixed-point forces (learned_terms.cuh)
// The per-atom arithmetic is the per-stage kernels' own, so the result is the
// same bit for bit as features + k_mlp_tc + k_adjoint.
//
// Shared memory (dynamic, 1024-byte aligned):
//   [0, 96 KB)          G operand (6 x 16 KB) -> a1 / d2 / d1 -> quarter-tile g (32 x 424 FP32)
//   [96 KB, +118 KB)    per-warp scratch (phases A and C) or the weight ring (2 x 48 KB, phase B)
//   then b1, b2, W3, energy partials (4 KB), barriers and flags
// Warps 0-15: compute and epilogue (warp w reads TMEM lanes 32 (w mod 4) ..
// +31 and column group w / 4); warp 16: TMA producer; warp 17: TMEM
// allocation and MMA issue.  Every wait is bounded: on expiry the CTA records
// MDPF_STATUS_TIMEOUT, drains its copies and MMAs in flight, frees its tensor
// memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "learned.cuh"
#include "learned_terms.cuh"
#include "tc_util.cuh"

namespace mdpf {
namespace {

constexpr int kFuWarps = 16;
constexpr int kFuThreads = 32 * kFuWarps + 64;
constexpr int kFuProducer = kFuWarps, kFuMma = kFuWarps + 1;
constexpr int kFuStage = 48 * 1024;
constexpr int kFuRes = 96 * 1024;
constexpr int kFuChunk = 32;    // triplets staged per adjoint pass (no effect on the result)
using FuAdj = AdjScratch<kFuChunk>;
constexpr int kFuWarpScr = ((int)sizeof(NbrSmem) + (sizeof(FuAdj) > sizeof(TripStage) ? (int)sizeof(FuAdj)
                                                                                      : (int)sizeof(TripStage)) +
                            15) & ~15;
constexpr int kFuScr = kFuWarps * kFuWarpScr > 2 * kFuStage ? kFuWarps * kFuWarpScr : 2 * kFuStage;
constexpr int kFuOffScr = kFuRes;
constexpr int kFuOffPar = kFuOffScr + kFuScr;
constexpr int kFuOffBar = kFuOffPar + 4096;
constexpr int kFuSmem = kFuOffBar + 128 + 1024;
static_assert(6 * 16384 <= kFuRes && 32 * kGRow * 4 <= kFuRes, "resident region");
static_assert(kFuSmem <= 232448, "shared memory");
static_assert(sizeof(NbrSmem) % 16 == 0, "scratch alignment");

enum { F_FULL = 0, F_EMPTY = 2, F_ACC = 4, F_EPI = 5, F_DRAIN = 6 };

__device__ __forceinline__ void fu_sync() { asm volatile("bar.sync 1, %0;" ::"r"(32 * kFuWarps) : "memory"); }

// One BF16 value into row r, column c of the swizzled K-major operand.
__device__ __forceinline__ void st_operand1(unsigned char *res, int r, int c, float x) {
    const int cc = c & 63;
    unsigned char *p = res + (c >> 6) * 16384 + r * 128 + ((((cc >> 3) ^ (r & 7))) << 4) + (cc & 7) * 2;
    *reinterpret_cast<__nv_bfloat16 *>(p) = __float2bfloat16_rn(x);
}

__global__ void __launch_bounds__(kFuThreads, 1)
k_fused(LearnedDev L, FusedTiles T, const __grid_constant__ MlpMaps maps, const float4 *pos4,
        unsigned long long *fx, unsigned long long *efx, uint32_t *status) {
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned base (128-byte swizzle atoms), by pointer arithmetic on the shared array so that
    // the compiler keeps the shared address space for every access through it
    unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = smem_u32(sm);
    unsigned char *res = sm;
    float *sb1 = (float *)(sm + kFuOffPar), *sb2 = sb1 + 256, *sw3 = sb2 + 128, *sEp = sw3 + 128;
    const uint32_t bar0 = sbase + kFuOffBar;
    auto bar = [&](int k) { return bar0 + 8u * (uint32_t)k; };
    volatile uint32_t *s_tmem = (volatile uint32_t *)(sm + kFuOffBar + 64);
    volatile int *s_abort = (volatile int *)(sm + kFuOffBar + 68);
    volatile int *s_issued = (volatile int *)(sm + kFuOffBar + 72);
    volatile int *s_consumed = (volatile int *)(sm + kFuOffBar + 76);
    int *s_next = (int *)(sm + kFuOffBar + 80);   // atom counters: phase A, phase C quarters 0-3

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x;
    const int row0 = T.first[tile], cnt = T.count[tile], e = T.el[tile];

    if (tid == 0) {
        mbar_init(bar(F_FULL), 1);
        mbar_init(bar(F_FULL + 1), 1);
        mbar_init(bar(F_EMPTY), 1);
        mbar_init(bar(F_EMPTY + 1), 1);
        mbar_init(bar(F_ACC), 1);
        mbar_init(bar(F_EPI), 32 * kFuWarps);
        mbar_init(bar(F_DRAIN), 1);
        *s_abort = 0;
        *s_issued = 0;
        *s_consumed = 0;
        s_next[0] = s_next[1] = s_next[2] = s_next[3] = s_next[4] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kFuMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32((const void *)s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int q = tid; q < 256; q += kFuThreads) sb1[q] = L.b1[e * kH1 + q];
    for (int q = tid; q < 128; q += kFuThreads) {
        sb2[q] = L.b2[e * kH2 + q];
        sw3[q] = L.W3[e * kH2 + q];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    // ---------------- phase A: features -> BF16 operand rows
    if (warp < kFuWarps) {
        unsigned char *scr = sm + kFuOffScr + warp * kFuWarpScr;
        NbrSmem &sn = *reinterpret_cast<NbrSmem *>(scr);
        TripStage &ts = *reinterpret_cast<TripStage *>(scr + sizeof(NbrSmem));
        bool out = false;
        for (;;) {
            int r = 0;
            if (lane == 0) r = atomicAdd(&s_next[0], 1);
            r = __shfl_sync(0xffffffffu, r, 0);
            if (r >= kRowTile) break;
            float v[12];
            if (r < cnt) {
                const int i = L.atom_of[row0 + r];
                int nc, nr, na;
                load_neighbours<true>(L, pos4, i, sn, lane, nc, nr, na);
                feature_row(sn, nr, na, ts, lane, v);
                if (L.lo != nullptr) {
#pragma unroll
                    for (int b = 0; b < 12; ++b) {
                        const int f = 32 * b + lane;
                        out |= (v[b] < L.lo[e * kNFeat + f]) || (v[b] > L.hi[e * kNFeat + f]);
                    }
                }
            } else {
#pragma unroll
                for (int b = 0; b < 12; ++b) v[b] = 0.f;
            }
#pragma unroll
            for (int b = 0; b < 12; ++b) st_operand1(res, r, 32 * b + lane, v[b]);
            __syncwarp();
        }
        if (__any_sync(0xffffffffu, out) && lane == 0) atomicOr(&L.lflags[1], 1u);
        proxy_fence();   // operand rows written through the generic proxy, read by the MMA
    }
    __syncthreads();     // operand complete; the scratch becomes the weight ring

    // ---------------- phase B: the MLP
    if (warp == kFuProducer) {
        if (lane == 0) {
            for (int c = 0; c < 20; ++c) {
                const int s = c & 1;
                if (c >= 2 && !mbar_wait(bar(F_EMPTY + s), ((c >> 1) - 1) & 1, s_abort)) break;
                // phases: 0 GEMM1, 1 GEMM2 (hi), 2 GEMM2 (lo), 3 GEMM3, 4 GEMM4
                const int g = c < 6 ? 0 : (c < 10 ? 1 : (c < 14 ? 2 : (c < 16 ? 3 : 4)));
                const int kc = c - (g == 0 ? 0 : (g == 1 ? 6 : (g == 2 ? 10 : (g == 3 ? 14 : 16))));
                const uint32_t B = sbase + kFuOffScr + s * kFuStage;
                const int x = kc * 64;
                const uint32_t fb = bar(F_FULL + s);
                if (g == 0) {
                    mbar_expect_tx(fb, 32 * 1024);
                    tma_2d(B, &maps.w1, x, e * kH1, fb);
                    tma_2d(B + 16384, &maps.w1, x, e * kH1 + 128, fb);
                } else if (g == 1 || g == 2) {
                    mbar_expect_tx(fb, 16 * 1024);
                    tma_2d(B, &maps.w2, x, e * kH2, fb);
                } else if (g == 3) {
                    mbar_expect_tx(fb, 32 * 1024);
                    tma_2d(B, &maps.w2t, x, e * kH1, fb);
                    tma_2d(B + 16384, &maps.w2t, x, e * kH1 + 128, fb);
                } else {
                    mbar_expect_tx(fb, 48 * 1024);
                    tma_2d(B, &maps.w1t, x, e * kNFeat, fb);
                    tma_2d(B + 16384, &maps.w1t, x, e * kNFeat + 128, fb);
                    tma_2d(B + 32768, &maps.w1t, x, e * kNFeat + 256, fb);
                }
                *s_issued = c + 1;
            }
        }
    } else if (warp == kFuMma) {
        if (lane == 0) {
            const uint32_t i256 = idesc_bf16(256), i128 = idesc_bf16(128);
            const uint32_t ra = sbase;
            int c = 0;
            bool ok = true;
            for (int g = 0; g < 5 && ok; ++g) {
                if (g > 0) {
                    if (!mbar_wait(bar(F_EPI), (g - 1) & 1, s_abort)) break;
                    tc_fence_after();
                }
                const int nk = g == 0 ? 6 : (g == 3 ? 2 : 4);
                for (int kc = 0; kc < nk; ++kc, ++c) {
                    const int s = c & 1;
                    if (!mbar_wait(bar(F_FULL + s), (c >> 1) & 1, s_abort)) {
                        ok = false;
                        break;
                    }
                    *s_consumed = c + 1;
                    tc_fence_after();
                    const uint32_t B = sbase + kFuOffScr + s * kFuStage;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t acc = g == 2 || (kc | k) != 0;   // GEMM2 (lo) adds onto GEMM2 (hi)
                        const uint32_t ko = 32u * k;
                        const uint64_t a = sdesc(ra + kc * 16384 + ko);
                        if (g == 0) {
                            mma_bf16(tmem, a, sdesc(B + ko), i256, acc);
                        } else if (g == 1 || g == 2) {
                            mma_bf16(tmem + 256, a, sdesc(B + ko), i128, acc);
                        } else if (g == 3) {
                            mma_bf16(tmem + 256, a, sdesc(B + ko), i256, acc);
                        } else {
                            mma_bf16(tmem, a, sdesc(B + ko), i256, acc);
                            mma_bf16(tmem + 256, a, sdesc(B + 32768 + ko), i128, acc);
                        }
                    }
                    mma_commit(bar(F_EMPTY + s));
                }
                if (ok) mma_commit(bar(F_ACC));
            }
        }
    } else {
        // ---------------- epilogues, then phase C: lane = tile row (TMEM lane), column group cg
        const int q4 = warp & 3, cg = warp >> 2;
        const int r = 32 * q4 + lane;
        const uint32_t tl = tmem + ((uint32_t)(32 * q4) << 16);
        float v[32], h[32];
        bool ok = true;
        // epi1: a1 = celu(H1 + b1): its BF16 value over the (consumed) G operand, a1 (FP32) over H1 in TMEM
        if ((ok = warp_wait(bar(F_ACC), 0, s_abort))) {
            tc_fence_after();
#pragma unroll 1
            for (int cc = 2 * cg; cc < 2 * cg + 2; ++cc) {
                tmem_ld32(tl + cc * 32, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float x = v[j] + sb1[cc * 32 + j];
                    v[j] = celu_e(x, exp10x_neg(x));
                }
                st_operand32(res, r, cc * 32, v);
                tmem_st32(tl + cc * 32, v);
            }
            proxy_fence();
            tc_fence_before();
            mbar_arrive(bar(F_EPI));
        }
        // epi1b: once GEMM2 has read the operand, the BF16 residuals a1 - bf16(a1) replace it
        if (ok && (ok = warp_wait(bar(F_ACC), 1, s_abort))) {
            tc_fence_after();
#pragma unroll 1
            for (int cc = 2 * cg; cc < 2 * cg + 2; ++cc) {
                tmem_ld32(tl + cc * 32, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = bf16_residual(v[j]);
                st_operand32(res, r, cc * 32, v);
            }
            proxy_fence();
            tc_fence_before();
            mbar_arrive(bar(F_EPI));
        }
        // epi2: energy partial and d2 = bf16(W3 * celu'(H2 + b2))
        if (ok && (ok = warp_wait(bar(F_ACC), 0, s_abort))) {
            tc_fence_after();
            float E = 0.f;
            tmem_ld32(tl + 256 + cg * 32, v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int c = cg * 32 + j;
                const float hv = v[j] + sb2[c], ex = exp10x_neg(hv);
                E = fmaf(sw3[c], celu_e(hv, ex), E);
                v[j] = sw3[c] * dcelu_e(hv, ex);
            }
            st_operand32(res, r, cg * 32, v);
            sEp[cg * 128 + r] = E;
            proxy_fence();
            tc_fence_before();
            mbar_arrive(bar(F_EPI));
        }
        fu_sync();   // energy partials of the four column groups are in shared memory
        if (ok && cg == 0) {
            const float E = ((sEp[r] + sEp[128 + r]) + sEp[256 + r]) + sEp[384 + r];
            const double Er = r < cnt ? (double)E + (double)L.b3[e] + L.e0[e] : 0.0;
            if (r < cnt) L.E_row[row0 + r] = Er;
            if (efx != nullptr) fx_warp_add_d(&efx[E_LEARN], Er);
        }
        // epi3: d1 = bf16(P1 * celu'(H1 + b1))
        if (ok && (ok = warp_wait(bar(F_ACC), 1, s_abort))) {
            tc_fence_after();
#pragma unroll 1
            for (int cc = 2 * cg; cc < 2 * cg + 2; ++cc) {
                tmem_ld32(tl + 256 + cc * 32, v);
                tmem_ld32(tl + cc * 32, h);   // a1, stored by epi1
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = v[j] * dcelu_from_a(h[j]);
                st_operand32(res, r, cc * 32, v);
            }
            proxy_fence();
            tc_fence_before();
            mbar_arrive(bar(F_EPI));
        }
        // GEMM4 done: g = dE/dG in TMEM columns 0..383; the operand region and the ring are free
        if (ok && (ok = warp_wait(bar(F_ACC), 0, s_abort))) tc_fence_after();

        // ---------------- phase C
        unsigned char *scr = sm + kFuOffScr + warp * kFuWarpScr;
        NbrSmem &sn = *reinterpret_cast<NbrSmem *>(scr);
        FuAdj &A = *reinterpret_cast<FuAdj *>(scr + sizeof(NbrSmem));
        float *gst = reinterpret_cast<float *>(res);
#pragma unroll 1
        for (int hh = 0; hh < 4; ++hh) {
            if (32 * hh >= cnt) break;   // the same in every warp
            if (ok && q4 == hh) {
                float *dst = gst + lane * kGRow;
#pragma unroll 1
                for (int cc = 3 * cg; cc < 3 * cg + 3; ++cc) {
                    tmem_ld32(tl + cc * 32, v);
                    float *d = dst + (cc < 2 ? 32 * cc : 64 + kAngStride * (cc - 2));
                    // rounded to BF16 as the per-stage path stores dE/dG, so both give the same forces
#pragma unroll
                    for (int j = 0; j < 32; ++j) d[j] = __bfloat162float(__float2bfloat16_rn(v[j]));
                }
            }
            fu_sync();
            for (;;) {
                int k = 0;
                if (lane == 0) k = atomicAdd(&s_next[1 + hh], 1);
                k = __shfl_sync(0xffffffffu, k, 0);
                const int rr = 32 * hh + k;
                if (k >= 32 || rr >= cnt || *s_abort) break;
                const int i = L.atom_of[row0 + rr];
                int nc, nr, na;
                load_neighbours<false>(L, pos4, i, sn, lane, nc, nr, na);
                adjoint_atom(i, sn, nc, nr, na, gst + k * kGRow, A, fx, lane, make_float2(L.core_a, L.core_rc),
                             efx != nullptr ? efx + E_LEARN : nullptr);
            }
            fu_sync();   // the quarter's g rows are no longer read
        }
        tc_fence_before();
    }
    __syncthreads();
    if (*s_abort) {
        if (tid == 0) {
            for (int c = *s_consumed; c < *s_issued; ++c) mbar_drain(bar(F_FULL + (c & 1)), (c >> 1) & 1);
            atomicOr(status, MDPF_STATUS_TIMEOUT);
            atomicOr(&L.lflags[3], 1u);
        }
        if (tid == 32 * kFuMma) {
            mma_commit(bar(F_DRAIN));
            mbar_drain(bar(F_DRAIN), 0);
        }
        __syncthreads();
    }
    if (warp == kFuMma) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

}  // namespace

cudaError_t learned_fused_prepare() {
    return cudaFuncSetAttribute(k_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, kFuSmem);
}

cudaError_t learned_fused(const LearnedDev &L, const FusedTiles &T, const MlpMaps &maps, const float4 *pos4,
                          unsigned long long *fx, unsigned long long *efx, uint32_t *status, cudaStream_t s) {
    if (T.n > 0) k_fused<<<T.n, kFuThreads, kFuSmem, s>>>(L, T, maps, pos4, fx, efx, status);
    return cudaGetLastError();
}

}  // namespace mdpf
