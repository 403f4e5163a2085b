// Per-element MLP on the 5th-generation tensor cores: forward energy and the
// input gradient dE/dG for one 128-row tile of same-element atoms per CTA.
//
//   GEMM1  H1 = G  W1^T      [128 x 256], K = 384   (TMEM columns   0..255)
//   epi1   a1 = celu(H1 + b1); hi = bf16(a1)          -> shared A operand; a1 (FP32) -> TMEM 0..255
//   GEMM2  H2 = hi W2^T      [128 x 128], K = 256   (TMEM columns 256..383)
//   epi1b  lo = bf16(a1 - hi)                         -> shared A operand (a1 read back from TMEM)
//   GEMM2' H2 += lo W2^T     (the same W2 chunks again)
//   epi2   E  = W3 . celu(H2 + b2) + b3 + e0;  d2 = bf16(W3 * celu'(H2 + b2))
//   GEMM3  P1 = d2 W2        [128 x 256], K = 128   (TMEM columns 256..511)
//   epi3   d1 = bf16(P1 * celu'(H1 + b1))           (celu' = 1 or 10 a1 + 1 from a1 in TMEM)
//   GEMM4  g  = d1 W1        [128 x 384], K = 256   (TMEM columns 0..255, 256..383)
//   epi4   g -> global, rounded to BF16 (the adjoint's input; half the bytes of FP32)
// a1 enters GEMM2 as the pair hi + lo of BF16 values (16 significant bits):
// rounding a1 to one BF16 value biases the energy through the curvature of
// the second CELU (~2e-3 kcal/mol/atom on a trained model, all atoms the same
// sign), the pair removes that bias; every other GEMM input is one BF16 value.
//
// Operands are BF16 in shared memory in the 128-byte-swizzled K-major layout
// (8-row x 128-byte atoms, the 16-byte unit index XOR-ed with the row index
// mod 8); weight and feature K-chunks of 64 arrive by TMA through a three-stage
// ring of 48 KB, the intermediate operands (a1, d2, d1) are written by the epilogue
// warps straight into that layout.  Accumulation is FP32 in tensor memory.
// Warps 0-15: epilogue (warp w reads TMEM lanes 32 (w mod 4) .. +31, i.e. those
// tile rows, and column group w / 4); warp 16: TMA producer; warp 17: TMEM
// allocation and MMA issue.
// Every wait is bounded (kTcWaitNs): on expiry the CTA records
// MDPF_STATUS_TIMEOUT, drains its copies and MMAs in flight, frees its tensor
// memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "learned.cuh"
#include "tc_util.cuh"

namespace mdpf {
namespace {

constexpr int kEpiWarps = 16;
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kTcThreads = kEpiThreads + 64;
constexpr int kProducerWarp = kEpiWarps, kMmaWarp = kEpiWarps + 1;
constexpr int kStageBytes = 48 * 1024;     // GEMM1: [G 16 KB][W1 32 KB]; GEMM2-4: [W 16/32/48 KB]
constexpr int kStages = 3;
constexpr int kResBytes = 64 * 1024;       // resident A operand: a1 / d2 / d1
constexpr int kOffRes = kStages * kStageBytes;
constexpr int kOffPar = kOffRes + kResBytes;   // b1[256] b2[128] w3[128] E partials[4][128], FP32
constexpr int kOffBar = kOffPar + 4096;
constexpr int kGStrideW = 20;                  // padded row (32-bit words) of a 32 x 32 BF16 staging block of g
constexpr int kSmemBytes = kOffBar + 128 + 1024;   // barriers/flags + 1024-byte alignment slack
static_assert(kSmemBytes <= 232448, "shared memory");
static_assert(kEpiWarps * 32 * kGStrideW * 4 <= kStages * kStageBytes, "g staging fits in the ring");
constexpr int kChunks = 20;                    // 6 + 4 + 4 + 2 + 4 K-chunks of 64 (GEMM1, GEMM2, GEMM2', 3, 4)
constexpr int kPhases = 5;

// barrier block: full[kStages] empty[kStages] acc epi drain, then (from byte 96) tmem address, abort
// flag, issued, consumed
enum { B_FULL = 0, B_EMPTY = kStages, B_ACC = 2 * kStages, B_EPI = 2 * kStages + 1, B_DRAIN = 2 * kStages + 2 };
static_assert(8 * (B_DRAIN + 1) <= 96, "barrier block");

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"r"(kEpiThreads) : "memory"); }

// K-chunk c of the operand stream: phase g (0 GEMM1, 1 GEMM2 with hi, 2 GEMM2 with lo, 3 GEMM3, 4 GEMM4)
// and its chunk index kc within the phase.
__device__ __forceinline__ void chunk_of(int c, int &g, int &kc) {
    if (c < 6) { g = 0; kc = c; }
    else if (c < 10) { g = 1; kc = c - 6; }
    else if (c < 14) { g = 2; kc = c - 10; }
    else if (c < 16) { g = 3; kc = c - 14; }
    else { g = 4; kc = c - 16; }
}
__device__ __forceinline__ int phase_chunks(int g) { return g == 0 ? 6 : (g == 3 ? 2 : 4); }

__global__ void __launch_bounds__(kTcThreads, 1)
k_mlp_tc(LearnedDev L, const __grid_constant__ MlpMaps maps, uint32_t *status, int gated, unsigned long long *efx) {
    if (gated && L.lflags[1]) return;
    if (L.n_tiles_live != nullptr && (int)blockIdx.x >= *L.n_tiles_live) return;
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned base (128-byte swizzle atoms), by pointer arithmetic on the shared array so that
    // the compiler keeps the shared address space for every access through it
    unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = smem_u32(sm);
    float *sb1 = (float *)(sm + kOffPar), *sb2 = sb1 + 256, *sw3 = sb2 + 128, *sEp = sw3 + 128;
    const uint32_t bar0 = sbase + kOffBar;
    auto bar = [&](int k) { return bar0 + 8u * (uint32_t)k; };
    volatile uint32_t *s_tmem = (volatile uint32_t *)(sm + kOffBar + 96);
    volatile int *s_abort = (volatile int *)(sm + kOffBar + 100);
    volatile int *s_issued = (volatile int *)(sm + kOffBar + 104);
    volatile int *s_consumed = (volatile int *)(sm + kOffBar + 108);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x;
    const int row0 = tile * kRowTile;
    const int e = L.tile_el[tile];

    if (tid == 0) {
        for (int k = 0; k < kStages; ++k) {
            mbar_init(bar(B_FULL + k), 1);
            mbar_init(bar(B_EMPTY + k), 1);
        }
        mbar_init(bar(B_ACC), 1);
        mbar_init(bar(B_EPI), kEpiThreads);
        mbar_init(bar(B_DRAIN), 1);
        *s_abort = 0;
        *s_issued = 0;
        *s_consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_u32((const void *)s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int q = tid; q < 256; q += kTcThreads) sb1[q] = L.b1[e * kH1 + q];
    for (int q = tid; q < 128; q += kTcThreads) {
        sb2[q] = L.b2[e * kH2 + q];
        sw3[q] = L.W3[e * kH2 + q];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    if (warp == kProducerWarp) {
        // ---------------- TMA producer
        if (lane == 0) {
            for (int c = 0; c < kChunks; ++c) {
                const int s = c % kStages;
                if (c >= kStages && !mbar_wait(bar(B_EMPTY + s), ((c / kStages) - 1) & 1, s_abort)) break;
                int g, kc;
                chunk_of(c, g, kc);
                const uint32_t A = sbase + s * kStageBytes, B = g == 0 ? A + 16384 : A;
                const int x = kc * 64;
                const uint32_t fb = bar(B_FULL + s);
                if (g == 0) {
                    mbar_expect_tx(fb, 48 * 1024);
                    tma_2d(A, &maps.g, x, row0, fb);
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
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issue
        if (lane == 0) {
            const uint32_t i256 = idesc_bf16(256), i128 = idesc_bf16(128);
            const uint32_t res = sbase + kOffRes;
            int c = 0;
            bool ok = true;
            for (int g = 0; g < kPhases && ok; ++g) {
                if (g > 0) {
                    if (!mbar_wait(bar(B_EPI), (g - 1) & 1, s_abort)) break;
                    tc_fence_after();
                }
                const int nk = phase_chunks(g);
                for (int kc = 0; kc < nk; ++kc, ++c) {
                    const int s = c % kStages;
                    if (!mbar_wait(bar(B_FULL + s), (c / kStages) & 1, s_abort)) {
                        ok = false;
                        break;
                    }
                    *s_consumed = c + 1;
                    tc_fence_after();
                    const uint32_t A = sbase + s * kStageBytes, B = g == 0 ? A + 16384 : A;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t acc = g == 2 || (kc | k) != 0;   // GEMM2' adds onto GEMM2
                        const uint32_t ko = 32u * k;
                        if (g == 0) {
                            mma_bf16(tmem, sdesc(A + ko), sdesc(B + ko), i256, acc);
                        } else if (g == 1 || g == 2) {
                            mma_bf16(tmem + 256, sdesc(res + kc * 16384 + ko), sdesc(B + ko), i128, acc);
                        } else if (g == 3) {
                            mma_bf16(tmem + 256, sdesc(res + kc * 16384 + ko), sdesc(B + ko), i256, acc);
                        } else {
                            const uint64_t a = sdesc(res + kc * 16384 + ko);
                            mma_bf16(tmem, a, sdesc(B + ko), i256, acc);
                            mma_bf16(tmem + 256, a, sdesc(B + 32768 + ko), i128, acc);
                        }
                    }
                    mma_commit(bar(B_EMPTY + s));
                }
                if (ok) mma_commit(bar(B_ACC));
            }
        }
    } else {
        // ---------------- epilogue: lane = tile row (TMEM lane), warp group cg = column range
        const int q4 = warp & 3, cg = warp >> 2;
        const int r = 32 * q4 + lane;
        const int row = row0 + r;
        const uint32_t tl = tmem + ((uint32_t)(32 * q4) << 16);
        unsigned char *res = sm + kOffRes;
        float v[32], h[32];
        bool ok = true;
        // epi1: a1 = celu(H1 + b1), columns 64 cg .. 64 cg + 63: its BF16 value to the operand, a1 itself
        // (FP32) over H1 in TMEM (read again by epi1b and epi3)
        if ((ok = warp_wait(bar(B_ACC), 0, s_abort))) {
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
            mbar_arrive(bar(B_EPI));
        }
        // epi1b: once GEMM2 has read the operand, the BF16 residuals a1 - bf16(a1) replace it
        if (ok && (ok = warp_wait(bar(B_ACC), 1, s_abort))) {
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
            mbar_arrive(bar(B_EPI));
        }
        // epi2: energy partial and d2 = bf16(W3 * celu'(H2 + b2)), columns 32 cg .. 32 cg + 31
        if (ok && (ok = warp_wait(bar(B_ACC), 0, s_abort))) {
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
            mbar_arrive(bar(B_EPI));
        }
        epi_sync();   // energy partials of the four column groups are in shared memory
        if (ok && cg == 0) {
            const float E = ((sEp[r] + sEp[128 + r]) + sEp[256 + r]) + sEp[384 + r];
            const double Er = L.atom_of[row] >= 0 ? (double)E + (double)L.b3[e] + L.e0[e] : 0.0;
            L.E_row[row] = Er;
            if (efx != nullptr) fx_warp_add_d(&efx[E_LEARN], Er);
        }
        // epi3: d1 = bf16(P1 * celu'(H1 + b1)), columns 64 cg .. 64 cg + 63
        if (ok && (ok = warp_wait(bar(B_ACC), 1, s_abort))) {
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
            mbar_arrive(bar(B_EPI));
        }
        // epi4: g = dE/dG, columns 96 cg .. 96 cg + 95, through a per-warp 32 x 32 staging
        // block (in the operand ring, idle once the last GEMM completed) for coalesced stores
        if (ok && warp_wait(bar(B_ACC), 0, s_abort)) {
            tc_fence_after();
            uint32_t *stg = reinterpret_cast<uint32_t *>(sm) + warp * 32 * kGStrideW;
            __nv_bfloat16 *gtile = static_cast<__nv_bfloat16 *>(L.g) + (size_t)(row0 + 32 * q4) * kNFeat;
#pragma unroll 1
            for (int cc = 3 * cg; cc < 3 * cg + 3; ++cc) {
                tmem_ld32(tl + cc * 32, v);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    *reinterpret_cast<uint4 *>(stg + lane * kGStrideW + 4 * q) =
                        make_uint4(pack_bf16(v[8 * q], v[8 * q + 1]), pack_bf16(v[8 * q + 2], v[8 * q + 3]),
                                   pack_bf16(v[8 * q + 4], v[8 * q + 5]), pack_bf16(v[8 * q + 6], v[8 * q + 7]));
                __syncwarp();
                // 32 rows x 64 bytes: lane takes 16 bytes (8 columns) of row (it * 32 + lane) / 4
#pragma unroll
                for (int it = 0; it < 4; ++it) {
                    const int f = it * 32 + lane, rr = f >> 2, c4 = f & 3;
                    *reinterpret_cast<uint4 *>(gtile + (size_t)rr * kNFeat + cc * 32 + 8 * c4) =
                        *reinterpret_cast<const uint4 *>(stg + rr * kGStrideW + 4 * c4);
                }
                __syncwarp();
            }
        }
        tc_fence_before();
    }
    __syncthreads();
    if (*s_abort) {
        // teardown after a timeout: let copies and MMAs in flight finish before freeing tensor memory
        if (tid == 0) {
            for (int c = *s_consumed; c < *s_issued; ++c) mbar_drain(bar(B_FULL + c % kStages), (c / kStages) & 1);
            atomicOr(status, MDPF_STATUS_TIMEOUT);
            atomicOr(&L.lflags[3], 1u);
        }
        if (tid == 32 * kMmaWarp) {
            mma_commit(bar(B_DRAIN));
            mbar_drain(bar(B_DRAIN), 0);
        }
        __syncthreads();
    }
    if (warp == kMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

}  // namespace

cudaError_t learned_mlp_tc_prepare() {
    return cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

cudaError_t learned_mlp_tc(const LearnedDev &L, const MlpMaps &maps, uint32_t *status, bool gated,
                           unsigned long long *efx, cudaStream_t s) {
    if (L.n_rows > 0)
        k_mlp_tc<<<L.n_rows / kRowTile, kTcThreads, kSmemBytes, s>>>(L, maps, status, gated ? 1 : 0, efx);
    return cudaGetLastError();
}

}  // namespace mdpf
