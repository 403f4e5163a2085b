// Weight gradients of the force-matching loss on the 5th-generation tensor
// cores:
//
//   dW1[e] = sum over the rows r of element e of  hbar1_r (x) G_r  +  tbar1_r (x) U_r     [256 x 384]
//   dW2[e] = sum over the rows r of element e of  hbar2_r (x) a1_r +  tbar2_r (x) ta1_r   [128 x 256]
//
// (the row adjoints of the MLP's primal and tangent passes times the
// features, their tangents, and the layer-1 activations and their tangents).
// Each is a GEMM whose K index runs over the rows, i.e. over the row tiles of
// element e and the two terms.  One CTA computes one 128 x 128 output tile
// over a contiguous run of one element's row tiles (a K split) and writes it
// as a partial sum; the splits are handed out in proportion to each element's
// tile count and summed afterwards in split order, so the result is
// reproducible bit for bit.
//
// The row arrays are BF16 [rows][width] (rounded where they are produced):
// the operands are MN-major.  The eight producer warps read them coalesced
// (one output row or column per thread, 64 rows per K chunk) and write them
// transposed into the 128-byte-swizzled K-major layout (8-row x 128-byte atoms, the 16-byte
// unit index XOR-ed with the row index mod 8) through a three-stage ring; rows
// past a frame's atoms are zero.  One thread of warp 8 issues
// tcgen05.mma kind::f16 (BF16 x BF16 -> FP32, M = N = 128) into 128 TMEM
// columns; warps 0-3 then read the accumulator (TMEM lanes 32 w .. 32 w + 31)
// and store the partial tile.  Every wait is bounded: on expiry the CTA
// records MDPF_STATUS_TIMEOUT, lets its MMAs in flight finish, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "learned.cuh"
#include "tc_util.cuh"

namespace mdpf {
namespace {

constexpr int kWgProd = 8;                       // producer warps (warps 0-3 also run the epilogue)
constexpr int kWgThreads = 32 * kWgProd + 32;    // + the MMA warp
constexpr int kWgMma = kWgProd;
constexpr int kWgStages = 3;
constexpr int kWgStage = 32 * 1024;              // [A 128 x 64][B 128 x 64] BF16
constexpr int kWgOffBar = kWgStages * kWgStage;
constexpr int kWgSmem = kWgOffBar + 128 + 1024;
enum { W_FULL = 0, W_EMPTY = kWgStages, W_ACC = 2 * kWgStages, W_DRAIN = 2 * kWgStages + 1 };
static_assert(8 * (W_DRAIN + 1) <= 64, "barrier block");

struct WgProblem {
    const __nv_bfloat16 *A[2];   // [rows][M]: the two terms
    const __nv_bfloat16 *B[2];   // [rows][N]
    int M, N;
    int off;             // offset of the gradient block within one element's parameters
};

struct WgArgs {
    WgProblem p[2];
    const int *atom_of;
    const int *etiles;   // [4][tiles_max]: live row tiles of each element, in order
    const int4 *split;   // [kWgSplits]: element (-1: unused), first and end index into its tile list
    int tiles_max;
    float *part;         // problem 0 partials [kWgSplits][M0][N0], then problem 1's
    uint32_t *status;
};

// The live row tiles of each element, and the K splits: kWgSplits handed out
// in proportion to the elements' tile counts (at least one per element that
// has tiles, at most one per tile).  The block stages the tile elements in
// shared memory 1024 at a time and warp 0 lists each element's tiles in
// ascending order by ballots; thread 0 then deals the splits.
constexpr int kWgTableThreads = 256, kWgTableChunk = 1024;

__global__ void __launch_bounds__(kWgTableThreads) k_wg_table(const int *tile_el, const int *n_live, int tiles_max,
                                                             int *etiles, int4 *split) {
    __shared__ int s_el[kWgTableChunk];
    const int t = threadIdx.x, lane = t & 31;
    const int live = *n_live;
    int cnt[4] = {0, 0, 0, 0};   // warp 0: tiles of each element listed so far (the same in every lane)
    for (int base = 0; base < live; base += kWgTableChunk) {
        const int m = min(kWgTableChunk, live - base);
        for (int k = t; k < m; k += kWgTableThreads) s_el[k] = tile_el[base + k];
        __syncthreads();
        if (t < 32) {
            for (int k0 = 0; k0 < m; k0 += 32) {
                const int e = k0 + lane < m ? s_el[k0 + lane] : -1;
#pragma unroll
                for (int ee = 0; ee < 4; ++ee) {
                    const unsigned int mask = __ballot_sync(0xffffffffu, e == ee);
                    if (e == ee) etiles[ee * tiles_max + cnt[ee] + __popc(mask & ((1u << lane) - 1u))] = base + k0 + lane;
                    cnt[ee] += __popc(mask);
                }
            }
        }
        __syncthreads();
    }
    if (t != 0) return;   // thread 0 is in warp 0, whose lanes all hold the counts
    const int total = cnt[0] + cnt[1] + cnt[2] + cnt[3];
    int se[4], used = 0;
    for (int e = 0; e < 4; ++e) {
        se[e] = cnt[e] > 0 ? max(1, (int)((long long)kWgSplits * cnt[e] / max(total, 1))) : 0;
        se[e] = min(se[e], cnt[e]);
        used += se[e];
    }
    while (used > kWgSplits) {   // at most 3 over: take from the element with the fewest tiles per split
        int best = -1;
        for (int e = 0; e < 4; ++e)
            if (se[e] > 1 && (best < 0 || cnt[e] * se[best] < cnt[best] * se[e])) best = e;
        if (best < 0) break;
        --se[best];
        --used;
    }
    while (used < kWgSplits) {   // the rest to the element with the most tiles per split
        int best = -1;
        for (int e = 0; e < 4; ++e)
            if (se[e] < cnt[e] && (best < 0 || cnt[e] * se[best] > cnt[best] * se[e])) best = e;
        if (best < 0) break;
        ++se[best];
        ++used;
    }
    int c = 0;
    for (int e = 0; e < 4; ++e)
        for (int j = 0; j < se[e] && c < kWgSplits; ++j, ++c)
            split[c] = make_int4(e, cnt[e] * j / se[e], cnt[e] * (j + 1) / se[e], 0);
    for (; c < kWgSplits; ++c) split[c] = make_int4(-1, 0, 0, 0);
}

__global__ void __launch_bounds__(kWgThreads, 2) k_wgrad_tc(WgArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t sbase = smem_u32(sm);
    const uint32_t bar0 = sbase + kWgOffBar;
    auto bar = [&](int k) { return bar0 + 8u * (uint32_t)k; };
    volatile uint32_t *s_tmem = (volatile uint32_t *)(sm + kWgOffBar + 64);
    volatile int *s_abort = (volatile int *)(sm + kWgOffBar + 68);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int job = blockIdx.x, prob = 0;
    const int jobs0 = (a.p[0].M / 128) * (a.p[0].N / 128) * kWgSplits;
    if (job >= jobs0) {
        job -= jobs0;
        prob = 1;
    }
    const WgProblem &P = a.p[prob];
    const int ntn = P.N / 128;
    const int tile = job / kWgSplits, sp = job % kWgSplits;
    const int m0 = (tile / ntn) * 128, n0 = (tile % ntn) * 128;
    const int4 spl = a.split[sp];
    const int e = spl.x;
    if (e < 0) return;   // unused split: the whole CTA
    const int nchunks = (spl.z - spl.y) * 4;   // per row tile: 2 terms x 2 halves of 64 rows
    float *out = a.part + (prob ? (size_t)kWgSplits * a.p[0].M * a.p[0].N : 0) + (size_t)sp * P.M * P.N;

    if (tid == 0) {
        for (int k = 0; k < kWgStages; ++k) {
            mbar_init(bar(W_FULL + k), 32 * kWgProd);
            mbar_init(bar(W_EMPTY + k), 1);
        }
        mbar_init(bar(W_ACC), 1);
        mbar_init(bar(W_DRAIN), 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kWgMma) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
                         smem_u32((const void *)s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    if (warp < kWgProd) {
        // ---------------- producers: thread = two adjacent rows of A (tid < 128) or of B and one half (32) of
        // the chunk's 64 K values; each 4-byte load brings both rows' values of one K index
        const bool isA = tid < 128;
        const int pr = tid & 63, kh = (tid >> 6) & 1;
        const int stride = isA ? P.M : P.N;
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % kWgStages;
            if (c >= kWgStages && !warp_wait(bar(W_EMPTY + s), ((c / kWgStages) - 1) & 1, s_abort)) {
                ok = false;   // the same in every lane of the warp
                break;
            }
            const int tl = a.etiles[e * a.tiles_max + spl.y + (c >> 2)];
            const int term = (c >> 1) & 1, r0 = tl * kRowTile + (c & 1) * 64;
            const unsigned int mk = __ballot_sync(0xffffffffu, a.atom_of[r0 + 32 * kh + lane] >= 0);
            const uint32_t *src = reinterpret_cast<const uint32_t *>((isA ? P.A[term] + m0 : P.B[term] + n0) +
                                                                     (size_t)(r0 + 32 * kh) * stride + 2 * pr);
            uint32_t x[32];   // BF16 bit patterns of rows 2 pr (low half) and 2 pr + 1 (high half)
#pragma unroll
            for (int j = 0; j < 32; ++j) x[j] = src[(size_t)j * (stride / 2)];
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (!((mk >> j) & 1u)) x[j] = 0u;   // rows past a frame's atoms are zero
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = 2 * pr + h;
                unsigned char *dst = sm + s * kWgStage + (isA ? 0 : 16384) + row * 128;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int u = 4 * kh + q;
                    uint32_t v[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) v[k] = h ? (x[8 * q + k] >> 16) : (x[8 * q + k] & 0xFFFFu);
                    uint4 w;
                    w.x = v[0] | (v[1] << 16);
                    w.y = v[2] | (v[3] << 16);
                    w.z = v[4] | (v[5] << 16);
                    w.w = v[6] | (v[7] << 16);
                    *reinterpret_cast<uint4 *>(dst + ((u ^ (row & 7)) << 4)) = w;
                }
            }
            proxy_fence();   // generic-proxy stores, read by the MMA
            mbar_arrive(bar(W_FULL + s));
        }
        // ---------------- epilogue (warps 0-3): the partial tile, row m = 32 w + lane
        if (warp < 4) {
            const bool acc = warp_wait(bar(W_ACC), 0, s_abort);
            if (ok && acc) {
                tc_fence_after();
                const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
                float *o = out + (size_t)(m0 + 32 * warp + lane) * P.N + n0;
#pragma unroll 1
                for (int cc = 0; cc < 4; ++cc) {
                    float v[32];
                    tmem_ld32(tl + 32 * cc, v);
                    if (nchunks == 0) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = 0.f;
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        *reinterpret_cast<float4 *>(o + 32 * cc + 4 * q) =
                            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
        }
        tc_fence_before();
    } else if (lane == 0) {
        // ---------------- MMA issue
        const uint32_t idesc = idesc_bf16(128);
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % kWgStages;
            if (!mbar_wait(bar(W_FULL + s), (c / kWgStages) & 1, s_abort)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t A = sbase + s * kWgStage, B = A + 16384;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mma_bf16(tmem, sdesc(A + 32u * k), sdesc(B + 32u * k), idesc, (c | k) != 0 ? 1u : 0u);
            mma_commit(bar(W_EMPTY + s));
        }
        if (ok) mma_commit(bar(W_ACC));
    }
    __syncthreads();
    if (*s_abort) {
        if (tid == 32 * kWgMma) {
            atomicOr(a.status, MDPF_STATUS_TIMEOUT);
            mma_commit(bar(W_DRAIN));
            mbar_drain(bar(W_DRAIN), 0);
        }
        __syncthreads();
    }
    if (warp == kWgMma) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
    }
}

// grad[e][off + j] = sum over the splits c of element e, in order, of part[c][j].
__global__ void k_wg_reduce(const float *part, const int4 *split, int len, int off, int per_element, float *grad) {
    const int e = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= len) return;
    float s = 0.f;
    for (int c = 0; c < kWgSplits; ++c)
        if (split[c].x == e) s += part[(size_t)c * len + j];
    grad[(size_t)e * per_element + off + j] = s;
}

}  // namespace

cudaError_t learned_wgrad_tc_prepare() {
    return cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem);
}

cudaError_t learned_wgrad_tc(const WgradIn &w, cudaStream_t s) {
    k_wg_table<<<1, kWgTableThreads, 0, s>>>(w.tile_el, w.n_live, w.tiles_max, w.etiles, w.split);
    WgArgs a{};
    a.p[0] = WgProblem{{w.bh1, w.bt1}, {w.G, w.U}, kH1, kNFeat, w.off_w1};
    a.p[1] = WgProblem{{w.bh2, w.bt2}, {w.a1, w.ta1}, kH2, kH1, w.off_w2};
    a.atom_of = w.atom_of;
    a.etiles = w.etiles;
    a.split = w.split;
    a.tiles_max = w.tiles_max;
    a.part = w.part;
    a.status = w.status;
    const int jobs = ((kH1 / 128) * (kNFeat / 128) + (kH2 / 128) * (kH1 / 128)) * kWgSplits;
    k_wgrad_tc<<<jobs, kWgThreads, kWgSmem, s>>>(a);
    const float *part1 = w.part + (size_t)kWgSplits * kH1 * kNFeat;
    k_wg_reduce<<<dim3((kH1 * kNFeat + 255) / 256, 4), 256, 0, s>>>(w.part, w.split, kH1 * kNFeat, w.off_w1,
                                                                       w.per_element, w.grad);
    k_wg_reduce<<<dim3((kH2 * kH1 + 255) / 256, 4), 256, 0, s>>>(part1, w.split, kH2 * kH1, w.off_w2,
                                                                       w.per_element, w.grad);
    return cudaGetLastError();
}

}  // namespace mdpf
