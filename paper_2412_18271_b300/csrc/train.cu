// Force-matching training of the learned potential on the device.
//
// One call evaluates, for a batch of B frames of N atoms each,
//   L = (1/B) sum_f ((E_f - E_ref,f) / N)^2  +  w * (1/(3 N B)) sum_{f,a,c} (F - F_ref)^2
// and its gradient in the FP32 master parameters:
//   1. rows: per frame, atoms grouped by element into 128-row tiles;
//   2. neighbours per frame (all pairs within 5.2 A, FP32 predicate, ascending);
//   3. features (FP32 and the BF16 GEMM copy), MLP energies and dE/dG on the
//      tensor cores, forces by the feature adjoint (with the model's repulsive
//      core, whose energy and forces have no parameters but enter E_f and F);
//   4. per frame: c = dL/dE_f, v = dL/dF;  U = J v by the feature JVP;
//   5. per row: primal and tangent passes of the MLP along U, then one reverse
//      sweep over both for sum_i [c E_i - U_i . dE_i/dG_i]; the row adjoints
//      are stored;
//   6. weight gradients as fixed-order reductions over the rows of each
//      element (split over the row range, splits summed in order), so the
//      gradient is reproducible bit for bit.
// Parameters (flat FP32, per element e = 0..3, kParamsPerElement each):
//   W1 [256][384], b1 [256], W2 [128][256], b2 [128], W3 [128], b3.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "learned.cuh"

namespace mdpf {
namespace {

constexpr int kOW1 = 0, kOb1 = kH1 * kNFeat, kOW2 = kOb1 + kH1, kOb2 = kOW2 + kH2 * kH1, kOW3 = kOb2 + kH2,
              kOb3 = kOW3 + kH2, kPPE = kOb3 + 1;
constexpr int kSplits = 8;     // row-range splits of the weight-matrix gradients
constexpr int kVSplits = 64;   // block-range splits of the bias / output-weight gradients
constexpr int kTrRows = 32;    // rows per block of the training MLP kernel (4 MMA n-tiles)
// its BF16 row planes: G and U (hi, lo), then a1 and ta1 (hi, lo); bt2 and bh2 (hi, lo) and the FP32
// s'(h1), s''(h1) t1 of the rows reuse the first; then each warp's ring of weight fragments (4 stages of
// two 16 x 16 BF16 tiles)
constexpr int kTrSmem = (4 * kTrRows * (kNFeat + 8) + 4 * kTrRows * (kH1 + 8) + 8 * 4 * 2 * 16 * 16) * 2;

// ------------------------------------------------------------ batch layout

// Per frame: atoms of each element and the frame's row tiles.
__global__ void k_tr_count(const int *el, int N, int *cnt, int *ntile) {
    __shared__ int c[4];
    const int f = blockIdx.x;
    if (threadIdx.x < 4) c[threadIdx.x] = 0;
    __syncthreads();
    for (int a = threadIdx.x; a < N; a += blockDim.x) atomicAdd(&c[el[(size_t)f * N + a]], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int e = 0; e < 4; ++e) {
            cnt[4 * f + e] = c[e];
            t += (c[e] + kRowTile - 1) / kRowTile;
        }
        ntile[f] = t;
    }
}

__global__ void k_tr_scan(int B, const int *ntile, int *tile_off, int *n_tiles_live) {
    if (threadIdx.x != 0) return;
    int t = 0;
    for (int f = 0; f < B; ++f) {
        tile_off[f] = t;
        t += ntile[f];
    }
    tile_off[B] = t;
    *n_tiles_live = t;
}

// Rows: within a frame, element groups in order H, C, N, O, each padded to
// 128 rows; within a group, atoms in index order (block-wide scans).
__global__ void __launch_bounds__(1024) k_tr_rows(const int *el, int N, const int *cnt, const int *tile_off,
                                                  int *row_of, int *atom_of, int *tile_el) {
    __shared__ unsigned long long warp_tot[32];
    __shared__ int base[4];
    const int f = blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
    int start[4];
    {
        int tt = tile_off[f];
        for (int e = 0; e < 4; ++e) {
            start[e] = tt;
            const int nt = (cnt[4 * f + e] + kRowTile - 1) / kRowTile;
            for (int q = t; q < nt; q += blockDim.x) tile_el[tt + q] = e;
            tt += nt;
        }
    }
    if (t < 4) base[t] = 0;
    __syncthreads();
    for (int a0 = 0; a0 < N; a0 += blockDim.x) {
        const int a = a0 + t;
        const int e = a < N ? el[(size_t)f * N + a] : -1;
        // packed per-element counters (16 bits each), inclusive scan over the block
        unsigned long long x = e >= 0 ? (1ull << (16 * e)) : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            unsigned long long y = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0ull;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long z = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += z;
            }
            warp_tot[lane] = y;
        }
        __syncthreads();
        const unsigned long long incl = x + (wid > 0 ? warp_tot[wid - 1] : 0ull);
        if (e >= 0) {
            const int rank = (int)((incl >> (16 * e)) & 0xFFFFull) - 1 + base[e];
            const int row = start[e] * kRowTile + rank;
            row_of[(size_t)f * N + a] = row;
            atom_of[row] = f * N + a;
        }
        __syncthreads();
        if (t < 4) base[t] += (int)((warp_tot[(blockDim.x >> 5) - 1] >> (16 * t)) & 0xFFFFull);
        __syncthreads();
    }
}

__global__ void k_tr_pos(const double *pos, int n, float4 *pos4) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < n) pos4[a] = make_float4((float)pos[3 * a], (float)pos[3 * a + 1], (float)pos[3 * a + 2], 0.f);
}

// Neighbours within the atom's own frame, brute force, ascending: one thread
// per atom, each walking its frame's atoms in index order and appending the
// ones within the list radius to its own row (the FP32 predicate evaluated
// with explicitly rounded operations, so no contraction changes it).  When a
// block's atoms share one frame, the frame's positions pass through shared
// memory 256 at a time; a block that straddles two frames reads them from
// global memory.
__device__ __forceinline__ bool tr_in_list(const float4 &pi, const float4 &pj, float rc2) {
    const float dx = __fsub_rn(pj.x, pi.x), dy = __fsub_rn(pj.y, pi.y), dz = __fsub_rn(pj.z, pi.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)) < rc2;
}

constexpr int kTrNbThreads = 256;

__global__ void __launch_bounds__(kTrNbThreads) k_tr_nb(LearnedDev L, const float4 *pos4, int N, uint32_t *status) {
    __shared__ float4 s_pj[kTrNbThreads];
    const int a0 = blockIdx.x * kTrNbThreads, t = threadIdx.x;
    const int i = a0 + t;
    const int alast = min(a0 + kTrNbThreads, L.n) - 1;
    const bool one_frame = a0 / N == alast / N;   // the same in every thread of the block
    const bool live = i < L.n;
    const int f0 = ((live ? i : alast) / N) * N;
    const float4 pi = pos4[live ? i : alast];
    const float rc2 = L.rc_list2;
    int *row = L.nb_idx + (size_t)(live ? i : 0) * kKmax;
    int m = 0;
    if (one_frame) {
        for (int c0 = 0; c0 < N; c0 += kTrNbThreads) {
            const int cn = min(kTrNbThreads, N - c0);
            __syncthreads();
            if (t < cn) s_pj[t] = pos4[f0 + c0 + t];
            __syncthreads();
            if (live) {
#pragma unroll 8
                for (int k = 0; k < cn; ++k) {
                    const int j = f0 + c0 + k;
                    if (j != i && tr_in_list(pi, s_pj[k], rc2)) {
                        if (m < kKmax) row[m] = j;
                        ++m;
                    }
                }
            }
        }
    } else if (live) {
        for (int j = f0; j < f0 + N; ++j) {
            if (j != i && tr_in_list(pi, pos4[j], rc2)) {
                if (m < kKmax) row[m] = j;
                ++m;
            }
        }
    }
    if (!live) return;
    L.nb_count[i] = min(m, kKmax);
    if (m > kKmax) atomicOr(status, MDPF_STATUS_NEIGHBOR_OVERFLOW);
}

// BF16 weights (and their transposes) and contiguous FP32 bias / output vectors from the master parameters.
__global__ void k_tr_weights(const float *P, __nv_bfloat16 *W1, __nv_bfloat16 *W1T, __nv_bfloat16 *W2,
                             __nv_bfloat16 *W2T, float *b1, float *b2, float *W3, float *b3) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int e = blockIdx.y;
    const float *p = P + (size_t)e * kPPE;
    if (q < kH1 * kNFeat) {
        const int a = q / kNFeat, f = q % kNFeat;
        const __nv_bfloat16 v = __float2bfloat16_rn(p[kOW1 + q]);
        W1[(size_t)e * kH1 * kNFeat + q] = v;
        W1T[(size_t)e * kNFeat * kH1 + (size_t)f * kH1 + a] = v;
    }
    if (q < kH2 * kH1) {
        const int b = q / kH1, a = q % kH1;
        const __nv_bfloat16 v = __float2bfloat16_rn(p[kOW2 + q]);
        W2[(size_t)e * kH2 * kH1 + q] = v;
        W2T[(size_t)e * kH1 * kH2 + (size_t)a * kH2 + b] = v;
    }
    if (q < kH1) b1[e * kH1 + q] = p[kOb1 + q];
    if (q < kH2) {
        b2[e * kH2 + q] = p[kOb2 + q];
        W3[e * kH2 + q] = p[kOW3 + q];
    }
    if (q == 0) b3[e] = p[kOb3];
}

// Feature range of the training data (per element and feature), order-free min/max.
__device__ __forceinline__ unsigned int ord_u(float f) {
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
// One block per row tile, one thread per feature.
__global__ void k_tr_range(LearnedDev L, unsigned int *rmin, unsigned int *rmax) {
    const int tile = blockIdx.x, f = threadIdx.x;
    if (tile >= *L.n_tiles_live || f >= kNFeat) return;
    const int e = L.tile_el[tile];
    unsigned int lo = 0xFFFFFFFFu, hi = 0u;
    for (int row = tile * kRowTile; row < (tile + 1) * kRowTile; ++row) {
        if (L.atom_of[row] < 0) continue;
        const unsigned int u = ord_u(L.G32[(size_t)row * kNFeat + f]);
        lo = min(lo, u);
        hi = max(hi, u);
    }
    if (hi != 0u) {
        atomicMin(&rmin[e * kNFeat + f], lo);
        atomicMax(&rmax[e * kNFeat + f], hi);
    }
}

// ------------------------------------------------------------ loss

__device__ double block_sum_d(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    return t;   // valid in thread 0
}

// Per frame: energy, energy-loss weight c (per row), force residual -> v, loss parts.
__global__ void k_tr_loss(LearnedDev L, int N, int B, double w_force, const int *tile_off, const double *E_ref,
                          const float *F_ref, const unsigned long long *fx, const unsigned long long *ecore,
                          float *c_row, float *v, double *loss_parts) {
    __shared__ double sh[32];
    __shared__ double s_c;
    const int f = blockIdx.x;
    const int r0 = tile_off[f] * kRowTile, r1 = tile_off[f + 1] * kRowTile;
    double e = 0.0;
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) e += L.E_row[r];
    const double Ef = block_sum_d(e, sh) + fx_val(ecore[f]);   // MLP rows + the repulsive core
    if (threadIdx.x == 0) {
        const double d = (Ef - E_ref[f]) / N;
        loss_parts[2 * f] = d * d / B;
        s_c = 2.0 * d / N / B;
    }
    __syncthreads();
    const float cf = (float)s_c;
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) c_row[r] = L.atom_of[r] >= 0 ? cf : 0.f;
    const double scale = 2.0 * w_force / (3.0 * N * B);
    double sse = 0.0;
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
        const size_t k = (size_t)f * 3 * N + q;
        const double d = fx_val(fx[k]) - (double)F_ref[k];
        v[k] = (float)(scale * d);
        sse += d * d;
    }
    const double S = block_sum_d(sse, sh);
    if (threadIdx.x == 0) loss_parts[2 * f + 1] = w_force * S / (3.0 * N * B);
}

__global__ void k_tr_loss_total(int B, const double *parts, double *loss3) {
    if (threadIdx.x != 0) return;
    double le = 0.0, lf = 0.0;
    for (int f = 0; f < B; ++f) {
        le += parts[2 * f];
        lf += parts[2 * f + 1];
    }
    loss3[0] = le + lf;
    loss3[1] = le;
    loss3[2] = lf;
}

// ------------------------------------------------------------ per-row reverse over the tangent pass

__device__ __forceinline__ float tr_s(float z) { return z > 0.f ? z : 0.1f * (__expf(10.f * z) - 1.f); }
__device__ __forceinline__ float tr_ds(float z) { return z >= 0.f ? 1.f : __expf(10.f * z); }
__device__ __forceinline__ float tr_dds(float z) { return z >= 0.f ? 0.f : 10.f * __expf(10.f * z); }

// Columns of a block's vector-gradient partials: sum over its real rows of bh1 (b1), bh2 (b2),
// c s(h2) - s'(h2) t2 (W3) and c (b3).
constexpr int kVb1 = 0, kVb2 = kH1, kVW3 = kH1 + kH2, kVb3 = kH1 + 2 * kH2, kVLen = kVb3 + 1;

// The row kernel's outputs for the weight-gradient GEMMs, rounded to BF16 (their operand type), and the
// per-block vector-gradient partials.
struct RowOut {
    __nv_bfloat16 *bh1, *bt1, *a1, *ta1;   // [rows][256]
    __nv_bfloat16 *bh2, *bt2;              // [rows][128]
    __nv_bfloat16 *u16;                    // [rows][384]: the tangents U
    float *vpart;                          // [rows / kTrRows][kVLen]
};

// kTrRows rows of one element per block, 8 warps, on the tensor cores through
// warp-level MMA (m16n8k16, BF16 operands, FP32 accumulation).  The weights are
// BF16 values already; every FP32 row operand X (features G, tangents U and
// the layer outputs that feed the next GEMM) enters as the pair
// hi = bf16(X), lo = bf16(X - hi), and W X is accumulated as W hi + W lo, so
// the products keep about 16 bits of X (the FP32 CUDA-core sums they replace
// kept 24; the rows' own features are FP32 values of a BF16 model).
//   layer 1   h1 = W1 G + b1, t1 = W1 U       (M = 256 units, N = 32 rows, K = 384)
//             a1 = s(h1), ta1 = s'(h1) t1
//   layer 2   h2 = W2 a1 + b2, t2 = W2 ta1    (M = 128, K = 256)
//             bt2 = -w3 s'(h2), bh2 = -w3 s''(h2) t2 + c w3 s'(h2), w3g = c s(h2) - s'(h2) t2
//   layer 1'  bta1 = W2^T bt2, ba1 = W2^T bh2 (M = 256, K = 128)
//             bt1 = s'(h1) bta1, bh1 = s''(h1) t1 bta1 + s'(h1) ba1
// The rows sit in shared memory as BF16 [row][k] planes (the MMA's B operand,
// read with ldmatrix); the A fragments (weight rows, K contiguous) reach a
// per-warp shared ring by cp.async three k-steps ahead of their MMAs.  Warp w owns units
// 32 w .. 32 w + 31 in layers 1 and 1' and units 16 w .. 16 w + 15 in layer
// 2; s'(h1) and s''(h1) t1 of its layer-1 fragments wait in shared memory
// for layer 1'.
constexpr int kXs = kNFeat + 8;   // BF16 row strides padded by 16 bytes (conflict-free ldmatrix rows)
constexpr int kAs = kH1 + 8;
constexpr int kBs = kH2 + 8;
constexpr int kPlaneX = kTrRows * kXs, kPlaneA = kTrRows * kAs, kPlaneB = kTrRows * kBs;
static_assert(4 * kPlaneB * 2 + 2 * kTrRows * kH1 * 4 <= 4 * kPlaneX * 2, "bt2 / bh2 planes and s', s'' t1 fit");
static_assert(kRowTile % kTrRows == 0, "a block's rows lie in one row tile (one element)");

__device__ __forceinline__ uint32_t tr_smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Fragments of two n-tiles (rows 8 j .. 8 j + 15) of a [row][k] plane at k-step k0: b[0..1] for n-tile j,
// b[2..3] for n-tile j + 1.
__device__ __forceinline__ void tr_frag_b2(const __nv_bfloat16 *plane, int ld, int j, int k0, int lane,
                                           uint32_t (&b)[4]) {
    const __nv_bfloat16 *p = plane + (size_t)(8 * j + ((lane >> 4) << 3) + (lane & 7)) * ld + k0 + ((lane >> 3) & 1) * 8;
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3])
                 : "r"(tr_smem_u32(p)));
}

__device__ __forceinline__ void tr_mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The weight (A) fragments travel through a per-warp ring of kTrRing k-steps in shared memory, filled by
// 16-byte cp.async copies kTrRing - 1 k-steps ahead of their MMAs.  A stage holds MT m-tiles of 16 rows x 16
// columns (32 bytes a row); the two 16-byte halves of rows 4..7 and 12..15 are swapped, so that the eight rows
// an ldmatrix reads lie in eight different bank groups.
constexpr int kTrRing = 4;
constexpr int kTrStage = 2 * 16 * 16;   // BF16 elements of a stage (two m-tiles)

static_assert(kTrSmem == (4 * kPlaneX + 4 * kPlaneA + 8 * kTrRing * kTrStage) * 2,
              "shared-memory size of the training MLP kernel");

__device__ __forceinline__ void tr_cp16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tr_smem_u32(dst)), "l"(src) : "memory");
}

template <int MT>
__device__ __forceinline__ void tr_ring_fill(const __nv_bfloat16 *W, int ldw, int m0, int k0, __nv_bfloat16 *stage,
                                             int lane) {
#pragma unroll
    for (int x = 0; x < MT; ++x) {
        const int c = lane + 32 * x, i = c >> 5, row = (c & 31) >> 1, half = c & 1;
        tr_cp16(stage + i * 256 + row * 16 + ((half ^ ((row >> 2) & 1)) << 3),
                W + (size_t)(m0 + 16 * i + row) * ldw + k0 + 8 * half);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// The A fragment of m-tile i of a stage (ldmatrix x4: rows 0-7 / 8-15, columns 0-7 / 8-15).
__device__ __forceinline__ void tr_frag_a_ring(const __nv_bfloat16 *stage, int i, int lane, uint32_t (&a)[4]) {
    const int mi = lane >> 3, r = (mi & 1) * 8 + (lane & 7), half = mi >> 1;
    const __nv_bfloat16 *p = stage + i * 256 + r * 16 + ((half ^ ((r >> 2) & 1)) << 3);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(tr_smem_u32(p)));
}

// D_h += W (P0 + P1), D_t += W (P2 + P3) over K = 16 KS for MT m-tiles of W (rows m0 + 16 i) and the four
// n-tiles of the block's rows; P0..P3 are consecutive [row][k] planes `plane` elements apart.  ring: the
// warp's kTrRing stages.
template <int MT, int KS>
__device__ __forceinline__ void tr_gemm(const __nv_bfloat16 *W, int ldw, int m0, const __nv_bfloat16 *P, int ld,
                                        int plane, __nv_bfloat16 *ring, int lane, float (&dh)[MT][4][4],
                                        float (&dt)[MT][4][4]) {
    __syncwarp();   // the ring's previous contents have been read by every lane
#pragma unroll
    for (int s = 0; s < kTrRing - 1; ++s) {
        if (s < KS) tr_ring_fill<MT>(W, ldw, m0, 16 * s, ring + s * kTrStage, lane);
        else asm volatile("cp.async.commit_group;" ::: "memory");
    }
#pragma unroll 1
    for (int ks = 0; ks < KS; ++ks) {
        const int kn = ks + kTrRing - 1;
        if (kn < KS) tr_ring_fill<MT>(W, ldw, m0, 16 * kn, ring + (kn % kTrRing) * kTrStage, lane);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group %0;" ::"n"(kTrRing - 1) : "memory");
        __syncwarp();
        uint32_t a[MT][4];
#pragma unroll
        for (int i = 0; i < MT; ++i) tr_frag_a_ring(ring + (ks % kTrRing) * kTrStage, i, lane, a[i]);
#pragma unroll
        for (int op = 0; op < 4; ++op) {
            uint32_t b[2][4];
            tr_frag_b2(P + op * plane, ld, 0, 16 * ks, lane, b[0]);
            tr_frag_b2(P + op * plane, ld, 2, 16 * ks, lane, b[1]);
#pragma unroll
            for (int i = 0; i < MT; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float(&d)[4] = op < 2 ? dh[i][j] : dt[i][j];
                    tr_mma(d, a[i], b[j >> 1][2 * (j & 1)], b[j >> 1][2 * (j & 1) + 1]);
                }
        }
        __syncwarp();   // every lane's ldmatrix of this stage is done before it is refilled
    }
}

// x as the BF16 pair (hi, lo) at [r][c] of two planes; returns hi = bf16(x).
__device__ __forceinline__ __nv_bfloat16 tr_put_pair(__nv_bfloat16 *hi, __nv_bfloat16 *lo, int idx, float x) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[idx] = h;
    lo[idx] = __float2bfloat16_rn(x - __bfloat162float(h));
    return h;
}

// Two per-lane column sums (units g and g + 8 of a fragment) summed over the four lanes of the quad
// (t4 = 0..3, xor 1 then xor 2: a fixed order) and stored by lane t4 = 0 at columns ca and cb.
__device__ __forceinline__ void tr_quad_sums(const float (&x)[2], const float (&y)[2], float *out, int ca, int cb,
                                             int t4) {
    float v[4] = {x[0], x[1], y[0], y[1]};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] += __shfl_xor_sync(0xffffffffu, v[k], 1);
        v[k] += __shfl_xor_sync(0xffffffffu, v[k], 2);
    }
    if (t4 == 0) {
        out[ca] = v[0];
        out[ca + 8] = v[1];
        out[cb] = v[2];
        out[cb + 8] = v[3];
    }
}

__global__ void __launch_bounds__(256, 1) k_mlp_train(LearnedDev L, const float *U, const float *c_row, RowOut o) {
    const int r0 = blockIdx.x * kTrRows;
    if (r0 >= *L.n_tiles_live * kRowTile) return;
    extern __shared__ __align__(16) unsigned char tr_smem[];
    __nv_bfloat16 *sX = reinterpret_cast<__nv_bfloat16 *>(tr_smem);              // G hi, G lo, U hi, U lo
    __nv_bfloat16 *sA = sX + 4 * kPlaneX;                                        // a1 hi, lo, ta1 hi, lo
    __nv_bfloat16 *sB = sX;                                                      // bt2 hi, lo, bh2 hi, lo
    __nv_bfloat16 *ring = sA + 4 * kPlaneA + (threadIdx.x >> 5) * kTrRing * kTrStage;   // the warp's weight ring
    __shared__ float sc[kTrRows];
    __shared__ int sreal[kTrRows];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int e = L.tile_el[r0 / kRowTile];
    if (t < kTrRows) {
        sreal[t] = L.atom_of[r0 + t] >= 0;
        sc[t] = c_row[r0 + t];
    }
    __syncthreads();
    for (int q = t; q < kTrRows * kNFeat / 4; q += 256) {
        const int r = q / (kNFeat / 4), f = 4 * (q % (kNFeat / 4));
        const bool re = sreal[r];
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 gv = re ? *reinterpret_cast<const float4 *>(L.G32 + (size_t)(r0 + r) * kNFeat + f) : z;
        const float4 uv = re ? *reinterpret_cast<const float4 *>(U + (size_t)(r0 + r) * kNFeat + f) : z;
        const float gs[4] = {gv.x, gv.y, gv.z, gv.w}, us[4] = {uv.x, uv.y, uv.z, uv.w};
        __align__(8) __nv_bfloat16 uh[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            tr_put_pair(sX, sX + kPlaneX, r * kXs + f + c, gs[c]);
            uh[c] = tr_put_pair(sX + 2 * kPlaneX, sX + 3 * kPlaneX, r * kXs + f + c, us[c]);
        }
        *reinterpret_cast<uint2 *>(o.u16 + (size_t)(r0 + r) * kNFeat + f) = *reinterpret_cast<const uint2 *>(uh);
    }
    __syncthreads();
    // ---- layer 1: units 32 w + 16 i + g (+ 8), rows 8 j + 2 t4 (+ 1)
    float h1[2][4][4], t1[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) h1[i][j][q] = t1[i][j][q] = 0.f;
    tr_gemm<2, kNFeat / 16>(L.W1 + (size_t)e * kH1 * kNFeat, kNFeat, 32 * w, sX, kXs, kPlaneX, ring, lane, h1, t1);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int u = 32 * w + 16 * i + g + 8 * (q >> 1);
            const float b = L.b1[e * kH1 + u];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = 8 * j + 2 * t4 + (q & 1);
                const float h = h1[i][j][q] + b, a1 = tr_s(h), ta1 = tr_ds(h) * t1[i][j][q];
                h1[i][j][q] = h;
                o.a1[(size_t)(r0 + r) * kH1 + u] = tr_put_pair(sA, sA + kPlaneA, r * kAs + u, a1);
                o.ta1[(size_t)(r0 + r) * kH1 + u] = tr_put_pair(sA + 2 * kPlaneA, sA + 3 * kPlaneA, r * kAs + u, ta1);
            }
        }
    __syncthreads();
    // s'(h1) and s''(h1) t1 of the warp's fragments go to the free tail of the G / U planes (FP32, columns
    // swizzled by the row so that a fragment's lanes hit 32 banks); layer 1' reads them back
    float *sD = reinterpret_cast<float *>(sX + 4 * kPlaneB);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int u = 32 * w + 16 * i + g + 8 * (q >> 1), r = 8 * j + 2 * t4 + (q & 1);
                const int idx = r * kH1 + (u ^ ((r & 7) << 2));
                sD[idx] = tr_ds(h1[i][j][q]);
                sD[kTrRows * kH1 + idx] = tr_dds(h1[i][j][q]) * t1[i][j][q];
            }
    // ---- layer 2: units 16 w + g (+ 8); the bt2 / bh2 planes replace the G / U planes
    {
        float h2[1][4][4], t2[1][4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) h2[0][j][q] = t2[0][j][q] = 0.f;
        tr_gemm<1, kH1 / 16>(L.W2 + (size_t)e * kH2 * kH1, kH1, 16 * w, sA, kAs, kPlaneA, ring, lane, h2, t2);
        float vb2[2] = {0.f, 0.f}, vw3[2] = {0.f, 0.f};   // unit g and g + 8: the lane's rows, then the quad's
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int v = 16 * w + g + 8 * (q >> 1);
            const float b = L.b2[e * kH2 + v], w3 = L.W3[e * kH2 + v];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = 8 * j + 2 * t4 + (q & 1);
                const float cr = sc[r];
                const float h = h2[0][j][q] + b, tt = t2[0][j][q];
                const float d1 = tr_ds(h);
                const float bt2 = -w3 * d1;
                const float bh2 = -w3 * tr_dds(h) * tt + cr * w3 * d1;
                if (sreal[r]) {
                    vb2[q >> 1] += bh2;
                    vw3[q >> 1] += cr * tr_s(h) - d1 * tt;
                }
                o.bt2[(size_t)(r0 + r) * kH2 + v] = tr_put_pair(sB, sB + kPlaneB, r * kBs + v, bt2);
                o.bh2[(size_t)(r0 + r) * kH2 + v] = tr_put_pair(sB + 2 * kPlaneB, sB + 3 * kPlaneB, r * kBs + v, bh2);
            }
        }
        tr_quad_sums(vb2, vw3, o.vpart + (size_t)blockIdx.x * kVLen, kVb2 + 16 * w + g, kVW3 + 16 * w + g, t4);
    }
    __syncthreads();
    // ---- layer 1' (the same units as layer 1)
    float bta1[2][4][4], ba1[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) bta1[i][j][q] = ba1[i][j][q] = 0.f;
    tr_gemm<2, kH2 / 16>(L.W2T + (size_t)e * kH1 * kH2, kH2, 32 * w, sB, kBs, kPlaneB, ring, lane, bta1, ba1);
    float vb1[2][2] = {{0.f, 0.f}, {0.f, 0.f}};   // [i][unit g, g + 8]
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int u = 32 * w + 16 * i + g + 8 * (q >> 1);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = 8 * j + 2 * t4 + (q & 1);
                const int idx = r * kH1 + (u ^ ((r & 7) << 2));
                const float d1 = sD[idx], dd = sD[kTrRows * kH1 + idx];
                const float bh1 = dd * bta1[i][j][q] + d1 * ba1[i][j][q];
                o.bt1[(size_t)(r0 + r) * kH1 + u] = __float2bfloat16_rn(d1 * bta1[i][j][q]);
                o.bh1[(size_t)(r0 + r) * kH1 + u] = __float2bfloat16_rn(bh1);
                if (sreal[r]) vb1[i][q >> 1] += bh1;
            }
        }
    float *vp = o.vpart + (size_t)blockIdx.x * kVLen;
    tr_quad_sums(vb1[0], vb1[1], vp, kVb1 + 32 * w + g, kVb1 + 32 * w + 16 + g, t4);
    if (t == 0) {
        float c = 0.f;
        for (int r = 0; r < kTrRows; ++r)
            if (sreal[r]) c += sc[r];
        vp[kVb3] = c;
    }
}

// Per (element, split, column): the block partials of the split's blocks of that element, in block order.
__global__ void k_vsum(LearnedDev L, const float *vpart, float *part) {
    const int e = blockIdx.y, sp = blockIdx.z;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kVLen) return;
    const int nb = *L.n_tiles_live * (kRowTile / kTrRows);
    const int b0 = (int)((long long)nb * sp / kVSplits), b1 = (int)((long long)nb * (sp + 1) / kVSplits);
    float s = 0.f;
    for (int b = b0; b < b1; ++b)
        if (L.tile_el[b / (kRowTile / kTrRows)] == e) s += vpart[(size_t)b * kVLen + j];
    part[((size_t)sp * 4 + e) * kVLen + j] = s;
}

// The vector gradients of element e: the split sums in split order.
__global__ void k_vfinal(const float *part, float *grad) {
    const int e = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kVLen) return;
    float s = 0.f;
    for (int sp = 0; sp < kVSplits; ++sp) s += part[((size_t)sp * 4 + e) * kVLen + j];
    const int col = j < kVb2 ? kOb1 + j : j < kVW3 ? kOb2 + (j - kVb2) : j < kVb3 ? kOW3 + (j - kVW3) : kOb3;
    grad[(size_t)e * kPPE + col] = s;
}

// ------------------------------------------------------------ weight gradients

// ------------------------------------------------------------ AdamW

__global__ void k_adamw(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                        float eps, float wd, float bc1, float bc2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / bc1, vh = vi / bc2;
    p[i] = p[i] - lr * (mh / (sqrtf(vh) + eps) + wd * p[i]);
}

}  // namespace
}  // namespace mdpf

using namespace mdpf;

struct mdpf_trainer {
    int device = 0;
    int max_frames = 0, N = 0, n_max = 0, tiles_max = 0, rows_max = 0;
    double w_force = 10.0;
    double e0[4] = {0, 0, 0, 0};
    LearnedDev L{};
    MlpMaps maps{};
    std::vector<void *> allocs;
    int *d_cnt = nullptr, *d_ntile = nullptr, *d_tile_off = nullptr, *d_live = nullptr;
    float4 *d_pos4 = nullptr;
    unsigned long long *d_fx = nullptr, *d_efx = nullptr;
    unsigned long long *d_ecore = nullptr;   // [max_frames] repulsive-core energy per frame (fixed point)
    uint32_t *d_status = nullptr;
    float *d_c = nullptr, *d_v = nullptr, *d_U = nullptr;
    RowOut ro{};
    float *d_part = nullptr;
    int *d_etiles = nullptr;
    int4 *d_wsplit = nullptr;
    double *d_lparts = nullptr;
    unsigned int *d_rmin = nullptr, *d_rmax = nullptr;
    std::string err;
    bool sticky = false;
};

namespace {
thread_local std::string g_tr_error;

template <typename T>
cudaError_t talloc(mdpf_trainer *t, T **p, size_t count) {
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
    if (e == cudaSuccess) t->allocs.push_back((void *)*p);
    return e;
}

void tr_free(mdpf_trainer *t) {
    if (!t) return;
    for (void *p : t->allocs) cudaFree(p);
    delete t;
}

int tr_fail(mdpf_trainer *t, int code, const std::string &m) {
    if (t) t->err = m; else g_tr_error = m;
    return code;
}
int tr_cuda(mdpf_trainer *t, cudaError_t e, const char *where) {
    std::string m = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
    if (t) {
        t->sticky = true;
        t->err = m;
    } else {
        g_tr_error = m;
    }
    return MDPF_ERR_CUDA;
}
}  // namespace

extern "C" {

const char *mdpf_trainer_last_error(const mdpf_trainer *t) { return t ? t->err.c_str() : g_tr_error.c_str(); }

int mdpf_trainer_create(const mdpf_train_params *p, mdpf_trainer **out) {
    if (!out) return tr_fail(nullptr, MDPF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!p) return tr_fail(nullptr, MDPF_ERR_INVALID_ARG, "params is NULL");
    if (p->max_frames < 1 || p->atoms_per_frame < 1 || (int64_t)p->max_frames * p->atoms_per_frame > (1 << 22))
        return tr_fail(nullptr, MDPF_ERR_INVALID_ARG, "max_frames, atoms_per_frame out of range");
    if (!(p->w_force >= 0.0)) return tr_fail(nullptr, MDPF_ERR_INVALID_ARG, "w_force must be >= 0");
    if (p->core_rc != 0.0 && (!(p->core_a > 0.0 && p->core_a <= 1e5) || !(p->core_rc > 0.0 && p->core_rc <= 2.0)))
        return tr_fail(nullptr, MDPF_ERR_INVALID_ARG, "core A must be in (0, 1e5] and r_c in (0, 2] (or r_c 0: none)");
    mdpf_trainer *t = new mdpf_trainer();
    t->max_frames = p->max_frames;
    t->N = p->atoms_per_frame;
    t->n_max = p->max_frames * p->atoms_per_frame;
    t->tiles_max = p->max_frames * ((p->atoms_per_frame + kRowTile - 1) / kRowTile + 4);
    t->rows_max = t->tiles_max * kRowTile;
    t->w_force = p->w_force;
    for (int e = 0; e < 4; ++e) t->e0[e] = p->e0[e];
    LearnedDev &L = t->L;
    cudaError_t ce = cudaSuccess;
#define TA(ptr, count)                                                                   \
    do {                                                                                 \
        if ((ce = talloc(t, &(ptr), (count))) != cudaSuccess) {                          \
            tr_cuda(nullptr, ce, "trainer allocation");                                  \
            tr_free(t);                                                                  \
            return ce == cudaErrorMemoryAllocation ? MDPF_ERR_OOM : MDPF_ERR_CUDA;       \
        }                                                                                \
    } while (0)
    const size_t R = t->rows_max, n = t->n_max;
    int *row_of, *atom_of, *tile_el, *live;
    __nv_bfloat16 *W1, *W1T, *W2, *W2T;
    float *b1, *b2, *W3, *b3;
    double *e0;
    CellGrid *grid;
    cudaGetDevice(&t->device);
    TA(t->d_cnt, 4 * (size_t)t->max_frames);
    TA(t->d_ntile, t->max_frames);
    TA(t->d_tile_off, t->max_frames + 1);
    TA(live, 1);
    t->d_live = live;
    TA(row_of, n);
    TA(atom_of, R);
    TA(tile_el, t->tiles_max);
    TA(L.nb_count, n);
    TA(L.nb_idx, n * kKmax);
    TA(L.pos_build, n);
    TA(grid, 1);
    TA(L.bbox, 8);
    TA(L.G16, R * kNFeat);
    TA(L.G32, R * kNFeat);
    {
        __nv_bfloat16 *gbuf = nullptr;   // dE/dG in BF16, as the tensor-core MLP writes it
        TA(gbuf, R * kNFeat);
        L.g = gbuf;
        L.g_f32 = 0;
    }
    TA(L.E_row, R);
    TA(W1, 4 * (size_t)kH1 * kNFeat);
    TA(W1T, 4 * (size_t)kH1 * kNFeat);
    TA(W2, 4 * (size_t)kH2 * kH1);
    TA(W2T, 4 * (size_t)kH2 * kH1);
    TA(b1, 4 * kH1);
    TA(b2, 4 * kH2);
    TA(W3, 4 * kH2);
    TA(b3, 4);
    TA(e0, 4);
    TA(L.lflags, 4);
    TA(L.lcount, 4);
    TA(t->d_pos4, n);
    TA(t->d_fx, 3 * n);
    TA(t->d_efx, E_SLOTS);
    TA(t->d_status, 4);
    TA(t->d_c, R);
    TA(t->d_v, 3 * n);
    TA(t->d_U, R * kNFeat);
    TA(t->ro.bh1, R * kH1);
    TA(t->ro.bt1, R * kH1);
    TA(t->ro.a1, R * kH1);
    TA(t->ro.ta1, R * kH1);
    TA(t->ro.bh2, R * kH2);
    TA(t->ro.bt2, R * kH2);
    TA(t->ro.u16, R * kNFeat);
    TA(t->ro.vpart, (R / kTrRows) * kVLen);
    TA(t->d_part, (size_t)kSplits * 4 * kH1 * kNFeat);
    static_assert((size_t)kWgSplits * (kH1 * kNFeat + kH2 * kH1) <= (size_t)kSplits * 4 * kH1 * kNFeat,
                  "partial buffer");
    static_assert((size_t)kVSplits * 4 * kVLen <= (size_t)kSplits * 4 * kH1 * kNFeat, "vector partial buffer");
    TA(t->d_etiles, 4 * (size_t)t->tiles_max);
    TA(t->d_wsplit, kWgSplits);
    TA(t->d_lparts, 2 * (size_t)t->max_frames);
    TA(t->d_ecore, (size_t)t->max_frames);
    TA(t->d_rmin, 4 * kNFeat);
    TA(t->d_rmax, 4 * kNFeat);
#undef TA
    L.n = t->n_max;
    L.n_rows = (int)R;
    L.n_tiles_live = live;
    L.row_of = row_of;
    L.atom_of = atom_of;
    L.tile_el = tile_el;
    L.rc_list = 5.2f;
    L.rc_list2 = (float)(5.2 * 5.2);
    L.half_skin2 = 0.f;
    L.grid = grid;
    L.W1 = W1;
    L.W1T = W1T;
    L.W2 = W2;
    L.W2T = W2T;
    L.b1 = b1;
    L.b2 = b2;
    L.W3 = W3;
    L.b3 = b3;
    L.e0 = e0;
    L.lo = L.hi = nullptr;
    L.core_a = (float)p->core_a;
    L.core_rc = (float)p->core_rc;
    cudaError_t e1 = cudaMemcpy(e0, t->e0, sizeof(double) * 4, cudaMemcpyHostToDevice);
    if (e1 == cudaSuccess) e1 = cudaMemset(atom_of, 0xFF, sizeof(int) * R);
    if (e1 == cudaSuccess) e1 = cudaMemset(L.G16, 0, sizeof(__nv_bfloat16) * R * kNFeat);
    if (e1 == cudaSuccess) e1 = cudaMemset(L.lflags, 0, sizeof(unsigned int) * 4);
    if (e1 == cudaSuccess) e1 = cudaMemset(t->d_rmin, 0xFF, sizeof(unsigned int) * 4 * kNFeat);
    if (e1 == cudaSuccess) e1 = cudaMemset(t->d_rmax, 0, sizeof(unsigned int) * 4 * kNFeat);
    if (e1 != cudaSuccess) {
        tr_cuda(nullptr, e1, "trainer initialisation");
        tr_free(t);
        return MDPF_ERR_CUDA;
    }
    // TMA descriptors of the tensor-core MLP operands
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    e1 = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e1 != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        tr_free(t);
        return tr_fail(nullptr, MDPF_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    }
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    auto one = [&](CUtensorMap *m, const void *ptr, uint64_t inner, uint64_t rows) {
        cuuint64_t dims[2] = {inner, rows};
        cuuint64_t strides[1] = {inner * 2};
        cuuint32_t box[2] = {64, 128};
        cuuint32_t estr[2] = {1, 1};
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    if (!one(&t->maps.g, L.G16, kNFeat, R) || !one(&t->maps.w1, W1, kNFeat, 4 * kH1) ||
        !one(&t->maps.w2, W2, kH1, 4 * kH2) || !one(&t->maps.w2t, W2T, kH2, 4 * kH1) ||
        !one(&t->maps.w1t, W1T, kH1, 4 * kNFeat)) {
        tr_free(t);
        return tr_fail(nullptr, MDPF_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    }
    e1 = learned_mlp_tc_prepare();
    if (e1 == cudaSuccess) e1 = learned_wgrad_tc_prepare();
    if (e1 == cudaSuccess) e1 = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrSmem);
    if (e1 != cudaSuccess) {
        tr_free(t);
        return tr_cuda(nullptr, e1, "training kernel attributes");
    }
    *out = t;
    return MDPF_OK;
}

void mdpf_trainer_destroy(mdpf_trainer *t) {
    if (!t) return;
    cudaDeviceSynchronize();
    tr_free(t);
}

int mdpf_trainer_loss_grad(mdpf_trainer *t, const float *d_params, float *d_grad, int32_t n_frames,
                           const double *d_pos, const int32_t *d_element, const double *d_E_ref,
                           const float *d_F_ref, double *d_loss3, void *stream) {
    if (!t) return MDPF_ERR_INVALID_ARG;
    if (t->sticky) return MDPF_ERR_CUDA;
    if (n_frames < 1 || n_frames > t->max_frames) return tr_fail(t, MDPF_ERR_INVALID_ARG, "n_frames out of range");
    if (!d_params || !d_grad || !d_pos || !d_element || !d_E_ref || !d_F_ref || !d_loss3)
        return tr_fail(t, MDPF_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int N = t->N, B = n_frames, n = B * N;
    LearnedDev L = t->L;
    L.n = n;
    L.el = d_element;
    // 1. rows
    k_tr_count<<<B, 256, 0, s>>>(d_element, N, t->d_cnt, t->d_ntile);
    k_tr_scan<<<1, 32, 0, s>>>(B, t->d_ntile, t->d_tile_off, t->d_live);
    cudaMemsetAsync(const_cast<int *>(L.atom_of), 0xFF, sizeof(int) * t->rows_max, s);
    k_tr_rows<<<B, 1024, 0, s>>>(d_element, N, t->d_cnt, t->d_tile_off, const_cast<int *>(L.row_of),
                                  const_cast<int *>(L.atom_of), const_cast<int *>(L.tile_el));
    // 2. positions, neighbours, weights
    k_tr_pos<<<(n + 255) / 256, 256, 0, s>>>(d_pos, n, t->d_pos4);
    cudaMemsetAsync(t->d_status, 0, sizeof(uint32_t), s);
    k_tr_nb<<<(n + kTrNbThreads - 1) / kTrNbThreads, kTrNbThreads, 0, s>>>(L, t->d_pos4, N, t->d_status);
    k_tr_weights<<<dim3((kH1 * kNFeat + 255) / 256, 4), 256, 0, s>>>(
        d_params, const_cast<__nv_bfloat16 *>(L.W1), const_cast<__nv_bfloat16 *>(L.W1T),
        const_cast<__nv_bfloat16 *>(L.W2), const_cast<__nv_bfloat16 *>(L.W2T), const_cast<float *>(L.b1),
        const_cast<float *>(L.b2), const_cast<float *>(L.W3), const_cast<float *>(L.b3));
    // 3. features, MLP (energies, dE/dG), forces
    cudaMemsetAsync(L.G16, 0, sizeof(__nv_bfloat16) * (size_t)t->rows_max * kNFeat, s);
    learned_features(L, t->d_pos4, true, s);
    k_tr_range<<<t->tiles_max, kNFeat, 0, s>>>(L, t->d_rmin, t->d_rmax);
    cudaError_t ce = learned_mlp_tc(L, t->maps, t->d_status, false, nullptr, s);
    if (ce != cudaSuccess) return tr_cuda(t, ce, "learned_mlp_tc");
    cudaMemsetAsync(t->d_fx, 0, sizeof(unsigned long long) * 3 * (size_t)n, s);
    cudaMemsetAsync(t->d_ecore, 0, sizeof(unsigned long long) * (size_t)B, s);
    learned_adjoint(L, t->d_pos4, t->d_fx, false, t->d_ecore, N, s);
    // 4. loss, c, v; U = J v
    k_tr_loss<<<B, 256, 0, s>>>(L, N, B, t->w_force, t->d_tile_off, d_E_ref, d_F_ref, t->d_fx, t->d_ecore, t->d_c,
                                 t->d_v, t->d_lparts);
    k_tr_loss_total<<<1, 32, 0, s>>>(B, t->d_lparts, d_loss3);
    learned_jvp(L, t->d_pos4, t->d_v, t->d_U, s);
    // 5. per-row reverse over the tangent pass
    k_mlp_train<<<t->rows_max / kTrRows, 256, kTrSmem, s>>>(L, t->d_U, t->d_c, t->ro);
    // 6. weight-matrix gradients on the tensor cores (K splits over each element's row tiles, summed in
    //    order); the bias and output-weight gradients from the row kernel's per-block column sums, summed by
    //    split in block order, then over the splits in order
    WgradIn wg{t->ro.bh1, t->ro.bt1, L.G16, t->ro.u16, t->ro.bh2, t->ro.bt2, t->ro.a1, t->ro.ta1,
               L.atom_of, L.tile_el, L.n_tiles_live, t->tiles_max, t->d_etiles, t->d_wsplit, t->d_part,
               d_grad, kPPE, kOW1, kOW2, t->d_status};
    ce = learned_wgrad_tc(wg, s);
    if (ce != cudaSuccess) return tr_cuda(t, ce, "learned_wgrad_tc");
    k_vsum<<<dim3((kVLen + 127) / 128, 4, kVSplits), 128, 0, s>>>(L, t->ro.vpart, t->d_part);
    k_vfinal<<<dim3((kVLen + 127) / 128, 4), 128, 0, s>>>(t->d_part, d_grad);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return tr_cuda(t, ce, "training launches");
    return MDPF_OK;
}

int mdpf_trainer_status(mdpf_trainer *t, uint32_t *status) {
    if (!t) return MDPF_ERR_INVALID_ARG;
    if (t->sticky) return MDPF_ERR_CUDA;
    uint32_t st = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&st, t->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return tr_cuda(t, e, "trainer status");
    if (status) *status = st;
    if (st & MDPF_STATUS_TIMEOUT) return tr_fail(t, MDPF_ERR_TIMEOUT, "tensor-core MLP wait timed out");
    if (st & MDPF_STATUS_NEIGHBOR_OVERFLOW) return tr_fail(t, MDPF_ERR_NEIGHBOR_OVERFLOW, "neighbour row over 128");
    return MDPF_OK;
}

int mdpf_trainer_feature_range(mdpf_trainer *t, float *lo, float *hi) {
    if (!t) return MDPF_ERR_INVALID_ARG;
    if (t->sticky) return MDPF_ERR_CUDA;
    std::vector<unsigned int> a(4 * kNFeat), b(4 * kNFeat);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(a.data(), t->d_rmin, sizeof(unsigned int) * a.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(b.data(), t->d_rmax, sizeof(unsigned int) * b.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return tr_cuda(t, e, "feature range");
    auto un = [](unsigned int u) {
        const unsigned int bits = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;
        float f;
        std::memcpy(&f, &bits, 4);
        return f;
    };
    for (int k = 0; k < 4 * kNFeat; ++k) {
        const bool seen = a[k] != 0xFFFFFFFFu;
        if (lo) lo[k] = seen ? un(a[k]) : 0.f;
        if (hi) hi[k] = seen ? un(b[k]) : 0.f;
    }
    return MDPF_OK;
}

int mdpf_adamw_step(float *d_params, const float *d_grad, float *d_m, float *d_v, int64_t n, int64_t step, double lr,
                    double beta1, double beta2, double eps, double weight_decay, void *stream) {
    if (!d_params || !d_grad || !d_m || !d_v || n < 0 || step < 1) return MDPF_ERR_INVALID_ARG;
    if (n == 0) return MDPF_OK;
    const float bc1 = (float)(1.0 - std::pow(beta1, (double)step)), bc2 = (float)(1.0 - std::pow(beta2, (double)step));
    k_adamw<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_params, d_grad, d_m, d_v, n, (float)lr,
                                                                        (float)beta1, (float)beta2, (float)eps,
                                                                        (float)weight_decay, bc1, bc2);
    return cudaGetLastError() == cudaSuccess ? MDPF_OK : MDPF_ERR_CUDA;
}

}  // extern "C"
