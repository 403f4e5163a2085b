// Learned-potential kernels: cell-list neighbour build, symmetry-function
// features, per-element MLP (forward and input gradient), feature adjoint,
// feature JVP.  The per-atom feature and adjoint arithmetic is in
// learned_terms.cuh (shared with the fused tile kernel).
//
//   E_i = W3 . celu(W2 celu(W1 G_i + b1) + b2) + b3 + e0,  celu(x) = max(x, 0.1 (exp(10 x) - 1))
// Every accumulation that feeds a result is done in a fixed order per lane, and
// forces are int64 fixed-point sums, so results are reproducible bit for bit.
#include <cuda_bf16.h>

#include "learned.cuh"
#include "learned_terms.cuh"

namespace mdpf {
namespace {

constexpr float kCeluAlpha = 0.1f;

// CELU(0.1) and its derivative, exp(10 x) from the fast exponential (as in the tensor-core MLP)
__device__ __forceinline__ float celu(float x) { return x > 0.f ? x : kCeluAlpha * (__expf(10.f * x) - 1.f); }
__device__ __forceinline__ float dcelu(float x) { return x >= 0.f ? 1.f : __expf(10.f * x); }
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ unsigned int ord_f(float f) {
    unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord_f(unsigned int u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

// ------------------------------------------------------------------ neighbour list
//
// One cooperative kernel: it returns at once unless a rebuild is requested
// (or forced); otherwise four phases separated by grid barriers:
//   A  bounding box (block min/max, then global ordered-int atomics) and the
//      first two moments of the positions per axis (fixed-point sums)
//   B  cell grid (computed identically by every block), cells cleared: the
//      bounding box cut to mean +- 4 standard deviations per axis, so that a
//      few atoms far from the rest (a gas-phase cluster evaporates) do not
//      stretch the cells; atoms outside the grid fall in its edge cells
//   C  cell fill (atomic slot per atom; overflow flagged, never written)
//   D  rows: every j != i in the 27 surrounding cells with
//      fl(fl(fl(dx^2) + fl(dy^2)) + fl(dz^2)) < fl32(rc^2), sorted ascending.
// The barrier counter is monotonic; its base for the next build is stored
// after the last barrier, so no reset is needed between launches.  Each wait
// gives up after limit_ns (MDPF_STATUS_TIMEOUT).

__device__ __forceinline__ unsigned long long nb_atom_add_release(unsigned long long *p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned long long nb_ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long nb_timer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool nb_barrier(unsigned long long *bar, unsigned long long target, uint32_t *status,
                                           long long limit_ns, int *s_fail) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int fail = 0;
        if (gridDim.x > 1) {
            __threadfence();
            nb_atom_add_release(bar, 1ull);
            const unsigned long long t0 = nb_timer();
            unsigned int spins = 0;
            while (nb_ld_acquire(bar) < target) {
                if ((++spins & 31u) == 0u && (long long)(nb_timer() - t0) > limit_ns) {
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

// Fixed-point scales of the position moments (sums over atoms of u = x - x0 and u^2, u clamped to
// +-1e4 A so that both products fit 32-bit integers: the conversions are the 32-bit ones), and the number
// of copies of the six sums that the blocks' adds are spread over.
constexpr float kMom1 = 64.f, kMom2 = 4.f, kMomClamp = 1.0e4f;
constexpr int kMomCopies = 8;

// The grid: per axis the bounding box [lo, hi], cut to mu +- 4 sigma of the
// positions (mom: the fixed-point sums, n atoms, x0 the reference position).
// Clamping a cell index to the grid never moves two indices further apart,
// so two atoms within the list radius stay in neighbouring cells wherever
// they are; the cut only decides how wide the cells are.
__device__ __forceinline__ CellGrid make_grid(const unsigned int *bb, const long long *mom, int n, float4 x0,
                                              float rc_list) {
    float lo[3], ext = 0.f, e3[3];
    const float ref[3] = {x0.x, x0.y, x0.z};
    for (int d = 0; d < 3; ++d) {
        lo[d] = unord_f(bb[d]);
        float hi = unord_f(bb[3 + d]);
        const double m1 = (double)mom[d] / ((double)kMom1 * n), m2 = (double)mom[3 + d] / ((double)kMom2 * n);
        const double sd = sqrt(fmax(m2 - m1 * m1, 0.0));
        const float cl = (float)(ref[d] + m1 - 4.0 * sd), ch = (float)(ref[d] + m1 + 4.0 * sd);
        if (cl < ch) {   // false for non-finite moments: the plain bounding box
            lo[d] = fmaxf(lo[d], cl);
            hi = fminf(hi, ch);
        }
        e3[d] = fmaxf(hi - lo[d], 0.f);
        ext = fmaxf(ext, e3[d]);
    }
    // cells a little wider than the list radius, so that rounding in the cell
    // index never puts two atoms within the radius more than one cell apart
    const float cs = fmaxf(rc_list * 1.001f, ext / (float)kMaxCellDim);
    CellGrid g;
    int nc = 1;
    for (int d = 0; d < 3; ++d) {
        g.lo[d] = lo[d];
        g.dim[d] = max(1, min((int)floorf(e3[d] / cs) + 1, kMaxCellDim + 1));  // non-finite input stays in bounds
        nc *= g.dim[d];
    }
    g.cs = cs;
    g.ncell = nc;
    return g;
}

__device__ __forceinline__ void cell_of(const CellGrid &g, float4 p, int &cx, int &cy, int &cz) {
    cx = min(max((int)floorf((p.x - g.lo[0]) / g.cs), 0), g.dim[0] - 1);
    cy = min(max((int)floorf((p.y - g.lo[1]) / g.cs), 0), g.dim[1] - 1);
    cz = min(max((int)floorf((p.z - g.lo[2]) / g.cs), 0), g.dim[2] - 1);
}

// Row of atom i by one warp: candidates of the 27 cells 32 at a time, accepted
// ones appended in shared memory (ballot order), then written out in ascending
// order (each entry's rank among the distinct entries).  Returns the row
// length (kKmax + 1 when the row overflowed).
// Candidates of the 27 cells around atom i, in (z, y, x) cell order and slot
// order within a cell: lane c < 27 reads cell c's count, a warp scan gives
// each cell's first candidate index, and the candidates are then taken 32 at
// a time across cells (three dependent memory trips per 32 candidates instead
// of per cell).
struct CellScan {
    int start[28];  // first candidate index of cell c; start[27] = total
    int cell[27];   // cell id, or -1 outside the grid
};

__device__ int build_row_warp(const LearnedDev &L, const float4 *pos4, const CellGrid &g, int i, int lane,
                              int *srow, CellScan &cs) {
    const float4 pi = pos4[i];
    int cx, cy, cz;
    cell_of(g, pi, cx, cy, cz);
    int cid = -1, ccnt = 0;
    if (lane < 27) {
        const int z = cz - 1 + lane / 9, y = cy - 1 + (lane / 3) % 3, x = cx - 1 + lane % 3;
        if (z >= 0 && z < g.dim[2] && y >= 0 && y < g.dim[1] && x >= 0 && x < g.dim[0]) {
            cid = (z * g.dim[1] + y) * g.dim[0] + x;
            ccnt = min(L.cell_cnt[cid], kCellCap);
        }
    }
    int incl = ccnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    if (lane < 27) {
        cs.start[lane] = incl - ccnt;
        cs.cell[lane] = cid;
    }
    if (lane == 27) cs.start[27] = total;
    __syncwarp();
    int m = 0;
    for (int k0 = 0; k0 < total; k0 += 32) {
        const int k = k0 + lane;
        int j = -1;
        bool in = false;
        if (k < total) {
            // the cell holding candidate k: the last c with start[c] <= k (empty cells share their start)
            int lo = 0, hi = 26;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (cs.start[mid] <= k) lo = mid;
                else hi = mid - 1;
            }
            j = L.cell_atoms[(size_t)cs.cell[lo] * kCellCap + (k - cs.start[lo])];
            if (j != i) {
                const float4 pj = pos4[j];
                const float dx = __fsub_rn(pj.x, pi.x), dy = __fsub_rn(pj.y, pi.y), dz = __fsub_rn(pj.z, pi.z);
                in = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)) < L.rc_list2;
            }
        }
        const unsigned int bal = __ballot_sync(0xffffffffu, in);
        const int pos = m + __popc(bal & ((1u << lane) - 1u));
        if (in && pos < kKmax) srow[pos] = j;
        m += __popc(bal);
    }
    __syncwarp();
    const int mm = min(m, kKmax);
    int *out = L.nb_idx + (size_t)i * kKmax;
    for (int p = lane; p < mm; p += 32) {
        const int v = srow[p];
        int rank = 0;
        for (int q = 0; q < mm; ++q) rank += srow[q] < v;
        out[rank] = v;
    }
    if (lane == 0) {
        L.nb_count[i] = mm;
        L.pos_build[i] = pi;
    }
    __syncwarp();
    return m > kKmax ? kKmax + 1 : m;
}

constexpr int kNbThreads = 256;

__global__ void __launch_bounds__(kNbThreads) k_nb_all(LearnedDev L, const float4 *pos4, uint32_t *status,
                                                        int forced, long long limit_ns) {
    if (!forced && L.lflags[0] == 0u) return;   // the same decision in every block
    __shared__ unsigned long long s_base;
    __shared__ int s_fail;
    __shared__ unsigned int s_bb[6];
    __shared__ unsigned long long s_mom[6];
    const int nb = gridDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    if (threadIdx.x == 0) s_base = *(volatile unsigned long long *)&L.nb_bar[1];
    if (threadIdx.x < 6) {
        s_bb[threadIdx.x] = threadIdx.x < 3 ? 0xFFFFFFFFu : 0u;
        s_mom[threadIdx.x] = 0ull;
    }
    __syncthreads();
    const unsigned long long base = s_base;
    const float4 x0 = pos4[0];
    // A: bounding box and moments (the global box and sums were reset by the previous build); the moments
    // are integer sums, so they do not depend on the order of the adds
    long long m[6] = {0, 0, 0, 0, 0, 0};
    for (int a = tid; a < L.n; a += stride) {
        const float4 p = pos4[a];
        atomicMin(&s_bb[0], ord_f(p.x));
        atomicMin(&s_bb[1], ord_f(p.y));
        atomicMin(&s_bb[2], ord_f(p.z));
        atomicMax(&s_bb[3], ord_f(p.x));
        atomicMax(&s_bb[4], ord_f(p.y));
        atomicMax(&s_bb[5], ord_f(p.z));
        const float q[3] = {p.x - x0.x, p.y - x0.y, p.z - x0.z};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float u = fminf(fmaxf(q[d], -kMomClamp), kMomClamp);   // non-finite positions stay bounded
            m[d] += __float2int_rn(u * kMom1);
            m[3 + d] += __float2int_rn(u * u * kMom2);
        }
    }
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        long long v = m[d];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v != 0) atomicAdd(&s_mom[d], (unsigned long long)v);
    }
    __syncthreads();
    if (threadIdx.x < 3) atomicMin(&L.bbox[threadIdx.x], s_bb[threadIdx.x]);
    else if (threadIdx.x < 6) atomicMax(&L.bbox[threadIdx.x], s_bb[threadIdx.x]);
    else if (threadIdx.x < 12 && s_mom[threadIdx.x - 6] != 0ull)
        atomicAdd(reinterpret_cast<unsigned long long *>(&L.bmom[6 * (blockIdx.x % kMomCopies) + threadIdx.x - 6]),
                  s_mom[threadIdx.x - 6]);
    if (!nb_barrier(L.nb_bar, base + nb, status, limit_ns, &s_fail)) return;
    // B: the grid (identical in every block), cells cleared
    // one thread per block reads the box and the sums (every thread reading the same few words made them a
    // hot spot) and forms the grid for the block
    __shared__ CellGrid s_grid;
    if (threadIdx.x == 0) {
        unsigned int bb[6];
        long long mom[6] = {0, 0, 0, 0, 0, 0};
        for (int d = 0; d < 6; ++d) bb[d] = *(volatile unsigned int *)&L.bbox[d];
        for (int k = 0; k < kMomCopies; ++k)
            for (int d = 0; d < 6; ++d) mom[d] += *(volatile long long *)&L.bmom[6 * k + d];
        s_grid = make_grid(bb, mom, L.n, x0, L.rc_list);
    }
    __syncthreads();
    const CellGrid g = s_grid;
    for (int c = tid; c < g.ncell; c += stride) L.cell_cnt[c] = 0;
    if (!nb_barrier(L.nb_bar, base + 2ull * nb, status, limit_ns, &s_fail)) return;
    // every block has read the box and the moments: reset them for the next build
    if (blockIdx.x == 0 && threadIdx.x < 6) L.bbox[threadIdx.x] = threadIdx.x < 3 ? 0xFFFFFFFFu : 0u;
    if (blockIdx.x == 0 && threadIdx.x < 6 * kMomCopies) L.bmom[threadIdx.x] = 0;
    // C: cell fill
    for (int a = tid; a < L.n; a += stride) {
        int cx, cy, cz;
        cell_of(g, pos4[a], cx, cy, cz);
        const int c = (cz * g.dim[1] + cy) * g.dim[0] + cx;
        const int slot = atomicAdd(&L.cell_cnt[c], 1);
        if (slot < kCellCap) L.cell_atoms[(size_t)c * kCellCap + slot] = a;
        else atomicOr(&L.lflags[2], 1u);
    }
    if (!nb_barrier(L.nb_bar, base + 3ull * nb, status, limit_ns, &s_fail)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (*(volatile unsigned int *)&L.lflags[2]) atomicOr(status, MDPF_STATUS_NEIGHBOR_OVERFLOW);
        L.lflags[2] = 0u;
        L.lflags[0] = 0u;
        L.lcount[0] += 1;
        L.nb_bar[1] = base + 3ull * nb;
        *L.grid = g;
    }
    // D: rows, one warp per atom
    __shared__ int srow[kNbThreads / 32][kKmax];
    __shared__ CellScan scs[kNbThreads / 32];
    __shared__ int s_max[kNbThreads / 32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    int longest = 0;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < L.n; i += nwarps)
        longest = max(longest, build_row_warp(L, pos4, g, i, lane, srow[wib], scs[wib]));
    if (lane == 0) s_max[wib] = longest;
    __syncthreads();
    if (threadIdx.x == 0) {
        int mx = 0;
        for (int w = 0; w < kNbThreads / 32; ++w) mx = max(mx, s_max[w]);
        if (mx > kKmax) atomicOr(status, MDPF_STATUS_NEIGHBOR_OVERFLOW);
        atomicMax((unsigned long long *)&L.lcount[2], (unsigned long long)mx);
    }
}

// Rows of small systems (n <= kNbSmallMax) by brute force, one warp per atom:
// every j != i in index order, 32 at a time, with the row predicate of the
// cell-list build (so the same rows, ascending by construction).  One plain
// launch with no grid barrier: below a few hundred atoms the four phases of
// the cell-list build cost more than the O(n^2) scan.  The last block to
// finish (an arrival count, no waiting) clears the rebuild request and counts
// the build.
constexpr int kNbSmallMax = 512;

__global__ void __launch_bounds__(kNbThreads) k_nb_small(LearnedDev L, const float4 *pos4, uint32_t *status,
                                                          int forced) {
    if (!forced && L.lflags[0] == 0u) return;   // the same decision in every block
    __shared__ int s_max[kNbThreads / 32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int i = blockIdx.x * (kNbThreads / 32) + wib;
    int m = 0;
    if (i < L.n) {
        const float4 pi = pos4[i];
        int *out = L.nb_idx + (size_t)i * kKmax;
        for (int j0 = 0; j0 < L.n; j0 += 32) {
            const int j = j0 + lane;
            bool in = false;
            if (j < L.n && j != i) {
                const float4 pj = pos4[j];
                const float dx = __fsub_rn(pj.x, pi.x), dy = __fsub_rn(pj.y, pi.y), dz = __fsub_rn(pj.z, pi.z);
                in = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)) < L.rc_list2;
            }
            const unsigned int bal = __ballot_sync(0xffffffffu, in);
            const int pos = m + __popc(bal & ((1u << lane) - 1u));
            if (in && pos < kKmax) out[pos] = j;
            m += __popc(bal);
        }
        if (lane == 0) {
            L.nb_count[i] = min(m, kKmax);
            L.pos_build[i] = pi;
        }
    }
    if (lane == 0) s_max[wib] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        int mx = 0;
        for (int w = 0; w < kNbThreads / 32; ++w) mx = max(mx, s_max[w]);
        if (mx > kKmax) atomicOr(status, MDPF_STATUS_NEIGHBOR_OVERFLOW);
        atomicMax((unsigned long long *)&L.lcount[2], (unsigned long long)min(mx, kKmax + 1));
        __threadfence();   // this block's read of the request precedes its arrival
        if (atomicAdd(&L.nb_bar[2], 1ull) == (unsigned long long)gridDim.x - 1ull) {
            L.nb_bar[2] = 0ull;
            L.lflags[0] = 0u;
            L.lcount[0] += 1;
        }
    }
}

// ------------------------------------------------------------------ features

constexpr int kFeatWarps = 2;   // warps (atoms) per block of k_features ...
constexpr int kAtomWarps = 4;   // ... and of k_adjoint and k_jvp (each measured best on c4)

// One warp per atom: neighbours, features (learned_terms.cuh), then the BF16
// GEMM input row (and the FP32 row when asked) and the range check.
__global__ void __launch_bounds__(32 * kFeatWarps) k_features(LearnedDev L, const float4 *pos4, int write_f32) {
    __shared__ NbrSmem sn[kFeatWarps];
    __shared__ TripStage st[kFeatWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kFeatWarps + w;
    if (i >= L.n) return;
    int cnt, nr, na;
    load_neighbours<true>(L, pos4, i, sn[w], lane, cnt, nr, na);
    float v[12];
    feature_row(sn[w], nr, na, st[w], lane, v);
    const int row = L.row_of[i];
    const int z = L.el[i];
    // every range load before the first store: a load that follows a store through a pointer that may alias
    // it is issued only after that store, so interleaving them costs an L2 round trip per column block
    bool out = false;
    if (L.lo != nullptr) {
#pragma unroll
        for (int b = 0; b < 12; ++b) {
            const int f = 32 * b + lane;
            out |= (v[b] < L.lo[z * kNFeat + f]) || (v[b] > L.hi[z * kNFeat + f]);
        }
    }
#pragma unroll
    for (int b = 0; b < 12; ++b) {
        const int f = 32 * b + lane;
        L.G16[(size_t)row * kNFeat + f] = __float2bfloat16_rn(v[b]);
        if (write_f32) L.G32[(size_t)row * kNFeat + f] = v[b];
    }
    if (__any_sync(0xffffffffu, out) && lane == 0) atomicOr(&L.lflags[1], 1u);
}

// ------------------------------------------------------------------ MLP (CUDA cores)
//
// Rows are grouped by element and padded to kRowTile, so every block of
// kMlpRows rows belongs to one element.  GEMM operands are rounded to BF16,
// products accumulate in FP32.

constexpr int kMlpRows = 8;

// BF16 = true: the tensor-core kernel's rounding points (BF16 features,
// activations and deltas); false: FP32 operands throughout (features from the
// FP32 copy), so the forces are the gradient of the evaluated energy to FP32
// rounding.  Weights are the model's (BF16-valued) in both.
template <bool BF16>
__global__ void __launch_bounds__(256) k_mlp_simt(LearnedDev L, int gated, unsigned long long *efx) {
    if (gated && L.lflags[1]) return;
    if (L.n_tiles_live != nullptr && (int)(blockIdx.x * kMlpRows / kRowTile) >= *L.n_tiles_live) return;
    __shared__ float sG[kMlpRows][kNFeat];
    __shared__ float sA1[kMlpRows][kH1];
    __shared__ float sH1d[kMlpRows][kH1];
    __shared__ float sD2[kMlpRows][kH2];
    __shared__ float sD1[kMlpRows][kH1];
    __shared__ float sE[kMlpRows][4];
    const int t = threadIdx.x;
    const int r0 = blockIdx.x * kMlpRows;
    const int e = L.tile_el[r0 / kRowTile];
    for (int q = t; q < kMlpRows * kNFeat; q += 256) {
        if (BF16) sG[q / kNFeat][q % kNFeat] = __bfloat162float(L.G16[(size_t)r0 * kNFeat + q]);
        else sG[q / kNFeat][q % kNFeat] = L.atom_of[r0 + q / kNFeat] >= 0 ? L.G32[(size_t)r0 * kNFeat + q] : 0.f;
    }
    __syncthreads();
    // layer 1: column a = t
    {
        const __nv_bfloat16 *W = L.W1T + (size_t)e * kNFeat * kH1;
        float acc[kMlpRows];
        const float b = L.b1[e * kH1 + t];
#pragma unroll
        for (int r = 0; r < kMlpRows; ++r) acc[r] = b;
        for (int k = 0; k < kNFeat; ++k) {
            const float wv = __bfloat162float(W[(size_t)k * kH1 + t]);
#pragma unroll
            for (int r = 0; r < kMlpRows; ++r) acc[r] = fmaf(sG[r][k], wv, acc[r]);
        }
#pragma unroll
        for (int r = 0; r < kMlpRows; ++r) {
            // BF16: the tensor-core kernels' operand pair hi + lo (both BF16) of celu(h1), and celu'
            // recovered from celu(h1) as they do (1, or 10 a + 1 below zero)
            const float a = celu(acc[r]);
            const float hi = bf16r(a);
            sA1[r][t] = BF16 ? hi + bf16r(a - hi) : a;
            sH1d[r][t] = BF16 ? (a >= 0.f ? 1.f : fmaf(10.f, a, 1.f)) : dcelu(acc[r]);
        }
    }
    __syncthreads();
    // layer 2 + output layer + delta2: column c = t < 128
    if (t < kH2) {
        const __nv_bfloat16 *W = L.W2T + (size_t)e * kH1 * kH2;
        float acc[kMlpRows];
        const float b = L.b2[e * kH2 + t];
#pragma unroll
        for (int r = 0; r < kMlpRows; ++r) acc[r] = b;
        for (int a = 0; a < kH1; ++a) {
            const float wv = __bfloat162float(W[(size_t)a * kH2 + t]);
#pragma unroll
            for (int r = 0; r < kMlpRows; ++r) acc[r] = fmaf(sA1[r][a], wv, acc[r]);
        }
        const float w3 = L.W3[e * kH2 + t];
#pragma unroll
        for (int r = 0; r < kMlpRows; ++r) {
            float ev = w3 * celu(acc[r]);
            for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
            if ((t & 31) == 0) sE[r][t >> 5] = ev;
            sD2[r][t] = BF16 ? bf16r(w3 * dcelu(acc[r])) : w3 * dcelu(acc[r]);
        }
    }
    __syncthreads();
    if (t < 32) {
        const int row = r0 + t;
        double Er = 0.0;
        if (t < kMlpRows && L.atom_of[row] >= 0)
            Er = (double)(sE[t][0] + sE[t][1] + sE[t][2] + sE[t][3]) + (double)L.b3[e] + L.e0[e];
        if (t < kMlpRows) L.E_row[row] = Er;
        if (efx != nullptr) {   // the block's energy into the fixed-point learned-energy slot
            const double ws = warp_sum_d(Er);
            if (t == 0 && ws != 0.0) fx_add_d(&efx[E_LEARN], ws);
        }
    }
    // backward through layer 2: delta1 = celu'(h1) * (W2^T delta2), column a = t
    {
        const __nv_bfloat16 *W = L.W2 + (size_t)e * kH2 * kH1;
        float acc[kMlpRows];
#pragma unroll
        for (int r = 0; r < kMlpRows; ++r) acc[r] = 0.f;
        for (int c = 0; c < kH2; ++c) {
            const float wv = __bfloat162float(W[(size_t)c * kH1 + t]);
#pragma unroll
            for (int r = 0; r < kMlpRows; ++r) acc[r] = fmaf(sD2[r][c], wv, acc[r]);
        }
#pragma unroll
        for (int r = 0; r < kMlpRows; ++r) sD1[r][t] = BF16 ? bf16r(acc[r] * sH1d[r][t]) : acc[r] * sH1d[r][t];
    }
    __syncthreads();
    // backward through layer 1: dE/dG = W1^T delta1, columns f = t, t + 256
    {
        const __nv_bfloat16 *W = L.W1 + (size_t)e * kH1 * kNFeat;
        for (int f = t; f < kNFeat; f += 256) {
            float acc[kMlpRows];
#pragma unroll
            for (int r = 0; r < kMlpRows; ++r) acc[r] = 0.f;
            for (int a = 0; a < kH1; ++a) {
                const float wv = __bfloat162float(W[(size_t)a * kNFeat + f]);
#pragma unroll
                for (int r = 0; r < kMlpRows; ++r) acc[r] = fmaf(sD1[r][a], wv, acc[r]);
            }
#pragma unroll
            for (int r = 0; r < kMlpRows; ++r) {
                const size_t q = (size_t)(r0 + r) * kNFeat + f;
                if (BF16) static_cast<__nv_bfloat16 *>(L.g)[q] = __float2bfloat16_rn(acc[r]);
                else static_cast<float *>(L.g)[q] = acc[r];
            }
        }
    }
}

// ------------------------------------------------------------------ adjoint

constexpr int kAdjChunk = 128;  // triplets staged per pass

// One warp per atom: g row into the padded per-warp layout, neighbours, then
// the chain rule of learned_terms.cuh (fixed-point force sums).
__global__ void __launch_bounds__(32 * kAtomWarps) k_adjoint(LearnedDev L, const float4 *pos4, unsigned long long *fx,
                                                             int gated, unsigned long long *ecore, int ecore_per) {
    if (gated && L.lflags[1]) return;
    __shared__ NbrSmem sn[kAtomWarps];
    __shared__ AdjScratch<kAdjChunk> sa[kAtomWarps];
    __shared__ __align__(16) float sg[kAtomWarps][kGRow];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kAtomWarps + w;
    if (i >= L.n) return;
    // all global loads first (neighbour row, then its positions alongside the g row), then the stores
    const int row = L.row_of[i];
    NbrFetch nf;
    fetch_neighbours(L, pos4, i, lane, nf);
    float gv[kNFeat / 32];
    if (L.g_f32) {
#pragma unroll
        for (int b = 0; b < kNFeat / 32; ++b) gv[b] = static_cast<const float *>(L.g)[(size_t)row * kNFeat + 32 * b + lane];
    } else {
#pragma unroll
        for (int b = 0; b < kNFeat / 32; ++b)
            gv[b] = __bfloat162float(static_cast<const __nv_bfloat16 *>(L.g)[(size_t)row * kNFeat + 32 * b + lane]);
    }
#pragma unroll
    for (int b = 0; b < kNFeat / 32; ++b) sg[w][g_col(32 * b + lane)] = gv[b];
    int cnt, nr, na;
    store_neighbours<false>(nf, sn[w], lane, cnt, nr, na);
    adjoint_atom(i, sn[w], cnt, nr, na, sg[w], sa[w], fx, lane, make_float2(L.core_a, L.core_rc),
                 ecore != nullptr ? ecore + i / ecore_per : nullptr);
}

// ------------------------------------------------------------------ feature JVP

// Per-warp staging of the JVP: one batch of 32 triplet slots (value and
// tangent factors), the pair-type table and the angular column sums, plus
// w_j = v_j - v_i and the tangent of r_ij for every neighbour.
struct JvpStage {
    float4 q[32];    // cos, sin of the scaled angle, 2^-31 fc(r_j) fc(r_k) = C, pair type
    float4 qd[32];   // cot, 32 x tangent of the scaled cosine, 2^-31 tangent of C, 0
    float4 b[32];    // radial-shell factors B_m of the 4 shells
    float4 bd[32];   // their tangents
    int4 type[10];   // as in the feature stage: first slot, triplets, first angular indices and count, e1 == e2
    float rcp[12];
    float acc[10][32];
    float4 w[kKmax];   // v_j - v_i (x, y, z), tangent of r_ij
};

// Tangent of the features along per-atom vectors v: U_i = sum_a dG_i/dx_a . v_a.
// The lane layout of the features: radial lane 16 h + k sums every second
// in-cutoff neighbour into four per-element registers; angular triplets laid
// out pair type by pair type in padded runs, lane 8 t4 + p taking slot t4 of
// each group of 4 for section p and its four shells, the four slot groups'
// sums combined by a reduce-scatter at each type change.  Per pair the
// tangent of r_ij is u_ij . (v_j - v_i); per triplet that of cos(theta) is
// ((u_k - c u_j)/r_j) . (v_j - v_i) + ((u_j - c u_k)/r_k) . (v_k - v_i).
__global__ void __launch_bounds__(32 * kAtomWarps) k_jvp(LearnedDev L, const float4 *pos4, const float *v, float *U) {
    __shared__ NbrSmem sn[kAtomWarps];
    __shared__ JvpStage st[kAtomWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kAtomWarps + w;
    if (i >= L.n) return;
    NbrSmem &s = sn[w];
    JvpStage &ts = st[w];
    int cnt, nr, na;
    {
        NbrFetch f;
        fetch_neighbours(L, pos4, i, lane, f);
        float3 vj[kKmax / 32];
        const float vix = v[3 * i], viy = v[3 * i + 1], viz = v[3 * i + 2];
#pragma unroll
        for (int k = 0; k < kKmax / 32; ++k)
            if (lane + 32 * k < f.cnt) vj[k] = make_float3(v[3 * f.j[k]], v[3 * f.j[k] + 1], v[3 * f.j[k] + 2]);
        store_neighbours<true>(f, s, lane, cnt, nr, na);
#pragma unroll
        for (int k = 0; k < kKmax / 32; ++k) {
            const int q = lane + 32 * k;
            if (q < cnt) {
                const float4 d = s.d[q];
                const float wx = vj[k].x - vix, wy = vj[k].y - viy, wz = vj[k].z - viz;
                ts.w[q] = make_float4(wx, wy, wz, d.x * wx + d.y * wy + d.z * wz);
            }
        }
        __syncwarp();
    }
    float out[12];
    {   // radial: d/de of sum_j exp(-eta (r - R_k)^2) fc(r) = (-2 eta (r - R_k) fc + fc') exp(.) rdot
        const int h = lane >> 4, k = lane & 15;
        const float Rk = 0.9f + (float)k * (4.3f / 16.f);
        float racc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int u = h; u < nr; u += 2) {
            const int q = s.rad[u];
            const float x = s.d[q].w - Rk;
            const float ex = exp_neg(-kEtaR * x * x);
            const float t = ex * (-2.f * kEtaR * x * s.fc[q].x + s.fc[q].y) * ts.w[q].w;
            const int e = s.el[q];
#pragma unroll
            for (int ee = 0; ee < 4; ++ee)
                if (ee == e) racc[ee] += t;
        }
        float tot[4];
#pragma unroll
        for (int ee = 0; ee < 4; ++ee) tot[ee] = racc[ee] + __shfl_xor_sync(0xffffffffu, racc[ee], 16);
        out[0] = h ? tot[1] : tot[0];
        out[1] = h ? tot[3] : tot[2];
    }
    {   // angular
        const int t4 = lane >> 3, p = lane & 7;
        const float thp = (float)(2 * p + 1) * (kPi / 16.f);
        const float cp = cosf(thp), sp = sinf(thp);
        int ne[4], stt[4], off[10];
#pragma unroll
        for (int e = 0; e < 4; ++e) ne[e] = s.nae[e];
        stt[0] = 0;
        stt[1] = ne[0];
        stt[2] = stt[1] + ne[1];
        stt[3] = stt[2] + ne[2];
        int total = 0;
#pragma unroll
        for (int P = 0; P < 10; ++P) {
            constexpr int e1s[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3}, e2s[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
            const int e1 = e1s[P], e2 = e2s[P];
            const int n = e1 == e2 ? ne[e1] * (ne[e1] - 1) / 2 : ne[e1] * ne[e2];
            if (lane == P) {
                ts.type[P] = make_int4(total, n, stt[e1] | (stt[e2] << 8) | (ne[e2] << 16), e1 == e2 ? 1 : 0);
                ts.rcp[P] = ne[e2] > 0 ? 1.f / (float)ne[e2] : 0.f;
            }
            off[P] = total;
            total += (n + 3) & ~3;
        }
#pragma unroll
        for (int k = 0; k < 10; ++k) ts.acc[k][lane] = 0.f;
        __syncwarp();
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        int curP = -1;
        const bool hi = (t4 & 2) != 0, lo = (t4 & 1) != 0;
        auto flush = [&]() {
            const float a0 = acc[0], a1 = acc[1], a2 = acc[2], a3 = acc[3];
            float k0 = hi ? a2 : a0, k1 = hi ? a3 : a1;
            const float s0 = hi ? a0 : a2, s1 = hi ? a1 : a3;
            k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
            k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
            float mine = lo ? k1 : k0;
            mine += __shfl_xor_sync(0xffffffffu, lo ? k0 : k1, 8);
            ts.acc[curP][lane] += mine;
#pragma unroll
            for (int mm = 0; mm < 4; ++mm) acc[mm] = 0.f;
        };
        for (int base = 0; base < total; base += 32) {
            const int slot = base + lane;
            int P = 0;
#pragma unroll
            for (int k = 1; k < 10; ++k) P += slot >= off[k] ? 1 : 0;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f), qd = q, bq = q, bdq = q;
            if (slot < total) {
                const int4 ty = ts.type[P];
                const int l = slot - ty.x;
                if (l < ty.y) {
                    const int a0 = ty.z & 255, b0 = (ty.z >> 8) & 255, c2 = ty.z >> 16;
                    int a, b;
                    if (ty.w) {
                        triplet_ab(l, c2, a, b);
                        a += a0;
                        b += a0;
                    } else {
                        a = (int)(((float)l + 0.5f) * ts.rcp[P]);
                        b = b0 + (l - a * c2);
                        a += a0;
                    }
                    const int qa = s.ang[a], qb = s.ang[b];
                    const float4 dj = s.d[qa], dk = s.d[qb], wj = ts.w[qa], wk = ts.w[qb];
                    const float rj = dj.w, rk = dk.w;
                    const float ct = dj.x * dk.x + dj.y * dk.y + dj.z * dk.z;
                    const float ctd = ((dk.x - ct * dj.x) * wj.x + (dk.y - ct * dj.y) * wj.y + (dk.z - ct * dj.z) * wj.z) /
                                          rj +
                                      ((dj.x - ct * dk.x) * wk.x + (dj.y - ct * dk.y) * wk.y + (dj.z - ct * dk.z) * wk.z) /
                                          rk;
                    const float cs = kAngScale * ct;
                    const float sn2 = sqrtf(1.f - cs * cs);
                    const float fj = s.fc[qa].z, fk = s.fc[qb].z;
                    q = make_float4(cs, sn2, kTwoPowM31 * fj * fk, 0.f);
                    qd = make_float4(cs / sn2, 32.f * kAngScale * ctd,
                                     kTwoPowM31 * (s.fc[qa].w * fk * wj.w + fj * s.fc[qb].w * wk.w), 0.f);
                    const float ravg = 0.5f * (rj + rk), ravgd = 0.5f * (wj.w + wk.w);
                    float bm[4], bdm[4];
#pragma unroll
                    for (int mm = 0; mm < 4; ++mm) {
                        const float x = ravg - (0.9f + (float)mm * 0.65f);
                        bm[mm] = __expf(-kEtaA * x * x);
                        bdm[mm] = -2.f * kEtaA * x * bm[mm] * ravgd;
                    }
                    bq = make_float4(bm[0], bm[1], bm[2], bm[3]);
                    bdq = make_float4(bdm[0], bdm[1], bdm[2], bdm[3]);
                }
            }
            q.w = __int_as_float(P);   // empty slots of a run carry its type and contribute zero
            ts.q[lane] = q;
            ts.qd[lane] = qd;
            ts.b[lane] = bq;
            ts.bd[lane] = bdq;
            __syncwarp();
            const int ng = min(32, total - base);   // a multiple of 4
            for (int u = 0; u < ng; u += 4) {
                const float4 qq = ts.q[u + t4], dd = ts.qd[u + t4];
                const int Pu = __float_as_int(ts.q[u].w);
                if (Pu != curP) {
                    if (curP >= 0) flush();
                    curP = Pu;
                }
                // A = 2^-31 x^32 and dA/dcos = 2^-31 32 x^31 (cos theta_p - cot sin theta_p), x = 1 + cos(theta - theta_p)
                const float x = 1.f + qq.x * cp + qq.y * sp;
                const float x2 = x * x, x4 = x2 * x2, x8 = x4 * x4, x16 = x8 * x8;
                const float x31 = x16 * x8 * x4 * x2 * x;
                const float A = x31 * x, dA = x31 * (cp - dd.x * sp);
                const float cB = dA * dd.y * qq.z + A * dd.z;   // multiplies B_m
                const float cBd = A * qq.z;                      // multiplies the tangent of B_m
                const float4 bb = ts.b[u + t4], bd = ts.bd[u + t4];
                acc[0] = fmaf(cB, bb.x, fmaf(cBd, bd.x, acc[0]));
                acc[1] = fmaf(cB, bb.y, fmaf(cBd, bd.y, acc[1]));
                acc[2] = fmaf(cB, bb.z, fmaf(cBd, bd.z, acc[2]));
                acc[3] = fmaf(cB, bb.w, fmaf(cBd, bd.w, acc[3]));
            }
            __syncwarp();
        }
        if (curP >= 0) flush();
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 10; ++k) out[2 + k] = ts.acc[k][lane];
    }
    float *row = U + (size_t)L.row_of[i] * kNFeat;
#pragma unroll
    for (int k = 0; k < kNFeat / 32; ++k) row[32 * k + lane] = out[k];
}

__global__ void k_learn_begin(LearnedDev L) {
    if (threadIdx.x == 0) L.lflags[1] = 0u;
}

// After a learned force evaluation: count a step that left the feature range
// (its forces came from the plain force field), or report it when the
// fallback is off.
__global__ void k_learn_end(LearnedDev L, uint32_t *status, int fallback) {
    if (threadIdx.x != 0 || L.lflags[1] == 0u) return;
    L.lcount[1] += 1;
    L.lflags[1] = 0u;   // ready for the next evaluation
    if (!fallback) atomicOr(status, MDPF_STATUS_OUT_OF_RANGE);
}

__global__ void k_fallback_clear(LearnedDev L, unsigned long long *fx, unsigned long long *efx) {
    if (L.lflags[1] == 0u) return;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < 3 * L.n) fx[q] = 0ull;
    if (q == 0 && efx != nullptr) efx[E_LEARN] = 0ull;
}

__global__ void k_import_g(LearnedDev L, const float *G) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= L.n * kNFeat) return;
    const int a = q / kNFeat, f = q % kNFeat;
    L.G16[(size_t)L.row_of[a] * kNFeat + f] = __float2bfloat16_rn(G[q]);
}

}  // namespace

// ------------------------------------------------------------------ launchers

void learned_begin(const LearnedDev &L, cudaStream_t s) { k_learn_begin<<<1, 32, 0, s>>>(L); }

void learned_fallback_clear(const LearnedDev &L, unsigned long long *fx, unsigned long long *efx, cudaStream_t s) {
    k_fallback_clear<<<(3 * L.n + 255) / 256 + 1, 256, 0, s>>>(L, fx, efx);
}

void learned_end(const LearnedDev &L, uint32_t *status, int fallback, cudaStream_t s) {
    k_learn_end<<<1, 32, 0, s>>>(L, status, fallback);
}

void learned_jvp(const LearnedDev &L, const float4 *pos4, const float *v, float *U, cudaStream_t s) {
    k_jvp<<<(L.n + kAtomWarps - 1) / kAtomWarps, 32 * kAtomWarps, 0, s>>>(L, pos4, v, U);
}

void learned_import_g(const LearnedDev &L, const float *G_atoms, cudaStream_t s) {
    k_import_g<<<(L.n * kNFeat + 255) / 256, 256, 0, s>>>(L, G_atoms);
}

int learned_nb_grid() {
    int dev = 0, sms = 0, occ = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_nb_all, kNbThreads, 0) != cudaSuccess || occ < 1)
        return 0;
    return sms * (occ < 4 ? occ : 4);
}

cudaError_t learned_neighbors(const LearnedDev &L, const float4 *pos4, bool forced, uint32_t *status,
                              cudaStream_t s) {
    int f = forced ? 1 : 0;
    if (L.n <= kNbSmallMax) {
        k_nb_small<<<(L.n + kNbThreads / 32 - 1) / (kNbThreads / 32), kNbThreads, 0, s>>>(L, pos4, status, f);
        return cudaGetLastError();
    }
    long long limit = 1000000000LL;   // 1 s per barrier wait
    const int want = (L.n + kNbThreads / 32 - 1) / (kNbThreads / 32);   // one warp per atom in the row phase
    const int grid = want < L.nb_grid ? want : L.nb_grid;
    LearnedDev Lc = L;
    const float4 *p = pos4;
    void *args[] = {&Lc, &p, &status, &f, &limit};
    return cudaLaunchCooperativeKernel((const void *)k_nb_all, dim3(grid > 0 ? grid : 1), dim3(kNbThreads), args, 0,
                                       s);
}

void learned_features(const LearnedDev &L, const float4 *pos4, bool write_f32, cudaStream_t s) {
    k_features<<<(L.n + kFeatWarps - 1) / kFeatWarps, 32 * kFeatWarps, 0, s>>>(L, pos4, write_f32 ? 1 : 0);
}

void learned_mlp(const LearnedDev &L, bool gated, bool fp32, unsigned long long *efx, cudaStream_t s) {
    if (L.n_rows <= 0) return;
    if (fp32) k_mlp_simt<false><<<L.n_rows / kMlpRows, 256, 0, s>>>(L, gated ? 1 : 0, efx);
    else k_mlp_simt<true><<<L.n_rows / kMlpRows, 256, 0, s>>>(L, gated ? 1 : 0, efx);
}

void learned_adjoint(const LearnedDev &L, const float4 *pos4, unsigned long long *fx, bool gated,
                     unsigned long long *ecore, int ecore_per, cudaStream_t s) {
    k_adjoint<<<(L.n + kAtomWarps - 1) / kAtomWarps, 32 * kAtomWarps, 0, s>>>(L, pos4, fx, gated ? 1 : 0, ecore,
                                                                               ecore_per > 0 ? ecore_per : 1);
}

}  // namespace mdpf
