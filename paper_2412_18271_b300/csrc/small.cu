// Persistent velocity-Verlet stepper of the learned potential for molecules
// of up to 32 atoms (the paper's per-step-overhead case: a 9-atom molecule,
// where launch latency and serial stage chains, not arithmetic, decide the
// step time).
//
// One cooperative launch of kSB blocks runs all n steps.  Each block keeps a
// slice of the network's weights in shared memory for the whole launch, so no
// weight is read from memory inside the step loop:
//   block b: W1 rows (hidden units) 32 b .. 32 b + 31 and the W2 columns of the
//   same units (all 128 rows), of every element, BF16, as the tensor-core
//   kernels use them.
// So a block's layer-1 activations are exactly the inputs of its W2 columns:
// layer 2 leaves the block as partial sums of z2, and layer 2' (W2^T delta2
// for the block's own units) needs no exchange.
// An MD step (positions x_{s+1} identical in every block):
//   features   block b, two warps per atom a = b + 8 p (warps p and p + 4):
//              warp p lists the neighbours by brute force over the molecule
//              (ascending index, as the neighbour list orders them) into
//              shared memory for both; then warp p computes the radial and
//              warp p + 4 the angular columns of learned_terms.cuh (the same
//              bits as one warp doing both), with their range checks; the
//              FP32 rows to the exchange buffer.                     barrier 0
//   layer 1    every block: all rows as BF16; z1 = W1 G + b1 for its 32 units
//              (warp MMA m16n8k16, K = 384, FP32 accumulation); a1 =
//              CELU(z1) kept as the BF16 pair hi + lo, CELU'(z1) kept;
//              the partial W2 a1 over its 32 units for all 128 units of
//              layer 2 (warp MMA, K = 32, hi and lo products apart).  barrier 1
//   layer 2    every block: z2 = b2 + the partials summed in block order for
//              all 128 units; delta2 = w3 CELU'(z2) (BF16); block 0 keeps
//              the energy terms w3 CELU(z2).  Layer 2': delta1 = CELU'(z1)
//              W2^T delta2 for its 32 units (warp MMA, K = 128; BF16).
//              Layer 1': the partial dE/dG = W1^T delta1 over its units for
//              all 384 features (warp MMA, K = 32).                  barrier 2
//   adjoint    block b, the same two warps per atom: dE/dG (sum of the
//              partials in block order; each warp its own columns), the chain
//              rule of learned_terms.cuh into fixed-point forces, warp p the
//              radial pairs (and the repulsive core), warp p + 4 the triplets,
//              each adding its own fixed-point sums.                 barrier 3
//   integration every block, the same FP64 arithmetic on the same sums (so
//              every block holds the same state): v += dt/2 a; (energy and
//              frames by block 0); v += dt/2 a; x += dt v.
// A step whose features left the model's training range runs the plain force
// field instead (block 0, all pairs and bonded terms of the molecule) and is
// counted, as on the per-stage path; with the fallback off the step reports
// MDPF_STATUS_OUT_OF_RANGE.
//
// Numerics follow the tensor-core MLP's rounding points: BF16 features, the
// BF16 pair hi + lo of a1, BF16 delta2 and delta1, BF16 weights, FP32
// accumulation (z2's sum over units taken per block, then over blocks).
// Every sum is taken in a fixed order or in integers, so runs repeat bit for
// bit; the forces differ from the stage kernels' only in rounding each atom's
// radial and angular parts to fixed point apart.  Every wait is a bounded grid
// barrier (1 s, MDPF_STATUS_TIMEOUT); the warp pairs' named barriers wait for
// a partner that runs the same code path.
#include "forcefield.cuh"
#include "grid_sync.cuh"
#include "learned_terms.cuh"
#include "tc_util.cuh"

namespace mdpf {
namespace {

constexpr int kSB = 8;                 // blocks
constexpr int kSThreads = 256;         // threads per block (8 warps)
constexpr int kSmallMax = 32;          // atoms
constexpr int kU1 = kH1 / kSB;         // 32 hidden units of layer 1 per block
constexpr int kW1Stride = kNFeat + 8;  // BF16 row strides padded by 16 bytes (conflict-free ldmatrix rows)
constexpr int kU1Stride = kU1 + 8;     // rows over the block's 32 units (W2 columns, a1, delta1)
constexpr int kD2Stride = kH2 + 8;
constexpr int kAdjChunkS = 128;  // triplets staged per adjoint pass of the angular warps (no effect on the result)

struct SmallArgs {
    LearnedDev L;
    PlainDev p;
    int n, fallback;
    double dt;
    const double *hdt_m, *mass;
    const float *qs;                   // q sqrt(ke) per atom (the plain fallback's Coulomb term)
    double *x, *v;
    unsigned long long *fxs;           // state forces F(x) (fixed point) on entry and on exit
    // exchange buffers (global)
    float *xG;                         // [32][384] features
    float *xZ2;                        // [kSB][32][128] partial W2 a1
    float *xPG;                        // [kSB][32][384] partial dE/dG
    unsigned long long *fac;           // [2][32][3] forces of a step (fixed point), by step parity
    unsigned long long *eacc;          // [2][4] energies of a step (fixed point): core, bond, angle, LJ + Coulomb
    unsigned int *flag;                // [2] range flag of a step
    const int *el_list;                // [4][32] atoms of each element, ascending
    const int *el_cnt;                 // [4]
    // traces and frames
    double *trace_u, *trace_k;
    int64_t *trace_step, *trace_fb;
    int trace_cap, energy_every;
    int64_t *step;
    uint32_t *status;
    double *scalars;
    Frames frames;
    int record_every;
    unsigned long long *bar;
    int64_t n_steps;
    long long limit_ns;
};

// Shared memory of a block.  The phases use disjoint parts of one union.
struct SmallSmem {
    __nv_bfloat16 w1[4][kU1][kW1Stride];     // W1 rows of the block's units
    __nv_bfloat16 w2[4][kH2][kU1Stride];     // W2 columns of the block's units (all 128 rows)
    float b1[4][kU1], b2[4][kH2], w3[4][kH2];
    union {
        struct {
            NbrSmem nb[4];        // atom b + 8 p's neighbours, shared by warps p and p + 4
            TripStage ts[4];      // the angular warp's staging
        } feat;
        __nv_bfloat16 g[kSmallMax][kW1Stride];                 // features, BF16
        struct {
            NbrSmem nb[4];                  // as in feat
            AdjScratch<32> asr[4];          // the radial warps' (they stage no triplets)
            AdjScratch<kAdjChunkS> asa[4];  // the angular warps'
            alignas(16) float sg[4][kGRow]; // dE/dG of atom b + 8 p: radial columns by warp p, angular by p + 4
        } adj;
    } u;
    __nv_bfloat16 a1hi[kSmallMax][kU1Stride], a1lo[kSmallMax][kU1Stride];   // CELU(z1) of the block's units, hi + lo
    float dc1[kSmallMax][kU1];               // CELU'(z1) of the block's units
    union {
        __nv_bfloat16 d2[kSmallMax][kD2Stride];   // delta2, all 128 units
        float zp[2][kSmallMax][kU1];               // layer 1: z1 over each half of K
    };
    __nv_bfloat16 d1[kSmallMax][kU1Stride];  // delta1 of the block's units
    float eat[kSmallMax];                    // block 0: w3 . CELU(z2) per atom
    double x[kSmallMax][3], vel[kSmallMax][3], h[kSmallMax], km[kSmallMax];
    float4 pos[kSmallMax];
    int el[kSmallMax];
    int el_list[4][kSmallMax], el_cnt[4];
    double red[8];
    int nbc[4][3];                           // neighbour row length, radial and angular counts of atom b + 8 p
    unsigned int pending;                    // status bits found after barrier 3, raised after the next barrier 0
    int s_fail;
};

static_assert(sizeof(SmallSmem) <= 227 * 1024, "a block's shared memory");

// ---- warp-level MMA (m16n8k16, BF16 in, FP32 accumulate) from shared memory
__device__ __forceinline__ void ldsm_x4(const void *p, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(const void *p, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2(const void *p, uint32_t (&r)[2]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment of rows m0..m0+15, columns k0..k0+15 of a row-major matrix (row stride `ld` elements).
__device__ __forceinline__ void frag_a(const __nv_bfloat16 *base, int ld, int m0, int k0, int lane, uint32_t (&a)[4]) {
    const int mi = lane >> 3, r = lane & 7;
    ldsm_x4(base + (size_t)(m0 + (mi & 1) * 8 + r) * ld + k0 + (mi >> 1) * 8, a);
}
// A fragment of the transpose: A(m, k) = S(k, m), S row-major (row stride `ld`); rows m0.., columns k0.. of A.
__device__ __forceinline__ void frag_at(const __nv_bfloat16 *S, int ld, int m0, int k0, int lane, uint32_t (&a)[4]) {
    const int mi = lane >> 3, r = lane & 7;
    ldsm_x4_t(S + (size_t)(k0 + (mi >> 1) * 8 + r) * ld + m0 + (mi & 1) * 8, a);
}
// B fragment (16 x 8, k x n) from n rows of a row-major [n][k] matrix: row pointers per n (lane & 7).
__device__ __forceinline__ void frag_b(const __nv_bfloat16 *row, int k0, int lane, uint32_t (&b)[2]) {
    ldsm_x2(row + k0 + ((lane >> 3) & 1) * 8, b);
}

// Atom `at`'s candidate neighbours: every other atom, ascending (the order of a neighbour-list row).
__device__ __forceinline__ void small_fetch(const SmallSmem &S, int n, int at, int lane, NbrFetch &f) {
    f.pi = S.pos[at];
    f.cnt = n - 1;
#pragma unroll
    for (int k = 0; k < kKmax / 32; ++k) {
        const int idx = lane + 32 * k;
        f.j[k] = 0;
        if (idx < n - 1) {
            const int j = idx < at ? idx : idx + 1;
            f.j[k] = j;
            f.pj[k] = S.pos[j];
            f.ej[k] = S.el[j];
        }
    }
}

// The B-operand row of atom slot `idx` of element e (slots past the element's count read atom 0's row;
// their output columns are discarded).
__device__ __forceinline__ int slot_atom(const SmallSmem &S, int e, int idx) {
    return idx < S.el_cnt[e] ? S.el_list[e][idx] : S.el_list[e][0];
}

// The two output columns of an MMA fragment lane (atom slots 8 nt + 2 t4 and the next): their atoms and
// whether they are real.  Read once, before any store, so that the stores of an epilogue (through pointers
// the compiler cannot tell from shared memory) do not force these shared reads to repeat after each.
struct EpiRows {
    int at[2];
    bool ok[2];
};
__device__ __forceinline__ EpiRows epi_rows(const SmallSmem &S, int e, int nt, int t4) {
    const int i0 = 8 * nt + 2 * t4, c = S.el_cnt[e];
    EpiRows r;
    r.at[0] = S.el_list[e][i0];       // i0 + 1 <= 31: within the element's list (unused slots hold 0)
    r.at[1] = S.el_list[e][i0 + 1];
    r.ok[0] = i0 < c;
    r.ok[1] = i0 + 1 < c;
    return r;
}

// Tasks (element e, n-tile of 8 atoms, m-tile) of one GEMM phase, enumerated in a fixed order: element,
// then n-tile, then m-tile.  Returns false past the last task.
__device__ __forceinline__ bool task_of(const SmallSmem &S, int id, int mtiles, int &e, int &nt, int &mt) {
    for (e = 0; e < 4; ++e) {
        const int nte = (S.el_cnt[e] + 7) >> 3;
        if (id < nte * mtiles) {
            nt = id / mtiles;
            mt = id - nt * mtiles;
            return true;
        }
        id -= nte * mtiles;
    }
    return false;
}

// Warps p and p + 4 of a block share atom b + 8 p in the feature and adjoint phases: warp p lists the
// neighbours into shared memory and both wait here (named barrier 1 + p, 64 threads) before reading them.
__device__ __forceinline__ void pair_sync(int p) { asm volatile("bar.sync %0, 64;" ::"r"(1 + p) : "memory"); }

// The neighbours of atom `at` into S.u.<phase>.nb[p] by warp p (ang false); the counts in every lane of both
// warps after the pair barrier.
template <bool ByElement>
__device__ __forceinline__ void pair_neighbours(SmallSmem &S, NbrSmem &nb, int n, int at, int p, bool ang, int lane,
                                                int &cnt, int &nr, int &na) {
    if (!ang) {
        NbrFetch f;
        small_fetch(S, n, at, lane, f);
        store_neighbours<ByElement>(f, nb, lane, cnt, nr, na);
        if (lane == 0) {
            S.nbc[p][0] = cnt;
            S.nbc[p][1] = nr;
            S.nbc[p][2] = na;
        }
    }
    pair_sync(p);
    cnt = S.nbc[p][0];
    nr = S.nbc[p][1];
    na = S.nbc[p][2];
}

__global__ void __launch_bounds__(kSThreads, 1) k_learned_small(SmallArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmallSmem &S = *reinterpret_cast<SmallSmem *>(smem_raw);
    const LearnedDev &L = a.L;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5, b = blockIdx.x;
    const int n = a.n;
    const int g4 = lane >> 2, t4 = lane & 3;   // MMA fragment coordinates
    const int64_t step0 = *a.step;
    unsigned long long epoch = 0;

    // ---- the block's weight slices, in 16-byte pieces
    for (int q = t; q < 4 * kU1 * (kNFeat / 8); q += kSThreads) {
        const int e = q / (kU1 * (kNFeat / 8)), r = q % (kU1 * (kNFeat / 8)), u = r / (kNFeat / 8), c = r % (kNFeat / 8);
        *reinterpret_cast<uint4 *>(&S.w1[e][u][8 * c]) =
            *reinterpret_cast<const uint4 *>(L.W1 + ((size_t)e * kH1 + kU1 * b + u) * kNFeat + 8 * c);
    }
    for (int q = t; q < 4 * kH2 * (kU1 / 8); q += kSThreads) {
        const int e = q / (kH2 * (kU1 / 8)), r = q % (kH2 * (kU1 / 8)), v = r / (kU1 / 8), c = r % (kU1 / 8);
        *reinterpret_cast<uint4 *>(&S.w2[e][v][8 * c]) =
            *reinterpret_cast<const uint4 *>(L.W2 + ((size_t)e * kH2 + v) * kH1 + kU1 * b + 8 * c);
    }
    for (int q = t; q < 4 * kU1; q += kSThreads) S.b1[q / kU1][q % kU1] = L.b1[(q / kU1) * kH1 + kU1 * b + q % kU1];
    for (int q = t; q < 4 * kH2; q += kSThreads) {
        S.b2[q / kH2][q % kH2] = L.b2[q];
        S.w3[q / kH2][q % kH2] = L.W3[q];
    }
    for (int q = t; q < 4 * kSmallMax; q += kSThreads) S.el_list[q / kSmallMax][q % kSmallMax] = a.el_list[q];
    if (t < 4) S.el_cnt[t] = a.el_cnt[t];
    if (t < n) S.el[t] = L.el[t];
    if (t == 0) S.pending = 0u;
    // ---- pre-phase (every block the same): v_{1/2} = v_0 + dt/2 a(x_0); x_1 = x_0 + dt v_{1/2}
    for (int q = t; q < 3 * n; q += kSThreads) {
        const int at = q / 3, c = q - 3 * at;
        const double h = a.hdt_m[at];
        const double v = fma(h, fx_val(a.fxs[q]), a.v[q]);
        const double x = fma(a.dt, v, a.x[q]);
        S.vel[at][c] = v;
        S.x[at][c] = x;
        reinterpret_cast<float *>(&S.pos[at])[c] = (float)x;
        if (c == 0) {
            S.h[at] = h * kFxInv;
            S.km[at] = 0.5 * a.mass[at] / kAcc;
            S.pos[at].w = a.qs[at];
        }
    }
    __syncthreads();

    for (int64_t s = 0; s < a.n_steps; ++s) {
        const int par = (int)(s & 1);
        const int64_t done = step0 + s + 1;
        const bool energy = done % a.energy_every == 0;
        const bool rec = a.record_every > 0 && done % a.record_every == 0;
        const int slot = rec ? (int)((done / a.record_every - 1) % a.frames.cap) : 0;
        const bool last = s + 1 == a.n_steps;
        unsigned long long *fac = a.fac + par * 3 * kSmallMax;
        unsigned long long *eacc = a.eacc + par * 4;
        bool bad = false;
        // ---- features of atoms b + 8 (w mod 4): warp w < 4 the radial columns, warp w + 4 the angular ones
        {
            const int pr = w & 3, at = b + kSB * pr;
            const bool ang = w >= 4;
            if (at < n) {
                int cnt, nr, na;
                pair_neighbours<true>(S, S.u.feat.nb[pr], n, at, pr, ang, lane, cnt, nr, na);
                float v[12];
                if (ang) feature_row<2>(S.u.feat.nb[pr], nr, na, S.u.feat.ts[pr], lane, v);
                else feature_row<1>(S.u.feat.nb[pr], nr, na, S.u.feat.ts[pr], lane, v);
                const int k0 = ang ? 2 : 0, k1 = ang ? 12 : 2;
                const int z = S.el[at];
                bool out = false;
                if (L.lo != nullptr) {   // every range load issued before the first store
#pragma unroll
                    for (int k = 0; k < 12; ++k) {
                        const int fi = 32 * k + lane;
                        if (k >= k0 && k < k1)
                            out |= (v[k] < L.lo[z * kNFeat + fi]) || (v[k] > L.hi[z * kNFeat + fi]);
                    }
                }
#pragma unroll
                for (int k = 0; k < 12; ++k)
                    if (k >= k0 && k < k1) a.xG[at * kNFeat + 32 * k + lane] = v[k];
                if (__any_sync(0xffffffffu, out) && lane == 0) {
                    atomicOr(&a.flag[par], 1u);
                    if (!a.fallback) atomicOr(a.status, MDPF_STATUS_OUT_OF_RANGE);
                }
            }
        }
        if (!grid_barrier(a.bar, ++epoch, a.status, a.limit_ns, &S.s_fail)) return;   // B0
        const bool out = *(volatile unsigned int *)&a.flag[par] != 0u;
        const bool plain = out && a.fallback;
        // Status bits are raised only before barrier 3 (here, or by the feature warps), so every block reads
        // the same status after it and all stop together.
        if (t == 0 && S.pending != 0u) {
            atomicOr(a.status, S.pending);
            S.pending = 0u;
        }
        if (b == 0) {   // the buffers of the next step (last read before this step's barrier 0)
            if (t == 0) a.flag[par ^ 1] = 0u;
            if (t < 3 * kSmallMax) a.fac[(par ^ 1) * 3 * kSmallMax + t] = 0ull;
            if (t < 4) a.eacc[(par ^ 1) * 4 + t] = 0ull;
            if (t == 0 && out) L.lcount[1] += 1;   // counted with the fallback on or off, as on the per-stage path
        }
        if (!plain) {
            // ---- layer 1: z1 = W1 G + b1 for the block's 32 units
            for (int q = t; q < n * (kNFeat / 4); q += kSThreads) {
                const int at = q / (kNFeat / 4), c = 4 * (q % (kNFeat / 4));
                const float4 gv = __ldcg(reinterpret_cast<const float4 *>(&a.xG[at * kNFeat + c]));
                *reinterpret_cast<uint2 *>(&S.u.g[at][c]) = make_uint2(pack_bf16(gv.x, gv.y), pack_bf16(gv.z, gv.w));
            }
            __syncthreads();
            // a task: (element, n-tile, half of K), both m-tiles of the block's 32 units, four chains in flight
            int e, nt, mt;
            for (int id = w; task_of(S, id, 2, e, nt, mt); id += 8) {
                float acc[2][2][4] = {};   // [m-tile][k parity]
                const __nv_bfloat16 *brow = &S.u.g[slot_atom(S, e, 8 * nt + (lane & 7))][0];
                const int k0 = mt * (kNFeat / 32);   // mt is the K half here
#pragma unroll 2
                for (int k2 = 0; k2 < kNFeat / 32; k2 += 2) {
#pragma unroll
                    for (int par = 0; par < 2; ++par) {
                        const int kk = k0 + k2 + par;
                        uint32_t A0[4], A1[4], B[2];
                        frag_b(brow, 16 * kk, lane, B);
                        frag_a(&S.w1[e][0][0], kW1Stride, 0, 16 * kk, lane, A0);
                        frag_a(&S.w1[e][0][0], kW1Stride, 16, 16 * kk, lane, A1);
                        mma16816(acc[0][par], A0, B);
                        mma16816(acc[1][par], A1, B);
                    }
                }
                const EpiRows er = epi_rows(S, e, nt, t4);
#pragma unroll
                for (int h = 0; h < 8; ++h) {
                    const int m = h >> 2, hh = h & 3;
                    const int ul = 16 * m + g4 + 8 * (hh >> 1);
                    if (er.ok[hh & 1]) S.zp[mt][er.at[hh & 1]][ul] = acc[m][0][hh] + acc[m][1][hh];
                }
            }
            __syncthreads();
            for (int q = t; q < n * kU1; q += kSThreads) {
                const int at = q / kU1, ul = q % kU1;
                const float z = (S.zp[0][at][ul] + S.zp[1][at][ul]) + S.b1[S.el[at]][ul];
                const float av = celu_e(z, exp10x_neg(z));
                const __nv_bfloat16 hi = __float2bfloat16_rn(av);
                S.a1hi[at][ul] = hi;
                S.a1lo[at][ul] = __float2bfloat16_rn(av - __bfloat162float(hi));
                S.dc1[at][ul] = dcelu_from_a(av);
            }
            __syncthreads();
            // partial z2 = W2 (hi + lo) over the block's 32 units, for all 128 units of layer 2; a task is
            // (element, n-tile, group of 4 m-tiles), its B fragments shared
            for (int id = w; task_of(S, id, kH2 / 64, e, nt, mt); id += 8) {
                const int ra = slot_atom(S, e, 8 * nt + (lane & 7));
                uint32_t Bh[2][2], Bl[2][2];
#pragma unroll
                for (int kk = 0; kk < kU1 / 16; ++kk) {
                    frag_b(&S.a1hi[ra][0], 16 * kk, lane, Bh[kk]);
                    frag_b(&S.a1lo[ra][0], 16 * kk, lane, Bl[kk]);
                }
                float acc[4][2][4] = {};   // [m-tile][hi, lo]: the hi and lo products apart
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int kk = 0; kk < kU1 / 16; ++kk) {
                        uint32_t A[4];
                        frag_a(&S.w2[e][0][0], kU1Stride, 16 * (4 * mt + j), 16 * kk, lane, A);
                        mma16816(acc[j][0], A, Bh[kk]);
                        mma16816(acc[j][1], A, Bl[kk]);
                    }
                const EpiRows er = epi_rows(S, e, nt, t4);
                float *zr[2] = {a.xZ2 + ((size_t)b * kSmallMax + er.at[0]) * kH2, a.xZ2 + ((size_t)b * kSmallMax + er.at[1]) * kH2};
#pragma unroll
                for (int h = 0; h < 16; ++h) {
                    const int j = h >> 2, hh = h & 3;
                    const int v = 16 * (4 * mt + j) + g4 + 8 * (hh >> 1);
                    if (er.ok[hh & 1]) zr[hh & 1][v] = acc[j][0][hh] + acc[j][1][hh];
                }
            }
            if (!grid_barrier(a.bar, ++epoch, a.status, a.limit_ns, &S.s_fail)) return;   // B1
            // ---- layer 2: z2 = b2 + the partials in block order, all 128 units (warp: one atom, lane: 4 units)
            for (int q = t; q < n * (kH2 / 4); q += kSThreads) {
                const int at = q / (kH2 / 4), v4 = 4 * (q % (kH2 / 4)), z = S.el[at];
                float4 zs = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int bb = 0; bb < kSB; ++bb) {
                    const float4 pv = __ldcg(reinterpret_cast<const float4 *>(&a.xZ2[((size_t)bb * kSmallMax + at) * kH2 + v4]));
                    zs.x += pv.x;
                    zs.y += pv.y;
                    zs.z += pv.z;
                    zs.w += pv.w;
                }
                const float zv[4] = {zs.x, zs.y, zs.z, zs.w};
                float ev = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float z2 = S.b2[z][v4 + k] + zv[k], ex = exp10x_neg(z2);
                    ev += S.w3[z][v4 + k] * celu_e(z2, ex);
                    S.d2[at][v4 + k] = __float2bfloat16_rn(S.w3[z][v4 + k] * dcelu_e(z2, ex));
                }
                ev = warp_sum_f(ev);   // the 32 lanes of this atom, a fixed butterfly
                if (b == 0 && lane == 0) S.eat[at] = ev;
            }
            __syncthreads();
            // ---- layer 2': delta1 = CELU'(z1) W2^T delta2 for the block's 32 units (K = 128, BF16)
            for (int id = w; task_of(S, id, kU1 / 16, e, nt, mt); id += 8) {
                float acc2[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};   // two K halves in flight
                const __nv_bfloat16 *brow = &S.d2[slot_atom(S, e, 8 * nt + (lane & 7))][0];
#pragma unroll
                for (int kk = 0; kk < kH2 / 16; ++kk) {
                    uint32_t A[4], B[2];
                    frag_at(&S.w2[e][0][0], kU1Stride, 16 * mt, 16 * kk, lane, A);
                    frag_b(brow, 16 * kk, lane, B);
                    mma16816(acc2[kk & 1], A, B);
                }
                const EpiRows er = epi_rows(S, e, nt, t4);
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int ul = 16 * mt + g4 + 8 * (h >> 1), at = er.at[h & 1];
                    if (er.ok[h & 1]) S.d1[at][ul] = __float2bfloat16_rn((acc2[0][h] + acc2[1][h]) * S.dc1[at][ul]);
                }
            }
            __syncthreads();
            // ---- layer 1': partial dE/dG = W1^T delta1 over the block's 32 units for all 384 features (warp MMA,
            // K = 32); a task is (element, n-tile, group of 6 m-tiles), its B fragments shared
            for (int id = w; task_of(S, id, kNFeat / 96, e, nt, mt); id += 8) {
                const __nv_bfloat16 *brow = &S.d1[slot_atom(S, e, 8 * nt + (lane & 7))][0];
                uint32_t B[2][2];
#pragma unroll
                for (int kk = 0; kk < kU1 / 16; ++kk) frag_b(brow, 16 * kk, lane, B[kk]);
                float acc[6][4] = {};
#pragma unroll
                for (int j = 0; j < 6; ++j)
#pragma unroll
                    for (int kk = 0; kk < kU1 / 16; ++kk) {
                        uint32_t A[4];
                        frag_at(&S.w1[e][0][0], kW1Stride, 16 * (6 * mt + j), 16 * kk, lane, A);
                        mma16816(acc[j], A, B[kk]);
                    }
                const EpiRows er = epi_rows(S, e, nt, t4);
                float *gr[2] = {a.xPG + ((size_t)b * kSmallMax + er.at[0]) * kNFeat,
                                a.xPG + ((size_t)b * kSmallMax + er.at[1]) * kNFeat};
#pragma unroll
                for (int h = 0; h < 24; ++h) {
                    const int j = h >> 2, hh = h & 3;
                    const int f = 16 * (6 * mt + j) + g4 + 8 * (hh >> 1);
                    if (er.ok[hh & 1]) gr[hh & 1][f] = acc[j][hh];
                }
            }
            if (!grid_barrier(a.bar, ++epoch, a.status, a.limit_ns, &S.s_fail)) return;   // B2
            // ---- adjoint of atoms b + 8 (w mod 4), warp w < 4 its radial pairs, warp w + 4 its triplets: dE/dG
            // (the warp's columns) summed in block order, rounded to BF16 as on the per-stage path
            {
                const int pr = w & 3, at = b + kSB * pr;
                const bool ang = w >= 4;
                if (at < n) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const int f4 = 128 * k + 4 * lane;
                        if ((f4 >= 64) != ang) continue;
                        float4 gs = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                        for (int bb = 0; bb < kSB; ++bb) {
                            const float4 v = __ldcg(reinterpret_cast<const float4 *>(
                                &a.xPG[((size_t)bb * kSmallMax + at) * kNFeat + f4]));
                            gs.x += v.x;
                            gs.y += v.y;
                            gs.z += v.z;
                            gs.w += v.w;
                        }
                        S.u.adj.sg[pr][g_col(f4 + 0)] = __bfloat162float(__float2bfloat16_rn(gs.x));
                        S.u.adj.sg[pr][g_col(f4 + 1)] = __bfloat162float(__float2bfloat16_rn(gs.y));
                        S.u.adj.sg[pr][g_col(f4 + 2)] = __bfloat162float(__float2bfloat16_rn(gs.z));
                        S.u.adj.sg[pr][g_col(f4 + 3)] = __bfloat162float(__float2bfloat16_rn(gs.w));
                    }
                    int cnt, nr, na;
                    pair_neighbours<false>(S, S.u.adj.nb[pr], n, at, pr, ang, lane, cnt, nr, na);
                    if (ang)
                        adjoint_atom<kAdjChunkS, 2>(at, S.u.adj.nb[pr], cnt, nr, na, S.u.adj.sg[pr], S.u.adj.asa[pr],
                                                    fac, lane);
                    else
                        adjoint_atom<32, 1>(at, S.u.adj.nb[pr], cnt, nr, na, S.u.adj.sg[pr], S.u.adj.asr[pr], fac, lane,
                                            make_float2(L.core_a, L.core_rc),
                                                    L.core_rc > 0.f ? &eacc[0] : nullptr);
                }
            }
        } else if (b == 0) {
            // ---- the plain force field for this step: all pairs (i < j) and every bonded term
            const PlainDev &p = a.p;
            float elj = 0.f, ec = 0.f, eb = 0.f, ea = 0.f;
            for (int q = t; q < n * (n - 1) / 2; q += kSThreads) {
                int i = 0, r = q;
                while (r >= n - 1 - i) {
                    r -= n - 1 - i;
                    ++i;
                }
                const int j = i + 1 + r;
                const uint32_t m = p.row_mask[((size_t)(i / 16) * p.n_chunks + j / 32) * 16 + (i % 16)];
                float dx, dy, dz;
                const float fs = pair_fs<true, true>(S.pos[i], p.lj[i], S.pos[j], p.lj[j], (m >> (j % 32)) & 1u, dx, dy,
                                                     dz, elj, ec);
                fx_add(&fac[3 * i + 0], -fs * dx);
                fx_add(&fac[3 * i + 1], -fs * dy);
                fx_add(&fac[3 * i + 2], -fs * dz);
                fx_add(&fac[3 * j + 0], fs * dx);
                fx_add(&fac[3 * j + 1], fs * dy);
                fx_add(&fac[3 * j + 2], fs * dz);
            }
            for (int q = t; q < p.n_bonds + p.n_angles; q += kSThreads) {
                const int4 r = bonded_rec(p, q);
                BondedGeom g;
                g.xa = S.pos[r.x];
                g.xb = S.pos[r.y];
                g.xc = r.z >= 0 ? S.pos[r.z] : make_float4(0.f, 0.f, 0.f, 0.f);
                g.par = r.z < 0 ? p.bond_par[r.w] : make_float2(0.f, 0.f);
                float3 fa, fb, fc;
                float e;
                bonded_forces(p, r, g, fa, fb, fc, e);
                if (r.z < 0) eb += e;
                else ea += e;
                fx_add(&fac[3 * r.x + 0], fa.x);
                fx_add(&fac[3 * r.x + 1], fa.y);
                fx_add(&fac[3 * r.x + 2], fa.z);
                fx_add(&fac[3 * r.y + 0], fb.x);
                fx_add(&fac[3 * r.y + 1], fb.y);
                fx_add(&fac[3 * r.y + 2], fb.z);
                if (r.z >= 0) {
                    fx_add(&fac[3 * r.z + 0], fc.x);
                    fx_add(&fac[3 * r.z + 1], fc.y);
                    fx_add(&fac[3 * r.z + 2], fc.z);
                }
            }
            // energies: bond, angle, LJ + Coulomb (pairs counted once) into the step's fixed-point slots
            const long long i1 = warp_sum_ll(fx_from_float(eb)), i2 = warp_sum_ll(fx_from_float(ea));
            const long long i3 = warp_sum_ll(fx_from_double((double)elj * (1.0 / 6.0) + (double)ec));
            if (lane == 0) {
                if (i1) atomicAdd(&eacc[1], (unsigned long long)i1);
                if (i2) atomicAdd(&eacc[2], (unsigned long long)i2);
                if (i3) atomicAdd(&eacc[3], (unsigned long long)i3);
            }
        }
        if (!grid_barrier(a.bar, ++epoch, a.status, a.limit_ns, &S.s_fail)) return;   // B3
        // every block reads the status after the same barrier, so all stop together
        const bool stop = energy && *(volatile uint32_t *)a.status != 0u;
        // ---- integration (every block, the same arithmetic on the same integers)
        double kin = 0.0;
        if (t < 3 * n) {
            const int at = t / 3, c = t - 3 * at;
            const long long F = (long long)__ldcg(&fac[t]);
            const double Fd = fx_exact(F);
            double v = fma(S.h[at], Fd, S.vel[at][c]);   // v_{s+1}
            double x = S.x[at][c];
            if (energy) kin = S.km[at] * (v * v);
            if (b == 0) {
                if (rec) {
                    a.frames.pos[((size_t)slot * n + at) * 3 + c] = x;
                    a.frames.forces[((size_t)slot * n + at) * 3 + c] = (float)(Fd * kFxInv);
                }
                if (last) a.fxs[t] = (unsigned long long)F;
                if (energy || last || stop) {
                    a.x[t] = x;
                    a.v[t] = v;
                }
            }
            if (!last && !stop) {
                v = fma(S.h[at], Fd, v);   // v_{s+3/2}
                x = fma(a.dt, v, x);       // x_{s+2}
                reinterpret_cast<float *>(&S.pos[at])[c] = (float)x;
            }
            S.vel[at][c] = v;
            S.x[at][c] = x;
            bad |= !finite_bits(v);
        }
        if (bad) atomicOr(&S.pending, MDPF_STATUS_NONFINITE);
        if (energy && b == 0) {
            const double ks = warp_sum_d(kin);   // 3 n <= 96 slots: warps 0..2
            double eu = 0.0;                     // learned: atom t's energy (its terms summed in block order)
            if (!plain && t < n) {
                const int z = S.el[t];
                eu = (double)S.eat[t] + (double)L.b3[z] + L.e0[z];
            }
            eu = warp_sum_d(eu);   // n <= 32: warp 0
            if (lane == 0 && w < 4) S.red[w] = ks;
            if (t == 0) S.red[4] = eu;
            __syncthreads();
            if (t == 0) {
                const double K = (S.red[0] + S.red[1]) + (S.red[2] + S.red[3]);
                double U;
                if (plain) {
                    U = (fx_exact((long long)__ldcg(&eacc[1])) + fx_exact((long long)__ldcg(&eacc[2])) +
                         fx_exact((long long)__ldcg(&eacc[3]))) * kFxInv;
                } else {
                    U = S.red[4] + fx_exact((long long)__ldcg(&eacc[0])) * kFxInv;
                }
                const int64_t ei = done / a.energy_every - 1;
                a.trace_u[ei % a.trace_cap] = U;
                a.trace_k[ei % a.trace_cap] = K;
                a.trace_step[ei % a.trace_cap] = done;
                if (a.trace_fb != nullptr) a.trace_fb[ei % a.trace_cap] = L.lcount[1];
                a.scalars[0] = U;
                a.scalars[1] = K;
                if (!isfinite(U) || !isfinite(K)) atomicOr(&S.pending, MDPF_STATUS_NONFINITE);
                if (rec) {
                    a.frames.energy[slot] = U;
                    a.frames.step[slot] = done;
                }
            }
        }
        __syncthreads();
        if (stop || last) {
            if (t == 0 && S.pending != 0u) atomicOr(a.status, S.pending);
            if (b == 0 && t == 0) *a.step = done;
            return;
        }
    }
}

}  // namespace
}  // namespace mdpf

namespace mdpf {

struct SmallBuf {
    float *xG = nullptr, *xZ2 = nullptr, *xPG = nullptr;
    unsigned long long *fac = nullptr, *eacc = nullptr;
    unsigned int *flag = nullptr;
    int *el_list = nullptr, *el_cnt = nullptr;
};

static void small_release(SmallBuf *b) {
    void *ptrs[] = {b->xG, b->xZ2, b->xPG, b->fac, b->eacc, b->flag, b->el_list, b->el_cnt};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete b;
}

int small_create(mdpf_ctx *c, const int32_t *element) {
    if (c->n > kSmallMax || c->n < 1) return MDPF_ERR_UNSUPPORTED;
    int dev = c->device, sms = 0, coop = 0, occ = 0, smem_max = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < kSB)
        return MDPF_ERR_UNSUPPORTED;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
        return MDPF_ERR_UNSUPPORTED;
    if (cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        smem_max < (int)sizeof(SmallSmem))
        return MDPF_ERR_UNSUPPORTED;
    if (cudaFuncSetAttribute(k_learned_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SmallSmem)) !=
        cudaSuccess) {
        cudaGetLastError();
        return MDPF_ERR_UNSUPPORTED;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_learned_small, kSThreads, sizeof(SmallSmem)) !=
            cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        return MDPF_ERR_UNSUPPORTED;
    }
    SmallBuf *b = new SmallBuf();
    std::vector<int> el_list(4 * kSmallMax, 0), el_cnt(4, 0);
    for (int i = 0; i < c->n; ++i) {
        const int e = element[i];
        el_list[e * kSmallMax + el_cnt[e]++] = i;
    }
    bool ok = cudaMalloc(&b->xG, sizeof(float) * kSmallMax * kNFeat) == cudaSuccess &&
              cudaMalloc(&b->xZ2, sizeof(float) * kSB * kSmallMax * kH2) == cudaSuccess &&
              cudaMalloc(&b->xPG, sizeof(float) * kSB * kSmallMax * kNFeat) == cudaSuccess &&
              cudaMalloc(&b->fac, sizeof(unsigned long long) * 2 * 3 * kSmallMax) == cudaSuccess &&
              cudaMalloc(&b->eacc, sizeof(unsigned long long) * 2 * 4) == cudaSuccess &&
              cudaMalloc(&b->flag, sizeof(unsigned int) * 2) == cudaSuccess &&
              cudaMalloc(&b->el_list, sizeof(int) * 4 * kSmallMax) == cudaSuccess &&
              cudaMalloc(&b->el_cnt, sizeof(int) * 4) == cudaSuccess;
    ok = ok && cudaMemcpy(b->el_list, el_list.data(), sizeof(int) * 4 * kSmallMax, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->el_cnt, el_cnt.data(), sizeof(int) * 4, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        small_release(b);
        return MDPF_ERR_UNSUPPORTED;
    }
    c->small = b;
    return MDPF_OK;
}

void small_free(mdpf_ctx *c) {
    if (c->small) small_release(static_cast<SmallBuf *>(c->small));
    c->small = nullptr;
}

cudaError_t launch_learned_small(mdpf_ctx *c, int64_t n_steps, cudaStream_t s) {
    SmallBuf *buf = static_cast<SmallBuf *>(c->small);
    SmallArgs a;
    a.L = learned_dev(c);
    a.p = plain_dev(c, c->d_pos4);
    a.n = c->n;
    a.fallback = learned_fallback_on(c);
    a.dt = c->dt;
    a.hdt_m = c->d_hdt_m;
    a.mass = c->d_mass;
    a.qs = c->d_charge_s;
    a.x = c->d_x;
    a.v = c->d_v;
    a.fxs = c->d_fx;
    a.xG = buf->xG;
    a.xZ2 = buf->xZ2;
    a.xPG = buf->xPG;
    a.fac = buf->fac;
    a.eacc = buf->eacc;
    a.flag = buf->flag;
    a.el_list = buf->el_list;
    a.el_cnt = buf->el_cnt;
    a.trace_u = c->d_trace_u;
    a.trace_k = c->d_trace_k;
    a.trace_step = c->d_trace_step;
    a.trace_fb = c->d_trace_fb;
    a.trace_cap = c->trace_cap;
    a.energy_every = c->energy_every;
    a.step = c->d_step;
    a.status = c->d_status;
    a.scalars = c->d_scalar;
    a.frames = c->frames;
    a.record_every = c->frames.cap > 0 ? c->record_every : 0;
    a.bar = reinterpret_cast<unsigned long long *>(c->d_barrier);
    a.n_steps = n_steps;
    a.limit_ns = 1000000000LL;  // 1 s per barrier wait
    cudaError_t e = cudaMemsetAsync(c->d_barrier, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf->fac, 0, sizeof(unsigned long long) * 2 * 3 * kSmallMax, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf->eacc, 0, sizeof(unsigned long long) * 2 * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf->flag, 0, sizeof(unsigned int) * 2, s);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel((const void *)k_learned_small, dim3(kSB), dim3(kSThreads), args,
                                       sizeof(SmallSmem), s);
}

}  // namespace mdpf
