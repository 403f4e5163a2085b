// Per-atom device code of the learned potential, shared by the per-stage
// kernels (learned.cu) and the fused tile kernel (fused.cu): the neighbour
// geometry of one atom, its symmetry-function features, and the chain rule
// from dE/dG back to forces.  Both callers run the same code, so the two paths
// give the same bits.
//
//   radial    G[i, 16 Zj + k]           = sum_j  exp(-16 (r_ij - R_k)^2) fc(r_ij; 5.2)
//   angular   G[i, 64 + 32 P + 8 m + p] = sum_{j<k} 2^-31 (1 + cos(theta - theta_p))^32
//                                         exp(-8 ((r_ij + r_ik)/2 - R_m)^2) fc(r_ij; 3.5) fc(r_ik; 3.5)
//   theta = acos(0.95 cos theta_ijk), cos(theta - theta_p) = c cos theta_p + sqrt(1 - c^2) sin theta_p
//   R_k = 0.9 + 4.3 k / 16,  R_m = 0.9 + 0.65 m,  theta_p = (2 p + 1) pi / 16
// plus, when the model has one, a repulsive pair core that the features cannot
// express (they vanish as r -> 0, so no network on them can keep two atoms
// apart):  E_core = sum_{i<j, r < rc} A (1 - x)^3 / x,  x = r / rc.
// The Gaussians exp(x), x <= 0, are one ex2.approx instruction on x log2(e)
// (subnormal results flush to zero): the relative error grows with |x| but
// stays below ~2e-6 wherever exp(x) is not negligible (x > -30), far inside
// the FP32 feature tolerance, and the features and the adjoint use the same
// one.  Square roots and reciprocals are the approximate single-instruction
// forms (a few ulp): every argument is bounded away from zero (distances
// between distinct atoms, 1 - (0.95 cos)^2 >= 0.0975).
#pragma once

#include "learned.cuh"

namespace mdpf {
namespace {

constexpr float kPi = 3.14159265358979f;
constexpr float kEtaR = 16.f, kEtaA = 8.f;
constexpr float kAngScale = 0.95f;
constexpr float kTwoPowM31 = 4.656612873077393e-10f;  // 2^-31 = 2^(1 - zeta), zeta = 32


// exp(x) for x <= 0 (see the header).
__device__ __forceinline__ float exp_neg(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x * 1.4426950408889634f));
    return y;
}
__device__ __forceinline__ int pair_index(int a, int b) {
    if (a > b) {
        int t = a;
        a = b;
        b = t;
    }
    return (a == 0 ? 0 : (a == 1 ? 4 : (a == 2 ? 7 : 9))) + (b - a);
}

// One atom's neighbours, per warp (5,008 bytes).
struct NbrSmem {
    int j[kKmax];
    float4 d[kKmax];              // unit vector from i to j (x, y, z) and r
    float4 fc[kKmax];             // fc(r; 5.2), fc'(r; 5.2), fc(r; 3.5), fc'(r; 3.5)
    signed char el[kKmax];
    unsigned char rad[kKmax];     // neighbours within the radial cutoff, in row order
    unsigned char ang[kKmax];     // neighbours within the angular cutoff (by element for the features)
    int nae[4];                   // angular neighbours of each element (features)
};

// Cosine cutoff and its derivative at both cutoffs from one approximate
// sine/cosine pair each (the single-instruction forms, absolute error ~1e-6
// on [0, pi], the range used; larger arguments give values that are dropped):
// fc(r; rc) = (1 + cos(pi r / rc)) / 2, fc' = -pi / (2 rc) sin(pi r / rc), zero from rc on.
__device__ __forceinline__ float4 cutoffs(float r) {
    float sr, cr, sa, ca;
    __sincosf(r * (kPi / kRcRad), &sr, &cr);
    __sincosf(r * (kPi / kRcAng), &sa, &ca);
    const bool inr = r < kRcRad, ina = r < kRcAng;
    return make_float4(inr ? 0.5f * cr + 0.5f : 0.f, inr ? (-0.5f * kPi / kRcRad) * sr : 0.f,
                       ina ? 0.5f * ca + 0.5f : 0.f, ina ? (-0.5f * kPi / kRcAng) * sa : 0.f);
}

// The repulsive core of one pair at r < rc: energy A (1 - x)^3 / x and its
// r-derivative -(A / rc) (1 - x)^2 (1 + 2 x) / x^2, x = r / rc (zero with its
// first two derivatives at rc, growing as 1/r below).
__device__ __forceinline__ void core_pair(float r, float a, float rc, float &e, float &dedr) {
    const float x = __fdividef(r, rc), ix = __fdividef(1.f, x), om = 1.f - x;
    const float om2 = om * om;
    e = a * om2 * om * ix;
    dedr = -__fdividef(a, rc) * om2 * (1.f + 2.f * x) * ix * ix;
}

// Atom i's neighbour row in registers: lane l holds entries l, l + 32, ...
struct NbrFetch {
    float4 pi;
    int cnt;
    int j[kKmax / 32];
    float4 pj[kKmax / 32];
    int ej[kKmax / 32];
};

// Issue every global load of atom i's neighbours: the count and the whole
// index row at once (the row is allocated at full length, so this needs no
// count), then the positions and elements of the entries below the count.
// Two dependent memory round trips in all.
__device__ __forceinline__ void fetch_neighbours(const LearnedDev &L, const float4 *pos4, int i, int lane,
                                                 NbrFetch &f) {
    f.pi = pos4[i];
    f.cnt = L.nb_count[i];
    const int *row = L.nb_idx + (size_t)i * kKmax;
#pragma unroll
    for (int k = 0; k < kKmax / 32; ++k) f.j[k] = row[lane + 32 * k];
#pragma unroll
    for (int k = 0; k < kKmax / 32; ++k) {
        if (lane + 32 * k < f.cnt) {
            f.pj[k] = pos4[f.j[k]];
            f.ej[k] = L.el[f.j[k]];
        }
    }
}

// The fetched row into shared memory (geometry and cutoff values per entry);
// returns the row length and the numbers of neighbours within the radial and
// angular cutoffs.  ByElement: the angular list element by element (and the
// per-element counts), as the features need; otherwise in row order.  The compacted in-cutoff lists do not depend on how far the
// list radius reaches beyond the cutoffs, so neither does any summation order
// below.
template <bool ByElement>
__device__ __forceinline__ void store_neighbours(const NbrFetch &f, NbrSmem &s, int lane, int &cnt, int &nr,
                                                 int &na) {
    cnt = f.cnt;
#pragma unroll
    for (int k = 0; k < kKmax / 32; ++k) {
        const int q = lane + 32 * k;
        if (q < cnt) {
            const float dx = f.pj[k].x - f.pi.x, dy = f.pj[k].y - f.pi.y, dz = f.pj[k].z - f.pi.z;
            const float d2 = dx * dx + dy * dy + dz * dz, ir = rsqrtf(d2), r = d2 * ir;
            s.j[q] = f.j[k];
            s.el[q] = (signed char)f.ej[k];
            s.d[q] = make_float4(dx * ir, dy * ir, dz * ir, r);
            s.fc[q] = cutoffs(r);
        }
    }
    __syncwarp();
    const unsigned int below = (1u << lane) - 1u;
    if (!ByElement) {   // both lists in row order
        nr = 0;
        na = 0;
        for (int base = 0; base < cnt; base += 32) {
            const int q = base + lane;
            const float r = q < cnt ? s.d[q].w : 1e30f;
            const unsigned int br = __ballot_sync(0xffffffffu, r < kRcRad);
            if (r < kRcRad) s.rad[nr + __popc(br & below)] = (unsigned char)q;
            nr += __popc(br);
            const unsigned int ba = __ballot_sync(0xffffffffu, r < kRcAng);
            if (r < kRcAng) s.ang[na + __popc(ba & below)] = (unsigned char)q;
            na += __popc(ba);
        }
        __syncwarp();
        return;
    }
    // radial list in row order; angular neighbours counted per element, then listed element by element
    nr = 0;
    int ne[4] = {0, 0, 0, 0};
    for (int base = 0; base < cnt; base += 32) {
        const int q = base + lane;
        const float r = q < cnt ? s.d[q].w : 1e30f;
        const unsigned int br = __ballot_sync(0xffffffffu, r < kRcRad);
        if (r < kRcRad) s.rad[nr + __popc(br & below)] = (unsigned char)q;
        nr += __popc(br);
        const int e = q < cnt ? s.el[q] : -1;
#pragma unroll
        for (int k = 0; k < 4; ++k) ne[k] += __popc(__ballot_sync(0xffffffffu, r < kRcAng && e == k));
    }
    int at[4] = {0, ne[0], ne[0] + ne[1], ne[0] + ne[1] + ne[2]};
    na = at[3] + ne[3];
    for (int base = 0; base < cnt; base += 32) {
        const int q = base + lane;
        const bool in = q < cnt && s.d[q].w < kRcAng;
        const int e = q < cnt ? s.el[q] : -1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned int b = __ballot_sync(0xffffffffu, in && e == k);
            if (in && e == k) s.ang[at[k] + __popc(b & below)] = (unsigned char)q;
            at[k] += __popc(b);
        }
    }
    if (lane < 4) s.nae[lane] = lane == 0 ? ne[0] : (lane == 1 ? ne[1] : (lane == 2 ? ne[2] : ne[3]));
    __syncwarp();
}

template <bool ByElement>
__device__ __forceinline__ void load_neighbours(const LearnedDev &L, const float4 *pos4, int i, NbrSmem &s, int lane,
                                                int &cnt, int &nr, int &na) {
    NbrFetch f;
    fetch_neighbours(L, pos4, i, lane, f);
    store_neighbours<ByElement>(f, s, lane, cnt, nr, na);
}

// Triplet t of the pairs (a, b), a < b, of na angular neighbours, in row-major order.
__device__ __forceinline__ void triplet_ab(int t, int na, int &a, int &b) {
    a = 0;
    while (t >= na - 1 - a) {
        t -= na - 1 - a;
        ++a;
    }
    b = a + 1 + t;
}
// Inverse of triplet_ab.
__device__ __forceinline__ int triplet_index(int a, int b, int na) { return a * (na - 1) - a * (a - 1) / 2 + (b - a - 1); }

// ------------------------------------------------------------------ features

// Per-warp staging of one batch of 32 triplet slots, the atom's pair-type
// table and its angular sums (2,512 bytes).
struct TripStage {
    float4 q[32];    // cos, sin of the scaled angle, 2^-31 fc(r_j) fc(r_k), pair type
    float4 b[32];    // radial-shell factors of the 4 shells
    int4 type[10];   // per pair type: first slot, triplets, first angular index of e1 | of e2 << 8 | count of
                     // e2 << 16, e1 == e2
    float rcp[12];   // 1 / (count of e2)
    float acc[10][32];   // angular block of each pair type: column 8 m + p of the block in lane 8 m + p
};

// Features of one atom whose neighbours are in s.  On return lane l holds
// G[32 b + l] in v[b], b = 0..11.
//   radial: lane 16 h + k sums the in-cutoff neighbours u = h, h + 2, ... into
//     its four per-element sums (registers), then the two halves are added;
//   angular: the angular neighbours are listed by element, so the triplets of
//     pair type (e1, e2) are the pairs (a, b) with a in e1's range and b in
//     e2's (a < b when e1 = e2).  The atom's triplets are laid out type by
//     type, each type's run padded to a multiple of 4 slots with empty
//     triplets, and processed in batches of 32 slots: each lane stages one
//     slot's geometry; then lane 8 t4 + p takes slot t4 of every group of 4
//     (all of one type), computes its angular factor for section p once and
//     adds it, times the 4 shell factors, to its 4 column sums (m = 0..3).
//     When the type changes, the four slot groups' sums are combined by a
//     reduce-scatter in a fixed order (lanes t4 and t4 ^ 2 first, then t4 and
//     t4 ^ 1), after which lane 8 m + p holds sum m of its section and adds it
//     to the shared sum of column 64 + 32 P + 8 m + p (each type is flushed
//     once: its slots are contiguous).
// Every sum is taken in a fixed order, so the result does not depend on the
// caller.  Part: 1 the radial columns only (v[0..1]), 2 the angular ones only
// (v[2..11]), 3 both; a part's values are the same bits in every case.
template <int Part = 3>
__device__ __forceinline__ void feature_row(const NbrSmem &s, int nr, int na, TripStage &ts, int lane, float (&v)[12]) {
    if (Part & 1) {
        const int h = lane >> 4, k = lane & 15;
        const float Rk = 0.9f + (float)k * (4.3f / 16.f);
        float racc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int u = h; u < nr; u += 2) {
            const int q = s.rad[u];
            const float x = s.d[q].w - Rk;
            const float t = exp_neg(-kEtaR * x * x);
            const float fc = s.fc[q].x;
            const int e = s.el[q];
#pragma unroll
            for (int ee = 0; ee < 4; ++ee)
                if (ee == e) racc[ee] = fmaf(t, fc, racc[ee]);
        }
        float tot[4];
#pragma unroll
        for (int ee = 0; ee < 4; ++ee) tot[ee] = racc[ee] + __shfl_xor_sync(0xffffffffu, racc[ee], 16);
        v[0] = h ? tot[1] : tot[0];   // column l      = 16 h + k:       element h
        v[1] = h ? tot[3] : tot[2];   // column 32 + l = 16 (2 + h) + k: element 2 + h
    }
    if (Part & 2) {
        const int t4 = lane >> 3, p = lane & 7;
        const float thp = (float)(2 * p + 1) * (kPi / 16.f);
        const float cp = cosf(thp), sp = sinf(thp);
        // the pair-type table (lane P writes type P) and the padded run starts (every lane)
        int ne[4], st[4], off[10];
#pragma unroll
        for (int e = 0; e < 4; ++e) ne[e] = s.nae[e];
        st[0] = 0;
        st[1] = ne[0];
        st[2] = st[1] + ne[1];
        st[3] = st[2] + ne[2];
        int total = 0;
#pragma unroll
        for (int P = 0; P < 10; ++P) {
            // elements (e1 <= e2) of pair type P, in the column order of the angular blocks
            constexpr int e1s[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3}, e2s[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
            const int e1 = e1s[P], e2 = e2s[P];
            const int n = e1 == e2 ? ne[e1] * (ne[e1] - 1) / 2 : ne[e1] * ne[e2];
            if (lane == P) {
                ts.type[P] = make_int4(total, n, st[e1] | (st[e2] << 8) | (ne[e2] << 16), e1 == e2 ? 1 : 0);
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
            // lanes t4 and t4 ^ 2 exchange the two sums the other keeps (m with bit 1 = its t4's bit 1) ...
            const float a0 = acc[0], a1 = acc[1], a2 = acc[2], a3 = acc[3];
            float k0 = hi ? a2 : a0, k1 = hi ? a3 : a1;
            const float s0 = hi ? a0 : a2, s1 = hi ? a1 : a3;
            k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
            k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
            // ... then lanes t4 and t4 ^ 1 the one with bit 0 = the other's t4's bit 0: lane 8 m + p has sum m
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
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f), bq = make_float4(0.f, 0.f, 0.f, 0.f);
            if (slot < total) {
                const int4 ty = ts.type[P];
                const int l = slot - ty.x;
                if (l < ty.y) {
                    const int a0 = ty.z & 255, b0 = (ty.z >> 8) & 255, c2 = ty.z >> 16;
                    int a, b;
                    if (ty.w) {   // both neighbours of one element: pairs a < b of its range
                        triplet_ab(l, c2, a, b);
                        a += a0;
                        b += a0;
                    } else {      // a in e1's range, b in e2's (exact: l < 2^14)
                        a = (int)(((float)l + 0.5f) * ts.rcp[P]);
                        b = b0 + (l - a * c2);
                        a += a0;
                    }
                    const int qa = s.ang[a], qb = s.ang[b];
                    const float4 dj = s.d[qa], dk = s.d[qb];
                    const float ct = dj.x * dk.x + dj.y * dk.y + dj.z * dk.z;
                    const float cs = kAngScale * ct;
                    const float s2 = 1.f - cs * cs;   // >= 1 - 0.95^2
                    q = make_float4(cs, s2 * rsqrtf(s2), kTwoPowM31 * s.fc[qa].z * s.fc[qb].z, 0.f);
                    const float ravg = 0.5f * (dj.w + dk.w);
                    float bm[4];
#pragma unroll
                    for (int mm = 0; mm < 4; ++mm) {
                        const float x = ravg - (0.9f + (float)mm * 0.65f);
                        bm[mm] = exp_neg(-kEtaA * x * x);
                    }
                    bq = make_float4(bm[0], bm[1], bm[2], bm[3]);
                }
            }
            q.w = __int_as_float(P);   // empty slots of a run carry its type and contribute zero
            ts.q[lane] = q;
            ts.b[lane] = bq;
            __syncwarp();
            const int ng = min(32, total - base);   // a multiple of 4
            for (int u = 0; u < ng; u += 4) {
                const float4 qq = ts.q[u + t4];
                const int Pu = __float_as_int(ts.q[u].w);   // the group's pair type, the same in every lane
                if (Pu != curP) {
                    if (curP >= 0) flush();
                    curP = Pu;
                }
                float x = 1.f + qq.x * cp + qq.y * sp;
                x *= x; x *= x; x *= x; x *= x; x *= x;  // ^32
                const float xc = x * qq.z;
                const float4 bb = ts.b[u + t4];
                acc[0] = fmaf(xc, bb.x, acc[0]);
                acc[1] = fmaf(xc, bb.y, acc[1]);
                acc[2] = fmaf(xc, bb.z, acc[2]);
                acc[3] = fmaf(xc, bb.w, acc[3]);
            }
            __syncwarp();
        }
        if (curP >= 0) flush();
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 10; ++k) v[2 + k] = ts.acc[k][lane];
    }
}

// ------------------------------------------------------------------ adjoint

// Angular blocks of a g row are stored kAngStride floats apart: a multiple of
// four, so that every 8-float run of a block is two 16-byte loads, and 4 mod
// 32 banks apart, so that lanes working on different element pairs mostly
// read different banks.  Rows are 16-byte aligned.
constexpr int kAngStride = 36;
constexpr int kGRow = 64 + 10 * kAngStride;   // floats of one g row in that layout

// Per-warp scratch of the adjoint: Chunk triplets are staged per pass (a
// multiple of 32; the result does not depend on it).
template <int Chunk>
struct AdjScratch {
    static_assert(Chunk % 32 == 0, "triplet t is always taken by lane t mod 32");
    float f[kKmax][3];                  // force on each neighbour (FP32, fixed summation order)
    float tj[Chunk][3], tk[Chunk][3];   // staged triplet contributions to j and k
};

// Column of feature f of a g row in the padded layout.
__device__ __forceinline__ int g_col(int f) { return f < 64 ? f : 64 + kAngStride * ((f - 64) >> 5) + ((f - 64) & 31); }

// F = -dE/dx by the chain rule through the features of atom i (neighbours in
// s, g = dE/dG_i in the padded layout): for every radial pair and angular
// triplet around atom i, the contraction of g with the derivative of the
// feature terms.  Each neighbour's radial force is written by the one lane
// that owns the pair; triplet contributions are staged per chunk and each lane
// then sums, in a fixed order, those of the triplets that contain its
// neighbour; the force on atom i is summed per lane and reduced over the warp
// in a fixed order.  Triplet t is taken by lane t mod 32 and each neighbour's
// force is one running sum (radial term, then its triplets in index order), so
// no sum depends on the chunk size.  The sums go to fx as int64 fixed point,
// so the result is reproducible bit for bit.
// core = (A, rc) of the repulsive core (rc == 0: none).  Every pair sits in
// both atoms' rows, so each side adds half of the pair's core energy and
// force; the half energies of atom i go to *ecore (fixed point) when ecore is
// set.  Part: 1 the radial pairs (and the core) only, 2 the angular triplets
// only, 3 both (two warps may share an atom that way: their fixed-point adds
// commute, though the split rounds each part to fixed point apart).
template <int Chunk, int Part = 3>
__device__ __forceinline__ void adjoint_atom(int i, const NbrSmem &s, int cnt, int nr, int na, const float *g,
                                             AdjScratch<Chunk> &A, unsigned long long *fx, int lane,
                                             float2 core = make_float2(0.f, 0.f),
                                             unsigned long long *ecore = nullptr) {
    for (int q = lane; q < cnt * 3; q += 32) (&A.f[0][0])[q] = 0.f;
    __syncwarp();
    float fix = 0.f, fiy = 0.f, fiz = 0.f;
    float ecore_i = 0.f;
    // radial pairs: dE/dr = sum_k g[16 Zj + k] dT_k/dr;  F_j = -dE/dr u,  F_i += dE/dr u
    for (int u = lane; (Part & 1) && u < nr; u += 32) {
        const int q = s.rad[u];
        const float4 d = s.d[q];
        const float r = d.w;
        const float fc = s.fc[q].x, dfc = s.fc[q].y;
        const float4 *gz = reinterpret_cast<const float4 *>(g + 16 * s.el[q]);
        float dEdr = 0.f;
#pragma unroll
        for (int k4 = 0; k4 < 4; ++k4) {
            const float4 g4 = gz[k4];
            const float gk[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const int k = 4 * k4 + kk;
                const float x = r - (0.9f + (float)k * (4.3f / 16.f));
                const float ex = exp_neg(-kEtaR * x * x);
                dEdr = fmaf(gk[kk], ex * (-2.f * kEtaR * x * fc + dfc), dEdr);
            }
        }
        if (r < core.y) {
            float ec, dc;
            core_pair(r, core.x, core.y, ec, dc);
            dEdr = fmaf(0.5f, dc, dEdr);
            ecore_i = fmaf(0.5f, ec, ecore_i);
        }
        const float sx = dEdr * d.x, sy = dEdr * d.y, sz = dEdr * d.z;
        A.f[q][0] = -sx;
        A.f[q][1] = -sy;
        A.f[q][2] = -sz;
        fix += sx;
        fiy += sy;
        fiz += sz;
    }
    __syncwarp();
    // angular triplets; cos and sin of theta_p = (2 p + 1) pi / 16 as literals (immediate operands)
    constexpr float cpv[8] = {9.807852804e-01f, 8.314696123e-01f, 5.555702330e-01f, 1.950903220e-01f, -1.950903220e-01f, -5.555702330e-01f, -8.314696123e-01f, -9.807852804e-01f};
    constexpr float spv[8] = {1.950903220e-01f, 5.555702330e-01f, 8.314696123e-01f, 9.807852804e-01f, 9.807852804e-01f, 8.314696123e-01f, 5.555702330e-01f, 1.950903220e-01f};
    const int ntrip = (Part & 2) ? na * (na - 1) / 2 : 0;
    int kcur[kKmax / 32] = {0, 0, 0, 0};
    for (int t0 = 0; t0 < ntrip; t0 += Chunk) {
        const int t1 = min(t0 + Chunk, ntrip);
        for (int t = t0 + lane; t < t1; t += 32) {
            int a, b;
            triplet_ab(t, na, a, b);
            const int qa = s.ang[a], qb = s.ang[b];
            const float4 dj = s.d[qa], dk = s.d[qb];
            const float rj = dj.w, rk = dk.w;
            const float irj = __fdividef(1.f, rj), irk = __fdividef(1.f, rk);
            const float ujx = dj.x, ujy = dj.y, ujz = dj.z;
            const float ukx = dk.x, uky = dk.y, ukz = dk.z;
            const float ct = ujx * ukx + ujy * uky + ujz * ukz;
            const float cs = kAngScale * ct;
            const float s2 = 1.f - cs * cs, isn = rsqrtf(s2);   // s2 >= 1 - 0.95^2
            const float sn2 = s2 * isn;
            const float cot = cs * isn;
            const float fj = s.fc[qa].z, fk = s.fc[qb].z;
            const float dfj = s.fc[qa].w, dfk = s.fc[qb].w;
            const float C = fj * fk;
            const float ravg = 0.5f * (rj + rk);
            const float4 *gp = reinterpret_cast<const float4 *>(g + 64 + kAngStride * pair_index(s.el[qa], s.el[qb]));
            // angular factors A_p = 2^-31 (1 + cos(theta - theta_p))^32 and their derivatives in cos(theta),
            // 2^-31 * 32 (1 + cos(theta - theta_p))^31 (cos theta_p - cot sin theta_p), both without their
            // power-of-two factors, which scale the three sums below exactly and are applied to them at the end
            float Ap[8], dAp[8];
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const float base = 1.f + cs * cpv[p] + sn2 * spv[p];
                const float b2 = base * base, b4 = b2 * b2, b8 = b4 * b4, b16 = b8 * b8;
                const float b31 = b16 * b8 * b4 * b2 * base;
                Ap[p] = b31 * base;
                dAp[p] = b31 * (cpv[p] - cot * spv[p]);
            }
            float Sc = 0.f, Sr = 0.f, SC = 0.f;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float x = ravg - (0.9f + (float)m * 0.65f);
                const float B = exp_neg(-kEtaA * x * x);
                const float dB = -2.f * kEtaA * x * B;
                const float4 ga = gp[2 * m], gb = gp[2 * m + 1];
                const float gv[8] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w};
                float sa_ = 0.f, sdA = 0.f;
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    sa_ = fmaf(gv[p], Ap[p], sa_);
                    sdA = fmaf(gv[p], dAp[p], sdA);
                }
                Sc = fmaf(sdA, B * C, Sc);
                Sr = fmaf(sa_, dB * C, Sr);
                SC = fmaf(sa_, B, SC);
            }
            Sc *= kTwoPowM31 * 32.f;
            Sr *= kTwoPowM31;
            SC *= kTwoPowM31;
            const float dEdrj = 0.5f * Sr + SC * dfj * fk, dEdrk = 0.5f * Sr + SC * fj * dfk;
            const float gc = Sc * kAngScale;
            const float gjx = gc * (ukx - ct * ujx) * irj + dEdrj * ujx;
            const float gjy = gc * (uky - ct * ujy) * irj + dEdrj * ujy;
            const float gjz = gc * (ukz - ct * ujz) * irj + dEdrj * ujz;
            const float gkx = gc * (ujx - ct * ukx) * irk + dEdrk * ukx;
            const float gky = gc * (ujy - ct * uky) * irk + dEdrk * uky;
            const float gkz = gc * (ujz - ct * ukz) * irk + dEdrk * ukz;
            float *tj = A.tj[t - t0], *tk = A.tk[t - t0];
            tj[0] = -gjx;
            tj[1] = -gjy;
            tj[2] = -gjz;
            tk[0] = -gkx;
            tk[1] = -gky;
            tk[2] = -gkz;
            fix += gjx + gkx;
            fiy += gjy + gky;
            fiz += gjz + gkz;
        }
        __syncwarp();
        if (ntrip <= Chunk) {
            // one chunk holds every triplet: the same sums, with partner loops of fixed length
#pragma unroll
            for (int sl = 0; sl < kKmax / 32; ++sl) {
                const int a = lane + 32 * sl;
                if (a >= na) continue;
                const int q = s.ang[a];
                float ax = A.f[q][0], ay = A.f[q][1], az = A.f[q][2];
                int t = a - 1;   // triplet (0, a); it grows by na - 2 - b from partner b to b + 1
#pragma unroll 4
                for (int b = 0; b < a; ++b) {
                    const float *v = A.tk[t];
                    ax += v[0];
                    ay += v[1];
                    az += v[2];
                    t += na - 2 - b;
                }
                const int ra = triplet_index(a, a + 1, na), rb = ra + (na - a - 1);
#pragma unroll 4
                for (int u = ra; u < rb; ++u) {
                    const float *v = A.tj[u];
                    ax += v[0];
                    ay += v[1];
                    az += v[2];
                }
                A.f[q][0] = ax;
                A.f[q][1] = ay;
                A.f[q][2] = az;
            }
            __syncwarp();
            continue;
        }
        // each lane, for its angular neighbours a = lane + 32 sl: the staged contributions of
        // this chunk, in triplet order.  Those of the triplets (b, a), b < a, come first (their
        // indices grow with b; kcur carries the next b across chunks), then those of (a, b),
        // b > a, whose indices are contiguous.  Over all chunks this is one running sum per
        // neighbour in triplet index order, whatever the chunk size.
#pragma unroll
        for (int sl = 0; sl < kKmax / 32; ++sl) {
            const int a = lane + 32 * sl;
            if (a >= na) continue;
            const int q = s.ang[a];
            float ax = A.f[q][0], ay = A.f[q][1], az = A.f[q][2];
            int b = kcur[sl];
            for (; b < a; ++b) {
                const int t = triplet_index(b, a, na);
                if (t >= t1) break;
                const float *v = A.tk[t - t0];
                ax += v[0];
                ay += v[1];
                az += v[2];
            }
            kcur[sl] = b;
            if (a + 1 < na) {
                const int ra = triplet_index(a, a + 1, na);
                const int lo = max(ra, t0), hi = min(ra + (na - a - 2), t1 - 1);
                for (int t = lo; t <= hi; ++t) {
                    const float *v = A.tj[t - t0];
                    ax += v[0];
                    ay += v[1];
                    az += v[2];
                }
            }
            A.f[q][0] = ax;
            A.f[q][1] = ay;
            A.f[q][2] = az;
        }
        __syncwarp();
    }
    for (int q = lane; q < cnt; q += 32) {
        const int j = s.j[q];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long v = fx_from_float(A.f[q][c]);
            if (v != 0) atomicAdd(&fx[3 * j + c], (unsigned long long)v);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fix += __shfl_xor_sync(0xffffffffu, fix, o);
        fiy += __shfl_xor_sync(0xffffffffu, fiy, o);
        fiz += __shfl_xor_sync(0xffffffffu, fiz, o);
    }
    if (lane == 0) {
        atomicAdd(&fx[3 * i + 0], (unsigned long long)fx_from_float(fix));
        atomicAdd(&fx[3 * i + 1], (unsigned long long)fx_from_float(fiy));
        atomicAdd(&fx[3 * i + 2], (unsigned long long)fx_from_float(fiz));
    }
    if (ecore != nullptr && core.y > 0.f) {
        // the core energy of atom i: lane sums reduced in a fixed order, one fixed-point add when nonzero
        double e = (double)ecore_i;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if (lane == 0 && e != 0.0) fx_add_d(ecore, e);
    }
    __syncwarp();
}

}  // namespace
}  // namespace mdpf
