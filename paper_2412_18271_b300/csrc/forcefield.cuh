// Force-field device routines shared by the kernel-sequence stepper and the
// persistent stepper: one bonded term, and one work item of the all-pairs
// LJ + Coulomb sum.
//
// The all-pairs sum is cut into 32-atom tiles (one atom per lane).  A work
// item is one of
//   ITEM_OFF64 (p, J)  tiles 2p and 2p+1 against tile J > 2p+1: every lane
//                      owns two i-atoms, so each j read serves two pairs;
//   ITEM_OFF32 (I, J)  tile I against tile J > I, one i-atom per lane;
//   ITEM_SELF  (I)     the pairs inside tile I;
//   ITEM_BONDED (I)    no pairs: a share of tile I's bonded terms, for a
//                      stepper that spreads them over more warps (the
//                      pair sum skips it).
// Off-diagonal items apply Newton's third law: the j-tile sits in shared
// memory, lane l meets j-lane (l + k) & 31 at step k, and the j-force
// accumulator travels with its j index (one lane down per step, three
// shuffles).  Two accumulators run half a tile apart (offsets k and k + 16)
// so that every step carries independent pair chains.  Self tiles evaluate
// each ordered pair once, keep the i-force only and halve the energy.
//
// Per-atom data: pos4 = (x, y, z, q sqrt(ke)), lj = (sigma/2, sqrt(24 eps)),
// so that sigma_ij = a_i + a_j and 24 eps_ij = b_i b_j (Lorentz-Berthelot).
// Pair terms, with s = sigma_ij / r:
//   E = 4 eps (s^12 - s^6) + ke q_i q_j / r
//   F_i = -fs d,  F_j = +fs d,  d = x_j - x_i,
//   fs = [24 eps (2 s^12 - s^6) + ke q_i q_j / r] / r^2
#pragma once

#include "device_util.cuh"

namespace mdpf {

enum { ITEM_OFF64 = 0, ITEM_OFF32 = 1, ITEM_SELF = 2, ITEM_BONDED = 3 };

// One bonded term t: bonds are t < n_bonds, angles follow.  A term is
// described by a record r = (i, j, -1, t) for a bond, (a, v, b, t) for an
// angle with vertex v; its evaluation is split into the record, a gather of
// what it reads (positions, bond parameters) and the arithmetic, so that a
// caller can keep records and issue the loads of several terms before
// evaluating any.  Energies are added to eb / ea, forces to the fixed-point
// accumulators.
struct BondedGeom {
    float4 xa, xb, xc;  // bond: x_i, x_j; angle: x_a, x_v, x_b
    float2 par;         // bond: r0, k
};

__device__ __forceinline__ int4 bonded_rec(const PlainDev &p, int t) {
    if (t < p.n_bonds) {
        const int2 b = p.bonds[t];
        return make_int4(b.x, b.y, -1, t);
    }
    const int4 an = p.angles[t - p.n_bonds];
    return make_int4(an.x, an.y, an.z, t);
}

__device__ __forceinline__ void bonded_gather(const PlainDev &p, const int4 &r, BondedGeom &g) {
    g.xa = p.pos4[r.x];
    g.xb = p.pos4[r.y];
    if (r.z >= 0) {
        g.xc = p.pos4[r.z];
    } else {
        g.xc = make_float4(0.f, 0.f, 0.f, 0.f);
        g.par = p.bond_par[r.w];
    }
}

// 1/sqrt(x) and 1/x as single PTX approximate instructions with subnormals
// flushed: x is a squared length here, never subnormal for a term or pair
// that is evaluated.
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Forces of one bonded term on its atoms: fa on r.x, fb on r.y, fc on r.z
// (angles; zero for a bond), and its energy.  Every output is always
// computed, whichever of them a caller uses, so that the FP32 values are the
// same in every kernel that evaluates the term.
//   bond  (i, j):   E = k/2 (r - r0)^2,  F_i = k (r - r0) / r d,  F_j = -F_i,  d = x_j - x_i
//   angle (a, v, b), u = x_a - x_v, w = x_b - x_v, theta = atan2(|u x w|, u.w):
//         E = k/2 (theta - theta0)^2,
//         F_a = k (theta - theta0) / |u x w| (w - (u.w / u.u) u),
//         F_b = k (theta - theta0) / |u x w| (u - (u.w / w.w) w),  F_v = -(F_a + F_b)
__device__ __forceinline__ void bonded_forces(const PlainDev &p, const int4 &r, const BondedGeom &g, float3 &fa,
                                              float3 &fb, float3 &fc, float &e) {
    if (r.z < 0) {
        const float4 xi = g.xa, xj = g.xb;
        const float2 par = g.par;
        const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float ir = rsqrt_approx(r2);
        const float dr = r2 * ir - par.x;
        e = 0.5f * par.y * dr * dr;
        const float gg = par.y * dr * ir;
        fa = make_float3(gg * dx, gg * dy, gg * dz);
        fb = make_float3(-fa.x, -fa.y, -fa.z);
        fc = make_float3(0.f, 0.f, 0.f);
    } else {
        const float4 xa = g.xa, xv = g.xb, xb = g.xc;
        const float ux = xa.x - xv.x, uy = xa.y - xv.y, uz = xa.z - xv.z;
        const float wx = xb.x - xv.x, wy = xb.y - xv.y, wz = xb.z - xv.z;
        const float uu = fmaf(ux, ux, fmaf(uy, uy, uz * uz)), ww = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
        const float c = fmaf(ux, wx, fmaf(uy, wy, uz * wz));
        const float cx = fmaf(uy, wz, -uz * wy), cy = fmaf(uz, wx, -ux * wz), cz = fmaf(ux, wy, -uy * wx);
        const float cr2 = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
        const float icr = rsqrt_approx(cr2);
        const float th = atan2f(cr2 * icr, c);
        const float dth = th - p.angle_theta0;
        e = 0.5f * p.angle_k * dth * dth;
        const float gk = p.angle_k * dth * icr;
        const float ca = c * rcp_approx(uu), cb = c * rcp_approx(ww);
        fa = make_float3(gk * fmaf(-ca, ux, wx), gk * fmaf(-ca, uy, wy), gk * fmaf(-ca, uz, wz));
        fc = make_float3(gk * fmaf(-cb, wx, ux), gk * fmaf(-cb, wy, uy), gk * fmaf(-cb, wz, uz));
        fb = make_float3(-(fa.x + fc.x), -(fa.y + fc.y), -(fa.z + fc.z));
    }
}

__device__ __forceinline__ void bonded_eval(const PlainDev &p, const int4 &r, const BondedGeom &g,
                                            unsigned long long *fx, float &eb, float &ea) {
    float3 fa, fb, fc;
    float e;
    bonded_forces(p, r, g, fa, fb, fc, e);
    if (r.z < 0) eb += e;
    else ea += e;
    fx_add(&fx[3 * r.x + 0], fa.x);
    fx_add(&fx[3 * r.x + 1], fa.y);
    fx_add(&fx[3 * r.x + 2], fa.z);
    fx_add(&fx[3 * r.y + 0], fb.x);
    fx_add(&fx[3 * r.y + 1], fb.y);
    fx_add(&fx[3 * r.y + 2], fb.z);
    if (r.z >= 0) {
        fx_add(&fx[3 * r.z + 0], fc.x);
        fx_add(&fx[3 * r.z + 1], fc.y);
        fx_add(&fx[3 * r.z + 2], fc.z);
    }
}

__device__ __forceinline__ void bonded_term(const PlainDev &p, int t, unsigned long long *fx, float &eb,
                                            float &ea) {
    if (t >= p.n_bonds + p.n_angles) return;
    const int4 r = bonded_rec(p, t);
    BondedGeom g;
    bonded_gather(p, r, g);
    bonded_eval(p, r, g, fx, eb, ea);
}

// One pair: returns fs (0 when skipped); accumulates energies (elj carries
// 24 eps (s^12 - s^6), i.e. six times the LJ energy).
template <bool MASKED, bool ENERGY>
__device__ __forceinline__ float pair_fs(const float4 &pi, const float2 &li, const float4 &pj, const float2 &lj,
                                         bool skip, float &dx, float &dy, float &dz, float &elj, float &ec) {
    dx = pj.x - pi.x;
    dy = pj.y - pi.y;
    dz = pj.z - pi.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float rinv = rsqrt_approx(r2);
    const float r2inv = rinv * rinv;
    const float sr = (li.x + lj.x) * rinv;
    const float s2 = sr * sr;
    const float s6 = s2 * s2 * s2;
    const float s12 = s6 * s6;
    const float e6 = li.y * lj.y;
    const float ecp = pi.w * pj.w * rinv;
    float fs = fmaf(e6, fmaf(2.f, s12, -s6), ecp) * r2inv;
    if (MASKED) fs = skip ? 0.f : fs;
    if (ENERGY) {
        const float el = e6 * (s12 - s6);
        elj += (MASKED && skip) ? 0.f : el;
        ec += (MASKED && skip) ? 0.f : ecp;
    }
    return fs;
}

__device__ __forceinline__ void rot3(float3 &v, int src) {
    v.x = __shfl_sync(0xffffffffu, v.x, src);
    v.y = __shfl_sync(0xffffffffu, v.y, src);
    v.z = __shfl_sync(0xffffffffu, v.z, src);
}

// Two i-atoms per lane against the j-tile in shared memory.
template <bool MASKED, bool ENERGY>
__device__ __forceinline__ void item_off64(const float4 *sj, const float2 *sab, const float4 &pi0, const float2 &li0,
                                           const float4 &pi1, const float2 &li1, uint32_t m0, uint32_t m1, int lane,
                                           float3 &fi0, float3 &fi1, float3 &fj, float &elj, float &ec) {
    float3 fa = make_float3(0.f, 0.f, 0.f), fb = make_float3(0.f, 0.f, 0.f);
    const int nxt = (lane + 1) & 31;
#pragma unroll 4
    for (int k = 0; k < 16; ++k) {
        const int sA = (lane + k) & 31, sB = (lane + k + 16) & 31;
        const float4 ja = sj[sA], jb = sj[sB];
        const float2 aa = sab[sA], ab = sab[sB];
        float dx, dy, dz, fs;
        fs = pair_fs<MASKED, ENERGY>(pi0, li0, ja, aa, (m0 >> sA) & 1u, dx, dy, dz, elj, ec);
        fi0.x = fmaf(-fs, dx, fi0.x); fi0.y = fmaf(-fs, dy, fi0.y); fi0.z = fmaf(-fs, dz, fi0.z);
        fa.x = fmaf(fs, dx, fa.x); fa.y = fmaf(fs, dy, fa.y); fa.z = fmaf(fs, dz, fa.z);
        fs = pair_fs<MASKED, ENERGY>(pi1, li1, ja, aa, (m1 >> sA) & 1u, dx, dy, dz, elj, ec);
        fi1.x = fmaf(-fs, dx, fi1.x); fi1.y = fmaf(-fs, dy, fi1.y); fi1.z = fmaf(-fs, dz, fi1.z);
        fa.x = fmaf(fs, dx, fa.x); fa.y = fmaf(fs, dy, fa.y); fa.z = fmaf(fs, dz, fa.z);
        fs = pair_fs<MASKED, ENERGY>(pi0, li0, jb, ab, (m0 >> sB) & 1u, dx, dy, dz, elj, ec);
        fi0.x = fmaf(-fs, dx, fi0.x); fi0.y = fmaf(-fs, dy, fi0.y); fi0.z = fmaf(-fs, dz, fi0.z);
        fb.x = fmaf(fs, dx, fb.x); fb.y = fmaf(fs, dy, fb.y); fb.z = fmaf(fs, dz, fb.z);
        fs = pair_fs<MASKED, ENERGY>(pi1, li1, jb, ab, (m1 >> sB) & 1u, dx, dy, dz, elj, ec);
        fi1.x = fmaf(-fs, dx, fi1.x); fi1.y = fmaf(-fs, dy, fi1.y); fi1.z = fmaf(-fs, dz, fi1.z);
        fb.x = fmaf(fs, dx, fb.x); fb.y = fmaf(fs, dy, fb.y); fb.z = fmaf(fs, dz, fb.z);
        rot3(fa, nxt);
        rot3(fb, nxt);
    }
    // fa now belongs to j-lane (lane + 16) & 31, fb to j-lane lane
    rot3(fa, (lane + 16) & 31);
    fj.x = fa.x + fb.x;
    fj.y = fa.y + fb.y;
    fj.z = fa.z + fb.z;
}

// One i-atom per lane against the j-tile in shared memory.
template <bool MASKED, bool ENERGY>
__device__ __forceinline__ void item_off32(const float4 *sj, const float2 *sab, const float4 &pi0, const float2 &li0,
                                           uint32_t m0, int lane, float3 &fi0, float3 &fj, float &elj, float &ec) {
    float3 fa = make_float3(0.f, 0.f, 0.f), fb = make_float3(0.f, 0.f, 0.f);
    const int nxt = (lane + 1) & 31;
#pragma unroll 2
    for (int k = 0; k < 16; ++k) {
        const int sA = (lane + k) & 31, sB = (lane + k + 16) & 31;
        const float4 ja = sj[sA], jb = sj[sB];
        const float2 aa = sab[sA], ab = sab[sB];
        float dx, dy, dz, fs;
        fs = pair_fs<MASKED, ENERGY>(pi0, li0, ja, aa, (m0 >> sA) & 1u, dx, dy, dz, elj, ec);
        fi0.x = fmaf(-fs, dx, fi0.x); fi0.y = fmaf(-fs, dy, fi0.y); fi0.z = fmaf(-fs, dz, fi0.z);
        fa.x = fmaf(fs, dx, fa.x); fa.y = fmaf(fs, dy, fa.y); fa.z = fmaf(fs, dz, fa.z);
        fs = pair_fs<MASKED, ENERGY>(pi0, li0, jb, ab, (m0 >> sB) & 1u, dx, dy, dz, elj, ec);
        fi0.x = fmaf(-fs, dx, fi0.x); fi0.y = fmaf(-fs, dy, fi0.y); fi0.z = fmaf(-fs, dz, fi0.z);
        fb.x = fmaf(fs, dx, fb.x); fb.y = fmaf(fs, dy, fb.y); fb.z = fmaf(fs, dz, fb.z);
        rot3(fa, nxt);
        rot3(fb, nxt);
    }
    rot3(fa, (lane + 16) & 31);
    fj.x = fa.x + fb.x;
    fj.y = fa.y + fb.y;
    fj.z = fa.z + fb.z;
}

// Pairs inside one tile: every ordered pair, i-force only, energy counted twice.
template <bool ENERGY>
__device__ __forceinline__ void item_self(const float4 *sj, const float2 *sab, const float4 &pi0, const float2 &li0,
                                          uint32_t m0, int lane, float3 &fi0, float &elj, float &ec) {
#pragma unroll 4
    for (int k = 1; k < 32; ++k) {
        const int s = (lane + k) & 31;
        float dx, dy, dz;
        const float fs = pair_fs<true, ENERGY>(pi0, li0, sj[s], sab[s], (m0 >> s) & 1u, dx, dy, dz, elj, ec);
        fi0.x = fmaf(-fs, dx, fi0.x); fi0.y = fmaf(-fs, dy, fi0.y); fi0.z = fmaf(-fs, dz, fi0.z);
    }
}

// Per-warp shared staging of one j-tile.
struct JTile {
    float4 pos[32];
    float2 ab[32];
};

// What a work item reads besides positions: its tiles, exclusion masks and
// LJ parameters (fixed for the lifetime of a context, so a caller that runs
// the same item many times can keep them).
struct ItemCtx {
    int4 item;
    int I0, J;
    bool masked;       // some pair of the item is excluded
    uint32_t m0, m1;   // exclusion masks of this lane's i-atoms (bit j: pair skipped)
    float2 b0, b1, bj; // LJ parameters of this lane's i-atoms and of j-atom J * 32 + lane
};

__device__ __forceinline__ void item_ctx(const PlainDev &p, const int4 &item, int lane, ItemCtx &c) {
    const int T = p.n_tiles;
    c.item = item;
    if (item.x == ITEM_BONDED) {  // no pair work, nothing to read
        c.I0 = c.J = item.y;
        c.masked = false;
        c.m0 = c.m1 = 0u;
        c.b0 = c.b1 = c.bj = make_float2(0.f, 0.f);
        return;
    }
    if (item.x == ITEM_OFF64) {
        c.I0 = 2 * item.y;
        c.J = item.z;
    } else if (item.x == ITEM_OFF32) {
        c.I0 = item.y;
        c.J = item.z;
    } else {
        c.I0 = item.y;
        c.J = item.y;
    }
    const int i0 = c.I0 * kTile + lane;
    c.bj = p.lj[c.J * kTile + lane];
    c.b0 = p.lj[i0];
    c.m0 = c.m1 = 0u;
    c.b1 = make_float2(0.f, 0.f);
    if (item.x == ITEM_SELF) {
        c.masked = true;
        c.m0 = p.tile_mask[tile_pair_index(c.I0, c.I0, T) * kTile + lane];
    } else if (item.x == ITEM_OFF32) {
        const int64_t tp = tile_pair_index(c.I0, c.J, T);
        c.masked = p.tile_flag[tp] != 0u;
        if (c.masked) c.m0 = p.tile_mask[tp * kTile + lane];
    } else {
        c.b1 = p.lj[i0 + kTile];
        const int64_t tp0 = tile_pair_index(c.I0, c.J, T), tp1 = tile_pair_index(c.I0 + 1, c.J, T);
        c.masked = (p.tile_flag[tp0] | p.tile_flag[tp1]) != 0u;
        if (c.masked) {
            c.m0 = p.tile_mask[tp0 * kTile + lane];
            c.m1 = p.tile_mask[tp1 * kTile + lane];
        }
    }
}

// One work item of the all-pairs sum: forces into fx (fixed point), energies
// added to the lane's FP32 accumulators (elj as 24 eps (s^12 - s^6)).
// With fi_out set, a 64x32 item returns its two i-forces there (fi_out[0],
// fi_out[1]) instead of adding them.
template <bool ENERGY>
__device__ __forceinline__ void item_eval(const PlainDev &p, const ItemCtx &c, int lane, JTile &jt,
                                          unsigned long long *fx, float &elj, float &ec, bool &bad,
                                          float3 *fi_out = nullptr) {
    if (c.item.x == ITEM_BONDED) return;
    const int i0 = c.I0 * kTile + lane, j = c.J * kTile + lane;
    __syncwarp();
    jt.pos[lane] = p.pos4[j];
    jt.ab[lane] = c.bj;
    __syncwarp();
    float3 fi0 = make_float3(0.f, 0.f, 0.f), fj = make_float3(0.f, 0.f, 0.f);
    float el = 0.f, eq = 0.f;
    if (c.item.x == ITEM_SELF) {
        item_self<ENERGY>(jt.pos, jt.ab, jt.pos[lane], jt.ab[lane], c.m0, lane, fi0, el, eq);
        el *= 0.5f;
        eq *= 0.5f;
    } else if (c.item.x == ITEM_OFF32) {
        const float4 a0 = p.pos4[i0];
        if (c.masked)
            item_off32<true, ENERGY>(jt.pos, jt.ab, a0, c.b0, c.m0, lane, fi0, fj, el, eq);
        else
            item_off32<false, ENERGY>(jt.pos, jt.ab, a0, c.b0, 0u, lane, fi0, fj, el, eq);
    } else {
        const int i1 = i0 + kTile;
        const float4 a0 = p.pos4[i0], a1 = p.pos4[i1];
        float3 fi1 = make_float3(0.f, 0.f, 0.f);
        if (c.masked)
            item_off64<true, ENERGY>(jt.pos, jt.ab, a0, c.b0, a1, c.b1, c.m0, c.m1, lane, fi0, fi1, fj, el, eq);
        else
            item_off64<false, ENERGY>(jt.pos, jt.ab, a0, c.b0, a1, c.b1, 0u, 0u, lane, fi0, fi1, fj, el, eq);
        if (fi_out != nullptr) {
            fi_out[1] = fi1;
        } else {
            fx_add(&fx[3 * i1 + 0], fi1.x);
            fx_add(&fx[3 * i1 + 1], fi1.y);
            fx_add(&fx[3 * i1 + 2], fi1.z);
        }
        bad |= !isfinite(fi1.x + fi1.y + fi1.z);
    }
    if (c.item.x != ITEM_SELF) {
        fx_add(&fx[3 * j + 0], fj.x);
        fx_add(&fx[3 * j + 1], fj.y);
        fx_add(&fx[3 * j + 2], fj.z);
    }
    if (fi_out != nullptr && c.item.x == ITEM_OFF64) {
        fi_out[0] = fi0;
    } else {
        fx_add(&fx[3 * i0 + 0], fi0.x);
        fx_add(&fx[3 * i0 + 1], fi0.y);
        fx_add(&fx[3 * i0 + 2], fi0.z);
    }
    bad |= !isfinite(fi0.x + fi0.y + fi0.z + fj.x + fj.y + fj.z + el + eq);
    if (ENERGY) {
        elj += el;
        ec += eq;
    }
}

template <bool ENERGY>
__device__ __forceinline__ void nonbonded_item(const PlainDev &p, int it, int lane, JTile &jt,
                                               unsigned long long *fx, float &elj, float &ec, bool &bad) {
    ItemCtx c;
    item_ctx(p, p.items[it], lane, c);
    item_eval<ENERGY>(p, c, lane, jt, fx, elj, ec, bad);
}

// ------------------------------------------------------------------ row decomposition
//
// The all-pairs sum of the context's kernels (the kernel-sequence all-pairs
// kernel and the persistent stepper) is computed row by row: the force on
// atom i is the sum over every j, each pair evaluated from both sides, so no
// force ever crosses from one row's owner to another's and the stepper can
// integrate a row as soon as its own sums are in.  Twice the pair arithmetic
// of a Newton-pair sum, but no j-force shuffles, no scattered adds and one
// grid barrier per MD step instead of two.
//
// A row group is 16 consecutive atoms; a chunk is 32 consecutive j-atoms.  A
// group's j-range is cut into kSlices slices, slice s holding the chunks
// s, s + kSlices, ...; one warp evaluates one (group, slice) task.  Lane
// (iq = lane / 8, q = lane % 8) owns the four i-atoms 16 g + 4 iq + (0..3)
// and meets j = 32 c + 8 k + q (k = 0..3) of every chunk c of the slice, so
// each j read serves four pairs.  The lane sums its pair forces in FP32 in
// that order (chunks ascending, k ascending); the eight q-lanes of an atom
// quad then add their sums by a butterfly (FP32 addition commutes, so all
// eight get the same bits), and the (atom, slice) sum is rounded to fixed
// point.  The force on an atom is the integer sum over slices of those values
// plus its bonded terms, so it does not depend on which kernel, warp or block
// evaluated a task: both steppers produce the same forces bit for bit.
//
// Skipped pairs (the atom itself, its 1-2 and 1-3 partners, padding atoms on
// either side) are bits of a dense mask: word a of (g, c) holds bit l for the
// pair (16 g + a, 32 c + l).  A chunk whose masks are all zero for the warp
// takes the unmasked loop.
constexpr int kRowGroup = 16;   // i-atoms per row group
constexpr int kSlices = 16;     // j-slices per group (one warp each)

// One j-chunk staged in shared memory by its warp.
struct RowStage {
    float4 pos[32];
    float2 lj[32];
};

// The lane's four i-atoms: positions, LJ parameters and force sums.
struct RowQuad {
    float4 p[4];
    float2 l[4];
    float3 f[4];
};

// The 16 pairs of one chunk for a lane: its four i-atoms against
// j = 8 k + q of the staged chunk; m[a] is the skip mask of i-atom a already
// shifted right by q (bit 8 k: pair with j-lane 8 k + q skipped).
template <bool MASKED, bool ENERGY>
__device__ __forceinline__ void chunk_pairs(const RowStage &st, int q, RowQuad &r, const uint4 &m, float &elj,
                                            float &ec) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 pj = st.pos[8 * k + q];
        const float2 bj = st.lj[8 * k + q];
        const uint32_t mk[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            float dx, dy, dz;
            const float fs = pair_fs<MASKED, ENERGY>(r.p[a], r.l[a], pj, bj, (mk[a] >> (8 * k)) & 1u, dx, dy, dz,
                                                     elj, ec);
            r.f[a].x = fmaf(-fs, dx, r.f[a].x);
            r.f[a].y = fmaf(-fs, dy, r.f[a].y);
            r.f[a].z = fmaf(-fs, dz, r.f[a].z);
        }
    }
}

// Task (g, s) for one warp: the lane's four FP32 row sums over the slice's
// chunks, after the q-butterfly (the same value in the eight q-lanes of an
// atom quad).  Energies (elj as 24 eps (s^12 - s^6), ec) are added to the
// lane's accumulators with every pair counted from both of its atoms.
template <bool ENERGY, typename Mid>
__device__ __forceinline__ void row_task(const PlainDev &p, const float4 *__restrict__ pos4, int g, int s, int lane,
                                         RowStage &st, RowQuad &r, float &elj, float &ec, Mid mid) {
    const int iq = lane >> 3, q = lane & 7;
    const int i0 = g * kRowGroup + 4 * iq;
    const int C = p.n_chunks;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        r.p[a] = pos4[i0 + a];
        r.l[a] = p.lj[i0 + a];
        r.f[a] = make_float3(0.f, 0.f, 0.f);
    }
    const uint4 *mrow = reinterpret_cast<const uint4 *>(p.row_mask + (size_t)g * C * kRowGroup) + iq;
    int c = s;
    float4 npos = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 nlj = make_float2(0.f, 0.f);
    uint4 nm = make_uint4(0u, 0u, 0u, 0u);
    if (c < C) {
        npos = pos4[32 * c + lane];
        nlj = p.lj[32 * c + lane];
        nm = mrow[(size_t)c * (kRowGroup / 4)];
    }
    mid();   // the caller's work that overlaps these first loads
    for (; c < C; c += kSlices) {
        __syncwarp();
        st.pos[lane] = npos;
        st.lj[lane] = nlj;
        const uint4 m = make_uint4(nm.x >> q, nm.y >> q, nm.z >> q, nm.w >> q);
        const bool any = (nm.x | nm.y | nm.z | nm.w) != 0u;
        const int cn = c + kSlices;
        if (cn < C) {   // prefetch the next chunk of the slice while this one is evaluated
            npos = pos4[32 * cn + lane];
            nlj = p.lj[32 * cn + lane];
            nm = mrow[(size_t)cn * (kRowGroup / 4)];
        }
        __syncwarp();
        if (__any_sync(0xffffffffu, any))
            chunk_pairs<true, ENERGY>(st, q, r, m, elj, ec);
        else
            chunk_pairs<false, ENERGY>(st, q, r, make_uint4(0u, 0u, 0u, 0u), elj, ec);
    }
#pragma unroll
    for (int o = 1; o <= 4; o <<= 1) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            r.f[a].x += __shfl_xor_sync(0xffffffffu, r.f[a].x, o);
            r.f[a].y += __shfl_xor_sync(0xffffffffu, r.f[a].y, o);
            r.f[a].z += __shfl_xor_sync(0xffffffffu, r.f[a].z, o);
        }
    }
}

// The fixed-point values a lane emits after row_task: the twelve (atom,
// component) sums of its atom quad, v = 3 a + component, are spread over the
// eight q-lanes: value q and (q < 4) value q + 8.  slot = 3 * (local atom) +
// component = 12 iq + v, local atom in [0, 16); slot_b < 0: none.
struct RowEmit {
    int slot_a, slot_b;
    long long va, vb;
};

__device__ __forceinline__ float quad_value(const RowQuad &r, int v) {
    // v in [0, 12): component v % 3 of atom v / 3, by selects (no local memory)
    float out = r.f[0].x;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        out = v == 3 * a + 0 ? r.f[a].x : out;
        out = v == 3 * a + 1 ? r.f[a].y : out;
        out = v == 3 * a + 2 ? r.f[a].z : out;
    }
    return out;
}

__device__ __forceinline__ RowEmit row_emit(int lane, const RowQuad &r) {
    const int iq = lane >> 3, q = lane & 7;
    RowEmit e;
    e.slot_a = 12 * iq + q;
    e.va = fx_from_float(quad_value(r, q));
    e.slot_b = q < 4 ? 12 * iq + 8 + q : -1;
    e.vb = q < 4 ? fx_from_float(quad_value(r, q + 8)) : 0;
    return e;
}

__device__ __forceinline__ bool quad_finite(const RowQuad &r) {
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) s += r.f[a].x + r.f[a].y + r.f[a].z;
    return isfinite(s);
}

// One entry of a row group's bonded list, with the positions it reads.
struct BondEntry {
    int4 rec;      // bonded_rec of the term
    float2 par;    // bond parameters (bonds)
    int slot;      // 3 * local atom (the atom this entry belongs to)
    int role;      // 0, 1, 2: the atom is rec.x, rec.y, rec.z; role 0 also counts the term's energy
};

__device__ __forceinline__ BondEntry bond_entry(const PlainDev &p, int e) {
    const int2 en = p.grp_ent[e];
    BondEntry b;
    b.rec = bonded_rec(p, en.x);
    b.par = b.rec.z < 0 ? p.bond_par[b.rec.w] : make_float2(0.f, 0.f);
    b.slot = 3 * (en.y >> 2);
    b.role = en.y & 3;
    return b;
}

__device__ __forceinline__ void bond_gather(const BondEntry &b, const float4 *pos4, BondedGeom &g) {
    g.xa = pos4[b.rec.x];
    g.xb = pos4[b.rec.y];
    g.xc = b.rec.z >= 0 ? pos4[b.rec.z] : make_float4(0.f, 0.f, 0.f, 0.f);
    g.par = b.par;
}

// The force of an entry's term on the entry's atom, and the term's energy
// when the entry has role 0 (eb for a bond, ea for an angle).
__device__ __forceinline__ float3 bond_entry_force(const PlainDev &p, const BondEntry &b, const BondedGeom &g,
                                                   float &eb, float &ea) {
    float3 fa, fb, fc;
    float e;
    bonded_forces(p, b.rec, g, fa, fb, fc, e);
    if (b.role == 0) {
        if (b.rec.z < 0) eb += e;
        else ea += e;
    }
    return b.role == 0 ? fa : (b.role == 1 ? fb : fc);
}

}  // namespace mdpf
