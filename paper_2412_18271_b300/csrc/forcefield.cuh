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

__device__ __forceinline__ void bonded_eval(const PlainDev &p, const int4 &r, const BondedGeom &g,
                                            unsigned long long *fx, float &eb, float &ea) {
    if (r.z < 0) {
        const float4 xi = g.xa, xj = g.xb;
        const float2 par = g.par;
        float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        float rr = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        float dr = rr - par.x;
        eb += 0.5f * par.y * dr * dr;
        float gg = par.y * dr / rr;
        fx_add(&fx[3 * r.x + 0], gg * dx);
        fx_add(&fx[3 * r.x + 1], gg * dy);
        fx_add(&fx[3 * r.x + 2], gg * dz);
        fx_add(&fx[3 * r.y + 0], -gg * dx);
        fx_add(&fx[3 * r.y + 1], -gg * dy);
        fx_add(&fx[3 * r.y + 2], -gg * dz);
    } else {
        const float4 xa = g.xa, xv = g.xb, xb = g.xc;
        float ux = xa.x - xv.x, uy = xa.y - xv.y, uz = xa.z - xv.z;
        float wx = xb.x - xv.x, wy = xb.y - xv.y, wz = xb.z - xv.z;
        float ru = sqrtf(fmaf(ux, ux, fmaf(uy, uy, uz * uz))), rw = sqrtf(fmaf(wx, wx, fmaf(wy, wy, wz * wz)));
        float c = fmaf(ux, wx, fmaf(uy, wy, uz * wz));
        float cx = fmaf(uy, wz, -uz * wy), cy = fmaf(uz, wx, -ux * wz), cz = fmaf(ux, wy, -uy * wx);
        float cr = sqrtf(fmaf(cx, cx, fmaf(cy, cy, cz * cz)));
        float th = atan2f(cr, c);
        float dth = th - p.angle_theta0;
        ea += 0.5f * p.angle_k * dth * dth;
        float cs = c / (ru * rw);
        float sn = cr / (ru * rw);
        // F_a = k dth / (sin |u|) (w^ - cos u^),  F_b = k dth / (sin |w|) (u^ - cos w^)
        float ga = p.angle_k * dth / (sn * ru);
        float gb = p.angle_k * dth / (sn * rw);
        float iu = 1.f / ru, iw = 1.f / rw;
        float fax = ga * (wx * iw - cs * ux * iu), fay = ga * (wy * iw - cs * uy * iu), faz = ga * (wz * iw - cs * uz * iu);
        float fbx = gb * (ux * iu - cs * wx * iw), fby = gb * (uy * iu - cs * wy * iw), fbz = gb * (uz * iu - cs * wz * iw);
        fx_add(&fx[3 * r.x + 0], fax);
        fx_add(&fx[3 * r.x + 1], fay);
        fx_add(&fx[3 * r.x + 2], faz);
        fx_add(&fx[3 * r.z + 0], fbx);
        fx_add(&fx[3 * r.z + 1], fby);
        fx_add(&fx[3 * r.z + 2], fbz);
        fx_add(&fx[3 * r.y + 0], -(fax + fbx));
        fx_add(&fx[3 * r.y + 1], -(fay + fby));
        fx_add(&fx[3 * r.y + 2], -(faz + fbz));
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
    const float rinv = rsqrtf(r2);
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

}  // namespace mdpf
