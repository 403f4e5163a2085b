// Persistent velocity-Verlet stepper for the plain force field.
//
// One cooperative launch runs all n steps of mdpf_step; the kernel never
// returns to the host between steps (the paper's timing table shows that for
// small systems launch overhead, not arithmetic, decides the step time; CUDA
// graphs were its remedy, a single resident kernel is the one used here).
//
// Each MD step costs two grid barriers:
//   forces       every warp evaluates its all-pairs work items at x_{s+1}
//                (FP32 copy P[s & 1]) and adds the forces into buffer
//                buf(s) (int64 fixed point).  The bonded terms a tile owns
//                (bond: first atom; angle: vertex) go with the tile's items
//                on the diagonal, the shortest ones: the first kSelfBonded
//                with its self item, the next kPairBonded with the 32x32 item
//                of its pair of tiles, the rest with a bonded-only item.
//                A block whose eight 64x32 items share their i-tiles sums
//                those i-forces in shared memory (as integers) and sends one
//                add per atom and component.  A warp keeps what its first
//                item reads besides positions (tiles, masks, LJ parameters,
//                bonded records) in registers for the whole launch.
//   grid barrier
//   integration  tile t by warp t / G of block t % G (one tile per SM while
//                the tiles fit), because FP64 throughput is the limit here;
//                the warp keeps its first tile's x, v in registers:
//                  v_{s+1} = v_{s+1/2} + dt/2 a          (end of step s, K)
//                  v_{s+3/2} = v_{s+1} + dt/2 a; x_{s+2} = x_{s+1} + dt v
//                  FP32 copy of x_{s+2} into P[(s + 1) & 1]  (start of step s+1)
//   grid barrier
// A pre-phase performs the first half-kick and drift from the forces left in
// the state buffer by mdpf_set_state or by the previous launch; the last step
// writes F(x_n) back there instead.
//
// Forces are integer sums of the same FP32 terms the kernel-sequence stepper
// adds, and every state update is an explicit FMA (v = fma(h, f, v),
// x = fma(dt, v, x)) in both, so both steppers produce the same trajectory bit
// for bit; energies are
// summed in a fixed order (pair and bonded energies per block in block order,
// kinetic energy per tile in tile order), so they are reproducible too.
//
// The grid barrier is a 64-bit arrival counter (release add, acquire poll)
// that waits at most limit_ns; on time-out the block records
// MDPF_STATUS_TIMEOUT and returns, and the others follow at their next
// barrier.  Co-residency of all blocks is guaranteed by the cooperative launch.
#include "forcefield.cuh"

namespace mdpf {

struct StepArgs {
    PlainDev p;
    int n, n_tiles;
    double dt;
    const double *hdt_m;          // dt/2 * kAcc / m
    const double *mass;
    const float *qs;
    float4 *P0, *P1;              // FP32 position buffers (x, y, z, q sqrt(ke))
    double *x, *v;
    unsigned long long *fxA;      // state forces F(x) on entry and exit; accumulator of odd steps
    unsigned long long *fxB;      // accumulator of even steps
    const int *own_off, *own;     // bonded terms owned by each tile (CSR over tiles)
    double *part;                 // [2][grid][4] per-block energies (bond, angle, LJ, Coulomb)
    double *tile_e;               // [2][T][4] per-tile kinetic energy (slot 2)
    double *trace_u, *trace_k;
    int64_t *trace_step;
    int trace_cap;
    int energy_every;
    int64_t *step;
    uint32_t *status;
    double *scalars;
    Frames frames;
    int record_every;
    unsigned long long *bar;      // arrival counter
    int64_t n_steps;
    long long limit_ns;
};

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long atom_add_release(unsigned long long *p, unsigned long long v) {
    unsigned long long old;
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier number `epoch` (1, 2, ...).  Returns false in every
// thread of the block if this block gave up waiting.
__device__ __forceinline__ bool grid_barrier(unsigned long long *bar, unsigned long long epoch, uint32_t *status,
                                             long long limit_ns, int *s_fail) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int fail = 0;
        if (gridDim.x > 1) {
            const unsigned long long target = epoch * gridDim.x;
            atom_add_release(bar, 1ull);
            const unsigned long long t0 = globaltimer();
            unsigned int spins = 0;
            while (ld_acquire(bar) < target) {
                if ((++spins & 31u) == 0u && (long long)(globaltimer() - t0) > limit_ns) {
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

constexpr int kStepThreads = 256;
constexpr int kStepWarps = kStepThreads / 32;
constexpr int kSelfBonded = 16;  // bonded terms of a tile evaluated with its self item ...
constexpr int kPairBonded = 0;   // ... with the 32x32 item of its pair of tiles; the rest with its bonded item
constexpr int kBondRegs = 4;     // bonded terms per lane whose records a warp keeps in registers

// Integration state of one atom (one lane).  A warp keeps the state of the
// first tile it integrates in registers for the whole launch and writes x, v
// back only on energy steps (where the status is checked and the launch may
// stop) and at the last step; further tiles go through memory.
struct AtomState {
    double x[3], v[3], h, m;
    float q;
};

__device__ __forceinline__ void load_state(const StepArgs &a, int at, AtomState &st) {
    if (at < a.n) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            st.x[q] = __ldcg(&a.x[3 * at + q]);
            st.v[q] = __ldcg(&a.v[3 * at + q]);
        }
        st.h = a.hdt_m[at];
        st.m = a.mass[at];
        st.q = a.qs[at];
    }
}

// Integration of tile t (one atom per lane) after all forces of the step are in.
__device__ __forceinline__ void integrate_tile(const StepArgs &a, int t, int64_t s, float4 *Pnext,
                                               unsigned long long *acc, bool energy, bool rec, int slot,
                                               AtomState &st, bool store) {
    const int lane = threadIdx.x & 31;
    const int at = t * kTile + lane;
    double kin = 0.0;
    const bool last = s + 1 == a.n_steps;
    if (at < a.n) {
        const double h = st.h;
        unsigned long long fi[3];
        double f[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) fi[q] = __ldcg(&acc[3 * at + q]);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            f[q] = fx_val(fi[q]);
            st.v[q] = fma(h, f[q], st.v[q]);  // v_{s+1}
            kin += st.v[q] * st.v[q];
        }
        kin *= 0.5 * st.m / kAcc;
        if (rec) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                a.frames.pos[((size_t)slot * a.n + at) * 3 + q] = st.x[q];
                a.frames.forces[((size_t)slot * a.n + at) * 3 + q] = (float)f[q];
            }
        }
        if (!last) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                st.v[q] = fma(h, f[q], st.v[q]);
                st.x[q] = fma(a.dt, st.v[q], st.x[q]);
                acc[3 * at + q] = 0ull;
            }
            Pnext[at] = make_float4((float)st.x[0], (float)st.x[1], (float)st.x[2], st.q);
        } else {
            // leave F(x_n) in the state buffer for the next launch
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                acc[3 * at + q] = 0ull;
                a.fxA[3 * at + q] = fi[q];
            }
        }
        if (store || last) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                a.x[3 * at + q] = st.x[q];
                a.v[3 * at + q] = st.v[q];
            }
        }
        if (!isfinite(kin)) atomicOr(a.status, MDPF_STATUS_NONFINITE);
    } else if (at < a.p.n_pad) {
        acc[3 * at] = acc[3 * at + 1] = acc[3 * at + 2] = 0ull;
    }
    if (energy) {
        const double sk = warp_sum_d(kin);
        if (lane == 0) a.tile_e[((size_t)(s & 1) * a.n_tiles + t) * 4 + 2] = sk;
    }
}

// The bonded terms that go with a work item, as up to two ranges of the
// owner lists: a self item takes the first kSelfBonded terms of its tile, the
// 32x32 item of a diagonal pair the next kPairBonded of both tiles, and the
// tile's bonded item the rest (the shares follow each item's pair work).
struct BondedList {
    int a0, na, b0, nb;
    __device__ __forceinline__ int size() const { return na + nb; }
    __device__ __forceinline__ int at(const int *own, int e) const { return e < na ? own[a0 + e] : own[b0 + e - na]; }
};

__device__ __forceinline__ BondedList bonded_list(const StepArgs &a, const int4 &item) {
    BondedList l{0, 0, 0, 0};
    if (item.x == ITEM_SELF) {
        l.a0 = a.own_off[item.y];
        l.na = min(a.own_off[item.y + 1] - l.a0, kSelfBonded);
    } else if (item.x == ITEM_OFF32) {
        l.a0 = a.own_off[item.y] + kSelfBonded;
        l.na = min(max(a.own_off[item.y + 1] - l.a0, 0), kPairBonded);
        l.b0 = a.own_off[item.z] + kSelfBonded;
        l.nb = min(max(a.own_off[item.z + 1] - l.b0, 0), kPairBonded);
    } else if (item.x == ITEM_BONDED) {
        l.a0 = a.own_off[item.y] + kSelfBonded + kPairBonded;
        l.na = max(a.own_off[item.y + 1] - l.a0, 0);
    }
    return l;
}

__global__ void __launch_bounds__(kStepThreads, 1) k_plain_persistent(StepArgs a) {
    __shared__ JTile jt[kStepWarps];
    __shared__ double red[kStepWarps][4];
    __shared__ long long ired[kStepWarps][6][kTile];  // the block's i-forces (fixed point) before one add
    __shared__ int s_uniform;
    __shared__ int s_fail;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    const int gwarp = gtid >> 5;
    const int nwarps = nthreads >> 5;
    const int64_t step0 = *a.step;
    unsigned long long epoch = 0;

    // ---- pre-phase: v_{1/2} = v_0 + dt/2 a(x_0); x_1 = x_0 + dt v_{1/2}; clear both accumulators
    for (int at = gtid; at < a.p.n_pad; at += nthreads) {
        if (at < a.n) {
            const double h = a.hdt_m[at];
            double x[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const double f = fx_val(a.fxA[3 * at + q]);
                const double v = fma(h, f, a.v[3 * at + q]);
                x[q] = fma(a.dt, v, a.x[3 * at + q]);
                a.v[3 * at + q] = v;
                a.x[3 * at + q] = x[q];
            }
            a.P0[at] = make_float4((float)x[0], (float)x[1], (float)x[2], a.qs[at]);
        } else {
            a.P0[at] = make_float4(0.f, 0.f, 0.f, 0.f);
            a.P1[at] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            a.fxA[3 * at + q] = 0ull;
            a.fxB[3 * at + q] = 0ull;
        }
    }
    if (!grid_barrier(a.bar, ++epoch, a.status, a.limit_ns, &s_fail)) return;
    // integration: tile t by warp t / G of block t % G (G blocks), one tile per SM while T <= G
    const int t_own = blockIdx.x + gridDim.x * w;
    AtomState own;
    if (t_own < a.n_tiles) load_state(a, t_own * kTile + lane, own);
    // the warp's first work item (its only one unless there are more items than warps): tiles, masks and LJ
    // parameters stay in registers, so a step loads only positions for it
    // A block whose eight warps each have one 64x32 item on the same pair of i-tiles (the usual case: the
    // items of a pair of i-tiles are listed together) adds their i-forces in shared memory as integers and
    // sends one fixed-point add per atom and component instead of eight.
    if (threadIdx.x == 0) {
        int u = (long long)nwarps >= a.p.n_items && (blockIdx.x + 1) * kStepWarps <= a.p.n_items;
        if (u) {
            const int4 i0 = a.p.items[blockIdx.x * kStepWarps];
            for (int k = 0; k < kStepWarps && u; ++k) {
                const int4 ik = a.p.items[blockIdx.x * kStepWarps + k];
                u = ik.x == ITEM_OFF64 && ik.y == i0.y;
            }
        }
        s_uniform = u;
    }
    __syncthreads();
    const bool uniform = s_uniform != 0;
    // Work items: warp w takes the contiguous run [w * per, (w + 1) * per), so that consecutive 64x32 items of
    // a warp share their i-tiles when there are more items than warps; the warp then sums those i-forces as
    // integers in registers and sends them once per run of equal i-tiles.
    const int per = (a.p.n_items + nwarps - 1) / nwarps;
    const int it_first = gwarp * per, it_end = min(it_first + per, a.p.n_items);
    ItemCtx first;
    BondedList first_bl{0, 0, 0, 0};
    int4 brec[kBondRegs];    // records of the first item's bonded terms lane, lane + 32, ...
    float2 bpar[kBondRegs];  // and their bond parameters
    if (it_first < a.p.n_items) {
        item_ctx(a.p, a.p.items[it_first], lane, first);
        first_bl = bonded_list(a, first.item);
#pragma unroll
        for (int k = 0; k < kBondRegs; ++k) {
            const int e = lane + 32 * k;
            if (e < first_bl.size()) {
                brec[k] = bonded_rec(a.p, first_bl.at(a.own, e));
                bpar[k] = brec[k].z < 0 ? a.p.bond_par[brec[k].w] : make_float2(0.f, 0.f);
            }
        }
    }

    for (int64_t s = 0; s < a.n_steps; ++s) {
        const float4 *Pcur = (s & 1) ? a.P1 : a.P0;
        float4 *Pnext = (s & 1) ? a.P0 : a.P1;
        unsigned long long *acc = (s & 1) ? a.fxA : a.fxB;
        const int64_t done = step0 + s + 1;  // steps completed after this iteration
        const bool energy = done % a.energy_every == 0;
        const bool rec = a.record_every > 0 && done % a.record_every == 0;
        const int slot = rec ? (int)((done / a.record_every - 1) % a.frames.cap) : 0;
        PlainDev p = a.p;
        p.pos4 = Pcur;
        float elj = 0.f, ec = 0.f, eb = 0.f, ea = 0.f;
        bool bad = false;
        int run_p = -1;         // i-tile pair of the current run of 64x32 items
        long long run_f[6] = {0, 0, 0, 0, 0, 0};  // its i-forces (fixed point), atoms 64 run_p + lane (+ 32)
        auto flush_run = [&]() {
            if (run_p < 0) return;
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    atomicAdd(&acc[3 * ((2 * run_p + h) * kTile + lane) + q], (unsigned long long)run_f[3 * h + q]);
        };
        for (int it = it_first; it < it_end; ++it) {
            ItemCtx later;
            if (it != it_first) item_ctx(p, p.items[it], lane, later);
            const ItemCtx &c = it == it_first ? first : later;
            float3 fio[2];
            if (energy)
                item_eval<true>(p, c, lane, jt[w], acc, elj, ec, bad, fio);
            else
                item_eval<false>(p, c, lane, jt[w], acc, elj, ec, bad, fio);
            if (c.item.x == ITEM_OFF64 && !uniform) {
                if (c.item.y != run_p) {
                    flush_run();
                    run_p = c.item.y;
#pragma unroll
                    for (int k = 0; k < 6; ++k) run_f[k] = 0;
                }
                run_f[0] += fx_from_float(fio[0].x);
                run_f[1] += fx_from_float(fio[0].y);
                run_f[2] += fx_from_float(fio[0].z);
                run_f[3] += fx_from_float(fio[1].x);
                run_f[4] += fx_from_float(fio[1].y);
                run_f[5] += fx_from_float(fio[1].z);
            }
            if (uniform) {
                ired[w][0][lane] = fx_from_float(fio[0].x);
                ired[w][1][lane] = fx_from_float(fio[0].y);
                ired[w][2][lane] = fx_from_float(fio[0].z);
                ired[w][3][lane] = fx_from_float(fio[1].x);
                ired[w][4][lane] = fx_from_float(fio[1].y);
                ired[w][5][lane] = fx_from_float(fio[1].z);
                __syncthreads();
                // thread k < 192: atom k % 64 of the tile pair, component k / 64
                if (threadIdx.x < 6 * kTile) {
                    const int q = threadIdx.x / (2 * kTile), at = threadIdx.x % (2 * kTile);
                    const int slot = (at / kTile) * 3 + q, l = at % kTile;
                    long long sum = 0;
#pragma unroll
                    for (int k = 0; k < kStepWarps; ++k) sum += ired[k][slot][l];
                    atomicAdd(&acc[3 * (2 * c.item.y * kTile + at) + q], (unsigned long long)sum);
                }
                __syncthreads();
            }
            // bonded terms: shares of the tile's list by item type (bonded_list)
            const int4 item = c.item;
            if (item.x != ITEM_OFF64) {
                int e0 = 0;
                BondedList bl = first_bl;
                if (it == it_first) {
                    // records in registers: every position load is issued before the first evaluation
                    BondedGeom g[kBondRegs];
#pragma unroll
                    for (int k = 0; k < kBondRegs; ++k)
                        if (lane + 32 * k < bl.size()) {
                            g[k].xa = p.pos4[brec[k].x];
                            g[k].xb = p.pos4[brec[k].y];
                            g[k].xc = brec[k].z >= 0 ? p.pos4[brec[k].z] : make_float4(0.f, 0.f, 0.f, 0.f);
                            g[k].par = bpar[k];
                        }
#pragma unroll
                    for (int k = 0; k < kBondRegs; ++k)
                        if (lane + 32 * k < bl.size()) bonded_eval(p, brec[k], g[k], acc, eb, ea);
                    e0 = 32 * kBondRegs;
                } else {
                    bl = bonded_list(a, item);
                }
                for (int e = e0 + lane; e < bl.size(); e += 32) bonded_term(p, bl.at(a.own, e), acc, eb, ea);
            }
        }
        flush_run();
        bad |= !isfinite(eb + ea);
        if (bad) atomicOr(a.status, MDPF_STATUS_NONFINITE);
        if (energy) {
            double v4[4] = {warp_sum_d((double)eb), warp_sum_d((double)ea), warp_sum_d((double)elj * (1.0 / 6.0)),
                            warp_sum_d((double)ec)};
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < 4; ++k) red[w][k] = v4[k];
            __syncthreads();
            if (threadIdx.x < 4) {
                double sum = 0.0;
                for (int q = 0; q < kStepWarps; ++q) sum += red[q][threadIdx.x];
                a.part[((size_t)(s & 1) * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = sum;
            }
        }
        if (!grid_barrier(a.bar, ++epoch, a.status, a.limit_ns, &s_fail)) return;
        if (t_own < a.n_tiles) integrate_tile(a, t_own, s, Pnext, acc, energy, rec, slot, own, energy);
        for (int t = t_own + gridDim.x * kStepWarps; t < a.n_tiles; t += gridDim.x * kStepWarps) {
            AtomState st;
            load_state(a, t * kTile + lane, st);
            integrate_tile(a, t, s, Pnext, acc, energy, rec, slot, st, true);
        }
        if (!grid_barrier(a.bar, ++epoch, a.status, a.limit_ns, &s_fail)) return;
        // ---- energies of step `done` (block 0, warp 0), read after the barrier
        if (energy && blockIdx.x == 0 && w == 0) {
            const double *pp = a.part + (size_t)(s & 1) * gridDim.x * 4;
            const double *te = a.tile_e + (size_t)(s & 1) * a.n_tiles * 4;
            double sl = 0, sc = 0, sb = 0, sa = 0, sk = 0;
            for (int b = lane; b < (int)gridDim.x; b += 32) {
                sb += pp[4 * b];
                sa += pp[4 * b + 1];
                sl += pp[4 * b + 2];
                sc += pp[4 * b + 3];
            }
            for (int t = lane; t < a.n_tiles; t += 32) sk += te[4 * t + 2];
            sl = warp_sum_d(sl);
            sc = warp_sum_d(sc);
            sb = warp_sum_d(sb);
            sa = warp_sum_d(sa);
            sk = warp_sum_d(sk);
            if (lane == 0) {
                const double U = sb + sa + sl + sc;
                const int64_t e = done / a.energy_every - 1;
                a.trace_u[e % a.trace_cap] = U;
                a.trace_k[e % a.trace_cap] = sk;
                a.trace_step[e % a.trace_cap] = done;
                a.scalars[0] = U;
                a.scalars[1] = sk;
                if (!isfinite(U) || !isfinite(sk)) atomicOr(a.status, MDPF_STATUS_NONFINITE);
                if (rec) {
                    a.frames.energy[slot] = U;
                    a.frames.step[slot] = done;
                }
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0 && s + 1 == a.n_steps) *a.step = done;
        // every block reads the status after the same barrier, so all stop together
        if (energy && *(volatile uint32_t *)a.status != 0u) {
            if (blockIdx.x == 0 && threadIdx.x == 0) *a.step = done;
            return;
        }
    }
}

int stepper_grid(const mdpf_ctx *ctx) {
    int dev = ctx->device, sms = 0, occ = 0, coop = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_plain_persistent, kStepThreads, 0) != cudaSuccess)
        return 0;
    if (occ < 1) return 0;
    int want = (ctx->n_items + kStepWarps - 1) / kStepWarps;
    if (want < 1) want = 1;
    return want < sms ? want : sms;  // one block per SM keeps one barrier arrival per SM
}

cudaError_t launch_plain_persistent(mdpf_ctx *ctx, int64_t n_steps, cudaStream_t s) {
    StepArgs a;
    a.p = plain_dev(ctx, ctx->d_pos4);
    a.n = ctx->n;
    a.n_tiles = ctx->n_tiles;
    a.dt = ctx->dt;
    a.hdt_m = ctx->d_hdt_m;
    a.mass = ctx->d_mass;
    a.qs = ctx->d_charge_s;
    a.P0 = ctx->d_pos4;
    a.P1 = ctx->d_pos4_b;
    a.x = ctx->d_x;
    a.v = ctx->d_v;
    a.fxA = ctx->d_fx_base;
    a.fxB = ctx->d_fx_base + 3 * (size_t)ctx->n_pad;
    a.own_off = ctx->d_own_off;
    a.own = ctx->d_own;
    a.part = ctx->d_part;
    a.tile_e = ctx->d_tile_e;
    a.trace_u = ctx->d_trace_u;
    a.trace_k = ctx->d_trace_k;
    a.trace_step = ctx->d_trace_step;
    a.trace_cap = ctx->trace_cap;
    a.energy_every = ctx->energy_every;
    a.step = ctx->d_step;
    a.status = ctx->d_status;
    a.scalars = ctx->d_scalar;
    a.frames = ctx->frames;
    a.record_every = ctx->frames.cap > 0 ? ctx->record_every : 0;
    a.bar = reinterpret_cast<unsigned long long *>(ctx->d_barrier);
    a.n_steps = n_steps;
    a.limit_ns = 1000000000LL;  // 1 s per barrier wait
    cudaError_t e = cudaMemsetAsync(ctx->d_barrier, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    void *args[] = {&a};
    return cudaLaunchCooperativeKernel((const void *)k_plain_persistent, dim3(ctx->step_grid), dim3(kStepThreads),
                                       args, 0, s);
}

}  // namespace mdpf
