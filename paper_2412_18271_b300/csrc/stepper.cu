// Persistent velocity-Verlet stepper for the plain force field.
//
// One cooperative launch runs all n steps of mdpf_step; the kernel never
// returns to the host between steps (the paper's timing table shows that for
// small systems launch overhead, not arithmetic, decides the step time; CUDA
// graphs were its remedy, a single resident kernel is the one used here).
//
// Block b owns the row groups b, b + G, ... (16 atoms each, G blocks): it
// computes every force on its atoms and integrates them itself, so an MD step
// costs one grid barrier.  While SMs are left over, one more block owns no
// group and sums the energies of each energy step after its barrier.
//   forces       warp w evaluates slice w of the group's all-pairs row sum
//                (forcefield.cuh, row decomposition) at x_{s+1} (FP32 copy
//                P[s & 1]) and the group's bonded entries dealt to it (each
//                term once per atom it moves); the fixed-point (atom, slice)
//                sums and the bonded forces meet in shared memory;
//   integration  thread t < 48 owns (atom t / 3, component t % 3) of the
//                group and keeps its x, v in registers for the whole launch
//                (first group; further groups go through memory):
//                  v_{s+1} = v_{s+1/2} + dt/2 a          (end of step s, K)
//                  v_{s+3/2} = v_{s+1} + dt/2 a; x_{s+2} = x_{s+1} + dt v
//                  FP32 copy of x_{s+2} into P[(s + 1) & 1]
//   grid barrier (the new positions are visible to every block).
// A pre-phase performs the first half-kick and drift from the forces left in
// the state buffer by mdpf_set_state or by the previous launch; the last step
// writes F(x_n) back there instead.
//
// The forces are the same integer sums the kernel-sequence stepper forms (the
// same row tasks, the same bonded FP32 values), and every state update is an
// explicit FMA (v = fma(h, f, v), x = fma(dt, v, x)) in both, so both steppers
// produce the same trajectory bit for bit.  Energies are summed in a fixed
// order (per block, then blocks in order), so they are reproducible too.
//
// The grid barrier is a 64-bit arrival counter (release add, acquire poll)
// that waits at most limit_ns; on time-out the block records
// MDPF_STATUS_TIMEOUT and returns, and the others follow at their next
// barrier.  Co-residency of all blocks is guaranteed by the cooperative launch.
#include "forcefield.cuh"
#include "grid_sync.cuh"

namespace mdpf {

struct StepArgs {
    PlainDev p;
    int n;
    double dt;
    const double *hdt_m;          // dt/2 * kAcc / m
    const double *mass;
    const float *qs;
    float4 *P0, *P1;              // FP32 position buffers (x, y, z, q sqrt(ke))
    double *x, *v;
    unsigned long long *fxs;      // state forces F(x) (fixed point) on entry and on exit
    long long *part;              // [2][grid][kPart] per-block energies (fixed point)
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

constexpr int kStepWarps = kSlices;              // warp w evaluates slice w of the block's group
constexpr int kStepThreads = 32 * kStepWarps;
constexpr int kSlots = 3 * kRowGroup;            // (atom, component) slots of a group
constexpr int kPart = 8;                         // per-block energies: bond, angle, LJ, Coulomb, kinetic
constexpr int kBondSmem = 256;                   // bonded entries of a group whose forces meet in shared memory

__device__ __forceinline__ float *comp_ptr(float4 *P, int at, int q) { return reinterpret_cast<float *>(P + at) + q; }

// Bonded entries of a group: entry e goes to warp e % 16, lane (e / 16) % 32,
// round e / 512.  A warp evaluates its entries between issuing the loads of
// its first j-chunk and using them.  The fixed-point force of entry
// e < kBondSmem goes to its own shared slot, and the integration thread of an
// atom adds its atom's slots (the entries are sorted by atom); further
// entries are added atomically.
__device__ __forceinline__ int bond_local(int w, int lane, int k) { return kStepWarps * (32 * k + lane) + w; }

__device__ __forceinline__ void bond_add(unsigned long long *bsum, int slot, const float3 &f, bool &bad) {
    atomicAdd(&bsum[slot + 0], (unsigned long long)fx_from_float(f.x));
    atomicAdd(&bsum[slot + 1], (unsigned long long)fx_from_float(f.y));
    atomicAdd(&bsum[slot + 2], (unsigned long long)fx_from_float(f.z));
    bad |= !isfinite(f.x + f.y + f.z);
}

__global__ void __launch_bounds__(kStepThreads, 1) k_plain_persistent(StepArgs a) {
    __shared__ RowStage stage[kStepWarps];
    __shared__ long long red[kStepWarps][kSlots];   // fixed-point (atom, slice) sums of the group, per warp
    __shared__ unsigned long long bsum[kSlots];      // bonded forces of entries >= kBondSmem (fixed point)
    __shared__ long long bstore[kBondSmem][3];       // fixed-point force of each bonded entry < kBondSmem
    __shared__ long long ered[kStepWarps][kPart];   // per-warp energies (fixed point)
    // the first group's state per slot: x, v, dt/2m scaled by 2^-32 (it multiplies the fixed-point force
    // directly), m / (2 kAcc) for the kinetic energy
    __shared__ double s_x[kSlots], s_v[kSlots], s_h[kSlots], s_k[kSlots];
    __shared__ BondEntry s_b0[kStepWarps][32];       // first group's round-0 bonded entry of each lane
    __shared__ int s_fail;
    const PlainDev &p = a.p;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int G = gridDim.x, g0 = blockIdx.x;
    const int64_t step0 = *a.step;
    unsigned long long epoch = 0;
    const int sa = t / 3, sq = t - 3 * (t / 3);   // integration slot of thread t < kSlots: atom sa, component sq
    if (t < kSlots) bsum[t] = 0ull;

    // ---- pre-phase: v_{1/2} = v_0 + dt/2 a(x_0); x_1 = x_0 + dt v_{1/2} for the block's atoms
    for (int g = g0; g < p.n_groups; g += G) {
        if (t < kSlots) {
            const int at = g * kRowGroup + sa;
            if (at < a.n) {
                const double h = a.hdt_m[at];
                const double f = fx_val(a.fxs[3 * at + sq]);
                const double v = fma(h, f, a.v[3 * at + sq]);
                const double x = fma(a.dt, v, a.x[3 * at + sq]);
                a.v[3 * at + sq] = v;
                a.x[3 * at + sq] = x;
                *comp_ptr(a.P0, at, sq) = (float)x;
                if (sq == 0) {
                    *comp_ptr(a.P0, at, 3) = a.qs[at];
                    *comp_ptr(a.P1, at, 3) = a.qs[at];
                }
                if (g == g0) {
                    s_x[t] = x;
                    s_v[t] = v;
                    s_h[t] = h * kFxInv;
                    s_k[t] = 0.5 * a.mass[at] / kAcc;
                }
            } else {   // padding atoms: every pair with them is masked
                *comp_ptr(a.P0, at, sq) = 0.f;
                *comp_ptr(a.P1, at, sq) = 0.f;
                if (sq == 0) {
                    *comp_ptr(a.P0, at, 3) = 0.f;
                    *comp_ptr(a.P1, at, 3) = 0.f;
                }
            }
        }
    }
    // the record of each lane's round-0 bonded entry of the first group stays in shared memory
    const int e_off0 = g0 < p.n_groups ? p.grp_off[g0] : 0;
    const int e_cnt0 = g0 < p.n_groups ? p.grp_off[g0 + 1] - e_off0 : 0;
    if (bond_local(w, lane, 0) < e_cnt0) s_b0[w][lane] = bond_entry(p, e_off0 + bond_local(w, lane, 0));
    // and an integration thread the range of its atom's entries
    const int ab0 = (t < kSlots && g0 < p.n_groups) ? p.grp_aoff[g0 * 17 + sa] : 0;
    const int ae0 = (t < kSlots && g0 < p.n_groups) ? p.grp_aoff[g0 * 17 + sa + 1] : 0;
    if (!grid_barrier(a.bar, ++epoch, a.status, a.limit_ns, &s_fail)) return;

    for (int64_t s = 0; s < a.n_steps; ++s) {
        const float4 *Pcur = (s & 1) ? a.P1 : a.P0;
        float4 *Pnext = (s & 1) ? a.P0 : a.P1;
        const int64_t done = step0 + s + 1;  // steps completed after this iteration
        const bool energy = done % a.energy_every == 0;
        const bool rec = a.record_every > 0 && done % a.record_every == 0;
        const int slot = rec ? (int)((done / a.record_every - 1) % a.frames.cap) : 0;
        const bool last = s + 1 == a.n_steps;
        float eb = 0.f, ea = 0.f;
        long long elj = 0, ec = 0, kin = 0;   // pair energies (per-task FP32 sums) and kinetic, fixed point
        bool bad = false;
        for (int g = g0; g < p.n_groups; g += G) {
            const bool first = g == g0;
            const int e_off = first ? e_off0 : p.grp_off[g];
            const int e_cnt = first ? e_cnt0 : p.grp_off[g + 1] - e_off;
            auto bonded = [&]() {
                for (int k = 0; bond_local(w, lane, k) < e_cnt; ++k) {
                    const int el = bond_local(w, lane, k);
                    const BondEntry b = (first && k == 0) ? s_b0[w][lane] : bond_entry(p, e_off + el);
                    BondedGeom bg;
                    bond_gather(b, Pcur, bg);
                    const float3 f = bond_entry_force(p, b, bg, eb, ea);
                    if (el < kBondSmem) {
                        bstore[el][0] = fx_from_float(f.x);
                        bstore[el][1] = fx_from_float(f.y);
                        bstore[el][2] = fx_from_float(f.z);
                        bad |= !isfinite(f.x + f.y + f.z);
                    } else {
                        bond_add(bsum, b.slot, f, bad);
                    }
                }
            };
            RowQuad r;
            float tl = 0.f, tc = 0.f;
            if (energy) {
                row_task<true>(p, Pcur, g, w, lane, stage[w], r, tl, tc, bonded);
                elj += fx_from_float(tl);
                ec += fx_from_float(tc);
            } else {
                row_task<false>(p, Pcur, g, w, lane, stage[w], r, tl, tc, bonded);
            }
            bad |= !quad_finite(r);
            const RowEmit em = row_emit(lane, r);
            red[w][em.slot_a] = em.va;
            if (em.slot_b >= 0) red[w][em.slot_b] = em.vb;
            __syncthreads();
            // ---- integration of the group: thread t < 48 takes (atom sa, component sq)
            if (t < kSlots) {
                const int at = g * kRowGroup + sa;
                long long F = (long long)bsum[t];
                bsum[t] = 0ull;
#pragma unroll
                for (int k = 0; k < kStepWarps; ++k) F += red[k][t];
                const int ab = first ? ab0 : p.grp_aoff[g * 17 + sa];
                const int ae = min(first ? ae0 : p.grp_aoff[g * 17 + sa + 1], kBondSmem);
#pragma unroll 4
                for (int e = ab; e < ae; ++e) F += bstore[e][sq];
                if (at < a.n) {
                    double x, v, h;
                    if (first) {
                        x = s_x[t];
                        v = s_v[t];
                        h = s_h[t];
                    } else {
                        x = __ldcg(&a.x[3 * at + sq]);
                        v = __ldcg(&a.v[3 * at + sq]);
                        h = a.hdt_m[at] * kFxInv;
                    }
                    // h * F with h = dt/2m 2^-32 and F the exact fixed-point sum: the same FMA as with the force
                    const double Fd = fx_exact(F);
                    v = fma(h, Fd, v);   // v_{s+1}
                    if (energy) {
                        const double km = first ? s_k[t] : 0.5 * a.mass[at] / kAcc;
                        kin += fx_from_double(km * (v * v));
                    }
                    if (rec) {
                        a.frames.pos[((size_t)slot * a.n + at) * 3 + sq] = x;
                        a.frames.forces[((size_t)slot * a.n + at) * 3 + sq] = (float)(Fd * kFxInv);
                    }
                    if (last) a.fxs[3 * at + sq] = (unsigned long long)F;   // F(x_n) for the next launch
                    if ((first && energy) || last) {
                        // energy steps: the status is checked there and the launch may stop
                        a.x[3 * at + sq] = x;
                        a.v[3 * at + sq] = v;
                    }
                    if (!last) {
                        v = fma(h, Fd, v);     // v_{s+3/2}
                        x = fma(a.dt, v, x);   // x_{s+2}
                        *comp_ptr(Pnext, at, sq) = (float)x;
                        if (!first) {
                            a.x[3 * at + sq] = x;
                            a.v[3 * at + sq] = v;
                        }
                    }
                    if (first) {
                        s_x[t] = x;
                        s_v[t] = v;
                    }
                    bad |= !finite_bits(v);
                }
            }
            if (g + G < p.n_groups) __syncthreads();   // red and bsum are reused by the next group
        }
        if (bad) atomicOr(a.status, MDPF_STATUS_NONFINITE);
        if (energy) {
            const long long e0 = warp_sum_ll(fx_from_float(eb)), e1 = warp_sum_ll(fx_from_float(ea));
            const long long e2 = warp_sum_ll(elj), e3 = warp_sum_ll(ec), e4 = warp_sum_ll(kin);
            if (lane == 0) {
                ered[w][0] = e0;
                ered[w][1] = e1;
                ered[w][2] = e2;
                ered[w][3] = e3;
                ered[w][4] = e4;
            }
            __syncthreads();
            if (t < 5) {
                long long sum = 0;
#pragma unroll
                for (int k = 0; k < kStepWarps; ++k) sum += ered[k][t];
                a.part[((size_t)(s & 1) * G + blockIdx.x) * kPart + t] = sum;
            }
        }
        if (!grid_barrier(a.bar, ++epoch, a.status, a.limit_ns, &s_fail)) return;
        // ---- energies of step `done`, read after the barrier by the last block: a block with no group when
        // the grid has one to spare, so the sum does not delay any group's next step
        if (energy && blockIdx.x == G - 1 && w == 0) {
            const long long *pp = a.part + (size_t)(s & 1) * G * kPart;
            long long ib = 0, ia = 0, il = 0, ic = 0, ik = 0;
            for (int b = lane; b < G; b += 32) {
                ib += pp[kPart * b];
                ia += pp[kPart * b + 1];
                il += pp[kPart * b + 2];
                ic += pp[kPart * b + 3];
                ik += pp[kPart * b + 4];
            }
            ib = warp_sum_ll(ib);
            ia = warp_sum_ll(ia);
            il = warp_sum_ll(il);
            ic = warp_sum_ll(ic);
            ik = warp_sum_ll(ik);
            // the pair sums hold 24 eps (s^12 - s^6) and q q / r for every pair counted from both atoms
            const double sb = fx_exact(ib) * kFxInv, sa2 = fx_exact(ia) * kFxInv;
            const double sl = fx_exact(il) * (kFxInv / 12.0), sc = fx_exact(ic) * (kFxInv * 0.5);
            const double sk = fx_exact(ik) * kFxInv;
            if (lane == 0) {
                const double U = sb + sa2 + sl + sc;
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
        if (blockIdx.x == 0 && t == 0 && last) *a.step = done;
        // every block reads the status after the same barrier, so all stop together
        if (energy && *(volatile uint32_t *)a.status != 0u) {
            if (blockIdx.x == 0 && t == 0) *a.step = done;
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
    // one block per group, one block per SM; with more than one group (a grid barrier anyway) one more block
    // for the per-step energy sums while SMs are left
    const int want = ctx->n_groups > 1 ? ctx->n_groups + 1 : 1;
    return want < sms ? want : sms;
}

cudaError_t launch_plain_persistent(mdpf_ctx *ctx, int64_t n_steps, cudaStream_t s) {
    StepArgs a;
    a.p = plain_dev(ctx, ctx->d_pos4);
    a.n = ctx->n;
    a.dt = ctx->dt;
    a.hdt_m = ctx->d_hdt_m;
    a.mass = ctx->d_mass;
    a.qs = ctx->d_charge_s;
    a.P0 = ctx->d_pos4;
    a.P1 = ctx->d_pos4_b;
    a.x = ctx->d_x;
    a.v = ctx->d_v;
    a.fxs = ctx->d_fx;
    a.part = ctx->d_part;
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
