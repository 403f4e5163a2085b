// Plain analytic force field and velocity-Verlet kernels (kernel-sequence path
// and the helpers that mdpf_compute / mdpf_set_state use).
//
// Energy terms (units kcal/mol, A):
//   bonds    E = k/2 (r - r0)^2
//   angles   E = k/2 (theta - theta0)^2, one per pair of bonds meeting at an atom
//   pairs    E = 4 eps_ij [(sigma_ij/r)^12 - (sigma_ij/r)^6] + ke q_i q_j / r
//            over every pair that is neither 1-2 nor 1-3, no cutoff
// Forces are accumulated as int64 fixed point (value * 2^32), so the result
// does not depend on the order in which warps finish.
#include "forcefield.cuh"

namespace mdpf {
namespace {

// ------------------------------------------------------------------ helpers

__global__ void k_zero_fx(unsigned long long *fx, int n3, unsigned long long *efx) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3) fx[i] = 0ull;
    if (efx != nullptr && i < E_SLOTS) efx[i] = 0ull;
}

__global__ void k_pos4_from_x(const double *x, const float *qs, float4 *pos4, int n, int n_pad) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < n) {
        pos4[a] = make_float4((float)x[3 * a], (float)x[3 * a + 1], (float)x[3 * a + 2], qs[a]);
    } else if (a < n_pad) {
        pos4[a] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void k_fx_to_forces(const unsigned long long *fx, int n3, double *f64, float *f32) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3) {
        double v = fx_val(fx[i]);
        if (f64) f64[i] = v;
        if (f32) f32[i] = (float)v;
    }
}

// out = {U, E_bond, E_angle, E_LJ, E_Coulomb, K}
__global__ void k_energy_out(const unsigned long long *efx, double *out) {
    int t = threadIdx.x;
    if (t < 5) out[1 + t] = fx_val(efx[t]);
    if (t == 0)
        out[0] = fx_val(efx[E_BOND]) + fx_val(efx[E_ANGLE]) + fx_val(efx[E_LJ]) + fx_val(efx[E_COUL]) +
                 fx_val(efx[E_LEARN]);
}

// The start of a single evaluation in one launch: FP32 positions (and
// charges) from FP64 x, padding rows zero, and the fixed-point force and
// energy sums cleared.
__global__ void k_eval_begin(const double *x, const float *qs, float4 *pos4, int n, int n_pad,
                             unsigned long long *fx, int n3, unsigned long long *efx) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) pos4[q] = make_float4((float)x[3 * q], (float)x[3 * q + 1], (float)x[3 * q + 2], qs[q]);
    else if (q < n_pad) pos4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q < n3) fx[q] = 0ull;
    if (q < E_SLOTS) efx[q] = 0ull;
}

// Its end in one launch: FP32 forces (f32 may be null), the energy terms as
// k_energy_out writes them, and the total energy to *energy (may be null).
__global__ void k_eval_end(const unsigned long long *fx, int n3, float *f32, const unsigned long long *efx,
                           double *out, double *energy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (f32 != nullptr && i < n3) f32[i] = (float)fx_val(fx[i]);
    if (blockIdx.x == 0) {
        const int t = threadIdx.x;
        if (t < 5) out[1 + t] = fx_val(efx[t]);
        if (t == 0) {
            const double U = fx_val(efx[E_BOND]) + fx_val(efx[E_ANGLE]) + fx_val(efx[E_LJ]) + fx_val(efx[E_COUL]) +
                             fx_val(efx[E_LEARN]);
            out[0] = U;
            if (energy != nullptr) *energy = U;
        }
    }
}

// An external provider's FP32 forces and FP64 energy into the fixed-point sums.
__global__ void k_provider_to_fx(const float *forces, const double *energy, int n, unsigned long long *fx,
                                 unsigned long long *efx, uint32_t *status) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < 3 * n) {
        const float f = forces[q];
        if (!isfinite(f)) atomicOr(status, MDPF_STATUS_NONFINITE);
        fx_add(&fx[q], f);
    }
    if (q == 0) {
        const double e = *energy;
        if (!isfinite(e) || fabs(e) > 1e9) atomicOr(status, MDPF_STATUS_NONFINITE);
        else fx_add_d(&efx[E_LEARN], e);
    }
}

// ------------------------------------------------------------------ bonded

__global__ void k_bonded(PlainDev p, unsigned long long *fx, unsigned long long *efx) {
    if (p.gate != nullptr && *p.gate == 0u) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    float eb = 0.f, ea = 0.f;
    if (t < p.n_bonds + p.n_angles) bonded_term(p, t, fx, eb, ea);
    if (!isfinite(eb + ea)) atomicOr(p.status, MDPF_STATUS_NONFINITE);
    if (efx != nullptr) {
        double sb = warp_sum_d((double)eb), sa = warp_sum_d((double)ea);
        if ((threadIdx.x & 31) == 0) {
            if (sb != 0.0) fx_add_d(&efx[E_BOND], sb);
            if (sa != 0.0) fx_add_d(&efx[E_ANGLE], sa);
        }
    }
}

// ------------------------------------------------------------------ all pairs

constexpr int kNbThreads = 256;

// One warp per (row group, slice) task of the row decomposition
// (forcefield.cuh); the lanes add their fixed-point (atom, slice) sums.
template <bool ENERGY>
__global__ void __launch_bounds__(kNbThreads) k_nonbonded(PlainDev p, unsigned long long *fx,
                                                          unsigned long long *efx, uint32_t *status) {
    if (p.gate != nullptr && *p.gate == 0u) return;
    __shared__ RowStage st[kNbThreads / 32];
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int slices = p.n_chunks < kSlices ? p.n_chunks : kSlices;
    const int tasks = p.n_groups * slices;
    double elj = 0.0, ec = 0.0;   // per-task FP32 sums (the same in both steppers) added in FP64
    bool bad = false;
    for (int task = warp; task < tasks; task += nwarps) {
        const int g = task / slices, sl = task - g * slices;
        RowQuad r;
        float tl = 0.f, tc = 0.f;
        row_task<ENERGY>(p, p.pos4, g, sl, lane, st[threadIdx.x >> 5], r, tl, tc, [] {});
        elj += tl;
        ec += tc;
        bad |= !quad_finite(r);
        const RowEmit e = row_emit(lane, r);
        const int base = 3 * g * kRowGroup;
        if (base + e.slot_a < 3 * p.n) atomicAdd(&fx[base + e.slot_a], (unsigned long long)e.va);
        if (e.slot_b >= 0 && base + e.slot_b < 3 * p.n) atomicAdd(&fx[base + e.slot_b], (unsigned long long)e.vb);
    }
    if (bad) atomicOr(status, MDPF_STATUS_NONFINITE);
    if (ENERGY) {
        // every pair was met from both of its atoms
        double e_lj = warp_sum_d(elj * (0.5 / 6.0));
        double e_c = warp_sum_d(ec * 0.5);
        if (lane == 0) {
            fx_add_d(&efx[E_LJ], e_lj);
            fx_add_d(&efx[E_COUL], e_c);
        }
    }
}

// ------------------------------------------------------------------ integrator

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the multiply-xor round
// with the Weyl-advanced key.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const unsigned int lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned int lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Langevin O step (BAOAB): atom a, step index `step`: three Box-Muller normals
// from Philox with counter (a, step low, step high, tag) and key = seed.
__device__ __forceinline__ void langevin_normals(unsigned long long seed, long long step, int a, double z[3]) {
    const uint4 r = philox4x32_10(make_uint4((unsigned int)a, (unsigned int)(unsigned long long)step,
                                             (unsigned int)((unsigned long long)step >> 32), 0x4C414E47u),
                                  make_uint2((unsigned int)seed, (unsigned int)(seed >> 32)));
    const double inv = 1.0 / 4294967296.0, two_pi = 6.283185307179586476925286766559;
    const double u0 = ((double)r.x + 0.5) * inv, u1 = ((double)r.y + 0.5) * inv;
    const double u2 = ((double)r.z + 0.5) * inv, u3 = ((double)r.w + 0.5) * inv;
    const double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
    z[0] = r0 * cos(two_pi * u1);
    z[1] = r0 * sin(two_pi * u1);
    z[2] = r1 * cos(two_pi * u3);
}

// Velocity Verlet:  v += dt/2 a(F);  x += dt v.
// Langevin (lang != null), BAOAB:  v += dt/2 a(F);  x += dt/2 v;  v = c1 v + c2 R;  x += dt/2 v.
// Then the FP32 copy is refreshed and the force accumulators cleared.  With a
// displacement check (learned mode), a neighbour-list rebuild is requested
// when the new FP32 position is more than skin/2 from the one at the last
// build, or when the completed-step count is a multiple of rebuild_every.
__global__ void k_kick_drift(int n, int n_pad, double dt, const double *hdt_over_m, double *x, double *v,
                             unsigned long long *fx, float4 *pos4, const float *qs, unsigned long long *efx,
                             LangevinDev lang, DispCheck dc) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < E_SLOTS && efx != nullptr) efx[a] = 0ull;
    if (a >= n) {
        if (a < n_pad) {
            fx[3 * a] = fx[3 * a + 1] = fx[3 * a + 2] = 0ull;
            pos4[a] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return;
    }
    const double h = hdt_over_m[a];
    double p[3];
    if (lang.c2 != nullptr) {
        double z[3];
        langevin_normals(lang.seed, *lang.step, a, z);
        const double c2 = lang.c2[a], hdt = 0.5 * dt;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double vc = fma(h, fx_val(fx[3 * a + c]), v[3 * a + c]);
            double xc = fma(hdt, vc, x[3 * a + c]);
            vc = fma(lang.c1, vc, c2 * z[c]);
            xc = fma(hdt, vc, xc);
            v[3 * a + c] = vc;
            x[3 * a + c] = xc;
            p[c] = xc;
            fx[3 * a + c] = 0ull;
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double vc = fma(h, fx_val(fx[3 * a + c]), v[3 * a + c]);
            double xc = fma(dt, vc, x[3 * a + c]);
            v[3 * a + c] = vc;
            x[3 * a + c] = xc;
            p[c] = xc;
            fx[3 * a + c] = 0ull;
        }
    }
    const float4 p4 = make_float4((float)p[0], (float)p[1], (float)p[2], qs[a]);
    pos4[a] = p4;
    if (dc.pos_build != nullptr) {
        if (a == 0 && dc.rebuild_every > 0 && (*lang.step % dc.rebuild_every) == 0) atomicOr(dc.flag, 1u);
        const float4 b = dc.pos_build[a];
        const float dx = p4.x - b.x, dy = p4.y - b.y, dz = p4.z - b.z;
        if (dx * dx + dy * dy + dz * dz > dc.half_skin2) atomicOr(dc.flag, 1u);
    }
}

// v += dt/2 a(F_new) (when do_kick); kinetic energy into the fixed-point slot (when energy).
__global__ void k_kick(int n, const double *hdt_over_m, const double *mass, double *v, const unsigned long long *fx,
                       unsigned long long *efx, int do_kick, int energy) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0;
    if (a < n) {
        const double h = hdt_over_m[a];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double vc = v[3 * a + c];
            if (do_kick) {
                vc = fma(h, fx_val(fx[3 * a + c]), vc);
                v[3 * a + c] = vc;
            }
            ke += vc * vc;
        }
        ke *= 0.5 * mass[a] / kAcc;
    }
    if (!energy) return;
    ke = warp_sum_d(ke);
    if ((threadIdx.x & 31) == 0 && ke != 0.0) fx_add_d(&efx[E_KIN], ke);
}

// End of a step, one kernel: v += dt/2 a(F_new); the kinetic energy on energy
// steps; the frame (positions, forces) when the completed step is recorded.
// The last block to finish (a ticket counter, reset by that block) then does
// the single-thread part: the step counter, and on energy steps the trace
// entry, the scalars and the non-finite check; the recorded frame's energy and
// step.
struct FinishArgs {
    const double *x;
    double *trace_u, *trace_k;
    int64_t *trace_step;
    int64_t *trace_fb;            // cumulative fallback evaluations per trace entry
    const long long *fb_count;    // learned mode: the device counter of fallback evaluations, else null
    int cap, energy_every, record_every;
    int64_t *step;
    uint32_t *status;
    double *scalars;
    unsigned int *ticket;
    Frames frames;
};

__global__ void k_kick_finish(int n, const double *hdt_over_m, const double *mass, double *v,
                              const unsigned long long *fx, unsigned long long *efx, int energy, FinishArgs f) {
    __shared__ int s_last;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s = *f.step + 1;   // the step being completed
    const bool rec = f.record_every > 0 && f.frames.cap > 0 && s % f.record_every == 0;
    const int slot = rec ? (int)((s / f.record_every - 1) % f.frames.cap) : 0;
    double ke = 0.0;
    if (a < n) {
        const double h = hdt_over_m[a];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double fc = fx_val(fx[3 * a + c]);
            const double vc = fma(h, fc, v[3 * a + c]);
            v[3 * a + c] = vc;
            ke += vc * vc;
            if (rec) {
                f.frames.pos[((size_t)slot * n + a) * 3 + c] = f.x[3 * a + c];
                f.frames.forces[((size_t)slot * n + a) * 3 + c] = (float)fc;
            }
        }
        ke *= 0.5 * mass[a] / kAcc;
    }
    if (energy) {
        ke = warp_sum_d(ke);
        if ((threadIdx.x & 31) == 0 && ke != 0.0) fx_add_d(&efx[E_KIN], ke);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(f.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    *f.ticket = 0u;
    __threadfence();
    *f.step = s;
    if (energy) {
        const double U = fx_val(__ldcg(&efx[E_BOND])) + fx_val(__ldcg(&efx[E_ANGLE])) + fx_val(__ldcg(&efx[E_LJ])) +
                         fx_val(__ldcg(&efx[E_COUL])) + fx_val(__ldcg(&efx[E_LEARN]));
        const double K = fx_val(__ldcg(&efx[E_KIN]));
        const int64_t e = s / f.energy_every - 1;
        f.trace_u[e % f.cap] = U;
        f.trace_k[e % f.cap] = K;
        f.trace_step[e % f.cap] = s;
        f.trace_fb[e % f.cap] = f.fb_count != nullptr ? (int64_t)__ldcg(f.fb_count) : 0;
        f.scalars[0] = U;
        f.scalars[1] = K;
        // fixed-point slots saturate rather than turn NaN: treat huge values as non-finite too
        const bool bad = !isfinite(U) || !isfinite(K) || fabs(U) > 1e9 || fabs(K) > 1e9;
        if (bad) atomicOr(f.status, MDPF_STATUS_NONFINITE);
    }
    if (rec) {
        f.frames.energy[slot] = f.scalars[0];
        f.frames.step[slot] = s;
    }
}

// Maxwell-Boltzmann initial velocities in one block (runs once per call, so
// one block of kMbThreads keeps every reduction in a fixed order):
//   v_a = sqrt(kB T / m_a) z_a, z_a three Box-Muller normals from Philox with
//   counter (a, 0, 0, 'MBV0') and key = seed; minus the centre-of-mass
//   velocity; for n >= 3 minus the rigid rotation w x (x_a - x_com), I w = L
//   (skipped when I is singular); then scaled to K = (3n - 6) kB T / 2.
constexpr int kMbThreads = 1024;

__device__ double mb_block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = kMbThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kMbThreads) k_init_velocities(int n, const double *mass, const double *x,
                                                                  double *v, double kT_acc, double k_target,
                                                                  unsigned long long seed) {
    __shared__ double sh[kMbThreads];
    __shared__ double s_q[16];
    const int t = threadIdx.x;
    const double inv = 1.0 / 4294967296.0, two_pi = 6.283185307179586476925286766559;
    double M = 0, P[3] = {0, 0, 0}, mx[3] = {0, 0, 0};
    for (int a = t; a < n; a += kMbThreads) {
        const uint4 r = philox4x32_10(make_uint4((unsigned int)a, 0u, 0u, 0x4D425630u),
                                      make_uint2((unsigned int)seed, (unsigned int)(seed >> 32)));
        const double u0 = ((double)r.x + 0.5) * inv, u1 = ((double)r.y + 0.5) * inv;
        const double u2 = ((double)r.z + 0.5) * inv, u3 = ((double)r.w + 0.5) * inv;
        const double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
        const double z[3] = {r0 * cos(two_pi * u1), r0 * sin(two_pi * u1), r1 * cos(two_pi * u3)};
        const double m = mass[a], sd = sqrt(kT_acc / m);
        M += m;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double vc = sd * z[c];
            v[3 * a + c] = vc;
            P[c] += m * vc;
            mx[c] += m * x[3 * a + c];
        }
    }
    M = mb_block_sum(M, sh);
    double vcm[3], com[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        vcm[c] = mb_block_sum(P[c], sh) / M;
        com[c] = mb_block_sum(mx[c], sh) / M;
    }
    double L[3] = {0, 0, 0}, I6[6] = {0, 0, 0, 0, 0, 0};   // I: xx yy zz xy xz yz
    for (int a = t; a < n; a += kMbThreads) {
        const double m = mass[a];
        const double r[3] = {x[3 * a] - com[0], x[3 * a + 1] - com[1], x[3 * a + 2] - com[2]};
        double vv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            vv[c] = v[3 * a + c] - vcm[c];
            v[3 * a + c] = vv[c];
        }
        L[0] += m * (r[1] * vv[2] - r[2] * vv[1]);
        L[1] += m * (r[2] * vv[0] - r[0] * vv[2]);
        L[2] += m * (r[0] * vv[1] - r[1] * vv[0]);
        const double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        I6[0] += m * (rr - r[0] * r[0]);
        I6[1] += m * (rr - r[1] * r[1]);
        I6[2] += m * (rr - r[2] * r[2]);
        I6[3] -= m * r[0] * r[1];
        I6[4] -= m * r[0] * r[2];
        I6[5] -= m * r[1] * r[2];
    }
    if (n >= 3) {
        double Ls[3], Is[6];
#pragma unroll
        for (int c = 0; c < 3; ++c) Ls[c] = mb_block_sum(L[c], sh);
#pragma unroll
        for (int c = 0; c < 6; ++c) Is[c] = mb_block_sum(I6[c], sh);
        if (t == 0) {
            const double a = Is[0], b = Is[1], c = Is[2], d = Is[3], e = Is[4], f = Is[5];
            // I = [[a d e] [d b f] [e f c]]; w = adj(I) L / det(I)
            const double A00 = b * c - f * f, A01 = e * f - d * c, A02 = d * f - e * b;
            const double A11 = a * c - e * e, A12 = d * e - a * f, A22 = a * b - d * d;
            const double det = a * A00 + d * A01 + e * A02, tr = a + b + c;
            const bool ok = fabs(det) > 1e-12 * tr * tr * tr;
            s_q[0] = ok ? (A00 * Ls[0] + A01 * Ls[1] + A02 * Ls[2]) / det : 0.0;
            s_q[1] = ok ? (A01 * Ls[0] + A11 * Ls[1] + A12 * Ls[2]) / det : 0.0;
            s_q[2] = ok ? (A02 * Ls[0] + A12 * Ls[1] + A22 * Ls[2]) / det : 0.0;
        }
        __syncthreads();
    } else if (t == 0) {
        s_q[0] = s_q[1] = s_q[2] = 0.0;
    }
    __syncthreads();
    const double w[3] = {s_q[0], s_q[1], s_q[2]};
    double K = 0;
    for (int a = t; a < n; a += kMbThreads) {
        const double r[3] = {x[3 * a] - com[0], x[3 * a + 1] - com[1], x[3 * a + 2] - com[2]};
        double vv[3] = {v[3 * a], v[3 * a + 1], v[3 * a + 2]};
        vv[0] -= w[1] * r[2] - w[2] * r[1];
        vv[1] -= w[2] * r[0] - w[0] * r[2];
        vv[2] -= w[0] * r[1] - w[1] * r[0];
#pragma unroll
        for (int c = 0; c < 3; ++c) v[3 * a + c] = vv[c];
        K += 0.5 * mass[a] * (vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]) / kAcc;
    }
    K = mb_block_sum(K, sh);
    const double sc = K > 0.0 ? sqrt(k_target / K) : 1.0;
    for (int q = t; q < 3 * n; q += kMbThreads) v[q] *= sc;
}

// Spin on a flag that nothing sets, for at most limit_ns of globaltimer.
__global__ void k_wait_timeout(uint32_t *status, volatile unsigned int *flag, long long limit_ns) {
    if (threadIdx.x != 0) return;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (*flag == 0u) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if ((long long)(t - t0) > limit_ns) {
            atomicOr(status, MDPF_STATUS_TIMEOUT);
            return;
        }
        __nanosleep(1000);
    }
}

}  // namespace

// ------------------------------------------------------------------ launchers

PlainDev plain_dev(const mdpf_ctx *ctx, const float4 *pos4) {
    PlainDev p;
    p.n = ctx->n;
    p.n_pad = ctx->n_pad;
    p.n_tiles = ctx->n_tiles;
    p.n_bonds = ctx->n_bonds;
    p.n_angles = ctx->n_angles;
    p.pos4 = pos4;
    p.lj = ctx->d_lj;
    p.bonds = ctx->d_bonds;
    p.bond_par = ctx->d_bond_par;
    p.angles = ctx->d_angles;
    p.angle_k = ctx->angle_k;
    p.angle_theta0 = ctx->angle_theta0;
    p.tile_mask = nullptr;
    p.tile_flag = nullptr;
    p.items = nullptr;
    p.n_items = 0;
    p.n_groups = ctx->n_groups;
    p.n_chunks = ctx->n_chunks;
    p.row_mask = ctx->d_row_mask;
    p.grp_off = ctx->d_grp_off;
    p.grp_ent = ctx->d_grp_ent;
    p.grp_aoff = ctx->d_grp_aoff;
    p.status = ctx->d_status;
    p.gate = nullptr;
    return p;
}

void launch_zero_fx(unsigned long long *fx, int n3, unsigned long long *efx, cudaStream_t s) {
    int m = n3 > E_SLOTS ? n3 : E_SLOTS;
    k_zero_fx<<<(m + 255) / 256, 256, 0, s>>>(fx, n3, efx);
}

void launch_pos4_from_x(const double *x, const float *qs, float4 *pos4, int n, int n_pad, cudaStream_t s) {
    k_pos4_from_x<<<(n_pad + 255) / 256, 256, 0, s>>>(x, qs, pos4, n, n_pad);
}

void launch_bonded(const PlainDev &p, unsigned long long *fx, unsigned long long *efx, cudaStream_t s) {
    int m = p.n_bonds + p.n_angles;
    if (m > 0) k_bonded<<<(m + 255) / 256, 256, 0, s>>>(p, fx, efx);
}

void launch_nonbonded(const PlainDev &p, unsigned long long *fx, unsigned long long *efx, bool energy,
                      cudaStream_t s) {
    const int slices = p.n_chunks < kSlices ? p.n_chunks : kSlices;
    int blocks = (p.n_groups * slices * 32 + kNbThreads - 1) / kNbThreads;
    if (blocks < 1) blocks = 1;
    if (energy)
        k_nonbonded<true><<<blocks, kNbThreads, 0, s>>>(p, fx, efx, p.status);
    else
        k_nonbonded<false><<<blocks, kNbThreads, 0, s>>>(p, fx, efx, p.status);
}

void launch_fx_to_forces(const unsigned long long *fx, int n, double *f64, float *f32, cudaStream_t s) {
    k_fx_to_forces<<<(3 * n + 255) / 256, 256, 0, s>>>(fx, 3 * n, f64, f32);
}

void launch_energy_out(const unsigned long long *efx, double *out6, cudaStream_t s) {
    k_energy_out<<<1, 32, 0, s>>>(efx, out6);
}

void launch_eval_begin(const double *x, const float *qs, float4 *pos4, int n, int n_pad, unsigned long long *fx,
                       int n3, unsigned long long *efx, cudaStream_t s) {
    int m = n_pad > n3 ? n_pad : n3;
    if (m < E_SLOTS) m = E_SLOTS;
    k_eval_begin<<<(m + 255) / 256, 256, 0, s>>>(x, qs, pos4, n, n_pad, fx, n3, efx);
}

void launch_eval_end(const unsigned long long *fx, int n, float *f32, const unsigned long long *efx, double *out6,
                     double *energy, cudaStream_t s) {
    const int m = f32 != nullptr ? 3 * n : 1;
    k_eval_end<<<(m + 255) / 256, 256, 0, s>>>(fx, 3 * n, f32, efx, out6, energy);
}

// FP64 integrator kernels use small blocks so that the (slow) FP64 work of a
// few thousand atoms spreads over many SMs.
constexpr int kIntThreads = 32;

void launch_kick_drift(mdpf_ctx *ctx, cudaStream_t s) {
    int m = ctx->n_pad > E_SLOTS ? ctx->n_pad : E_SLOTS;
    const DispCheck dc = ctx->mode == MDPF_MODE_LEARNED ? learned_disp_check(ctx) : DispCheck{nullptr, nullptr, 0.f, 0};
    k_kick_drift<<<(m + kIntThreads - 1) / kIntThreads, kIntThreads, 0, s>>>(
        ctx->n, ctx->n_pad, ctx->dt, ctx->d_hdt_m, ctx->d_x, ctx->d_v, ctx->d_fx, ctx->d_pos4, ctx->d_charge_s,
        ctx->d_efx, LangevinDev{ctx->d_lang_c2, ctx->lang_c1, ctx->lang_seed, ctx->d_step}, dc);
}

void launch_kick_finish(mdpf_ctx *ctx, bool energy, cudaStream_t s) {
    FinishArgs f{ctx->d_x,          ctx->d_trace_u,   ctx->d_trace_k,      ctx->d_trace_step, ctx->d_trace_fb,
                 learned_fallback_counter(ctx), ctx->trace_cap, ctx->energy_every, ctx->record_every,
                 ctx->d_step,       ctx->d_status,    ctx->d_scalar,       ctx->d_status + 3, ctx->frames};
    k_kick_finish<<<(ctx->n + kIntThreads - 1) / kIntThreads, kIntThreads, 0, s>>>(
        ctx->n, ctx->d_hdt_m, ctx->d_mass, ctx->d_v, ctx->d_fx, ctx->d_efx, energy ? 1 : 0, f);
}

// Kinetic energy of the current velocities into efx[E_KIN] (no kick).
void launch_provider_to_fx(const float *forces, const double *energy, int n, unsigned long long *fx,
                           unsigned long long *efx, uint32_t *status, cudaStream_t s) {
    k_provider_to_fx<<<(3 * n + 255) / 256, 256, 0, s>>>(forces, energy, n, fx, efx, status);
}

void launch_kinetic(mdpf_ctx *ctx, cudaStream_t s) {
    k_kick<<<(ctx->n + kIntThreads - 1) / kIntThreads, kIntThreads, 0, s>>>(ctx->n, ctx->d_hdt_m, ctx->d_mass,
                                                                              ctx->d_v, ctx->d_fx, ctx->d_efx, 0, 1);
}

void launch_init_velocities(mdpf_ctx *ctx, double temperature_K, unsigned long long seed, cudaStream_t s) {
    const double kB = 0.0019872041;   // kcal/mol/K
    const int dof = 3 * ctx->n - 6 > 1 ? 3 * ctx->n - 6 : 1;
    k_init_velocities<<<1, kMbThreads, 0, s>>>(ctx->n, ctx->d_mass, ctx->d_x, ctx->d_v, kB * temperature_K * kAcc,
                                               0.5 * dof * kB * temperature_K, seed);
}

void launch_wait_timeout(uint32_t *status, unsigned int *flag, long long limit_ns, cudaStream_t s) {
    k_wait_timeout<<<1, 32, 0, s>>>(status, flag, limit_ns);
}

}  // namespace mdpf
