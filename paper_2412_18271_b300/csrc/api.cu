// C ABI entry points of libmdpf (declared in include/mdpf.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "forcefield.cuh"

using namespace mdpf;

namespace {
thread_local std::string g_create_error;
}

namespace mdpf {

int fail(mdpf_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg; else g_create_error = msg;
    return code;
}

int cuda_fail(mdpf_ctx *ctx, cudaError_t e, const char *where) {
    std::string m = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
    if (ctx) {
        ctx->sticky = true;
        ctx->err = m;
    } else {
        g_create_error = m;
    }
    return MDPF_ERR_CUDA;
}

static cudaEvent_t prof_event(mdpf_ctx *c) {
    if (!c->prof_free.empty()) {
        cudaEvent_t e = c->prof_free.back();
        c->prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

int prof_harvest(mdpf_ctx *c) {
    for (auto &r : c->prof_pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return cuda_fail(c, e, "profile events");
        c->prof_ms[r.slot] += ms;
        c->prof_n[r.slot] += 1;
        c->prof_free.push_back(r.a);
        c->prof_free.push_back(r.b);
    }
    c->prof_pending.clear();
    return MDPF_OK;
}

cudaEvent_t prof_begin(mdpf_ctx *c, cudaStream_t s) {
    if (!c->profiling) return nullptr;
    if (c->prof_pending.size() >= 2048) prof_harvest(c);
    cudaEvent_t a = prof_event(c);
    if (a) cudaEventRecord(a, s);
    return a;
}

void prof_end(mdpf_ctx *c, int slot, cudaEvent_t a, cudaStream_t s) {
    if (!c->profiling || !a) return;
    cudaEvent_t b = prof_event(c);
    if (!b) return;
    cudaEventRecord(b, s);
    c->prof_pending.push_back({slot, a, b});
}

}  // namespace mdpf

#define CK(ctx, x)                                               \
    do {                                                         \
        cudaError_t e_ = (x);                                    \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #x);  \
    } while (0)

#define GUARD(ctx)                                         \
    do {                                                   \
        if ((ctx) == nullptr) return MDPF_ERR_INVALID_ARG; \
        if ((ctx)->sticky) return MDPF_ERR_CUDA;           \
    } while (0)

static void free_ctx(mdpf_ctx *c) {
    if (!c) return;
    small_free(c);
    learned_free(c);
    for (auto &r : c->prof_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->prof_free) cudaEventDestroy(e);
    void *ptrs[] = {c->d_element, c->d_mass, c->d_hdt_m, c->d_pos4, c->d_pos4_b, c->d_pos4_c, c->d_lj,
                    c->d_charge_s, c->d_bonds, c->d_bond_par, c->d_angles, c->d_excl_off, c->d_excl_idx,
                    c->d_row_mask, c->d_grp_off, c->d_grp_ent, c->d_grp_aoff, c->d_x, c->d_v, c->d_fx_base, c->d_fx_c,
                    c->d_efx, c->d_efx_c, c->d_trace_u, c->d_trace_k, c->d_trace_step, c->d_trace_fb, c->d_step, c->d_status,
                    c->d_xc, c->d_fc, c->d_scalar, c->d_barrier, c->d_part, c->d_lang_c2, c->frames.pos,
                    c->frames.energy, c->frames.forces,
                    c->frames.step};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (auto &g : c->lgraph)
        if (g) cudaGraphExecDestroy(g);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

template <typename T>
static cudaError_t dalloc(T **p, size_t count) {
    return cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
}

extern "C" {

const char *mdpf_last_error(const mdpf_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int mdpf_create(const mdpf_topology *t, const mdpf_params *prm, mdpf_ctx **out) {
    if (out == nullptr) return fail(nullptr, MDPF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (t == nullptr || prm == nullptr) return fail(nullptr, MDPF_ERR_INVALID_ARG, "topology or params is NULL");
    const int n = t->n_atoms;
    if (n < 1) return fail(nullptr, MDPF_ERR_INVALID_ARG, "n_atoms must be >= 1");
    if (n > (1 << 22)) return fail(nullptr, MDPF_ERR_INVALID_ARG, "n_atoms too large");
    if (!t->element || !t->mass || !t->charge) return fail(nullptr, MDPF_ERR_INVALID_ARG, "NULL per-atom array");
    if (t->n_bonds < 0 || (t->n_bonds > 0 && (!t->bonds || !t->bond_r0 || !t->bond_k)))
        return fail(nullptr, MDPF_ERR_INVALID_ARG, "bad bond arrays");
    if (prm->mode != MDPF_MODE_PLAIN && prm->mode != MDPF_MODE_LEARNED && prm->mode != MDPF_MODE_CALLBACK)
        return fail(nullptr, MDPF_ERR_INVALID_ARG, "unknown mode");
    if (prm->integrator != MDPF_INTEGRATOR_VERLET && prm->integrator != MDPF_INTEGRATOR_LANGEVIN)
        return fail(nullptr, MDPF_ERR_INVALID_ARG, "unknown integrator");
    if (prm->integrator == MDPF_INTEGRATOR_LANGEVIN &&
        (!(prm->friction_per_ps > 0.0) || !std::isfinite(prm->friction_per_ps) || !(prm->temperature_K >= 0.0) ||
         !std::isfinite(prm->temperature_K)))
        return fail(nullptr, MDPF_ERR_INVALID_ARG, "Langevin needs friction_per_ps > 0 and temperature_K >= 0");
    if (prm->mode == MDPF_MODE_CALLBACK &&
        (!prm->provider || !prm->provider_pos || !prm->provider_energy || !prm->provider_forces))
        return fail(nullptr, MDPF_ERR_INVALID_ARG, "callback mode needs the provider function and its three buffers");
    if (prm->mode == MDPF_MODE_LEARNED && (!(prm->skin >= 0.0) || !std::isfinite(prm->skin) || prm->skin > 10.0 ||
                                           prm->rebuild_every < 0))
        return fail(nullptr, MDPF_ERR_INVALID_ARG, "skin must be in [0, 10] and rebuild_every >= 0");
    if (prm->mode == MDPF_MODE_LEARNED && prm->mlp_kernel != MDPF_MLP_TENSOR && prm->mlp_kernel != MDPF_MLP_SIMT &&
        prm->mlp_kernel != MDPF_MLP_SIMT_FP32 && prm->mlp_kernel != MDPF_MLP_FUSED)
        return fail(nullptr, MDPF_ERR_INVALID_ARG, "unknown mlp_kernel");
    if (prm->mode == MDPF_MODE_LEARNED) {
        std::string msg;
        const int vrc = learned_validate(prm, msg);
        if (vrc != MDPF_OK) return fail(nullptr, vrc, msg);
    }
    if (!(prm->dt_fs > 0.0) || !std::isfinite(prm->dt_fs))
        return fail(nullptr, MDPF_ERR_INVALID_ARG, "dt_fs must be > 0");
    if (prm->trace_capacity < 0 || prm->record_every < 0 || prm->max_frames < 0)
        return fail(nullptr, MDPF_ERR_INVALID_ARG, "negative capacity");
    if (prm->stepper != MDPF_STEPPER_PERSISTENT && prm->stepper != MDPF_STEPPER_KERNELS)
        return fail(nullptr, MDPF_ERR_INVALID_ARG, "unknown stepper");
    if (prm->record_every > 0 && prm->max_frames <= 0)
        return fail(nullptr, MDPF_ERR_INVALID_ARG, "record_every needs max_frames > 0");
    if (prm->energy_every < 0) return fail(nullptr, MDPF_ERR_INVALID_ARG, "energy_every < 0");
    {
        const int ee = prm->energy_every > 0 ? prm->energy_every : 1;
        if (prm->record_every > 0 && prm->record_every % ee != 0)
            return fail(nullptr, MDPF_ERR_INVALID_ARG, "record_every must be a multiple of energy_every");
    }
    for (int i = 0; i < n; ++i) {
        if (t->element[i] < 0 || t->element[i] > 3)
            return fail(nullptr, MDPF_ERR_INVALID_ARG, "element out of range");
        if (!(t->mass[i] > 0.0) || !std::isfinite(t->mass[i]))
            return fail(nullptr, MDPF_ERR_INVALID_ARG, "mass must be > 0");
        if (!std::isfinite(t->charge[i])) return fail(nullptr, MDPF_ERR_INVALID_ARG, "charge not finite");
    }
    for (int b = 0; b < t->n_bonds; ++b) {
        int a = t->bonds[2 * b], c = t->bonds[2 * b + 1];
        if (a < 0 || a >= n || c < 0 || c >= n || a == c)
            return fail(nullptr, MDPF_ERR_INVALID_ARG, "bad bond index");
        if (!std::isfinite(t->bond_r0[b]) || !std::isfinite(t->bond_k[b]))
            return fail(nullptr, MDPF_ERR_INVALID_ARG, "bond parameter not finite");
    }
    for (int e = 0; e < 4; ++e)
        if (!(t->lj_sigma[e] >= 0.0) || !(t->lj_eps[e] >= 0.0))
            return fail(nullptr, MDPF_ERR_INVALID_ARG, "LJ parameters must be >= 0");

    mdpf_ctx *c = new mdpf_ctx();
    c->mode = prm->mode;
    c->n = n;
    c->n_pad = (n + kPad - 1) / kPad * kPad;
    c->n_tiles = c->n_pad / kTile;
    c->n_bonds = t->n_bonds;
    c->dt = prm->dt_fs;
    c->coulomb_k = prm->coulomb_k > 0 ? prm->coulomb_k : kCoulombDefault;
    c->trace_cap = prm->trace_capacity > 0 ? prm->trace_capacity : 4096;
    c->record_every = prm->record_every;
    c->max_frames = prm->max_frames;
    // learned and callback modes, and Langevin dynamics, always step with the per-step kernel sequence
    c->stepper = prm->mode == MDPF_MODE_PLAIN && prm->integrator == MDPF_INTEGRATOR_VERLET ? prm->stepper
                                                                                          : MDPF_STEPPER_KERNELS;
    if (prm->mode == MDPF_MODE_CALLBACK) {
        c->prov_fn = prm->provider;
        c->prov_user = prm->provider_user;
        c->prov_pos = prm->provider_pos;
        c->prov_energy = prm->provider_energy;
        c->prov_forces = prm->provider_forces;
    }
    c->energy_every = prm->energy_every > 0 ? prm->energy_every : 1;
    c->angle_k = (float)t->angle_k;
    c->angle_theta0 = (float)(t->angle_theta0_deg * M_PI / 180.0);
    c->h_mass.assign(t->mass, t->mass + n);

    auto bail = [&](int code) {
        std::string m = c->err;
        free_ctx(c);
        g_create_error = m;
        return code;
    };
#define CKC(x)                                                                           \
    do {                                                                                 \
        cudaError_t e_ = (x);                                                            \
        if (e_ != cudaSuccess) {                                                         \
            cuda_fail(c, e_, #x);                                                        \
            return bail(e_ == cudaErrorMemoryAllocation ? MDPF_ERR_OOM : MDPF_ERR_CUDA); \
        }                                                                                \
    } while (0)

    CKC(cudaGetDevice(&c->device));
    CKC(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    const int np = c->n_pad;
    // host-side preparation of per-atom constants
    std::vector<float> qs(np, 0.f);
    std::vector<float2> lj(np, make_float2(0.f, 0.f));
    std::vector<double> hdt(n);
    const double sk = std::sqrt(c->coulomb_k);
    for (int i = 0; i < n; ++i) {
        qs[i] = (float)(t->charge[i] * sk);
        lj[i] = make_float2((float)(0.5 * t->lj_sigma[t->element[i]]),
                            (float)std::sqrt(24.0 * t->lj_eps[t->element[i]]));
        hdt[i] = 0.5 * c->dt * kAcc / t->mass[i];
    }
    std::vector<int2> bonds(t->n_bonds);
    std::vector<float2> bpar(t->n_bonds);
    for (int b = 0; b < t->n_bonds; ++b) {
        bonds[b] = make_int2(t->bonds[2 * b], t->bonds[2 * b + 1]);
        bpar[b] = make_float2((float)t->bond_r0[b], (float)t->bond_k[b]);
    }
    CKC(dalloc(&c->d_element, n));
    CKC(dalloc(&c->d_mass, n));
    CKC(dalloc(&c->d_hdt_m, n));
    if (prm->integrator == MDPF_INTEGRATOR_LANGEVIN) {
        const double kB = 0.0019872041;   // kcal/mol/K
        c->lang_c1 = std::exp(-prm->friction_per_ps * 1e-3 * c->dt);
        c->lang_seed = prm->seed;
        std::vector<double> c2(n);
        for (int i = 0; i < n; ++i)
            c2[i] = std::sqrt((1.0 - c->lang_c1 * c->lang_c1) * kB * prm->temperature_K * kAcc / t->mass[i]);
        CKC(dalloc(&c->d_lang_c2, n));
        CKC(cudaMemcpy(c->d_lang_c2, c2.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    }
    CKC(dalloc(&c->d_pos4, np));
    CKC(dalloc(&c->d_pos4_c, np));
    CKC(dalloc(&c->d_lj, np));
    CKC(dalloc(&c->d_charge_s, np));
    CKC(dalloc(&c->d_bonds, t->n_bonds));
    CKC(dalloc(&c->d_bond_par, t->n_bonds));
    CKC(dalloc(&c->d_x, 3 * (size_t)n));
    CKC(dalloc(&c->d_v, 3 * (size_t)n));
    CKC(dalloc(&c->d_xc, 3 * (size_t)n));
    CKC(dalloc(&c->d_fc, 3 * (size_t)n));
    CKC(dalloc(&c->d_fx_base, 6 * (size_t)np));
    c->d_fx = c->d_fx_base;
    CKC(dalloc(&c->d_fx_c, 3 * (size_t)np));
    CKC(dalloc(&c->d_efx, E_SLOTS));
    CKC(dalloc(&c->d_efx_c, E_SLOTS));
    CKC(dalloc(&c->d_trace_u, c->trace_cap));
    CKC(dalloc(&c->d_trace_k, c->trace_cap));
    CKC(dalloc(&c->d_trace_step, c->trace_cap));
    CKC(dalloc(&c->d_trace_fb, c->trace_cap));
    CKC(cudaMemset(c->d_trace_fb, 0, sizeof(int64_t) * c->trace_cap));
    CKC(dalloc(&c->d_step, 1));
    CKC(dalloc(&c->d_status, 4));
    CKC(dalloc(&c->d_scalar, 16));
    CKC(dalloc(&c->d_barrier, 8));
    if (c->record_every > 0) {
        c->frames.cap = c->max_frames;
        c->frames.every = c->record_every;
        CKC(dalloc(&c->frames.pos, (size_t)c->max_frames * n * 3));
        CKC(dalloc(&c->frames.forces, (size_t)c->max_frames * n * 3));
        CKC(dalloc(&c->frames.energy, c->max_frames));
        CKC(dalloc(&c->frames.step, c->max_frames));
    }
    cudaStream_t s = c->stream;
    CKC(cudaMemcpyAsync(c->d_element, t->element, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    CKC(cudaMemcpyAsync(c->d_mass, t->mass, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CKC(cudaMemcpyAsync(c->d_hdt_m, hdt.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CKC(cudaMemcpyAsync(c->d_lj, lj.data(), sizeof(float2) * np, cudaMemcpyHostToDevice, s));
    CKC(cudaMemcpyAsync(c->d_charge_s, qs.data(), sizeof(float) * np, cudaMemcpyHostToDevice, s));
    if (t->n_bonds > 0) {
        CKC(cudaMemcpyAsync(c->d_bonds, bonds.data(), sizeof(int2) * t->n_bonds, cudaMemcpyHostToDevice, s));
        CKC(cudaMemcpyAsync(c->d_bond_par, bpar.data(), sizeof(float2) * t->n_bonds, cudaMemcpyHostToDevice, s));
    }
    CKC(cudaMemsetAsync(c->d_status, 0, sizeof(uint32_t) * 4, s));
    CKC(cudaMemsetAsync(c->d_step, 0, sizeof(int64_t), s));
    CKC(cudaMemsetAsync(c->d_barrier, 0, sizeof(unsigned int) * 8, s));
    CKC(cudaMemsetAsync(c->d_scalar, 0, sizeof(double) * 16, s));
    CKC(cudaMemsetAsync(c->d_x, 0, sizeof(double) * 3 * n, s));
    CKC(cudaMemsetAsync(c->d_v, 0, sizeof(double) * 3 * n, s));
    CKC(cudaMemsetAsync(c->d_fx_base, 0, sizeof(unsigned long long) * 6 * np, s));
    int rc = build_exclusions(c);
    if (rc != MDPF_OK) return bail(rc);
    if (c->mode == MDPF_MODE_LEARNED) {
        rc = learned_create(c, t, prm);
        if (rc != MDPF_OK) return bail(rc);
        // molecules of up to 32 atoms step in one persistent launch when the device allows it; otherwise the
        // per-step graph of the stage kernels stays in use
        if (prm->integrator == MDPF_INTEGRATOR_VERLET && prm->stepper == MDPF_STEPPER_PERSISTENT)
            small_create(c, t->element);
    }
    if (c->stepper == MDPF_STEPPER_PERSISTENT) {
        c->step_grid = stepper_grid(c);
        if (c->step_grid < 1) {
            fail(c, MDPF_ERR_UNSUPPORTED, "cooperative launch of the persistent stepper is not available");
            return bail(MDPF_ERR_UNSUPPORTED);
        }
        // bonded entries of each row group: every term once per atom it moves (bond: 2, angle: 3), so that
        // a group's owner computes every bonded force on its atoms; the angle list comes from the device
        std::vector<int4> angles(c->n_angles);
        if (c->n_angles > 0)
            CKC(cudaMemcpy(angles.data(), c->d_angles, sizeof(int4) * c->n_angles, cudaMemcpyDeviceToHost));
        const int NG = c->n_groups;
        std::vector<std::vector<int2>> ent(NG);
        auto add = [&](int atom, int term, int role) {
            ent[atom / 16].push_back(make_int2(term, ((atom % 16) << 2) | role));
        };
        for (int b = 0; b < t->n_bonds; ++b) {
            add(t->bonds[2 * b], b, 0);
            add(t->bonds[2 * b + 1], b, 1);
        }
        for (int k = 0; k < c->n_angles; ++k) {
            add(angles[k].x, t->n_bonds + k, 0);
            add(angles[k].y, t->n_bonds + k, 1);
            add(angles[k].z, t->n_bonds + k, 2);
        }
        std::vector<int> grp_off(NG + 1, 0), grp_aoff((size_t)NG * 17, 0);
        std::vector<int2> grp_flat;
        for (int g = 0; g < NG; ++g) {
            // by local atom (stable: term order within an atom), with each atom's range recorded
            std::stable_sort(ent[g].begin(), ent[g].end(),
                             [](const int2 &u, const int2 &v) { return (u.y >> 2) < (v.y >> 2); });
            for (size_t e = 0; e < ent[g].size(); ++e) grp_aoff[(size_t)g * 17 + (ent[g][e].y >> 2) + 1]++;
            for (int a = 0; a < 16; ++a) grp_aoff[(size_t)g * 17 + a + 1] += grp_aoff[(size_t)g * 17 + a];
            grp_flat.insert(grp_flat.end(), ent[g].begin(), ent[g].end());
            grp_off[g + 1] = (int)grp_flat.size();
        }
        grp_flat.push_back(make_int2(0, 0));
        CKC(dalloc(&c->d_part, 2 * (size_t)c->step_grid * 8));
        CKC(dalloc(&c->d_grp_off, NG + 1));
        CKC(dalloc(&c->d_grp_ent, grp_flat.size()));
        CKC(dalloc(&c->d_grp_aoff, grp_aoff.size()));
        CKC(cudaMemcpy(c->d_grp_aoff, grp_aoff.data(), sizeof(int) * grp_aoff.size(), cudaMemcpyHostToDevice));
        CKC(dalloc(&c->d_pos4_b, np));
        CKC(cudaMemset(c->d_pos4_b, 0, sizeof(float4) * np));   // padding atoms stay at finite positions
        CKC(cudaMemcpy(c->d_grp_off, grp_off.data(), sizeof(int) * (NG + 1), cudaMemcpyHostToDevice));
        CKC(cudaMemcpy(c->d_grp_ent, grp_flat.data(), sizeof(int2) * grp_flat.size(), cudaMemcpyHostToDevice));
    }
#undef CKC
    *out = c;
    return MDPF_OK;
}

void mdpf_destroy(mdpf_ctx *ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_ctx(ctx);
}

int mdpf_sizes(const mdpf_ctx *ctx, int32_t *n_atoms, int32_t *n_angles) {
    if (!ctx) return MDPF_ERR_INVALID_ARG;
    if (n_atoms) *n_atoms = ctx->n;
    if (n_angles) *n_angles = ctx->n_angles;
    return MDPF_OK;
}

// External provider evaluation at the FP64 device positions x into (fx, efx)
// (zeroed first when `zero`): positions into the caller's buffer, the host
// call, then the provider's FP32 forces and FP64 energy into fixed point.
static int enqueue_provider(mdpf_ctx *c, const double *x, unsigned long long *fx, unsigned long long *efx,
                            uint32_t *status, bool zero, cudaStream_t s) {
    if (zero) launch_zero_fx(fx, 3 * c->n_pad, efx, s);
    CK(c, cudaMemcpyAsync(c->prov_pos, x, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToDevice, s));
    const int rc = c->prov_fn(c->prov_user, (void *)s);
    if (rc != 0) return fail(c, MDPF_ERR_CALLBACK, "the force provider returned " + std::to_string(rc));
    launch_provider_to_fx(c->prov_forces, c->prov_energy, c->n, fx, efx, status, s);
    CK(c, cudaGetLastError());
    return MDPF_OK;
}

// Force evaluation into (fx, efx) at the FP32 positions pos4 (learned mode:
// with a fresh neighbour list).
static int enqueue_forces(mdpf_ctx *c, const float4 *pos4, unsigned long long *fx, unsigned long long *efx,
                          uint32_t *status, bool energy, cudaStream_t s, bool zeroed = false) {
    if (!zeroed) launch_zero_fx(fx, 3 * c->n_pad, efx, s);
    if (c->mode == MDPF_MODE_LEARNED) return learned_enqueue_forces(c, pos4, fx, efx, status, true, false, s);
    PlainDev p = plain_dev(c, pos4);
    p.status = status;
    launch_bonded(p, fx, energy ? efx : nullptr, s);
    launch_nonbonded(p, fx, efx, energy, s);
    return MDPF_OK;
}

int mdpf_compute_device(mdpf_ctx *c, const double *d_pos, double *d_energy, float *d_forces, void *stream) {
    GUARD(c);
    if (!d_pos) return fail(c, MDPF_ERR_INVALID_ARG, "d_pos is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    // positions and cleared sums in one launch; forces, energy terms and the caller's energy in one
    launch_eval_begin(d_pos, c->d_charge_s, c->d_pos4_c, c->n, c->n_pad, c->d_fx_c, 3 * c->n_pad, c->d_efx_c, s);
    {
        const int rc = c->mode == MDPF_MODE_CALLBACK
                           ? enqueue_provider(c, d_pos, c->d_fx_c, c->d_efx_c, c->d_status + 1, false, s)
                           : enqueue_forces(c, c->d_pos4_c, c->d_fx_c, c->d_efx_c, c->d_status + 1, true, s, true);
        if (rc != MDPF_OK) return rc;
    }
    launch_eval_end(c->d_fx_c, c->n, d_forces, c->d_efx_c, c->d_scalar + 2, d_energy, s);
    CK(c, cudaGetLastError());
    return MDPF_OK;
}

int mdpf_compute(mdpf_ctx *c, const double *pos, double *energy, double *forces, double *terms) {
    GUARD(c);
    if (!pos) return fail(c, MDPF_ERR_INVALID_ARG, "pos is NULL");
    cudaStream_t s = c->stream;
    CK(c, cudaMemsetAsync(c->d_status + 1, 0, sizeof(uint32_t), s));
    CK(c, cudaMemcpyAsync(c->d_xc, pos, sizeof(double) * 3 * c->n, cudaMemcpyHostToDevice, s));
    launch_pos4_from_x(c->d_xc, c->d_charge_s, c->d_pos4_c, c->n, c->n_pad, s);
    {
        const int rc = c->mode == MDPF_MODE_CALLBACK
                           ? enqueue_provider(c, c->d_xc, c->d_fx_c, c->d_efx_c, c->d_status + 1, true, s)
                           : enqueue_forces(c, c->d_pos4_c, c->d_fx_c, c->d_efx_c, c->d_status + 1, true, s);
        if (rc != MDPF_OK) return rc;
    }
    launch_fx_to_forces(c->d_fx_c, c->n, c->d_fc, nullptr, s);
    launch_energy_out(c->d_efx_c, c->d_scalar + 2, s);
    CK(c, cudaGetLastError());
    double e6[6];
    uint32_t st = 0;
    if (forces) CK(c, cudaMemcpyAsync(forces, c->d_fc, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToHost, s));
    CK(c, cudaMemcpyAsync(e6, c->d_scalar + 2, sizeof(double) * 6, cudaMemcpyDeviceToHost, s));
    CK(c, cudaMemcpyAsync(&st, c->d_status + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    if (energy) *energy = e6[0];
    if (terms) std::memcpy(terms, e6 + 1, sizeof(double) * 4);
    if ((st & MDPF_STATUS_NONFINITE) || !std::isfinite(e6[0]))
        return fail(c, MDPF_ERR_NONFINITE, "non-finite energy or forces");
    if (st & MDPF_STATUS_NEIGHBOR_OVERFLOW) return fail(c, MDPF_ERR_NEIGHBOR_OVERFLOW, "neighbour list overflow");
    if (st & MDPF_STATUS_OUT_OF_RANGE) return fail(c, MDPF_ERR_OUT_OF_RANGE, "features out of training range");
    return MDPF_OK;
}

int mdpf_set_state(mdpf_ctx *c, const double *pos, const double *vel) {
    GUARD(c);
    if (!pos || !vel) return fail(c, MDPF_ERR_INVALID_ARG, "pos or vel is NULL");
    cudaStream_t s = c->stream;
    CK(c, cudaMemcpyAsync(c->d_x, pos, sizeof(double) * 3 * c->n, cudaMemcpyHostToDevice, s));
    CK(c, cudaMemcpyAsync(c->d_v, vel, sizeof(double) * 3 * c->n, cudaMemcpyHostToDevice, s));
    CK(c, cudaMemsetAsync(c->d_status, 0, sizeof(uint32_t), s));
    CK(c, cudaMemsetAsync(c->d_step, 0, sizeof(int64_t), s));
    launch_pos4_from_x(c->d_x, c->d_charge_s, c->d_pos4, c->n, c->n_pad, s);
    {
        const int rc = c->mode == MDPF_MODE_CALLBACK
                           ? enqueue_provider(c, c->d_x, c->d_fx, c->d_efx, c->d_status, true, s)
                           : enqueue_forces(c, c->d_pos4, c->d_fx, c->d_efx, c->d_status, true, s);
        if (rc != MDPF_OK) return rc;
    }
    launch_kinetic(c, s);
    launch_energy_out(c->d_efx, c->d_scalar + 2, s);
    CK(c, cudaGetLastError());
    double e6[6];
    uint32_t st = 0;
    CK(c, cudaMemcpyAsync(e6, c->d_scalar + 2, sizeof(double) * 6, cudaMemcpyDeviceToHost, s));
    CK(c, cudaMemcpyAsync(&st, c->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    double uk[2] = {e6[0], e6[5]};
    CK(c, cudaMemcpy(c->d_scalar, uk, sizeof(double) * 2, cudaMemcpyHostToDevice));
    c->h_initial = e6[0] + e6[5];
    c->steps = 0;
    c->force_evals = 0;
    c->state_set = true;
    if ((st & MDPF_STATUS_NONFINITE) || !std::isfinite(c->h_initial))
        return fail(c, MDPF_ERR_NONFINITE, "non-finite initial energy");
    if (st & MDPF_STATUS_NEIGHBOR_OVERFLOW) return fail(c, MDPF_ERR_NEIGHBOR_OVERFLOW, "neighbour list overflow");
    if (st & MDPF_STATUS_OUT_OF_RANGE) return fail(c, MDPF_ERR_OUT_OF_RANGE, "features out of training range");
    return MDPF_OK;
}

int mdpf_get_state(mdpf_ctx *c, double *pos, double *vel) {
    GUARD(c);
    cudaStream_t s = c->stream;
    if (pos) CK(c, cudaMemcpyAsync(pos, c->d_x, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToHost, s));
    if (vel) CK(c, cudaMemcpyAsync(vel, c->d_v, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    return MDPF_OK;
}

// One learned-mode MD step: kick-drift, rebuild check, learned forces, kick.
static int enqueue_learned_step(mdpf_ctx *c, bool energy, cudaStream_t s) {
    launch_kick_drift(c, s);   // also requests a list rebuild when one is due
    cudaEvent_t pn = prof_begin(c, s);
    const int rc = learned_enqueue_forces(c, c->d_pos4, c->d_fx, c->d_efx, c->d_status, false, false, s);
    if (rc != MDPF_OK) return rc;
    prof_end(c, MDPF_PROF_NONBONDED, pn, s);
    launch_kick_finish(c, energy, s);
    return MDPF_OK;
}

// The learned step as a CUDA graph (index 1: energy step), captured once on
// the context's own stream; null when capture is not available, in which
// case the same kernels are launched one by one.
static cudaGraphExec_t learned_step_graph(mdpf_ctx *c, bool energy) {
    const int k = energy ? 1 : 0;
    if (c->lgraph[k] != nullptr || c->lgraph_failed) return c->lgraph[k];
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    bool ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        const int rc = enqueue_learned_step(c, energy, c->stream);
        const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        ok = rc == MDPF_OK && e == cudaSuccess && g != nullptr;
    }
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();   // capture errors are not sticky; clear them
    if (!ok) {
        if (ex) cudaGraphExecDestroy(ex);
        c->lgraph_failed = true;
        c->err.clear();
        c->sticky = false;
        return nullptr;
    }
    c->lgraph[k] = ex;
    return ex;
}

static int enqueue_steps(mdpf_ctx *c, int64_t n_steps, cudaStream_t s) {
    if (n_steps == 0) return MDPF_OK;
    if (c->small != nullptr) {
        cudaEvent_t ps = prof_begin(c, s);
        CK(c, launch_learned_small(c, n_steps, s));
        prof_end(c, MDPF_PROF_STEPPER, ps, s);
        c->steps += n_steps;
        c->force_evals += n_steps;
        return MDPF_OK;
    }
    if (c->stepper == MDPF_STEPPER_PERSISTENT) {
        cudaEvent_t ps = prof_begin(c, s);
        CK(c, launch_plain_persistent(c, n_steps, s));
        prof_end(c, MDPF_PROF_STEPPER, ps, s);
        c->steps += n_steps;
        c->force_evals += n_steps;
        return MDPF_OK;
    }
    cudaEvent_t ps = prof_begin(c, s);
    for (int64_t k = 0; k < n_steps; ++k) {
        const bool energy = (c->steps + k + 1) % c->energy_every == 0;
        if (c->mode == MDPF_MODE_CALLBACK) {
            launch_kick_drift(c, s);   // also zeroes the force and energy sums
            const int rc = enqueue_provider(c, c->d_x, c->d_fx, c->d_efx, c->d_status, false, s);
            if (rc != MDPF_OK) return rc;
            launch_kick_finish(c, energy, s);
            continue;
        }
        if (c->mode == MDPF_MODE_LEARNED) {
            cudaGraphExec_t ex = c->profiling ? nullptr : learned_step_graph(c, energy);
            if (ex != nullptr) {
                CK(c, cudaGraphLaunch(ex, s));
            } else {
                const int rc = enqueue_learned_step(c, energy, s);
                if (rc != MDPF_OK) return rc;
            }
            continue;
        }
        launch_kick_drift(c, s);
        PlainDev p = plain_dev(c, c->d_pos4);
        launch_bonded(p, c->d_fx, energy ? c->d_efx : nullptr, s);
        cudaEvent_t pn = prof_begin(c, s);
        launch_nonbonded(p, c->d_fx, c->d_efx, energy, s);
        prof_end(c, MDPF_PROF_NONBONDED, pn, s);
        launch_kick_finish(c, energy, s);
    }
    prof_end(c, MDPF_PROF_STEP, ps, s);
    CK(c, cudaGetLastError());
    c->steps += n_steps;
    c->force_evals += n_steps;
    return MDPF_OK;
}

static int status_to_code(mdpf_ctx *c, uint32_t st) {
    if (st & MDPF_STATUS_TIMEOUT) return fail(c, MDPF_ERR_TIMEOUT, "device-side wait timed out");
    if (st & MDPF_STATUS_NONFINITE) return fail(c, MDPF_ERR_NONFINITE, "energy or state became non-finite");
    if (st & MDPF_STATUS_NEIGHBOR_OVERFLOW) return fail(c, MDPF_ERR_NEIGHBOR_OVERFLOW, "neighbour list overflow");
    if (st & MDPF_STATUS_OUT_OF_RANGE) return fail(c, MDPF_ERR_OUT_OF_RANGE, "features out of training range");
    return MDPF_OK;
}

int mdpf_step(mdpf_ctx *c, int64_t n_steps) {
    GUARD(c);
    if (n_steps < 0) return fail(c, MDPF_ERR_INVALID_ARG, "n_steps < 0");
    if (!c->state_set) return fail(c, MDPF_ERR_INVALID_ARG, "mdpf_set_state has not been called");
    int rc = enqueue_steps(c, n_steps, c->stream);
    if (rc != MDPF_OK) return rc;
    uint32_t st = 0;
    CK(c, cudaMemcpyAsync(&st, c->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return status_to_code(c, st);
}

int mdpf_step_async(mdpf_ctx *c, int64_t n_steps, void *stream) {
    GUARD(c);
    if (n_steps < 0) return fail(c, MDPF_ERR_INVALID_ARG, "n_steps < 0");
    if (!c->state_set) return fail(c, MDPF_ERR_INVALID_ARG, "mdpf_set_state has not been called");
    return enqueue_steps(c, n_steps, (cudaStream_t)stream);
}

int mdpf_get_counters(mdpf_ctx *c, mdpf_counters *out) {
    GUARD(c);
    if (!out) return fail(c, MDPF_ERR_INVALID_ARG, "out is NULL");
    double uk[2];
    uint32_t st = 0;
    int64_t dstep = 0;
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaMemcpy(uk, c->d_scalar, sizeof(double) * 2, cudaMemcpyDeviceToHost));
    CK(c, cudaMemcpy(&st, c->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    CK(c, cudaMemcpy(&dstep, c->d_step, sizeof(int64_t), cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(*out));
    out->steps = dstep;
    out->force_evals = c->force_evals;
    out->frames = c->record_every > 0 ? dstep / c->record_every : 0;
    out->status = st;
    out->potential = uk[0];
    out->kinetic = uk[1];
    out->h_initial = c->h_initial;
    out->h_now = uk[0] + uk[1];
    if (c->learned != nullptr) {
        const int rc = learned_counter_values(c, &out->rebuilds, &out->fallbacks, &out->max_disp);
        if (rc != MDPF_OK) return rc;
    }
    return MDPF_OK;
}

int mdpf_init_velocities(mdpf_ctx *c, double temperature_K, uint64_t seed) {
    GUARD(c);
    if (!(temperature_K >= 0.0) || !std::isfinite(temperature_K))
        return fail(c, MDPF_ERR_INVALID_ARG, "temperature must be finite and >= 0");
    if (!c->state_set) return fail(c, MDPF_ERR_INVALID_ARG, "set the state (positions) with mdpf_set_state first");
    cudaStream_t s = c->stream;
    launch_init_velocities(c, temperature_K, (unsigned long long)seed, s);
    // K of the new velocities (fixed-point slot, as everywhere else) and H0 = U + K
    CK(c, cudaMemsetAsync(c->d_efx + E_KIN, 0, sizeof(unsigned long long), s));
    launch_kinetic(c, s);
    CK(c, cudaGetLastError());
    unsigned long long kfx = 0;
    double u = 0;
    CK(c, cudaMemcpyAsync(&kfx, c->d_efx + E_KIN, sizeof(kfx), cudaMemcpyDeviceToHost, s));
    CK(c, cudaMemcpyAsync(&u, c->d_scalar, sizeof(u), cudaMemcpyDeviceToHost, s));
    CK(c, cudaStreamSynchronize(s));
    const double k = (double)(long long)kfx * kFxInv;
    CK(c, cudaMemcpy(c->d_scalar + 1, &k, sizeof(k), cudaMemcpyHostToDevice));
    c->h_initial = u + k;
    return MDPF_OK;
}

int mdpf_get_trace(mdpf_ctx *c, double *U, double *K, int64_t *step, int64_t max_n, int64_t *n_out) {
    GUARD(c);
    if (max_n < 0) return fail(c, MDPF_ERR_INVALID_ARG, "max_n < 0");
    int64_t dstep = 0;
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaMemcpy(&dstep, c->d_step, sizeof(int64_t), cudaMemcpyDeviceToHost));
    const int64_t n_energy = dstep / c->energy_every;
    int64_t cnt = n_energy < c->trace_cap ? n_energy : c->trace_cap;
    if (cnt > max_n) cnt = max_n;
    std::vector<double> hu(c->trace_cap), hk(c->trace_cap);
    std::vector<int64_t> hs(c->trace_cap);
    CK(c, cudaMemcpy(hu.data(), c->d_trace_u, sizeof(double) * c->trace_cap, cudaMemcpyDeviceToHost));
    CK(c, cudaMemcpy(hk.data(), c->d_trace_k, sizeof(double) * c->trace_cap, cudaMemcpyDeviceToHost));
    CK(c, cudaMemcpy(hs.data(), c->d_trace_step, sizeof(int64_t) * c->trace_cap, cudaMemcpyDeviceToHost));
    int64_t start = n_energy - cnt;
    for (int64_t k = 0; k < cnt; ++k) {
        int64_t slot = (start + k) % c->trace_cap;
        if (U) U[k] = hu[slot];
        if (K) K[k] = hk[slot];
        if (step) step[k] = hs[slot];
    }
    if (n_out) *n_out = cnt;
    return MDPF_OK;
}

int mdpf_get_trace_fallbacks(mdpf_ctx *c, int64_t *fallbacks, int64_t max_n, int64_t *n_out) {
    GUARD(c);
    if (max_n < 0) return fail(c, MDPF_ERR_INVALID_ARG, "max_n < 0");
    int64_t dstep = 0;
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaMemcpy(&dstep, c->d_step, sizeof(int64_t), cudaMemcpyDeviceToHost));
    const int64_t n_energy = dstep / c->energy_every;
    int64_t cnt = n_energy < c->trace_cap ? n_energy : c->trace_cap;
    if (cnt > max_n) cnt = max_n;
    std::vector<int64_t> hf(c->trace_cap);
    CK(c, cudaMemcpy(hf.data(), c->d_trace_fb, sizeof(int64_t) * c->trace_cap, cudaMemcpyDeviceToHost));
    const int64_t start = n_energy - cnt;
    for (int64_t k = 0; k < cnt; ++k)
        if (fallbacks) fallbacks[k] = hf[(start + k) % c->trace_cap];
    if (n_out) *n_out = cnt;
    return MDPF_OK;
}

int mdpf_get_frames(mdpf_ctx *c, int64_t max_n, double *pos, double *energy, float *forces, int64_t *step,
                    int64_t *n_out) {
    GUARD(c);
    if (max_n < 0) return fail(c, MDPF_ERR_INVALID_ARG, "max_n < 0");
    if (n_out) *n_out = 0;
    if (c->record_every <= 0) return MDPF_OK;
    int64_t dstep = 0;
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaMemcpy(&dstep, c->d_step, sizeof(int64_t), cudaMemcpyDeviceToHost));
    int64_t total = dstep / c->record_every;
    int64_t cnt = total < c->frames.cap ? total : c->frames.cap;
    if (cnt > max_n) cnt = max_n;
    const size_t n3 = 3 * (size_t)c->n;
    for (int64_t k = 0; k < cnt; ++k) {
        int64_t f = total - cnt + k;
        int slot = (int)(f % c->frames.cap);
        if (pos)
            CK(c, cudaMemcpy(pos + k * n3, c->frames.pos + slot * n3, sizeof(double) * n3, cudaMemcpyDeviceToHost));
        if (forces)
            CK(c, cudaMemcpy(forces + k * n3, c->frames.forces + slot * n3, sizeof(float) * n3,
                             cudaMemcpyDeviceToHost));
        if (energy) CK(c, cudaMemcpy(energy + k, c->frames.energy + slot, sizeof(double), cudaMemcpyDeviceToHost));
        if (step) CK(c, cudaMemcpy(step + k, c->frames.step + slot, sizeof(int64_t), cudaMemcpyDeviceToHost));
    }
    if (n_out) *n_out = cnt;
    return MDPF_OK;
}

int mdpf_get_exclusions(mdpf_ctx *c, int32_t *offset, int32_t *idx, int64_t capacity, int64_t *total) {
    GUARD(c);
    if (total) *total = c->excl_total;
    if (offset) CK(c, cudaMemcpy(offset, c->d_excl_off, sizeof(int32_t) * (c->n + 1), cudaMemcpyDeviceToHost));
    if (idx) {
        if (capacity < c->excl_total) return fail(c, MDPF_ERR_INVALID_ARG, "capacity too small");
        if (c->excl_total > 0)
            CK(c, cudaMemcpy(idx, c->d_excl_idx, sizeof(int32_t) * c->excl_total, cudaMemcpyDeviceToHost));
    }
    return MDPF_OK;
}

int mdpf_get_angles(mdpf_ctx *c, int32_t *angles, int64_t capacity, int64_t *n_out) {
    GUARD(c);
    if (n_out) *n_out = c->n_angles;
    if (angles) {
        if (capacity < c->n_angles) return fail(c, MDPF_ERR_INVALID_ARG, "capacity too small");
        std::vector<int4> h(c->n_angles);
        if (c->n_angles > 0)
            CK(c, cudaMemcpy(h.data(), c->d_angles, sizeof(int4) * c->n_angles, cudaMemcpyDeviceToHost));
        for (int k = 0; k < c->n_angles; ++k) {
            angles[3 * k] = h[k].x;
            angles[3 * k + 1] = h[k].y;
            angles[3 * k + 2] = h[k].z;
        }
    }
    return MDPF_OK;
}

int mdpf_debug_set_status(mdpf_ctx *c, uint32_t bits) {
    GUARD(c);
    uint32_t st = 0;
    CK(c, cudaStreamSynchronize(c->stream));
    CK(c, cudaMemcpy(&st, c->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    st = bits == 0 ? 0u : (st | bits);
    CK(c, cudaMemcpy(c->d_status, &st, sizeof(uint32_t), cudaMemcpyHostToDevice));
    return MDPF_OK;
}

int mdpf_debug_wait_timeout(mdpf_ctx *c, int32_t limit_us) {
    GUARD(c);
    if (limit_us < 1 || limit_us > 2000000) return fail(c, MDPF_ERR_INVALID_ARG, "limit_us out of [1, 2e6]");
    CK(c, cudaMemsetAsync(c->d_barrier + 7, 0, sizeof(unsigned int), c->stream));
    launch_wait_timeout(c->d_status, c->d_barrier + 7, (long long)limit_us * 1000LL, c->stream);
    CK(c, cudaGetLastError());
    uint32_t st = 0;
    CK(c, cudaMemcpyAsync(&st, c->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return status_to_code(c, st);
}

int mdpf_set_profiling(mdpf_ctx *c, int32_t enable) {
    GUARD(c);
    int rc = prof_harvest(c);
    if (rc != MDPF_OK) return rc;
    for (int k = 0; k < MDPF_PROF_SLOTS; ++k) {
        c->prof_ms[k] = 0.0;
        c->prof_n[k] = 0;
    }
    c->profiling = enable != 0;
    return MDPF_OK;
}

int mdpf_get_profile(mdpf_ctx *c, int32_t slot, double *total_ms, int64_t *launches) {
    GUARD(c);
    if (slot < 0 || slot >= MDPF_PROF_SLOTS) return fail(c, MDPF_ERR_INVALID_ARG, "bad profile slot");
    int rc = prof_harvest(c);
    if (rc != MDPF_OK) return rc;
    if (total_ms) *total_ms = c->prof_ms[slot];
    if (launches) *launches = c->prof_n[slot];
    return MDPF_OK;
}

}  // extern "C"
