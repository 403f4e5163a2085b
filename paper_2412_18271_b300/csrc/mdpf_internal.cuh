// Internal declarations shared by the CUDA sources of libmdpf.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mdpf.h"

namespace mdpf {

// (kcal/mol/A/amu) -> A/fs^2, i.e. 1 kcal/mol = 4.184e-4 amu A^2/fs^2.
constexpr double kAcc = 4.184e-4;
constexpr double kCoulombDefault = 332.06371;

// Fixed-point accumulation of forces and energies: value * 2^32 in int64.
// Integer addition is associative, so results do not depend on the order in
// which threads add their contributions.
constexpr double kFxScale = 4294967296.0;
constexpr double kFxInv = 1.0 / 4294967296.0;

constexpr int kTile = 32;          // atoms per tile (one per lane)
constexpr int kPad = 64;           // atoms are padded to a multiple of 64 (two tiles)
constexpr int kMaxExclPerAtom = 255;

// Energy slot layout (int64 fixed point): bond, angle, LJ, Coulomb, kinetic, learned.
// E_LEARN holds the learned model's energy, or the external provider's in callback mode.
enum { E_BOND = 0, E_ANGLE = 1, E_LJ = 2, E_COUL = 3, E_KIN = 4, E_LEARN = 5, E_SLOTS = 8 };

__host__ __device__ inline int64_t tile_pair_index(int I, int J, int T) {
    // upper triangle (I <= J), row-major
    return (int64_t)I * T - (int64_t)I * (I - 1) / 2 + (J - I);
}

// Per-system constant data on the device (plain path).
struct PlainDev {
    int n, n_pad, n_tiles;
    int n_bonds, n_angles;
    const float4 *pos4;      // x, y, z, q*sqrt(ke)   [n_pad]
    const float2 *lj;        // sigma/2, sqrt(24 eps)  [n_pad]
    const int2 *bonds;       // [n_bonds]
    const float2 *bond_par;  // r0, k                  [n_bonds]
    const int4 *angles;      // a, v, b, 0             [n_angles]
    float angle_k, angle_theta0;
    const uint32_t *tile_mask;  // [n_tile_pairs][32]: bit j of word i set = pair skipped
    const uint32_t *tile_flag;  // [n_tile_pairs]: 1 if any bit set in the tile
    const int4 *items;          // [n_items] work items of the Newton-pair tile sum (forcefield.cuh)
    int n_items;
    // row decomposition of the all-pairs sum (forcefield.cuh): groups of 16 i-atoms, chunks of 32 j-atoms
    int n_groups, n_chunks;
    const uint32_t *row_mask;   // [n_groups][n_chunks][16]: bit l of word a set = pair (16g+a, 32c+l) skipped
    const int *grp_off;         // [n_groups + 1] bonded entries of each group (CSR)
    const int2 *grp_ent;        // (term, (local atom << 2) | role): role 0, 1, 2 = the term's atom r.x, r.y, r.z;
                                // sorted by local atom within a group
    const int *grp_aoff;        // [n_groups][17]: entries of local atom a are [grp_aoff[a], grp_aoff[a+1]) of the group
    uint32_t *status;           // device status word
    const unsigned int *gate;   // if set, the kernels run only when *gate != 0 (learned-mode fallback)
};

// Langevin (BAOAB) parameters for the kick-drift kernel; c2 == null: velocity Verlet.
struct LangevinDev {
    const double *c2;        // [n] sqrt((1 - c1^2) kB T / m) in A/fs
    double c1;               // exp(-gamma dt)
    unsigned long long seed;
    const int64_t *step;     // completed steps (the noise counter)
};

// Learned mode: the neighbour-list displacement check done in the kick-drift kernel.
struct DispCheck {
    const float4 *pos_build;   // positions at the last list build, or null (no check)
    unsigned int *flag;        // set to request a rebuild
    float half_skin2;          // (skin / 2)^2
    int rebuild_every;         // also request one when the completed-step count is a multiple of this
};

struct Frames {
    double *pos;      // [cap][n][3]
    double *energy;   // [cap]
    float *forces;    // [cap][n][3]
    int64_t *step;    // [cap]
    int cap;
    int every;
};

}  // namespace mdpf

struct mdpf_ctx {
    int device = 0;
    int mode = MDPF_MODE_PLAIN;
    int n = 0, n_pad = 0, n_tiles = 0, n_bonds = 0, n_angles = 0;
    double dt = 0.5, coulomb_k = mdpf::kCoulombDefault;
    int trace_cap = 4096;
    int record_every = 0, max_frames = 0, energy_every = 1;
    int stepper = 0;                       // 0 persistent, 1 per-step kernel sequence
    int64_t excl_total = 0;

    // topology on the device
    int32_t *d_element = nullptr;
    double *d_mass = nullptr;
    double *d_hdt_m = nullptr;      // dt/2 * kAcc / m  [n]
    float4 *d_pos4 = nullptr;       // state positions, FP32 copy for force kernels
    float4 *d_pos4_b = nullptr;     // second position buffer of the persistent stepper
    float4 *d_pos4_c = nullptr;     // compute() positions
    float2 *d_lj = nullptr;
    float *d_charge_s = nullptr;    // q * sqrt(ke) [n_pad]
    int2 *d_bonds = nullptr;
    float2 *d_bond_par = nullptr;
    int4 *d_angles = nullptr;
    int32_t *d_excl_off = nullptr;
    int32_t *d_excl_idx = nullptr;
    uint32_t *d_row_mask = nullptr;        // [n_groups][n_chunks][16] skip masks of the row decomposition
    int *d_grp_off = nullptr;              // [n_groups + 1] bonded entries per row group
    int2 *d_grp_ent = nullptr;
    int *d_grp_aoff = nullptr;             // [n_groups][17] per-atom entry ranges within a group
    int n_groups = 0, n_chunks = 0;        // row groups (16 atoms) and j-chunks (32 atoms) holding real atoms
    float angle_k = 0, angle_theta0 = 0;

    // integrator state
    double *d_x = nullptr;          // [n][3]
    double *d_v = nullptr;          // [n][3]
    unsigned long long *d_fx_base = nullptr; // [2][n_pad][3] fixed-point force buffers
    unsigned long long *d_fx = nullptr;      // = d_fx_base: forces at the current x (state)
    unsigned long long *d_fx_c = nullptr;    // compute() forces
    unsigned long long *d_efx = nullptr;     // [E_SLOTS] fixed-point energies (state)
    unsigned long long *d_efx_c = nullptr;   // compute() energies
    double *d_trace_u = nullptr, *d_trace_k = nullptr;
    int64_t *d_trace_step = nullptr;
    int64_t *d_trace_fb = nullptr;         // learned mode: fallback evaluations so far, per trace entry
    int64_t *d_step = nullptr;             // device step counter
    uint32_t *d_status = nullptr;          // [0] state, [1] compute(), [3] block ticket of the kick-finish kernel
    double *d_xc = nullptr;                // compute() FP64 position staging [n][3]
    double *d_fc = nullptr;                // compute() FP64 forces out [n][3]
    double *d_scalar = nullptr;            // [16]: [0] U, [1] K of the state; [2..7] compute outputs
    unsigned int *d_barrier = nullptr;     // [8]: [0..1] grid-barrier counter (u64), [7] timeout flag
    mdpf::Frames frames{};

    // persistent stepper
    long long *d_part = nullptr;           // [2][step_grid][8] per-block energies (fixed point)
    int step_grid = 0;                     // blocks of the persistent stepper

    // Langevin (BAOAB) integrator: per-atom noise amplitude, damping factor, seed
    double *d_lang_c2 = nullptr;
    double lang_c1 = 1.0;
    unsigned long long lang_seed = 0;

    // callback mode: the caller's force provider and its device buffers
    mdpf_force_fn prov_fn = nullptr;
    void *prov_user = nullptr;
    double *prov_pos = nullptr, *prov_energy = nullptr;
    float *prov_forces = nullptr;

    // learned mode (learned_host.cu)
    void *learned = nullptr;               // mdpf::LearnedHost
    void *small = nullptr;                 // mdpf::SmallBuf: the persistent small-molecule stepper (small.cu), or null
    cudaGraphExec_t lgraph[2] = {nullptr, nullptr};   // learned step as a graph: [0] plain step, [1] energy step
    bool lgraph_failed = false;

    int64_t steps = 0, force_evals = 0;
    double h_initial = 0;
    bool state_set = false;

    cudaStream_t stream = nullptr;
    // profiling: event pairs recorded around launches of profiled kernels
    bool profiling = false;
    struct ProfRec {
        int slot;
        cudaEvent_t a, b;
    };
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> prof_free;
    double prof_ms[MDPF_PROF_SLOTS] = {0};
    int64_t prof_n[MDPF_PROF_SLOTS] = {0};
    std::vector<double> h_mass;
    std::string err;
    bool sticky = false;
};

namespace mdpf {

// status helpers (api.cu)
int fail(mdpf_ctx *ctx, int code, const std::string &msg);
int cuda_fail(mdpf_ctx *ctx, cudaError_t e, const char *where);

// profiling (api.cu): bracket a launch with events when profiling is on
cudaEvent_t prof_begin(mdpf_ctx *ctx, cudaStream_t s);
void prof_end(mdpf_ctx *ctx, int slot, cudaEvent_t a, cudaStream_t s);
int prof_harvest(mdpf_ctx *ctx);

// exclusions.cu
int build_exclusions(mdpf_ctx *ctx);

// plain.cu
PlainDev plain_dev(const mdpf_ctx *ctx, const float4 *pos4);
void launch_zero_fx(unsigned long long *fx, int n3, unsigned long long *efx, cudaStream_t s);
void launch_pos4_from_x(const double *x, const float *charge_s, float4 *pos4, int n, int n_pad, cudaStream_t s);
void launch_bonded(const PlainDev &p, unsigned long long *fx, unsigned long long *efx, cudaStream_t s);
void launch_nonbonded(const PlainDev &p, unsigned long long *fx, unsigned long long *efx, bool energy,
                      cudaStream_t s);
void launch_fx_to_forces(const unsigned long long *fx, int n, double *f64, float *f32, cudaStream_t s);
void launch_energy_out(const unsigned long long *efx, double *out6, cudaStream_t s);
// a single evaluation's first and last launches: positions and cleared sums; forces, energy terms and total
void launch_eval_begin(const double *x, const float *qs, float4 *pos4, int n, int n_pad, unsigned long long *fx,
                       int n3, unsigned long long *efx, cudaStream_t s);
void launch_eval_end(const unsigned long long *fx, int n, float *f32, const unsigned long long *efx, double *out6,
                     double *energy, cudaStream_t s);
void launch_kick_drift(mdpf_ctx *ctx, cudaStream_t s);
void launch_kick_finish(mdpf_ctx *ctx, bool energy, cudaStream_t s);
void launch_kinetic(mdpf_ctx *ctx, cudaStream_t s);
void launch_provider_to_fx(const float *forces, const double *energy, int n, unsigned long long *fx,
                           unsigned long long *efx, uint32_t *status, cudaStream_t s);
void launch_wait_timeout(uint32_t *status, unsigned int *flag, long long limit_ns, cudaStream_t s);
// Maxwell-Boltzmann velocities of the current positions into d_v (one block)
void launch_init_velocities(mdpf_ctx *ctx, double temperature_K, unsigned long long seed, cudaStream_t s);

// learned_host.cu
int learned_validate(const mdpf_params *prm, std::string &msg);
int learned_create(mdpf_ctx *ctx, const mdpf_topology *t, const mdpf_params *prm);
void learned_free(mdpf_ctx *ctx);
int learned_enqueue_forces(mdpf_ctx *ctx, const float4 *pos4, unsigned long long *fx, unsigned long long *efx,
                           uint32_t *status, bool forced_build, bool write_f32, cudaStream_t s);
DispCheck learned_disp_check(const mdpf_ctx *ctx);
int learned_counter_values(mdpf_ctx *ctx, int64_t *rebuilds, int64_t *fallbacks, double *max_disp);
// device counter of evaluations that fell back to the plain force field (learned mode), else null
const long long *learned_fallback_counter(const mdpf_ctx *ctx);

// small.cu: the persistent learned stepper for molecules of up to 32 atoms
int small_create(mdpf_ctx *ctx, const int32_t *element);   // MDPF_OK, or MDPF_ERR_UNSUPPORTED (not used then)
void small_free(mdpf_ctx *ctx);
cudaError_t launch_learned_small(mdpf_ctx *ctx, int64_t n_steps, cudaStream_t s);

// stepper.cu
int stepper_grid(const mdpf_ctx *ctx);
cudaError_t launch_plain_persistent(mdpf_ctx *ctx, int64_t n_steps, cudaStream_t s);

}  // namespace mdpf
