/*
 * mdpf.h -- C ABI of the B300 MD force provider.
 *
 * The contract is the force provider of arXiv 2412.18271 ("OpenMM-Python-
 * Force"): the MD engine hands the provider the current positions, the
 * provider returns the potential energy and the forces, and the engine then
 * advances the state (Methods section: the callable registered with the force
 * object returns an energy, and forces are obtained by differentiating it when
 * they are not returned explicitly; Results section, "Example: Ethanol": NVE
 * velocity-Verlet runs on the forces so obtained).  Here the provider and the
 * integrator both run as CUDA kernels on one GPU behind this ABI:
 *
 *   mdpf_create(topology, params)            build a context (device buffers, exclusions)
 *   mdpf_compute(ctx, positions, &E, forces) one energy/force evaluation   (host buffers)
 *   mdpf_step(ctx, n_steps)                  n velocity-Verlet steps, entirely on the device
 *
 * Units: A, fs, amu, e, kcal/mol.  Forces are -dE/dx in kcal/mol/A.
 *
 * Conventions shared by every entry point:
 *  - Return value: MDPF_OK (0) or a negative MDPF_ERR_* code.  Nothing aborts
 *    or exits the process.  mdpf_last_error() gives a message for the last
 *    failure on a context.
 *  - A CUDA error is sticky: once a context reports MDPF_ERR_CUDA every later
 *    call on it returns MDPF_ERR_CUDA; destroy it.
 *  - Inputs are copied; the caller keeps ownership of every pointer it passes.
 *    Host output buffers are caller-owned and must hold the stated sizes.
 *  - A context is not thread-safe; calls on one context must be serialised.
 *  - Array layouts are C row-major: "[N,3]" means x0 y0 z0 x1 y1 z1 ...
 */
#ifndef MDPF_H
#define MDPF_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MDPF_API __attribute__((visibility("default")))
#else
#define MDPF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define MDPF_OK 0
#define MDPF_ERR_INVALID_ARG (-1)       /* bad pointer, size or value; nothing was changed */
#define MDPF_ERR_CUDA (-2)              /* CUDA runtime error; sticky */
#define MDPF_ERR_OOM (-3)               /* device allocation failed */
#define MDPF_ERR_NEIGHBOR_OVERFLOW (-4) /* a neighbour or exclusion list exceeded its capacity */
#define MDPF_ERR_NONFINITE (-5)         /* energy or state became NaN/Inf */
#define MDPF_ERR_TIMEOUT (-6)           /* a bounded device-side wait gave up */
#define MDPF_ERR_OUT_OF_RANGE (-7)      /* learned features left the training range and fallback is off */
#define MDPF_ERR_CALLBACK (-9)          /* the external force provider reported an error */
#define MDPF_ERR_UNSUPPORTED (-8)       /* feature not available in this build or mode */

/* device status-word bits (mdpf_counters.status), one per failure kind */
#define MDPF_STATUS_NONFINITE 0x1u
#define MDPF_STATUS_NEIGHBOR_OVERFLOW 0x2u
#define MDPF_STATUS_TIMEOUT 0x4u
#define MDPF_STATUS_OUT_OF_RANGE 0x8u

#define MDPF_MODE_PLAIN 0   /* analytic bonded + all-pairs LJ + Coulomb */
#define MDPF_MODE_LEARNED 1 /* symmetry-function features + per-element MLP */
#define MDPF_MODE_CALLBACK 2 /* forces from a caller-supplied force provider (mdpf_force_fn) */

typedef struct mdpf_ctx mdpf_ctx;

/*
 * Topology and force-field parameters of a gas-phase system (no periodic
 * images, no cutoff on the plain nonbonded sum).  Copied by mdpf_create.
 *   element   [N]        0=H 1=C 2=N 3=O
 *   mass      [N]        amu (> 0)
 *   charge    [N]        e
 *   bonds     [n_bonds,2] atom indices, each pair distinct and in [0,N)
 *   bond_r0   [n_bonds]  A;   bond energy k/2 (r - r0)^2
 *   bond_k    [n_bonds]  kcal/mol/A^2
 *   angle_k, angle_theta0_deg: one harmonic angle k/2 (theta - theta0)^2 per
 *             pair of bonds sharing an atom (derived from the bond graph)
 *   lj_sigma, lj_eps [4] per element; pairs mix by Lorentz-Berthelot
 *             (sigma_ij = (sigma_i + sigma_j)/2, eps_ij = sqrt(eps_i eps_j)).
 * Pairs that are bonded (1-2) or share a bonded neighbour (1-3) are excluded
 * from the LJ + Coulomb sum; 1-4 and farther pairs are included unscaled.
 */
typedef struct mdpf_topology {
    int32_t n_atoms;
    const int32_t *element;
    const double *mass;
    const double *charge;
    int32_t n_bonds;
    const int32_t *bonds;
    const double *bond_r0;
    const double *bond_k;
    double angle_k;
    double angle_theta0_deg;
    double lj_sigma[4];
    double lj_eps[4];
} mdpf_topology;

/*
 * Run parameters.  Zero-initialise and set what you need; zeros select the
 * documented defaults.
 *   mode          MDPF_MODE_PLAIN or MDPF_MODE_LEARNED
 *   dt_fs         velocity-Verlet time step in fs (> 0)
 *   coulomb_k     Coulomb constant in kcal A/(mol e^2); 0 selects 332.06371
 *   trace_capacity  energy trace ring length (0 selects 4096)
 *   record_every  store a frame (positions, energy, forces) every this many
 *                 steps into a device ring of max_frames entries (0 = off)
 *   stepper       MDPF_STEPPER_PERSISTENT (0): mdpf_step runs as one resident
 *                 cooperative kernel with bounded grid barriers;
 *                 MDPF_STEPPER_KERNELS (1): one kernel sequence per step.
 *                 Both give the same trajectory bit for bit (plain mode).
 *                 Learned mode with velocity Verlet: PERSISTENT runs
 *                 molecules of up to 32 atoms as one resident cooperative
 *                 kernel (8 blocks, each holding a slice of the network's
 *                 weights; the same model and rounding points as the
 *                 tensor-core path, not the same bits), larger systems as
 *                 one CUDA graph of the stage kernels per step; KERNELS
 *                 always uses the stage kernels.
 *   energy_every  evaluate U and K every this many steps (0 selects 1); the
 *                 trace holds one entry per such step; record_every must be a
 *                 multiple of it.  Forces are evaluated every step regardless.
 */
#define MDPF_STEPPER_PERSISTENT 0
#define MDPF_STEPPER_KERNELS 1

/*
 * External force provider (MDPF_MODE_CALLBACK), the callable the MD engine
 * calls for energy and forces each step.  For every force evaluation the
 * library copies the positions (FP64 [N][3], A) into the caller's device
 * buffer provider_pos on cuda_stream, then calls fn(user, cuda_stream) on the
 * host.  The provider enqueues its work on cuda_stream (or finishes it before
 * returning) and writes the potential energy (one FP64, kcal/mol) to
 * provider_energy and the forces (FP32 [N][3], kcal/mol/A) to provider_forces,
 * both caller-owned device buffers; the library then turns them into its
 * fixed-point sums on the same stream.  A nonzero return aborts the call with
 * MDPF_ERR_CALLBACK.  Steps run one kernel sequence per step with the provider
 * called between its kick-drift and kick (no graph, no persistent kernel).  The
 * function and the buffers must stay valid for the context's lifetime.
 */
typedef int (*mdpf_force_fn)(void *user, void *cuda_stream);

typedef struct mdpf_params {
    int32_t mode;
    double dt_fs;
    double coulomb_k;
    int32_t trace_capacity;
    int32_t record_every;
    int32_t max_frames;
    int32_t stepper;
    int32_t energy_every;
    /* learned mode only */
    const void *model;       /* model blob (layout below); copied by mdpf_create */
    uint64_t model_bytes;
    double skin;             /* neighbour-list skin in A (0 selects 1.0); list radius = 5.2 + skin */
    int32_t rebuild_every;   /* rebuild the list every this many steps (0 selects 20) */
    int32_t fallback;        /* 1: a step whose features leave the model's range uses the plain
                                force field; 0: such a step reports MDPF_ERR_OUT_OF_RANGE */
    int32_t mlp_kernel;      /* MDPF_MLP_TENSOR (0): tcgen05 tensor cores, TMA-fed;
                                MDPF_MLP_SIMT (1): CUDA cores.  Same rounding points (BF16
                                GEMM inputs, FP32 accumulation); sums differ in order only.
                                MDPF_MLP_SIMT_FP32 (2): CUDA cores with FP32 operands (no BF16
                                rounding of features, activations or deltas), so the forces are
                                the gradient of the evaluated energy to FP32 rounding.
                                MDPF_MLP_FUSED (3): features, tensor-core MLP and force adjoint
                                in one kernel, one CTA per tile of at most 128 atoms of one
                                element; the features and dE/dG stay on chip.  Same arithmetic
                                as MDPF_MLP_TENSOR: identical energies and forces. */
    /* integrator: MDPF_INTEGRATOR_VERLET (0, NVE) or MDPF_INTEGRATOR_LANGEVIN (1): BAOAB
     *   v += dt/2 a;  x += dt/2 v;  v = c1 v + c2 R;  x += dt/2 v;  F = F(x);  v += dt/2 a
     * with c1 = exp(-gamma dt), c2 = sqrt((1 - c1^2) kB T / m) and R three normals per atom and step
     * from Philox4x32-10 (counter: atom, step index, tag; key: seed) by Box-Muller.  Langevin runs
     * the per-step kernel sequence (the persistent stepper is velocity Verlet only). */
    int32_t integrator;
    double friction_per_ps;   /* gamma in 1/ps (> 0 for Langevin) */
    double temperature_K;     /* bath temperature */
    uint64_t seed;            /* noise stream */
    /* callback mode only */
    mdpf_force_fn provider;
    void *provider_user;
    double *provider_pos;     /* device [N][3] FP64, written by the library */
    double *provider_energy;  /* device, 1 FP64, written by the provider */
    float *provider_forces;   /* device [N][3] FP32, written by the provider */
} mdpf_params;
#define MDPF_INTEGRATOR_VERLET 0
#define MDPF_INTEGRATOR_LANGEVIN 1
#define MDPF_MLP_TENSOR 0
#define MDPF_MLP_SIMT 1
#define MDPF_MLP_SIMT_FP32 2
#define MDPF_MLP_FUSED 3

/*
 * Learned mode (MDPF_MODE_LEARNED).  Per atom, 384 symmetry-function features
 * (64 radial: 16 Gaussians exp(-16 (r - R_k)^2), R_k = 0.9 + k 4.3/16, per
 * neighbour element, cosine cutoff 5.2 A; 320 angular: for each unordered
 * neighbour-element pair P (HH HC HN HO CC CN CO NN NO OO), 4 radial shells
 * R_m = 0.9 + m 2.6/4 (eta 8) x 8 angular sections theta_p = (2p+1) pi/16 of
 * 2^(1-32) (1 + cos(theta - theta_p))^32 with theta = acos(0.95 cos theta_ijk),
 * cutoff 3.5 A) feed a per-element MLP 384 -> 256 -> 128 -> 1 with CELU(0.1):
 * E = sum_i W3 . celu(W2 celu(W1 G_i + b1) + b2) + b3 + e0, plus an optional
 * repulsive pair core E_core = sum_{i<j, r_ij < rc} A (1 - r/rc)^3 (rc/r)
 * (the features vanish as r -> 0, so the network alone cannot keep two atoms
 * from merging).  Forces are the analytic adjoint -dE/dx.  The GEMM operands
 * run in BF16 (features and back-propagated deltas rounded to BF16; layer 1's
 * CELU output enters the second GEMM as a pair hi + lo of BF16 values, which
 * removes the energy bias one rounding would cause), accumulations in FP32,
 * energies and the state in FP64.  The plain topology (bonds, charges, LJ) is
 * still required: it is the fallback force field.
 *
 * Model blob (little endian): 64-byte header {char magic[8] = "MDPFMLP1";
 * int32 version = 1, n_elem = 4, n_feat = 384, h1 = 256, h2 = 128, flags
 * (bit 0: feature ranges follow; bit 1: repulsive core present); float64
 * celu_alpha; float64 core_A (kcal/mol, in (0, 1e5]), float64 core_rc (A, in
 * (0, 2]), both read only with flag bit 1; 8 reserved bytes},
 * then per element: uint16 W1[256][384] (BF16 bits), float32 b1[256],
 * uint16 W2[128][256] (BF16 bits), float32 b2[128], float32 W3[128],
 * float32 b3, float32 pad, float64 e0; then, if flags & 1, float32
 * lo[4][384], hi[4][384] (the training range of each feature, per element).
 */

/* Counters and diagnostics of a context. */
typedef struct mdpf_counters {
    int64_t steps;          /* velocity-Verlet steps taken since create / set_state */
    int64_t force_evals;    /* force evaluations by mdpf_step */
    int64_t frames;         /* frames recorded so far (ring holds the last max_frames) */
    uint32_t status;        /* MDPF_STATUS_* bits seen on the device */
    uint32_t reserved;
    double potential;       /* U at the last energy step, kcal/mol */
    double kinetic;         /* K at the last energy step, kcal/mol */
    double h_initial;       /* U + K right after the last set_state / init_velocities */
    double h_now;           /* U + K at the last energy step */
    int64_t rebuilds;       /* learned mode: neighbour-list builds so far (0 otherwise) */
    int64_t fallbacks;      /* learned mode: force evaluations whose features left the model's range
                               (they used the plain force field when the fallback is on) */
    double max_disp;        /* learned mode: largest displacement of an atom since the last list build, A */
} mdpf_counters;

/*
 * Build a context on the current CUDA device.  Copies the topology, derives
 * angles and the 1-2/1-3 exclusion set on the device, allocates every buffer
 * the path needs (the context owns them until mdpf_destroy).
 * Errors: INVALID_ARG (N < 1, bad index, non-positive mass or dt, unknown
 * mode or stepper; learned mode: missing or malformed model blob, skin
 * outside [0, 10]), OOM, CUDA, NEIGHBOR_OVERFLOW (an atom with more than 255
 * excluded partners), UNSUPPORTED (cooperative launch unavailable for the
 * persistent stepper; a model blob whose celu_alpha is not 0.1).  The blob
 * is checked on the host before any device work.  On error *out is NULL.
 */
/* Paper: the force object built around the force callable (Methods, Fig. 1). */
MDPF_API int mdpf_create(const mdpf_topology *topology, const mdpf_params *params, mdpf_ctx **out);

/* Free every device buffer and the context.  NULL is ignored. */
/* Paper: no counterpart (lifetime of the context). */
MDPF_API void mdpf_destroy(mdpf_ctx *ctx);

/* Message for the last failure on ctx (or of the last failed mdpf_create when ctx is NULL). */
/* Paper: no counterpart (error reporting). */
MDPF_API const char *mdpf_last_error(const mdpf_ctx *ctx);

/* Number of atoms, and the number of angles derived from the bond graph. */
/* Paper: no counterpart (sizes of the derived topology). */
MDPF_API int mdpf_sizes(const mdpf_ctx *ctx, int32_t *n_atoms, int32_t *n_angles);

/*
 * One energy/force evaluation at host positions pos [N,3] (A, FP64).  Writes
 * the potential energy (FP64, kcal/mol) to *energy and forces [N,3]
 * (kcal/mol/A) to the host buffer forces; either output may be NULL.  Does
 * not change the integrator state.  terms (may be NULL) receives the four
 * components {bond, angle, LJ, Coulomb} (zero in learned mode unless the
 * evaluation fell back to the plain force field).  Synchronous.  Learned
 * mode: returns NEIGHBOR_OVERFLOW when a neighbour row or cell exceeded its
 * capacity (128), and OUT_OF_RANGE when the features left the model's range
 * with the fallback off (the outputs then hold the model's values).
 */
/* Paper: the callable that returns the energy and the forces for given positions (Methods). */
MDPF_API int mdpf_compute(mdpf_ctx *ctx, const double *pos, double *energy, double *forces, double *terms);

/*
 * Device-pointer form of mdpf_compute: d_pos [N,3] FP64 device positions,
 * d_energy one FP64 device scalar, d_forces [N,3] FP32 device forces, all
 * enqueued on cuda_stream (a cudaStream_t; NULL = legacy default stream).
 * Asynchronous: results are valid once the stream reaches this point.  In
 * learned mode it shares the neighbour list and feature buffers with
 * mdpf_step: do not run the two concurrently on different streams.
 */
/* Paper: the callable that returns the energy and the forces for given positions (Methods). */
MDPF_API int mdpf_compute_device(mdpf_ctx *ctx, const double *d_pos, double *d_energy, float *d_forces,
                                 void *cuda_stream);

/*
 * Set the integrator state from host buffers pos [N,3] (A) and vel [N,3]
 * (A/fs), FP64.  Evaluates forces at pos, resets the step counter, the energy
 * trace and the status word, and records h_initial.
 */
/* Paper: the engine state the NVE runs start from (Results, "Example: Ethanol"). */
MDPF_API int mdpf_set_state(mdpf_ctx *ctx, const double *pos, const double *vel);

/* Copy the current state to host buffers (any may be NULL): pos, vel [N,3] FP64. */
/* Paper: the coordinates compared between runs (Results, "Example: Ethanol", Fig. 3). */
MDPF_API int mdpf_get_state(mdpf_ctx *ctx, double *pos, double *vel);

/*
 * Advance n_steps velocity-Verlet steps of dt_fs on the device:
 *   v += dt/2 a;  x += dt v;  F = F(x);  v += dt/2 a
 * with FP32 forces and FP64 positions, velocities, energies.  The whole loop
 * runs in one persistent kernel (or one kernel sequence per step); the host
 * is not involved between steps.  Returns NONFINITE if U or K became
 * non-finite, TIMEOUT if a device-side grid barrier gave up (the state is then
 * undefined; call mdpf_set_state).  Synchronous.
 */
/* Paper: the NVE velocity-Verlet runs (Results, "Example: Ethanol", Fig. 2); the whole loop on the device answers the per-step overhead of Table 2. */
MDPF_API int mdpf_step(mdpf_ctx *ctx, int64_t n_steps);

/*
 * Asynchronous mdpf_step on cuda_stream; status is checked by the next
 * synchronous call.  The synchronous calls run on the context's own stream:
 * the caller must let work enqueued on cuda_stream finish (or order the
 * streams) before calling mdpf_set_state, mdpf_get_state or mdpf_compute on
 * the same context.
 */
/* Paper: the NVE runs (Results, "Example: Ethanol"), enqueued without a host wait (Table 2's overhead). */
MDPF_API int mdpf_step_async(mdpf_ctx *ctx, int64_t n_steps, void *cuda_stream);

/* Counters, energies of the current state and the device status word. */
/* Paper: the energies and their conservation in the NVE runs (Results, "Example: Ethanol", Fig. 2). */
MDPF_API int mdpf_get_counters(mdpf_ctx *ctx, mdpf_counters *out);

/*
 * Maxwell-Boltzmann velocities at temperature_K (>= 0) for the current
 * positions (set them with mdpf_set_state first), drawn on the device:
 * v_i = sqrt(kB T / m_i) z_i with three standard normals per atom by
 * Box-Muller from Philox4x32-10 (counter: atom, 0, 0, 0x4D425630; key: seed),
 * then the centre-of-mass velocity and, for N >= 3 with a non-singular
 * inertia tensor, the rigid rotation are removed, and the velocities are
 * scaled so that K = (3N - 6) kB T / 2 (at least one degree of freedom).
 * Positions, forces and the step counter are unchanged; h_initial becomes
 * U + K.  These are the starting velocities of the NVE runs the engine
 * integrates (Results, "Example: Ethanol").  Errors: INVALID_ARG (bad
 * temperature, no state set), CUDA.  Synchronous.
 */
/* Paper: the starting velocities of the NVE runs (Results, "Example: Ethanol"). */
MDPF_API int mdpf_init_velocities(mdpf_ctx *ctx, double temperature_K, uint64_t seed);

/*
 * Energy trace, oldest first: one entry per energy step (every energy_every
 * steps), the most recent min(count, trace_capacity) of them.  U[k], K[k] in
 * kcal/mol after step step[k] (any output may be NULL).  *n_out receives the
 * count written (at most max_n).
 */
/* Paper: the potential, kinetic and total energy traces (Results, "Example: Ethanol", Figs. 2 and 4). */
MDPF_API int mdpf_get_trace(mdpf_ctx *ctx, double *U, double *K, int64_t *step, int64_t max_n, int64_t *n_out);

/*
 * Beside each energy-trace entry (same order and count as mdpf_get_trace):
 * the number of force evaluations so far, since mdpf_create, whose features
 * left the learned model's range (fallback evaluations; always 0 outside
 * learned mode).  Two consecutive entries one step apart that differ show a
 * step run on the plain force field; a step whose force field differs from
 * its predecessor's is a switch step, across which H is not conserved (the
 * two potentials differ), so drift is judged on the steps between switches.
 */
/* Paper: the NVE energy-conservation criterion (Results, "Example: Ethanol", Fig. 2). */
MDPF_API int mdpf_get_trace_fallbacks(mdpf_ctx *ctx, int64_t *fallbacks, int64_t max_n, int64_t *n_out);

/*
 * Recorded frames, oldest first (at most max_frames of them): pos [n,N,3]
 * FP64, energy [n] FP64, forces [n,N,3] FP32, step [n] int64 (any may be
 * NULL).  A frame is taken after every record_every-th step.
 */
/* Paper: the recorded trajectory frames (Results, "Example: Ethanol", Fig. 3). */
MDPF_API int mdpf_get_frames(mdpf_ctx *ctx, int64_t max_n, double *pos, double *energy, float *forces,
                             int64_t *step, int64_t *n_out);

/*
 * The 1-2/1-3 exclusion set built on the device by mdpf_create, as CSR:
 * offset [N+1] int32 and idx [capacity] int32, each row ascending.  *total
 * receives the number of entries (idx may be NULL to query it).
 */
/* Paper: no counterpart (topology of the analytic force field). */
MDPF_API int mdpf_get_exclusions(mdpf_ctx *ctx, int32_t *offset, int32_t *idx, int64_t capacity, int64_t *total);

/* Angles (a, vertex, b) derived on the device, [n_angles,3] int32, vertex-major order. */
/* Paper: no counterpart (topology of the analytic force field). */
MDPF_API int mdpf_get_angles(mdpf_ctx *ctx, int32_t *angles, int64_t capacity, int64_t *n_out);

/*
 * Fault injection for tests (host side; no GPU fault is raised).  The given
 * MDPF_STATUS_* bits are OR-ed into the device status word and reported by
 * the next mdpf_step / mdpf_get_counters; bits == 0 clears the word.
 */
/* Paper: no counterpart (failure detection). */
MDPF_API int mdpf_debug_set_status(mdpf_ctx *ctx, uint32_t bits);

/*
 * Bounded device-side wait on a flag that nothing sets: spins at most
 * limit_us microseconds (1..2,000,000), then records MDPF_STATUS_TIMEOUT and
 * returns MDPF_ERR_TIMEOUT.  Exercises the timeout path of the grid barrier
 * without hanging the GPU.
 */
/* Paper: no counterpart (failure detection). */
MDPF_API int mdpf_debug_wait_timeout(mdpf_ctx *ctx, int32_t limit_us);

/*
 * Check of the tensor-core operand path the MLP kernels share (tests only; no
 * context).  One CTA stores A [128 x 64] and B [n x 64] (BF16, row-major,
 * device pointers d_a and d_b, caller-owned) into its shared memory at byte
 * offsets a_off and b_off with the swizzled K-major store the MLP epilogues
 * use for their operands, issues the four tcgen05 MMAs of one 64-wide K chunk
 * with the MLP kernels' descriptors, and writes D = A B^T [128 x n] (FP32,
 * row-major) to d_d.  n: 128 or 256; offsets: multiples of 1024, the operands
 * disjoint and inside 225 KB; otherwise MDPF_ERR_INVALID_ARG.  Asynchronous
 * on cuda_stream (NULL: the default stream); if the bounded completion wait
 * expires the kernel ORs MDPF_STATUS_TIMEOUT into *d_status (a device word
 * the caller clears) and writes no D.
 */
/* Paper: no counterpart (test of the tensor-core helpers). */
MDPF_API int mdpf_debug_tc_probe(const void *d_a, const void *d_b, float *d_d, int32_t n, int32_t a_off,
                                 int32_t b_off, uint32_t *d_status, void *cuda_stream);

/*
 * Learned-path stages at host positions pos [N,3] (for parity checks; any
 * output may be NULL):
 *   neighbours  rows of the cell-list neighbour list (radius 5.2 + skin, FP32
 *               predicate fl(fl(fl(dx^2) + fl(dy^2)) + fl(dz^2)) < fl32(rc^2)),
 *               each row ascending: count [N], idx [N][max_per_atom] int32;
 *   features    G [N][384] FP32 (atom order);
 *   mlp         from caller features G [N][384] (FP32, rounded to BF16 as the
 *               GEMM input): atomic energies E_i [N] FP64 and dE/dG [N][384] FP32.
 * MDPF_ERR_UNSUPPORTED unless the context is in learned mode.
 */
/* Paper: the ML force module the plugin wraps (Methods), stage by stage. */
MDPF_API int mdpf_learned_neighbors(mdpf_ctx *ctx, const double *pos, int32_t max_per_atom, int32_t *count,
                                    int32_t *idx);
/* Paper: the ML force module the plugin wraps (Methods), stage by stage. */
MDPF_API int mdpf_learned_features(mdpf_ctx *ctx, const double *pos, float *G);
/* Paper: the ML force module the plugin wraps (Methods), stage by stage. */
MDPF_API int mdpf_learned_mlp(mdpf_ctx *ctx, const float *G, double *E_atom, float *dEdG);

/*
 * Learned-mode counters: neighbour-list rebuilds, force evaluations (steps,
 * set_state, compute) whose features left the model's range (these used the
 * plain force field when the fallback is on), and the largest neighbour row
 * seen.
 */
/* Paper: the ML force module the plugin wraps (Methods); fallback counting has no counterpart. */
MDPF_API int mdpf_learned_counters(mdpf_ctx *ctx, int64_t *rebuilds, int64_t *fallback_steps, int32_t *max_row);

/*
 * Force-matching training of the learned potential on the device.  The caller
 * owns every tensor (device pointers; e.g. torch tensors' data_ptr()):
 *   parameters  flat FP32, per element e = 0..3 (H, C, N, O), 131,585 each
 *               (526,340 in total): W1 [256][384], b1 [256], W2 [128][256],
 *               b2 [128], W3 [128], b3 (the forward rounds W1, W2 to BF16);
 *   batch       n_frames frames of atoms_per_frame atoms: positions
 *               [n][3] FP64 (A), elements [n] int32, reference energies
 *               [n_frames] FP64 (kcal/mol), reference forces [n][3] FP32.
 * mdpf_trainer_loss_grad enqueues on cuda_stream:
 *   L = (1/B) sum_f ((E_f - E_ref,f)/N)^2 + w_force (1/(3 N B)) sum (F - F_ref)^2
 * into d_loss3 = {L, energy part, force part} (FP64) and dL/dparams into
 * d_grad (same layout).  The force term's gradient is reverse mode over the
 * MLP's tangent pass along U = J dL/dF (feature JVP); every reduction runs in
 * a fixed order, so the gradient is reproducible bit for bit.  Neighbours: all
 * pairs within 5.2 A of the same frame.  The trainer also tracks the min/max
 * of every feature per element over all batches it has seen
 * (mdpf_trainer_feature_range, host [4][384] each).  mdpf_trainer_status
 * synchronises and reports NEIGHBOR_OVERFLOW (a row over 128) or TIMEOUT.
 * mdpf_adamw_step: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr (m/(1-b1^t) / (sqrt(v/(1-b2^t)) + eps) + weight_decay p), step t >= 1.
 */
typedef struct mdpf_trainer mdpf_trainer;
typedef struct mdpf_train_params {
    int32_t max_frames;        /* frames per batch, at most */
    int32_t atoms_per_frame;   /* N, the same for every frame */
    double w_force;            /* force-loss weight (10) */
    double e0[4];              /* per-element self energies (not trained) */
    double core_a, core_rc;    /* the model's repulsive core (kcal/mol, A; core_rc 0: none).  It has no
                                  trained parameters; its energy and forces are part of E_f and F. */
} mdpf_train_params;
#define MDPF_TRAIN_PARAMS_PER_ELEMENT 131585
/* Paper: forces of an energy model by automatic differentiation (Methods); training has no counterpart. */
MDPF_API int mdpf_trainer_create(const mdpf_train_params *params, mdpf_trainer **out);
/* Paper: no counterpart (lifetime of the trainer). */
MDPF_API void mdpf_trainer_destroy(mdpf_trainer *trainer);
/* Paper: no counterpart (error reporting). */
MDPF_API const char *mdpf_trainer_last_error(const mdpf_trainer *trainer);
/* Paper: forces of an energy model by automatic differentiation (Methods); the force-matching gradient has no counterpart. */
MDPF_API int mdpf_trainer_loss_grad(mdpf_trainer *trainer, const float *d_params, float *d_grad, int32_t n_frames,
                                    const double *d_pos, const int32_t *d_element, const double *d_E_ref,
                                    const float *d_F_ref, double *d_loss3, void *cuda_stream);
/* Paper: no counterpart (error reporting). */
MDPF_API int mdpf_trainer_status(mdpf_trainer *trainer, uint32_t *status);
/* Paper: no counterpart (the range behind the plain fallback). */
MDPF_API int mdpf_trainer_feature_range(mdpf_trainer *trainer, float *lo, float *hi);
/* Paper: no counterpart (the optimiser of the training). */
MDPF_API int mdpf_adamw_step(float *d_params, const float *d_grad, float *d_m, float *d_v, int64_t n, int64_t step,
                             double lr, double beta1, double beta2, double eps, double weight_decay,
                             void *cuda_stream);

/*
 * Feature JVP at host positions pos [N,3] along host vectors v [N,3]:
 * U [N][384] FP32 = sum_a dG/dx_a . v_a (the tangent the training gradient
 * uses; for parity checks).  Learned mode only.
 */
/* Paper: no counterpart (the tangent the training gradient uses). */
MDPF_API int mdpf_learned_jvp(mdpf_ctx *ctx, const double *pos, const float *v, float *U);

/*
 * Per-kernel device timing with CUDA events recorded on the launching stream
 * around every launch of the profiled kernels (off by default; costs two event
 * records per launch).  Slots: MDPF_PROF_NONBONDED (all-pairs tile kernel of
 * the kernel-sequence stepper), MDPF_PROF_STEPPER (persistent step-loop
 * kernel), MDPF_PROF_STEP (one whole mdpf_step call on the device); learned
 * mode: MDPF_PROF_NONBONDED times the whole learned force evaluation, and
 * MDPF_PROF_LEARN_NEIGHBORS / _FEATURES / _MLP / _ADJOINT its stages, or
 * MDPF_PROF_LEARN_FUSED the fused features-MLP-adjoint kernel.
 * mdpf_get_profile synchronises the recorded events and returns the summed
 * duration in ms and the number of launches since mdpf_set_profiling(ctx, 1).
 */
#define MDPF_PROF_NONBONDED 0
#define MDPF_PROF_STEPPER 1
#define MDPF_PROF_STEP 2
#define MDPF_PROF_LEARN_NEIGHBORS 3
#define MDPF_PROF_LEARN_FEATURES 4
#define MDPF_PROF_LEARN_MLP 5
#define MDPF_PROF_LEARN_ADJOINT 6
#define MDPF_PROF_LEARN_FUSED 7
#define MDPF_PROF_SLOTS 8
/* Paper: the per-step timings of Table 2. */
MDPF_API int mdpf_set_profiling(mdpf_ctx *ctx, int32_t enable);
/* Paper: the per-step timings of Table 2. */
MDPF_API int mdpf_get_profile(mdpf_ctx *ctx, int32_t slot, double *total_ms, int64_t *launches);

/*
 * All-pairs LJ + Coulomb energy and forces for callers that cannot allocate
 * device memory (an engine calling its force provider inside its own step
 * loop and memory pool, code that must not trigger the synchronisation that
 * cudaMalloc/cudaFree imply, or a host that only passes pointers into buffers
 * it already owns).  The paper has no counterpart of this entry point.
 *
 * Every pair i < j of the n_atoms atoms interacts (no exclusions, no bonded
 * terms, no cutoff), with the same per-element Lorentz-Berthelot LJ and
 * Coulomb terms and the same kernels as mdpf_compute_device; for a system
 * without bonds the two give the same results.
 *   d_pos     [N,3] FP64 device positions (A)        -- caller-owned input
 *   d_element [N]   int32 device elements 0..3       -- caller-owned input
 *                   (an element outside 0..3 yields NaN results)
 *   d_charge  [N]   FP64 device charges (e)          -- caller-owned input
 *   lj_sigma, lj_eps [4] host arrays, per element; coulomb_k 0 selects 332.06371
 *   d_energy  one FP64 device scalar (kcal/mol), or NULL
 *   d_forces  [N,3] FP32 device forces (kcal/mol/A), or NULL (not both NULL)
 * All work is enqueued on cuda_stream; the call returns without waiting.
 *
 * Memory: the call allocates nothing.  Its working memory is one fixed array
 * of about 390 KB in the library's device data, held by every GPU that loads
 * the library until the process exits; it limits n_atoms to 2048 (larger
 * values return MDPF_ERR_INVALID_ARG).  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress, with that device
 * current) and keeps it with the device's current context; a call that finds
 * another context current (the old one was destroyed, e.g. by
 * cudaDeviceReset) looks it up again.  Make the first call on a device, and
 * the first after a reset, before any stream capture.  All calls share
 * the array and each call clears what it accumulates, so calls that overlap
 * on the GPU (different streams, or different host threads) race and must be
 * serialised by the caller.  Errors are reported by the return code and
 * mdpf_last_error(NULL).
 */
MDPF_API int mdpf_pairs_noalloc(int32_t n_atoms, const double *d_pos, const int32_t *d_element, const double *d_charge,
                                const double lj_sigma[4], const double lj_eps[4], double coulomb_k, double *d_energy,
                                float *d_forces, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MDPF_H */
