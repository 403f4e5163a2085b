// Learned-potential path: device data and kernel launchers.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "device_util.cuh"

namespace mdpf {

constexpr int kNFeat = 384, kH1 = 256, kH2 = 128;
constexpr int kKmax = 128;          // neighbour-row capacity
constexpr int kCellCap = 128;       // atoms per cell capacity
constexpr int kMaxCellDim = 32;     // cells per dimension at most (larger systems get larger cells)
constexpr int kRowTile = 128;       // element groups of MLP rows are padded to this
constexpr float kRcRad = 5.2f, kRcAng = 3.5f;

// Cell grid of the current neighbour build (filled on the device).
struct CellGrid {
    float lo[3];
    float cs;
    int dim[3];
    int ncell;
};

// Everything the learned kernels read or write.
struct LearnedDev {
    int n, n_rows;
    const int *n_tiles_live;     // device count of row tiles in use (training batches), or null: all n_rows / 128
    const int *el;               // [n]
    const int *row_of;           // [n] atom -> MLP row
    const int *atom_of;          // [n_rows] MLP row -> atom, -1 on padding rows
    const int *tile_el;          // [n_rows / kRowTile] element of each row tile
    // neighbour list
    float rc_list2;              // fl32(rc_list^2)
    float rc_list;
    float half_skin2;            // (skin/2)^2
    int *nb_count;               // [n]
    int *nb_idx;                 // [n][kKmax]
    float4 *pos_build;           // [n] positions at the last build
    int *cell_cnt;               // [max cells]
    int *cell_atoms;             // [max cells][kCellCap]
    CellGrid *grid;
    unsigned int *bbox;          // [6] ordered-int min/max (empty box between builds)
    long long *bmom;             // [8][6] fixed-point sums of u = x - x0 and u^2 per axis, x0 = atom 0, spread
                                 // over 8 copies (zero between builds)
    unsigned long long *nb_bar;  // [3] grid-barrier arrival counter, base of the next build; small-build arrivals
    int nb_grid;                 // blocks of the cooperative neighbour kernel
    // features and MLP
    __nv_bfloat16 *G16;          // [n_rows][384] GEMM input
    float *G32;                  // [n_rows][384] FP32 features (parity output) or null
    void *g;                     // [n_rows][384] dE/dG (the adjoint's input): BF16, or FP32 when g_f32
    int g_f32;                   // 1: the FP32-operand MLP variant, whose forces are the exact FP32 gradient
    double *E_row;               // [n_rows]
    const __nv_bfloat16 *W1, *W1T, *W2, *W2T;  // [4][256][384], [4][384][256], [4][128][256], [4][256][128]
    const float *b1, *b2, *W3, *b3;            // [4][256], [4][128], [4][128], [4]
    const double *e0;                          // [4]
    const float *lo, *hi;                      // [4][384] training range, or null
    float core_a, core_rc;       // short-range repulsive core A (kcal/mol), r_c (A); core_rc == 0: none
    unsigned int *lflags;        // [0] rebuild requested, [1] out of range this step, [2] overflow, [3] MLP timeout
    long long *lcount;           // [0] rebuilds, [1] fallback steps, [2] max row length
};

// TMA descriptors of the MLP operands (BF16, 2-D, 64 x 128 boxes, 128-byte swizzle):
// features G16 [n_rows][384], W1 [4*256][384], W2 [4*128][256], W2T [4*256][128], W1T [4*384][256].
struct MlpMaps {
    CUtensorMap g, w1, w2, w2t, w1t;
};

// Tiles of the fused kernel: tile t covers MLP rows first[t] .. first[t] + count[t] - 1,
// 1 <= count[t] <= kRowTile, all atoms of element el[t].
struct FusedTiles {
    const int *first, *count, *el;
    int n;
};

// the context's learned-path data and whether out-of-range steps fall back (learned_host.cu)
const LearnedDev &learned_dev(const mdpf_ctx *c);
int learned_fallback_on(const mdpf_ctx *c);

// launchers (learned.cu)
// neighbour list (cooperative launch; learned_nb_grid() gives its grid size, 0 if unavailable)
int learned_nb_grid();
cudaError_t learned_neighbors(const LearnedDev &L, const float4 *pos4, bool forced, uint32_t *status,
                              cudaStream_t s);
void learned_features(const LearnedDev &L, const float4 *pos4, bool write_f32, cudaStream_t s);
// MLP on the CUDA cores; efx (or null) receives the summed energy in its learned-energy slot
void learned_mlp(const LearnedDev &L, bool gated, bool fp32, unsigned long long *efx, cudaStream_t s);
// forces into fx; the core energy of atom i goes to ecore[i / ecore_per] (fixed point) unless ecore is null
void learned_adjoint(const LearnedDev &L, const float4 *pos4, unsigned long long *fx, bool gated,
                     unsigned long long *ecore, int ecore_per, cudaStream_t s);
void learned_begin(const LearnedDev &L, cudaStream_t s);
// a step that left the feature range: drop the model's forces and energy (fused path, before the plain force field)
void learned_fallback_clear(const LearnedDev &L, unsigned long long *fx, unsigned long long *efx, cudaStream_t s);
void learned_end(const LearnedDev &L, uint32_t *status, int fallback, cudaStream_t s);
void learned_import_g(const LearnedDev &L, const float *G_atoms, cudaStream_t s);
// feature JVP: U [n_rows][384] (rows of the atoms) = sum_a dG/dx_a . v_a, v [n][3]
void learned_jvp(const LearnedDev &L, const float4 *pos4, const float *v, float *U, cudaStream_t s);

// tensor-core MLP (mlp_tc.cu): forward energy and dE/dG, one 128-row tile per CTA
cudaError_t learned_mlp_tc_prepare();
cudaError_t learned_mlp_tc(const LearnedDev &L, const MlpMaps &maps, uint32_t *status, bool gated,
                           unsigned long long *efx, cudaStream_t s);

// training (wgrad_tc.cu): dW1 and dW2 of the force-matching loss on the tensor cores, as K-split GEMMs
// over each element's row tiles, the splits summed in order into grad[e * per_element + off + ...]
constexpr int kWgSplits = 24;
struct WgradIn {
    const __nv_bfloat16 *bh1, *bt1, *G, *U;   // BF16 [rows][256], [rows][256], [rows][384], [rows][384]
    const __nv_bfloat16 *bh2, *bt2, *a1, *ta1;  // BF16 [rows][128], [rows][128], [rows][256], [rows][256]
    const int *atom_of, *tile_el, *n_live;
    int tiles_max;
    int *etiles;                          // scratch [4][tiles_max]
    int4 *split;                          // scratch [kWgSplits]
    float *part;                          // scratch kWgSplits * (256 * 384 + 128 * 256) floats
    float *grad;
    int per_element, off_w1, off_w2;
    uint32_t *status;
};
cudaError_t learned_wgrad_tc_prepare();
cudaError_t learned_wgrad_tc(const WgradIn &w, cudaStream_t s);

// fused features -> MLP -> adjoint (fused.cu): energies per row, the energy slot of efx and fixed-point
// forces fx, with G and dE/dG kept on chip; sets the range flag like the feature kernel
cudaError_t learned_fused_prepare();
cudaError_t learned_fused(const LearnedDev &L, const FusedTiles &T, const MlpMaps &maps, const float4 *pos4,
                          unsigned long long *fx, unsigned long long *efx, uint32_t *status, cudaStream_t s);

}  // namespace mdpf
