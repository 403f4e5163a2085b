// Learned mode: model-blob parsing, device buffers, the per-evaluation kernel
// sequence (neighbours -> features -> MLP -> adjoint, or the plain force field
// when the features leave the model's range), and the parity entry points.
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "learned.cuh"

namespace mdpf {

struct LearnedHost {
    LearnedDev dev{};
    std::vector<void *> allocs;
    int fallback = 1;
    int rebuild_every = 20;
    double skin = 1.0;
    int n_rows = 0;
    std::vector<int> row_of;
    float *d_Gin = nullptr;     // [n][384] staging for mdpf_learned_mlp
    float *d_vin = nullptr;     // [n][3] tangent staging for mdpf_learned_jvp (allocated on first use)
    float *d_U = nullptr;       // [n_rows][384] JVP output (allocated on first use)
    unsigned int *d_disp = nullptr;   // max squared displacement (float bits) for the counters
    int mlp_kernel = MDPF_MLP_TENSOR;
    MlpMaps maps{};
    FusedTiles ft{};
};

static int fused_tile_count(const std::vector<int> &cnt, int run) {
    int t = 0;
    for (int c : cnt) t += (c + run - 1) / run;
    return t;
}

// Tiles of the fused kernel: each element's atoms (rows start[e] .. start[e] + cnt[e] - 1) in
// near-equal runs of at most kRowTile.  The run length is the smallest one that keeps the tiles
// within one wave over the SMs (one CTA per SM), or kRowTile when even that needs more waves.
static void fused_tiling(const std::vector<int> &cnt, const std::vector<int> &start, int sms, std::vector<int> &first,
                         std::vector<int> &count, std::vector<int> &el) {
    int run = kRowTile;
    if (sms > 0 && fused_tile_count(cnt, kRowTile) <= sms) {
        run = 1;
        while (fused_tile_count(cnt, run) > sms) ++run;
    }
    for (int e = 0; e < (int)cnt.size(); ++e) {
        if (cnt[e] == 0) continue;
        const int nt = (cnt[e] + run - 1) / run, base = cnt[e] / nt, rem = cnt[e] % nt;
        for (int t = 0, off = 0; t < nt; ++t) {
            const int len = base + (t < rem ? 1 : 0);
            first.push_back(start[e] + off);
            count.push_back(len);
            el.push_back(e);
            off += len;
        }
    }
}

// 2-D BF16 tensor maps with 64 x 128 boxes and 128-byte swizzle for the MLP operands.
static int make_maps(mdpf_ctx *c, LearnedHost *h) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || fn == nullptr)
        return fail(c, MDPF_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const LearnedDev &L = h->dev;
    auto one = [&](CUtensorMap *m, const void *ptr, uint64_t inner, uint64_t rows) {
        cuuint64_t dims[2] = {inner, rows};
        cuuint64_t strides[1] = {inner * 2};
        cuuint32_t box[2] = {64, 128};
        cuuint32_t estr[2] = {1, 1};
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    if (!one(&h->maps.g, L.G16, kNFeat, (uint64_t)L.n_rows) || !one(&h->maps.w1, L.W1, kNFeat, 4 * kH1) ||
        !one(&h->maps.w2, L.W2, kH1, 4 * kH2) || !one(&h->maps.w2t, L.W2T, kH2, 4 * kH1) ||
        !one(&h->maps.w1t, L.W1T, kH1, 4 * kNFeat))
        return fail(c, MDPF_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    e = learned_mlp_tc_prepare();
    if (e != cudaSuccess) return cuda_fail(c, e, "learned_mlp_tc_prepare");
    e = learned_fused_prepare();
    if (e != cudaSuccess) return cuda_fail(c, e, "learned_fused_prepare");
    return MDPF_OK;
}

// The MLP (energy per row and dE/dG) on the selected units.
static void enqueue_mlp(LearnedHost *h, uint32_t *status, bool gated, unsigned long long *efx, cudaStream_t s) {
    if (h->mlp_kernel == MDPF_MLP_TENSOR || h->mlp_kernel == MDPF_MLP_FUSED)
        learned_mlp_tc(h->dev, h->maps, status, gated, efx, s);
    else learned_mlp(h->dev, gated, h->mlp_kernel == MDPF_MLP_SIMT_FP32, efx, s);
}

static LearnedHost *lh(const mdpf_ctx *c) { return static_cast<LearnedHost *>(c->learned); }

const LearnedDev &learned_dev(const mdpf_ctx *c) { return lh(c)->dev; }
int learned_fallback_on(const mdpf_ctx *c) { return lh(c)->fallback; }

template <typename T>
static cudaError_t lalloc(LearnedHost *h, T **p, size_t count) {
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
    if (e == cudaSuccess) h->allocs.push_back((void *)*p);
    return e;
}

void learned_free(mdpf_ctx *c) {
    LearnedHost *h = lh(c);
    if (!h) return;
    for (void *p : h->allocs) cudaFree(p);
    delete h;
    c->learned = nullptr;
}

static constexpr size_t kHeader = 64;
static constexpr size_t kPerElement = (size_t)kH1 * kNFeat * 2 + kH1 * 4 + (size_t)kH2 * kH1 * 2 + kH2 * 4 +
                                      kH2 * 4 + 4 + 4 + 8;

// Host-side check of a model blob (no device work): shape, CELU constant, size.
int learned_validate(const mdpf_params *prm, std::string &msg) {
    const unsigned char *blob = static_cast<const unsigned char *>(prm->model);
    if (blob == nullptr || prm->model_bytes < kHeader) return msg = "learned mode needs a model blob", MDPF_ERR_INVALID_ARG;
    if (std::memcmp(blob, "MDPFMLP1", 8) != 0) return msg = "model blob: bad magic", MDPF_ERR_INVALID_ARG;
    int32_t hdr[6];
    double alpha;
    std::memcpy(hdr, blob + 8, sizeof(hdr));
    std::memcpy(&alpha, blob + 32, sizeof(alpha));
    if (hdr[0] != 1 || hdr[1] != 4 || hdr[2] != kNFeat || hdr[3] != kH1 || hdr[4] != kH2)
        return msg = "model blob: unexpected version or shape", MDPF_ERR_INVALID_ARG;
    if (std::fabs(alpha - 0.1) > 1e-12) return msg = "model blob: CELU alpha must be 0.1", MDPF_ERR_UNSUPPORTED;
    const bool ranges = (hdr[5] & 1) != 0;
    const size_t expect = kHeader + 4 * kPerElement + (ranges ? 2 * 4 * kNFeat * sizeof(float) : 0);
    if (prm->model_bytes != expect) return msg = "model blob: wrong size", MDPF_ERR_INVALID_ARG;
    if (hdr[5] & 2) {   // repulsive core: A (kcal/mol) and r_c (A) in the header
        double core[2];
        std::memcpy(core, blob + 40, sizeof(core));
        if (!(core[0] > 0.0 && core[0] <= 1e5) || !(core[1] > 0.0 && core[1] <= 2.0))
            return msg = "model blob: core A must be in (0, 1e5] kcal/mol and r_c in (0, 2] A", MDPF_ERR_INVALID_ARG;
    }
    if (hdr[5] & ~3) return msg = "model blob: unknown flag bits", MDPF_ERR_INVALID_ARG;
    return MDPF_OK;
}

int learned_create(mdpf_ctx *c, const mdpf_topology *t, const mdpf_params *prm) {
    std::string msg;
    const int vrc = learned_validate(prm, msg);
    if (vrc != MDPF_OK) return fail(c, vrc, msg);
    const unsigned char *blob = static_cast<const unsigned char *>(prm->model);
    int32_t hdr[6];
    std::memcpy(hdr, blob + 8, sizeof(hdr));
    const bool ranges = (hdr[5] & 1) != 0;

    LearnedHost *h = new LearnedHost();
    c->learned = h;
    if (hdr[5] & 2) {
        double core[2];
        std::memcpy(core, blob + 40, sizeof(core));
        h->dev.core_a = (float)core[0];
        h->dev.core_rc = (float)core[1];
    }
    h->fallback = prm->fallback != 0;
    h->rebuild_every = prm->rebuild_every > 0 ? prm->rebuild_every : 20;
    h->skin = prm->skin > 0 ? prm->skin : 1.0;
    h->mlp_kernel = prm->mlp_kernel;
    const int n = c->n;

    // weights: W and W^T per element (the transposes serve the GEMMs that contract over the other index)
    std::vector<uint16_t> W1(4 * (size_t)kH1 * kNFeat), W1T(W1.size()), W2(4 * (size_t)kH2 * kH1), W2T(W2.size());
    std::vector<float> b1(4 * kH1), b2(4 * kH2), W3(4 * kH2), b3(4), lo, hi;
    std::vector<double> e0(4);
    size_t off = kHeader;
    for (int e = 0; e < 4; ++e) {
        uint16_t *w1 = W1.data() + (size_t)e * kH1 * kNFeat;
        std::memcpy(w1, blob + off, (size_t)kH1 * kNFeat * 2);
        off += (size_t)kH1 * kNFeat * 2;
        std::memcpy(b1.data() + e * kH1, blob + off, kH1 * 4);
        off += kH1 * 4;
        uint16_t *w2 = W2.data() + (size_t)e * kH2 * kH1;
        std::memcpy(w2, blob + off, (size_t)kH2 * kH1 * 2);
        off += (size_t)kH2 * kH1 * 2;
        std::memcpy(b2.data() + e * kH2, blob + off, kH2 * 4);
        off += kH2 * 4;
        std::memcpy(W3.data() + e * kH2, blob + off, kH2 * 4);
        off += kH2 * 4;
        std::memcpy(&b3[e], blob + off, 4);
        off += 8;
        std::memcpy(&e0[e], blob + off, 8);
        off += 8;
        for (int a = 0; a < kH1; ++a)
            for (int f = 0; f < kNFeat; ++f)
                W1T[(size_t)e * kNFeat * kH1 + (size_t)f * kH1 + a] = w1[(size_t)a * kNFeat + f];
        for (int b = 0; b < kH2; ++b)
            for (int a = 0; a < kH1; ++a) W2T[(size_t)e * kH1 * kH2 + (size_t)a * kH2 + b] = w2[(size_t)b * kH1 + a];
    }
    if (ranges) {
        lo.resize(4 * kNFeat);
        hi.resize(4 * kNFeat);
        std::memcpy(lo.data(), blob + off, 4 * kNFeat * 4);
        off += 4 * kNFeat * 4;
        std::memcpy(hi.data(), blob + off, 4 * kNFeat * 4);
    }

    // MLP rows: atoms grouped by element, each group padded to kRowTile rows
    std::vector<int> cnt(4, 0);
    for (int i = 0; i < n; ++i) cnt[t->element[i]]++;
    std::vector<int> start(5, 0);
    for (int e = 0; e < 4; ++e) start[e + 1] = start[e] + (cnt[e] + kRowTile - 1) / kRowTile * kRowTile;
    const int n_rows = start[4];
    h->n_rows = n_rows;
    h->row_of.assign(n, 0);
    std::vector<int> atom_of(n_rows > 0 ? n_rows : 1, -1), tile_el(n_rows / kRowTile + 1, 0), fill(start.begin(), start.end() - 1);
    for (int i = 0; i < n; ++i) {
        const int r = fill[t->element[i]]++;
        h->row_of[i] = r;
        atom_of[r] = i;
    }
    for (int e = 0; e < 4; ++e)
        for (int r = start[e]; r < start[e + 1]; r += kRowTile) tile_el[r / kRowTile] = e;
    std::vector<int> ft_first, ft_count, ft_el;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 0;
        fused_tiling(cnt, start, sms, ft_first, ft_count, ft_el);
    }

    LearnedDev &L = h->dev;
    L.n = n;
    L.n_rows = n_rows;
    L.el = c->d_element;
    const float rc = (float)(5.2 + h->skin);
    L.rc_list = rc;
    L.rc_list2 = (float)((5.2 + h->skin) * (5.2 + h->skin));
    L.half_skin2 = (float)(0.25 * h->skin * h->skin);
    const int max_cells = (kMaxCellDim + 1) * (kMaxCellDim + 1) * (kMaxCellDim + 1);
    int *d_row_of, *d_atom_of, *d_tile_el;
    __nv_bfloat16 *dW1, *dW1T, *dW2, *dW2T;
    float *db1, *db2, *dW3, *db3, *dlo = nullptr, *dhi = nullptr;
    double *de0;
    cudaError_t err = cudaSuccess;
#define LA(p, nelem)                                                  \
    do {                                                              \
        if ((err = lalloc(h, &(p), (nelem))) != cudaSuccess) {        \
            cuda_fail(c, err, "learned allocation");                  \
            return err == cudaErrorMemoryAllocation ? MDPF_ERR_OOM : MDPF_ERR_CUDA; \
        }                                                             \
    } while (0)
    LA(d_row_of, n);
    LA(d_atom_of, atom_of.size());
    LA(d_tile_el, tile_el.size());
    LA(L.nb_count, n);
    LA(L.nb_idx, (size_t)n * kKmax);
    LA(L.pos_build, n);
    LA(L.cell_cnt, max_cells);
    LA(L.cell_atoms, (size_t)max_cells * kCellCap);
    LA(L.grid, 1);
    LA(L.bbox, 8);
    LA(L.bmom, 48);
    LA(L.nb_bar, 3);
    LA(L.G16, (size_t)n_rows * kNFeat);
    LA(L.G32, (size_t)n_rows * kNFeat);
    {   // dE/dG: room for FP32 (the FP32-operand variant), BF16 otherwise
        float *gbuf = nullptr;
        LA(gbuf, (size_t)n_rows * kNFeat);
        L.g = gbuf;
        L.g_f32 = h->mlp_kernel == MDPF_MLP_SIMT_FP32 ? 1 : 0;
    }
    LA(L.E_row, n_rows);
    LA(dW1, W1.size());
    LA(dW1T, W1T.size());
    LA(dW2, W2.size());
    LA(dW2T, W2T.size());
    LA(db1, b1.size());
    LA(db2, b2.size());
    LA(dW3, W3.size());
    LA(db3, 4);
    LA(de0, 4);
    if (ranges) {
        LA(dlo, lo.size());
        LA(dhi, hi.size());
    }
    LA(L.lflags, 4);
    LA(h->d_disp, 1);
    LA(L.lcount, 4);
    LA(h->d_Gin, (size_t)n * kNFeat);
    int *d_ft_first, *d_ft_count, *d_ft_el;
    LA(d_ft_first, ft_first.size());
    LA(d_ft_count, ft_count.size());
    LA(d_ft_el, ft_el.size());
#undef LA
#define LC(x)                                                         \
    do {                                                              \
        if ((err = (x)) != cudaSuccess) return cuda_fail(c, err, #x); \
    } while (0)
    LC(cudaMemcpy(d_row_of, h->row_of.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    LC(cudaMemcpy(d_atom_of, atom_of.data(), sizeof(int) * atom_of.size(), cudaMemcpyHostToDevice));
    LC(cudaMemcpy(d_tile_el, tile_el.data(), sizeof(int) * tile_el.size(), cudaMemcpyHostToDevice));
    LC(cudaMemcpy(dW1, W1.data(), 2 * W1.size(), cudaMemcpyHostToDevice));
    LC(cudaMemcpy(dW1T, W1T.data(), 2 * W1T.size(), cudaMemcpyHostToDevice));
    LC(cudaMemcpy(dW2, W2.data(), 2 * W2.size(), cudaMemcpyHostToDevice));
    LC(cudaMemcpy(dW2T, W2T.data(), 2 * W2T.size(), cudaMemcpyHostToDevice));
    LC(cudaMemcpy(db1, b1.data(), 4 * b1.size(), cudaMemcpyHostToDevice));
    LC(cudaMemcpy(db2, b2.data(), 4 * b2.size(), cudaMemcpyHostToDevice));
    LC(cudaMemcpy(dW3, W3.data(), 4 * W3.size(), cudaMemcpyHostToDevice));
    LC(cudaMemcpy(db3, b3.data(), 16, cudaMemcpyHostToDevice));
    LC(cudaMemcpy(de0, e0.data(), 32, cudaMemcpyHostToDevice));
    if (ranges) {
        LC(cudaMemcpy(dlo, lo.data(), 4 * lo.size(), cudaMemcpyHostToDevice));
        LC(cudaMemcpy(dhi, hi.data(), 4 * hi.size(), cudaMemcpyHostToDevice));
    }
    if (!ft_first.empty()) {
        LC(cudaMemcpy(d_ft_first, ft_first.data(), sizeof(int) * ft_first.size(), cudaMemcpyHostToDevice));
        LC(cudaMemcpy(d_ft_count, ft_count.data(), sizeof(int) * ft_count.size(), cudaMemcpyHostToDevice));
        LC(cudaMemcpy(d_ft_el, ft_el.data(), sizeof(int) * ft_el.size(), cudaMemcpyHostToDevice));
    }
    h->ft = FusedTiles{d_ft_first, d_ft_count, d_ft_el, (int)ft_first.size()};
    LC(cudaMemset(L.G16, 0, sizeof(__nv_bfloat16) * (size_t)n_rows * kNFeat));
    LC(cudaMemset(L.E_row, 0, sizeof(double) * (size_t)(n_rows > 0 ? n_rows : 1)));
    LC(cudaMemset(L.lflags, 0, sizeof(unsigned int) * 4));
    LC(cudaMemset(L.lcount, 0, sizeof(long long) * 4));
    LC(cudaMemset(L.nb_count, 0, sizeof(int) * n));
    LC(cudaMemset(L.nb_bar, 0, sizeof(unsigned long long) * 3));
    LC(cudaMemset(L.bmom, 0, sizeof(long long) * 48));
    {
        const unsigned int empty_box[8] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u, 0u, 0u, 0u, 0u};
        LC(cudaMemcpy(L.bbox, empty_box, sizeof(empty_box), cudaMemcpyHostToDevice));
    }
    L.nb_grid = learned_nb_grid();
    if (L.nb_grid < 1) return fail(c, MDPF_ERR_UNSUPPORTED, "cooperative launch of the neighbour build is not available");
    unsigned int one = 1u;
    LC(cudaMemcpy(L.lflags, &one, sizeof(one), cudaMemcpyHostToDevice));
#undef LC
    L.row_of = d_row_of;
    L.atom_of = d_atom_of;
    L.tile_el = d_tile_el;
    L.W1 = dW1;
    L.W1T = dW1T;
    L.W2 = dW2;
    L.W2T = dW2T;
    L.b1 = db1;
    L.b2 = db2;
    L.W3 = dW3;
    L.b3 = db3;
    L.e0 = de0;
    L.lo = dlo;
    L.hi = dhi;
    return make_maps(c, h);
}

int learned_enqueue_forces(mdpf_ctx *c, const float4 *pos4, unsigned long long *fx, unsigned long long *efx,
                           uint32_t *status, bool forced_build, bool write_f32, cudaStream_t s) {
    LearnedHost *h = lh(c);
    const LearnedDev &L = h->dev;
    // the range flag is cleared by the end-of-evaluation kernel; single evaluations clear it first (a model
    // without ranges never raises it)
    if (forced_build && L.lo != nullptr) learned_begin(L, s);
    cudaEvent_t ev = prof_begin(c, s);
    cudaError_t ce = learned_neighbors(L, pos4, forced_build, status, s);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "learned_neighbors");
    prof_end(c, MDPF_PROF_LEARN_NEIGHBORS, ev, s);
    // with the fallback on, a step that left the range skips the model and runs the plain force field;
    // with it off, the model's forces are used and the step reports MDPF_STATUS_OUT_OF_RANGE
    const bool gated = h->fallback != 0;
    if (h->mlp_kernel == MDPF_MLP_FUSED && !write_f32) {
        // one kernel; the range is known only when it ends, so a step that left it drops the model's
        // forces and energy afterwards
        ev = prof_begin(c, s);
        ce = learned_fused(L, h->ft, h->maps, pos4, fx, efx, status, s);
        if (ce != cudaSuccess) return cuda_fail(c, ce, "learned_fused");
        prof_end(c, MDPF_PROF_LEARN_FUSED, ev, s);
        if (L.lo == nullptr) return MDPF_OK;
        if (gated) {
            learned_fallback_clear(L, fx, efx, s);
            PlainDev p = plain_dev(c, pos4);
            p.status = status;
            p.gate = L.lflags + 1;
            launch_bonded(p, fx, efx, s);
            launch_nonbonded(p, fx, efx, true, s);
        }
        learned_end(L, status, h->fallback, s);
        return MDPF_OK;
    }
    ev = prof_begin(c, s);
    learned_features(L, pos4, write_f32 || h->mlp_kernel == MDPF_MLP_SIMT_FP32, s);
    prof_end(c, MDPF_PROF_LEARN_FEATURES, ev, s);
    ev = prof_begin(c, s);
    enqueue_mlp(h, status, gated, efx, s);
    prof_end(c, MDPF_PROF_LEARN_MLP, ev, s);
    ev = prof_begin(c, s);
    learned_adjoint(L, pos4, fx, gated, efx != nullptr ? efx + E_LEARN : nullptr, L.n, s);
    prof_end(c, MDPF_PROF_LEARN_ADJOINT, ev, s);
    if (L.lo == nullptr) return MDPF_OK;   // no feature ranges: no evaluation can leave them
    if (gated) {
        PlainDev p = plain_dev(c, pos4);
        p.status = status;
        p.gate = L.lflags + 1;
        launch_bonded(p, fx, efx, s);
        launch_nonbonded(p, fx, efx, true, s);
    }
    learned_end(L, status, h->fallback, s);
    return MDPF_OK;
}

// The per-step rebuild request, checked by the kick-drift kernel: an atom moved more than skin/2 since the
// last build, or the completed-step count is a multiple of rebuild_every.
__global__ void k_max_disp2(int n, const float4 *pos4, const float4 *pos_build, unsigned int *out) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    float d2 = 0.f;
    if (a < n) {
        const float4 p = pos4[a], b = pos_build[a];
        const float dx = p.x - b.x, dy = p.y - b.y, dz = p.z - b.z;
        d2 = dx * dx + dy * dy + dz * dz;
    }
    for (int o = 16; o > 0; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    // non-negative floats order like their bit patterns
    if ((threadIdx.x & 31) == 0 && d2 > 0.f) atomicMax(out, __float_as_uint(d2));
}

// Counters of the learned path for mdpf_get_counters: list rebuilds, evaluations that left the
// feature range, and the largest displacement of an atom (FP32 state positions) since the last
// list build, in A.  Synchronous on the context's stream.
int learned_counter_values(mdpf_ctx *c, int64_t *rebuilds, int64_t *fallbacks, double *max_disp) {
    LearnedHost *h = lh(c);
    long long v[4];
    unsigned int bits = 0;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemcpy(v, h->dev.lcount, sizeof(v), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_disp, 0, sizeof(unsigned int), c->stream);
    if (e == cudaSuccess) {
        k_max_disp2<<<(c->n + 255) / 256, 256, 0, c->stream>>>(c->n, c->d_pos4, h->dev.pos_build, h->d_disp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, h->d_disp, sizeof(bits), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "learned counters");
    float d2;
    std::memcpy(&d2, &bits, sizeof(d2));
    *rebuilds = v[0];
    *fallbacks = v[1];
    *max_disp = std::sqrt((double)d2);
    return MDPF_OK;
}

const long long *learned_fallback_counter(const mdpf_ctx *c) {
    return c->learned != nullptr ? lh(c)->dev.lcount + 1 : nullptr;
}

DispCheck learned_disp_check(const mdpf_ctx *c) {
    const LearnedHost *h = lh(c);
    return DispCheck{h->dev.pos_build, h->dev.lflags, h->dev.half_skin2, h->rebuild_every};
}

}  // namespace mdpf

using namespace mdpf;

#define LGUARD(c)                                                                           \
    do {                                                                                    \
        if ((c) == nullptr) return MDPF_ERR_INVALID_ARG;                                    \
        if ((c)->sticky) return MDPF_ERR_CUDA;                                              \
        if ((c)->learned == nullptr) return fail((c), MDPF_ERR_UNSUPPORTED, "not in learned mode"); \
    } while (0)
#define LCK(c, x)                                                 \
    do {                                                          \
        cudaError_t e_ = (x);                                     \
        if (e_ != cudaSuccess) return cuda_fail((c), e_, #x);     \
    } while (0)

// Upload host positions and refresh the compute-side FP32 copy.
static int stage_positions(mdpf_ctx *c, const double *pos) {
    LCK(c, cudaMemcpyAsync(c->d_xc, pos, sizeof(double) * 3 * c->n, cudaMemcpyHostToDevice, c->stream));
    launch_pos4_from_x(c->d_xc, c->d_charge_s, c->d_pos4_c, c->n, c->n_pad, c->stream);
    return MDPF_OK;
}

extern "C" {

int mdpf_learned_neighbors(mdpf_ctx *c, const double *pos, int32_t max_per_atom, int32_t *count, int32_t *idx) {
    LGUARD(c);
    if (!pos || max_per_atom < 1) return fail(c, MDPF_ERR_INVALID_ARG, "pos is NULL or max_per_atom < 1");
    LearnedHost *h = lh(c);
    int rc = stage_positions(c, pos);
    if (rc != MDPF_OK) return rc;
    LCK(c, cudaMemsetAsync(c->d_status + 1, 0, sizeof(uint32_t), c->stream));
    LCK(c, learned_neighbors(h->dev, c->d_pos4_c, true, c->d_status + 1, c->stream));
    std::vector<int> cnt(c->n), rows((size_t)c->n * kKmax);
    uint32_t st = 0;
    LCK(c, cudaMemcpyAsync(cnt.data(), h->dev.nb_count, sizeof(int) * c->n, cudaMemcpyDeviceToHost, c->stream));
    LCK(c, cudaMemcpyAsync(rows.data(), h->dev.nb_idx, sizeof(int) * rows.size(), cudaMemcpyDeviceToHost, c->stream));
    LCK(c, cudaMemcpyAsync(&st, c->d_status + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    LCK(c, cudaStreamSynchronize(c->stream));
    if (st & MDPF_STATUS_NEIGHBOR_OVERFLOW) return fail(c, MDPF_ERR_NEIGHBOR_OVERFLOW, "neighbour row over capacity");
    for (int i = 0; i < c->n; ++i) {
        if (cnt[i] > max_per_atom) return fail(c, MDPF_ERR_NEIGHBOR_OVERFLOW, "row longer than max_per_atom");
        if (count) count[i] = cnt[i];
        if (idx) std::memcpy(idx + (size_t)i * max_per_atom, rows.data() + (size_t)i * kKmax, sizeof(int) * cnt[i]);
    }
    return MDPF_OK;
}

int mdpf_learned_features(mdpf_ctx *c, const double *pos, float *G) {
    LGUARD(c);
    if (!pos) return fail(c, MDPF_ERR_INVALID_ARG, "pos is NULL");
    LearnedHost *h = lh(c);
    int rc = stage_positions(c, pos);
    if (rc != MDPF_OK) return rc;
    LCK(c, cudaMemsetAsync(c->d_status + 1, 0, sizeof(uint32_t), c->stream));
    learned_begin(h->dev, c->stream);
    LCK(c, learned_neighbors(h->dev, c->d_pos4_c, true, c->d_status + 1, c->stream));
    learned_features(h->dev, c->d_pos4_c, true, c->stream);
    std::vector<float> rows((size_t)h->n_rows * kNFeat);
    uint32_t st = 0;
    if (!rows.empty())
        LCK(c, cudaMemcpyAsync(rows.data(), h->dev.G32, sizeof(float) * rows.size(), cudaMemcpyDeviceToHost, c->stream));
    LCK(c, cudaMemcpyAsync(&st, c->d_status + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    LCK(c, cudaStreamSynchronize(c->stream));
    if (st & MDPF_STATUS_NEIGHBOR_OVERFLOW) return fail(c, MDPF_ERR_NEIGHBOR_OVERFLOW, "neighbour row over capacity");
    if (G)
        for (int i = 0; i < c->n; ++i)
            std::memcpy(G + (size_t)i * kNFeat, rows.data() + (size_t)h->row_of[i] * kNFeat, sizeof(float) * kNFeat);
    return MDPF_OK;
}

int mdpf_learned_mlp(mdpf_ctx *c, const float *G, double *E_atom, float *dEdG) {
    LGUARD(c);
    if (!G) return fail(c, MDPF_ERR_INVALID_ARG, "G is NULL");
    LearnedHost *h = lh(c);
    LCK(c, cudaMemcpyAsync(h->d_Gin, G, sizeof(float) * (size_t)c->n * kNFeat, cudaMemcpyHostToDevice, c->stream));
    LCK(c, cudaMemsetAsync(c->d_status + 1, 0, sizeof(uint32_t), c->stream));
    learned_import_g(h->dev, h->d_Gin, c->stream);
    if (h->mlp_kernel == MDPF_MLP_SIMT_FP32)
        for (int i = 0; i < c->n; ++i)
            LCK(c, cudaMemcpyAsync(h->dev.G32 + (size_t)h->row_of[i] * kNFeat, G + (size_t)i * kNFeat,
                                   sizeof(float) * kNFeat, cudaMemcpyHostToDevice, c->stream));
    enqueue_mlp(h, c->d_status + 1, false, nullptr, c->stream);
    std::vector<double> E(h->n_rows);
    std::vector<float> g((size_t)h->n_rows * kNFeat);
    if (h->n_rows > 0) {
        LCK(c, cudaMemcpyAsync(E.data(), h->dev.E_row, sizeof(double) * h->n_rows, cudaMemcpyDeviceToHost, c->stream));
        if (h->dev.g_f32) {
            LCK(c, cudaMemcpyAsync(g.data(), h->dev.g, sizeof(float) * g.size(), cudaMemcpyDeviceToHost, c->stream));
        } else {
            std::vector<__nv_bfloat16> gb(g.size());
            LCK(c, cudaMemcpyAsync(gb.data(), h->dev.g, sizeof(__nv_bfloat16) * gb.size(), cudaMemcpyDeviceToHost,
                                   c->stream));
            LCK(c, cudaStreamSynchronize(c->stream));
            for (size_t q = 0; q < g.size(); ++q) g[q] = __bfloat162float(gb[q]);
        }
    }
    uint32_t st = 0;
    LCK(c, cudaMemcpyAsync(&st, c->d_status + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    LCK(c, cudaStreamSynchronize(c->stream));
    if (st & MDPF_STATUS_TIMEOUT) return fail(c, MDPF_ERR_TIMEOUT, "tensor-core MLP wait timed out");
    for (int i = 0; i < c->n; ++i) {
        const int r = h->row_of[i];
        if (E_atom) E_atom[i] = E[r];
        if (dEdG) std::memcpy(dEdG + (size_t)i * kNFeat, g.data() + (size_t)r * kNFeat, sizeof(float) * kNFeat);
    }
    return MDPF_OK;
}

int mdpf_learned_jvp(mdpf_ctx *c, const double *pos, const float *v, float *U) {
    LGUARD(c);
    if (!pos || !v) return fail(c, MDPF_ERR_INVALID_ARG, "pos or v is NULL");
    LearnedHost *h = lh(c);
    if (h->d_vin == nullptr) {
        cudaError_t e = lalloc(h, &h->d_vin, 3 * (size_t)c->n);
        if (e == cudaSuccess) e = lalloc(h, &h->d_U, (size_t)h->n_rows * kNFeat);
        if (e != cudaSuccess) return cuda_fail(c, e, "learned JVP scratch");
    }
    int rc = stage_positions(c, pos);
    if (rc != MDPF_OK) return rc;
    LCK(c, cudaMemcpyAsync(h->d_vin, v, sizeof(float) * 3 * c->n, cudaMemcpyHostToDevice, c->stream));
    LCK(c, cudaMemsetAsync(c->d_status + 1, 0, sizeof(uint32_t), c->stream));
    LCK(c, learned_neighbors(h->dev, c->d_pos4_c, true, c->d_status + 1, c->stream));
    learned_jvp(h->dev, c->d_pos4_c, h->d_vin, h->d_U, c->stream);
    std::vector<float> rows((size_t)h->n_rows * kNFeat);
    uint32_t st = 0;
    LCK(c, cudaMemcpyAsync(rows.data(), h->d_U, sizeof(float) * rows.size(), cudaMemcpyDeviceToHost, c->stream));
    LCK(c, cudaMemcpyAsync(&st, c->d_status + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    LCK(c, cudaStreamSynchronize(c->stream));
    if (st & MDPF_STATUS_NEIGHBOR_OVERFLOW) return fail(c, MDPF_ERR_NEIGHBOR_OVERFLOW, "neighbour row over capacity");
    if (U)
        for (int i = 0; i < c->n; ++i)
            std::memcpy(U + (size_t)i * kNFeat, rows.data() + (size_t)h->row_of[i] * kNFeat, sizeof(float) * kNFeat);
    return MDPF_OK;
}

int mdpf_learned_counters(mdpf_ctx *c, int64_t *rebuilds, int64_t *fallback_steps, int32_t *max_row) {
    LGUARD(c);
    long long v[4];
    LCK(c, cudaStreamSynchronize(c->stream));
    LCK(c, cudaMemcpy(v, lh(c)->dev.lcount, sizeof(v), cudaMemcpyDeviceToHost));
    if (rebuilds) *rebuilds = v[0];
    if (fallback_steps) *fallback_steps = v[1];
    if (max_row) *max_row = (int32_t)v[2];
    return MDPF_OK;
}

}  // extern "C"
