// All-pairs LJ + Coulomb evaluation that allocates no device memory.
//
// Some callers cannot call cudaMalloc when they need forces: an MD engine that
// calls its force provider from inside its step loop under its own memory
// pool, code that must not trigger the device synchronisation cudaMalloc and
// cudaFree imply, or a host that only hands out pointers into buffers it
// already owns.  mdpf_pairs_noalloc serves them: the caller passes its own
// device inputs and outputs, and the working memory the kernels need (FP32
// positions, fixed-point force accumulators, work items, tile flags) lives in
// one fixed-size array in the library's device data segment, which every GPU
// that loads the library holds until the process exits.
//
// The arithmetic is the library's all-pairs routine (forcefield.cuh), so for
// a system without bonds the results equal those of mdpf_compute_device.
// The paper has no counterpart of this entry point.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <mutex>

#include "forcefield.cuh"

namespace mdpf {
namespace {

constexpr int kNaMaxAtoms = 2048;                             // largest system accepted
constexpr int kNaTiles = kNaMaxAtoms / kTile;                 // 64
constexpr int kNaTilePairs = kNaTiles * (kNaTiles + 1) / 2;   // 2080
constexpr int kNaMaxItems = (kNaTiles / 2) * (kNaTiles / 2 - 1) + 3 * (kNaTiles / 2);  // 1088

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kOffPos = 0;
constexpr size_t kOffLj = kOffPos + align256(sizeof(float4) * kNaMaxAtoms);
constexpr size_t kOffFx = kOffLj + align256(sizeof(float2) * kNaMaxAtoms);
constexpr size_t kOffEfx = kOffFx + align256(sizeof(unsigned long long) * 3 * kNaMaxAtoms);
constexpr size_t kOffItems = kOffEfx + align256(sizeof(unsigned long long) * E_SLOTS);
constexpr size_t kOffMask = kOffItems + align256(sizeof(int4) * kNaMaxItems);
constexpr size_t kOffFlag = kOffMask + align256(sizeof(uint32_t) * kNaTilePairs * kTile);
constexpr size_t kOffStatus = kOffFlag + align256(sizeof(uint32_t) * kNaTilePairs);
constexpr size_t kNaScratchBytes = kOffStatus + 256;          // ~390 KB

// Shared by every call on a device; see mdpf_pairs_noalloc in include/mdpf.h.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

struct NaView {
    float4 *pos4;
    float2 *lj;
    unsigned long long *fx, *efx;
    int4 *items;
    uint32_t *mask, *flag, *status;
};

NaView view(unsigned char *base) {
    NaView v;
    v.pos4 = reinterpret_cast<float4 *>(base + kOffPos);
    v.lj = reinterpret_cast<float2 *>(base + kOffLj);
    v.fx = reinterpret_cast<unsigned long long *>(base + kOffFx);
    v.efx = reinterpret_cast<unsigned long long *>(base + kOffEfx);
    v.items = reinterpret_cast<int4 *>(base + kOffItems);
    v.mask = reinterpret_cast<uint32_t *>(base + kOffMask);
    v.flag = reinterpret_cast<uint32_t *>(base + kOffFlag);
    v.status = reinterpret_cast<uint32_t *>(base + kOffStatus);
    return v;
}

struct NaParams {
    float a[4], b[4];   // sigma/2 and sqrt(24 eps) per element
    float sqrt_ke;
};

// Fill the scratch for one call: FP32 positions and parameters (padding atoms
// far away with zero charge and zero eps, so every pair touching one adds
// exactly zero), cleared accumulators, cleared tile flags/masks, work items.
__global__ void k_na_prep(NaView v, int n, int n_pad, int T, int n_items, int n_mask_words, const double *x,
                          const int32_t *el, const double *q, NaParams prm) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n_pad) {
        if (g < n) {
            const int e = el[g];
            const bool ok = e >= 0 && e < 4;
            v.pos4[g] = make_float4((float)x[3 * g], (float)x[3 * g + 1], (float)x[3 * g + 2],
                                    (float)(q[g] * prm.sqrt_ke));
            v.lj[g] = ok ? make_float2(prm.a[e], prm.b[e]) : make_float2(nanf(""), nanf(""));
        } else {
            v.pos4[g] = make_float4(1.0e5f + 8.0f * (float)g, 1.0e5f, 1.0e5f, 0.f);
            v.lj[g] = make_float2(0.f, 0.f);
        }
        v.fx[3 * g] = v.fx[3 * g + 1] = v.fx[3 * g + 2] = 0ull;
    }
    if (g < E_SLOTS) v.efx[g] = 0ull;
    if (g < 4) v.status[g] = 0u;
    if (g < n_mask_words) v.mask[g] = 0u;
    if (g < T * (T + 1) / 2) v.flag[g] = 0u;
    if (g < n_items) {
        // 64x32 items of row p occupy [p (T - 1 - p), (p + 1)(T - 2 - p)); the diagonal blocks follow
        const int n64 = (T / 2) * (T / 2 - 1);
        if (g < n64) {
            int p = 0;
            while ((p + 1) * (T - 2 - p) <= g) ++p;
            const int J = 2 * p + 2 + (g - p * (T - 1 - p));
            v.items[g] = make_int4(ITEM_OFF64, p, J, 0);
        } else {
            const int d = g - n64, p = d / 3, r = d % 3;
            v.items[g] = r == 0 ? make_int4(ITEM_OFF32, 2 * p, 2 * p + 1, 0)
                                : make_int4(ITEM_SELF, 2 * p + (r - 1), 0, 0);
        }
    }
}

__global__ void __launch_bounds__(256, 2) k_na_pairs(PlainDev p, unsigned long long *fx, unsigned long long *efx) {
    __shared__ JTile jt[8];
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    float elj = 0.f, ec = 0.f;
    bool bad = false;
    for (int it = warp; it < p.n_items; it += nwarps) nonbonded_item<true>(p, it, lane, jt[threadIdx.x >> 5], fx, elj, ec, bad);
    if (bad) atomicOr(p.status, MDPF_STATUS_NONFINITE);
    const double e_lj = warp_sum_d((double)elj * (1.0 / 6.0));
    const double e_c = warp_sum_d((double)ec);
    if (lane == 0) {
        fx_add_d(&efx[E_LJ], e_lj);
        fx_add_d(&efx[E_COUL], e_c);
    }
}

__global__ void k_na_out(const unsigned long long *fx, const unsigned long long *efx, const uint32_t *status, int n,
                         double *energy, float *forces) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (forces != nullptr && g < 3 * n) forces[g] = (float)fx_val(fx[g]);
    if (g == 0 && energy != nullptr) {
        const double e = fx_val(efx[E_LJ]) + fx_val(efx[E_COUL]);
        *energy = (*status & MDPF_STATUS_NONFINITE) ? nan("") : e;
    }
}

std::mutex g_na_mutex;
unsigned char *g_na_ptr[64] = {nullptr};
CUcontext g_na_ctx[64] = {nullptr};      // the context each cached address belongs to

// The calling thread's current context (the driver call reached through the runtime, so the library
// needs no link-time dependency on the driver library), or null when it cannot be determined.
CUcontext current_context() {
    static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
        looked_up = true;
    }
    CUcontext c = nullptr;
    if (fn == nullptr || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

}  // namespace
}  // namespace mdpf

using namespace mdpf;

extern "C" int mdpf_pairs_noalloc(int32_t n, const double *d_pos, const int32_t *d_element, const double *d_charge,
                                  const double lj_sigma[4], const double lj_eps[4], double coulomb_k,
                                  double *d_energy, float *d_forces, void *cuda_stream) {
    if (n < 1 || n > kNaMaxAtoms)
        return fail(nullptr, MDPF_ERR_INVALID_ARG,
                    "mdpf_pairs_noalloc: n_atoms must be in [1, 2048] (its fixed scratch holds 2048 atoms)");
    if (!d_pos || !d_element || !d_charge || !lj_sigma || !lj_eps || (!d_energy && !d_forces))
        return fail(nullptr, MDPF_ERR_INVALID_ARG, "mdpf_pairs_noalloc: NULL pointer argument");
    for (int e = 0; e < 4; ++e)
        if (!(lj_sigma[e] >= 0.0) || !(lj_eps[e] >= 0.0) || !std::isfinite(lj_sigma[e]) || !std::isfinite(lj_eps[e]))
            return fail(nullptr, MDPF_ERR_INVALID_ARG, "mdpf_pairs_noalloc: LJ parameters must be finite and >= 0");
    const double ke = coulomb_k > 0 ? coulomb_k : kCoulombDefault;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(nullptr, MDPF_ERR_UNSUPPORTED, "mdpf_pairs_noalloc: device index >= 64");
    unsigned char *base = nullptr;
    {
        // once per device (and again if the device's context was replaced, e.g. after cudaDeviceReset),
        // with that device current: the device address of the scratch array
        std::lock_guard<std::mutex> lock(g_na_mutex);
        const CUcontext cur = current_context();   // null before the runtime made a context current: look up
        if (g_na_ptr[dev] == nullptr || cur == nullptr || cur != g_na_ctx[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
            g_na_ptr[dev] = static_cast<unsigned char *>(ptr);
            g_na_ctx[dev] = cur;
        }
        base = g_na_ptr[dev];
    }
    const int n_pad = (n + kPad - 1) / kPad * kPad;
    const int T = n_pad / kTile;
    const int n_items = (T / 2) * (T / 2 - 1) + 3 * (T / 2);
    const int n_mask_words = T * (T + 1) / 2 * kTile;
    NaView v = view(base);
    NaParams prm;
    for (int k = 0; k < 4; ++k) {
        prm.a[k] = (float)(0.5 * lj_sigma[k]);
        prm.b[k] = (float)std::sqrt(24.0 * lj_eps[k]);
    }
    prm.sqrt_ke = (float)std::sqrt(ke);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int m = n_mask_words > n_pad ? n_mask_words : n_pad;
    k_na_prep<<<(m + 255) / 256, 256, 0, s>>>(v, n, n_pad, T, n_items, n_mask_words, d_pos, d_element, d_charge, prm);
    PlainDev p{};
    p.n = n;
    p.n_pad = n_pad;
    p.n_tiles = T;
    p.pos4 = v.pos4;
    p.lj = v.lj;
    p.tile_mask = v.mask;
    p.tile_flag = v.flag;
    p.items = v.items;
    p.n_items = n_items;
    p.status = v.status;
    int blocks = (n_items * 32 + 255) / 256;
    k_na_pairs<<<blocks, 256, 0, s>>>(p, v.fx, v.efx);
    k_na_out<<<(3 * n + 255) / 256, 256, 0, s>>>(v.fx, v.efx, v.status, n, d_energy, d_forces);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "mdpf_pairs_noalloc launch");
    return MDPF_OK;
}
