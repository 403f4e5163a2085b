// Exclusion set (1-2 and 1-3 partners), derived angles and the skip masks of
// the all-pairs kernels' row decomposition, built on the device.
//
// A pair (i, j) is left out of the nonbonded sum when the atoms are bonded or
// share a bonded neighbour; every pair of bonds that meets at an atom carries
// one harmonic angle.  Both sets come from the bond graph: adjacency rows are
// built by a counting sort, each row is sorted, and an atom's exclusion row is
// the sorted union of its neighbours and its neighbours' neighbours.
#include "mdpf_internal.cuh"

namespace mdpf {
namespace {

__global__ void k_degree(const int2 *bonds, int nb, int *deg) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) {
        atomicAdd(&deg[bonds[b].x], 1);
        atomicAdd(&deg[bonds[b].y], 1);
    }
}

// Exclusive prefix sum of in[0..n) into out[0..n], out[n] = total.  One block
// of 1024 threads walks the array in chunks (set-up only).
__global__ void k_scan(const int *in, int *out, int n) {
    __shared__ int s[1024];
    __shared__ int carry;
    const int t = threadIdx.x;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        int v = (base + t < n) ? in[base + t] : 0;
        s[t] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            int add = (t >= off) ? s[t - off] : 0;
            __syncthreads();
            s[t] += add;
            __syncthreads();
        }
        if (base + t < n) out[base + t] = carry + s[t] - v;
        __syncthreads();
        if (t == 1023) carry += s[1023];
        __syncthreads();
    }
    if (t == 0) out[n] = carry;
}

__global__ void k_adj_fill(const int2 *bonds, int nb, const int *off, int *cursor, int *adj) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) {
        int a = bonds[b].x, c = bonds[b].y;
        adj[off[a] + atomicAdd(&cursor[a], 1)] = c;
        adj[off[c] + atomicAdd(&cursor[c], 1)] = a;
    }
}

__global__ void k_row_sort(const int *off, int *data, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = off[i], hi = off[i + 1];
    for (int p = lo + 1; p < hi; ++p) {
        int v = data[p], q = p - 1;
        while (q >= lo && data[q] > v) {
            data[q + 1] = data[q];
            --q;
        }
        data[q + 1] = v;
    }
}

// Exclusion row of atom i.  Count mode (out_off == nullptr) writes the row
// length to count[i]; write mode stores the sorted row at out_idx[out_off[i]].
__global__ void k_excl_rows(const int *adj_off, const int *adj, int n, int *count, const int *out_off,
                            int *out_idx, uint32_t *status) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cand[kMaxExclPerAtom + 1];
    int m = 0;
    bool over = false;
    for (int p = adj_off[i]; p < adj_off[i + 1]; ++p) {
        int j = adj[p];
        if (m <= kMaxExclPerAtom) cand[m++] = j; else over = true;
        for (int q = adj_off[j]; q < adj_off[j + 1]; ++q) {
            int k = adj[q];
            if (k == i) continue;
            if (m <= kMaxExclPerAtom) cand[m++] = k; else over = true;
        }
    }
    // insertion sort + unique
    for (int p = 1; p < m; ++p) {
        int v = cand[p], q = p - 1;
        while (q >= 0 && cand[q] > v) {
            cand[q + 1] = cand[q];
            --q;
        }
        cand[q + 1] = v;
    }
    int u = 0;
    for (int p = 0; p < m; ++p)
        if (u == 0 || cand[p] != cand[u - 1]) cand[u++] = cand[p];
    if (over || u > kMaxExclPerAtom) {
        atomicOr(status, MDPF_STATUS_NEIGHBOR_OVERFLOW);
        u = 0;
    }
    if (out_off == nullptr) {
        count[i] = u;
    } else {
        int base = out_off[i];
        for (int p = 0; p < u; ++p) out_idx[base + p] = cand[p];
    }
}

__global__ void k_angle_count(const int *adj_off, int n, int *cnt) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) {
        int d = adj_off[v + 1] - adj_off[v];
        cnt[v] = d * (d - 1) / 2;
    }
}

__global__ void k_angle_fill(const int *adj_off, const int *adj, const int *ang_off, int n, int4 *angles) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int w = ang_off[v];
    for (int p = adj_off[v]; p < adj_off[v + 1]; ++p)
        for (int q = p + 1; q < adj_off[v + 1]; ++q) angles[w++] = make_int4(adj[p], v, adj[q], 0);
}

// Skip masks of the row decomposition: word (g, c, a) holds bit l for the
// pair (16 g + a, 32 c + l).  Thread i sets the bits of its own words only:
// the atom itself and its excluded partners.
__global__ void k_row_masks(const int *excl_off, const int *excl_idx, int n, int C, uint32_t *mask) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t *row = mask + (size_t)(i / 16) * C * 16 + (i % 16);
    row[(size_t)(i / kTile) * 16] |= 1u << (i % kTile);
    for (int p = excl_off[i]; p < excl_off[i + 1]; ++p) {
        int j = excl_idx[p];
        row[(size_t)(j / kTile) * 16] |= 1u << (j % kTile);
    }
}

// Padding atoms (index >= n) never interact: all bits of a padding row, and
// the bits of padding j-atoms in every row.
__global__ void k_row_pad(int n, int n_groups, int C, uint32_t *mask) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= (int64_t)n_groups * C * 16) return;
    const int a = (int)(w % 16), c = (int)((w / 16) % C), g = (int)(w / (16 * (int64_t)C));
    const int i = 16 * g + a;
    if (i >= n) {
        mask[w] = 0xffffffffu;
        return;
    }
    const int vj = n - kTile * c;   // real j-atoms in chunk c
    if (vj >= kTile) return;
    mask[w] |= vj <= 0 ? 0xffffffffu : (0xffffffffu << vj);
}

}  // namespace

int build_exclusions(mdpf_ctx *ctx) {
    const int n = ctx->n, nb = ctx->n_bonds;
    cudaStream_t s = ctx->stream;
    int *d_deg = nullptr, *d_adj_off = nullptr, *d_adj = nullptr, *d_cursor = nullptr, *d_cnt = nullptr,
        *d_ang_off = nullptr;
    cudaError_t e;
    auto cleanup = [&]() {
        cudaFree(d_deg);
        cudaFree(d_adj_off);
        cudaFree(d_adj);
        cudaFree(d_cursor);
        cudaFree(d_cnt);
        cudaFree(d_ang_off);
    };
#define TRY(x)                                      \
    do {                                            \
        e = (x);                                    \
        if (e != cudaSuccess) {                     \
            cleanup();                              \
            return cuda_fail(ctx, e, #x);           \
        }                                           \
    } while (0)
    TRY(cudaMalloc(&d_deg, sizeof(int) * (n + 1)));
    TRY(cudaMalloc(&d_adj_off, sizeof(int) * (n + 1)));
    TRY(cudaMalloc(&d_adj, sizeof(int) * (2 * (size_t)nb + 1)));
    TRY(cudaMalloc(&d_cursor, sizeof(int) * (n + 1)));
    TRY(cudaMalloc(&d_cnt, sizeof(int) * (n + 1)));
    TRY(cudaMalloc(&d_ang_off, sizeof(int) * (n + 1)));
    TRY(cudaMemsetAsync(d_deg, 0, sizeof(int) * (n + 1), s));
    TRY(cudaMemsetAsync(d_cursor, 0, sizeof(int) * (n + 1), s));
    const int B = 256;
    if (nb > 0) k_degree<<<(nb + B - 1) / B, B, 0, s>>>(ctx->d_bonds, nb, d_deg);
    k_scan<<<1, 1024, 0, s>>>(d_deg, d_adj_off, n);
    if (nb > 0) k_adj_fill<<<(nb + B - 1) / B, B, 0, s>>>(ctx->d_bonds, nb, d_adj_off, d_cursor, d_adj);
    k_row_sort<<<(n + B - 1) / B, B, 0, s>>>(d_adj_off, d_adj, n);
    // exclusions: count, scan, fill
    k_excl_rows<<<(n + B - 1) / B, B, 0, s>>>(d_adj_off, d_adj, n, d_cnt, nullptr, nullptr, ctx->d_status);
    TRY(cudaMalloc(&ctx->d_excl_off, sizeof(int) * (n + 1)));
    k_scan<<<1, 1024, 0, s>>>(d_cnt, ctx->d_excl_off, n);
    // angles: count, scan
    k_angle_count<<<(n + B - 1) / B, B, 0, s>>>(d_adj_off, n, d_cnt);
    k_scan<<<1, 1024, 0, s>>>(d_cnt, d_ang_off, n);
    int totals[2] = {0, 0};
    uint32_t status = 0;
    TRY(cudaMemcpyAsync(&totals[0], ctx->d_excl_off + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    TRY(cudaMemcpyAsync(&totals[1], d_ang_off + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    TRY(cudaMemcpyAsync(&status, ctx->d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    if (status & MDPF_STATUS_NEIGHBOR_OVERFLOW) {
        cleanup();
        return fail(ctx, MDPF_ERR_NEIGHBOR_OVERFLOW, "an atom has more than 255 excluded partners");
    }
    ctx->excl_total = totals[0];
    ctx->n_angles = totals[1];
    TRY(cudaMalloc(&ctx->d_excl_idx, sizeof(int) * ((size_t)totals[0] + 1)));
    k_excl_rows<<<(n + B - 1) / B, B, 0, s>>>(d_adj_off, d_adj, n, nullptr, ctx->d_excl_off, ctx->d_excl_idx,
                                               ctx->d_status);
    TRY(cudaMalloc(&ctx->d_angles, sizeof(int4) * ((size_t)totals[1] + 1)));
    k_angle_fill<<<(n + B - 1) / B, B, 0, s>>>(d_adj_off, d_adj, d_ang_off, n, ctx->d_angles);
    // skip masks of the row decomposition
    // only groups and chunks that hold real atoms take part (padding rows and padding j-atoms inside them are
    // masked)
    const int C = (n + kTile - 1) / kTile, NG = (n + 15) / 16;
    ctx->n_groups = NG;
    ctx->n_chunks = C;
    const size_t nwords = (size_t)NG * C * 16;
    TRY(cudaMalloc(&ctx->d_row_mask, sizeof(uint32_t) * nwords));
    TRY(cudaMemsetAsync(ctx->d_row_mask, 0, sizeof(uint32_t) * nwords, s));
    k_row_masks<<<(n + B - 1) / B, B, 0, s>>>(ctx->d_excl_off, ctx->d_excl_idx, n, C, ctx->d_row_mask);
    k_row_pad<<<(unsigned)((nwords + B - 1) / B), B, 0, s>>>(n, NG, C, ctx->d_row_mask);
    TRY(cudaGetLastError());
    TRY(cudaStreamSynchronize(s));
    cleanup();
#undef TRY
    return MDPF_OK;
}

}  // namespace mdpf
