// Dynamic update (Section 3.5, Theorem update): apply a batch of link
// insertions/deletions to the canonical graph and inject the correction fluid
// d (P' - P) H into F, keeping H.
//
// The old links (key = source << 32 | target, value = old position) and the
// batch entries (value = nnz + batch index) are concatenated and sorted with
// the stable radix sort, so each run of equal keys lists the old link first
// and then the batch operations in batch order; the last operation decides.
// A source j is "touched" when its set of out-links (or a weight) changes,
// i.e. when column j of P changes; only those columns contribute to
// d (P' - P) H, and for them the whole old column is withdrawn and the whole
// new column injected (every entry changes when out(j) or W_j changes).
#include <cuda_runtime.h>

#include "di_internal.cuh"

namespace di {

using Off = uint32_t;

__global__ void k_check_batch(const int32_t *src, const int32_t *dst, const double *w, const int8_t *op,
                              int64_t m, int64_t n, unsigned *err)
{
    unsigned e = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (src[k] < 0 || src[k] >= n || dst[k] < 0 || dst[k] >= n) e |= 1u;
        if (op[k] != 1 && op[k] != -1) e |= 2u;
        if (w && op[k] == 1 && !(isfinite(w[k]) && w[k] > 0.0)) e |= 4u;
    }
    if (e) atomicOr(err, e);
}

__global__ void k_keys_old(const Off *rp, const int32_t *col, int64_t n, uint64_t *keys, uint32_t *vals)
{
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < n; r += nwarps)
        for (Off e = rp[r] + lane; e < rp[r + 1]; e += 32) {
            keys[e] = ((uint64_t)r << 32) | (uint32_t)col[e];
            vals[e] = e;
        }
}

__global__ void k_keys_batch(const int32_t *src, const int32_t *dst, int64_t m, int64_t nnz,
                             uint64_t *keys, uint32_t *vals)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        keys[nnz + k] = ((uint64_t)(uint32_t)src[k] << 32) | (uint32_t)dst[k];
        vals[nnz + k] = (uint32_t)(nnz + k);
    }
}

// Resolve each run of equal keys: keep[e] = 1 at a run start whose link is
// present after the batch; nw[e] its weight; touched[source] = 1 if the
// link's presence or weight changed.
__global__ void k_resolve(const uint64_t *keys, const uint32_t *vals, int64_t tot, int64_t nnz,
                          const double *wold, const double *wb, const int8_t *op, uint8_t *keep,
                          double *nw, uint8_t *touched)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[e];
        if (e > 0 && keys[e - 1] == key) {
            keep[e] = 0;
            continue;
        }
        int64_t q = e;
        const bool has_old = vals[e] < (uint64_t)nnz;
        int64_t last = -1;
        while (q < tot && keys[q] == key) {
            if (vals[q] >= (uint64_t)nnz) last = (int64_t)vals[q] - nnz;
            q++;
        }
        bool present = has_old;
        double wv = has_old && wold ? wold[vals[e]] : 1.0;
        if (last >= 0) {
            present = op[last] == 1;
            if (present) wv = wb ? wb[last] : 1.0;
        }
        keep[e] = present ? 1 : 0;
        nw[e] = wv;
        bool changed = present != has_old;
        if (present && has_old && wold && wv != wold[vals[e]]) changed = true;
        if (changed) touched[key >> 32] = 1;
    }
}

__global__ void k_compact_new(const uint64_t *keys, const uint8_t *keep, const uint64_t *pos, int64_t tot,
                              const double *nw, int32_t *col, uint32_t *rows, double *wout)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[e]) continue;
        const int64_t k = (int64_t)pos[e];
        col[k] = (int32_t)(uint32_t)(keys[e] & 0xffffffffull);
        rows[k] = (uint32_t)(keys[e] >> 32);
        if (wout) wout[k] = nw[e];
    }
}

template <typename P>
__global__ void k_row_ptr_u(const uint32_t *rows, int64_t m, int64_t n, P *rp)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = rows[k];
        const int64_t rprev = k > 0 ? (int64_t)rows[k - 1] : -1;
        for (int64_t q = rprev + 1; q <= r; q++) rp[q] = (P)k;
        if (k == m - 1)
            for (int64_t q = r + 1; q <= n; q++) rp[q] = (P)m;
    }
}

__global__ void k_zero_u32(uint32_t *a, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = 0;
}

__global__ void k_row_sums_u(const uint32_t *rp, const double *w, int64_t n, double *wsum,
                             unsigned long long *ndang)
{
    unsigned long long c = 0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = rp[j], b = rp[j + 1];
        if (a == b) c++;
        if (wsum) {
            double s = 0.0;
            for (uint32_t e = a; e < b; e++) s = (e == a) ? w[e] : s + w[e];
            wsum[j] = s;
        }
    }
    if (c) atomicAdd(ndang, c);
}

// F += sign * d H_j P[:, j] for every touched column j (one warp per node).
__global__ void k_inject(const uint8_t *touched, const Off *rp, const int32_t *col, const double *w,
                         const double *wsum, const double *H, int64_t n, double sd, double *F)
{
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = warp; j < n; j += nwarps) {
        if (!touched[j]) continue;
        const Off a = rp[j], b = rp[j + 1];
        if (a == b) continue;
        const double h = sd * H[j];
        const double unit = w ? h / wsum[j] : h / (double)(b - a);
        for (Off e = a + lane; e < b; e += 32) atomicAdd(F + col[e], w ? unit * w[e] : unit);
    }
}

static unsigned grid_for(int64_t work, int threads)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

di_status update_edges(di_graph_s *g, di_state_s *st, int64_t m, const int32_t *src, const int32_t *dst,
                       const double *wb, const int8_t *op, cudaStream_t s)
{
    const int64_t n = g->n, nnz = g->nnz;
    const int64_t tot = nnz + m;
    if (tot >= (int64_t(1) << 32)) return DI_ERR_INVALID_ARG;
    Temps t(s);
    unsigned *err;
    DI_TRY(t.get(&err, 1));
    DI_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
    k_check_batch<<<grid_for(m, 256), 256, 0, s>>>(src, dst, g->weighted ? wb : nullptr, op, m, n, err);
    count_launches(1);
    unsigned herr = 0;
    DI_CUDA(cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    if (herr) return DI_ERR_INVALID_ARG;
    if (m == 0) return DI_OK;

    uint64_t *keys, *keys2, *pos, *total;
    uint32_t *vals, *vals2;
    uint8_t *keep, *touched;
    double *nw;
    DI_TRY(t.get(&keys, tot));
    DI_TRY(t.get(&keys2, tot));
    DI_TRY(t.get(&vals, tot));
    DI_TRY(t.get(&vals2, tot));
    DI_TRY(t.get(&keep, tot));
    DI_TRY(t.get(&pos, tot));
    DI_TRY(t.get(&total, 1));
    DI_TRY(t.get(&nw, tot));
    DI_TRY(t.get(&touched, n));
    DI_CUDA(cudaMemsetAsync(touched, 0, n, s));
    const Off *rp = static_cast<const Off *>(g->rp);
    k_keys_old<<<grid_for(n * 32, 256), 256, 0, s>>>(rp, g->col, n, keys, vals);
    count_launches(1);
    k_keys_batch<<<grid_for(m, 256), 256, 0, s>>>(src, dst, m, nnz, keys, vals);
    count_launches(1);
    const int b = bits_for(n);
    int lo[16], cnt[16], np = 0;
    for (int x = 0; x < b; x += 8) { lo[np] = x; cnt[np] = b - x < 8 ? b - x : 8; np++; }
    for (int x = 0; x < b; x += 8) { lo[np] = 32 + x; cnt[np] = b - x < 8 ? b - x : 8; np++; }
    DI_TRY(radix_sort_pairs(&keys, &vals, &keys2, &vals2, tot, lo, cnt, np, s));
    k_resolve<<<grid_for(tot, 256), 256, 0, s>>>(keys, vals, tot, nnz, g->w, g->weighted ? wb : nullptr,
                                                 op, keep, nw, touched);
    count_launches(1);
    DI_TRY(scan_exclusive<uint8_t>(keep, pos, tot, total, s));
    uint64_t mnew = 0;
    DI_CUDA(cudaMemcpyAsync(&mnew, total, sizeof(mnew), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));

    // new canonical structure
    int32_t *ncol = nullptr;
    double *nwv = nullptr, *nwsum = nullptr;
    uint32_t *nrp = nullptr, *rows = nullptr;
    DI_TRY(t.get(&rows, mnew));
    DI_TRY(dalloc_t(&ncol, mnew, s));
    DI_TRY(dalloc_t(&nrp, n + 1, s));
    if (g->weighted) {
        DI_TRY(dalloc_t(&nwv, mnew, s));
        DI_TRY(dalloc_t(&nwsum, n, s));
    }
    k_compact_new<<<grid_for(tot, 256), 256, 0, s>>>(keys, keep, pos, tot, nw, ncol, rows, nwv);
    count_launches(1);
    if (mnew == 0) {
        k_zero_u32<<<grid_for(n + 1, 256), 256, 0, s>>>(nrp, n + 1);
        count_launches(1);
    } else {
        k_row_ptr_u<uint32_t><<<grid_for(mnew, 256), 256, 0, s>>>(rows, (int64_t)mnew, n, nrp);
        count_launches(1);
    }
    unsigned long long *ndang;
    DI_TRY(t.get(&ndang, 1));
    DI_CUDA(cudaMemsetAsync(ndang, 0, sizeof(unsigned long long), s));
    k_row_sums_u<<<grid_for(n, 256), 256, 0, s>>>(nrp, nwv, n, nwsum, ndang);
    count_launches(1);

    // F += d (P' - P) H: withdraw the old columns, inject the new ones
    if (st) {
        k_inject<<<grid_for(n * 32, 256), 256, 0, s>>>(touched, rp, g->col, g->w, g->wsum, st->H, n,
                                                       -st->d, st->F);
        count_launches(1);
        k_inject<<<grid_for(n * 32, 256), 256, 0, s>>>(touched, nrp, ncol, nwv, nwsum, st->H, n, st->d,
                                                       st->F);
        count_launches(1);
    }
    DI_CUDA(cudaGetLastError());
    unsigned long long hd = 0;
    DI_CUDA(cudaMemcpyAsync(&hd, ndang, sizeof(hd), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));

    // install P'
    dfree(g->rp, s);
    dfree(g->col, s);
    dfree(g->w, s);
    dfree(g->wsum, s);
    dfree(g->cp, s);
    dfree(g->crow, s);
    dfree(g->cw, s);
    g->rp = nrp;
    g->col = ncol;
    g->w = nwv;
    g->wsum = nwsum;
    g->cp = nullptr;
    g->crow = nullptr;
    g->cw = nullptr;
    g->nnz = (int64_t)mnew;
    g->n_dangling = (int64_t)hd;
    DI_CUDA(cudaStreamSynchronize(s));
    return DI_OK;
}

}  // namespace di
