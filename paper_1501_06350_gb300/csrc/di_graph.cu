// Graph builder (Section 2.1, Eq. def-p): validation, canonical out-CSR
// (rows sorted by target, duplicate links merged with weights summed in input
// order), row weight sums W_j, dangling count, and the in-link structure.
//
// Every link becomes one 64-bit key (source << 32 | target) carrying its input
// position; a stable LSD radix sort over the target bits then the source bits
// orders the keys by (source, target) with ties in input order, which makes the
// merge of duplicates and the resulting index arrays bit-exact.
#include <cuda_runtime.h>

#include "di_internal.cuh"

namespace di {

enum : unsigned { ERR_PTR = 1u, ERR_IDX = 2u, ERR_W = 4u };

__global__ void k_validate(const int64_t *ptr, const int32_t *idx, const void *w, int wdt, int64_t n,
                           int64_t nnz, unsigned *err)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned e = 0;
    if (tid == 0 && (ptr[0] != 0 || ptr[n] != nnz)) e |= ERR_PTR;
    for (int64_t r = tid; r < n; r += stride)
        if (ptr[r + 1] < ptr[r]) e |= ERR_PTR;
    for (int64_t k = tid; k < nnz; k += stride) {
        int32_t c = idx[k];
        if (c < 0 || (int64_t)c >= n) e |= ERR_IDX;
        if (wdt == DI_W_F32) {
            float x = static_cast<const float *>(w)[k];
            if (!(isfinite(x) && x > 0.0f)) e |= ERR_W;
        } else if (wdt == DI_W_F64) {
            double x = static_cast<const double *>(w)[k];
            if (!(isfinite(x) && x > 0.0)) e |= ERR_W;
        }
    }
    if (e) atomicOr(err, e);
}

// Row lookup table for link-parallel kernels: tab[q] is the row holding link
// q * 2^KEY_BUCKET_SHIFT (each such link lies in exactly one non-empty row,
// which writes it); tab[nbk] = n - 1.
template <typename P>
__global__ void k_bucket_rows(const P *ptr, int64_t n, int64_t nbk, uint32_t *tab)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = ptr[r], b = ptr[r + 1];
        if (a >= b) continue;
        const int64_t q0 = (a + (1 << KEY_BUCKET_SHIFT) - 1) >> KEY_BUCKET_SHIFT;
        const int64_t q1 = (b - 1) >> KEY_BUCKET_SHIFT;
        for (int64_t q = q0; q <= q1; q++) tab[q] = (uint32_t)r;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) tab[nbk] = (uint32_t)(n - 1);
}

// key = (source << 32 | target), value = input position, for every input
// link, one thread per link: the row of link e is the largest r with
// ptr[r] <= e, searched between the rows of the bucket starts around e.
__global__ void k_make_keys(const int64_t *ptr, const int32_t *idx, int64_t n, int64_t nnz, int layout,
                            const uint32_t *tab, uint64_t *keys, uint32_t *vals)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e >> KEY_BUCKET_SHIFT;
        int64_t lo = __ldg(tab + q), hi = __ldg(tab + q + 1);   // ptr[lo] <= e, row(e) <= hi
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (__ldg(ptr + mid) <= e) lo = mid;
            else hi = mid - 1;
        }
        const uint64_t r = (uint64_t)lo;
        const uint64_t t = (uint32_t)idx[e];
        keys[e] = layout == DI_LAYOUT_CSR ? ((r << 32) | t) : ((t << 32) | r);
        vals[e] = (uint32_t)e;
    }
}

__global__ void k_mark_runs(const uint64_t *keys, int64_t m, uint8_t *keep)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        keep[e] = (e == 0 || keys[e] != keys[e - 1]) ? 1 : 0;
}

// For every run start: write the merged link (low 32 bits of the key) and the
// high 32 bits (row id) to `rows`; weights summed over the run in order.
__global__ void k_compact(const uint64_t *keys, const uint32_t *vals, const uint8_t *keep,
                          const uint64_t *pos, int64_t m, const void *w, int wdt, int32_t *col,
                          uint32_t *rows, double *wout)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[e]) continue;
        const uint64_t key = keys[e];
        const int64_t k = (int64_t)pos[e];
        col[k] = (int32_t)(uint32_t)(key & 0xffffffffull);
        rows[k] = (uint32_t)(key >> 32);
        if (wout) {
            double s = 0.0;
            int64_t q = e;
            do {
                const uint32_t v = vals[q];
                const double x = wdt == DI_W_F32 ? (double)static_cast<const float *>(w)[v]
                                                 : static_cast<const double *>(w)[v];
                s = (q == e) ? x : s + x;
                q++;
            } while (q < m && keys[q] == key);
            wout[k] = s;
        }
    }
}

// Row pointers from the (sorted) row id of every merged link.
template <typename P>
__global__ void k_row_ptr(const uint32_t *rows, int64_t m, int64_t n, P *rp)
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

template <typename P>
__global__ void k_fill(P *a, int64_t n, P v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

// W_j, left-to-right in row order (Eq. def-p denominator); dangling count.
__global__ void k_row_sums(const uint32_t *rp, const double *w, int64_t n, double *wsum,
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
    // one atomic per warp (one counter for the whole grid)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(ndang, c);
}

__global__ void k_expand_rows(const uint32_t *rp, int64_t n, const int32_t *col, uint64_t *keys,
                              uint32_t *vals)
{
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < n; r += nwarps)
        for (uint32_t e = rp[r] + lane; e < rp[r + 1]; e += 32) {
            keys[e] = ((uint64_t)(uint32_t)col[e] << 32) | (uint64_t)r;
            vals[e] = e;
        }
}

__global__ void k_split_csc(const uint64_t *keys, const uint32_t *vals, int64_t m, const double *w,
                            int32_t *crow, uint32_t *rows, double *cw)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[k];
        crow[k] = (int32_t)(uint32_t)(key & 0xffffffffull);
        rows[k] = (uint32_t)(key >> 32);
        if (cw) cw[k] = w[vals[k]];
    }
}

__global__ void k_rp_to_i64(const uint32_t *rp, int64_t n, int64_t *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = rp[i];
}

static unsigned grid_for(int64_t work, int threads)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

di_status row_bucket_table(const uint32_t *rp, int64_t n, int64_t nnz, uint32_t *tab, cudaStream_t s)
{
    const int64_t nbk = (nnz + (1 << KEY_BUCKET_SHIFT) - 1) >> KEY_BUCKET_SHIFT;
    k_bucket_rows<uint32_t><<<grid_for(n, 256), 256, 0, s>>>(rp, n, nbk, tab);
    count_launches(1);
    DI_CUDA(cudaGetLastError());
    return DI_OK;
}

static di_status build(di_graph_s *g, int64_t n, int64_t nnz, const int64_t *ptr_d,
                       const int32_t *idx_d, const void *w_d, int wdt, int layout, cudaStream_t s)
{
    Temps t(s);
    unsigned *err;
    DI_TRY(t.get(&err, 1));
    DI_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned), s));
    k_validate<<<grid_for(nnz > n ? nnz : n, 256), 256, 0, s>>>(ptr_d, idx_d, w_d, wdt, n, nnz, err);
    count_launches(1);
    DI_CUDA(cudaGetLastError());
    unsigned herr = 0;
    DI_CUDA(cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    if (herr) return DI_ERR_BAD_GRAPH;

    g->n = n;
    g->weighted = wdt != DI_W_NONE;
    uint64_t *keys, *keys2;
    uint32_t *vals, *vals2;
    DI_TRY(t.get(&keys, nnz));
    DI_TRY(t.get(&keys2, nnz));
    DI_TRY(t.get(&vals, nnz));
    DI_TRY(t.get(&vals2, nnz));
    if (nnz > 0) {
        const int64_t nbk = (nnz + (1 << KEY_BUCKET_SHIFT) - 1) >> KEY_BUCKET_SHIFT;
        uint32_t *tab;
        DI_TRY(t.get(&tab, nbk + 1));
        k_bucket_rows<int64_t><<<grid_for(n, 256), 256, 0, s>>>(ptr_d, n, nbk, tab);
        k_make_keys<<<grid_for(nnz, 256), 256, 0, s>>>(ptr_d, idx_d, n, nnz, layout, tab, keys, vals);
        count_launches(2);
        DI_CUDA(cudaGetLastError());
        const int b = bits_for(n);
        int lo[16], cnt[16], np = 0;
        for (int x = 0; x < b; x += 8) { lo[np] = x; cnt[np] = b - x < 8 ? b - x : 8; np++; }
        for (int x = 0; x < b; x += 8) { lo[np] = 32 + x; cnt[np] = b - x < 8 ? b - x : 8; np++; }
        DI_TRY(radix_sort_pairs(&keys, &vals, &keys2, &vals2, nnz, lo, cnt, np, s));
    }
    uint8_t *keep;
    uint64_t *pos, *total;
    DI_TRY(t.get(&keep, nnz));
    DI_TRY(t.get(&pos, nnz));
    DI_TRY(t.get(&total, 1));
    k_mark_runs<<<grid_for(nnz, 256), 256, 0, s>>>(keys, nnz, keep);
    count_launches(1);
    DI_TRY(scan_exclusive<uint8_t>(keep, pos, nnz, total, s));
    uint64_t m = 0;
    DI_CUDA(cudaMemcpyAsync(&m, total, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    g->nnz = (int64_t)m;
    g->off64 = false;

    uint32_t *rows;
    DI_TRY(t.get(&rows, m));
    DI_TRY(dalloc_t(&g->col, m, s));
    if (g->weighted) DI_TRY(dalloc_t(&g->w, m, s));
    DI_TRY(dalloc_t(reinterpret_cast<uint32_t **>(&g->rp), n + 1 + RP_PAD, s));
    DI_CUDA(cudaMemsetAsync(static_cast<uint32_t *>(g->rp) + n + 1, 0, sizeof(uint32_t) * RP_PAD, s));
    k_compact<<<grid_for(nnz, 256), 256, 0, s>>>(keys, vals, keep, pos, nnz, w_d, wdt, g->col, rows,
                                                 g->w);
    count_launches(1);
    uint32_t *rp = static_cast<uint32_t *>(g->rp);
    if (m == 0) {
        k_fill<uint32_t><<<grid_for(n + 1, 256), 256, 0, s>>>(rp, n + 1, 0u);
        count_launches(1);
    } else {
        k_row_ptr<uint32_t><<<grid_for(m, 256), 256, 0, s>>>(rows, (int64_t)m, n, rp);
        count_launches(1);
    }
    unsigned long long *ndang;
    DI_TRY(t.get(&ndang, 1));
    DI_CUDA(cudaMemsetAsync(ndang, 0, sizeof(unsigned long long), s));
    if (g->weighted) DI_TRY(dalloc_t(&g->wsum, n, s));
    k_row_sums<<<grid_for(n, 256), 256, 0, s>>>(rp, g->w, n, g->wsum, ndang);
    count_launches(1);
    DI_CUDA(cudaGetLastError());
    unsigned long long hd = 0;
    DI_CUDA(cudaMemcpyAsync(&hd, ndang, sizeof(hd), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    g->n_dangling = (int64_t)hd;
    return DI_OK;
}

di_status graph_build_csc(di_graph_s *g, cudaStream_t s)
{
    if (g->cp) return DI_OK;
    const int64_t n = g->n, m = g->nnz;
    Temps t(s);
    uint64_t *keys, *keys2;
    uint32_t *vals, *vals2, *rows;
    DI_TRY(t.get(&keys, m));
    DI_TRY(t.get(&keys2, m));
    DI_TRY(t.get(&vals, m));
    DI_TRY(t.get(&vals2, m));
    DI_TRY(t.get(&rows, m));
    int64_t *cp = nullptr;
    int32_t *crow = nullptr;
    double *cw = nullptr;
    DI_TRY(dalloc_t(&cp, n + 1, s));
    DI_TRY(dalloc_t(&crow, m, s));
    if (g->weighted) DI_TRY(dalloc_t(&cw, m, s));
    const uint32_t *rp = static_cast<const uint32_t *>(g->rp);
    if (m > 0) {
        k_expand_rows<<<grid_for(n * 32, 256), 256, 0, s>>>(rp, n, g->col, keys, vals);
        count_launches(1);
        const int b = bits_for(n);
        int lo[8], cnt[8], np = 0;
        for (int x = 0; x < b; x += 8) { lo[np] = 32 + x; cnt[np] = b - x < 8 ? b - x : 8; np++; }
        DI_TRY(radix_sort_pairs(&keys, &vals, &keys2, &vals2, m, lo, cnt, np, s));
        k_split_csc<<<grid_for(m, 256), 256, 0, s>>>(keys, vals, m, g->w, crow, rows, cw);
        count_launches(1);
        k_row_ptr<int64_t><<<grid_for(m, 256), 256, 0, s>>>(rows, m, n, cp);
        count_launches(1);
    } else {
        k_fill<int64_t><<<grid_for(n + 1, 256), 256, 0, s>>>(cp, n + 1, (int64_t)0);
        count_launches(1);
    }
    DI_CUDA(cudaGetLastError());
    DI_CUDA(cudaStreamSynchronize(s));
    g->cp = cp;
    g->crow = crow;
    g->cw = cw;
    return DI_OK;
}

// ---------------------------------------------------------------- hot targets
// In-degree of every page; a bucket of about a quarter octave per in-degree
// (integer only: 4 * floor(log2 x) + the two bits after the leading one).
__device__ __forceinline__ int indeg_bucket(unsigned x)
{
    if (x == 0) return 0;
    const int lg = 31 - __clz(x);
    const unsigned frac = lg >= 2 ? (x >> (lg - 2)) & 3u : (x << (2 - lg)) & 3u;
    return 1 + 4 * lg + (int)frac;
}

__global__ void k_indeg(const int32_t *col, int64_t nnz, unsigned *indeg)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(indeg + col[e], 1u);
}

__global__ void k_indeg_hist(const unsigned *indeg, int64_t n, unsigned long long *hist)
{
    __shared__ unsigned long long h[130];
    for (int b = threadIdx.x; b < 130; b += blockDim.x) h[b] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(h + indeg_bucket(indeg[i]), 1ull);
    __syncthreads();
    for (int b = threadIdx.x; b < 130; b += blockDim.x)
        if (h[b]) atomicAdd(hist + b, h[b]);
}

__global__ void k_hot_assign(const unsigned *indeg, int64_t n, int bmin, unsigned min_indeg, int *slot_of,
                             int32_t *hot_node, unsigned *nhot)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned x = indeg[i];
        int sl = -1;
        if (x >= min_indeg && indeg_bucket(x) >= bmin) {
            sl = (int)atomicAdd(nhot, 1u);
            hot_node[sl] = (int32_t)i;
        }
        slot_of[i] = sl;
    }
}

__global__ void k_pcol(const int32_t *col, int64_t nnz, const int *slot_of, int32_t *pcol)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = col[e];
        const int sl = slot_of[c];
        pcol[e] = sl >= 0 ? (int32_t)(0x80000000u | (unsigned)sl) : c;
    }
}

__global__ void k_w32(const double *w, int64_t nnz, float *w32)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        w32[e] = (float)w[e];
}

// Push copy of the link targets: links into the (at most HOT_K) pages with
// the most in-links are tagged with their slot so that the push can add them
// up in shared memory first (one global add per CTA and page instead of one
// per link: the many adds into one address would otherwise serialise).
di_status graph_build_push_targets(di_graph_s *g, cudaStream_t s)
{
    if (g->pcol && g->pcol_version == g->version) return DI_OK;
    const int64_t n = g->n, m = g->nnz;
    dfree(g->pcol, s);
    g->pcol = nullptr;
    dfree(g->w32, s);
    g->w32 = nullptr;
    if (!g->hot_node) DI_TRY(dalloc_t(&g->hot_node, HOT_K, s));
    DI_TRY(dalloc_t(&g->pcol, m, s));
    if (g->weighted) {   // link weights for the FP32-fluid push
        DI_TRY(dalloc_t(&g->w32, m, s));
        k_w32<<<grid_for(m, 256), 256, 0, s>>>(g->w, m, g->w32);
        count_launches(1);
    }
    Temps t(s);
    unsigned *nhot;
    unsigned long long *hist;
    if (!g->slot_of) DI_TRY(dalloc_t(&g->slot_of, n, s));
    int *slot_of = g->slot_of;
    DI_TRY(t.get(&hist, 130));
    DI_TRY(t.get(&nhot, 1));
    DI_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * 130, s));
    DI_CUDA(cudaMemsetAsync(nhot, 0, sizeof(unsigned), s));
    if (!g->indeg) {   // counted once; link updates keep it current
        DI_TRY(dalloc_t(&g->indeg, n, s));
        DI_CUDA(cudaMemsetAsync(g->indeg, 0, sizeof(unsigned) * n, s));
        k_indeg<<<grid_for(m, 256), 256, 0, s>>>(g->col, m, g->indeg);
        count_launches(1);
    }
    const unsigned *indeg = g->indeg;
    k_indeg_hist<<<grid_for(n, 256) < 1024 ? grid_for(n, 256) : 1024, 256, 0, s>>>(indeg, n, hist);
    count_launches(1);
    unsigned long long hh[130];
    DI_CUDA(cudaMemcpyAsync(hh, hist, sizeof(hh), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    // smallest bucket whose tail fits in HOT_K slots
    int bmin = 130;
    unsigned long long tail = 0;
    for (int b = 129; b >= 1; b--) {
        if (tail + hh[b] > (unsigned long long)HOT_K) break;
        tail += hh[b];
        bmin = b;
    }
    k_hot_assign<<<grid_for(n, 256), 256, 0, s>>>(indeg, n, bmin, HOT_MIN_INDEG, slot_of, g->hot_node, nhot);
    count_launches(1);
    k_pcol<<<grid_for(m, 256), 256, 0, s>>>(g->col, m, slot_of, g->pcol);
    count_launches(1);
    DI_CUDA(cudaGetLastError());
    unsigned nh = 0;
    DI_CUDA(cudaMemcpyAsync(&nh, nhot, sizeof(nh), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    g->nhot = (int)nh;
    g->pcol_version = g->version;
    return DI_OK;
}

di_status graph_export(di_graph_s *g, bool csc, int64_t *ptr, int32_t *idx, double *w, int mem,
                       cudaStream_t s)
{
    const int64_t n = g->n, m = g->nnz;
    if (csc) DI_TRY(graph_build_csc(g, s));
    Temps t(s);
    int64_t *p64 = nullptr;
    if (csc) {
        p64 = g->cp;
    } else {
        DI_TRY(t.get(&p64, n + 1));
        k_rp_to_i64<<<grid_for(n + 1, 256), 256, 0, s>>>(static_cast<const uint32_t *>(g->rp), n, p64);
        count_launches(1);
    }
    const cudaMemcpyKind kind = mem == DI_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (ptr) DI_CUDA(cudaMemcpyAsync(ptr, p64, sizeof(int64_t) * (n + 1), kind, s));
    if (idx && m) DI_CUDA(cudaMemcpyAsync(idx, csc ? g->crow : g->col, sizeof(int32_t) * m, kind, s));
    if (w && m) {
        const double *src = csc ? g->cw : g->w;
        if (src) {
            DI_CUDA(cudaMemcpyAsync(w, src, sizeof(double) * m, kind, s));
        } else {
            double *ones;
            DI_TRY(t.get(&ones, m));
            k_fill<double><<<grid_for(m, 256), 256, 0, s>>>(ones, m, 1.0);
            count_launches(1);
            DI_CUDA(cudaMemcpyAsync(w, ones, sizeof(double) * m, kind, s));
        }
    }
    DI_CUDA(cudaGetLastError());
    DI_CUDA(cudaStreamSynchronize(s));
    return DI_OK;
}

di_status graph_create(int64_t n, int64_t nnz, const int64_t *ptr, const int32_t *idx, const void *w,
                       int wdt, int layout, int mem, cudaStream_t s, di_graph_s *g)
{
    pool_keep(g->device);
    Temps t(s);
    const int64_t *ptr_d = ptr;
    const int32_t *idx_d = idx;
    const void *w_d = w;
    if (mem == DI_MEM_HOST) {
        int64_t *p;
        int32_t *i;
        DI_TRY(t.get(&p, n + 1));
        DI_TRY(t.get(&i, nnz));
        DI_CUDA(cudaMemcpyAsync(p, ptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
        if (nnz) DI_CUDA(cudaMemcpyAsync(i, idx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s));
        ptr_d = p;
        idx_d = i;
        if (wdt != DI_W_NONE) {
            const size_t es = wdt == DI_W_F32 ? 4 : 8;
            uint8_t *wb;
            DI_TRY(t.get(&wb, es * nnz));
            if (nnz) DI_CUDA(cudaMemcpyAsync(wb, w, es * nnz, cudaMemcpyHostToDevice, s));
            w_d = wb;
        }
    }
    return build(g, n, nnz, ptr_d, idx_d, w_d, wdt, layout, s);
}

void graph_release(di_graph_s *g)
{
    reverse_release(g);
    cudaStream_t s = 0;
    dfree(g->rp, s);
    dfree(g->col, s);
    dfree(g->w, s);
    dfree(g->wsum, s);
    dfree(g->cp, s);
    dfree(g->crow, s);
    dfree(g->cw, s);
    dfree(g->pcol, s);
    dfree(g->w32, s);
    dfree(g->hot_node, s);
    dfree(g->slot_of, s);
    dfree(g->indeg, s);
    cudaStreamSynchronize(s);
    g->slot_of = nullptr;
    g->pcol = nullptr;
    g->w32 = nullptr;
    g->hot_node = nullptr;
    g->indeg = nullptr;
    g->rp = nullptr;
    g->col = nullptr;
    g->w = g->wsum = g->cw = nullptr;
    g->cp = nullptr;
    g->crow = nullptr;
}

}  // namespace di
