// Adjoint of the solve (backward pass; not in the paper).
//
// For a loss L = g . x with x = (1 - d)(I - d P)^-1 Z (Section 2.1), the
// adjoint lambda solves (I - d P)^T lambda = g, i.e. lambda = g + d P^T lambda.
// That is the fluid diffusion of Section 3.1 on the reverse graph: diffusing
// node i moves F_i into H_i and sends d F_i P[i][j] to every j with a link
// j -> i.  The reverse graph is built once per graph version from the in-link
// structure: node i's row lists the sources j of its in-links with weight
// P[i][j] = w(j,i) / W_j, and every node's push factor is d (row sums of W are
// 1 by construction), so the sweep kernels of the forward solve run on it
// unchanged.
//
// P^T is not column-substochastic (its rows are: they are the columns of P),
// so the L1 argument of Theorem 1 does not carry over; the infinity norm does:
// lambda - H = (I - d P^T)^-1 F and |P^T v|_inf <= |v|_inf give
// |lambda - H|_inf <= |F|_inf / (1 - d), which is the stop test here.  The
// frontier threshold is capped at (1 - d)/2 x max |F_i| so that max |F|
// shrinks by at least (1 + d)/2 per sweep.
//
// Gradients: dL/dZ = (1 - d) lambda, and for a link j -> k with
// P[k][j] = w(j,k) / W_j, dL/dw(j,k) = d x_j / W_j (lambda_k - (P^T lambda)_j).
// The diffusion keeps H + F = g + d P^T H exactly (Eq. HnFn on the reverse
// graph), so d (P^T H)_j = H_j + F_j - g_j per node, without a row reduction.
#include <cuda_runtime.h>
#include <new>

#include "di_internal.cuh"

namespace di {

using Off = uint32_t;

static unsigned grid_for(int64_t work, int threads)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

__global__ void k_rp32(const int64_t *cp, int64_t n, Off *rp)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
        rp[i] = (Off)cp[i];
}

// Weight of reverse link i -> j (in-link j -> i of the forward graph): P[i][j].
__global__ void k_rev_weights(const int32_t *crow, const double *cw, const Off *rp, const double *wsum, int64_t nnz,
                              double *pw)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = crow[e];
        pw[e] = cw ? cw[e] / wsum[j] : 1.0 / (double)(rp[j + 1] - rp[j]);
    }
}

__global__ void k_ones(double *a, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = 1.0;
}

__global__ void k_scale_into(double *out, const double *in, int64_t n, double a)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a * in[i];
}

// dL/dw per link of the out-CSR, in its order, one thread per link: the row
// j of link e is the largest j with rp[j] <= e, searched between the rows of
// the bucket starts around e (tab, see row_bucket_table).
__global__ void k_grad_w(const Off *rp, const uint32_t *tab, const int32_t *col, const double *wsum, int64_t n,
                         int64_t nnz, const double *x, const double *lam, const double *F, const double *g, double d,
                         double *grad)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = e >> KEY_BUCKET_SHIFT;
        int64_t lo = __ldg(tab + q), hi = __ldg(tab + q + 1);   // rp[lo] <= e, row(e) <= hi
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (__ldg(rp + mid) <= (Off)e) lo = mid;
            else hi = mid - 1;
        }
        const int64_t j = lo;
        const double W = wsum ? wsum[j] : (double)(__ldg(rp + j + 1) - __ldg(rp + j));
        const double t = lam[j] + F[j] - g[j];   // d (P^T H)_j
        grad[e] = x[j] / W * (d * lam[col[e]] - t);
    }
}

static void release_reverse(di_graph_s *g)
{
    if (g->rev_state) {
        state_free(g->rev_state);
        delete g->rev_state;
        g->rev_state = nullptr;
    }
    if (g->rev) {
        graph_release(g->rev);
        delete g->rev;
        g->rev = nullptr;
    }
    g->rev_version = -1;
}

void reverse_release(di_graph_s *g) { release_reverse(g); }

// The reverse graph and its solver state for the current graph version.
di_status graph_build_reverse(di_graph_s *g, cudaStream_t s)
{
    if (g->rev && g->rev_version == g->version) return DI_OK;
    release_reverse(g);
    DI_TRY(graph_build_csc(g, s));
    const int64_t n = g->n, m = g->nnz;
    di_graph_s *r = new (std::nothrow) di_graph_s;
    if (!r) return DI_ERR_OOM;
    g->rev = r;
    r->device = g->device;
    r->n = n;
    r->nnz = m;
    r->weighted = true;
    Off *rp = nullptr;
    DI_TRY(dalloc_t(&rp, n + 1 + RP_PAD, s));
    DI_CUDA(cudaMemsetAsync(rp + n + 1, 0, sizeof(Off) * RP_PAD, s));
    r->rp = rp;
    DI_TRY(dalloc_t(&r->col, m, s));
    DI_TRY(dalloc_t(&r->w, m, s));
    DI_TRY(dalloc_t(&r->wsum, n, s));
    k_rp32<<<grid_for(n + 1, 256), 256, 0, s>>>(g->cp, n, rp);
    if (m) DI_CUDA(cudaMemcpyAsync(r->col, g->crow, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s));
    k_rev_weights<<<grid_for(m, 256), 256, 0, s>>>(g->crow, g->weighted ? g->cw : nullptr,
                                                   static_cast<const Off *>(g->rp), g->wsum, m, r->w);
    k_ones<<<grid_for(n, 256), 256, 0, s>>>(r->wsum, n);
    count_launches(3);
    DI_CUDA(cudaGetLastError());
    di_state_s *st = new (std::nothrow) di_state_s;
    if (!st) return DI_ERR_OOM;
    g->rev_state = st;
    st->g = r;
    st->device = r->device;
    st->prep_version = r->version;
    DI_TRY(state_alloc(st, s));
    g->rev_version = g->version;
    return DI_OK;
}

di_status adjoint(di_graph_s *g, double d, const double *gvec, const double *x, double tol, const di_opts *o,
                  double *lambda, double *grad_Z, double *grad_w, di_info *info, cudaStream_t s)
{
    DI_TRY(graph_build_reverse(g, s));
    di_graph_s *r = g->rev;
    di_state_s *st = g->rev_state;
    const int64_t n = g->n;
    st->d = d;
    // F_0 = g, H_0 = 0 (the padding past n stays 0 from allocation)
    DI_CUDA(cudaMemcpyAsync(st->F, gvec, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    DI_CUDA(cudaMemsetAsync(st->H, 0, sizeof(double) * n, s));
    di_info inf = {};
    di_status rc = solve_loop(r, st, tol, o, &inf, s, false, nullptr, true);
    if (rc != DI_OK && rc != DI_ERR_NOT_CONVERGED) return rc;
    if (lambda) DI_CUDA(cudaMemcpyAsync(lambda, st->H, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (grad_Z) {
        k_scale_into<<<grid_for(n, 256), 256, 0, s>>>(grad_Z, st->H, n, 1.0 - d);
        count_launches(1);
    }
    if (grad_w && g->nnz) {
        const int64_t nbk = (g->nnz + (1 << KEY_BUCKET_SHIFT) - 1) >> KEY_BUCKET_SHIFT;
        uint32_t *tab = nullptr;
        DI_TRY(dalloc_t(&tab, nbk + 1, s));
        di_status rt = row_bucket_table(static_cast<const Off *>(g->rp), n, g->nnz, tab, s);
        if (rt == DI_OK) {
            k_grad_w<<<grid_for(g->nnz, 256), 256, 0, s>>>(static_cast<const Off *>(g->rp), tab, g->col,
                                                           g->weighted ? g->wsum : nullptr, n, g->nnz, x, st->H,
                                                           st->F, gvec, d, grad_w);
            count_launches(1);
        }
        dfree(tab, s);
        DI_TRY(rt);
    }
    DI_CUDA(cudaGetLastError());
    DI_CUDA(cudaStreamSynchronize(s));
    if (info) *info = inf;
    return rc;
}

}  // namespace di
