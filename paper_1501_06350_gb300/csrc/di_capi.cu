// extern "C" entry points of libdi.so (declared in include/di.h): argument
// checks, device selection, host<->device staging, then the device code.
#include <cuda_runtime.h>
#include <math.h>
#include <new>
#include <string.h>

#include "di_internal.cuh"

namespace {

using namespace di;

// Makes the handle's device current for the duration of a call.
struct DeviceScope {
    int prev = -1;
    bool ok = true;
    explicit DeviceScope(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceScope()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

bool mem_ok(int mem) { return mem == DI_MEM_HOST || mem == DI_MEM_DEVICE; }

// Stage n doubles to the device if they live on the host.
di_status stage_in(const double *p, int64_t n, int mem, Temps &t, const double **out, cudaStream_t s)
{
    if (!p || mem == DI_MEM_DEVICE) {
        *out = p;
        return DI_OK;
    }
    double *d;
    DI_TRY(t.get(&d, n));
    DI_CUDA(cudaMemcpyAsync(d, p, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    *out = d;
    return DI_OK;
}

template <typename T>
di_status stage_in_t(const T *p, int64_t n, int mem, Temps &t, const T **out, cudaStream_t s)
{
    if (!p || mem == DI_MEM_DEVICE) {
        *out = p;
        return DI_OK;
    }
    T *d;
    DI_TRY(t.get(&d, n));
    if (n) DI_CUDA(cudaMemcpyAsync(d, p, sizeof(T) * n, cudaMemcpyHostToDevice, s));
    *out = d;
    return DI_OK;
}

di_status opts_ok(const di_opts *o)
{
    if (!(o->theta_factor > 0.0 && o->theta_factor <= 1.0)) return DI_ERR_INVALID_ARG;
    if (o->max_sweeps < 1 || o->check_every < 1) return DI_ERR_INVALID_ARG;
    if (o->precision != DI_PREC_F64 && o->precision != DI_PREC_F32) return DI_ERR_INVALID_ARG;
    if (o->precision == DI_PREC_F32 && !(o->refine_ratio > 0.0 && o->refine_ratio < 1.0))
        return DI_ERR_INVALID_ARG;
    if (o->hub_deg < 32 || o->hub_deg > 65536 || o->piece < 128 || o->piece > 65536) return DI_ERR_INVALID_ARG;
    return DI_OK;
}

// Re-derive what a state keeps about its graph after a structural update.
di_status prepare(di_graph_s *g, di_state_s *st, cudaStream_t s)
{
    if (st->prep_version == g->version) return DI_OK;
    // the captured sweep loops read the moved buffers through the state's
    // pointer block, rewritten by the next solve: they stay valid
    st->dscale_d = -1.0;
    DI_TRY(state_prepare_graph(g, st, s));
    st->prep_version = g->version;
    return DI_OK;
}

di_status finish_solve(di_graph_s *g, di_state_s *st, di_status rc, const di_opts *o, double *H_out,
                       di_info *info_out, di_info &info, int mem, cudaStream_t s)
{
    if (rc != DI_OK && rc != DI_ERR_NOT_CONVERGED) return rc;
    if (H_out) DI_TRY(copy_out_H(st, H_out, o->normalize != 0, info.l_dangling, mem, s));
    if (info_out) *info_out = info;
    (void)g;
    return rc;
}

}  // namespace

extern "C" {

void di_opts_default(di_opts *o)
{
    if (!o) return;
    o->theta_factor = 1.0;
    o->max_sweeps = 100000;
    o->check_every = 8;
    o->use_graph = 1;
    o->normalize = 0;
    o->profile = 0;
    o->precision = DI_PREC_F64;
    o->refine_ratio = 1e-5;
    o->hub_deg = 256;
    o->piece = 1024;
}

const char *di_status_str(di_status s)
{
    switch (s) {
    case DI_OK: return "DI_OK";
    case DI_ERR_INVALID_ARG: return "DI_ERR_INVALID_ARG";
    case DI_ERR_BAD_GRAPH: return "DI_ERR_BAD_GRAPH";
    case DI_ERR_OOM: return "DI_ERR_OOM";
    case DI_ERR_NOT_CONVERGED: return "DI_ERR_NOT_CONVERGED";
    case DI_ERR_CUDA: return "DI_ERR_CUDA";
    case DI_ERR_DEVICE_TIMEOUT: return "DI_ERR_DEVICE_TIMEOUT";
    }
    return "DI_ERR_UNKNOWN";
}

int di_last_cuda_error(void) { return di::last_cuda(); }

int64_t di_kernel_launches(void) { return di::launches(); }

di_status di_graph_create(int64_t n, int64_t nnz, const int64_t *ptr, const int32_t *idx, const void *w,
                          int w_dtype, int layout, int mem, void *stream, di_graph_t *out)
{
    if (!out) return DI_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || n >= (int64_t(1) << 31) || nnz < 0 || nnz >= (int64_t(1) << 32)) return DI_ERR_INVALID_ARG;
    if (!ptr || (nnz > 0 && !idx)) return DI_ERR_INVALID_ARG;
    if (w_dtype != DI_W_NONE && w_dtype != DI_W_F32 && w_dtype != DI_W_F64) return DI_ERR_INVALID_ARG;
    if (w_dtype != DI_W_NONE && nnz > 0 && !w) return DI_ERR_INVALID_ARG;
    if (layout != DI_LAYOUT_CSR && layout != DI_LAYOUT_CSC) return DI_ERR_INVALID_ARG;
    if (!mem_ok(mem)) return DI_ERR_INVALID_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return note_cuda(e);
    di_graph_s *g = new (std::nothrow) di_graph_s;
    if (!g) return DI_ERR_OOM;
    g->device = dev;
    di_status rc = graph_create(n, nnz, ptr, idx, w, w_dtype, layout, mem, as_stream(stream), g);
    if (rc != DI_OK) {
        graph_release(g);
        delete g;
        return rc;
    }
    *out = g;
    return DI_OK;
}

di_status di_graph_destroy(di_graph_t g)
{
    if (!g) return DI_ERR_INVALID_ARG;
    DeviceScope ds(g->device);
    graph_release(g);
    delete g;
    return DI_OK;
}

di_status di_graph_info(di_graph_t g, int64_t *n, int64_t *nnz, int64_t *n_dangling, int *weighted)
{
    if (!g) return DI_ERR_INVALID_ARG;
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (n_dangling) *n_dangling = g->n_dangling;
    if (weighted) *weighted = g->weighted ? 1 : 0;
    return DI_OK;
}

di_status di_graph_export_csr(di_graph_t g, int64_t *ptr, int32_t *idx, double *w, int mem, void *stream)
{
    if (!g || !mem_ok(mem)) return DI_ERR_INVALID_ARG;
    DeviceScope ds(g->device);
    return graph_export(g, false, ptr, idx, w, mem, as_stream(stream));
}

di_status di_graph_export_csc(di_graph_t g, int64_t *ptr, int32_t *idx, double *w, int mem, void *stream)
{
    if (!g || !mem_ok(mem)) return DI_ERR_INVALID_ARG;
    DeviceScope ds(g->device);
    return graph_export(g, true, ptr, idx, w, mem, as_stream(stream));
}

di_status di_state_create(di_graph_t g, di_state_t *out)
{
    if (!g || !out) return DI_ERR_INVALID_ARG;
    *out = nullptr;
    DeviceScope ds(g->device);
    di_state_s *st = new (std::nothrow) di_state_s;
    if (!st) return DI_ERR_OOM;
    st->g = g;
    st->device = g->device;
    st->prep_version = g->version;
    di_status rc = state_alloc(st, 0);
    if (rc != DI_OK) {
        state_free(st);
        delete st;
        return rc;
    }
    *out = st;
    return DI_OK;
}

di_status di_state_destroy(di_state_t s)
{
    if (!s) return DI_ERR_INVALID_ARG;
    DeviceScope ds(s->device);
    state_free(s);
    delete s;
    return DI_OK;
}

di_status di_solve(di_graph_t g, di_state_t st, double d, const double *Z, double tol, const di_opts *opts,
                   double *H_out, di_info *info, int mem, void *stream)
{
    if (!g || !st || st->g != g || !mem_ok(mem)) return DI_ERR_INVALID_ARG;
    if (!(d > 0.0 && d < 1.0) || !(tol > 0.0) || !isfinite(tol)) return DI_ERR_INVALID_ARG;
    di_opts o;
    di_opts_default(&o);
    if (opts) o = *opts;
    DI_TRY(opts_ok(&o));
    DeviceScope ds(g->device);
    cudaStream_t s = as_stream(stream);
    Temps t(s);
    const double *Zd = nullptr;
    DI_TRY(stage_in(Z, g->n, mem, t, &Zd, s));
    if (Zd) {
        bool ok = false;
        DI_TRY(check_finite(Zd, g->n, &ok, s));
        if (!ok) return DI_ERR_INVALID_ARG;
    }
    DI_TRY(prepare(g, st, s));
    st->d = d;
    di_info inf = {};
    di_status rc = solve_loop(g, st, tol, &o, &inf, s, true, Zd);
    if (rc == DI_OK || rc == DI_ERR_NOT_CONVERGED) {
        st->have_problem = true;
        st->problem_version = g->version;
    }
    return finish_solve(g, st, rc, &o, H_out, info, inf, mem, s);
}

di_status di_resume(di_graph_t g, di_state_t st, double tol, const di_opts *opts, double *H_out, di_info *info,
                    int mem, void *stream)
{
    if (!g || !st || st->g != g || !mem_ok(mem)) return DI_ERR_INVALID_ARG;
    if (!(tol > 0.0) || !isfinite(tol)) return DI_ERR_INVALID_ARG;
    if (!st->have_problem || st->problem_version != g->version) return DI_ERR_INVALID_ARG;
    di_opts o;
    di_opts_default(&o);
    if (opts) o = *opts;
    DI_TRY(opts_ok(&o));
    DeviceScope ds(g->device);
    cudaStream_t s = as_stream(stream);
    DI_TRY(prepare(g, st, s));
    di_info inf = {};
    di_status rc = solve_loop(g, st, tol, &o, &inf, s, false, nullptr);
    return finish_solve(g, st, rc, &o, H_out, info, inf, mem, s);
}

di_status di_update_edges(di_graph_t g, di_state_t st, int64_t m, const int32_t *src, const int32_t *dst,
                          const double *w, const int8_t *op, int mem, void *stream)
{
    if (!g || !st || st->g != g || !mem_ok(mem) || m < 0) return DI_ERR_INVALID_ARG;
    if (m > 0 && (!src || !dst || !op)) return DI_ERR_INVALID_ARG;
    if (g->weighted && m > 0 && !w) return DI_ERR_INVALID_ARG;
    if (!st->have_problem || st->problem_version != g->version) return DI_ERR_INVALID_ARG;
    DeviceScope ds(g->device);
    cudaStream_t s = as_stream(stream);
    Temps t(s);
    const int32_t *sd = nullptr, *dd = nullptr;
    const int8_t *od = nullptr;
    const double *wd = nullptr;
    DI_TRY(stage_in_t(src, m, mem, t, &sd, s));
    DI_TRY(stage_in_t(dst, m, mem, t, &dd, s));
    DI_TRY(stage_in_t(op, m, mem, t, &od, s));
    if (g->weighted) DI_TRY(stage_in(w, m, mem, t, &wd, s));
    DI_TRY(prepare(g, st, s));
    di_status rc = update_edges(g, st, m, sd, dd, wd, od, s);
    if (rc != DI_OK) return rc;
    if (m > 0) {
        g->version++;
        st->problem_version = g->version;
    }
    return DI_OK;
}

di_status di_state_export(di_state_t st, double *H, double *F, double *l, int mem, void *stream)
{
    if (!st || !mem_ok(mem)) return DI_ERR_INVALID_ARG;
    DeviceScope ds(st->device);
    cudaStream_t s = as_stream(stream);
    const cudaMemcpyKind k = mem == DI_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const int64_t n = st->g->n;
    if (H) DI_CUDA(cudaMemcpyAsync(H, st->H, sizeof(double) * n, k, s));
    if (F) DI_CUDA(cudaMemcpyAsync(F, st->F, sizeof(double) * n, k, s));
    if (l) DI_TRY(state_l(st->g, st, l, s));
    DI_CUDA(cudaStreamSynchronize(s));
    return DI_OK;
}

di_status di_state_import(di_state_t st, const double *H, const double *F, double d, int mem, void *stream)
{
    if (!st || !H || !F || !mem_ok(mem) || !(d > 0.0 && d < 1.0)) return DI_ERR_INVALID_ARG;
    DeviceScope ds(st->device);
    cudaStream_t s = as_stream(stream);
    const int64_t n = st->g->n;
    Temps t(s);
    const double *Hd = nullptr, *Fd = nullptr;
    DI_TRY(stage_in(H, n, mem, t, &Hd, s));
    DI_TRY(stage_in(F, n, mem, t, &Fd, s));
    bool ok1 = false, ok2 = false;
    DI_TRY(check_finite(Hd, n, &ok1, s));
    DI_TRY(check_finite(Fd, n, &ok2, s));
    if (!ok1 || !ok2) return DI_ERR_INVALID_ARG;
    DI_CUDA(cudaMemcpyAsync(st->H, Hd, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    DI_CUDA(cudaMemcpyAsync(st->F, Fd, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    DI_CUDA(cudaStreamSynchronize(s));
    st->d = d;
    st->have_problem = true;
    st->problem_version = st->g->version;
    return DI_OK;
}

di_status di_autotune(di_graph_t g, double d, double tol, int32_t precision, int32_t budget, const char *cache_path,
                      di_opts *out, double *best_ms, double *default_ms, int32_t *trials, void *stream)
{
    if (!g || !out || budget < 1) return DI_ERR_INVALID_ARG;
    if (!(d > 0.0 && d < 1.0) || !(tol > 0.0) || !isfinite(tol)) return DI_ERR_INVALID_ARG;
    if (precision != DI_PREC_F64 && precision != DI_PREC_F32) return DI_ERR_INVALID_ARG;
    DeviceScope ds(g->device);
    double b = 0.0, dm = 0.0;
    int tr = 0, fc = 0;
    di_status rc = autotune(g, d, tol, precision, budget, cache_path, out, &b, &dm, &tr, &fc, as_stream(stream));
    if (rc != DI_OK) return rc;
    if (best_ms) *best_ms = b;
    if (default_ms) *default_ms = dm;
    if (trials) *trials = fc ? 0 : tr;
    return DI_OK;
}

di_status di_solve_batch(di_graph_t g, int32_t B, double d, const double *Z, double tol, const di_opts *opts,
                         double *H_out, double *resid_out, di_info *info, int mem, void *stream)
{
    if (!g || !mem_ok(mem) || B < 1 || B > 64) return DI_ERR_INVALID_ARG;
    if (!(d > 0.0 && d < 1.0) || !(tol > 0.0) || !isfinite(tol)) return DI_ERR_INVALID_ARG;
    di_opts o;
    di_opts_default(&o);
    if (opts) o = *opts;
    o.precision = DI_PREC_F32;
    DI_TRY(opts_ok(&o));
    DeviceScope ds(g->device);
    cudaStream_t s = as_stream(stream);
    Temps t(s);
    const double *Zd = nullptr;
    DI_TRY(stage_in(Z, g->n * (int64_t)B, mem, t, &Zd, s));
    if (Zd) {
        bool ok = false;
        DI_TRY(check_finite(Zd, g->n * (int64_t)B, &ok, s));
        if (!ok) return DI_ERR_INVALID_ARG;
    }
    return solve_batch(g, B, d, Zd, tol, &o, H_out, resid_out, info, mem, s);
}

di_status di_adjoint(di_graph_t g, double d, const double *gvec, const double *x, double tol, const di_opts *opts,
                     double *lambda_out, double *grad_Z_out, double *grad_w_out, di_info *info, int mem,
                     void *stream)
{
    if (!g || !gvec || !mem_ok(mem)) return DI_ERR_INVALID_ARG;
    if (!(d > 0.0 && d < 1.0) || !(tol > 0.0) || !isfinite(tol)) return DI_ERR_INVALID_ARG;
    if (grad_w_out && !x) return DI_ERR_INVALID_ARG;
    di_opts o;
    di_opts_default(&o);
    if (opts) o = *opts;
    DI_TRY(opts_ok(&o));
    if (o.precision != DI_PREC_F64) return DI_ERR_INVALID_ARG;
    DeviceScope ds(g->device);
    cudaStream_t s = as_stream(stream);
    const int64_t n = g->n;
    Temps t(s);
    const double *gd = nullptr, *xd = nullptr;
    DI_TRY(stage_in(gvec, n, mem, t, &gd, s));
    DI_TRY(stage_in(x, n, mem, t, &xd, s));
    bool ok = false;
    DI_TRY(check_finite(gd, n, &ok, s));
    if (!ok) return DI_ERR_INVALID_ARG;
    if (xd) {
        DI_TRY(check_finite(xd, n, &ok, s));
        if (!ok) return DI_ERR_INVALID_ARG;
    }
    double *lam = lambda_out, *gz = grad_Z_out, *gw = grad_w_out;
    const int64_t m = g->nnz;
    if (mem == DI_MEM_HOST) {
        if (lam) DI_TRY(t.get(&lam, n));
        if (gz) DI_TRY(t.get(&gz, n));
        if (gw) DI_TRY(t.get(&gw, m > 0 ? m : 1));
    }
    di_info inf = {};
    di_status rc = adjoint(g, d, gd, xd, tol, &o, lam, gz, gw, &inf, s);
    if (rc != DI_OK && rc != DI_ERR_NOT_CONVERGED) return rc;
    if (mem == DI_MEM_HOST) {
        if (lam) DI_CUDA(cudaMemcpyAsync(lambda_out, lam, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        if (gz) DI_CUDA(cudaMemcpyAsync(grad_Z_out, gz, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        if (gw && m) DI_CUDA(cudaMemcpyAsync(grad_w_out, gw, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
        DI_CUDA(cudaStreamSynchronize(s));
    }
    if (info) *info = inf;
    return rc;
}

di_status di_frontier_select(di_graph_t g, const double *F, double theta, int32_t *ids, int64_t *count,
                             int mem, void *stream)
{
    if (!g || !F || !ids || !count || !mem_ok(mem) || !(theta >= 0.0) || !isfinite(theta))
        return DI_ERR_INVALID_ARG;
    DeviceScope ds(g->device);
    cudaStream_t s = as_stream(stream);
    Temps t(s);
    const double *Fd = nullptr;
    DI_TRY(stage_in(F, g->n, mem, t, &Fd, s));
    int32_t *idd = ids;
    if (mem == DI_MEM_HOST) DI_TRY(t.get(&idd, g->n));
    DI_TRY(select_only(g, Fd, theta, idd, count, s));
    if (mem == DI_MEM_HOST && *count)
        DI_CUDA(cudaMemcpyAsync(ids, idd, sizeof(int32_t) * (*count), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    return DI_OK;
}

di_status di_residual_l1(di_graph_t g, const double *v, double *out, int mem, void *stream)
{
    if (!g || !v || !out || !mem_ok(mem)) return DI_ERR_INVALID_ARG;
    DeviceScope ds(g->device);
    cudaStream_t s = as_stream(stream);
    Temps t(s);
    const double *vd = nullptr;
    DI_TRY(stage_in(v, g->n, mem, t, &vd, s));
    return l1_device(g, vd, out, s);
}

}  // extern "C"
