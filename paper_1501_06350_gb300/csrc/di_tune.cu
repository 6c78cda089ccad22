// Autotuner for the solver's launch shape (not in the paper).
//
// The knobs: the DI-argmax threshold factor c (Section 3.4; c < 1 diffuses more
// nodes per sweep, so fewer sweeps of the fixed selection cost are needed), the
// degree-bin threshold between rows pushed by the warp that owns them and rows
// cut into pieces for many warps, the piece size, and for the FP32 form the
// refinement ratio.  One pass of coordinate search, each candidate timed as a
// from-scratch solve of the graph with a uniform teleport vector (device time,
// best of two runs), starting from the library defaults.  The result is cached
// in a plain text file, one line per tuned problem, keyed by the graph's shape
// (nodes, links, dangling nodes, weighted, rows above 256 links, largest row),
// the damping, the tolerance and the precision.
#include <cuda_runtime.h>
#include <math.h>
#include <new>
#include <stdio.h>
#include <string.h>

#include "di_internal.cuh"

namespace di {

using Off = uint32_t;

__global__ void k_shape(const Off *rp, int64_t n, unsigned long long *hubs, unsigned *maxdeg)
{
    unsigned long long h = 0;
    unsigned m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Off deg = rp[i + 1] - rp[i];
        if (deg > 256) h++;
        m = deg > m ? deg : m;
    }
    // one atomic of each kind per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        h += __shfl_xor_sync(0xffffffffu, h, o);
        const unsigned y = __shfl_xor_sync(0xffffffffu, m, o);
        m = y > m ? y : m;
    }
    if ((threadIdx.x & 31) == 0) {
        if (h) atomicAdd(hubs, h);
        atomicMax(maxdeg, m);
    }
}

static di_status shape_key(di_graph_s *g, double d, double tol, int precision, char *key, size_t cap,
                           cudaStream_t s)
{
    Temps t(s);
    unsigned long long *hubs;
    unsigned *maxdeg;
    DI_TRY(t.get(&hubs, 1));
    DI_TRY(t.get(&maxdeg, 1));
    DI_CUDA(cudaMemsetAsync(hubs, 0, sizeof(unsigned long long), s));
    DI_CUDA(cudaMemsetAsync(maxdeg, 0, sizeof(unsigned), s));
    int64_t blocks = (g->n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_shape<<<(unsigned)blocks, 256, 0, s>>>(static_cast<const Off *>(g->rp), g->n, hubs, maxdeg);
    count_launches(1);
    unsigned long long hh = 0;
    unsigned mm = 0;
    DI_CUDA(cudaMemcpyAsync(&hh, hubs, sizeof(hh), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaMemcpyAsync(&mm, maxdeg, sizeof(mm), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    snprintf(key, cap, "n=%lld nnz=%lld dangling=%lld weighted=%d rows_over_256=%llu max_row=%u d=%.17g tol=%.17g prec=%d",
             (long long)g->n, (long long)g->nnz, (long long)g->n_dangling, g->weighted ? 1 : 0, hh, mm, d, tol,
             precision);
    return DI_OK;
}

// Cache line: "<key> | theta_factor=<c> hub_deg=<h> piece=<p> refine_ratio=<r> best_ms=<t> default_ms=<t>"
static bool cache_lookup(const char *path, const char *key, di_opts *o, double *best_ms, double *default_ms)
{
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    const size_t kl = strlen(key);
    while (fgets(line, sizeof line, f)) {
        if (strncmp(line, key, kl) != 0 || strncmp(line + kl, " | ", 3) != 0) continue;
        double c = 0, r = 0, b = 0, dm = 0;
        int h = 0, p = 0;
        if (sscanf(line + kl + 3, "theta_factor=%lf hub_deg=%d piece=%d refine_ratio=%lf best_ms=%lf default_ms=%lf",
                   &c, &h, &p, &r, &b, &dm) == 6) {
            o->theta_factor = c;
            o->hub_deg = h;
            o->piece = p;
            o->refine_ratio = r;
            *best_ms = b;
            *default_ms = dm;
            found = true;   // the last matching line wins
        }
    }
    fclose(f);
    return found;
}

static void cache_store(const char *path, const char *key, const di_opts *o, double best_ms, double default_ms)
{
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s | theta_factor=%.17g hub_deg=%d piece=%d refine_ratio=%.17g best_ms=%.6f default_ms=%.6f\n", key,
            o->theta_factor, o->hub_deg, o->piece, o->refine_ratio, best_ms, default_ms);
    fclose(f);
}

// Best of two from-scratch solves with options o (device time of the loop).
static di_status time_solve(di_graph_s *g, di_state_s *st, double d, double tol, const di_opts *o, double *ms,
                            cudaStream_t s)
{
    double best = INFINITY;
    for (int rep = 0; rep < 2; rep++) {
        di_info info = {};
        st->d = d;
        di_status rc = solve_loop(g, st, tol, o, &info, s, true, nullptr);
        if (rc == DI_ERR_NOT_CONVERGED) {
            *ms = INFINITY;
            return DI_OK;
        }
        DI_TRY(rc);
        if (info.time_ms < best) best = info.time_ms;
    }
    *ms = best;
    return DI_OK;
}

di_status autotune(di_graph_s *g, double d, double tol, int precision, int budget, const char *cache,
                   di_opts *best, double *best_ms, double *default_ms, int *trials, int *from_cache,
                   cudaStream_t s)
{
    di_opts o;
    di_opts_default(&o);
    o.precision = precision;
    char key[512];
    DI_TRY(shape_key(g, d, tol, precision, key, sizeof key, s));
    *trials = 0;
    *from_cache = 0;
    if (cache && cache_lookup(cache, key, &o, best_ms, default_ms)) {
        *best = o;
        *from_cache = 1;
        return DI_OK;
    }
    di_state_s *st = new (std::nothrow) di_state_s;
    if (!st) return DI_ERR_OOM;
    st->g = g;
    st->device = g->device;
    st->prep_version = g->version;
    di_status rc = state_alloc(st, s);
    double cur = INFINITY;
    if (rc == DI_OK) rc = time_solve(g, st, d, tol, &o, &cur, s);
    *default_ms = cur;
    int used = 1;
    // one pass of coordinate search
    const double thetas[] = {0.7, 0.5, 0.35, 0.25, 0.15};
    const int hubs[] = {64, 128, 512, 1024, 4096};
    const int pieces[] = {256, 512, 2048, 4096};
    const double ratios[] = {1e-3, 1e-4, 1e-6};
    for (int stage = 0; stage < 4 && rc == DI_OK; stage++) {
        const int count = stage == 0 ? 5 : stage == 1 ? 5 : stage == 2 ? 4 : (precision == DI_PREC_F32 ? 3 : 0);
        di_opts stage_best = o;
        for (int k = 0; k < count && rc == DI_OK && used < budget; k++) {
            di_opts c = o;
            if (stage == 0) c.theta_factor = thetas[k];
            if (stage == 1) c.hub_deg = hubs[k];
            if (stage == 2) c.piece = pieces[k];
            if (stage == 3) c.refine_ratio = ratios[k];
            double ms = INFINITY;
            rc = time_solve(g, st, d, tol, &c, &ms, s);
            used++;
            if (rc == DI_OK && ms < cur) {
                cur = ms;
                stage_best = c;
            }
        }
        o = stage_best;
    }
    state_free(st);
    delete st;
    if (rc != DI_OK) return rc;
    *best = o;
    *best_ms = cur;
    *trials = used;
    if (cache) cache_store(cache, key, &o, cur, *default_ms);
    return DI_OK;
}

}  // namespace di
