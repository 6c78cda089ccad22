// The D-Iteration sweep on the GPU (Section 3.1, Eq. defF; Section 3.4).
//
// One sweep diffuses a whole frontier S_t = { i : |F_i| >= theta_t } at once:
//
//   select  (k_select)  one CTA per tile of TILE consecutive nodes: reads F,
//           adds |F_i| to a fixed-order per-tile partial of |F|_1, tests the
//           DI-argmax threshold, *takes* the fluid of the selected nodes
//           (H_i += F_i, F_i = 0) and writes one frontier entry per selected
//           non-dangling node (row start, d F_i / W_i, local link prefix).
//           The last CTA to finish sums the tile partials in a fixed order
//           (|F_t|_1, hence the next threshold and the stop test), and cuts
//           the frontier's links into work items of PUSH_ITEM links.
//   push    (k_push)    persistent CTAs pull work items from a queue and
//           scatter d F_i P[k][i] to every out-neighbour k with FP64 atomic
//           adds; each link is mapped to its entry by a binary search over
//           the tile's link prefix held in shared memory.
//
// Diffusing the set S_t at once keeps Eq. HnFn exact: with G = F restricted
// to S_t, H' = H + G and F' = F - G + d P G, so H' + F' = F_0 + d P H'.  Every
// selected node loses (1 - d) of its fluid (all of it if dangling), which is
// the argument of Theorem 3.
#include <cuda_runtime.h>
#include <new>
#include <string.h>

#include "di_internal.cuh"

namespace di {

using Off = uint32_t;
constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned long long ABS_MASK = 0x7fffffffffffffffull;

__device__ __forceinline__ unsigned long long abs_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & ABS_MASK;
}

// Deterministic block sum: xor-butterfly in each warp, then warp 0 over the
// warp partials.  The result is returned to every thread.
template <int NT>
__device__ __forceinline__ double block_sum_det(double v, double *sm)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double x = lane < NT / 32 ? sm[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
        if (lane == 0) sm[NT / 32] = x;
    }
    __syncthreads();
    double r = sm[NT / 32];
    __syncthreads();
    return r;
}

template <int NT>
__device__ __forceinline__ unsigned long long block_exscan_u64(unsigned long long v,
                                                              unsigned long long *sm,
                                                              unsigned long long *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long ws = lane < NT / 32 ? sm[lane] : 0;
        unsigned long long inc = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane < NT / 32) sm[lane] = inc - ws;
        if (lane == NT / 32 - 1) sm[NT / 32] = inc;
    }
    __syncthreads();
    unsigned long long r = sm[warp] + x - v;
    *total = sm[NT / 32];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ init
// Section 3.1: F_0 = (1 - d) Z, H_0 = 0.
__global__ void k_init(double *F, double *H, const double *Z, int64_t n, double one_minus_d, double zu)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        F[i] = one_minus_d * (Z ? Z[i] : zu);
        H[i] = 0.0;
    }
}

// d / W_j (weighted) or d / out(j): the factor turning taken fluid into the
// per-unit-weight share pushed along column j of P (Eq. def-p).
__global__ void k_dscale(const Off *rp, const double *wsum, int64_t n, double d, double *dscale)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Off deg = rp[i + 1] - rp[i];
        dscale[i] = deg == 0 ? 0.0 : (wsum ? d / wsum[i] : d / (double)deg);
    }
}

__global__ void k_scale(double *out, const double *in, int64_t n, double a)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a * in[i];
}

// Load the SEL_PER_THREAD fluid values of this thread (0 past the end).
__device__ __forceinline__ void load4(const double *F, int64_t i0, int64_t n, double f[4])
{
    if (i0 + 3 < n) {
        const double2 a = *reinterpret_cast<const double2 *>(F + i0);
        const double2 b = *reinterpret_cast<const double2 *>(F + i0 + 2);
        f[0] = a.x; f[1] = a.y; f[2] = b.x; f[3] = b.y;
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++) f[k] = (i0 + k < n) ? F[i0 + k] : 0.0;
    }
}

// --------------------------------------------------------------- reduce
// |v|_1 (and, with H, the dangling history l = sum of H_i over dangling i)
// with the same per-thread order and block tree as the selection, summed
// over tiles in a fixed order by the last CTA.
enum { RED_PLAIN = 0, RED_INIT = 1, RED_FINAL = 2 };

__global__ void __launch_bounds__(SEL_THREADS) k_reduce(const double *v, const double *H, const Off *rp,
                                                       int64_t n, int64_t ntiles, double *part_l1,
                                                       double *part_l, DevCtl *ctl, int mode)
{
    __shared__ double sm[SEL_THREADS / 32 + 1];
    __shared__ int s_last;
    const int64_t tile = blockIdx.x;
    const int64_t i0 = tile * TILE + (int64_t)threadIdx.x * SEL_PER_THREAD;
    double f[4];
    load4(v, i0, n, f);
    double a = fabs(f[0]);
    a += fabs(f[1]);
    a += fabs(f[2]);
    a += fabs(f[3]);
    double l = 0.0;
    if (H) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int64_t i = i0 + k;
            if (i < n && rp[i + 1] == rp[i]) l += H[i];
        }
    }
    a = block_sum_det<SEL_THREADS>(a, sm);
    l = block_sum_det<SEL_THREADS>(l, sm);
    if (threadIdx.x == 0) {
        part_l1[tile] = a;
        part_l[tile] = l;
        __threadfence();
        const unsigned t = atomicAdd(&ctl->ticket2, 1u);
        s_last = (t == (unsigned)(ntiles - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double sa = 0.0, sl = 0.0;
    for (int64_t k = threadIdx.x; k < ntiles; k += SEL_THREADS) {
        sa += __ldcg(part_l1 + k);
        sl += __ldcg(part_l + k);
    }
    sa = block_sum_det<SEL_THREADS>(sa, sm);
    sl = block_sum_det<SEL_THREADS>(sl, sm);
    if (threadIdx.x == 0) {
        ctl->ticket2 = 0;
        if (mode == RED_INIT) {
            ctl->l1 = sa;
            ctl->theta = ctl->theta_factor * sa / (double)n;
            ctl->done = sa <= ctl->stop_l1 ? 1u : 0u;
        } else {
            ctl->final_l1 = sa;
            ctl->final_l = sl;
        }
    }
}

// --------------------------------------------------------------- select
__global__ void __launch_bounds__(SEL_THREADS)
    k_select(const Off *__restrict__ rp, const double *__restrict__ dscale, double *F, double *H,
             int64_t n, int64_t ntiles, Off *ent_row, Off *ent_epos, double *ent_val,
             unsigned *tile_cnt, unsigned long long *tile_edges, unsigned *tile_diff, double *tile_l1,
             unsigned *item_tile, unsigned *item_sub, DevCtl *ctl, int use_cond,
             cudaGraphConditionalHandle cond, int32_t *sel_ids, unsigned long long *stats)
{
    __shared__ double sm[SEL_THREADS / 32 + 1];
    __shared__ unsigned long long smu[SEL_THREADS / 32 + 1];
    __shared__ int s_last;
    volatile DevCtl *vc = ctl;
    if (vc->done) {
        // Nothing left to do: make sure a graph while-loop ends here too.
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
        return;
    }
    const double theta = vc->theta;
    const unsigned long long tb = abs_bits(theta);
    const int64_t tile = blockIdx.x;
    const int64_t i0 = tile * TILE + (int64_t)threadIdx.x * SEL_PER_THREAD;

    double f[4];
    load4(F, i0, n, f);
    double a = fabs(f[0]);
    a += fabs(f[1]);
    a += fabs(f[2]);
    a += fabs(f[3]);
    bool sel[4];
    int nsel = 0;
    unsigned long long mb = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const unsigned long long b = abs_bits(f[k]);
        sel[k] = (i0 + k < n) && b != 0 && b >= tb;
        nsel += sel[k];
        mb = b > mb ? b : mb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(FULL, mb, o);
        mb = y > mb ? y : mb;
    }
    if ((threadIdx.x & 31) == 0 && mb) atomicMax(&ctl->maxbits, mb);
    Off r[5] = {0, 0, 0, 0, 0};
    unsigned my_cnt = 0;
    unsigned long long my_edges = 0;
    if (nsel) {
#pragma unroll
        for (int k = 0; k < 5; k++) r[k] = (i0 + k <= n) ? rp[i0 + k] : 0;
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (sel[k] && r[k + 1] > r[k]) {
                my_cnt++;
                my_edges += r[k + 1] - r[k];
            }
    }
    unsigned long long tot_cnt, tot_edges, tot_diff;
    const unsigned long long pos = block_exscan_u64<SEL_THREADS>(my_cnt, smu, &tot_cnt);
    unsigned long long epos = block_exscan_u64<SEL_THREADS>(my_edges, smu, &tot_edges);
    unsigned long long spos = block_exscan_u64<SEL_THREADS>((unsigned long long)nsel, smu, &tot_diff);
    if (nsel) {
        const int64_t slot0 = tile * TILE + (int64_t)pos;
        int q = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (!sel[k]) continue;
            const int64_t i = i0 + k;
            if (sel_ids) sel_ids[tile * TILE + (int64_t)(spos++)] = (int32_t)i;
            H[i] += f[k];
            F[i] = 0.0;
            const Off deg = r[k + 1] - r[k];
            if (deg) {
                ent_row[slot0 + q] = r[k];
                ent_epos[slot0 + q] = (Off)epos;
                ent_val[slot0 + q] = f[k] * dscale[i];
                epos += deg;
                q++;
            }
        }
    }
    a = block_sum_det<SEL_THREADS>(a, sm);
    if (threadIdx.x == 0) {
        tile_l1[tile] = a;
        tile_cnt[tile] = (unsigned)tot_cnt;
        tile_edges[tile] = tot_edges;
        tile_diff[tile] = (unsigned)tot_diff;
        __threadfence();
        const unsigned t = atomicAdd(&ctl->ticket, 1u);
        s_last = (t == (unsigned)(ntiles - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // ---- epilogue: one CTA, fixed-order totals and the push work items
    double sa = 0.0;
    unsigned long long sd = 0, se = 0, sc = 0;
    for (int64_t k = threadIdx.x; k < ntiles; k += SEL_THREADS) {
        sa += __ldcg(tile_l1 + k);
        sd += __ldcg(tile_diff + k);
        se += __ldcg(tile_edges + k);
        sc += __ldcg(tile_cnt + k);
    }
    sa = block_sum_det<SEL_THREADS>(sa, sm);
    unsigned long long tmp;
    block_exscan_u64<SEL_THREADS>(sd, smu, &sd);
    block_exscan_u64<SEL_THREADS>(se, smu, &se);
    block_exscan_u64<SEL_THREADS>(sc, smu, &sc);
    unsigned long long carry = 0;
    for (int64_t c = 0; c < ntiles; c += SEL_THREADS) {
        const int64_t k = c + threadIdx.x;
        unsigned long long ns = 0;
        if (k < ntiles) ns = (__ldcg(tile_edges + k) + PUSH_ITEM - 1) / PUSH_ITEM;
        const unsigned long long base = carry + block_exscan_u64<SEL_THREADS>(ns, smu, &tmp);
        for (unsigned long long s = 0; s < ns; s++) {
            item_tile[base + s] = (unsigned)k;
            item_sub[base + s] = (unsigned)s;
        }
        carry += tmp;
    }
    if (threadIdx.x == 0) {
        ctl->l1 = sa;
        ctl->nitems = (unsigned)carry;
        ctl->item_next = 0;
        ctl->total_edges = se;
        ctl->total_entries = sc;
        ctl->diffusions += sd;
        ctl->edge_pushes += se;
        const unsigned long long sweep = ctl->sweep + 1;
        ctl->sweep = sweep;
        if (stats && sweep <= (unsigned long long)STAT_CAP) {
            stats[2 * (sweep - 1)] = se;
            stats[2 * (sweep - 1) + 1] = sc;
        }
        unsigned done = 0;
        if (sa <= ctl->stop_l1) done = 1;
        else if (sweep >= ctl->max_sweeps) done = 2;
        double th = ctl->theta_factor * sa / (double)n;
        // A sweep that took nothing left F unchanged; the largest |F_i| passes
        // the DI-argmax test exactly, so never ask for more than that (covers
        // a rounded average above every equal fluid, and factors above 1).
        const double fmax = __longlong_as_double((long long)__ldcg(&ctl->maxbits));
        if (sd == 0 && fmax < th) th = fmax;
        ctl->theta = th;
        ctl->maxbits = 0;
        ctl->ticket = 0;
        __threadfence();
        ctl->done = done;
        if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
    }
}

// ----------------------------------------------------------------- push
template <bool WEIGHTED>
__global__ void __launch_bounds__(PUSH_THREADS)
    k_push(const Off *__restrict__ ent_row, const Off *__restrict__ ent_epos,
           const double *__restrict__ ent_val, const unsigned *__restrict__ tile_cnt,
           const unsigned long long *__restrict__ tile_edges, const unsigned *__restrict__ item_tile,
           const unsigned *__restrict__ item_sub, const int32_t *__restrict__ col,
           const double *__restrict__ w, double *F, DevCtl *ctl)
{
    __shared__ Off s_epos[TILE + 1];
    __shared__ unsigned s_item;
    const unsigned nitems = ((volatile DevCtl *)ctl)->nitems;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ctl->item_next, 1u);
        __syncthreads();
        const unsigned item = s_item;
        if (item >= nitems) break;
        const unsigned t = __ldg(item_tile + item);
        const unsigned sub = __ldg(item_sub + item);
        const unsigned cnt = __ldg(tile_cnt + t);
        const Off et = (Off)__ldg(tile_edges + t);
        const Off a = (Off)sub * PUSH_ITEM;
        const Off b = et - a < (Off)PUSH_ITEM ? et : a + PUSH_ITEM;
        const int64_t slot0 = (int64_t)t * TILE;
        for (unsigned k = threadIdx.x; k < cnt; k += PUSH_THREADS) s_epos[k] = __ldg(ent_epos + slot0 + k);
        if (threadIdx.x == 0) s_epos[cnt] = et;
        __syncthreads();
        for (Off e = a + threadIdx.x; e < b; e += PUSH_THREADS) {
            unsigned lo = 0, hi = cnt;  // s_epos[lo] <= e < s_epos[hi]
            while (hi - lo > 1) {
                const unsigned mid = (lo + hi) >> 1;
                if (s_epos[mid] <= e) lo = mid;
                else hi = mid;
            }
            const Off link = __ldg(ent_row + slot0 + lo) + (e - s_epos[lo]);
            const double v = __ldg(ent_val + slot0 + lo);
            const int32_t c = __ldg(col + link);
            atomicAdd(F + c, WEIGHTED ? v * __ldg(w + link) : v);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- host side
static unsigned grid_for(int64_t work, int threads)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

static int push_grid(int device)
{
    static int cached = 0;
    if (!cached) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push<false>, PUSH_THREADS, 0);
        if (per_sm < 1) per_sm = 1;
        cached = per_sm * sm_count(device);
    }
    return cached;
}

di_status state_alloc(di_state_s *st, cudaStream_t s)
{
    di_graph_s *g = st->g;
    const int64_t n = g->n;
    st->ntiles = (n + TILE - 1) / TILE;
    st->max_items = st->ntiles + g->nnz / PUSH_ITEM + 2;
    const int64_t slots = st->ntiles * TILE;
    DI_TRY(dalloc_t(&st->F, slots, s));
    DI_TRY(dalloc_t(&st->H, slots, s));
    DI_TRY(dalloc_t(&st->dscale, n, s));
    DI_TRY(dalloc_t(reinterpret_cast<Off **>(&st->ent_row), slots, s));
    DI_TRY(dalloc_t(reinterpret_cast<Off **>(&st->ent_epos), slots, s));
    DI_TRY(dalloc_t(&st->ent_val, slots, s));
    DI_TRY(dalloc_t(&st->tile_cnt, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_edges, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_diff, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_l1, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_l, st->ntiles, s));
    DI_TRY(dalloc_t(&st->item_tile, st->max_items, s));
    DI_TRY(dalloc_t(&st->item_sub, st->max_items, s));
    DI_TRY(dalloc_t(&st->ctl, 1, s));
    DI_TRY(dalloc_t(&st->stats, 2 * STAT_CAP, s));
    DI_CUDA(cudaMemsetAsync(st->ctl, 0, sizeof(DevCtl), s));
    DI_CUDA(cudaMemsetAsync(st->F, 0, sizeof(double) * slots, s));
    DI_CUDA(cudaMemsetAsync(st->H, 0, sizeof(double) * slots, s));
    DI_CUDA(cudaMallocHost(reinterpret_cast<void **>(&st->host_ctl), sizeof(DevCtl)));
    memset(st->host_ctl, 0, sizeof(DevCtl));
    DI_CUDA(cudaEventCreate(&st->ev0));
    DI_CUDA(cudaEventCreate(&st->ev1));
    DI_CUDA(cudaEventCreate(&st->evp0));
    DI_CUDA(cudaEventCreate(&st->evp1));
    DI_CUDA(cudaStreamSynchronize(s));
    return DI_OK;
}

di_status state_free(di_state_s *st)
{
    cudaStream_t s = 0;
    if (st->gexec) cudaGraphExecDestroy(st->gexec);
    if (st->gstream) cudaStreamDestroy(st->gstream);
    void *bufs[] = {st->F, st->H, st->dscale, st->ent_row, st->ent_epos, st->ent_val, st->tile_cnt,
                    st->tile_edges, st->tile_diff, st->tile_l1, st->tile_l, st->item_tile,
                    st->item_sub, st->ctl, st->stats};
    for (void *p : bufs) dfree(p, s);
    if (st->host_ctl) cudaFreeHost(st->host_ctl);
    if (st->ev0) cudaEventDestroy(st->ev0);
    if (st->ev1) cudaEventDestroy(st->ev1);
    if (st->evp0) cudaEventDestroy(st->evp0);
    if (st->evp1) cudaEventDestroy(st->evp1);
    for (int i = 0; i < st->npev; i++) cudaEventDestroy(st->pev[i]);
    delete[] st->pev;
    st->pev = nullptr;
    st->npev = 0;
    cudaStreamSynchronize(s);
    return DI_OK;
}

static void launch_select(di_graph_s *g, di_state_s *st, cudaStream_t s, int use_cond,
                          cudaGraphConditionalHandle h, int32_t *sel_ids = nullptr)
{
    k_select<<<(unsigned)st->ntiles, SEL_THREADS, 0, s>>>(
        static_cast<const Off *>(g->rp), st->dscale, st->F, st->H, g->n, st->ntiles,
        static_cast<Off *>(st->ent_row), static_cast<Off *>(st->ent_epos), st->ent_val, st->tile_cnt,
        st->tile_edges, st->tile_diff, st->tile_l1, st->item_tile, st->item_sub, st->ctl, use_cond, h,
        sel_ids, st->stats);
    count_launches(1);
}

static void launch_push(di_graph_s *g, di_state_s *st, cudaStream_t s)
{
    const int grid = push_grid(st->device);
    if (g->weighted)
        k_push<true><<<grid, PUSH_THREADS, 0, s>>>(
            static_cast<const Off *>(st->ent_row), static_cast<const Off *>(st->ent_epos), st->ent_val,
            st->tile_cnt, st->tile_edges, st->item_tile, st->item_sub, g->col, g->w, st->F, st->ctl);
    else
        k_push<false><<<grid, PUSH_THREADS, 0, s>>>(
            static_cast<const Off *>(st->ent_row), static_cast<const Off *>(st->ent_epos), st->ent_val,
            st->tile_cnt, st->tile_edges, st->item_tile, st->item_sub, g->col, nullptr, st->F, st->ctl);
    count_launches(1);
}

static di_status build_graph_exec(di_graph_s *g, di_state_s *st)
{
    if (st->gexec) return DI_OK;
    (void)push_grid(st->device);  // occupancy query outside the capture
    if (!st->gstream) DI_CUDA(cudaStreamCreateWithFlags(&st->gstream, cudaStreamNonBlocking));
    cudaGraph_t graph;
    DI_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return note_cuda(e);
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return note_cuda(e);
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(st->gstream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        launch_select(g, st, st->gstream, 1, h);
        launch_push(g, st, st->gstream);
        cudaGraph_t out = nullptr;
        e = cudaStreamEndCapture(st->gstream, &out);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&st->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        st->gexec = nullptr;
        return note_cuda(e);
    }
    return DI_OK;
}

di_status l1_device(di_graph_s *g, const double *v, double *out_host, cudaStream_t s)
{
    const int64_t ntiles = (g->n + TILE - 1) / TILE;
    Temps t(s);
    double *p1, *p2;
    DevCtl *ctl;
    DI_TRY(t.get(&p1, ntiles));
    DI_TRY(t.get(&p2, ntiles));
    DI_TRY(t.get(&ctl, 1));
    DI_CUDA(cudaMemsetAsync(ctl, 0, sizeof(DevCtl), s));
    k_reduce<<<(unsigned)ntiles, SEL_THREADS, 0, s>>>(v, nullptr, static_cast<const Off *>(g->rp), g->n,
                                                      ntiles, p1, p2, ctl, RED_PLAIN);
    count_launches(1);
    DI_CUDA(cudaGetLastError());
    DI_CUDA(cudaMemcpyAsync(out_host, &ctl->final_l1, sizeof(double), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    return DI_OK;
}

di_status solve_loop(di_graph_s *g, di_state_s *st, double tol, const di_opts *o, di_info *info,
                     cudaStream_t s, bool fresh, const double *Z_dev)
{
    const int64_t n = g->n;
    const double d = st->d;
    if (fresh) {
        k_init<<<grid_for(n, 256), 256, 0, s>>>(st->F, st->H, Z_dev, n, 1.0 - d, 1.0 / (double)n);
        count_launches(1);
    }
    if (st->dscale_d != d) {
        k_dscale<<<grid_for(n, 256), 256, 0, s>>>(static_cast<const Off *>(g->rp), g->wsum, n, d,
                                                  st->dscale);
        count_launches(1);
        st->dscale_d = d;
    }
    DevCtl *hc = st->host_ctl;
    memset(hc, 0, sizeof(DevCtl));
    hc->d = d;
    hc->theta_factor = o->theta_factor;
    hc->stop_l1 = (1.0 - d) * tol;
    hc->max_sweeps = (unsigned long long)o->max_sweeps;
    DI_CUDA(cudaMemcpyAsync(st->ctl, hc, sizeof(DevCtl), cudaMemcpyHostToDevice, s));
    k_reduce<<<(unsigned)st->ntiles, SEL_THREADS, 0, s>>>(st->F, nullptr, static_cast<const Off *>(g->rp),
                                                          n, st->ntiles, st->tile_l1, st->tile_l,
                                                          st->ctl, RED_INIT);
    count_launches(1);
    DI_CUDA(cudaGetLastError());

    double push_ms = 0.0;
    int64_t push_launches = 0, push_edges = 0, push_entries = 0;
    const bool graph_mode = o->use_graph && !o->profile;
    if (graph_mode) DI_TRY(build_graph_exec(g, st));
    if (o->profile && !st->pev) {
        st->pev = new (std::nothrow) cudaEvent_t[2 * STAT_CAP];
        if (!st->pev) return DI_ERR_OOM;
    }
    int npairs = 0;
    DI_CUDA(cudaEventRecord(st->ev0, s));
    if (graph_mode) {
        DI_CUDA(cudaGraphLaunch(st->gexec, s));
    } else {
        for (;;) {
            for (int k = 0; k < o->check_every; k++) {
                launch_select(g, st, s, 0, cudaGraphConditionalHandle{});
                if (o->profile && npairs < STAT_CAP) {
                    while (st->npev < 2 * (npairs + 1)) DI_CUDA(cudaEventCreate(&st->pev[st->npev++]));
                    DI_CUDA(cudaEventRecord(st->pev[2 * npairs], s));
                    launch_push(g, st, s);
                    DI_CUDA(cudaEventRecord(st->pev[2 * npairs + 1], s));
                    npairs++;
                } else {
                    launch_push(g, st, s);
                }
            }
            DI_CUDA(cudaGetLastError());
            DI_CUDA(cudaMemcpyAsync(hc, st->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s));
            DI_CUDA(cudaStreamSynchronize(s));
            if (hc->done) break;
        }
    }
    DI_CUDA(cudaEventRecord(st->ev1, s));
    k_reduce<<<(unsigned)st->ntiles, SEL_THREADS, 0, s>>>(st->F, st->H, static_cast<const Off *>(g->rp),
                                                          n, st->ntiles, st->tile_l1, st->tile_l,
                                                          st->ctl, RED_FINAL);
    count_launches(1);
    DI_CUDA(cudaGetLastError());
    DI_CUDA(cudaMemcpyAsync(hc, st->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    DI_CUDA(cudaEventElapsedTime(&ms, st->ev0, st->ev1));
    if (graph_mode) count_launches(2 * (hc->sweep > 0 ? (int64_t)hc->sweep : 1));
    if (npairs) {
        // push launch i follows selection i; selections past the converged
        // sweep returned at once and their pushes found no work
        static unsigned long long hstats[2 * STAT_CAP];
        const int ran = (int)((int64_t)hc->sweep < npairs ? (int64_t)hc->sweep : npairs);
        DI_CUDA(cudaMemcpy(hstats, st->stats, sizeof(unsigned long long) * 2 * ran, cudaMemcpyDeviceToHost));
        for (int i = 0; i < ran; i++) {
            if (hstats[2 * i] == 0) continue;
            float pm = 0.f;
            DI_CUDA(cudaEventElapsedTime(&pm, st->pev[2 * i], st->pev[2 * i + 1]));
            push_ms += pm;
            push_launches++;
            push_edges += (int64_t)hstats[2 * i];
            push_entries += (int64_t)hstats[2 * i + 1];
        }
    }
    if (info) {
        info->resid_l1 = hc->final_l1;
        info->l_dangling = hc->final_l;
        info->bound = hc->final_l1 / (1.0 - d);
        info->bound_completed = hc->final_l1 / (1.0 - d - d * hc->final_l);
        info->sweeps = (int64_t)hc->sweep;
        info->diffusions = (int64_t)hc->diffusions;
        info->edge_pushes = (int64_t)hc->edge_pushes;
        info->time_ms = ms;
        info->push_ms = push_ms;
        info->push_launches = push_launches;
        info->push_edges = push_edges;
        info->push_entries = push_entries;
    }
    if (hc->done == 2) return DI_ERR_NOT_CONVERGED;
    if (hc->done != 1) return DI_ERR_CUDA;
    return DI_OK;
}

di_status copy_out_H(di_state_s *st, double *H_out, bool normalize, double l, int mem, cudaStream_t s)
{
    const int64_t n = st->g->n;
    const double d = st->d;
    const double *src = st->H;
    Temps t(s);
    if (normalize) {
        double *tmp;
        DI_TRY(t.get(&tmp, n));
        k_scale<<<grid_for(n, 256), 256, 0, s>>>(tmp, st->H, n, (1.0 - d) / (1.0 - d - d * l));
        count_launches(1);
        src = tmp;
    }
    DI_CUDA(cudaMemcpyAsync(H_out, src, sizeof(double) * n,
                            mem == DI_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    DI_CUDA(cudaStreamSynchronize(s));
    return DI_OK;
}

__global__ void k_finite(const double *v, int64_t n, unsigned *bad)
{
    unsigned b = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) b = 1;
    if (b) atomicOr(bad, 1u);
}

di_status check_finite(const double *v, int64_t n, bool *ok, cudaStream_t s)
{
    Temps t(s);
    unsigned *bad;
    DI_TRY(t.get(&bad, 1));
    DI_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned), s));
    k_finite<<<grid_for(n, 256), 256, 0, s>>>(v, n, bad);
    count_launches(1);
    unsigned hb = 0;
    DI_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    *ok = hb == 0;
    return DI_OK;
}

// l = sum of H over dangling nodes for the state's current H.
di_status state_l(di_graph_s *g, di_state_s *st, double *l, cudaStream_t s)
{
    Temps t(s);
    DevCtl *ctl;
    DI_TRY(t.get(&ctl, 1));
    DI_CUDA(cudaMemsetAsync(ctl, 0, sizeof(DevCtl), s));
    k_reduce<<<(unsigned)st->ntiles, SEL_THREADS, 0, s>>>(st->F, st->H, static_cast<const Off *>(g->rp),
                                                          g->n, st->ntiles, st->tile_l1, st->tile_l, ctl,
                                                          RED_FINAL);
    count_launches(1);
    DI_CUDA(cudaGetLastError());
    DI_CUDA(cudaMemcpyAsync(l, &ctl->final_l, sizeof(double), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    return DI_OK;
}

// ------------------------------------------------------- frontier alone
__global__ void k_compact_ids(const int32_t *sel_ids, const unsigned *tile_diff, const uint64_t *base,
                              int32_t *ids)
{
    const int64_t t = blockIdx.x;
    const unsigned c = tile_diff[t];
    for (unsigned k = threadIdx.x; k < c; k += blockDim.x) ids[base[t] + k] = sel_ids[t * TILE + k];
}

// Runs the solver's own selection kernel once on a scratch state holding a
// copy of F (threshold given, stop test disabled) and compacts the ids it
// reports, tile by tile, into ascending order.
di_status select_only(di_graph_s *g, const double *F, double theta, int32_t *ids, int64_t *count,
                      cudaStream_t s)
{
    const int64_t n = g->n;
    di_state_s st;
    st.g = g;
    st.device = g->device;
    di_status rc = state_alloc(&st, s);
    if (rc == DI_OK) {
        Temps t(s);
        int32_t *sel_ids = nullptr;
        uint64_t *base = nullptr, *tot = nullptr;
        rc = t.get(&sel_ids, st.ntiles * TILE);
        if (rc == DI_OK) rc = t.get(&base, st.ntiles);
        if (rc == DI_OK) rc = t.get(&tot, 1);
        if (rc == DI_OK) {
            DevCtl *hc = st.host_ctl;
            memset(hc, 0, sizeof(DevCtl));
            hc->theta = theta;
            hc->stop_l1 = -1.0;
            hc->max_sweeps = ~0ull;
            hc->theta_factor = 1.0;
            cudaMemcpyAsync(st.ctl, hc, sizeof(DevCtl), cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(st.F, F, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
            k_dscale<<<grid_for(n, 256), 256, 0, s>>>(static_cast<const Off *>(g->rp), g->wsum, n, 0.85,
                                                      st.dscale);
            count_launches(1);
            launch_select(g, &st, s, 0, cudaGraphConditionalHandle{}, sel_ids);
            rc = scan_exclusive<uint32_t>(st.tile_diff, base, st.ntiles, tot, s);
            if (rc == DI_OK) {
                k_compact_ids<<<(unsigned)st.ntiles, 256, 0, s>>>(sel_ids, st.tile_diff, base, ids);
                count_launches(1);
                uint64_t c = 0;
                cudaError_t e = cudaGetLastError();
                if (e == cudaSuccess) e = cudaMemcpyAsync(&c, tot, sizeof(c), cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) rc = note_cuda(e);
                *count = (int64_t)c;
            }
        }
    }
    state_free(&st);
    return rc;
}

}  // namespace di
