// Batched personalised solves: up to 64 teleport vectors Z_c on one graph
// (topic-sensitive PageRank, Section 2.1 remark on Z), solved together.
//
// The fluid of all columns of a node is stored contiguously (node-major,
// BW = 64 columns, FP32): diffusing node i for every column at once costs one
// read of its out-links for 64 problems, and the push of one link adds 64
// contiguous FP32 values (256 B, one half-warp of 16-byte vector reductions)
// into its target's row.  Each column keeps its own DI-argmax threshold
// theta_c = c |F_c|_1 / n (Section 3.4) and its own stop test
// |F_c|_1 / (1 - d) <= tol (Theorem 1, Eq. SL); a node is taken when one of its
// active columns passes, and then all its columns are diffused (any amount is
// a valid diffusion of Eq. defF).
//
// Precision: the sweeps move FP32 fluid and add the taken fluid to an FP32
// accumulator D; a cycle ends per column at refine_ratio x its starting
// |F_c|_1, then H += D in FP64 and the FP64 fluid R becomes R + d P D - D
// (Eq. HnFn, computed in FP64 by a pull over the in-links of every node:
// deterministic, no atomics except for rows split across warps).  By
// linearity that is the exact residual (1-d) Z + d P H - H of the new H
// whatever the rounding of D, so the stop test, applied to the FP64 |R_c|_1,
// is certified in FP64; D's rounding only leaves the next cycle a slightly
// larger residual (about 6e-8 of the fluid taken, like the FP32 fluid itself).
//
// One sweep: k_bsel (per-column partials of the fluid, frontier mask, and the
// take of the selected rows: F_i -> V_i = (d/W_i) F_i, D_i += F_i, F_i = 0) ->
// k_btot (per-column totals, thresholds, stop tests) -> k_bpush (scatter the V
// rows along the links; rows longer than BHUB are cut into static pieces).  A
// sweep whose totals end the cycle does not push what its selection took; that
// fluid is in D, and the refinement's d P D pushes it exactly.  The sweep loop
// is one CUDA graph with a device-side while condition, launched per cycle.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "di_internal.cuh"

namespace di {

using Off = uint32_t;
constexpr int BW = 64;            // columns per node (fixed; fewer are zero-padded)
constexpr int BT = 256;           // threads per CTA
constexpr int BWARP_NODES = 128; // nodes per selection warp
constexpr int BTILE = 1024;       // nodes per selection tile (8 warps x 128 nodes)
constexpr Off BHUB = 256;         // longer rows are pushed as static pieces
constexpr Off BPIECE = 256;       // links per piece
constexpr Off PULL_CH = 512;      // in-links per refinement chunk
constexpr unsigned FULLM = 0xffffffffu;
constexpr int BMAX_CYCLES = 64;
constexpr int UNR = 4;            // link pairs in flight per push iteration

struct BCtl {
    float theta[BW];              // per-column threshold (FP32, rounded up); +inf when inactive
    float l1f[BW];                // per-column |F_c|_1 bound of the last selection
    double l1[BW];                // exact |R_c|_1 after the last refinement
    double sweep_stop[BW];        // per-column end of the current cycle
    double stop;                  // (1 - d) tol
    double theta_factor;
    double refine_ratio;
    unsigned long long act;       // columns still iterating in this cycle
    unsigned long long pending;   // columns whose refined |R_c|_1 is still above stop
    unsigned long long live;      // the caller's columns (bit c set for c < B)
    unsigned long long sweep, max_sweeps, edge_pushes, diffusions, sweep_links;
    unsigned col_on[BW];          // per-column decision of the last totals
    unsigned done;                // 0 running, 1 cycle over, 2 sweep cap
    unsigned push_ready;
    unsigned ticket;
    unsigned pad;
};

static unsigned grid_for(int64_t work, int threads)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

__device__ __forceinline__ void red_v4(float *a, float4 v)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(a), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

// ------------------------------------------------------------ setup kernels
// Static hub bits (one per node, 32-node words) and the pieces of hub rows.
__global__ void k_bhubbits(const Off *rp, int64_t n, int64_t words, unsigned *hubbits)
{
    for (int64_t wi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; wi < words;
         wi += (int64_t)gridDim.x * blockDim.x) {
        unsigned word = 0;
        for (int b = 0; b < 32; b++) {
            const int64_t i = wi * 32 + b;
            if (i < n && rp[i + 1] - rp[i] > BHUB) word |= 1u << b;
        }
        hubbits[wi] = word;
    }
}

// Chunk counts per row: hub pieces of the out-rows (0 for short rows), or
// refinement chunks of the in-rows (at least 1 per row).
__global__ void k_bchunks(const Off *rp, int64_t n, Off limit, Off len, int at_least_one, uint32_t *cnt)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Off deg = rp[i + 1] - rp[i];
        uint32_t c = deg > limit ? (deg + len - 1) / len : 0u;
        if (at_least_one && c == 0) c = 1;
        cnt[i] = c;
    }
}

__global__ void k_bchunk_fill(const Off *rp, int64_t n, Off len, const uint32_t *cnt, const uint64_t *pos,
                              uint32_t *c_row, uint32_t *c_start, uint32_t *c_len)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Off a = rp[i], b = rp[i + 1];
        const uint64_t p = pos[i];
        for (uint32_t c = 0; c < cnt[i]; c++) {
            const Off s = a + c * len;
            c_row[p + c] = (uint32_t)i;
            c_start[p + c] = s;
            c_len[p + c] = (b - s < len) ? b - s : len;
        }
    }
}

__global__ void k_bdscale(const Off *rp, const double *wsum, int64_t n, double d, float *dscale)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Off deg = rp[i + 1] - rp[i];
        dscale[i] = deg == 0 ? 0.0f : (float)(wsum ? d / wsum[i] : d / (double)deg);
    }
}

// R = (1 - d) Z (zero-padded to BW columns), H = D = 0.
__global__ void k_binit(const double *Z, int B, int64_t n, int64_t slots, double one_minus_d, double zu, double *R,
                        double *H, float *D)
{
    const int64_t total = slots * BW;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / BW;
        const int c = (int)(k % BW);
        double z = 0.0;
        if (i < n && c < B) z = Z ? Z[i * B + c] : zu;
        R[k] = one_minus_d * z;
        H[k] = 0.0;
        D[k] = 0.0f;
    }
}

// ------------------------------------------------------------------ sweep
// Half-warp h of a warp handles node base + 2 it + h; lane q = lane & 15 owns
// columns 4q .. 4q + 3.  A warp covers BWARP_NODES nodes (4 mask words).
__global__ void __launch_bounds__(BT) k_bsel(float *F, int64_t n, float *__restrict__ D, float *__restrict__ V,
                                            const float *__restrict__ dscale, unsigned *mask, float *tl1,
                                            unsigned *tmax, unsigned *tcnt, BCtl *ctl, int use_cond,
                                            cudaGraphConditionalHandle cond)
{
    constexpr int NWORD = BWARP_NODES / 32;
    __shared__ float s_l1[BT / 32][BW];
    __shared__ unsigned s_mx[BT / 32][BW];
    __shared__ unsigned s_cnt[BT / 32];
    volatile BCtl *vc = ctl;
    if (vc->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            vc->push_ready = 0;
            if (use_cond) cudaGraphSetConditional(cond, 0u);
        }
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, half = lane >> 4, q = lane & 15;
    const int64_t base = ((int64_t)blockIdx.x * (BT / 32) + warp) * BWARP_NODES;
    float th[4];
#pragma unroll
    for (int k = 0; k < 4; k++) th[k] = vc->theta[4 * q + k];
    float a[4] = {0.f, 0.f, 0.f, 0.f};
    unsigned m[4] = {0u, 0u, 0u, 0u};
    unsigned words[NWORD];
    unsigned cnt = 0;
#pragma unroll
    for (int wd = 0; wd < NWORD; wd++) {
        unsigned word = 0;
#pragma unroll
        for (int it = 0; it < 16; it++) {
            const int64_t i = base + 32 * wd + 2 * it + half;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < n) v = __ldcg(reinterpret_cast<const float4 *>(F + i * BW + 4 * q));
            const float x[4] = {fabsf(v.x), fabsf(v.y), fabsf(v.z), fabsf(v.w)};
            bool s = false;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                a[k] = __fadd_ru(a[k], x[k]);
                const unsigned xb = __float_as_uint(x[k]);
                m[k] = xb > m[k] ? xb : m[k];
                s |= (x[k] != 0.0f) && (x[k] >= th[k]);
            }
            const unsigned b = __ballot_sync(FULLM, s);
            word |= (unsigned)((b & 0xffffu) != 0u) << (2 * it);
            word |= (unsigned)((b >> 16) != 0u) << (2 * it + 1);
            // take the selected node now (its row is in registers): the partials
            // above are those of the fluid before the take
            if ((half ? (b >> 16) : (b & 0xffffu)) != 0u) {
                *reinterpret_cast<float4 *>(F + i * BW + 4 * q) = make_float4(0.f, 0.f, 0.f, 0.f);
                float4 *dp = reinterpret_cast<float4 *>(D + i * BW + 4 * q);
                float4 dd = *dp;
                dd.x += v.x;
                dd.y += v.y;
                dd.z += v.z;
                dd.w += v.w;
                *dp = dd;
                const float sc = __ldg(dscale + i);
                *reinterpret_cast<float4 *>(V + i * BW + 4 * q) = make_float4(v.x * sc, v.y * sc, v.z * sc, v.w * sc);
            }
        }
        words[wd] = word;
        cnt += __popc(word);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
        a[k] = __fadd_ru(a[k], __shfl_xor_sync(FULLM, a[k], 16));
        const unsigned y = __shfl_xor_sync(FULLM, m[k], 16);
        m[k] = y > m[k] ? y : m[k];
    }
    if (lane < 16) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            s_l1[warp][4 * q + k] = a[k];
            s_mx[warp][4 * q + k] = m[k];
        }
    }
    if (lane < NWORD) {
        unsigned wv = words[0];
#pragma unroll
        for (int wd = 1; wd < NWORD; wd++)
            if (lane == wd) wv = words[wd];
        mask[base / 32 + lane] = wv;
    }
    if (lane == 0) s_cnt[warp] = cnt;
    __syncthreads();
    if (threadIdx.x < BW) {
        const int c = threadIdx.x;
        float t = s_l1[0][c];
        unsigned mx = s_mx[0][c];
#pragma unroll
        for (int w = 1; w < BT / 32; w++) {
            t = __fadd_ru(t, s_l1[w][c]);
            mx = s_mx[w][c] > mx ? s_mx[w][c] : mx;
        }
        tl1[(int64_t)blockIdx.x * BW + c] = t;
        tmax[(int64_t)blockIdx.x * BW + c] = mx;
    }
    if (threadIdx.x == 0) {
        unsigned cc = 0;
#pragma unroll
        for (int w = 0; w < BT / 32; w++) cc += s_cnt[w];
        tcnt[blockIdx.x] = cc;
    }
}

// Per-column totals in a fixed order (every partial rounded up: an upper
// bound of |F_c|_1): CTA c sums column c, decides whether the column has
// reached the end of its cycle and sets its next threshold; the last CTA to
// finish assembles the active set and the loop decision.
__global__ void __launch_bounds__(BT) k_btot(const float *tl1, const unsigned *tmax, const unsigned *tcnt,
                                            int64_t ntiles, int64_t n, BCtl *ctl, int use_cond,
                                            cudaGraphConditionalHandle cond)
{
    __shared__ float s_l1[BT / 32];
    __shared__ unsigned s_mx[BT / 32];
    __shared__ unsigned long long s_c[BT / 32];
    __shared__ int s_last;
    volatile BCtl *vc = ctl;
    if (vc->done) return;
    const int c = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float t = 0.0f;
    unsigned mx = 0;
    for (int64_t k = threadIdx.x; k < ntiles; k += BT) {
        t = __fadd_ru(t, tl1[k * BW + c]);
        const unsigned y = tmax[k * BW + c];
        mx = y > mx ? y : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t = __fadd_ru(t, __shfl_xor_sync(FULLM, t, o));
        const unsigned y = __shfl_xor_sync(FULLM, mx, o);
        mx = y > mx ? y : mx;
    }
    if (lane == 0) {
        s_l1[warp] = t;
        s_mx[warp] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float tt = s_l1[0];
        unsigned m2 = s_mx[0];
        for (int w = 1; w < BT / 32; w++) {
            tt = __fadd_ru(tt, s_l1[w]);
            m2 = s_mx[w] > m2 ? s_mx[w] : m2;
        }
        const bool was_on = (vc->act >> c) & 1ull;
        const bool on = was_on && !((double)tt <= vc->sweep_stop[c]);
        float th = __double2float_ru(vc->theta_factor * (double)tt / (double)n);
        const float mxf = __uint_as_float(m2);
        if (th > mxf) th = mxf;   // the largest fluid passes the exact test
        vc->theta[c] = on ? th : __int_as_float(0x7f800000);
        vc->l1f[c] = tt;
        vc->col_on[c] = on ? 1u : 0u;
        __threadfence();
        s_last = atomicAdd((unsigned *)&ctl->ticket, 1u) == BW - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    unsigned long long cnt = 0;
    for (int64_t k = threadIdx.x; k < ntiles; k += BT) cnt += tcnt[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULLM, cnt, o);
    if (lane == 0) s_c[warp] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long act = 0;
        for (int k = 0; k < BW; k++)
            if (vc->col_on[k]) act |= 1ull << k;
        const unsigned long long sweep = vc->sweep;
        vc->edge_pushes = vc->edge_pushes + vc->sweep_links;
        vc->sweep_links = 0;
        const unsigned done = act == 0 ? 1u : (sweep >= vc->max_sweeps ? 2u : 0u);
        vc->act = act;
        if (!done) {
            unsigned long long nsel = 0;
            for (int w = 0; w < BT / 32; w++) nsel += s_c[w];
            vc->diffusions = vc->diffusions + nsel;
        }
        vc->ticket = 0;
        vc->push_ready = done ? 0u : 1u;
        __threadfence();
        vc->done = done;
        if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
    }
}

// Scatter: unit u < words is a mask word (its non-hub selected nodes, links
// enumerated two at a time, one per half-warp); unit u >= words is hub piece
// u - words (pushed if its row is selected).
__global__ void __launch_bounds__(BT) k_bpush(float *F, const float *V, const Off *__restrict__ rp,
                                             const int32_t *__restrict__ col, const float *__restrict__ w32,
                                             const unsigned *__restrict__ mask, const unsigned *__restrict__ hubbits,
                                             int64_t words, const uint32_t *__restrict__ pc_row,
                                             const uint32_t *__restrict__ pc_start, const uint32_t *__restrict__ pc_len,
                                             int64_t npieces, BCtl *ctl)
{
    __shared__ unsigned long long s_links[BT / 32];
    volatile BCtl *vc = ctl;
    if (!vc->push_ready) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) vc->sweep = vc->sweep + 1;
    const int lane = threadIdx.x & 31, half = lane >> 4, q = lane & 15;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long links = 0;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < words + npieces; u += nw) {
        if (u < words) {
            const unsigned sel = mask[u] & ~hubbits[u];
            if (!sel) continue;
            const int64_t i = u * 32 + lane;
            Off r0 = 0, deg = 0;
            if ((sel >> lane) & 1u) {
                r0 = rp[i];
                deg = rp[i + 1] - r0;
            }
            Off incl = deg;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const Off y = __shfl_up_sync(FULLM, incl, o);
                if (lane >= o) incl += y;
            }
            const Off total = __shfl_sync(FULLM, incl, 31);
            const Off excl = incl - deg;
            links += total;
            // 4 link pairs in flight per iteration: all loads first, then the adds
            for (Off e = 0; e < total; e += 2 * UNR) {
                Off link[UNR];
                int64_t src[UNR];
#pragma unroll
                for (int k = 0; k < UNR; k++) {
                    const Off ee0 = e + 2 * k + half;
                    const Off ee = ee0 < total ? ee0 : total - 1;
                    int j = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const Off ex = __shfl_sync(FULLM, excl, j + step);
                        if (ex <= ee) j += step;
                    }
                    link[k] = __shfl_sync(FULLM, r0, j) + (ee - __shfl_sync(FULLM, excl, j));
                    src[k] = u * 32 + j;
                }
                int32_t c[UNR];
                float4 v[UNR];
#pragma unroll
                for (int k = 0; k < UNR; k++) {
                    c[k] = __ldg(col + link[k]);
                    v[k] = __ldg(reinterpret_cast<const float4 *>(V + src[k] * BW + 4 * q));
                    if (w32) {
                        const float wl = __ldg(w32 + link[k]);
                        v[k].x *= wl;
                        v[k].y *= wl;
                        v[k].z *= wl;
                        v[k].w *= wl;
                    }
                }
#pragma unroll
                for (int k = 0; k < UNR; k++)
                    if (e + 2 * k + half < total) red_v4(F + (int64_t)c[k] * BW + 4 * q, v[k]);
            }
        } else {
            const int64_t p = u - words;
            const uint32_t row = pc_row[p];
            if (!((mask[row >> 5] >> (row & 31)) & 1u)) continue;
            const Off s0 = pc_start[p], len = pc_len[p];
            links += len;
            const float4 v0 = __ldg(reinterpret_cast<const float4 *>(V + (int64_t)row * BW + 4 * q));
            for (Off e = half; e < len; e += 2 * UNR) {
                int32_t c[UNR];
                float4 v[UNR];
#pragma unroll
                for (int k = 0; k < UNR; k++) {
                    const Off link = s0 + (e + 2 * k < len ? e + 2 * k : len - 1);
                    c[k] = __ldg(col + link);
                    v[k] = v0;
                    if (w32) {
                        const float wl = __ldg(w32 + link);
                        v[k].x *= wl;
                        v[k].y *= wl;
                        v[k].z *= wl;
                        v[k].w *= wl;
                    }
                }
#pragma unroll
                for (int k = 0; k < UNR; k++)
                    if (e + 2 * k < len) red_v4(F + (int64_t)c[k] * BW + 4 * q, v[k]);
            }
        }
    }
    if (lane == 0) s_links[threadIdx.x >> 5] = links;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < BT / 32; k++) t += s_links[k];
        if (t) atomicAdd((unsigned long long *)&ctl->sweep_links, t);
    }
}

// ------------------------------------------------------------- refinement
// R_i += d sum_{j -> i} P[i][j] D_j - D_i and H_i += D_i, by chunks of the
// in-rows (the reverse graph: rrp/rcol/rw with rw = P[i][j]).  A warp per
// chunk, lane l owns columns 2l, 2l + 1.  A row cut into several chunks adds
// its partial sums atomically; its first chunk also applies -D_i and H_i.
__global__ void __launch_bounds__(BT) k_bpull(const Off *rrp, const int32_t *rcol, const double *rw,
                                             const uint32_t *c_row, const uint32_t *c_start, const uint32_t *c_len,
                                             int64_t nch, double d, const double *D, double *R, double *H)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nch; t += nw) {
        const uint32_t i = c_row[t];
        const Off s0 = c_start[t], len = c_len[t];
        const bool whole = s0 == rrp[i] && s0 + len == rrp[i + 1];
        const bool first = s0 == rrp[i];
        double ax = 0.0, ay = 0.0;
        for (Off e = s0; e < s0 + len; e++) {
            const int32_t j = __ldg(rcol + e);
            const double p = __ldg(rw + e);
            const double2 dj = __ldcg(reinterpret_cast<const double2 *>(D + (int64_t)j * BW) + lane);
            ax += p * dj.x;
            ay += p * dj.y;
        }
        double2 *rp2 = reinterpret_cast<double2 *>(R + (int64_t)i * BW) + lane;
        double2 *hp2 = reinterpret_cast<double2 *>(H + (int64_t)i * BW) + lane;
        const double2 di = __ldcg(reinterpret_cast<const double2 *>(D + (int64_t)i * BW) + lane);
        if (whole) {
            double2 r = *rp2;
            r.x += d * ax - di.x;
            r.y += d * ay - di.y;
            *rp2 = r;
        } else {
            atomicAdd(&rp2->x, first ? d * ax - di.x : d * ax);
            atomicAdd(&rp2->y, first ? d * ay - di.y : d * ay);
        }
        if (first) {
            double2 h = *hp2;
            h.x += di.x;
            h.y += di.y;
            *hp2 = h;
        }
    }
}

// D64 = D: the FP64 copy the pull reads (one conversion per value instead of
// one per link and value; FP64 work is scarce on this part).
__global__ void k_bwiden(const float *D, int64_t total, double *D64)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total / 4;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = reinterpret_cast<const float4 *>(D)[k];
        reinterpret_cast<double2 *>(D64)[2 * k] = make_double2((double)v.x, (double)v.y);
        reinterpret_cast<double2 *>(D64)[2 * k + 1] = make_double2((double)v.z, (double)v.w);
    }
}

// F = fl(R) (FP32), D = 0, per-column exact |R_c|_1 partials (FP64, fixed
// order) and max |F_c| per tile of BTILE nodes.
__global__ void __launch_bounds__(BT) k_bconv(const double *R, float *F, float *D, int64_t slots, double *tl1d,
                                             unsigned *tmax)
{
    __shared__ double s_a[BT / 32][BW];
    __shared__ unsigned s_m[BT / 32][BW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = ((int64_t)blockIdx.x * (BT / 32) + warp) * BWARP_NODES;
    double a0 = 0.0, a1 = 0.0;
    unsigned m0 = 0, m1 = 0;
    for (int it = 0; it < BWARP_NODES; it++) {
        const int64_t i = base + it;
        if (i >= slots) break;
        const double2 r = reinterpret_cast<const double2 *>(R + i * BW)[lane];
        const float2 f = make_float2((float)r.x, (float)r.y);
        reinterpret_cast<float2 *>(F + i * BW)[lane] = f;
        reinterpret_cast<float2 *>(D + i * BW)[lane] = make_float2(0.0f, 0.0f);
        a0 += fabs(r.x);
        a1 += fabs(r.y);
        const unsigned b0 = __float_as_uint(fabsf(f.x)), b1 = __float_as_uint(fabsf(f.y));
        m0 = b0 > m0 ? b0 : m0;
        m1 = b1 > m1 ? b1 : m1;
    }
    s_a[warp][2 * lane] = a0;
    s_a[warp][2 * lane + 1] = a1;
    s_m[warp][2 * lane] = m0;
    s_m[warp][2 * lane + 1] = m1;
    __syncthreads();
    if (threadIdx.x < BW) {
        const int c = threadIdx.x;
        double t = s_a[0][c];
        unsigned mx = s_m[0][c];
        for (int w = 1; w < BT / 32; w++) {
            t += s_a[w][c];
            mx = s_m[w][c] > mx ? s_m[w][c] : mx;
        }
        tl1d[(int64_t)blockIdx.x * BW + c] = t;
        tmax[(int64_t)blockIdx.x * BW + c] = mx;
    }
}

// Per-column exact totals after a refinement: stop test, next cycle targets,
// first thresholds of the cycle.
__global__ void __launch_bounds__(1024) k_bcycle(const double *tl1d, const unsigned *tmax, int64_t ntiles, int64_t n,
                                                BCtl *ctl)
{
    __shared__ double s_a[16][BW];
    __shared__ unsigned s_m[16][BW];
    const int c = threadIdx.x & (BW - 1), g = threadIdx.x >> 6;
    double t = 0.0;
    unsigned mx = 0;
    for (int64_t k = g; k < ntiles; k += 16) {
        t += tl1d[k * BW + c];
        const unsigned y = tmax[k * BW + c];
        mx = y > mx ? y : mx;
    }
    s_a[g][c] = t;
    s_m[g][c] = mx;
    __syncthreads();
    if (threadIdx.x < BW) {
        double tt = s_a[0][c];
        unsigned m2 = s_m[0][c];
        for (int gg = 1; gg < 16; gg++) {
            tt += s_a[gg][c];
            m2 = s_m[gg][c] > m2 ? s_m[gg][c] : m2;
        }
        s_a[0][c] = tt;
        s_m[0][c] = m2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long pend = 0;
        for (int k = 0; k < BW; k++) {
            ctl->l1[k] = s_a[0][k];
            if (((ctl->live >> k) & 1ull) && s_a[0][k] > ctl->stop) pend |= 1ull << k;
            const double target = ctl->refine_ratio * s_a[0][k];
            ctl->sweep_stop[k] = target > 0.5 * ctl->stop ? target : 0.5 * ctl->stop;
        }
        ctl->pending = pend;
        ctl->act = pend;
        ctl->sweep_links = 0;
        ctl->push_ready = 0;
        if (ctl->done != 2u) ctl->done = pend ? 0u : 1u;
    }
    __syncthreads();
    if (threadIdx.x < BW) {
        const bool on = (ctl->act >> c) & 1ull;
        float th = __double2float_ru(ctl->theta_factor * s_a[0][c] / (double)n);
        const float mxf = __uint_as_float(s_m[0][c]);
        if (th > mxf) th = mxf;
        ctl->theta[c] = on ? th : __int_as_float(0x7f800000);
    }
}

// H (n x BW, FP64) to the caller's n x B layout.
__global__ void k_bgather(const double *H, int64_t n, int B, double *out)
{
    const int64_t total = n * B;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = H[(k / B) * BW + (k % B)];
}

// ------------------------------------------------------------------- host
struct BatchBufs {
    int64_t n = 0, slots = 0, ntiles = 0, words = 0, npieces = 0, nch = 0;
    float *F = nullptr, *V = nullptr, *dscale = nullptr, *D = nullptr;
    double *H = nullptr, *R = nullptr, *D64 = nullptr;
    unsigned *mask = nullptr, *hubbits = nullptr, *tmax = nullptr, *tcnt = nullptr;
    float *tl1 = nullptr;
    double *tl1d = nullptr;
    uint32_t *pc_row = nullptr, *pc_start = nullptr, *pc_len = nullptr;
    uint32_t *ch_row = nullptr, *ch_start = nullptr, *ch_len = nullptr;
    BCtl *ctl = nullptr;
};

static void launch_sweep(di_graph_s *g, BatchBufs &b, cudaStream_t s, int use_cond, cudaGraphConditionalHandle h,
                         int grid, cudaEvent_t ev_a = nullptr, cudaEvent_t ev_b = nullptr)
{
    k_bsel<<<(unsigned)b.ntiles, BT, 0, s>>>(b.F, b.n, b.D, b.V, b.dscale, b.mask, b.tl1, b.tmax, b.tcnt, b.ctl,
                                             use_cond, h);
    k_btot<<<BW, BT, 0, s>>>(b.tl1, b.tmax, b.tcnt, b.ntiles, b.n, b.ctl, use_cond, h);
    if (ev_a) cudaEventRecord(ev_a, s);
    k_bpush<<<grid, BT, 0, s>>>(b.F, b.V, static_cast<const Off *>(g->rp), g->col, g->weighted ? g->w32 : nullptr,
                                b.mask, b.hubbits, b.words, b.pc_row, b.pc_start, b.pc_len, b.npieces, b.ctl);
    if (ev_b) cudaEventRecord(ev_b, s);
    count_launches(3);
}

static di_status refine(di_graph_s *g, BatchBufs &b, double d, cudaStream_t s)
{
    di_graph_s *r = g->rev;
    k_bwiden<<<grid_for(b.slots * BW / 4, BT), BT, 0, s>>>(b.D, b.slots * BW, b.D64);
    k_bpull<<<grid_for(b.nch * 32, BT), BT, 0, s>>>(static_cast<const Off *>(r->rp), r->col, r->w, b.ch_row,
                                                    b.ch_start, b.ch_len, b.nch, d, b.D64, b.R, b.H);
    k_bconv<<<(unsigned)b.ntiles, BT, 0, s>>>(b.R, b.F, b.D, b.slots, b.tl1d, b.tmax);
    k_bcycle<<<1, 1024, 0, s>>>(b.tl1d, b.tmax, b.ntiles, b.n, b.ctl);
    count_launches(4);
    DI_CUDA(cudaGetLastError());
    return DI_OK;
}

di_status solve_batch(di_graph_s *g, int B, double d, const double *Z, double tol, const di_opts *o, double *H_out,
                      double *resid_out, di_info *info, int mem, cudaStream_t s)
{
    const int64_t n = g->n;
    DI_TRY(graph_build_reverse(g, s));        // in-links with P[i][j], for the refinement
    DI_TRY(graph_build_push_targets(g, s));   // FP32 copy of the weights
    BatchBufs b;
    b.n = n;
    b.ntiles = (n + BTILE - 1) / BTILE;
    b.slots = b.ntiles * BTILE;
    b.words = b.slots / 32;
    Temps t(s);
    DI_TRY(t.get(&b.F, b.slots * BW));
    DI_TRY(t.get(&b.V, b.slots * BW));
    DI_TRY(t.get(&b.D, b.slots * BW));
    DI_TRY(t.get(&b.H, b.slots * BW));
    DI_TRY(t.get(&b.R, b.slots * BW));
    DI_TRY(t.get(&b.D64, b.slots * BW));
    DI_TRY(t.get(&b.dscale, n));
    DI_TRY(t.get(&b.mask, b.words));
    DI_TRY(t.get(&b.hubbits, b.words));
    DI_TRY(t.get(&b.tl1, b.ntiles * BW));
    DI_TRY(t.get(&b.tl1d, b.ntiles * BW));
    DI_TRY(t.get(&b.tmax, b.ntiles * BW));
    DI_TRY(t.get(&b.tcnt, b.ntiles));
    DI_TRY(t.get(&b.ctl, 1));
    const Off *rp = static_cast<const Off *>(g->rp);
    // static pieces of the long out-rows, chunks of the in-rows
    uint32_t *cnt;
    uint64_t *pos, *tot;
    DI_TRY(t.get(&cnt, n + 1));
    DI_TRY(t.get(&pos, n + 1));
    DI_TRY(t.get(&tot, 2));
    k_bchunks<<<grid_for(n, 256), 256, 0, s>>>(rp, n, BHUB, BPIECE, 0, cnt);
    DI_TRY(scan_exclusive<uint32_t>(cnt, pos, n, tot, s));
    uint64_t hv = 0;
    DI_CUDA(cudaMemcpyAsync(&hv, tot, sizeof(hv), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    b.npieces = (int64_t)hv;
    DI_TRY(t.get(&b.pc_row, b.npieces + 1));
    DI_TRY(t.get(&b.pc_start, b.npieces + 1));
    DI_TRY(t.get(&b.pc_len, b.npieces + 1));
    k_bchunk_fill<<<grid_for(n, 256), 256, 0, s>>>(rp, n, BPIECE, cnt, pos, b.pc_row, b.pc_start, b.pc_len);
    const Off *rrp = static_cast<const Off *>(g->rev->rp);
    k_bchunks<<<grid_for(n, 256), 256, 0, s>>>(rrp, n, PULL_CH, PULL_CH, 1, cnt);
    DI_TRY(scan_exclusive<uint32_t>(cnt, pos, n, tot + 1, s));
    DI_CUDA(cudaMemcpyAsync(&hv, tot + 1, sizeof(hv), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    b.nch = (int64_t)hv;
    DI_TRY(t.get(&b.ch_row, b.nch + 1));
    DI_TRY(t.get(&b.ch_start, b.nch + 1));
    DI_TRY(t.get(&b.ch_len, b.nch + 1));
    k_bchunk_fill<<<grid_for(n, 256), 256, 0, s>>>(rrp, n, PULL_CH, cnt, pos, b.ch_row, b.ch_start, b.ch_len);
    k_bhubbits<<<grid_for(b.words, 256), 256, 0, s>>>(rp, n, b.words, b.hubbits);
    k_bdscale<<<grid_for(n, 256), 256, 0, s>>>(rp, g->weighted ? g->wsum : nullptr, n, d, b.dscale);
    DI_CUDA(cudaMemsetAsync(b.F, 0, sizeof(float) * b.slots * BW, s));
    DI_CUDA(cudaMemsetAsync(b.mask, 0, sizeof(unsigned) * b.words, s));
    k_binit<<<grid_for(b.slots * BW, 256), 256, 0, s>>>(Z, B, n, b.slots, 1.0 - d, 1.0 / (double)n, b.R, b.H, b.D);
    count_launches(7);
    BCtl hc;
    memset(&hc, 0, sizeof(hc));
    hc.stop = (1.0 - d) * tol;
    hc.theta_factor = o->theta_factor;
    hc.refine_ratio = o->refine_ratio;
    hc.live = B >= 64 ? ~0ull : ((1ull << B) - 1ull);
    hc.max_sweeps = (unsigned long long)o->max_sweeps;
    DI_CUDA(cudaMemcpyAsync(b.ctl, &hc, sizeof(hc), cudaMemcpyHostToDevice, s));
    // the first "refinement" only converts R = (1 - d) Z (D = 0)
    k_bconv<<<(unsigned)b.ntiles, BT, 0, s>>>(b.R, b.F, b.D, b.slots, b.tl1d, b.tmax);
    k_bcycle<<<1, 1024, 0, s>>>(b.tl1d, b.tmax, b.ntiles, b.n, b.ctl);
    count_launches(2);
    DI_CUDA(cudaGetLastError());

    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bpush, BT, 0);
    const int grid = (per_sm < 1 ? 1 : per_sm) * sm_count(g->device);
    const bool graph_mode = o->use_graph && !o->profile;
    cudaGraphExec_t gx = nullptr;
    cudaStream_t cs = nullptr;
    if (graph_mode) {
        DI_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph;
        DI_CUDA(cudaGraphCreate(&graph, 0));
        cudaGraphConditionalHandle h;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            launch_sweep(g, b, cs, 1, h, grid);
            cudaGraph_t out = nullptr;
            e = cudaStreamEndCapture(cs, &out);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gx, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cs);
            return note_cuda(e);
        }
    }
    cudaEvent_t e0, e1, pa = nullptr, pb = nullptr;
    DI_CUDA(cudaEventCreate(&e0));
    DI_CUDA(cudaEventCreate(&e1));
    if (o->profile) {
        DI_CUDA(cudaEventCreate(&pa));
        DI_CUDA(cudaEventCreate(&pb));
    }
    double push_ms = 0.0;
    int64_t push_launches = 0, push_links = 0;
    DI_CUDA(cudaEventRecord(e0, s));
    DI_CUDA(cudaMemcpyAsync(&hc, b.ctl, sizeof(hc), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    int64_t refinements = 0;
    di_status rc = DI_OK;
    for (int cycle = 0; hc.done == 0; cycle++) {
        if (cycle == BMAX_CYCLES) {
            hc.done = 2;
            break;
        }
        if (graph_mode) {
            cudaError_t e = cudaGraphLaunch(gx, s);
            if (e != cudaSuccess) {
                rc = note_cuda(e);
                break;
            }
        } else {
            for (;;) {
                for (int k = 0; k < o->check_every; k++) {
                    if (o->profile) {
                        // one sweep at a time: time its push, and take its links
                        // from the totals of the next sweep
                        launch_sweep(g, b, s, 0, cudaGraphConditionalHandle{}, grid, pa, pb);
                        DI_CUDA(cudaMemcpyAsync(&hc, b.ctl, sizeof(hc), cudaMemcpyDeviceToHost, s));
                        DI_CUDA(cudaStreamSynchronize(s));
                        if (hc.push_ready) {
                            float pm = 0.f;
                            DI_CUDA(cudaEventElapsedTime(&pm, pa, pb));
                            push_ms += pm;
                            push_launches++;
                            push_links += (int64_t)hc.sweep_links;
                        }
                        if (hc.done) break;
                    } else {
                        launch_sweep(g, b, s, 0, cudaGraphConditionalHandle{}, grid);
                    }
                }
                DI_CUDA(cudaMemcpyAsync(&hc, b.ctl, sizeof(hc), cudaMemcpyDeviceToHost, s));
                DI_CUDA(cudaStreamSynchronize(s));
                if (hc.done) break;
            }
        }
        rc = refine(g, b, d, s);
        if (rc != DI_OK) break;
        refinements++;
        DI_CUDA(cudaMemcpyAsync(&hc, b.ctl, sizeof(hc), cudaMemcpyDeviceToHost, s));
        DI_CUDA(cudaStreamSynchronize(s));
    }
    DI_CUDA(cudaEventRecord(e1, s));
    if (gx) cudaGraphExecDestroy(gx);
    if (cs) cudaStreamDestroy(cs);
    if (rc != DI_OK) return rc;
    if (graph_mode) count_launches(3 * (int64_t)(hc.sweep + refinements));
    if (H_out) {
        double *dst = H_out;
        if (mem == DI_MEM_HOST) DI_TRY(t.get(&dst, n * B));
        k_bgather<<<grid_for(n * B, 256), 256, 0, s>>>(b.H, n, B, dst);
        count_launches(1);
        if (mem == DI_MEM_HOST)
            DI_CUDA(cudaMemcpyAsync(H_out, dst, sizeof(double) * n * B, cudaMemcpyDeviceToHost, s));
    }
    DI_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    DI_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (pa) cudaEventDestroy(pa);
    if (pb) cudaEventDestroy(pb);
    if (resid_out) {
        if (mem == DI_MEM_HOST) {
            for (int c = 0; c < B; c++) resid_out[c] = hc.l1[c];
        } else {
            DI_CUDA(cudaMemcpyAsync(resid_out, &b.ctl->l1[0], sizeof(double) * B, cudaMemcpyDeviceToDevice, s));
            DI_CUDA(cudaStreamSynchronize(s));
        }
    }
    if (info) {
        double worst = 0.0;
        for (int c = 0; c < B; c++) worst = hc.l1[c] > worst ? hc.l1[c] : worst;
        memset(info, 0, sizeof(*info));
        info->resid_l1 = worst;
        info->bound = worst / (1.0 - d);
        info->sweeps = (int64_t)hc.sweep;
        info->diffusions = (int64_t)hc.diffusions;
        info->edge_pushes = (int64_t)hc.edge_pushes;
        info->time_ms = ms;
        info->refinements = refinements;
        info->push_ms = push_ms;
        info->push_launches = push_launches;
        info->push_edges = push_links;
    }
    if (hc.done == 2) return DI_ERR_NOT_CONVERGED;
    return DI_OK;
}

}  // namespace di
