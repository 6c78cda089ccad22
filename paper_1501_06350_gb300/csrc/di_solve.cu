// The D-Iteration sweep on the GPU (Section 3.1, Eq. defF; Section 3.4).
//
// One sweep diffuses a whole frontier S_t = { i : |F_i| >= theta_t } at once:
//
//   select  (k_select)  one CTA per tile of TILE consecutive nodes (tile ids
//           handed out in launch order).  Reads F, adds |F_i| to an exact
//           fixed-point partial of |F|_1, applies the DI-argmax threshold,
//           *takes* the fluid of the selected nodes (H_i += F_i, F_i = 0) and
//           appends one frontier entry per selected node with out-links:
//           rows of at most HUB_DEG links go to a dense, ascending entry
//           array (tile offsets by a decoupled look-back scan), longer rows
//           are cut into pieces of PIECE links on a separate queue.  The
//           last CTA sums the tile partials (|F_t|_1, hence the next
//           threshold and the stop test).
//   push    (k_push)    warp-centric: a warp takes 32 consecutive entries,
//           prefix-sums their degrees with shuffles, and walks their links
//           32 at a time (coalesced reads of the link targets), adding
//           d F_i P[k][i] to F_k with FP64 atomic adds; hub pieces are
//           walked by one warp each.  No block barrier anywhere.
//
// Diffusing the set S_t at once keeps Eq. HnFn exact: with G = F restricted
// to S_t, H' = H + G and F' = F - G + d P G, so H' + F' = F_0 + d P H'.  Every
// selected node loses (1 - d) of its fluid (all of it if dangling), which is
// the argument of Theorem 3.
//
// FP64 arithmetic is scarce on this part, so |F|_1 inside the sweep is summed
// exactly as 128-bit integers (|F_i| rounded up to a multiple of 2^-fx_shift,
// fx_shift chosen from the initial |F|_1 so the sum stays below 2^113); the
// sum is order-independent, hence deterministic, and an upper bound.
#include <cuda_runtime.h>
#include <new>
#include <string.h>

#include "di_internal.cuh"

namespace di {

using Off = uint32_t;
typedef unsigned __int128 u128;
constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned long long ABS_MASK = 0x7fffffffffffffffull;
constexpr int FX_TOP = 112;            // the initial |F|_1 is scaled below 2^FX_TOP
constexpr unsigned SPIN_MAX = 1u << 22;

__device__ __forceinline__ unsigned long long abs_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & ABS_MASK;
}

// L2 eviction priorities (PTX createpolicy / .L2::cache_hint).  The fluid
// vector F is the target of every atomic add and is read and written by every
// sweep, so its lines are kept with evict_last; the streams that are read
// once per sweep (link targets, frontier entries, row pointers, H, scale
// factors) are marked evict_first so that they do not push F out of L2.
__device__ __forceinline__ unsigned long long pol_last()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long pol_first()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void red_add_f64(double *a, double v, unsigned long long pol)
{
    asm volatile("red.global.add.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(a), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ double2 ld_f64x2(const double *a, unsigned long long pol)
{
    double2 r;
    asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                 : "=d"(r.x), "=d"(r.y)
                 : "l"(a), "l"(pol));
    return r;
}
__device__ __forceinline__ double ld_f64(const double *a, unsigned long long pol)
{
    double r;
    asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(a), "l"(pol));
    return r;
}
__device__ __forceinline__ void st_f64(double *a, double v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(a), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ double ldnc_f64(const double *a, unsigned long long pol)
{
    double r;
    asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(a), "l"(pol));
    return r;
}
__device__ __forceinline__ unsigned ldnc_u32(const unsigned *a, unsigned long long pol)
{
    unsigned r;
    asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(a), "l"(pol));
    return r;
}
__device__ __forceinline__ int ldnc_s32(const int *a, unsigned long long pol)
{
    int r;
    asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(a), "l"(pol));
    return r;
}

// |x| (given by its IEEE bits b, sign cleared) in units of 2^-sh, rounded up.
__device__ __forceinline__ u128 to_fixed(unsigned long long b, int sh)
{
    const int e = (int)(b >> 52);
    unsigned long long m = b & 0x000fffffffffffffull;
    int ex = e;
    if (e == 0) ex = 1;
    else m |= 0x0010000000000000ull;
    const int s = ex - 1075 + sh;   // value = m * 2^(s - sh)
    if (m == 0) return 0;
    if (s >= 0) return s >= 75 ? ~(u128)0 >> 1 : ((u128)m << s);
    if (s <= -64) return 1;
    const unsigned long long q = m >> (-s);
    return (u128)q + ((q << (-s)) != m ? 1 : 0);
}

__device__ __forceinline__ double from_fixed(u128 v, int sh)
{
    const double hi = (double)(unsigned long long)(v >> 64);
    const double lo = (double)(unsigned long long)v;
    return scalbn(fma(hi, 18446744073709551616.0, lo), -sh);
}

__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int o)
{
    const unsigned long long lo = __shfl_xor_sync(FULL, (unsigned long long)v, o);
    const unsigned long long hi = __shfl_xor_sync(FULL, (unsigned long long)(v >> 64), o);
    return ((u128)hi << 64) | lo;
}

// Deterministic block sum of doubles: xor butterfly per warp, then warp 0
// over the warp partials.  Returned to every thread.
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

// Load the 8 fluid values of this thread with the F eviction priority.
__device__ __forceinline__ void load8_keep(const double *F, int64_t i0, int64_t n, double f[8],
                                          unsigned long long pol)
{
    if (i0 + 7 < n) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const double2 a = ld_f64x2(F + i0 + 2 * q, pol);
            f[2 * q] = a.x;
            f[2 * q + 1] = a.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; k++) f[k] = (i0 + k < n) ? ld_f64(F + i0 + k, pol) : 0.0;
    }
}

// Load the SEL_PER_THREAD (= 8) consecutive values of this thread (0 past the end).
__device__ __forceinline__ void load8(const double *F, int64_t i0, int64_t n, double f[8])
{
    if (i0 + 7 < n) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const double2 a = *reinterpret_cast<const double2 *>(F + i0 + 2 * q);
            f[2 * q] = a.x;
            f[2 * q + 1] = a.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; k++) f[k] = (i0 + k < n) ? F[i0 + k] : 0.0;
    }
}

// --------------------------------------------------------------- reduce
// FP64 |v|_1 (and, with H, l = sum of H_i over dangling i): per-thread order,
// warp butterfly, warp partials in order, tile partials in a fixed strided
// order by the last CTA.  Used at the start (threshold, fixed-point scale)
// and at the end of a solve (reported residual).
enum { RED_PLAIN = 0, RED_INIT = 1, RED_FINAL = 2 };

__global__ void __launch_bounds__(SEL_THREADS) k_reduce(const double *v, const double *H, const Off *rp,
                                                       int64_t n, int64_t ntiles, double *part_l1,
                                                       double *part_l, DevCtl *ctl, int mode)
{
    __shared__ double sm[SEL_THREADS / 32 + 1];
    __shared__ int s_last;
    const int64_t tile = blockIdx.x;
    const int64_t i0 = tile * TILE + (int64_t)threadIdx.x * SEL_PER_THREAD;
    double f[8];
    load8(v, i0, n, f);
    double a = fabs(f[0]);
#pragma unroll
    for (int k = 1; k < 8; k++) a += fabs(f[k]);
    double l = 0.0;
    if (H) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
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
            int e = 0;
            if (sa > 0.0) frexp(sa, &e);    // sa < 2^e
            ctl->fx_shift = FX_TOP - 1 - e;  // |F|_1 scaled below 2^(FX_TOP-1), room to grow 2x
        } else {
            ctl->final_l1 = sa;
            ctl->final_l = sl;
        }
    }
}

// --------------------------------------------------------------- select
// Per-thread counters packed for one block scan:
//   bits 0..11 dense entries, 12..23 nodes taken, 24..63 links.
constexpr int PK_TAKEN = 12;
constexpr int PK_LINKS = 24;
// look-back word: tag (24 bits) | flag (2 bits) | inclusive-or-local count (38 bits)
constexpr unsigned long long LB_AGG = 1ull, LB_PRE = 2ull;

__device__ __forceinline__ unsigned long long lb_word(unsigned tag, unsigned long long flag,
                                                      unsigned long long v)
{
    return ((unsigned long long)(tag & 0xffffffu) << 40) | (flag << 38) | v;
}

__global__ void __launch_bounds__(SEL_THREADS)
    k_select(const Off *__restrict__ rp, const double *__restrict__ dscale, double *F, double *H,
             int64_t n, int64_t ntiles, Off *ent_row, Off *ent_deg, double *ent_val, Off *pc_row,
             Off *pc_len, double *pc_val, unsigned *tile_cnt, unsigned long long *tile_edges,
             unsigned *tile_diff, unsigned long long *tile_fx, unsigned long long *tile_max,
             unsigned long long *lb_status, unsigned *lb_epoch, DevCtl *ctl, int use_cond,
             cudaGraphConditionalHandle cond, int32_t *sel_ids, unsigned long long *stats)
{
    __shared__ unsigned long long smu[SEL_THREADS / 32 + 1];
    __shared__ unsigned long long s_fx[SEL_THREADS / 32][2];
    __shared__ unsigned long long s_mx[SEL_THREADS / 32];
    __shared__ unsigned long long s_base;
    __shared__ unsigned s_tile;
    __shared__ int s_last;
    volatile DevCtl *vc = ctl;
    if (vc->done) {
        // Nothing left to do: the push that follows must find no work (its
        // counts still describe the frontier it has already pushed), and a
        // graph while-loop must end here too.
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            vc->nent = 0;
            vc->npieces_done = 0;
            if (use_cond) cudaGraphSetConditional(cond, 0u);
        }
        return;
    }
    const double theta = vc->theta;
    const int fxs = vc->fx_shift;
    const unsigned tag = *((volatile unsigned *)lb_epoch) + 1u;
    const unsigned long long tb = abs_bits(theta);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(&ctl->tile_next, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t i0 = tile * TILE + (int64_t)threadIdx.x * SEL_PER_THREAD;

    const unsigned long long keep = pol_last(), stream = pol_first();
    double f[8];
    load8_keep(F, i0, n, f, keep);
    u128 fx = 0;
    unsigned selm = 0;
    unsigned long long mb = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const unsigned long long b = abs_bits(f[k]);
        fx += to_fixed(b, fxs);
        if ((i0 + k < n) && b != 0 && b >= tb) selm |= 1u << k;
        mb = b > mb ? b : mb;
    }
    Off r[9];
    unsigned long long packed = (unsigned long long)__popc(selm) << PK_TAKEN;
    unsigned npc = 0;
    if (selm) {
#pragma unroll
        for (int k = 0; k < 9; k++) r[k] = (i0 + k <= n) ? ldnc_u32(rp + i0 + k, stream) : 0;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const Off deg = r[k + 1] - r[k];
            if (!((selm >> k) & 1u) || deg == 0) continue;
            packed += (unsigned long long)deg << PK_LINKS;
            if (deg <= (Off)HUB_DEG) packed += 1ull;
            else npc += (deg + PIECE - 1) / PIECE;
        }
    }
    // warp partials of |F|_1 (exact integers) and of max |F_i|
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fx += shfl_xor_u128(fx, o);
        const unsigned long long y = __shfl_xor_sync(FULL, mb, o);
        mb = y > mb ? y : mb;
    }
    if (lane == 0) {
        s_fx[warp][0] = (unsigned long long)fx;
        s_fx[warp][1] = (unsigned long long)(fx >> 64);
        s_mx[warp] = mb;
    }
    unsigned long long tot;
    const unsigned long long pre = block_exscan_u64<SEL_THREADS>(packed, smu, &tot);
    const unsigned long long cnt = tot & 0xfff;

    // tile offset in the dense entry array: decoupled look-back over the
    // tiles handed out before this one (they are all running or done)
    if (threadIdx.x == 0) {
        unsigned long long base = 0;
        if (tile == 0) {
            atomicExch(lb_status, lb_word(tag, LB_PRE, cnt));
        } else {
            atomicExch(lb_status + tile, lb_word(tag, LB_AGG, cnt));
            for (int64_t p = tile - 1; p >= 0; p--) {
                unsigned long long wv = 0;
                unsigned it = 0;
                for (; it < SPIN_MAX; it++) {
                    wv = *((volatile unsigned long long *)(lb_status + p));
                    if ((unsigned)(wv >> 40) == (tag & 0xffffffu) && ((wv >> 38) & 3ull)) break;
                    __nanosleep(64);
                }
                if (it == SPIN_MAX) {          // give up: flag the error, keep positions in range
                    atomicOr(&ctl->err, 1u);
                    break;
                }
                base += wv & ((1ull << 38) - 1);
                if (((wv >> 38) & 3ull) == LB_PRE) break;
            }
            atomicExch(lb_status + tile, lb_word(tag, LB_PRE, base + cnt));
        }
        s_base = base;
    }
    __syncthreads();
    if (selm) {
        unsigned long long pos = s_base + (pre & 0xfff);
        unsigned spos = (unsigned)((pre >> PK_TAKEN) & 0xfff);
        const int64_t slot0 = tile * TILE;
        unsigned pbase = npc ? (unsigned)atomicAdd(&ctl->npieces, (unsigned long long)npc) : 0u;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if (!((selm >> k) & 1u)) continue;
            const int64_t i = i0 + k;
            st_f64(H + i, ld_f64(H + i, stream) + f[k], stream);
            st_f64(F + i, 0.0, keep);
            if (sel_ids) sel_ids[slot0 + spos++] = (int32_t)i;
            const Off deg = r[k + 1] - r[k];
            if (deg == 0) continue;
            const double v = f[k] * ldnc_f64(dscale + i, stream);
            if (deg <= (Off)HUB_DEG) {
                ent_row[pos] = r[k];
                ent_deg[pos] = deg;
                ent_val[pos] = v;
                pos++;
            } else {
                for (Off o = 0; o < deg; o += PIECE) {
                    pc_row[pbase] = r[k] + o;
                    pc_len[pbase] = deg - o < (Off)PIECE ? deg - o : (Off)PIECE;
                    pc_val[pbase] = v;
                    pbase++;
                }
            }
        }
    }
    if (threadIdx.x == 0) {
        u128 t = 0;
        unsigned long long mx = 0;
#pragma unroll
        for (int w = 0; w < SEL_THREADS / 32; w++) {
            t += ((u128)s_fx[w][1] << 64) | s_fx[w][0];
            mx = s_mx[w] > mx ? s_mx[w] : mx;
        }
        tile_fx[2 * tile] = (unsigned long long)t;
        tile_fx[2 * tile + 1] = (unsigned long long)(t >> 64);
        tile_max[tile] = mx;
        tile_cnt[tile] = (unsigned)cnt;
        tile_edges[tile] = tot >> PK_LINKS;
        tile_diff[tile] = (unsigned)((tot >> PK_TAKEN) & 0xfff);
        __threadfence();
        const unsigned tk = atomicAdd(&ctl->ticket, 1u);
        s_last = (tk == (unsigned)(ntiles - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // ---- epilogue: one CTA; integer totals are order-free, hence exact
    u128 sfx = 0;
    unsigned long long sd = 0, se = 0, sc = 0, mx = 0;
#pragma unroll 4
    for (int64_t k = threadIdx.x; k < ntiles; k += SEL_THREADS) {
        sfx += ((u128)__ldcg(tile_fx + 2 * k + 1) << 64) | __ldcg(tile_fx + 2 * k);
        sd += __ldcg(tile_diff + k);
        se += __ldcg(tile_edges + k);
        sc += __ldcg(tile_cnt + k);
        const unsigned long long m = __ldcg(tile_max + k);
        mx = m > mx ? m : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sfx += shfl_xor_u128(sfx, o);
        sd += __shfl_xor_sync(FULL, sd, o);
        se += __shfl_xor_sync(FULL, se, o);
        sc += __shfl_xor_sync(FULL, sc, o);
        const unsigned long long y = __shfl_xor_sync(FULL, mx, o);
        mx = y > mx ? y : mx;
    }
    __shared__ unsigned long long s_red[6][SEL_THREADS / 32];
    if (lane == 0) {
        s_red[0][warp] = (unsigned long long)sfx;
        s_red[1][warp] = (unsigned long long)(sfx >> 64);
        s_red[2][warp] = sd;
        s_red[3][warp] = se;
        s_red[4][warp] = sc;
        s_red[5][warp] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sfx = 0;
        sd = se = sc = mx = 0;
        for (int w = 0; w < SEL_THREADS / 32; w++) {
            sfx += ((u128)s_red[1][w] << 64) | s_red[0][w];
            sd += s_red[2][w];
            se += s_red[3][w];
            sc += s_red[4][w];
            mx = s_red[5][w] > mx ? s_red[5][w] : mx;
        }
        const double sa = from_fixed(sfx, fxs);
        ctl->l1 = sa;
        ctl->nent = sc;
        ctl->npieces_done = *((volatile unsigned long long *)&ctl->npieces);
        ctl->npieces = 0;
        ctl->total_edges = se;
        ctl->diffusions += sd;
        ctl->edge_pushes += se;
        const unsigned long long sweep = ctl->sweep + 1;
        ctl->sweep = sweep;
        if (stats && sweep <= (unsigned long long)STAT_CAP) {
            stats[2 * (sweep - 1)] = se;
            stats[2 * (sweep - 1) + 1] = sc;
        }
        unsigned done = 0;
        // the integer sum rounds every |F_i| up, so it bounds |F_t|_1 from above
        if (sa <= ctl->stop_l1) done = 1;
        else if (sweep >= ctl->max_sweeps) done = 2;
        if (ctl->err) done = 3;
        double th = ctl->theta_factor * sa / (double)n;
        // A sweep that took nothing left F unchanged; the largest |F_i| passes
        // the DI-argmax test exactly, so never ask for more than that (this
        // covers a rounded average above every one of several equal fluids).
        const double fmax = __longlong_as_double((long long)mx);
        if (sd == 0 && fmax < th) th = fmax;
        ctl->theta = th;
        ctl->ticket = 0;
        ctl->tile_next = 0;
        *lb_epoch = tag;
        __threadfence();
        ctl->done = done;
        if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
    }
}

// ----------------------------------------------------------------- push
// Warp-centric push.  Work unit u < nchunks: entries [32u, 32u + 32) of the
// dense frontier; u >= nchunks: hub piece u - nchunks.  Lane j of a chunk
// owns entry 32u + j; the chunk's links are enumerated 32 at a time and each
// lane finds the entry of its link by a binary search over the lanes'
// exclusive degree prefixes (shuffles only).
template <bool WEIGHTED>
__global__ void __launch_bounds__(PUSH_THREADS)
    k_push(const Off *__restrict__ ent_row, const Off *__restrict__ ent_deg,
           const double *__restrict__ ent_val, const Off *__restrict__ pc_row,
           const Off *__restrict__ pc_len, const double *__restrict__ pc_val,
           const int32_t *__restrict__ col, const double *__restrict__ w, double *F, const DevCtl *ctl)
{
    const unsigned long long nent = ((volatile const DevCtl *)ctl)->nent;
    const unsigned long long npc = ((volatile const DevCtl *)ctl)->npieces_done;
    const unsigned long long keep = pol_last(), stream = pol_first();
    const int lane = threadIdx.x & 31;
    const unsigned long long nchunks = (nent + 31) / 32;
    const unsigned long long nunits = nchunks + npc;
    const unsigned long long wid = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long u = wid; u < nunits; u += nw) {
        if (u < nchunks) {
            const unsigned long long k = u * 32 + lane;
            Off row = 0, deg = 0;
            double val = 0.0;
            if (k < nent) {
                row = ldnc_u32(ent_row + k, stream);
                deg = ldnc_u32(ent_deg + k, stream);
                val = ldnc_f64(ent_val + k, stream);
            }
            Off incl = deg;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const Off y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            const Off total = __shfl_sync(FULL, incl, 31);
            const Off excl = incl - deg;
            // lanes' links are e = base + lane; four groups in flight
            for (Off base = 0; base < total; base += 128) {
                int32_t c[4];
                double v[4];
#pragma unroll
                for (int g = 0; g < 4; g++) {
                    const Off e = base + (Off)(g * 32 + lane);
                    const Off eq = e < total ? e : total - 1;
                    int j = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const Off ex = __shfl_sync(FULL, excl, j + step);
                        if (ex <= eq) j += step;
                    }
                    const Off rj = __shfl_sync(FULL, row, j);
                    const Off xj = __shfl_sync(FULL, excl, j);
                    const double vj = __shfl_sync(FULL, val, j);
                    c[g] = -1;
                    v[g] = vj;
                    if (e < total) {
                        const Off link = rj + (e - xj);
                        c[g] = ldnc_s32(col + link, stream);
                        if (WEIGHTED) v[g] = vj * ldnc_f64(w + link, stream);
                    }
                }
#pragma unroll
                for (int g = 0; g < 4; g++)
                    if (c[g] >= 0) red_add_f64(F + c[g], v[g], keep);
            }
        } else {
            const unsigned long long p = u - nchunks;
            const Off row = ldnc_u32(pc_row + p, stream), len = ldnc_u32(pc_len + p, stream);
            const double val = ldnc_f64(pc_val + p, stream);
            for (Off base = 0; base < len; base += 128) {
                int32_t c[4];
                double v[4];
#pragma unroll
                for (int g = 0; g < 4; g++) {
                    const Off e = base + (Off)(g * 32 + lane);
                    c[g] = -1;
                    v[g] = val;
                    if (e < len) {
                        c[g] = ldnc_s32(col + row + e, stream);
                        if (WEIGHTED) v[g] = val * ldnc_f64(w + row + e, stream);
                    }
                }
#pragma unroll
                for (int g = 0; g < 4; g++)
                    if (c[g] >= 0) red_add_f64(F + c[g], v[g], keep);
            }
        }
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
    st->max_items = g->nnz / PIECE + g->nnz / HUB_DEG + 2;
    const int64_t slots = st->ntiles * TILE;
    DI_TRY(dalloc_t(&st->F, slots, s));
    DI_TRY(dalloc_t(&st->H, slots, s));
    DI_TRY(dalloc_t(&st->dscale, n, s));
    DI_TRY(dalloc_t(&st->ent_row, n, s));
    DI_TRY(dalloc_t(&st->ent_deg, n, s));
    DI_TRY(dalloc_t(&st->ent_val, n, s));
    DI_TRY(dalloc_t(&st->pc_row, st->max_items, s));
    DI_TRY(dalloc_t(&st->pc_len, st->max_items, s));
    DI_TRY(dalloc_t(&st->pc_val, st->max_items, s));
    DI_TRY(dalloc_t(&st->tile_cnt, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_edges, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_diff, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_fx, 2 * st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_max, st->ntiles, s));
    DI_TRY(dalloc_t(&st->lb_status, st->ntiles, s));
    DI_TRY(dalloc_t(&st->lb_epoch, 1, s));
    DI_TRY(dalloc_t(&st->tile_l1, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_l, st->ntiles, s));
    DI_TRY(dalloc_t(&st->ctl, 1, s));
    DI_TRY(dalloc_t(&st->stats, 2 * STAT_CAP, s));
    DI_CUDA(cudaMemsetAsync(st->ctl, 0, sizeof(DevCtl), s));
    DI_CUDA(cudaMemsetAsync(st->lb_status, 0, sizeof(unsigned long long) * st->ntiles, s));
    DI_CUDA(cudaMemsetAsync(st->lb_epoch, 0, sizeof(unsigned), s));
    DI_CUDA(cudaMemsetAsync(st->F, 0, sizeof(double) * slots, s));
    DI_CUDA(cudaMemsetAsync(st->H, 0, sizeof(double) * slots, s));
    DI_CUDA(cudaMallocHost(reinterpret_cast<void **>(&st->host_ctl), sizeof(DevCtl)));
    memset(st->host_ctl, 0, sizeof(DevCtl));
    DI_CUDA(cudaEventCreate(&st->ev0));
    DI_CUDA(cudaEventCreate(&st->ev1));
    DI_CUDA(cudaStreamSynchronize(s));
    return DI_OK;
}

di_status state_free(di_state_s *st)
{
    cudaStream_t s = 0;
    if (st->gexec) cudaGraphExecDestroy(st->gexec);
    if (st->gstream) cudaStreamDestroy(st->gstream);
    void *bufs[] = {st->F, st->H, st->dscale, st->ent_row, st->ent_deg, st->ent_val, st->pc_row,
                    st->pc_len, st->pc_val, st->tile_cnt, st->tile_edges, st->tile_diff, st->tile_fx,
                    st->tile_max, st->lb_status, st->lb_epoch, st->tile_l1, st->tile_l, st->ctl,
                    st->stats};
    for (void *p : bufs) dfree(p, s);
    if (st->host_ctl) cudaFreeHost(st->host_ctl);
    if (st->ev0) cudaEventDestroy(st->ev0);
    if (st->ev1) cudaEventDestroy(st->ev1);
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
        static_cast<const Off *>(g->rp), st->dscale, st->F, st->H, g->n, st->ntiles, st->ent_row,
        st->ent_deg, st->ent_val, st->pc_row, st->pc_len, st->pc_val, st->tile_cnt, st->tile_edges,
        st->tile_diff, st->tile_fx, st->tile_max, st->lb_status, st->lb_epoch, st->ctl, use_cond, h,
        sel_ids, st->stats);
    count_launches(1);
}

static void launch_push(di_graph_s *g, di_state_s *st, cudaStream_t s)
{
    const int grid = push_grid(st->device);
    if (g->weighted)
        k_push<true><<<grid, PUSH_THREADS, 0, s>>>(st->ent_row, st->ent_deg, st->ent_val, st->pc_row,
                                                  st->pc_len, st->pc_val, g->col, g->w, st->F, st->ctl);
    else
        k_push<false><<<grid, PUSH_THREADS, 0, s>>>(st->ent_row, st->ent_deg, st->ent_val, st->pc_row,
                                                   st->pc_len, st->pc_val, g->col, nullptr, st->F,
                                                   st->ctl);
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
    if (hc->err || hc->done == 3) return DI_ERR_DEVICE_TIMEOUT;
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
            hc->fx_shift = 0;
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
