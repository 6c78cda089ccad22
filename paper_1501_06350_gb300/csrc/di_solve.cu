// The D-Iteration sweep on the GPU (Section 3.1, Eq. defF; Section 3.4).
//
// One sweep diffuses the frontier S_t = { i : |F_i| >= theta_t }:
//
//   select  (k_select)  streams F once: an exact fixed-point partial of
//           |F_t|_1 and max |F_i| per tile, the DI-argmax test, and the
//           frontier as a bit mask (one bit per node); selected hub rows
//           (more than hub_deg links) go to a short list instead.
//   plan    (k_plan)    every CTA sums the tile partials (integers, so all
//           CTAs agree exactly), decides the stop test |F_t|_1/(1-d) <= tol
//           (Theorem 1, Eq. SL) and the next threshold, and takes the fluid
//           of the selected hubs (F is quiescent here), cutting their rows
//           into pieces of `piece` links.
//   push    (k_push)    warp-centric: a warp takes 32 nodes with their mask
//           word, takes the fluid of the set ones with an atomic exchange,
//           moves it into H, and scatters d F_i P[k][i] along their links with
//           FP64 atomic adds; hub pieces are scattered the same way.  No block
//           barrier inside the loop.
//
// Each atomic take-and-push is one elementary diffusion of Eq. defF (with
// whatever fluid the node holds at that moment), so Eq. HnFn holds exactly
// for any interleaving; every taken node loses (1 - d) of its fluid (all of it
// if dangling), which is the argument of Theorem 3.  Nothing is taken before
// the stop test, so the |F|_1 the test certifies is that of the final state.
//
// FP64 arithmetic is scarce on this part (about 1/64 of the FP32 rate), so
// |F|_1 inside the sweep is summed in FP32 with every value and every partial
// sum rounded upward (an upper bound of the exact sum, in a fixed order, hence
// deterministic), and the push adds the contributions to the most linked-to
// pages in shared memory as 64-bit fixed-point integers (native integer
// atomics) before one FP64 add per page and CTA.
#include <cuda_runtime.h>
#include <new>
#include <string.h>
#include <vector>

#include "di_internal.cuh"

namespace di {

using Off = uint32_t;
constexpr unsigned FULL = 0xffffffffu;
constexpr unsigned long long ABS_MASK = 0x7fffffffffffffffull;

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
// The cache-hinted loads and stores move raw 64-bit words: a double-typed
// asm operand that is later reinterpreted as an integer costs an FP64
// instruction per value on this part, and FP64 issue is scarce.
__device__ __forceinline__ void ld_b64x2(const double *a, unsigned long long pol, unsigned long long &x,
                                         unsigned long long &y)
{
    asm volatile("ld.global.L2::cache_hint.v2.b64 {%0, %1}, [%2], %3;" : "=l"(x), "=l"(y) : "l"(a), "l"(pol));
}
__device__ __forceinline__ unsigned long long ld_b64(const double *a, unsigned long long pol)
{
    unsigned long long r;
    asm volatile("ld.global.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(r) : "l"(a), "l"(pol));
    return r;
}
__device__ __forceinline__ void st_b64(double *a, unsigned long long v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(a), "l"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ double ldnc_f64(const double *a, unsigned long long pol)
{
    unsigned long long r;
    asm volatile("ld.global.nc.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(r) : "l"(a), "l"(pol));
    return __longlong_as_double((long long)r);
}
__device__ __forceinline__ uint4 ldnc_u32x4(const unsigned *a, unsigned long long pol)
{
    uint4 r;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(a), "l"(pol));
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

// |x| (given by the IEEE bits b of a double, sign cleared) as FP32 bits,
// rounded upward (values below FLT_MIN become FLT_MIN, overflow becomes inf).
__device__ __forceinline__ unsigned f32_up_bits(unsigned long long b)
{
    if (b == 0) return 0u;
    const int e = (int)(b >> 52) - 1023 + 127;
    if (e >= 255) return 0x7f800000u;
    if (e <= 0) return 0x00800000u;
    const unsigned lo = (unsigned)b, hi = (unsigned)(b >> 32);
    const unsigned mf = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned up = (lo & 0x1fffffffu) != 0u;
    return ((unsigned)e << 23) + mf + up;    // a carry moves into the exponent
}

// Same, rounded downward (values below FLT_MIN become 0).
__device__ __forceinline__ unsigned f32_down_bits(unsigned long long b)
{
    const int e = (int)(b >> 52) - 1023 + 127;
    if (e >= 255) return 0x7f7fffffu;
    if (e <= 0) return 0u;
    const unsigned lo = (unsigned)b, hi = (unsigned)(b >> 32);
    return ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
}

// v * 2^sh rounded to the nearest 64-bit integer (two's complement), from the
// bits of v; |v| * 2^sh must stay below 2^62.
__device__ __forceinline__ long long to_fixed64(double v, int sh)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ffu);
    if (ex == 0) return 0;   // zero or subnormal: below every scale used here
    const unsigned long long m = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;
    const int s = ex - 1075 + sh;
    long long q;
    if (s >= 0) q = (long long)(m << (s < 10 ? s : 10));
    else if (s > -64) q = (long long)((m + (1ull << (-s - 1))) >> (-s));
    else q = 0;
    return (b >> 63) ? -q : q;
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
// Unweighted rows read d / out(j) from the table of k_dtab when given (FP64
// division is slow on this part; the table holds the same quotients).
__global__ void k_dscale(const Off *rp, const double *wsum, const double *dtab, int64_t n, double d,
                         double *dscale)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Off deg = rp[i + 1] - rp[i];
        double v;
        if (deg == 0) v = 0.0;
        else if (wsum) v = d / wsum[i];
        else if (dtab && deg <= (Off)DTAB_MAX) v = __ldg(dtab + deg);
        else v = d / (double)deg;
        dscale[i] = v;
    }
}

// d / k for k = 0 .. DTAB_MAX (0 at k = 0): the same division as k_dscale,
// so a row's share from the table is bit for bit its d / out(j).
__global__ void k_dtab(double d, double *dtab)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= DTAB_MAX; k += gridDim.x * blockDim.x)
        dtab[k] = k == 0 ? 0.0 : d / (double)k;
}

__global__ void k_scale(double *out, const double *in, int64_t n, double a)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a * in[i];
}

// Load the IEEE bits of the P consecutive fluid values of this thread (0
// past the end) with the eviction priority of F.
template <int P>
__device__ __forceinline__ void loadP_keep(const double *F, int64_t i0, int64_t n, unsigned long long *fb,
                                           unsigned long long pol)
{
    if (i0 + P - 1 < n) {
#pragma unroll
        for (int q = 0; q < P / 2; q++) ld_b64x2(F + i0 + 2 * q, pol, fb[2 * q], fb[2 * q + 1]);
    } else {
#pragma unroll
        for (int k = 0; k < P; k++) fb[k] = (i0 + k < n) ? ld_b64(F + i0 + k, pol) : 0ull;
    }
}

// Load the P consecutive values of this thread (0 past the end).
template <int P>
__device__ __forceinline__ void loadP(const double *F, int64_t i0, int64_t n, double *f)
{
    if (i0 + P - 1 < n) {
#pragma unroll
        for (int q = 0; q < P / 2; q++) {
            const double2 a = *reinterpret_cast<const double2 *>(F + i0 + 2 * q);
            f[2 * q] = a.x;
            f[2 * q + 1] = a.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < P; k++) f[k] = (i0 + k < n) ? F[i0 + k] : 0.0;
    }
}

// --------------------------------------------------------------- reduce
// FP64 |v|_1 (and, with H, l = sum of H_i over dangling i): per-thread order,
// warp butterfly, warp partials in order, tile partials in a fixed strided
// order by the last CTA.  Used at the start (threshold) and at the end of a
// solve (reported residual), and after every refinement pass of the FP32
// form, where it also writes the FP32 copy of the fluid (v32, every slot of
// the tile, 0 past n) and sets the targets of the next cycle.
enum { RED_PLAIN = 0, RED_INIT = 1, RED_FINAL = 2, RED_CYCLE = 3 };

// Deterministic block max of non-negative doubles (returned to every thread).
template <int NT>
__device__ __forceinline__ double block_max(double v, double *sm)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double x = lane < NT / 32 ? sm[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(FULL, x, o));
        if (lane == 0) sm[NT / 32] = x;
    }
    __syncthreads();
    double r = sm[NT / 32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SEL_THREADS) k_reduce(const double *v, const double *H, const Off *rp,
                                                       int64_t n, int64_t ntiles, double *part_l1,
                                                       double *part_l, double *part_max, DevCtl *ctl, int mode,
                                                       float *v32)
{
    __shared__ double sm[SEL_THREADS / 32 + 1];
    __shared__ int s_last;
    const int64_t tile = blockIdx.x;
    const int64_t i0 = tile * TILE + (int64_t)threadIdx.x * SEL_PER_THREAD;
    constexpr int P = SEL_PER_THREAD;
    double f[P];
    loadP<P>(v, i0, n, f);
    if (v32) {
        static_assert(P % 4 == 0, "whole 16-byte stores");
#pragma unroll
        for (int q = 0; q < P / 4; q++)
            *reinterpret_cast<float4 *>(v32 + i0 + 4 * q) =
                make_float4((float)f[4 * q], (float)f[4 * q + 1], (float)f[4 * q + 2], (float)f[4 * q + 3]);
    }
    // the largest |f| by the integer order of the magnitude bits (the same as
    // the FP64 order for non-NaN values; integer compares keep the narrow FP64
    // pipe of this part for the sum)
    double a = fabs(f[0]);
    unsigned long long mxb = abs_bits(f[0]);
#pragma unroll
    for (int k = 1; k < P; k++) {
        a += fabs(f[k]);
        const unsigned long long b = abs_bits(f[k]);
        mxb = b > mxb ? b : mxb;
    }
    double mxv = __longlong_as_double((long long)mxb);
    double l = 0.0;
    if (H) {
#pragma unroll
        for (int k = 0; k < P; k++) {
            const int64_t i = i0 + k;
            if (i < n && rp[i + 1] == rp[i]) l += H[i];
        }
    }
    a = block_sum_det<SEL_THREADS>(a, sm);
    l = block_sum_det<SEL_THREADS>(l, sm);
    if (part_max) mxv = block_max<SEL_THREADS>(mxv, sm);
    if (threadIdx.x == 0) {
        part_l1[tile] = a;
        part_l[tile] = l;
        if (part_max) part_max[tile] = mxv;
        __threadfence();
        const unsigned t = atomicAdd(&ctl->ticket2, 1u);
        s_last = (t == (unsigned)(ntiles - 1));
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double sa = 0.0, sl = 0.0, smx = 0.0;
    for (int64_t k = threadIdx.x; k < ntiles; k += SEL_THREADS) {
        sa += __ldcg(part_l1 + k);
        sl += __ldcg(part_l + k);
        if (part_max) smx = fmax(smx, __ldcg(part_max + k));
    }
    sa = block_sum_det<SEL_THREADS>(sa, sm);
    sl = block_sum_det<SEL_THREADS>(sl, sm);
    if (part_max) smx = block_max<SEL_THREADS>(smx, sm);
    if (threadIdx.x == 0) {
        ctl->ticket2 = 0;
        ctl->final_max = smx;
        if (mode == RED_INIT || mode == RED_CYCLE) {
            // a loop that ended in its stop test leaves the hubs of its last
            // selection listed (nobody took them): start the next one clean
            ctl->npieces = 0;
            ctl->push_ready = 0;
            ctl->l1 = sa;
            ctl->theta = ctl->theta_factor * sa / (double)n;
            if (mode == RED_INIT) {
                ctl->sweep_stop = ctl->stop_l1;
                ctl->done = (ctl->inf_norm ? smx : sa) <= ctl->stop_l1 ? 1u : 0u;
            } else {
                // FP32 cycle: run to refine_ratio x the exact |F|_1 (never
                // further than half the final target); a reached sweep cap
                // stays reached
                const double target = ctl->refine_ratio * sa;
                ctl->sweep_stop = target > 0.5 * ctl->stop_l1 ? target : 0.5 * ctl->stop_l1;
                if (ctl->done != 2u) ctl->done = sa <= ctl->stop_l1 ? 1u : 0u;
            }
        } else {
            ctl->final_l1 = sa;
            ctl->final_l = sl;
        }
    }
}

// ------------------------------------------------------ fluid word types
// The sweep kernels move the fluid either as FP64 (the plain form) or as FP32
// (the iterative-refinement form); these overloads give the raw-word access
// to either.
template <typename T>
struct FluidWord;
template <>
struct FluidWord<double> {
    typedef unsigned long long U;
    static constexpr unsigned long long ABS = ABS_MASK;
};
template <>
struct FluidWord<float> {
    typedef unsigned U;
    static constexpr unsigned ABS = 0x7fffffffu;
};

__device__ __forceinline__ double word_val(unsigned long long b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ float word_val(unsigned b) { return __uint_as_float(b); }

__device__ __forceinline__ unsigned ld_b32(const float *a, unsigned long long pol)
{
    unsigned r;
    asm volatile("ld.global.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(r) : "l"(a), "l"(pol));
    return r;
}
__device__ __forceinline__ unsigned long long ld_word(const double *a, unsigned long long pol) { return ld_b64(a, pol); }
__device__ __forceinline__ unsigned ld_word(const float *a, unsigned long long pol) { return ld_b32(a, pol); }
__device__ __forceinline__ void st_word(double *a, unsigned long long v, unsigned long long pol) { st_b64(a, v, pol); }
__device__ __forceinline__ void st_word(float *a, unsigned v, unsigned long long pol)
{
    asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(pol) : "memory");
}

// The P consecutive fluid words of a selection thread (0 past the end).
template <int P>
__device__ __forceinline__ void loadw_keep(const double *F, int64_t i0, int64_t n, unsigned long long *fb,
                                           unsigned long long pol)
{
    loadP_keep<P>(F, i0, n, fb, pol);
}
template <int P>
__device__ __forceinline__ void loadw_keep(const float *F, int64_t i0, int64_t n, unsigned *fb,
                                           unsigned long long pol)
{
    static_assert(P % 4 == 0, "whole 16-byte words");
    if (i0 + P - 1 < n) {
#pragma unroll
        for (int q = 0; q < P / 4; q++)
            asm volatile("ld.global.L2::cache_hint.v4.b32 {%0, %1, %2, %3}, [%4], %5;"
                         : "=r"(fb[4 * q]), "=r"(fb[4 * q + 1]), "=r"(fb[4 * q + 2]), "=r"(fb[4 * q + 3])
                         : "l"(F + i0 + 4 * q), "l"(pol));
    } else {
#pragma unroll
        for (int k = 0; k < P; k++) fb[k] = (i0 + k < n) ? ld_b32(F + i0 + k, pol) : 0u;
    }
}

// |x| as FP32 bits rounded upward / downward (exact for FP32 fluid).
__device__ __forceinline__ unsigned up32(unsigned long long b) { return f32_up_bits(b); }
__device__ __forceinline__ unsigned up32(unsigned b) { return b; }
__device__ __forceinline__ unsigned down32(unsigned long long b) { return f32_down_bits(b); }
__device__ __forceinline__ unsigned down32(unsigned b) { return b; }

// Bits of the smallest fluid magnitude that passes |F_i| >= theta: for FP32
// fluid, theta rounded up to the next FP32 value (subnormals included), so
// that the test on FP32 words is the exact test against the FP64 theta.
__device__ __forceinline__ unsigned long long theta_word(double th, const double *) { return abs_bits(th); }
__device__ __forceinline__ unsigned theta_word(double th, const float *)
{
    const unsigned long long b = abs_bits(th);
    if (b < (0x381ull << 52)) return (unsigned)ceil(__longlong_as_double((long long)b) * 0x1p149);
    return f32_up_bits(b);
}

// --------------------------------------------------------------- select
// One CTA of SEL_THREADS per tile of TILE nodes.  The tile is read in
// SEL_ROUNDS rounds; in round q warp w covers the 64 nodes
// tile + q * 2 SEL_THREADS + 64 w, lane l its nodes l and 32 + l, so every
// load instruction of a warp reads 32 consecutive words (coalesced) and every
// frontier mask word is one warp ballot.  Per node: the exact DI-argmax test
// on the raw fluid word, and FP32 upper-bound partials of |F|_1 and of
// max |F_i| taken from the word's upper 32 bits (sign, exponent, 20 mantissa
// bits), which bound |x| from below as they are and from above with one
// unit added in their last place (at most 2^-20 above |x|).  Selected hubs
// are listed in the tile's own region of the hub list (no global atomics).
// Fluid arrays hold whole tiles, zero past n, so the tail needs no test.
__device__ __forceinline__ unsigned hi_word(unsigned long long b) { return (unsigned)(b >> 32); }
__device__ __forceinline__ unsigned hi_word(unsigned b) { return b; }
// FP32 bits bounding |x| from above, from the upper word of its FP64 bits
// (0 stays 0: a zero word never contributes).
__device__ __forceinline__ unsigned up_hi(unsigned hi, bool nonzero)
{
    if (hi < 0x38100000u) return nonzero ? 0x00800000u : 0u;   // below FLT_MIN: FLT_MIN
    if (hi >= 0x47f00000u) return 0x7f800000u;                 // beyond FLT_MAX: +inf
    return ((hi - 0x38000000u) << 3) + 8u;
}
// FP32 bits bounding |x| from below (truncation to the FP32 grid).
__device__ __forceinline__ unsigned down_hi(unsigned hi)
{
    if (hi < 0x38100000u) return 0u;
    if (hi >= 0x47f00000u) return 0x7f7fffffu;
    return (hi - 0x38000000u) << 3;
}

constexpr int SEL_ROUNDS = TILE / (2 * SEL_THREADS);   // rounds of 64 nodes per warp
constexpr int SEL_PHASE64 = 2;                         // rounds per load phase (FP64 words)
constexpr int SEL_CTAS = 4;                            // resident selection CTAs per SM (FP64 words)
static_assert(SEL_ROUNDS % SEL_PHASE64 == 0, "whole phases per tile");
constexpr int SEL_WORDS = TILE / 32;                   // mask words per tile

template <typename T>
__global__ void __launch_bounds__(SEL_THREADS, sizeof(T) == 8 ? SEL_CTAS : 1)
    k_select(const T *F, int64_t n, unsigned *mask, const unsigned *__restrict__ hubbits,
             const GraphPtrs *__restrict__ gp, const uint64_t *__restrict__ hub_base, unsigned *tile_hub,
             unsigned *tile_cnt, unsigned *tile_diff, float *tile_l1f, unsigned *tile_maxf, unsigned *tile_maxu,
             DevCtl *ctl, int use_cond, cudaGraphConditionalHandle cond, int32_t *sel_ids)
{
    typedef typename FluidWord<T>::U U;
    constexpr bool F64 = sizeof(U) == 8;
    constexpr int R = SEL_ROUNDS;
    constexpr int NW = SEL_THREADS / 32;
    static_assert(TILE <= 65535, "per-tile counts are packed in 16 bits");
    static_assert(R * 2 * SEL_THREADS == TILE, "whole rounds per tile");
    __shared__ float s_fx[NW];
    __shared__ unsigned s_mx[NW], s_mu[NW], s_cnt[NW], s_hub[NW];
    __shared__ unsigned s_hubw[NW][2 * R];     // each warp's selected-hub words
    __shared__ unsigned s_selw[SEL_WORDS];     // selected words in node order (verification output)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tile = blockIdx.x;
    const int64_t t0 = tile * TILE;
    const unsigned long long keep = pol_last();
    // FP64 words: the tile is read in phases of PH rounds (few registers:
    // four CTAs fit on an SM, so that every tile of a graph up to 4.9M pages
    // runs in one wave; 14.6 against 16.3 µs per launch on 4M pages).  FP32
    // words: in one phase, two CTAs per SM (11.5 against 13.0 µs in phases).
    // The first phase's fluid words are requested before the control block is
    // read, so the two round trips overlap (F is readable whatever the block
    // says).
    constexpr int PH = sizeof(U) == 8 ? SEL_PHASE64 : R;
    U fb[2 * PH];
    auto load_phase = [&](int p) {
#pragma unroll
        for (int qq = 0; qq < PH; qq++) {
            const int64_t seg = t0 + (int64_t)(p * PH + qq) * 2 * SEL_THREADS + 64 * warp;
            fb[2 * qq] = ld_word(F + seg + lane, keep);
            fb[2 * qq + 1] = ld_word(F + seg + 32 + lane, keep);
        }
    };
    load_phase(0);
    // control fields: independent L2 loads (not volatile ones, which would
    // be issued one after another)
    const unsigned done0 = __ldcg(&ctl->done);
    const double theta0 = __ldcg(&ctl->theta);
    volatile DevCtl *vc = ctl;
    if (done0) {
        // Nothing left to do: the push that follows must find no work, and a
        // graph while-loop must end here too.
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            vc->push_ready = 0;
            if (use_cond) cudaGraphSetConditional(cond, 0u);
        }
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) vc->npieces = 0;   // the last push is over
    // a selected node holds fluid (the zero words past n never qualify, even
    // at theta = 0)
    U tb = theta_word(theta0, F);
    tb = tb > (U)1 ? tb : (U)1;
    float fx = 0.0f;
    unsigned hmax = 0, nbits = 0, nsel = 0, nhubs = 0;
#pragma unroll 1
    for (int p = 0; p < R / PH; p++) {
    if (p) load_phase(p);
#pragma unroll
    for (int kk = 0; kk < 2 * PH; kk++) {
        const int k = 2 * PH * p + kk;
        const int q = k >> 1, h = k & 1;
        const int wt = 32 * q + 2 * warp + h;              // mask word inside the tile
        const U b = fb[kk] & FluidWord<T>::ABS;
        const unsigned sw = __ballot_sync(FULL, b >= tb);
        const unsigned hw = __ldg(hubbits + tile * SEL_WORDS + wt);
        const unsigned hi = hi_word(b);
        fx = __fadd_ru(fx, __uint_as_float(F64 ? up_hi(hi, b != 0) : hi));
        hmax = hi > hmax ? hi : hmax;
        const unsigned bits = sw & ~hw;   // taken by the push
        const unsigned hs = sw & hw;      // taken by the plan
        if (lane == 0) {
            mask[tile * SEL_WORDS + wt] = bits;
            s_hubw[warp][k] = hs;
            if (sel_ids) s_selw[wt] = sw;
        }
        nbits += __popc(bits);
        nsel += __popc(sw);
        nhubs += __popc(hs);
    }
    }
    // tile partials in a fixed order (warp butterfly, then warp 0 over the warps)
    unsigned mb = F64 ? down_hi(hmax) : hmax, mu = F64 ? up_hi(hmax, hmax != 0) : hmax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fx = __fadd_ru(fx, __shfl_xor_sync(FULL, fx, o));
        const unsigned y = __shfl_xor_sync(FULL, mb, o);
        mb = y > mb ? y : mb;
        const unsigned yu = __shfl_xor_sync(FULL, mu, o);
        mu = yu > mu ? yu : mu;
    }
    if (lane == 0) {
        s_fx[warp] = fx;
        s_mx[warp] = mb;
        s_mu[warp] = mu;
        s_cnt[warp] = nbits | (nsel << 16);
        s_hub[warp] = nhubs;
    }
    __syncthreads();
    // selected hubs: the warps' lists one after another in the tile's region
    if (nhubs) {
        uint64_t pb = hub_base[tile];
        for (int w = 0; w < warp; w++) pb += s_hub[w];
        unsigned *hub_list = gp->hub_list;
        const unsigned lt = (1u << lane) - 1u;
#pragma unroll
        for (int k = 0; k < 2 * R; k++) {
            const unsigned hs = s_hubw[warp][k];
            if ((hs >> lane) & 1u)
                hub_list[pb + __popc(hs & lt)] =
                    (unsigned)(t0 + (int64_t)(k >> 1) * 2 * SEL_THREADS + 64 * warp + 32 * (k & 1) + lane);
            pb += __popc(hs);
        }
    }
    if (warp == 0) {
        float t = lane < NW ? s_fx[lane] : 0.0f;
        unsigned mx = lane < NW ? s_mx[lane] : 0u, mxu = lane < NW ? s_mu[lane] : 0u;
        unsigned c = lane < NW ? s_cnt[lane] : 0u, nh = lane < NW ? s_hub[lane] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t = __fadd_ru(t, __shfl_xor_sync(FULL, t, o));
            const unsigned y = __shfl_xor_sync(FULL, mx, o);
            mx = y > mx ? y : mx;
            const unsigned yu = __shfl_xor_sync(FULL, mxu, o);
            mxu = yu > mxu ? yu : mxu;
            c += __shfl_xor_sync(FULL, c, o);
            nh += __shfl_xor_sync(FULL, nh, o);
        }
        if (lane == 0) {
            tile_l1f[tile] = t;
            tile_maxf[tile] = mx;
            tile_maxu[tile] = mxu;
            tile_cnt[tile] = c & 0xffffu;
            tile_diff[tile] = c >> 16;
            tile_hub[tile] = nh;
        }
    }
    // verification output: ascending ids of the selected nodes of the tile
    if (sel_ids) {
        __shared__ unsigned s_pre[SEL_WORDS];
        static_assert(SEL_WORDS == 32 * 8, "warp 0 scans 8 words per lane");
        if (warp == 0) {
            unsigned c8[8], sum = 0;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                c8[j] = __popc(s_selw[8 * lane + j]);
                sum += c8[j];
            }
            unsigned incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            unsigned run = incl - sum;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                s_pre[8 * lane + j] = run;
                run += c8[j];
            }
        }
        __syncthreads();
        const unsigned lt = (1u << lane) - 1u;
#pragma unroll
        for (int k = 0; k < 2 * R; k++) {
            const int wt = 32 * (k >> 1) + 2 * warp + (k & 1);
            const unsigned sw = s_selw[wt];
            if ((sw >> lane) & 1u)
                sel_ids[t0 + s_pre[wt] + __popc(sw & lt)] = (int32_t)(t0 + 32 * wt + lane);
        }
    }
}

// ----------------------------------------------------------------- plan
// Every CTA sums the tile partials; CTA 0 updates the control block.  Then
// the selected hubs are taken (no push is running, so nobody else writes the
// fluid) and their rows cut into pieces for the push.
//
// Ft is the array the fluid is taken from, Fd the array pushes land in, Hs
// the FP64 array the taken fluid is added to.  A sweep has Ft = Fd (F, or the
// FP32 fluid) and Hs = H (or the cycle accumulator D).  The refinement pass
// (SUB) takes from D, adds to H, and lands in the FP64 fluid F, from which it
// also subtracts the taken amount: F + d P D - D.
template <typename T, bool SUB>
__global__ void __launch_bounds__(SEL_THREADS, 1)
    k_plan(T *Ft, T *Fd, double *Hs, const GraphPtrs *__restrict__ gp, const double *__restrict__ dscale,
           int64_t n, int64_t ntiles, const unsigned *tile_cnt, const unsigned *tile_diff, const float *tile_l1f,
           const unsigned *tile_maxf, const unsigned *tile_maxu, const uint64_t *__restrict__ hub_base,
           const unsigned *__restrict__ tile_hub, DevCtl *ctl, int use_cond, cudaGraphConditionalHandle cond,
           unsigned long long *stats)
{
    typedef typename FluidWord<T>::U U;
    constexpr int NW = SEL_THREADS / 32;
    __shared__ unsigned long long s_red[4][NW];
    __shared__ float s_l1[NW];
    __shared__ unsigned s_go;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Off *__restrict__ rp = gp->rp;
    const unsigned *__restrict__ hub_list = gp->hub_list;
    const uint64_t hub_cap = gp->hub_cap;
    const unsigned long long stream = pol_first(), keep = pol_last();
    // Warps over the tiles, lanes over a tile's selected hubs (32 at a time).
    // The first round of each warp is requested before the control block and
    // the tile partials, so its three dependent loads (count, id, node data)
    // overlap the reduction; every index is clamped to its array, so a list
    // left by an earlier sweep (the selection of this one returned early) is
    // read harmlessly and then not used.
    // control fields, requested at once (volatile loads would be issued one
    // after another); only the selection, the previous plan and the previous
    // push wrote them, all finished
    const unsigned done0 = __ldcg(&ctl->done);
    int c_inf = 0;
    unsigned long long c_sweep = 0, c_max_sweeps = 0, c_links = 0, c_hot = 0, c_pushes = 0, c_diff = 0;
    double c_stop = 0.0, c_d = 0.0, c_tf = 0.0, c_cap = 0.0;
    if (threadIdx.x == 0) {
        c_inf = __ldcg(&ctl->inf_norm);
        c_sweep = __ldcg(&ctl->sweep);
        c_max_sweeps = __ldcg(&ctl->max_sweeps);
        c_stop = __ldcg(&ctl->sweep_stop);
        if (blockIdx.x == 0) {
            c_links = __ldcg(&ctl->sweep_links);
            c_hot = __ldcg(&ctl->sweep_hot);
            c_pushes = __ldcg(&ctl->edge_pushes);
            c_diff = __ldcg(&ctl->diffusions);
            c_d = __ldcg(&ctl->d);
            c_tf = __ldcg(&ctl->theta_factor);
            c_cap = __ldcg(&ctl->inf_cap);
        }
    }
    const int64_t gw = ((int64_t)blockIdx.x * SEL_THREADS + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * (SEL_THREADS / 32);
    struct HubTake {
        unsigned i;
        U fbits;
        Off r0, r1;
        unsigned long long hb;
        double ds;
    };
    auto load_hub = [&](int64_t tw, unsigned h, unsigned nt, HubTake &t) -> bool {
        if (h >= nt) return false;
        const uint64_t q = __ldg(hub_base + tw) + h;
        if (q >= hub_cap) return false;
        t.i = hub_list[q];
        if (t.i >= (uint64_t)n) return false;
        t.fbits = ld_word(Ft + t.i, keep);
        t.r0 = ldnc_u32(rp + t.i, stream);
        t.r1 = ldnc_u32(rp + t.i + 1, stream);
        t.hb = ld_b64(Hs + t.i, stream);
        t.ds = ldnc_f64(dscale + t.i, stream);
        return true;
    };
    unsigned nt0 = 0;
    HubTake first = {};
    bool have_first = false;
    if (gw < ntiles) {
        nt0 = __ldg(tile_hub + gw);
        have_first = load_hub(gw, lane, nt0, first);
    }
    volatile DevCtl *vc = ctl;
    if (done0) return;   // the selection has already closed the loop
    // fixed order: thread-strided tiles, xor butterfly, warps in order; every
    // partial rounded upward, so every CTA gets the same upper bound
    float sfx = 0.0f;
    unsigned long long sd = 0, sc = 0, mx = 0, mu = 0;
    for (int64_t k = threadIdx.x; k < ntiles; k += SEL_THREADS) {
        sfx = __fadd_ru(sfx, __ldg(tile_l1f + k));
        sd += __ldg(tile_diff + k);
        sc += __ldg(tile_cnt + k);
        const unsigned long long m = __ldg(tile_maxf + k), mm = __ldg(tile_maxu + k);
        mx = m > mx ? m : mx;
        mu = mm > mu ? mm : mu;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sfx = __fadd_ru(sfx, __shfl_xor_sync(FULL, sfx, o));
        sd += __shfl_xor_sync(FULL, sd, o);
        sc += __shfl_xor_sync(FULL, sc, o);
        const unsigned long long y = __shfl_xor_sync(FULL, mx, o);
        mx = y > mx ? y : mx;
        const unsigned long long yu = __shfl_xor_sync(FULL, mu, o);
        mu = yu > mu ? yu : mu;
    }
    if (lane == 0) {
        s_l1[warp] = sfx;
        s_red[0][warp] = sd;
        s_red[1][warp] = sc;
        s_red[2][warp] = mx;
        s_red[3][warp] = mu;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sfx = s_l1[0];
        sd = sc = mx = mu = 0;
        for (int w = 0; w < NW; w++) {
            if (w) sfx = __fadd_ru(sfx, s_l1[w]);
            sd += s_red[0][w];
            sc += s_red[1][w];
            mx = s_red[2][w] > mx ? s_red[2][w] : mx;
            mu = s_red[3][w] > mu ? s_red[3][w] : mu;
        }
        const double sa = (double)sfx;
        const bool inf_norm = c_inf != 0;
        const unsigned long long sweep = c_sweep;
        unsigned done = 0;
        // every |F_i| and every partial sum was rounded up: an upper bound of
        // |F_t|_1 (or of max |F_i| in the infinity-norm mode)
        if ((inf_norm ? (double)__uint_as_float((unsigned)mu) : sa) <= c_stop) done = 1;
        else if (sweep >= c_max_sweeps) done = 2;
        s_go = done == 0;
        if (blockIdx.x == 0) {
            // fold the links of the previous push into the totals
            const unsigned long long links = c_links;
            vc->edge_pushes = c_pushes + links;
            if (stats && sweep >= 1 && sweep <= (unsigned long long)STAT_CAP) {
                stats[3 * (sweep - 1)] = links;
                stats[3 * (sweep - 1) + 2] = c_hot;
            }
            vc->sweep_links = 0;
            vc->sweep_hot = 0;
            vc->l1 = sa;
            // hot_scale >= V / 8, V a bound on what one sweep adds into one
            // page (the push keeps 8 hot_scale of headroom per page).  Plain
            // solve: a unit of fluid can be taken again after each hop inside
            // one sweep, keeping d of it per hop, so the fluid taken in one
            // sweep is at most |F|_1 / (1 - d) and V = d |F|_1 / (1 - d).
            // Reverse graph (infinity norm): a page j receives d f_i P[i][j]
            // from the pages i that link to it in the reverse graph, and the
            // column sums of P are at most 1, so no page ever holds more than
            // max |F| / (1 - d) during the sweep and V = d max |F| / (1 - d).
            // (The refinement pass takes each node once: V = d |D|_1 < sa.)
            {
                const double hop = c_d / (1.0 - c_d);
                const double base = inf_norm ? (double)__uint_as_float((unsigned)mu) : sa;
                vc->hot_scale = base * fmax(inf_norm ? 8.0 : 1.0, 0.125 * hop);
            }
            if (!done) {
                vc->diffusions = c_diff + sd;
                vc->nent = sc;
                if (stats && sweep < (unsigned long long)STAT_CAP) stats[3 * sweep + 1] = sc;
                double th = c_tf * sa / (double)n;
                // A sweep that took nothing leaves F unchanged; the largest |F_i|
                // passes the DI-argmax test exactly, so never ask for more than
                // that (this covers a rounded average above several equal fluids).
                const double fmax = (double)__uint_as_float((unsigned)mx);
                if (sd == 0 && fmax < th) th = fmax;
                // infinity-norm mode: theta <= inf_cap max |F_i| with inf_cap + d < 1,
                // so max |F| shrinks by at least inf_cap + d per sweep
                if (inf_norm && c_cap * fmax < th) th = c_cap * fmax;
                vc->theta = th;
            }
            vc->push_ready = done ? 0u : 1u;
            vc->done = done;   // read by the next kernels only (kernel order makes it visible)
            if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
        }
    }
    __syncthreads();
    if (!s_go) return;
    // take the selected hubs (no push is running: F is quiescent), one lane
    // each, and cut their rows into pieces; one piece-queue reservation per
    // warp and round
    Off *pc_row = gp->pc_row, *pc_len = gp->pc_len;
    double *pc_val = gp->pc_val;
    const Off piece = gp->piece;
    for (int64_t tw = gw; tw < ntiles; tw += nwarps) {
        const unsigned nt = tw == gw ? nt0 : __ldg(tile_hub + tw);
        for (unsigned h0 = 0; h0 < nt; h0 += 32) {
            HubTake t = {};
            const bool mine = (tw == gw && h0 == 0) ? have_first : load_hub(tw, h0 + lane, nt, t);
            if (tw == gw && h0 == 0) t = first;
            unsigned np = 0;
            Off deg = 0;
            double v = 0.0;
            if (mine) {
                const double f = (double)word_val(t.fbits);
                st_b64(Hs + t.i, (unsigned long long)__double_as_longlong(__longlong_as_double((long long)t.hb) + f),
                       stream);
                st_word(Ft + t.i, (U)0, keep);
                if (SUB) red_add_f64(reinterpret_cast<double *>(Fd) + t.i, -f, keep);
                deg = t.r1 - t.r0;
                v = f * t.ds;
                np = (deg + piece - 1) / piece;
            }
            unsigned incl = np;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned wtot = __shfl_sync(FULL, incl, 31);
            unsigned long long wbase = 0;
            if (lane == 31 && wtot) wbase = atomicAdd((unsigned long long *)&ctl->npieces, (unsigned long long)wtot);
            wbase = __shfl_sync(FULL, wbase, 31);
            // the warp's pieces written 32 at a time, one per lane (a hub of
            // 50,000 links has about a hundred: one lane writing them all was
            // the plan's longest chain)
            const unsigned excl = incl - np;
            for (unsigned b0 = 0; b0 < wtot; b0 += 32) {
                const unsigned e = b0 + lane;
                const unsigned eq = e < wtot ? e : wtot - 1;
                int h = 0;   // the lane whose hub holds piece eq
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (__shfl_sync(FULL, excl, h + step) <= eq) h += step;
                const Off r0 = __shfl_sync(FULL, t.r0, h), dh = __shfl_sync(FULL, deg, h);
                const double vh = __shfl_sync(FULL, v, h);
                const Off o = (eq - __shfl_sync(FULL, excl, h)) * piece;
                if (e < wtot) {
                    pc_row[wbase + e] = r0 + o;
                    pc_len[wbase + e] = dh - o < piece ? dh - o : piece;
                    pc_val[wbase + e] = vh;
                }
            }
        }
    }
}

// ----------------------------------------------------------------- push
__device__ __forceinline__ unsigned long long atom_exch_word(double *a, unsigned long long pol)
{
    unsigned long long old;
    asm volatile("atom.global.exch.L2::cache_hint.b64 %0, [%1], %2, %3;"
                 : "=l"(old)
                 : "l"(a), "l"(0ull), "l"(pol)
                 : "memory");
    return old;
}
__device__ __forceinline__ unsigned atom_exch_word(float *a, unsigned long long pol)
{
    unsigned old;
    asm volatile("atom.global.exch.L2::cache_hint.b32 %0, [%1], %2, %3;"
                 : "=r"(old)
                 : "l"(a), "r"(0u), "l"(pol)
                 : "memory");
    return old;
}
__device__ __forceinline__ void red_add(double *a, double v, unsigned long long pol) { red_add_f64(a, v, pol); }
__device__ __forceinline__ void red_add(float *a, float v, unsigned long long pol)
{
    asm volatile("red.global.add.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ float ldnc_f32(const float *a, unsigned long long pol)
{
    unsigned r;
    asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(r) : "l"(a), "l"(pol));
    return __uint_as_float(r);
}

// Per-link value of a weighted push: the node's share times the link weight
// (FP64 weights for FP64 fluid, the FP32 copy for FP32 fluid).
__device__ __forceinline__ double link_weight(const double *w, const float *, Off link, unsigned long long pol)
{
    return ldnc_f64(w + link, pol);
}
__device__ __forceinline__ float link_weight(const float *w32, Off link, unsigned long long pol)
{
    return ldnc_f32(w32 + link, pol);
}

// Shared-memory accumulation for the hot pages: FP64 contributions as 64-bit
// fixed point (native integer atomics; the shared FP64 add is not native),
// FP32 contributions with the native shared FP32 add.
// Returns false (nothing added) for a contribution too large for the fixed
// point, |v| 2^hot_shift >= 2^59; the caller then adds it in global memory.
// (hot_scale bounds every sweep so that this does not happen; the check keeps
// a contribution from ever being converted out of range.)
__device__ __forceinline__ bool hot_add(unsigned long long *s_hot, int slot, double v, int hot_shift)
{
    const int ex = (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ffu);
    if (ex == 0) return v == 0.0;   // a subnormal contribution goes to global memory as it is
    if (ex - 1023 + hot_shift > 58) return false;
    atomicAdd(s_hot + slot, (unsigned long long)to_fixed64(v, hot_shift));
    return true;
}
__device__ __forceinline__ bool hot_add(unsigned long long *s_hot, int slot, float v, int)
{
    atomicAdd(reinterpret_cast<float *>(s_hot) + slot, v);
    return true;
}
// a 2^-sh as the nearest double (ties to even), the same value as
// scalbn((double)a, -sh), built with integer instructions: the FP64 pipe of
// this part is narrow, and every CTA converts up to HOT_K sums at its end.
// |a| < 2^62; a result outside the normal range takes the FP64 route.
__device__ __forceinline__ double fixed64_to_double(long long a, int sh)
{
    if (a == 0) return 0.0;
    const unsigned long long sgn = a < 0 ? 0x8000000000000000ull : 0ull;
    const unsigned long long u = a < 0 ? (unsigned long long)(-a) : (unsigned long long)a;
    int msb = 63 - __clzll((long long)u);
    unsigned long long mant;
    if (msb <= 52) {
        mant = u << (52 - msb);
    } else {
        const int s = msb - 52;
        const unsigned long long rem = u & ((1ull << s) - 1ull), half = 1ull << (s - 1);
        mant = u >> s;
        if (rem > half || (rem == half && (mant & 1ull))) mant++;
        if (mant >> 53) {
            mant >>= 1;
            msb++;
        }
    }
    const int be = msb - sh + 1023;
    if (be < 1 || be > 2046) return scalbn((double)a, -sh);
    return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | (mant & 0x000fffffffffffffull)));
}
__device__ __forceinline__ void hot_flush(double *Fd, const int32_t *hot_node, const unsigned long long *s_hot,
                                          int k, int hot_shift, unsigned long long keep)
{
    const long long a = (long long)s_hot[k];
    if (a != 0) red_add_f64(Fd + __ldg(hot_node + k), fixed64_to_double(a, hot_shift), keep);
}
__device__ __forceinline__ void hot_flush(float *Fd, const int32_t *hot_node, const unsigned long long *s_hot,
                                          int k, int, unsigned long long keep)
{
    const float a = reinterpret_cast<const float *>(s_hot)[k];
    if (a != 0.0f) red_add(Fd + __ldg(hot_node + k), a, keep);
}

// Scatter helper: 4 x 32 links in flight per warp.  lane_link(e) gives the
// link and the value for the warp's e-th link (e < total).  Targets tagged
// in the push copy of the links (hot pages) are added in shared memory.
template <typename T, bool WEIGHTED, typename LinkOf>
__device__ __forceinline__ void scatter_links(unsigned total, LinkOf lane_link, const int32_t *pcol,
                                              const double *w, const float *w32, T *Fd,
                                              unsigned long long *s_hot, const int32_t *hot_node, int hot_shift,
                                              unsigned long long keep, unsigned long long stream, unsigned &hotc)
{
    const int lane = threadIdx.x & 31;
    for (unsigned base = 0; base < total; base += 128) {
        int32_t c[4];
        T v[4];
        bool ok[4];
#pragma unroll
        for (int g = 0; g < 4; g++) {
            const unsigned e = base + (unsigned)(g * 32 + lane);
            Off link;
            T vj;
            lane_link(e < total ? e : total - 1, link, vj);
            ok[g] = e < total;
            c[g] = 0;
            v[g] = vj;
            if (ok[g]) {
                c[g] = ldnc_s32(pcol + link, stream);
                if (WEIGHTED) {
                    if constexpr (sizeof(T) == 8) v[g] = vj * link_weight(w, w32, link, stream);
                    else v[g] = vj * link_weight(w32, link, stream);
                }
            }
        }
#pragma unroll
        for (int g = 0; g < 4; g++) {
            if (!ok[g]) continue;
            if (c[g] >= 0) {
                red_add(Fd + c[g], v[g], keep);
            } else {
                hotc++;
                if (!hot_add(s_hot, c[g] & 0x7fffffff, v[g], hot_shift))
                    red_add(Fd + __ldg(hot_node + (c[g] & 0x7fffffff)), v[g], keep);
            }
        }
    }
}

// Asynchronous 16-byte (and one 4-byte) copies from global to shared memory,
// with an L2 eviction priority; completion is waited for per thread.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, unsigned long long pol)
{
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Per-warp staging area of the push (dynamic shared memory): the fluid words,
// d/W_j and the 129 row pointers of the warp's next unit.
constexpr int STAGE_RP = 132;   // row pointers per warp (129 used; rows of 16 bytes)
template <typename T>
__host__ __device__ constexpr bool push_staged()
{
    return sizeof(T) == 4;
}
template <typename T>
__host__ __device__ constexpr int push_stage_bytes()
{
    return push_staged<T>() ? (PUSH_THREADS / 32) * (128 * (int)sizeof(T) + 128 * 8 + STAGE_RP * 4) : 0;
}

// Warp-centric take and push.  Work unit u < nunits: the 128 nodes
// [128u, 128u + 128), lane l owning nodes 128u + 4l .. 4l + 3 and their bits
// of mask words 4u .. 4u + 3; u >= nunits: hub piece u - nunits.
// FP64 fluid: the take is an atomic exchange of F_i issued with the unit's
// row pointer and d/W_j loads, so it also picks up fluid that reached the node
// earlier in the same sweep.  FP32 fluid: while a unit's links are pushed, the
// warp's next unit is already on its way into shared memory (fluid words,
// d/W_j, row pointers, by cp.async), so its take waits for no global round
// trip: a selected node's fluid f is read from that snapshot and taken by
// adding -f to F_i (fluid that arrived since stays for a later sweep, a valid
// diffusion order).  (Measured on the 4M-page graph: the snapshot take costs
// 2-3 more sweeps per solve in both precisions; it saves 4.6% of each FP32
// push and nothing of an FP64 one, whose atomic traffic bounds it.)  Either
// way the history gets the taken fluid by a reduction.  The taken nodes'
// links are dealt to the lanes 128 at a time; a link finds its node by a
// binary search over the unit's link offsets in shared memory.  Ft / Fd / Hs
// / SUB as for k_plan.  At most 64 registers: four CTAs of 256 threads per SM.
template <typename T, bool WEIGHTED, bool SUB>
__global__ void __launch_bounds__(PUSH_THREADS, 4)
    k_push(T *Ft, T *Fd, double *Hs, const GraphPtrs *__restrict__ gp, const double *__restrict__ dscale,
           const unsigned *__restrict__ mask, int64_t ngroups, int64_t n, const int32_t *__restrict__ hot_node,
           DevCtl *ctl)
{
    typedef typename FluidWord<T>::U U;
    const Off *__restrict__ rp = gp->rp;
    const Off *__restrict__ pc_row = gp->pc_row;
    const Off *__restrict__ pc_len = gp->pc_len;
    const double *__restrict__ pc_val = gp->pc_val;
    const int32_t *__restrict__ pcol = gp->pcol;
    const double *__restrict__ w = gp->w;
    const float *__restrict__ w32 = gp->w32;
    const int nhot = gp->nhot;
    constexpr int Q = 4;
    constexpr int NWP = PUSH_THREADS / 32;
    __shared__ unsigned long long s_links[NWP];
    __shared__ unsigned s_hotc[NWP];
    __shared__ unsigned long long s_hot[HOT_K];   // FP64: fixed point, units of 2^-hot_shift; FP32: floats
    // per warp, the current unit's 128 nodes: link offset of each node inside
    // the unit's link list, its first link, its per-link value
    __shared__ unsigned s_start[NWP][32 * 4];
    __shared__ Off s_row[NWP][32 * 4];
    __shared__ T s_val[NWP][32 * 4];
    extern __shared__ __align__(16) unsigned char s_stage[];
    constexpr bool STAGED = push_staged<T>();
    const int wq = threadIdx.x >> 5;
    U *const g_f = reinterpret_cast<U *>(s_stage) + wq * 128;
    double *const g_ds = reinterpret_cast<double *>(s_stage + NWP * 128 * sizeof(U)) + wq * 128;
    Off *const g_rp = reinterpret_cast<Off *>(s_stage + NWP * 128 * (sizeof(U) + 8)) + wq * STAGE_RP;
    // control fields, requested at once (the plan that wrote them is over)
    const unsigned ready = __ldcg(&ctl->push_ready);
    const double hot_scale = __ldcg(&ctl->hot_scale);
    const unsigned long long npieces0 = __ldcg(&ctl->npieces);
    volatile DevCtl *vc = ctl;
    if (!ready) return;
    // 8 hot_scale bounds what this sweep adds into one page, for every d
    // (k_plan derives it): with 2^(e-1) <= hot_scale < 2^e, units of
    // 2^(e - 58) keep every slot below 2^61.
    int e = 0;
    frexp(hot_scale, &e);
    const int hot_shift = 58 - e;
    for (int k = threadIdx.x; k < nhot; k += PUSH_THREADS) s_hot[k] = 0ull;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        vc->sweep = vc->sweep + 1;    // (the plan reads it; it is stable until here)
    }
    // unit and piece counts stay below 2^32 (n / 128 units; pieces <= links)
    const unsigned npc = (unsigned)npieces0;
    const unsigned long long keep = pol_last(), stream = pol_first();
    const int lane = threadIdx.x & 31;
    const unsigned nunits = (unsigned)(ngroups / Q);
    const unsigned wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned nw = (gridDim.x * blockDim.x) >> 5;
    unsigned long long links = 0;
    unsigned hotc = 0;   // this lane's links into hot pages
    // a unit holding a page below n is staged (row pointers are padded past
    // rp[n] to a whole unit; fluid and d/W_j arrays hold whole tiles)
    auto stage = [&](unsigned un) {
        const size_t i0 = (size_t)un * 128;
        if (!STAGED || un >= nunits || (int64_t)i0 >= n) return;
        constexpr int FW = 16 / (int)sizeof(U);   // fluid words per 16-byte copy
#pragma unroll
        for (int c = lane; c < 128 / FW; c += 32)
            cp_async16(g_f + c * FW, reinterpret_cast<const U *>(Ft) + i0 + c * FW, keep);
#pragma unroll
        for (int c = lane; c < 64; c += 32) cp_async16(g_ds + 2 * c, dscale + i0 + 2 * c, stream);
        cp_async16(g_rp + 4 * lane, rp + i0 + 4 * lane, stream);
        if (lane == 0) cp_async4(g_rp + 128, rp + i0 + 128);
        cp_async_commit();
    };
    // the mask word of the warp's next unit is loaded one unit ahead
    unsigned mw_next = wid < nunits ? ldnc_u32(mask + (size_t)wid * Q + (lane >> 3), stream) : 0u;
    if (STAGED) stage(wid);
    for (unsigned u = wid; u < nunits + npc; u += nw) {
        if (u < nunits) {
            const unsigned mw = mw_next;
            {
                const unsigned un = u + nw;
                mw_next = un < nunits ? ldnc_u32(mask + (size_t)un * Q + (lane >> 3), stream) : 0u;
            }
            const unsigned bits = (mw >> (Q * (lane & 7))) & ((1u << Q) - 1u);
            const unsigned long long i0 = (unsigned long long)u * (32 * Q) + (unsigned long long)lane * Q;
            if (STAGED) {
                cp_async_wait_all();
                __syncwarp();
            }
            Off r[Q + 1];
            T val[Q];
            unsigned c1 = 0, c2 = 0, c3 = 0, tot = 0;
            const bool any = __any_sync(FULL, bits) != 0;
            if (!STAGED && !any) continue;
            if (bits) {
                unsigned dg[Q];
                if (STAGED) {
#pragma unroll
                    for (int k = 0; k <= Q; k++) r[k] = g_rp[Q * lane + k];
#pragma unroll
                    for (int k = 0; k < Q; k++) {
                        dg[k] = 0;
                        val[k] = (T)0;
                        if (!((bits >> k) & 1u)) continue;
                        // take (Eq. defF): the fluid of the snapshot, withdrawn
                        // by a reduction and added to the history
                        const T fw = word_val(g_f[Q * lane + k]);
                        const double f = (double)fw;
                        red_add(Ft + i0 + k, -fw, keep);
                        red_add_f64(Hs + i0 + k, f, stream);
                        if (SUB) red_add_f64(reinterpret_cast<double *>(Fd) + i0 + k, -f, keep);
                        dg[k] = r[k + 1] - r[k];
                        val[k] = (T)(f * g_ds[Q * lane + k]);
                    }
                } else {
                    U fb[Q];
                    double ds[Q];
#pragma unroll
                    for (int k = 0; k < Q; k++) {
                        fb[k] = 0;
                        ds[k] = 0.0;
                        if (!((bits >> k) & 1u)) continue;
                        // take (Eq. defF): whatever fluid the node holds now
                        fb[k] = atom_exch_word(Ft + i0 + k, keep);
                        ds[k] = ldnc_f64(dscale + i0 + k, stream);
                    }
                    {
                        // i0 is a multiple of 4: one 16-byte load for the first four
                        const uint4 r4 = ldnc_u32x4(rp + i0, stream);
                        r[0] = r4.x;
                        r[1] = r4.y;
                        r[2] = r4.z;
                        r[3] = r4.w;
                        r[4] = ldnc_u32(rp + i0 + Q, stream);
                    }
#pragma unroll
                    for (int k = 0; k < Q; k++) {
                        dg[k] = 0;
                        val[k] = (T)0;
                        if (!((bits >> k) & 1u)) continue;
                        const double f = (double)word_val(fb[k]);
                        red_add_f64(Hs + i0 + k, f, stream);
                        if (SUB) red_add_f64(reinterpret_cast<double *>(Fd) + i0 + k, -f, keep);
                        dg[k] = r[k + 1] - r[k];
                        val[k] = (T)(f * ds[k]);
                    }
                }
                c1 = dg[0];
                c2 = c1 + dg[1];
                c3 = c2 + dg[2];
                tot = c3 + dg[3];
            } else {
#pragma unroll
                for (int k = 0; k <= Q; k++) r[k] = 0;
#pragma unroll
                for (int k = 0; k < Q; k++) val[k] = (T)0;
            }
            if (STAGED) {
                // the staging area is free: the next unit's copies go out now
                // and land while this unit's links are pushed
                __syncwarp();
                stage(u + nw);
                if (!any) continue;
            }
            unsigned incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned total = __shfl_sync(FULL, incl, 31);
            const unsigned excl = incl - tot;
            links += total;
            // park the unit's nodes in shared memory: a link then finds its
            // node by a binary search over the 128 starts (shared loads, the
            // lanes of a batch mostly read the same entries)
            __syncwarp();
            s_start[wq][Q * lane] = excl;
            s_start[wq][Q * lane + 1] = excl + c1;
            s_start[wq][Q * lane + 2] = excl + c2;
            s_start[wq][Q * lane + 3] = excl + c3;
#pragma unroll
            for (int k = 0; k < Q; k++) {
                s_row[wq][Q * lane + k] = r[k];
                s_val[wq][Q * lane + k] = val[k];
            }
            __syncwarp();
            auto lane_link = [&](unsigned e, Off &link, T &vj) {
                int k = 0;
#pragma unroll
                for (int step = 64; step > 0; step >>= 1)
                    if (s_start[wq][k + step] <= e) k += step;
                link = s_row[wq][k] + (e - s_start[wq][k]);
                vj = s_val[wq][k];
            };
            scatter_links<T, WEIGHTED>(total, lane_link, pcol, w, w32, Fd, s_hot, hot_node, hot_shift, keep, stream,
                                       hotc);
        } else {
            const unsigned p = u - nunits;
            const Off row = ldnc_u32(pc_row + p, stream), len = ldnc_u32(pc_len + p, stream);
            const T pv = (T)ldnc_f64(pc_val + p, stream);
            links += len;
            auto piece_link = [&](unsigned e, Off &link, T &vj) {
                link = row + e;
                vj = pv;
            };
            scatter_links<T, WEIGHTED>(len, piece_link, pcol, w, w32, Fd, s_hot, hot_node, hot_shift, keep, stream,
                                       hotc);
        }
    }
    if (STAGED) cp_async_wait_all();   // (nothing is left in flight at exit)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hotc += __shfl_xor_sync(FULL, hotc, o);
    if (lane == 0) {
        s_links[threadIdx.x >> 5] = links;
        s_hotc[threadIdx.x >> 5] = hotc;
    }
    __syncthreads();
    // one global add per hot page this CTA touched
    for (int k = threadIdx.x; k < nhot; k += PUSH_THREADS) hot_flush(Fd, hot_node, s_hot, k, hot_shift, keep);
    if (threadIdx.x == 0) {
        unsigned long long t = 0, th = 0;
        for (int q = 0; q < NWP; q++) {
            t += s_links[q];
            th += s_hotc[q];
        }
        if (t) atomicAdd((unsigned long long *)&ctl->sweep_links, t);
        if (th) atomicAdd((unsigned long long *)&ctl->sweep_hot, th);
    }
}

// Static hub bit mask: node i has more than hub_deg out-links.
// One node per thread, one word per warp (ballot); the grid covers whole
// words.  tile_hubs[t] counts the hub nodes of selection tile t.
__global__ void k_hubbits(const Off *rp, int64_t n, int64_t words, Off hub_deg, unsigned *hubbits,
                          unsigned *tile_hubs, unsigned long long *count)
{
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words * 32;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool hub = i < n && rp[i + 1] - rp[i] > hub_deg;
        const unsigned word = __ballot_sync(0xffffffffu, hub);
        if ((threadIdx.x & 31) == 0) {
            hubbits[i >> 5] = word;
            c += __popc(word);
            if (word) atomicAdd(tile_hubs + i / TILE, (unsigned)__popc(word));
        }
    }
    if (c) atomicAdd(count, c);
}

// ------------------------------------------------------------- host side
static unsigned grid_for(int64_t work, int threads)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (1 << 20)) b = 1 << 20;
    return (unsigned)b;
}

// Sweep variants: FP64 fluid, FP32 fluid, FP64 refinement pass.
enum SweepKind { SW_F64 = 0, SW_F32 = 1, SW_REFINE = 2 };

static int push_grid(int device, SweepKind kind, bool weighted)
{
    static int cached[3][2];
    int &c = cached[kind][weighted ? 1 : 0];
    if (!c) {
        int per_sm = 0;
        const void *fn = nullptr;
        if (kind == SW_F32) fn = weighted ? (const void *)k_push<float, true, false> : (const void *)k_push<float, false, false>;
        else if (kind == SW_REFINE) fn = weighted ? (const void *)k_push<double, true, true> : (const void *)k_push<double, false, true>;
        else fn = weighted ? (const void *)k_push<double, true, false> : (const void *)k_push<double, false, false>;
        const int smem = kind == SW_F32 ? push_stage_bytes<float>() : push_stage_bytes<double>();
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PUSH_THREADS, smem);
        if (per_sm < 1) per_sm = 1;
        c = per_sm * sm_count(device);
    }
    return c;
}

// Buffers derived from the graph's degrees: static hub bit mask, hub list
// and hub-piece queue capacities.  Called at creation and after updates.
di_status state_prepare_graph(di_graph_s *g, di_state_s *st, cudaStream_t s)
{
    DI_TRY(graph_build_push_targets(g, s));
    const int64_t words = st->ntiles * TILE / 32;
    Temps t(s);
    unsigned long long *cnt;
    unsigned *tile_hubs;
    DI_TRY(t.get(&cnt, 1));
    DI_TRY(t.get(&tile_hubs, st->ntiles));
    DI_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
    DI_CUDA(cudaMemsetAsync(tile_hubs, 0, sizeof(unsigned) * st->ntiles, s));
    k_hubbits<<<grid_for(words * 32, 256), 256, 0, s>>>(static_cast<const Off *>(g->rp), g->n, words,
                                                   (Off)st->hub_deg, st->hubbits, tile_hubs, cnt);
    count_launches(1);
    // each tile lists its selected hubs in a region of its own
    DI_TRY(scan_exclusive<uint32_t>(tile_hubs, st->hub_base, st->ntiles, nullptr, s));
    DI_CUDA(cudaGetLastError());
    unsigned long long nh = 0;
    DI_CUDA(cudaMemcpyAsync(&nh, cnt, sizeof(nh), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    if ((int64_t)nh + 1 > st->nhub_cap) {
        dfree(st->hub_list, s);
        st->hub_list = nullptr;
        DI_TRY(dalloc_t(&st->hub_list, nh + 1, s));
        st->nhub_cap = (int64_t)nh + 1;
    }
    const int64_t need = g->nnz / st->piece + (int64_t)nh + 2;
    if (need > st->max_items) {
        dfree(st->pc_row, s);
        dfree(st->pc_len, s);
        dfree(st->pc_val, s);
        st->pc_row = st->pc_len = nullptr;
        st->pc_val = nullptr;
        DI_TRY(dalloc_t(&st->pc_row, need, s));
        DI_TRY(dalloc_t(&st->pc_len, need, s));
        DI_TRY(dalloc_t(&st->pc_val, need, s));
        st->max_items = need;
    }
    return DI_OK;
}

// Apply the degree-bin threshold and piece size of a solve: the hub bits and
// the piece queue follow them, and the captured sweep loops are rebuilt.
di_status state_set_bins(di_graph_s *g, di_state_s *st, int hub_deg, int piece, cudaStream_t s)
{
    if (hub_deg == st->hub_deg && piece == st->piece) return DI_OK;
    st->hub_deg = hub_deg;
    st->piece = piece;
    return state_prepare_graph(g, st, s);
}

// Write the current positions of the moving buffers into the state's block.
di_status state_sync_ptrs(di_graph_s *g, di_state_s *st, cudaStream_t s)
{
    GraphPtrs *h = st->host_gp;
    // the push reads four row pointers at a time with a 16-byte load
    if (reinterpret_cast<uintptr_t>(g->rp) % 16 != 0) return DI_ERR_CUDA;
    h->rp = static_cast<const Off *>(g->rp);
    h->pcol = g->pcol;
    h->w = g->w;
    h->w32 = g->w32;
    h->hub_list = st->hub_list;
    h->hub_cap = (uint64_t)st->nhub_cap;
    h->pc_row = st->pc_row;
    h->pc_len = st->pc_len;
    h->pc_val = st->pc_val;
    h->nhot = g->nhot;
    h->piece = (Off)st->piece;
    DI_CUDA(cudaMemcpyAsync(st->gp, h, sizeof(GraphPtrs), cudaMemcpyHostToDevice, s));
    return DI_OK;
}

di_status state_alloc(di_state_s *st, cudaStream_t s)
{
    di_graph_s *g = st->g;
    const int64_t n = g->n;
    st->ntiles = (n + TILE - 1) / TILE;
    const int64_t slots = st->ntiles * TILE;
    DI_TRY(dalloc_t(&st->F, slots, s));
    DI_TRY(dalloc_t(&st->H, slots, s));
    DI_TRY(dalloc_t(&st->dscale, slots, s));   // whole tiles: the push stages whole units
    DI_CUDA(cudaMemsetAsync(st->dscale, 0, sizeof(double) * slots, s));
    DI_TRY(dalloc_t(&st->dtab, DTAB_MAX + 1, s));
    DI_TRY(dalloc_t(&st->mask, slots / 32, s));
    DI_TRY(dalloc_t(&st->hubbits, slots / 32, s));
    DI_TRY(dalloc_t(&st->tile_cnt, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_hub, st->ntiles, s));
    DI_TRY(dalloc_t(&st->hub_base, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_diff, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_l1f, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_maxf, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_maxu, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_max, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_l1, st->ntiles, s));
    DI_TRY(dalloc_t(&st->tile_l, st->ntiles, s));
    DI_TRY(dalloc_t(&st->ctl, 1, s));
    DI_TRY(dalloc_t(&st->gp, 1, s));
    DI_TRY(dalloc_t(&st->stats, 3 * STAT_CAP, s));
    DI_CUDA(cudaMemsetAsync(st->ctl, 0, sizeof(DevCtl), s));
    DI_CUDA(cudaMemsetAsync(st->mask, 0, sizeof(unsigned) * (slots / 32), s));
    DI_CUDA(cudaMemsetAsync(st->F, 0, sizeof(double) * slots, s));
    DI_CUDA(cudaMemsetAsync(st->H, 0, sizeof(double) * slots, s));
    DI_TRY(state_prepare_graph(g, st, s));
    DI_CUDA(cudaMallocHost(reinterpret_cast<void **>(&st->host_ctl), sizeof(DevCtl)));
    memset(st->host_ctl, 0, sizeof(DevCtl));
    DI_CUDA(cudaMallocHost(reinterpret_cast<void **>(&st->host_gp), sizeof(GraphPtrs)));
    memset(st->host_gp, 0, sizeof(GraphPtrs));
    DI_CUDA(cudaEventCreate(&st->ev0));
    DI_CUDA(cudaEventCreate(&st->ev1));
    DI_CUDA(cudaStreamSynchronize(s));
    return DI_OK;
}

di_status state_free(di_state_s *st)
{
    cudaStream_t s = 0;
    if (st->gexec) cudaGraphExecDestroy(st->gexec);
    if (st->gexec32) cudaGraphExecDestroy(st->gexec32);
    if (st->gstream) cudaStreamDestroy(st->gstream);
    void *bufs[] = {st->F, st->H, st->dscale, st->dtab, st->tile_hub, st->hub_base, st->mask, st->hubbits, st->hub_list, st->pc_row, st->pc_len,
                    st->pc_val, st->tile_cnt, st->tile_diff, st->tile_l1f, st->tile_maxf, st->tile_l1,
                    st->tile_l, st->ctl, st->stats, st->F32, st->D, st->rctl, st->tile_maxu, st->tile_max,
                    st->gp};
    for (void *p : bufs) dfree(p, s);
    if (st->host_ctl) cudaFreeHost(st->host_ctl);
    if (st->host_gp) cudaFreeHost(st->host_gp);
    if (st->host_rctl) cudaFreeHost(st->host_rctl);
    if (st->ev0) cudaEventDestroy(st->ev0);
    if (st->ev1) cudaEventDestroy(st->ev1);
    for (int i = 0; i < st->npev; i++) cudaEventDestroy(st->pev[i]);
    delete[] st->pev;
    st->pev = nullptr;
    st->npev = 0;
    cudaStreamSynchronize(s);
    return DI_OK;
}

// The arrays one sweep works on (see k_plan): take from Ft, push into Fd,
// add the taken fluid to Hs, under control block ctl.
struct Sweep {
    SweepKind kind;
    void *Ft;
    void *Fd;
    double *Hs;
    DevCtl *ctl;
};

static Sweep sweep_of(di_state_s *st, SweepKind kind)
{
    if (kind == SW_F32) return Sweep{kind, st->F32, st->F32, st->D, st->ctl};
    if (kind == SW_REFINE) return Sweep{kind, st->D, st->F, st->H, st->rctl};
    return Sweep{kind, st->F, st->F, st->H, st->ctl};
}

static void launch_select(di_graph_s *g, di_state_s *st, const Sweep &w, cudaStream_t s, int use_cond,
                          cudaGraphConditionalHandle h, int32_t *sel_ids = nullptr)
{
    if (w.kind == SW_F32)
        k_select<float><<<(unsigned)st->ntiles, SEL_THREADS, 0, s>>>(
            static_cast<const float *>(w.Ft), g->n, st->mask, st->hubbits, st->gp, st->hub_base, st->tile_hub, st->tile_cnt,
            st->tile_diff, st->tile_l1f, st->tile_maxf, st->tile_maxu, w.ctl, use_cond, h, sel_ids);
    else
        k_select<double><<<(unsigned)st->ntiles, SEL_THREADS, 0, s>>>(
            static_cast<const double *>(w.Ft), g->n, st->mask, st->hubbits, st->gp, st->hub_base, st->tile_hub, st->tile_cnt,
            st->tile_diff, st->tile_l1f, st->tile_maxf, st->tile_maxu, w.ctl, use_cond, h, sel_ids);
    count_launches(1);
}

static void launch_plan(di_graph_s *g, di_state_s *st, const Sweep &w, cudaStream_t s, int use_cond,
                        cudaGraphConditionalHandle h)
{
    unsigned long long *stats = w.kind == SW_REFINE ? nullptr : st->stats;
#define DI_PLAN_ARGS                                                                                   \
    w.Hs, st->gp, st->dscale, g->n, st->ntiles, st->tile_cnt, st->tile_diff, st->tile_l1f, st->tile_maxf, \
        st->tile_maxu, st->hub_base, st->tile_hub, w.ctl, use_cond, h, stats
    if (w.kind == SW_F32)
        k_plan<float, false><<<PLAN_CTAS, SEL_THREADS, 0, s>>>(static_cast<float *>(w.Ft),
                                                               static_cast<float *>(w.Fd), DI_PLAN_ARGS);
    else if (w.kind == SW_REFINE)
        k_plan<double, true><<<PLAN_CTAS, SEL_THREADS, 0, s>>>(static_cast<double *>(w.Ft),
                                                               static_cast<double *>(w.Fd), DI_PLAN_ARGS);
    else
        k_plan<double, false><<<PLAN_CTAS, SEL_THREADS, 0, s>>>(static_cast<double *>(w.Ft),
                                                                static_cast<double *>(w.Fd), DI_PLAN_ARGS);
#undef DI_PLAN_ARGS
    count_launches(1);
}

static void launch_push(di_graph_s *g, di_state_s *st, const Sweep &w, cudaStream_t s)
{
    const int grid = push_grid(st->device, w.kind, g->weighted);
    const int64_t ngroups = st->ntiles * TILE / 32;
#define DI_PUSH_ARGS w.Hs, st->gp, st->dscale, st->mask, ngroups, g->n, g->hot_node, w.ctl
    const int sm32 = push_stage_bytes<float>(), sm64 = push_stage_bytes<double>();
    float *f32t = static_cast<float *>(w.Ft), *f32d = static_cast<float *>(w.Fd);
    double *f64t = static_cast<double *>(w.Ft), *f64d = static_cast<double *>(w.Fd);
    if (w.kind == SW_F32) {
        if (g->weighted) k_push<float, true, false><<<grid, PUSH_THREADS, sm32, s>>>(f32t, f32d, DI_PUSH_ARGS);
        else k_push<float, false, false><<<grid, PUSH_THREADS, sm32, s>>>(f32t, f32d, DI_PUSH_ARGS);
    } else if (w.kind == SW_REFINE) {
        if (g->weighted) k_push<double, true, true><<<grid, PUSH_THREADS, sm64, s>>>(f64t, f64d, DI_PUSH_ARGS);
        else k_push<double, false, true><<<grid, PUSH_THREADS, sm64, s>>>(f64t, f64d, DI_PUSH_ARGS);
    } else {
        if (g->weighted) k_push<double, true, false><<<grid, PUSH_THREADS, sm64, s>>>(f64t, f64d, DI_PUSH_ARGS);
        else k_push<double, false, false><<<grid, PUSH_THREADS, sm64, s>>>(f64t, f64d, DI_PUSH_ARGS);
    }
#undef DI_PUSH_ARGS
    count_launches(1);
}

static di_status build_graph_exec(di_graph_s *g, di_state_s *st, SweepKind kind)
{
    cudaGraphExec_t &gx = kind == SW_F32 ? st->gexec32 : st->gexec;
    if (gx) return DI_OK;
    const Sweep w = sweep_of(st, kind);
    (void)push_grid(st->device, kind, g->weighted);  // occupancy query outside the capture
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
        launch_select(g, st, w, st->gstream, 1, h);
        launch_plan(g, st, w, st->gstream, 1, h);
        launch_push(g, st, w, st->gstream);
        cudaGraph_t out = nullptr;
        e = cudaStreamEndCapture(st->gstream, &out);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gx, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        gx = nullptr;
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
                                                      ntiles, p1, p2, nullptr, ctl, RED_PLAIN, nullptr);
    count_launches(1);
    DI_CUDA(cudaGetLastError());
    DI_CUDA(cudaMemcpyAsync(out_host, &ctl->final_l1, sizeof(double), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    return DI_OK;
}

// The same reduction as l1_device, into buffers the caller provides (the
// allocation-free entry point passes its static scratch here).
di_status l1_device_into(di_graph_s *g, const double *v, double *part_l1, double *part_l, DevCtl *ctl,
                         double *out_host, cudaStream_t s)
{
    const int64_t ntiles = (g->n + TILE - 1) / TILE;
    DI_CUDA(cudaMemsetAsync(ctl, 0, sizeof(DevCtl), s));
    k_reduce<<<(unsigned)ntiles, SEL_THREADS, 0, s>>>(v, nullptr, static_cast<const Off *>(g->rp), g->n,
                                                      ntiles, part_l1, part_l, nullptr, ctl, RED_PLAIN, nullptr);
    count_launches(1);
    DI_CUDA(cudaGetLastError());
    DI_CUDA(cudaMemcpyAsync(out_host, &ctl->final_l1, sizeof(double), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    return DI_OK;
}

// Buffers of the FP32-fluid form, allocated on its first use.
static di_status state_alloc_f32(di_state_s *st, cudaStream_t s)
{
    if (st->F32) return DI_OK;
    const int64_t slots = st->ntiles * TILE;
    DI_TRY(dalloc_t(&st->D, slots, s));
    DI_CUDA(cudaMemsetAsync(st->D, 0, sizeof(double) * slots, s));
    DI_TRY(dalloc_t(&st->rctl, 1, s));
    DI_CUDA(cudaMallocHost(reinterpret_cast<void **>(&st->host_rctl), sizeof(DevCtl)));
    DI_TRY(dalloc_t(&st->F32, slots, s));
    return DI_OK;
}

// Sweeps until the control block says done (1 reached its sweep_stop, 2 sweep
// cap): one CUDA-graph launch, or launches polled every check_every sweeps
// (with CUDA events around every push when profiling).
struct PushProfile {
    int npairs = 0;
};

static di_status run_sweeps(di_graph_s *g, di_state_s *st, SweepKind kind, const di_opts *o, cudaStream_t s,
                            PushProfile &pp)
{
    const Sweep w = sweep_of(st, kind);
    DevCtl *hc = st->host_ctl;
    const bool graph_mode = o->use_graph && !o->profile;
    if (graph_mode) {
        DI_TRY(build_graph_exec(g, st, kind));
        DI_CUDA(cudaGraphLaunch(kind == SW_F32 ? st->gexec32 : st->gexec, s));
        return DI_OK;
    }
    for (;;) {
        for (int k = 0; k < o->check_every; k++) {
            launch_select(g, st, w, s, 0, cudaGraphConditionalHandle{});
            launch_plan(g, st, w, s, 0, cudaGraphConditionalHandle{});
            if (o->profile && pp.npairs < STAT_CAP) {
                while (st->npev < 2 * (pp.npairs + 1)) DI_CUDA(cudaEventCreate(&st->pev[st->npev++]));
                DI_CUDA(cudaEventRecord(st->pev[2 * pp.npairs], s));
                launch_push(g, st, w, s);
                DI_CUDA(cudaEventRecord(st->pev[2 * pp.npairs + 1], s));
                pp.npairs++;
            } else {
                launch_push(g, st, w, s);
            }
        }
        DI_CUDA(cudaGetLastError());
        DI_CUDA(cudaMemcpyAsync(hc, st->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s));
        DI_CUDA(cudaStreamSynchronize(s));
        if (hc->done) return DI_OK;
    }
}

// One refinement pass of the FP32 form: H += D, F += d P D - D, D = 0 (a
// single sweep of the push machinery over every node with D != 0, into the
// FP64 fluid), then the exact |F|_1, the FP32 copy of F and the next cycle's
// targets (k_reduce, RED_CYCLE).
static di_status refine_pass(di_graph_s *g, di_state_s *st, cudaStream_t s)
{
    DevCtl *r = st->host_rctl;
    memset(r, 0, sizeof(DevCtl));
    r->theta = 0.0;                 // every node with D != 0
    r->stop_l1 = -1.0;
    r->sweep_stop = -1.0;           // one sweep, never "converged"
    r->theta_factor = 1.0;
    r->max_sweeps = ~0ull;
    DI_CUDA(cudaMemcpyAsync(st->rctl, r, sizeof(DevCtl), cudaMemcpyHostToDevice, s));
    const Sweep w = sweep_of(st, SW_REFINE);
    launch_select(g, st, w, s, 0, cudaGraphConditionalHandle{});
    launch_plan(g, st, w, s, 0, cudaGraphConditionalHandle{});
    launch_push(g, st, w, s);
    k_reduce<<<(unsigned)st->ntiles, SEL_THREADS, 0, s>>>(st->F, nullptr, static_cast<const Off *>(g->rp), g->n,
                                                          st->ntiles, st->tile_l1, st->tile_l, st->tile_max, st->ctl, RED_CYCLE,
                                                          st->F32);
    count_launches(1);
    DI_CUDA(cudaGetLastError());
    return DI_OK;
}

constexpr int MAX_CYCLES = 64;   // FP32-form cycles per call (each gains >= 1/refine_ratio)

di_status solve_loop(di_graph_s *g, di_state_s *st, double tol, const di_opts *o, di_info *info,
                     cudaStream_t s, bool fresh, const double *Z_dev, bool inf_norm)
{
    const int64_t n = g->n;
    const double d = st->d;
    const bool f32 = o->precision == DI_PREC_F32;
    if (f32) DI_TRY(state_alloc_f32(st, s));
    DI_TRY(state_set_bins(g, st, o->hub_deg, o->piece, s));
    DI_TRY(state_sync_ptrs(g, st, s));
    if (fresh) {
        k_init<<<grid_for(n, 256), 256, 0, s>>>(st->F, st->H, Z_dev, n, 1.0 - d, 1.0 / (double)n);
        count_launches(1);
    }
    if (st->dscale_d != d) {
        k_dtab<<<grid_for(DTAB_MAX + 1, 256), 256, 0, s>>>(d, st->dtab);
        k_dscale<<<grid_for(n, 256), 256, 0, s>>>(static_cast<const Off *>(g->rp), g->wsum, st->dtab, n, d,
                                                  st->dscale);
        count_launches(2);
        st->dscale_d = d;
    }
    DevCtl *hc = st->host_ctl;
    memset(hc, 0, sizeof(DevCtl));
    hc->d = d;
    hc->theta_factor = o->theta_factor;
    hc->stop_l1 = (1.0 - d) * tol;
    hc->refine_ratio = o->refine_ratio;
    hc->max_sweeps = (unsigned long long)o->max_sweeps;
    hc->inf_norm = inf_norm ? 1 : 0;
    hc->inf_cap = 0.5 * (1.0 - d);
    DI_CUDA(cudaMemcpyAsync(st->ctl, hc, sizeof(DevCtl), cudaMemcpyHostToDevice, s));
    k_reduce<<<(unsigned)st->ntiles, SEL_THREADS, 0, s>>>(st->F, nullptr, static_cast<const Off *>(g->rp),
                                                          n, st->ntiles, st->tile_l1, st->tile_l, st->tile_max,
                                                          st->ctl, f32 ? RED_CYCLE : RED_INIT,
                                                          f32 ? st->F32 : nullptr);
    count_launches(1);
    DI_CUDA(cudaGetLastError());

    double push_ms = 0.0;
    int64_t push_launches = 0, push_edges = 0, push_entries = 0, push_hot = 0;
    int64_t refinements = 0, refine_links = 0;
    if (o->profile && !st->pev) {
        st->pev = new (std::nothrow) cudaEvent_t[2 * STAT_CAP];
        if (!st->pev) return DI_ERR_OOM;
    }
    PushProfile pp;
    DI_CUDA(cudaEventRecord(st->ev0, s));
    if (!f32) {
        DI_TRY(run_sweeps(g, st, SW_F64, o, s, pp));
    } else {
        // cycles: FP32 sweeps to the cycle target, then the FP64 refinement;
        // the stop test is the one on the refined (exact) |F|_1
        DI_CUDA(cudaMemcpyAsync(hc, st->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s));
        DI_CUDA(cudaStreamSynchronize(s));
        for (int cycle = 0; hc->done == 0; cycle++) {
            if (cycle == MAX_CYCLES) {
                hc->done = 2;
                break;
            }
            DI_TRY(run_sweeps(g, st, SW_F32, o, s, pp));
            DI_TRY(refine_pass(g, st, s));
            refinements++;
            DI_CUDA(cudaMemcpyAsync(hc, st->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s));
            DI_CUDA(cudaMemcpyAsync(st->host_rctl, st->rctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s));
            DI_CUDA(cudaStreamSynchronize(s));
            refine_links += (int64_t)st->host_rctl->sweep_links;
        }
    }
    DI_CUDA(cudaEventRecord(st->ev1, s));
    const unsigned done = hc->done;   // (graph mode: read below)
    k_reduce<<<(unsigned)st->ntiles, SEL_THREADS, 0, s>>>(st->F, st->H, static_cast<const Off *>(g->rp),
                                                          n, st->ntiles, st->tile_l1, st->tile_l, st->tile_max,
                                                          st->ctl, RED_FINAL, nullptr);
    count_launches(1);
    DI_CUDA(cudaGetLastError());
    DI_CUDA(cudaMemcpyAsync(hc, st->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s));
    DI_CUDA(cudaStreamSynchronize(s));
    if (f32) hc->done = done;   // a cycle cap decided on the host
    float ms = 0.f;
    DI_CUDA(cudaEventElapsedTime(&ms, st->ev0, st->ev1));
    if (o->use_graph && !o->profile) count_launches(3 * ((int64_t)hc->sweep + refinements + 1));
    if (pp.npairs) {
        // push launch i follows selection i; selections past the converged
        // sweep returned at once and their pushes found no work
        std::vector<unsigned long long> hstats(3 * STAT_CAP);
        const int ran = (int)((int64_t)hc->sweep < pp.npairs ? (int64_t)hc->sweep : pp.npairs);
        DI_CUDA(cudaMemcpy(hstats.data(), st->stats, sizeof(unsigned long long) * 3 * ran, cudaMemcpyDeviceToHost));
        for (int i = 0; i < ran; i++) {
            if (hstats[3 * i] == 0) continue;
            float pm = 0.f;
            DI_CUDA(cudaEventElapsedTime(&pm, st->pev[2 * i], st->pev[2 * i + 1]));
            push_ms += pm;
            push_launches++;
            push_edges += (int64_t)hstats[3 * i];
            push_entries += (int64_t)hstats[3 * i + 1];
            push_hot += (int64_t)hstats[3 * i + 2];
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
        info->push_hot_links = push_hot;
        info->refinements = refinements;
        info->refine_links = refine_links;
        info->resid_inf = hc->final_max;
        if (inf_norm) info->bound = hc->final_max / (1.0 - d);
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
                                                          g->n, st->ntiles, st->tile_l1, st->tile_l, nullptr, ctl,
                                                          RED_FINAL, nullptr);
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
            state_sync_ptrs(g, &st, s);
            k_dscale<<<grid_for(n, 256), 256, 0, s>>>(static_cast<const Off *>(g->rp), g->wsum, nullptr, n, 0.85,
                                                      st.dscale);
            count_launches(1);
            launch_select(g, &st, sweep_of(&st, SW_F64), s, 0, cudaGraphConditionalHandle{}, sel_ids);
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
