// Device primitives of the graph builder: a deterministic exclusive scan and a
// stable LSD radix sort of (uint64 key, uint32 value) pairs.  Both are plain
// three-phase designs (per-tile reduce / scan of tile totals / per-tile
// rewrite), written for sm_103a with warp shuffles and __match_any_sync.
#include <cuda_runtime.h>

#include "di_internal.cuh"

namespace di {

static thread_local int g_last_cuda = 0;
static unsigned long long g_launches = 0;

void count_launches(int64_t k) { __atomic_fetch_add(&g_launches, (unsigned long long)k, __ATOMIC_RELAXED); }
int64_t launches() { return (int64_t)__atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

di_status note_cuda(cudaError_t e)
{
    g_last_cuda = (int)e;
    if (e == cudaErrorMemoryAllocation) return DI_ERR_OOM;
    return DI_ERR_CUDA;
}

int last_cuda() { return g_last_cuda; }

di_status dalloc(void **p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return note_cuda(e);
    }
    return DI_OK;
}

void dfree(void *p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

int sm_count(int device)
{
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) v = 1;
    return v > 0 ? v : 1;
}

constexpr unsigned FULL = 0xffffffffu;

// Exclusive scan of one value per thread across a block of NT threads.
// smem needs NT/32 + 1 slots.  Returns the exclusive prefix; *total = block sum.
template <int NT>
__device__ __forceinline__ uint64_t block_exscan(uint64_t v, uint64_t *smem, uint64_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t ws = lane < NT / 32 ? smem[lane] : 0;
        uint64_t incl = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane < NT / 32) smem[lane] = incl - ws;
        if (lane == NT / 32 - 1) smem[NT / 32] = incl;
    }
    __syncthreads();
    uint64_t r = smem[warp] + x - v;
    *total = smem[NT / 32];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------- scan
constexpr int SCAN_NT = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_NT * SCAN_ITEMS;

template <typename T>
__global__ void __launch_bounds__(SCAN_NT) k_scan_reduce(const T *in, int64_t n, uint64_t *part)
{
    __shared__ uint64_t sm[SCAN_NT / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    uint64_t s = 0;
#pragma unroll 4
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t i = base + k * SCAN_NT + threadIdx.x;
        if (i < n) s += (uint64_t)in[i];
    }
    uint64_t tot;
    block_exscan<SCAN_NT>(s, sm, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_partials(uint64_t *part, int64_t nb, uint64_t *total)
{
    __shared__ uint64_t sm[1024 / 32 + 1];
    uint64_t carry = 0;
    for (int64_t c = 0; c < nb; c += 1024) {
        int64_t i = c + threadIdx.x;
        uint64_t v = i < nb ? part[i] : 0;
        uint64_t tot;
        uint64_t ex = block_exscan<1024>(v, sm, &tot);
        if (i < nb) part[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_NT) k_scan_down(const T *in, int64_t n, const uint64_t *part,
                                                      uint64_t *out)
{
    __shared__ uint64_t sm[SCAN_NT / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint64_t v[SCAN_ITEMS];
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t i = base + k;
        v[k] = i < n ? (uint64_t)in[i] : 0;
        s += v[k];
    }
    uint64_t tot;
    uint64_t run = part[blockIdx.x] + block_exscan<SCAN_NT>(s, sm, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; k++) {
        int64_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
}

template <typename T>
di_status scan_exclusive(const T *in, uint64_t *out, int64_t n, uint64_t *total_dev, cudaStream_t s)
{
    if (n <= 0) {
        if (total_dev) DI_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(uint64_t), s));
        return DI_OK;
    }
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    Temps t(s);
    uint64_t *part;
    DI_TRY(t.get(&part, nb));
    k_scan_reduce<T><<<(unsigned)nb, SCAN_NT, 0, s>>>(in, n, part);
    k_scan_partials<<<1, 1024, 0, s>>>(part, nb, total_dev);
    k_scan_down<T><<<(unsigned)nb, SCAN_NT, 0, s>>>(in, n, part, out);
    count_launches(3);
    DI_CUDA(cudaGetLastError());
    return DI_OK;
}

template di_status scan_exclusive<uint8_t>(const uint8_t *, uint64_t *, int64_t, uint64_t *, cudaStream_t);
template di_status scan_exclusive<uint32_t>(const uint32_t *, uint64_t *, int64_t, uint64_t *, cudaStream_t);
template di_status scan_exclusive<uint64_t>(const uint64_t *, uint64_t *, int64_t, uint64_t *, cudaStream_t);

// ------------------------------------------------------------- radix sort
constexpr int RS_NT = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_NT * RS_ITEMS;
constexpr int RS_WARPS = RS_NT / 32;

__global__ void __launch_bounds__(RS_NT) k_radix_hist(const uint64_t *keys, int64_t n, int shift,
                                                     int nbits, int64_t ntiles, uint32_t *hist)
{
    __shared__ uint32_t cnt[256];
    const int ndig = 1 << nbits;
    const uint64_t mask = (uint64_t)ndig - 1;
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int k = 0; k < RS_ITEMS; k++) {
        int64_t i = base + k * RS_NT + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & mask], 1u);
    }
    __syncthreads();
    if (threadIdx.x < ndig) hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: keys of the tile are ranked in index order (item k of
// thread t is index k*RS_NT + t, so items are walked k-major, warps in order,
// lanes in order).
__global__ void __launch_bounds__(RS_NT) k_radix_scatter(const uint64_t *kin, const uint32_t *vin,
                                                        uint64_t *kout, uint32_t *vout, int64_t n,
                                                        int shift, int nbits, int64_t ntiles,
                                                        const uint64_t *offs)
{
    __shared__ uint32_t s_wcnt[RS_WARPS][256];
    __shared__ uint32_t s_run[256];
    __shared__ uint64_t s_base[256];
    const int ndig = 1 << nbits;
    const uint64_t mask = (uint64_t)ndig - 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    s_run[threadIdx.x] = 0;
    if (threadIdx.x < ndig) s_base[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int k = 0; k < RS_ITEMS; k++) {
        const int64_t i = base + (int64_t)k * RS_NT + threadIdx.x;
        const bool valid = i < n;
        uint64_t key = 0;
        uint32_t val = 0;
        int dg = 256;  // sentinel for past-the-end slots
        if (valid) {
            key = kin[i];
            val = vin[i];
            dg = (int)((key >> shift) & mask);
        }
        const unsigned peers = __match_any_sync(FULL, dg);
        const unsigned lrank = __popc(peers & lt);
        for (int q = lane; q < 256; q += 32) s_wcnt[warp][q] = 0;
        __syncwarp();
        if (valid && lrank == 0) s_wcnt[warp][dg] = __popc(peers);
        __syncthreads();
        {
            const int dgt = threadIdx.x;  // one digit per thread (RS_NT == 256)
            uint32_t run = s_run[dgt];
#pragma unroll
            for (int w = 0; w < RS_WARPS; w++) {
                uint32_t c = s_wcnt[w][dgt];
                s_wcnt[w][dgt] = run;
                run += c;
            }
            s_run[dgt] = run;
        }
        __syncthreads();
        if (valid) {
            const uint64_t pos = s_base[dg] + s_wcnt[warp][dg] + lrank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

di_status radix_sort_pairs(uint64_t **keys, uint32_t **vals, uint64_t **keys_alt, uint32_t **vals_alt,
                           int64_t n, const int *bit_lo, const int *bit_cnt, int npass, cudaStream_t s)
{
    if (n <= 1) return DI_OK;
    const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    Temps t(s);
    uint32_t *hist;
    uint64_t *offs;
    DI_TRY(t.get(&hist, (size_t)256 * ntiles));
    DI_TRY(t.get(&offs, (size_t)256 * ntiles));
    for (int p = 0; p < npass; p++) {
        const int nb = bit_cnt[p];
        if (nb <= 0) continue;
        const int ndig = 1 << nb;
        k_radix_hist<<<(unsigned)ntiles, RS_NT, 0, s>>>(*keys, n, bit_lo[p], nb, ntiles, hist);
        DI_TRY(scan_exclusive<uint32_t>(hist, offs, (int64_t)ndig * ntiles, nullptr, s));
        k_radix_scatter<<<(unsigned)ntiles, RS_NT, 0, s>>>(*keys, *vals, *keys_alt, *vals_alt, n,
                                                          bit_lo[p], nb, ntiles, offs);
        count_launches(2);
        DI_CUDA(cudaGetLastError());
        uint64_t *tk = *keys;
        *keys = *keys_alt;
        *keys_alt = tk;
        uint32_t *tv = *vals;
        *vals = *vals_alt;
        *vals_alt = tv;
    }
    return DI_OK;
}

}  // namespace di
