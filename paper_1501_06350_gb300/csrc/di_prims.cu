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

// The library's scratch comes from the device's default stream-ordered pool.
// By default the pool returns freed memory to the driver at every
// synchronisation, so each graph build, update or solve with host inputs
// mapped and unmapped its temporaries again (about 3 ms of a 4M-page build).
// Keeping up to POOL_KEEP bytes of freed memory in the pool (an attribute of
// this process's pool, gone with the process) lets them be reused.  The bound
// is sized for the largest graphs this library targets on a 288 GB part: a
// link update of a 557M-link graph allocates its new 2.2 GB link arrays while
// the old ones are still live, and with a 2 GiB bound those pages were mapped
// afresh at every update.
constexpr uint64_t POOL_KEEP = 16ull << 30;
void pool_keep(int device)
{
    static bool done[64] = {};
    if (device < 0 || device >= 64 || done[device]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = POOL_KEEP;
        if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess) done[device] = true;
    }
    cudaGetLastError();
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
// One LSD pass = a per-tile digit histogram, an exclusive scan of the
// histograms in (digit, tile) order, and a stable scatter.  A tile is 2048
// pairs; warp w of its CTA holds the tile's items [256 w, 256 w + 256) with
// item k of lane l at 256 w + 32 k + l, so walking k-major inside a warp and
// warps in order visits the tile in index order.
constexpr int RS_NT = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_NT * RS_ITEMS;
constexpr int RS_WARPS = RS_NT / 32;
constexpr int RS_WITEMS = RS_ITEMS * 32;
static_assert(RS_NT == 256, "one digit per thread");

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

// Stable scatter.  Every item gets its rank among the tile's items of the same
// digit (index order: within a warp by item and lane, __match_any_sync groups
// the lanes of one digit; warps in order through per-warp counts); the tile is
// reordered by digit in shared memory and written out with consecutive
// threads writing consecutive positions of each digit's run.
__global__ void __launch_bounds__(RS_NT) k_radix_scatter(const uint64_t *kin, const uint32_t *vin,
                                                        uint64_t *kout, uint32_t *vout, int64_t n,
                                                        int shift, int nbits, int64_t ntiles,
                                                        const uint64_t *offs)
{
    __shared__ uint64_t s_key[RS_TILE];
    __shared__ uint32_t s_val[RS_TILE];
    __shared__ uint32_t s_wcnt[RS_WARPS][256];   // per-warp digit counts, then offsets
    __shared__ uint32_t s_dstart[256];           // tile-local start of each digit's run
    __shared__ uint32_t s_wsum[RS_WARPS];
    __shared__ uint64_t s_gbase[256];            // global start of the run of each digit
    const int ndig = 1 << nbits;
    const uint64_t mask = (uint64_t)ndig - 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int q = threadIdx.x; q < RS_WARPS * 256; q += RS_NT) (&s_wcnt[0][0])[q] = 0;
    s_gbase[threadIdx.x] = threadIdx.x < ndig ? offs[(int64_t)threadIdx.x * ntiles + blockIdx.x] : 0ull;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
    const int64_t w0 = t0 + (int64_t)warp * RS_WITEMS;
    uint64_t key[RS_ITEMS];
    uint32_t val[RS_ITEMS];
    int dg[RS_ITEMS];
    uint32_t rk[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; k++) {
        const int64_t i = w0 + 32 * k + lane;
        key[k] = 0;
        val[k] = 0;
        dg[k] = 256;   // past the end
        if (i < n) {
            key[k] = kin[i];
            val[k] = vin[i];
            dg[k] = (int)((key[k] >> shift) & mask);
        }
    }
#pragma unroll
    for (int k = 0; k < RS_ITEMS; k++) {
        const unsigned peers = __match_any_sync(FULL, dg[k]);
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (lane == leader && dg[k] < 256) {
            // only this lane touches this warp's count of this digit now
            before = s_wcnt[warp][dg[k]];
            s_wcnt[warp][dg[k]] = before + (uint32_t)__popc(peers);
        }
        before = __shfl_sync(FULL, before, leader);
        rk[k] = before + (uint32_t)__popc(peers & lt);
    }
    __syncthreads();
    // per digit (one per thread): offsets of the warps, then the tile's runs
    {
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; w++) {
            const uint32_t c = s_wcnt[w][d];
            s_wcnt[w][d] = run;
            run += c;
        }
        uint32_t incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        uint32_t prev = 0;
        for (int w = 0; w < warp; w++) prev += s_wsum[w];
        s_dstart[d] = prev + incl - run;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RS_ITEMS; k++) {
        if (dg[k] < 256) {
            const uint32_t lp = s_dstart[dg[k]] + s_wcnt[warp][dg[k]] + rk[k];
            s_key[lp] = key[k];
            s_val[lp] = val[k];
        }
    }
    __syncthreads();
    const int cnt = (int)(n - t0 < RS_TILE ? n - t0 : RS_TILE);
    for (int j = threadIdx.x; j < cnt; j += RS_NT) {
        const uint64_t kk = s_key[j];
        const int d = (int)((kk >> shift) & mask);
        const uint64_t pos = s_gbase[d] + (uint64_t)(j - (int)s_dstart[d]);
        kout[pos] = kk;
        vout[pos] = s_val[j];
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
