// di_residual_l1_noalloc: the |v|_1 reduction of di_residual_l1 for callers
// that cannot allocate device memory (see include/di.h).  Its scratch lives in
// one file-scope device array; host code reaches it only through the address
// cudaGetSymbolAddress returns, looked up once per device.
#include <cuda_runtime.h>
#include <mutex>

#include "di_internal.cuh"

namespace {

using namespace di;

// Largest graph served: 2^16 * 2048 = 134,217,728 nodes, i.e. this many
// reduction tiles of TILE nodes.
constexpr int64_t NOALLOC_MAX_NODES = (int64_t(1) << 16) * 2048;
constexpr int64_t NOALLOC_MAX_TILES = (NOALLOC_MAX_NODES + TILE - 1) / TILE;
constexpr size_t CTL_BYTES = (sizeof(DevCtl) + 255) / 256 * 256;
constexpr size_t SCRATCH_BYTES = CTL_BYTES + 2 * NOALLOC_MAX_TILES * sizeof(double);

// Control block, then the FP64 tile partials of |v|_1 and of the dangling sum.
static __device__ __align__(256) unsigned char g_l1_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES];

// Device address of g_l1_scratch on the current device (looked up on the
// first call made with that device current).
di_status scratch_on(int device, unsigned char **out)
{
    if (device < 0 || device >= MAX_DEVICES) return DI_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_l1_scratch);
        if (e != cudaSuccess) return note_cuda(e);
        g_addr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_addr[device]);
    return DI_OK;
}

}  // namespace

extern "C" di_status di_residual_l1_noalloc(di_graph_t g, const double *v, double *out, void *stream)
{
    if (!g || !v || !out) return DI_ERR_INVALID_ARG;
    if (g->n > NOALLOC_MAX_NODES) return DI_ERR_INVALID_ARG;
    // v must be device (or managed) memory of the graph's device: a host
    // vector would have to be staged through an allocation, and a kernel must
    // never be handed a host address
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, v) != cudaSuccess) {
        (void)cudaGetLastError();
        return DI_ERR_INVALID_ARG;
    }
    if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) || pa.device != g->device)
        return DI_ERR_INVALID_ARG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return DI_ERR_CUDA;
    if (prev != g->device && cudaSetDevice(g->device) != cudaSuccess) return DI_ERR_CUDA;
    unsigned char *base = nullptr;
    di_status rc = scratch_on(g->device, &base);
    if (rc == DI_OK) {
        DevCtl *ctl = reinterpret_cast<DevCtl *>(base);
        double *part_l1 = reinterpret_cast<double *>(base + CTL_BYTES);
        double *part_l = part_l1 + NOALLOC_MAX_TILES;
        rc = l1_device_into(g, v, part_l1, part_l, ctl, out, static_cast<cudaStream_t>(stream));
    }
    if (prev != g->device) cudaSetDevice(prev);
    return rc;
}
