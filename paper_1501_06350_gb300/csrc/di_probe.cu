// di_probe_atomic_adds: the throughput of FP64 atomic additions at random
// pages of an L2-resident vector on this GPU, the resource the push spends
// per link (it is not a step of the method; it gives the push's roofline).
#include <cuda_runtime.h>

#include "di_internal.cuh"

namespace {

// m additions of 1.0 at pseudo-random slots of a[0, n) (n a power of two):
// the slot is a multiplicative hash of the operation's index, so no index is
// read and every lane adds at its own random address.
__global__ void k_probe_red(double *a, unsigned n_mask, unsigned long long m)
{
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned h = (unsigned)(i * 0x9e3779b97f4a7c15ull >> 32);
        asm volatile("red.global.add.f64 [%0], %1;" ::"l"(a + (h & n_mask)), "d"(1.0) : "memory");
    }
}

}  // namespace

extern "C" di_status di_probe_atomic_adds(int device, double *gops, void *stream)
{
    using namespace di;
    if (!gops || device < 0) return DI_ERR_INVALID_ARG;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return DI_ERR_CUDA;
    if (prev != device && cudaSetDevice(device) != cudaSuccess) return DI_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    di_status rc = DI_OK;
    const unsigned n = 1u << 22;                 // 4M doubles: 32 MB, held in L2
    const unsigned long long m = 1ull << 25;     // 32M additions per launch
    double *a = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 0.f;
    rc = dalloc(reinterpret_cast<void **>(&a), sizeof(double) * n, s);
    if (rc == DI_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = DI_ERR_CUDA;
    if (rc == DI_OK && cudaMemsetAsync(a, 0, sizeof(double) * n, s) != cudaSuccess) rc = DI_ERR_CUDA;
    const unsigned grid = (unsigned)(16 * sm_count(device));
    for (int rep = 0; rc == DI_OK && rep < 4; rep++) {   // the first launch warms L2 and is not counted
        cudaEventRecord(e0, s);
        k_probe_red<<<grid, 256, 0, s>>>(a, n - 1u, m);
        count_launches(1);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = DI_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (rc == DI_OK && cudaGetLastError() != cudaSuccess) rc = DI_ERR_CUDA;
    if (rc == DI_OK) *gops = (double)m / (best * 1e-3) / 1e9;
    if (a) dfree(a, s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    if (prev != device) cudaSetDevice(prev);
    return rc;
}
