// Poisson log-likelihood for callers that cannot allocate device memory.
//
// spect_poisson_ll needs a plan, and creating a plan calls cudaMalloc.  This
// entry point computes the same sums without a plan: its per-block partial
// sums live in a fixed array compiled into the library (g_ll_partials), which
// every GPU that loads the library keeps until the process exits.  It calls
// no cudaMalloc, cudaFree or allocating library routine.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "geometry.cuh"
#include "internal.h"

namespace {

constexpr int kLlThreads = 256;
constexpr int kLlPerThread = 16;
constexpr size_t kLlPerBlock = (size_t)kLlThreads * kLlPerThread;  // 4096 bins per block
constexpr int kLlMaxBlocks = 16384;                                 // 128 KiB of partial sums
constexpr size_t kLlMaxCount = kLlPerBlock * kLlMaxBlocks;          // 67,108,864 bins
constexpr int kMaxDevices = 64;

// One FP64 partial sum per block.  Shared by every call on a device.
static __device__ __align__(256) double g_ll_partials[kLlMaxBlocks];

// Device address of g_ll_partials, looked up once per device.
double* g_partials_addr[kMaxDevices] = {};
std::mutex g_setup_lock;

// Block b sums bins [b * kLlPerBlock, (b + 1) * kLlPerBlock) in a fixed order:
// y log(p + s) - (p + s) in FP64 (the y == 0 term is -(p + s)), and writes
// the gradient y / (p + s) - 1 with respect to p when grad is not NULL.
__global__ void __launch_bounds__(kLlThreads) ll_partial_kernel(const float* __restrict__ y, const float* __restrict__ p,
                                                                float s, size_t count, double* __restrict__ partials,
                                                                float* __restrict__ grad)
{
    __shared__ double red[kLlThreads / 32];
    const size_t base = (size_t)blockIdx.x * kLlPerBlock;
    double acc = 0.0;
#pragma unroll 4
    for (int r = 0; r < kLlPerThread; ++r) {
        const size_t b = base + (size_t)r * kLlThreads + threadIdx.x;
        if (b < count) {
            const float yv = __ldg(y + b);
            const float lam = __ldg(p + b) + s;
            double term = -(double)lam;
            if (yv != 0.f) term += (double)yv * (double)logf(lam);
            acc += term;
            if (grad) grad[b] = (lam > 0.f ? yv / lam : 0.f) - 1.f;
        }
    }
    const double tot = spect::block_sum_f64(acc, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// Sum of the block partials in a fixed order: thread t adds partials t,
// t + 256, t + 512, ... in turn, then the block reduction of
// block_sum_f64.  The order depends only on n_blocks, so a given count
// always gives bitwise the same total.  With n_blocks == 0 the total is 0.
__global__ void __launch_bounds__(kLlThreads) ll_total_kernel(const double* __restrict__ partials, int n_blocks,
                                                              double* __restrict__ out)
{
    __shared__ double red[kLlThreads / 32];
    double acc = 0.0;
    for (int b = threadIdx.x; b < n_blocks; b += kLlThreads) acc += partials[b];
    const double total = spect::block_sum_f64(acc, red);
    if (threadIdx.x == 0) out[0] = total;
}

int noalloc_fail(int status, const char* msg)
{
    spect_internal_set_error(msg);
    return status;
}

}  // namespace

extern "C" int spect_poisson_ll_noalloc(const float* y, const float* p, float s, size_t count, double* ll_dev,
                                        float* grad_proj, void* stream)
{
    if (!y || !p || !ll_dev) return noalloc_fail(SPECT_EINVAL, "y, p and ll must be device pointers");
    const auto aligned16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
    if (!aligned16(y) || !aligned16(p) || (grad_proj && !aligned16(grad_proj)))
        return noalloc_fail(SPECT_EINVAL, "y, p and grad must be 16-byte aligned");
    if (!(s == s) || s - s != 0.f) return noalloc_fail(SPECT_EINVAL, "s must be finite");
    if (count > kLlMaxCount) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "count %zu exceeds the %zu bins the built-in scratch of "
                      "spect_poisson_ll_noalloc covers; use spect_poisson_ll", count, kLlMaxCount);
        return noalloc_fail(SPECT_EINVAL, msg);
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(SPECT_ECUDA, "cudaGetDevice failed");
    }
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(SPECT_EINVAL, "device index out of range");
    double* partials = nullptr;
    {
        // First call on this device (which is current): look up the device
        // address of the built-in array.  The host-side symbol itself is not a
        // device address and must never be passed to a kernel.
        std::lock_guard<std::mutex> guard(g_setup_lock);
        if (!g_partials_addr[dev]) {
            void* addr = nullptr;
            e = cudaGetSymbolAddress(&addr, g_ll_partials);
            if (e != cudaSuccess || !addr) {
                cudaGetLastError();
                return noalloc_fail(SPECT_ECUDA, "cudaGetSymbolAddress of the built-in scratch failed");
            }
            g_partials_addr[dev] = static_cast<double*>(addr);
        }
        partials = g_partials_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int n_blocks = (int)((count + kLlPerBlock - 1) / kLlPerBlock);
    if (n_blocks > 0) ll_partial_kernel<<<n_blocks, kLlThreads, 0, st>>>(y, p, s, count, partials, grad_proj);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        ll_total_kernel<<<1, kLlThreads, 0, st>>>(partials, n_blocks, ll_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return noalloc_fail(SPECT_ECUDA, cudaGetErrorString(e));
    return SPECT_OK;
}
