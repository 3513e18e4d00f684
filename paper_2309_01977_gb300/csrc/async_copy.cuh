// Bulk asynchronous copies into shared memory (cp.async.bulk, completing on
// an mbarrier) and bounded mbarrier waits, shared by the sm_100-family
// kernels.  A wait gives up after kWaitCycles (about 2 s) and returns false;
// the caller then records SPECT_ETIMEDOUT and leaves, so that no kernel can
// spin forever on a copy that never lands.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "spect.h"

namespace spect {

constexpr long long kWaitCycles = 4000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Makes barrier initialisation visible to the async proxy (and the cluster).
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Wait until the phase of `bar` with the given parity has completed, for
// at most `limit` SM clock cycles; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_for(uint32_t bar, uint32_t parity, long long limit)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) { return mbar_wait_for(bar, parity, kWaitCycles); }

// A timed-out wait: one thread records SPECT_ETIMEDOUT in the status word
// `err`; every thread of the CTA learns of it at this barrier (so that all
// leave together).  Returns true when no thread timed out.
__device__ __forceinline__ bool sync_ok(bool ok, int* err)
{
    const int bad = __syncthreads_or(!ok);
    if (bad && threadIdx.x == 0 && err) atomicExch(err, SPECT_ETIMEDOUT);
    return !bad;
}

// Arrive on `bar` and announce `bytes` of copies that complete on it.
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Global -> shared copy of `bytes` (multiple of 16; both addresses 16-byte
// aligned) that completes its bytes on `bar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tma_load_1d(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    mbar_expect_tx(bar, bytes);
    bulk_load(dst, src, bytes, bar);
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// its later async-proxy ones (a bulk copy overwriting data just read).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Ask L2 to fetch `bytes` (multiple of 16, 16-byte aligned address) ahead of
// use: a hint, no data returns to the SM and nothing waits on it.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

}  // namespace spect
