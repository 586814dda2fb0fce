// mpr_tma.cuh -- Tensor Memory Accelerator (TMA) bulk tensor copies and mbarrier waits in inline
// PTX: 2-D tiled copies global -> shared memory that complete on a shared-memory mbarrier, and a
// wait on the barrier's phase with a time limit (a copy that never lands cannot hang a block).
#pragma once

#include <cuda.h>   // CUtensorMap (the 128-byte descriptor; built on the host)
#include <stdint.h>

namespace mpr {
namespace tma {

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
    // make the initialised barrier visible to the async proxy (the TMA unit)
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses before later async-proxy (TMA) writes.
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival that also announces `bytes` of transactions the current phase waits for.
__device__ __forceinline__ void arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Box of the tensor map at element coordinates (x, y) -> dst; completes `bar`'s transactions.
// x * element size must be a multiple of 16 bytes; x and y may lie outside the tensor (fill 0).
__device__ __forceinline__ void load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                        int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits until phase `parity` of *bar has completed; false after limit_ns without completion.
__device__ __forceinline__ bool wait(uint64_t* bar, uint32_t parity, long long limit_ns)
{
    if (try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (try_wait(bar, parity)) return true;
        if ((long long)(globaltimer() - t0) > limit_ns) return false;
    }
}

}  // namespace tma
}  // namespace mpr
