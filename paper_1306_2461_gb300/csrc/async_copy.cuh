// Asynchronous copies global -> shared completing on an mbarrier, with a bounded wait:
// untiled bulk copies (cp.async.bulk) and 2-D tiled tensor copies (cp.async.bulk.tensor,
// the TMA unit) that stage an iteration tile's flow estimate and I2 window in shared
// memory.
#pragma once

#include <stdint.h>

namespace of {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long gtimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Warm L2 with `bytes` bytes at p (both multiples of 16, inside one allocation): a hint,
// nothing waits for it.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make the barrier's initialisation (and generic-proxy writes to shared memory) visible
// to the asynchronous proxy.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order generic-proxy writes to global memory (made visible to this thread by a grid
// barrier) before this thread's later asynchronous-proxy reads.
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Add `bytes` to the transaction count of the barrier's current phase without arriving:
// copies may then complete on the phase before the arrival that closes it.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// dst (shared) <- src (global), `bytes` a multiple of 16, both addresses 16-byte aligned.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// One 2-D box of the tensor described by the tensor map at `map` (a kernel parameter:
// param space) into shared memory at dst, completing on bar. (x, y) is the box's first
// element; x times the element size must be a multiple of 16 bytes. Elements outside
// the tensor (negative or beyond its extent) are written as zeros and still count
// towards the box's bytes.
__device__ __forceinline__ void tma_load_2d(void *dst, const void *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the barrier phase with the given parity to complete, giving up after
// timeout_ns (and after a matching number of polls, should the timer stall).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long timeout_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer_ns();
    const long long cap = timeout_ns / 64 + 10000;
    for (long long it = 0; it < cap; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((long long)(gtimer_ns() - t0) > timeout_ns) return false;
    }
    return false;
}

}  // namespace of
