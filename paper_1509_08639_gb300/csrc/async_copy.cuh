// async_copy.cuh -- bulk copies into shared memory, mbarriers and bounded
// waits, shared by the kernels of the miner (sm_103a inline PTX).
//
// Every wait here gives up after a fixed number of tries, records
// ERR_TIMEOUT in the batch's error word and returns false, so a kernel whose
// partner never arrives ends instead of spinning forever.
#pragma once
#include "internal.h"

namespace mine {

__device__ __forceinline__ uint32_t s2u(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s2u(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival that also announces `bytes` of transaction on the barrier.
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s2u(bar)),
                 "r"(bytes)
                 : "memory");
}

// TMA bulk copy global -> shared (16-byte aligned addresses, size % 16 == 0).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            s2u(dst)),
        "l"(src), "r"(bytes), "r"(s2u(bar))
        : "memory");
}

// L2 policy for data read once: its lines are the first to be evicted, so a
// stream of them does not push out what is read again soon (the direction
// codes the traceback reads next).
__device__ __forceinline__ uint64_t l2_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void bulk_g2s_once(void *dst, const void *src, uint32_t bytes,
                                              unsigned long long *bar, uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            s2u(dst)),
        "l"(src), "r"(bytes), "r"(s2u(bar)), "l"(policy)
        : "memory");
}

// Test the phase; a thread whose phase is incomplete may be suspended for up
// to kWaitHintNs before the test returns false (no busy spinning).
__device__ __forceinline__ bool mbar_test(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(s2u(bar)), "r"(parity), "r"(kWaitHintNs)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity; gives up after kMbarTries tests
// (at most about kMbarTries * kWaitHintNs), records ERR_TIMEOUT and returns
// false.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, int32_t *err)
{
    for (uint32_t it = 0; it < kMbarTries; ++it)
        if (mbar_test(bar, parity)) return true;
    atomicCAS(err, 0, ERR_TIMEOUT);
    return false;
}

// Spin until *flag >= v (shared memory, written by another warp of the CTA);
// gives up after `tries` tests (0: kWaitLimit).
__device__ __forceinline__ bool flag_wait_ge(const int32_t *flag, int32_t v, int32_t *err,
                                             uint32_t tries = 0)
{
    const uint32_t n = tries ? tries : kWaitLimit;
    for (uint32_t it = 0; it < n; ++it) {
        if (*(volatile const int32_t *)flag >= v) return true;
        __nanosleep(32);
    }
    atomicCAS(err, 0, ERR_TIMEOUT);
    return false;
}

}  // namespace mine
