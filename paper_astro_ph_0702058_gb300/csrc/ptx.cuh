// Hand-written PTX wrappers: mbarriers, bulk (TMA) global->shared copies,
// the MUFU reciprocal square root, the global timer and a bounded grid barrier.
#pragma once

#include <cstdint>

namespace nb {

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Makes initialised barriers visible to the async (TMA) proxy.
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase with the given parity; gives up after ~2 s of wall
// time or 2^26 polls and returns false (the caller records a timeout).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && global_timer_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}

// Device-scope acquire load (pairs with the fence before an arrival).
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Barrier of all CTAs of a cooperative launch (all co-resident): thread 0 of
// each CTA fences the CTA's stores, adds 1 to *ctr (zero at launch) and waits
// until it reaches `target` + CTAs (target: thread 0's count of arrivals
// expected so far, advanced here).  Gives up after ~1 s of wall time and
// returns false (the caller records a timeout); every thread of the CTA calls
// it and gets the same answer through *s_ok.
__device__ __forceinline__ bool grid_barrier(unsigned long long *ctr, unsigned long long &target,
                                             const unsigned ctas, int *s_ok)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        target += ctas;
        __threadfence();
        atomicAdd(ctr, 1ull);
        bool ok = false;
        const uint64_t t0 = global_timer_ns();
        for (uint32_t it = 0; it < (1u << 26); ++it) {
            if (ld_acquire_gpu(ctr) >= target) {
                ok = true;
                break;
            }
            if ((it & 63u) == 63u && global_timer_ns() - t0 > 1000000000ull) break;
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// One bulk asynchronous copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned) from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                         uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// 16-byte asynchronous copy from global to shared memory through L2 only
// (cp.async.cg, the generic proxy: ordered by barriers like a load), then the
// commit and the wait for all of this thread's copies.
__device__ __forceinline__ void cp_async16_cg(void *dst_smem, const void *src_gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst_smem)), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Approximate reciprocal square root on the MUFU unit.
__device__ __forceinline__ float rsqrt_mufu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

}  // namespace nb
