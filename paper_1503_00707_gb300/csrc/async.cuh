// Asynchronous bulk copies (cp.async.bulk, global -> shared) completing on
// mbarriers, with bounded waits: a wait gives up after a fixed number of
// polls so that a kernel can report DVM_ETIMEOUT instead of hanging.
#pragma once
#include <cstdint>

namespace dvm {

constexpr uint32_t WAIT_POLLS = 1u << 22;

__device__ inline uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ inline void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ inline void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ inline void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// plain arrival (no transaction bytes)
__device__ inline void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ inline void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after WAIT_POLLS polls (with back-off, about a
// second in all).
__device__ inline bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (uint32_t t = 0; t < WAIT_POLLS; t++) {
        if (mbar_try_wait(bar, parity)) return true;
        if (t > 32) __nanosleep(128);
    }
    return false;
}

__device__ inline uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One wait that suspends the thread until the phase completes or about
// 20 us pass, so that waiting warps leave the issue slots to the others.
__device__ inline bool mbar_try_wait_suspend(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}

// Bounded suspending wait: gives up after about a second of global time
// (or 2^20 tries, whichever comes first).
__device__ inline bool mbar_wait_suspend(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait_suspend(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t t = 0; t < (1u << 20); t++) {
        if (mbar_try_wait_suspend(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) break;
    }
    return false;
}

// Per-thread asynchronous copies global -> shared (cp.async, the L1TEX path),
// completed by commit groups.  `dep` is an unused operand that makes the copy
// wait until the value it names has been computed: passing a result derived
// from the last read of the destination orders that read before the refill.
__device__ inline void cp_async16(void *dst, const void *src, uint32_t dep)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16; // %2" ::"r"(smem_u32(dst)), "l"(src), "r"(dep)
                 : "memory");
}
__device__ inline void cp_async8(void *dst, const void *src, uint32_t dep)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8; // %2" ::"r"(smem_u32(dst)), "l"(src), "r"(dep)
                 : "memory");
}
// Prefetch of the line holding src into L2.
__device__ inline void prefetch_l2(const void *src) { asm volatile("prefetch.global.L2 [%0];" ::"l"(src)); }

// Bulk prefetch of [src, src + bytes) into L2 (bytes a multiple of 16).
__device__ inline void prefetch_l2_bulk(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace dvm

namespace dvm {

// Bulk copy shared -> global in the bulk-group completion mechanism: the
// issuing thread commits the group and waits until the copy has finished
// reading shared memory before that memory is reused or released.
__device__ inline void bulk_s2g(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ inline void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ inline void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

}  // namespace dvm
