// bulk.cuh -- bulk asynchronous copies between global and shared memory
// (cp.async.bulk, completion on an mbarrier for loads and on bulk groups for
// stores) for the streaming passes over particle arrays: one instruction
// moves a 16 KB tile, so the load/store queues of the SM stay short, and
// every wait is bounded.
#pragma once
#include <cstdint>

#include "device.cuh"

namespace smc {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mb_init(uint64_t* mb, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(mb)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mb_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// one arrival that also expects `bytes` of transactions
__device__ __forceinline__ void mb_expect_tx(uint64_t* mb, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(smem_addr(mb)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mb_test(uint64_t* mb, uint32_t phase) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(smem_addr(mb)), "r"(phase) : "memory");
    return done != 0;
}
// Waits for the phase with parity `phase`: `limit` polls, then (after
// raising ST_TIMEOUT) once more with the full bound, so that no copy is left
// in flight when the caller goes on.  Returns false if the first bound ran
// out.
__device__ __forceinline__ bool mb_wait(uint64_t* mb, uint32_t phase, uint32_t* status,
                                        uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        if (mb_test(mb, phase)) return true;
        if (it > 64) __nanosleep(64);
    }
    raise_status(status, ST_TIMEOUT);
    for (uint32_t it = 0; it < kSpinLimit; ++it) {
        if (mb_test(mb, phase)) break;
        if (it > 64) __nanosleep(64);
    }
    return false;
}
// global -> shared, `bytes` a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* mb) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(mb)) : "memory");
}
// bulk_load with an L2 eviction policy for the source lines
__device__ __forceinline__ void bulk_load_hint(void* dst, const void* src, uint32_t bytes,
                                               uint64_t* mb, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;"
        :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(mb)), "l"(pol) : "memory");
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// shared -> global in the current bulk group (same alignment rules)
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                 :: "l"(dst), "r"(smem_addr(src)), "r"(bytes) : "memory");
}
// bulk_store with an L2 eviction policy for the destination lines
__device__ __forceinline__ void bulk_store_hint(void* dst, const void* src, uint32_t bytes,
                                                uint64_t pol) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;"
                 :: "l"(dst), "r"(smem_addr(src)), "r"(bytes), "l"(pol) : "memory");
}
__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// at most N bulk groups of this thread still reading shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" :: "n"(N) : "memory");
}
// every bulk group of this thread complete (writes visible)
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
// generic-proxy shared-memory writes before an async-proxy read of them
__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace smc
