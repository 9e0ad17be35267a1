// Inline-PTX helpers shared by the kernels that stage data with the bulk-copy
// engine (cp.async.bulk), synchronise through mbarriers and drive the
// 5th-generation tensor cores (tcgen05).  sm_103a only.
#pragma once

#include <cstdint>

namespace tn {
namespace {

constexpr long long kWaitCycles = 4000000000LL;       // bounded waits: ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on one phase of an mbarrier; false after ~2 s.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Global -> shared bulk copy completing `bytes` transaction bytes on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Named barrier 1 over the first `n` threads of the block (n a multiple of 32).
template <int n>
__device__ __forceinline__ void named_bar() {
    asm volatile("bar.sync 1, %0;" ::"n"(n) : "memory");
}
// The same, returning the AND of `p` over those threads.
template <int n>
__device__ __forceinline__ bool named_bar_and(bool p) {
    uint32_t r;
    asm volatile(
        "{\n"
        " .reg .pred a, b;\n"
        " setp.ne.u32 a, %1, 0;\n"
        " bar.red.and.pred b, 1, %2, a;\n"
        " selp.u32 %0, 1, 0, b;\n"
        "}\n"
        : "=r"(r)
        : "r"((uint32_t)p), "n"(n)
        : "memory");
    return r != 0;
}

}  // namespace
}  // namespace tn
