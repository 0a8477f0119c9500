// Inline-PTX wrappers shared by the pipelined kernels: mbarriers, bulk
// asynchronous copies (cp.async.bulk) and bounded waits.
#pragma once

#include <stdint.h>

#include "common.cuh"

namespace sqrtba {

constexpr uint64_t WAIT_NS = 2000000000ull;  // every device-side wait gives up after 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar) : "memory");
}
// count arrivals at once (on behalf of warps that skip a phase)
__device__ __forceinline__ void mbar_arrive_cnt(uint32_t bar, uint32_t count) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the phase of `parity`; false after `limit` ns (WAIT_NS = 2 s
// unless a test shortens it) or when another warp has aborted (honour_abort);
// a timeout raises ERRBIT_TIMEOUT.
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, uint32_t* err,
                          bool honour_abort = true, uint64_t limit = WAIT_NS) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (honour_abort && *abort_flag) return false;
        if (global_ns() - t0 > limit) {
            *abort_flag = 1;
            atomicOr(err, ERRBIT_TIMEOUT);
            return false;
        }
    }
}

// Bounded wait until *p == v (a shared-memory word another warp of the CTA
// sets); false after `limit` ns or when another warp has aborted; a timeout
// raises ERRBIT_TIMEOUT.
__device__ inline bool seq_wait(volatile int* p, int v, volatile int* abort_flag, uint32_t* err,
                                uint64_t limit = WAIT_NS) {
    if (*p == v) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (*p == v) return true;
        if (*abort_flag) return false;
        if (global_ns() - t0 > limit) {
            *abort_flag = 1;
            atomicOr(err, ERRBIT_TIMEOUT);
            return false;
        }
    }
}

}  // namespace sqrtba
