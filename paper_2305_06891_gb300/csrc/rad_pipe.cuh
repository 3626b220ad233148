// Shared-memory pipeline primitives (inline PTX, sm_100 family): mbarriers,
// 1-D bulk copies (global -> shared, completing on an mbarrier's
// transaction count), 4-byte asynchronous copies that arrive on an
// mbarrier when they land, and bounded waits.
#pragma once

#include <cstdint>

namespace rad {
namespace pipe {

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(unsigned long long* b, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count));
}
// makes the initialised barriers visible to the asynchronous proxy
__device__ __forceinline__ void bar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void bar_arrive(unsigned long long* b) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(saddr(b)) : "memory");
}
// the caller's arrival, announcing `bytes` of bulk-copy transactions
__device__ __forceinline__ void bar_arrive_tx(unsigned long long* b, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}\n" ::"r"(
                     saddr(b)),
                 "r"(bytes)
                 : "memory");
}
// bytes (a multiple of 16) from global src to shared dst (both 16-byte
// aligned); completes `bytes` transactions on barrier b
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, unsigned long long* b) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(saddr(dst)),
        "l"(src), "r"(bytes), "r"(saddr(b))
        : "memory");
}
// one 4-byte asynchronous copy global -> shared
__device__ __forceinline__ void cp4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(saddr(dst)), "l"(src) : "memory");
}
// the caller's arrival on b, taken when all its earlier cp.async copies
// have landed (counts as one of the barrier's expected arrivals)
__device__ __forceinline__ void cp_arrive(unsigned long long* b) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// *p += v with release semantics at GPU scope (cumulative: writes this
// thread has observed, including its CTA's writes ordered before it by a
// barrier, become visible to a reader that acquires the new value)
__device__ __forceinline__ void red_release_add(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// one test of phase `parity`; the thread may be suspended in hardware for
// up to about a microsecond (the hint) while the phase is incomplete
__device__ __forceinline__ bool bar_test(unsigned long long* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(saddr(b)), "r"(parity), "r"(1000u)
        : "memory");
    return ok != 0;
}

// Waits are bounded twice over: by wall time (kWaitNs) and by a count of
// tests; a wait that gives up raises *abort, which the CTA's other roles
// poll in their own waits.
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s
constexpr unsigned kWaitTests = 1u << 26;

__device__ __forceinline__ bool bar_wait(unsigned long long* b, uint32_t parity, volatile int* abort) {
    if (bar_test(b, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (unsigned it = 1; it < kWaitTests; ++it) {
        if (bar_test(b, parity)) return true;
        if ((it & 15) == 0 && (*abort || now_ns() - t0 > kWaitNs)) break;
    }
    *abort = 1;
    return false;
}

// waits until *p >= target (p written by other CTAs, read with acquire)
__device__ __forceinline__ bool count_wait(const int* p, int target, volatile int* abort) {
    if (ld_acquire(p) >= target) return true;
    const unsigned long long t0 = now_ns();
    for (unsigned it = 1; it < kWaitTests; ++it) {
        __nanosleep(128);
        if (ld_acquire(p) >= target) return true;
        if ((it & 15) == 0 && (*abort || now_ns() - t0 > kWaitNs)) break;
    }
    *abort = 1;
    return false;
}

}  // namespace pipe
}  // namespace rad
