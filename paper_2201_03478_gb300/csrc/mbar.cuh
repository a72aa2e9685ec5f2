// mbar.cuh -- shared-memory barriers (mbarrier) with bounded waits, and
// asynchronous global -> shared copies (cp.async), for the warp-specialized
// kernels (the tensor-core contraction, the FP32 interpolation).
//
// Every wait is bounded in wall time (%globaltimer): a wait that expires
// returns false, and the caller raises the plan's device error flag and stops,
// so that a protocol fault surfaces as SL_ERR_TIMEOUT at the next
// sl_plan_sync instead of hanging the GPU.
#pragma once

#include <cstdint>

namespace sl {

constexpr unsigned long long kMsWaitNs = 1000000000ull;   // bound of every mbarrier wait: 1 s
constexpr unsigned kMsSuspendNs = 20000;                  // suspend-time hint of one mbarrier test

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}

// One test of the phase; a thread whose phase is not complete is suspended in
// hardware until it completes or kMsSuspendNs pass (no spinning on the issue
// slots other warps need).
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(done) : "r"(bar), "r"(parity), "n"(kMsSuspendNs) : "memory");
    return done != 0;
}

// Waits for the completion of the mbarrier phase of the given parity, for at
// most limit_ns of wall time; false when the limit expired.  The wall clock is
// read only once the first test has failed (reading it is slow).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns = kMsWaitNs) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}

// Arrives on the barrier once every cp.async this thread issued before has
// landed (the barrier's expected count includes this arrival).
__device__ __forceinline__ void mbar_arrive_cp_async(uint32_t bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" :: "r"(bar) : "memory");
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(smem_u32(dst)), "l"(src) : "memory");
}
// 8-byte copy; with ok == false nothing is read and the destination is zero-filled
__device__ __forceinline__ void cp_async8(void *dst, const void *src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" :: "r"(smem_u32(dst)), "l"(src), "r"(ok ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(NPEND) : "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace sl
