// Bulk asynchronous global->shared copies completed through an mbarrier
// (cp.async.bulk + mbarrier transaction counts, sm_90 and later, used here on
// sm_103a), with bounded waits.  Under IBLBM_EMULATE the same calls are served
// by host code: the copy happens at issue time and the barrier is a packed
// 64-bit word updated with atomics.
#pragma once

#include "iblbm_dev.cuh"

namespace iblbm {

#ifndef IBLBM_EMULATE

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Barrier expecting `count` arrivals per phase.  Call from one thread, then
// fence_bar_init() and a block barrier before any other use.
__device__ __forceinline__ void bar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_bar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One arrival that also raises the phase's expected transaction bytes.
__device__ __forceinline__ void bar_arrive_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// Plain arrival (release semantics: the caller's earlier shared-memory reads are done).
__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Contiguous copy of `bytes` (multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// One poll; the thread may be suspended in hardware for up to kBarSuspendNs while
// the phase is incomplete (woken early when it completes), so waiting warps do
// not take issue slots from working ones.
constexpr unsigned kBarSuspendNs = 500;
__device__ __forceinline__ bool bar_test(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(kBarSuspendNs)
        : "memory");
    return ok != 0;
}

#else   // host emulation

// word layout: bit 63 phase parity | bits 48..62 arrivals per phase |
// bits 32..47 arrivals pending | bits 0..31 transaction bytes pending (signed)
inline uint64_t emu_bar_pack(unsigned ph, unsigned cnt, unsigned pend, int tx) {
    return ((uint64_t)ph << 63) | ((uint64_t)(cnt & 0x7fffu) << 48) | ((uint64_t)(pend & 0xffffu) << 32) |
           (uint64_t)(uint32_t)tx;
}
inline void emu_bar_update(uint64_t* bar, int arrivals, int dtx) {
    uint64_t o = __atomic_load_n(bar, __ATOMIC_SEQ_CST), n;
    do {
        unsigned ph = (unsigned)(o >> 63), cnt = (unsigned)(o >> 48) & 0x7fffu, pend = (unsigned)(o >> 32) & 0xffffu;
        int tx = (int)(uint32_t)o;
        pend -= arrivals;
        tx += dtx;
        if (pend == 0 && tx == 0) {
            ph ^= 1u;
            pend = cnt;
        }
        n = emu_bar_pack(ph, cnt, pend, tx);
    } while (!__atomic_compare_exchange_n(bar, &o, n, false, __ATOMIC_SEQ_CST, __ATOMIC_SEQ_CST));
}
inline void bar_init(uint64_t* bar, unsigned count) {
    __atomic_store_n(bar, emu_bar_pack(0, count, count, 0), __ATOMIC_SEQ_CST);
}
inline void fence_bar_init() {}
inline void bar_arrive_tx(uint64_t* bar, unsigned bytes) { emu_bar_update(bar, 1, (int)bytes); }
inline void bar_arrive(uint64_t* bar) { emu_bar_update(bar, 1, 0); }
inline void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    if (emu::drop_bulk_copies()) return;   // test hook: a copy that never lands
    std::memcpy(dst, src, bytes);
    emu_bar_update(bar, 0, -(int)bytes);
}
inline bool bar_test(uint64_t* bar, unsigned parity) {
    const bool done = (unsigned)(__atomic_load_n(bar, __ATOMIC_SEQ_CST) >> 63) != parity;
    if (!done) emu::yield();
    return done;
}

#endif

// Wait for the phase of the given parity to complete; false after `limit` polls.
__device__ __forceinline__ bool bar_wait(uint64_t* bar, unsigned parity, long limit) {
    for (long it = 0; it < limit; ++it)
        if (bar_test(bar, parity)) return true;
    return false;
}

}  // namespace iblbm
