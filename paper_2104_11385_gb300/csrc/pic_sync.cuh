// pic_sync.cuh -- device-side synchronisation helpers shared by the particle
// kernel and the self-test of its bounded wait: shared-memory addresses,
// %globaltimer, mbarrier init / expect-tx / bounded wait, and cp.async copies
// with their group waits (inline PTX).
#pragma once
#include <cstdint>

#define PIC_WAIT_LIMIT_NS 2000000000ull  // every device wait gives up after 2 s

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bounded wait on an mbarrier phase: gives up after limit_ns of %globaltimer
// (2 s by default) and returns false; the caller records the error and leaves.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase,
                                                  uint64_t limit_ns = PIC_WAIT_LIMIT_NS) {
    const uint32_t a = smem_u32(bar);
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
            "selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(a), "r"(phase)
            : "memory");
        if (done) return true;
        if ((it & 255u) == 0u) {
            uint64_t now = globaltimer();
            if (it == 0) t0 = now;
            else if (now - t0 > limit_ns) return false;
        }
    }
}

}  // namespace

namespace {

// Ampere-style asynchronous copies global -> shared (cp.async, 8 bytes per
// thread): the copy completes without the issuing thread waiting, and
// cp.async.wait_group makes the thread's own earlier groups visible to it.
__device__ __forceinline__ void cp_async_8(void* smem_dst, const void* gmem_src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem_dst)),
                 "l"(__cvta_generic_to_global(gmem_src))
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace
