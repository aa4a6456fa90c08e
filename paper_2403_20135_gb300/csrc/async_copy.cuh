// Bulk asynchronous copies (global -> shared, cp.async.bulk) completed on
// shared-memory mbarriers, and a bounded wait on an mbarrier phase (device
// code only).  A wait gives up after kWaitLimit polls or kWaitNs nanoseconds
// of the global timer, whichever comes first, and returns false; the callers
// turn that into an error flag instead of spinning forever.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace sdc {

constexpr uint32_t kWaitLimit = 1u << 22;
constexpr unsigned long long kWaitNs = 1000000000ull;   // one second

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}

__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;"); }

__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t phase) {
    uint32_t done = 0;
    const unsigned long long t0 = global_ns();
    for (uint32_t it = 0; it < kWaitLimit && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(phase));
        if (!done && (it & 255u) == 255u && global_ns() - t0 > kWaitNs) break;
    }
    return done != 0;
}

// dst and src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(mbar))
        : "memory");
}

__device__ __forceinline__ void expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

// cp.async (Ampere-style asynchronous copies, per thread): 16 or 8 bytes,
// completed by commit groups and cp.async.wait_group.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Programmatic dependent launch (griddepcontrol): a kernel launched with the
// programmatic-serialisation attribute is scheduled as its predecessor in the
// stream retires, or earlier once every block of the predecessor has issued
// pdl_release(); pdl_wait() returns once every prerequisite grid has
// completed and its memory is visible (at once when there is none).  Only
// the sweep releases its dependents early: dependents that start early hold
// shared memory and registers while they wait, which measured slower for
// the transform kernels (whose successors compete with the other state
// chain's kernels) and faster for the sweep (whose one-wave grid leaves the
// next synthesis room to prefetch its table while the sweep drains).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

}  // namespace sdc
