// Synchronisation primitives of the persistent kernels: acquire / release
// accesses to global words, a device-wide barrier whose last arriving block
// takes a decision for the whole grid, and mbarrier-tracked bulk copies into
// shared memory.  Every wait is bounded in time.
#pragma once

#include "slk_internal.cuh"

namespace {

constexpr unsigned long long kSyncTimeoutNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned ld_acq(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acq_i(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_ar(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Words of one device-wide barrier (zeroed before the launch).
struct GridBarrier {
    unsigned arrive, gen, error, pad;
};

// Device-wide barrier of a cooperative grid.  The last block to arrive runs
// decide() in its thread 0 -- every block's writes made before the barrier
// are visible there -- and publishes the answer with the new generation
// (bit 31); the other blocks learn it from the load that releases them.
// Returns 1 (decide() said stop), 0 (go on) or -1 (a wait gave up after
// kSyncTimeoutNs, or another block's did; gb->error is then non-zero).
template <class Decide>
__device__ int grid_barrier(GridBarrier* gb, unsigned nblocks, Decide decide) {
    __shared__ int s_res;
    __syncthreads();
    if (threadIdx.x == 0) {
        int res = 0;
        const unsigned gen = ld_acq(&gb->gen);
        __threadfence();
        const unsigned prev = atom_add_ar(&gb->arrive, 1u);
        if (prev == nblocks - 1) {
            gb->arrive = 0;
            const unsigned done = decide() ? 0x80000000u : 0u;
            st_rel(&gb->gen, ((gen + 1u) & 0x7fffffffu) | done);
            res = done ? 1 : 0;
        } else {
            const unsigned long long t0 = globaltimer_ns();
            unsigned polls = 0, v;
            while ((v = ld_acq(&gb->gen)) == gen) {
                if ((++polls & 63u) == 0u) {
                    if (ld_acq(&gb->error) != 0u) { res = -1; break; }
                    if (globaltimer_ns() - t0 > kSyncTimeoutNs) {
                        atomicOr(&gb->error, 1u);
                        res = -1;
                        break;
                    }
                }
            }
            if (res == 0) res = (v & 0x80000000u) ? 1 : 0;
        }
        s_res = res;
    }
    __syncthreads();
    return s_res;
}

// ---------------------------------------------------------------- mbarrier + bulk copy

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init1(unsigned long long* b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(b)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long* b) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test_parity(unsigned long long* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity`; false after kSyncTimeoutNs.
__device__ __noinline__ bool mbar_wait_parity(unsigned long long* b, uint32_t parity) {
    if (mbar_test_parity(b, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_test_parity(b, parity))
        if (globaltimer_ns() - t0 > kSyncTimeoutNs) return false;
    return true;
}
// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) writes.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One contiguous global -> shared copy through the bulk-copy unit; both
// addresses 16-byte aligned, bytes a multiple of 16.  Completion is counted
// on mbarrier b (transaction bytes).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         unsigned long long* b) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(b))
        : "memory");
}

}  // namespace
