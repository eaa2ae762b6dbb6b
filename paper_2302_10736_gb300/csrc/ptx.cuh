// ptx.cuh - thin inline-PTX helpers for sm_100+/sm_103a: mbarrier, bulk
// (TMA, non-tensor) copies between global and shared memory, programmatic
// dependent launch controls.
#pragma once

#include <cstdint>

namespace pf {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Bring the line of a valid global address into L2 (a hint: no data returned,
// no ordering; L2 is the point of coherence, so a later load after a
// programmatic-dependent-launch wait still sees what the previous grid wrote)
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make the barrier initialisation visible to the async (TMA) proxy
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait on phase `phase`: gives up after `limit` polls (each try_wait
// suspends the thread for a hardware-chosen while), returns false then.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, phase)) return true;
        __nanosleep(64);
    }
    return false;
}

// global -> shared bulk copy completing on `bar` (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// shared -> global bulk copy in the current bulk group (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// wait until the shared-memory sources of all committed bulk stores were read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// order this thread's generic-proxy shared-memory writes before later async-proxy reads
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Grid-wide barrier for a cooperative launch (every CTA resident).  `state`
// (zero initially) holds a launch parity at [0] and two arrival counters at
// [32] and [64], on separate 128-byte lines.  A launch uses the counter of
// its parity, which is zero when it starts: the k-th barrier of the launch
// (k = 0, 1, ...) is complete when the counter reaches (k + 1) nblocks, and
// every waiting CTA polls the counter itself.  The CTA that completes barrier
// 0 flips the parity for the next launch (every CTA has read it by then), and
// CTA 0 zeroes the other counter, which the previous launch used.  So the
// barrier needs no per-launch host state (graph replays work).  Waiting is
// bounded: after `limit_ns` of the global timer the CTA records
// `timeout_code` in *err and returns false (uniformly for the whole CTA).
__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct GridBar {
    unsigned int *cnt;     // thread 0: this launch's arrival counter
    unsigned int parity;   // thread 0: this launch's parity
};

// at kernel start, before any CTA can have arrived
__device__ __forceinline__ GridBar grid_barrier_begin(unsigned int *state)
{
    GridBar b{nullptr, 0u};
    if (threadIdx.x == 0) {
        b.parity = *(volatile unsigned int *)state & 1u;
        b.cnt = state + 32u + 32u * b.parity;
        if (blockIdx.x == 0) *(volatile unsigned int *)(state + 32u + 32u * (b.parity ^ 1u)) = 0u;
    }
    return b;
}

__device__ __forceinline__ bool grid_barrier(const GridBar &b, unsigned int *state, unsigned int nblocks,
                                             unsigned int k, int *err, int timeout_code, uint64_t limit_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int target = (k + 1u) * nblocks;
        __threadfence();   // this CTA's global writes before its arrival
        unsigned int arrived;
        asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(b.cnt) : "memory");
        if (arrived + 1u == target) {
            if (k == 0) *(volatile unsigned int *)state = b.parity ^ 1u;
        } else {
            const uint64_t t0 = global_timer_ns();
            for (;;) {
                unsigned int c;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(c) : "l"(b.cnt) : "memory");
                if ((int)(c - target) >= 0) break;
                if (global_timer_ns() - t0 > limit_ns) {
                    atomicExch(err, timeout_code);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// programmatic dependent launch: let the next kernel in the stream start its
// prologue now / wait until the previous kernel's results are visible
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

}  // namespace pf
