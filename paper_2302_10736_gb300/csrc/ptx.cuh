// ptx.cuh - thin inline-PTX helpers for sm_100+/sm_103a: mbarrier, bulk
// (TMA, non-tensor) copies between global and shared memory, programmatic
// dependent launch controls.
#pragma once

#include <cstdint>

namespace pf {

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

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
// holds {arrival count, generation} in global memory, both zero initially;
// the last CTA to arrive resets the count and advances the generation, so
// the barrier needs no per-launch host state (graph replays work).  Thread 0
// of every CTA reads the generation once, at kernel start (grid_barrier_gen):
// it cannot move before this CTA arrives, and each barrier advances it by
// one, so arriving needs no further read.  Waiting is bounded: after
// `limit_ns` of the global timer the CTA records `timeout_code` in *err and
// returns false (uniformly for the whole CTA).
__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int grid_barrier_gen(const unsigned int *state)
{
    return threadIdx.x == 0 ? *(const volatile unsigned int *)(state + 1) : 0u;
}

__device__ __forceinline__ bool grid_barrier(unsigned int *state, unsigned int nblocks, unsigned int &gen, int *err,
                                             int timeout_code, uint64_t limit_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = state + 1;
        const unsigned int g0 = gen;
        int ok = 1;
        __threadfence();   // this CTA's global writes before its arrival
        const unsigned int arrived = atomicAdd(state, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(state, 0u);
            // release everyone: the reset (and everything before it) is visible
            // to a CTA that sees the new generation
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(state + 1) : "memory");
        } else {
            const uint64_t t0 = global_timer_ns();
            while (*vgen == g0) {
                if (global_timer_ns() - t0 > limit_ns) {
                    atomicExch(err, timeout_code);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();   // acquire the other CTAs' writes
        gen = g0 + 1;
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
