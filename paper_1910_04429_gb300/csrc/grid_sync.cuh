// A bounded grid-wide barrier for cooperative launches (every CTA resident):
// the exact recomputation behind wrapped products and the persistent batched
// transform kernel step through their phases with it.
#pragma once
#include "pa_internal.h"

namespace pa {

struct GridBarrier {
    u32* count;   // zeroed before the launch; every CTA adds one per barrier
    u32 ctas;
    u32 passed;   // barriers this CTA has passed
    u32 limit;    // polls before a wait gives up
    u32* sticky;  // the kernel's device-wide status word
    u32* status;  // the launching stream's status word, or null
};

// All CTAs of the grid reach this point before any leaves it; their global
// writes before it are visible to all after it. A wait that runs out of polls
// marks PA_STATUS_TIMEOUT in both status words and goes on, so the kernel
// always terminates (the cooperative launch makes every CTA resident, so the
// limit is not reached in normal operation).
__device__ __forceinline__ void grid_sync(GridBarrier& g) {
    __syncthreads();
    g.passed++;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(g.count, 1u);
        const u32 target = g.passed * g.ctas;
        u32 spins = 0, v;
        while (true) {
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(g.count) : "memory");
            if (v >= target) break;
            if (++spins > g.limit) {
                atomicOr(g.sticky, PA_STATUS_TIMEOUT);
                if (g.status) atomicOr(g.status, PA_STATUS_TIMEOUT);
                break;
            }
            __nanosleep(128);
        }
        __threadfence();
    }
    __syncthreads();
}

}  // namespace pa
