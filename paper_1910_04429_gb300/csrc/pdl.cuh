// Programmatic dependent launch between the kernels of one hash: each kernel
// waits, before touching global memory, until its predecessor has completed
// and its writes are visible; the next kernel on the stream may be scheduled
// as each CTA exits (the implicit trigger), which takes part of its launch
// latency off the critical path. No kernel triggers its dependents early:
// CTAs of the next kernel scheduled next to running ones and waiting there
// slowed the running kernel more than the earlier launch saved (n = 10^6:
// 29.8 -> 27.2 us per hash back to back; n = 10^8: 0.3565 -> 0.3554 ms).
// (The wait is a no-op for a kernel launched without the attribute.)
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace pa {

__device__ __forceinline__ void pdl_begin() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// kernel<<<grid, block, smem, st>>>(args...) with programmatic stream serialization
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace pa
