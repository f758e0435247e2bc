// Programmatic dependent launch between the kernels of one hash: each kernel
// lets the next one on its stream be scheduled as soon as all of its own CTAs
// have started, and waits, before touching global memory, until its
// predecessor has completed and its writes are visible. The launch latency of
// a kernel then overlaps the tail of the one before it. (Both instructions are
// no-ops for a kernel launched without the attribute.)
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace pa {

__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

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
