// Programmatic dependent launch for the kernels of one leapfrog step.
//
// Every step kernel starts with griddepcontrol.wait (it returns once the
// previous kernel of the stream has completed and its writes are visible)
// and ends with griddepcontrol.launch_dependents.  Launched through
// launch_k, with programmatic stream serialization allowed, the next kernel's
// CTAs can therefore be scheduled while the previous kernel drains, instead
// of after it; inside a captured CUDA graph the dependency becomes a
// programmatic edge.  A kernel launched without the attribute executes the
// wait as a no-op.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace smx {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace smx
