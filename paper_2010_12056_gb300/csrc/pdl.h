// Programmatic dependent launch (CUDA 11.8+, sm_90 and later): a kernel launched
// with the programmatic-stream-serialization attribute may start while the
// kernel before it on the same stream is still running.  Its blocks run their
// independent prologue, then wait (griddepcontrol.wait) until that kernel has
// completed and its writes are visible; a kernel signals early
// (griddepcontrol.launch_dependents) that its successor may be scheduled.
// Every kernel launched this way calls wait() in every thread before its first
// read of an earlier kernel's output and before it can exit, so that ordering
// stays transitive along the stream.  Without the attribute both instructions
// return at once.
#pragma once

#include <cuda_runtime.h>

namespace pdl {

__device__ __forceinline__ void wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

inline void set_attr(cudaLaunchAttribute& a) {
    a.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    a.val.programmaticStreamSerializationAllowed = 1;
}

// <<<grid, block, smem, st>>> with the attribute
template <typename... KArgs, typename... Args>
cudaError_t launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    set_attr(attr[0]);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace pdl
