// Programmatic dependent launch for the kernels of one decode.
//
// Consecutive kernels of a decode on one stream are launched with
// programmatic stream serialization, so the launch of the next kernel may
// overlap the end of the previous one. Each such kernel calls pdl_wait()
// before its first global memory access: it waits until the previous kernel
// on the stream has completed and its writes are visible. No kernel releases
// its dependents early: the release happens as each CTA exits, so waiting
// CTAs of the next kernel never sit on the SMs beside running ones (an early
// release made them take issue slots from the running kernel and from other
// streams' decodes, measured slower). A kernel launched without the attribute
// passes the wait at once.
#pragma once

#include <cuda_runtime.h>

namespace ldpc {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace ldpc
