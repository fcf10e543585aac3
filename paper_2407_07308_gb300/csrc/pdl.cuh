// pdl.cuh -- programmatic dependent launch for the hot kernels.
//
// A kernel launched with launch_pdl may have its CTAs made resident while
// the previous kernel on its stream is still finishing (that kernel lets its
// dependents launch once all of its CTAs have started); every such kernel
// first calls pdl_begin(), which lets its own dependents launch and then
// waits until all prerequisite grids have completed and their memory
// operations are visible -- before it reads or writes any global memory.
// In a captured graph the launches become programmatic edges.  A kernel
// launched without the attribute passes pdl_begin() at once.
//
// Off by default (FHE_PDL 0: plain launches): measured on the 16-pair
// comparison, the waiting CTAs hold SM slots that the concurrent stream's
// kernels would use, 2415 against 2454 slot-comparisons/s.
#pragma once
#include <cuda_runtime.h>

#include <utility>

#ifndef FHE_PDL
#define FHE_PDL 0
#endif

__device__ __forceinline__ void pdl_begin()
{
#if FHE_PDL
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

template <class... KArgs, class... Args>
inline void launch_pdl(void (*kernel)(KArgs...), int grid, int block, cudaStream_t s, Args &&...args)
{
#if FHE_PDL
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);  // errors surface in cudaGetLastError
#else
    kernel<<<grid, block, 0, s>>>(std::forward<Args>(args)...);
#endif
}
