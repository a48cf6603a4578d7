// Programmatic dependent launch (sm_90 and later, here sm_103a).  A kernel
// launched with launch_pdl is launched ahead, while the kernel before it in
// the stream is still running, so its launch and the placement of its CTAs
// overlap that kernel's end; its threads then wait in pdl_wait() until the
// kernel before has completed and its writes are visible.  Every kernel
// launched this way calls pdl_wait() before its first global memory access,
// so the stream's order holds as for a plain launch.  The kernels do not
// signal early completion (griddepcontrol.launch_dependents): with that
// signal at a kernel's start the results were wrong, without it they are
// bit for bit those of plain launches and the step is about 1% shorter.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace uccsd {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t stream, Args &&...args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace uccsd
