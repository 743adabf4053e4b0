// pdl.cuh -- programmatic dependent launch between the kernels of one step.
//
// The step's kernels form a chain in one stream (and one CUDA graph). Launched with the
// programmatic-serialisation attribute, a kernel may be scheduled while its predecessor's
// last blocks are still running; it then waits in pdl_wait(), before it touches any memory,
// until the predecessor has completed and its writes are visible. What this hides is the
// launch gap between consecutive kernels; no kernel reads anything before the wait, and no
// kernel signals early, so the order of memory effects is that of plain stream order.
#pragma once
#include <cuda_runtime.h>
#include <utility>

namespace dem {

__device__ __forceinline__ void pdl_wait() {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 900)
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

// kernel<<<grid, block, 0, st>>>(args...), with programmatic serialisation when pdl is set
template <typename... KArgs, typename... Args>
inline void launch_k(bool pdl, void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t st,
                     Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace dem
