// Kernel launch with an optional programmatic dependence on the kernel before
// it on the stream (shared by the row, column and table translation units).
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace sg {

// Launch with the programmatic-stream-serialization attribute when pdl:
// the kernel may then start before its predecessor on the stream finishes,
// and must call griddep_wait before reading anything that predecessor
// writes, and read it coherently (ld_cg_hint or TMA, never the
// non-coherent path, which presumes data fixed for the kernel's lifetime).
template <typename... KArgs, typename... Args>
cudaError_t launch_ex(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                      Args &&...args)
{
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace sg
