// Column-pass kernels that stage the kernel spectra one (target, component)
// step at a time (k_cols<float, NS, LC, true>), instantiated apart from the
// all-at-once ones so the two sets compile in parallel.
#include "sg_cols.cuh"
#include "sg_internal.h"

namespace sg {

ColsKernelF32 cols_kernel_steps(int nsrc, int L)
{
    if (nsrc == 1) {
        if (L == 4096) return k_cols<float, 1, 4096, true>;
        if (L == 2048) return k_cols<float, 1, 2048, true>;
        if (L == 1024) return k_cols<float, 1, 1024, true>;
        if (L == 512) return k_cols<float, 1, 512, true>;
        if (L == 256) return k_cols<float, 1, 256, true>;
        return k_cols<float, 1, 0, true>;
    }
    if (L == 4096) return k_cols<float, 2, 4096, true>;
    if (L == 2048) return k_cols<float, 2, 2048, true>;
    if (L == 1024) return k_cols<float, 2, 1024, true>;
    if (L == 512) return k_cols<float, 2, 512, true>;
    if (L == 256) return k_cols<float, 2, 256, true>;
    return k_cols<float, 2, 0, true>;
}

cudaError_t set_cols_steps_smem_limits(int max_optin)
{
    for (int nsrc = 1; nsrc <= 2; ++nsrc)
        for (int L : {0, 256, 512, 1024, 2048, 4096}) {
            const cudaError_t e = cudaFuncSetAttribute((const void *)cols_kernel_steps(nsrc, L),
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, max_optin);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

}  // namespace sg
