// Programmatic dependent launch for the single-pass kernels (block,
// real-signal block and mixed-radix).
#pragma once
#include <cuda_runtime.h>

namespace fftseg {

// Launches kernel k with programmatic stream serialization: its blocks may
// start while the previous kernel in the stream runs, so k must call
// grid_dependency_wait before its first global access on the data path.
template <class K, class A>
cudaError_t launch_programmatic(K k, unsigned grid, unsigned block, size_t smem, cudaStream_t st, const A &a)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace fftseg
