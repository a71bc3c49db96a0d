// nef_launch.cuh -- programmatic dependent launch for the kernels of a sweep and of
// the fold-in step (CUDA-only: included by the .cu translation units).
//
// A sweep is a chain of dependent kernels, many of them small.  Launched with the
// programmatic-serialization attribute, a kernel may be scheduled while its
// predecessor in the stream still runs; it begins with pdl_wait(), which blocks
// until every prerequisite grid has completed and its memory operations are
// visible (and returns at once for a plain launch), so no kernel touches global
// memory before its predecessor is done.  pdl_trigger() right after lets the next
// kernel's launch start.  What overlaps is launch latency and CTA start-up, never
// data access, so the results are those of plain stream order.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <utility>

namespace nef {

// Kernels launched by this library in this process (read through kernel_launches()).
inline std::atomic<long long> g_kernel_launches{0};

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// kernel<<<grid, block, smem, st>>>(args...) with the programmatic-serialization attribute.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
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
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace nef
