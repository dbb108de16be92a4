// Programmatic dependent launch between consecutive kernels of a stream.
//
// A kernel launched with the programmatic-serialization attribute may start
// once every block of the kernel before it in the stream has signalled
// (griddepcontrol.launch_dependents) or exited: its blocks take the SMs that
// the earlier kernel's last blocks leave free, set up shared memory and then
// wait (griddepcontrol.wait) until the earlier kernel has completed and its
// writes are visible.  Every pass kernel that is launched this way waits
// before it touches global memory other than the plan's own twiddle tables
// (a generic pass kernel: every thread at its start; a pipelined one: the
// thread that issues the first TMA load, before a block barrier that all
// other global accesses follow), so reads after writes and writes after reads
// of the previous kernel's buffers stay ordered as in plain stream order.
// The pass kernels signal late (after their stores, or when a persistent
// block starts its last tile).  Both instructions are no-ops for a kernel
// launched without the attribute.
#pragma once
#include <cuda_runtime.h>

namespace moa {

// Let the next kernel in the stream start launching (its blocks still wait).
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// Wait until the previous kernel in the stream has completed and its memory
// operations are visible.
__device__ __forceinline__ void pdl_wait_prior() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch `kern` on `stream`; with `dependent`, as a programmatic dependent
// launch of the kernel before it in the stream.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_maybe_dependent(void (*kern)(KArgs...), unsigned grid, int threads, size_t smem,
                                          cudaStream_t stream, int dependent, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = dependent ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

}  // namespace moa
