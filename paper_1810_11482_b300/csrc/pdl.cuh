// Programmatic dependent launch (device and launch side), for step kernels
// that are launched back to back on one stream.
//
// A kernel opens with pdl_prologue(): griddepcontrol.wait blocks until the
// kernel ahead of it on the stream has finished and its memory is visible
// (so nothing is read or written before that, and stream order keeps its
// meaning), and griddepcontrol.launch_dependents lets the launch behind it
// place its CTAs as soon as SM room frees up.  Launched without the
// attribute (launch_pdl with pdl = false, or <<< >>>) both are no-ops.
#pragma once

#include <cuda_runtime.h>

namespace hxc {
namespace k {

__device__ __forceinline__ void pdl_prologue() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launches `kernel` (grid g, block b, no dynamic shared memory) on `s`, with
// programmatic stream serialization when `pdl`.
template <typename... Params, typename... Args>
cudaError_t launch_pdl(void (*kernel)(Params...), unsigned g, unsigned b, cudaStream_t s, bool pdl,
                       Args... args) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(g);
    lc.blockDim = dim3(b);
    lc.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = at;
    lc.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&lc, kernel, static_cast<Params>(args)...);
}

}  // namespace k
}  // namespace hxc
