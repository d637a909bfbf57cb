// Programmatic dependent launch for the kernels of one pipeline step.
//
// A chained launch is prepared while the kernel before it in the stream is
// still running and starts as that kernel's last blocks exit, instead of
// after its completion has gone through the stream's ordering.  No kernel
// releases its dependents earlier (griddepcontrol.launch_dependents): blocks
// of the next kernel resident early, waiting for this one, measured slower
// on every workload tried.
//
// Device side.  chain_wait() returns once every kernel the launch depends on
// has completed and its writes are visible; in a launch that was not chained
// it returns at once.  Every thread of a kernel that may be chained calls it
// before it reads or writes memory that earlier work in the stream touches:
// the kernel then cannot complete before its predecessor, so the guarantee
// carries down a chain.
//
// Host side.  launch_kernel(kern, grid, block, smem, stream, chain, args...)
// launches kern; with chain set the launch carries the programmatic stream
// serialization attribute.  Chain a launch only when the work before it in
// the stream is a kernel of the same step (not a copy, a memset or an event
// wait), so that the relaxed dependency is the one on that kernel.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace veckm {

__device__ __forceinline__ void chain_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                          cudaStream_t s, bool chain, Args &&...args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = chain ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace veckm
