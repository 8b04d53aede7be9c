// Programmatic dependent launch (sm_90 and later) for the chains of dependent kernels of the
// cycle and the Krylov loop: a kernel launched with the programmatic stream-serialisation
// attribute may be scheduled while the previous kernel of the stream is still running, so its
// launch and block set-up overlap that kernel's execution. Every kernel launched this way calls
// grid_dependency_wait() as its first statement, before any access to global memory; the wait
// returns once the previous kernel has completed and its writes are visible, so no read or write
// can race with it. Right after its own wait, each such kernel allows its dependents to launch
// (griddepcontrol.launch_dependents): the next kernel's blocks are dispatched while this one
// runs and wait in their grid_dependency_wait(). A dependent grid launches only once every block
// of this grid has issued the trigger or exited, i.e. all of them are resident, so waiting
// dependents cannot hold the resources that this grid's blocks still need.
// Inside a stream capture the attribute becomes a programmatic edge of the graph.
//
// EMG_PDL=0 in the environment launches these kernels the ordinary way (for comparisons).
#pragma once
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>

__device__ __forceinline__ void grid_dependency_wait() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

inline bool pdl_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("EMG_PDL");
    return !(v && std::strcmp(v, "0") == 0);
  }();
  return on;
}

// kernel<<<grid, block, smem, st>>>(args...) with programmatic stream serialisation.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
