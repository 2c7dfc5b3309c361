// Launch behind the previous kernel of the stream with programmatic dependent
// launch: the launch is processed while that kernel finishes, and the kernel
// calls griddep_wait() before it touches anything the previous kernels write.
// FCFS_PDL=0 in the environment turns the attribute off (the work is the same;
// some profilers need it), and a launch that refuses it runs without it.
#pragma once

#include <cstdlib>
#include <utility>

#include "fcfs_common.cuh"

namespace fcfs {

inline bool pdl_allowed() {
  static const bool ok = !(getenv("FCFS_PDL") && atoi(getenv("FCFS_PDL")) == 0);
  return ok;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_after(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                         Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_allowed() ? 1 : 0;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
  if (e != cudaSuccess && cfg.numAttrs == 1) {
    cudaGetLastError();
    cfg.numAttrs = 0;
    e = cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
  }
  count_launch(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace fcfs
