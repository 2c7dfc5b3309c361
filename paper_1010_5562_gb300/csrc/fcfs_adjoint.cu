// Adjoint of the block transform and edge chaining.
#include <algorithm>

#include "fcfs_common.cuh"

namespace fcfs {

// gE[e] = g_axis[ev0[e]] + g_axis[ev1[e]]: an edge moves both of its corners.
__global__ void edge_chain_kernel(const float* __restrict__ gx, const float* __restrict__ gy,
                                  const int32_t* __restrict__ ev0, const int32_t* __restrict__ ev1,
                                  const int8_t* __restrict__ eaxis, long long E, float* __restrict__ gE) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (long long)gridDim.x * blockDim.x) {
    const float* g = eaxis[e] == 0 ? gx : gy;
    gE[e] = g[ev0[e]] + g[ev1[e]];
  }
}

}  // namespace fcfs

using namespace fcfs;

extern "C" {

fcfs_status fcfs_edge_chain(const float* gx, const float* gy, const int32_t* ev0, const int32_t* ev1,
                            const int8_t* eaxis, int64_t E, float* gE, void* stream) {
  if (E < 0) return FCFS_EINVAL;
  if (E == 0) return FCFS_OK;
  if (!gx || !gy || !ev0 || !ev1 || !eaxis || !gE) return FCFS_EINVAL;
  const int blocks = (int)std::min<long long>((E + 255) / 256, 4096);
  edge_chain_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(gx, gy, ev0, ev1, eaxis, E, gE);
  count_launch(1);
  return cudaGetLastError() == cudaSuccess ? FCFS_OK : FCFS_ECUDA;
}

size_t fcfs_adjoint_workspace_size(int64_t, int32_t, int32_t, int32_t) { return 0; }

fcfs_status fcfs_adjoint(const int32_t*, const int32_t*, const int8_t*, int64_t, int32_t, int32_t, int32_t,
                         const float*, float*, float*, void*, size_t, void*) {
  return FCFS_EUNSUPPORTED;
}

size_t fcfs_batch_workspace_size(int64_t, int32_t, int32_t, int32_t, int32_t) { return 0; }

fcfs_status fcfs_batch(const int32_t*, const int32_t*, const int8_t*, const int64_t*, int32_t, int64_t, int32_t,
                       int32_t, int32_t, uint32_t, float*, int64_t*, void*, size_t, void*) {
  return FCFS_EUNSUPPORTED;
}

}  // extern "C"
