// Forward block for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they need a transform: a plugin whose host framework owns every device
// byte and forbids raw allocations, a real-time loop where an allocation would
// stall the device, or a memory-pool callback that must not re-enter the
// allocator.  fcfs_forward_noalloc serves them: its scratch space is a fixed
// array compiled into this library (a file-scope __device__ array), so neither
// the caller nor the library allocates anything per call.
//
// The array is FCFS_NOALLOC_SCRATCH_BYTES long and every GPU that loads the
// library keeps it until the process exits.  All calls share it: it keeps the
// previous call's contents (the sincos tables are reused when T matches, the
// accumulators are zeroed by each call), so calls that overlap on the GPU --
// on different streams, or from different host threads without ordering --
// race and must not be issued.  Clips whose workspace does not fit are run
// with fewer vertex splits; if even one split does not fit the call is
// rejected with FCFS_EUNSUPPORTED.
#include <mutex>

#include "fcfs_common.cuh"

namespace fcfs {

fcfs_status make_plan_ex(int64_t V, int32_t T, int32_t K, int32_t prec, bool single, Plan& pl);

// The scratch array.  In host code its name is only a stand-in for the symbol,
// not a device address: the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FCFS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the first call on a device does this set-up).
fcfs_status scratch_on_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FCFS_ECUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return FCFS_ECUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return FCFS_OK;
}

// Shrink the vertex-split count until the workspace fits the array.
fcfs_status fit_plan(Plan& pl, size_t cap) {
  if (pl.total <= cap) return FCFS_OK;
  const size_t per_split = (size_t)pl.M2 * pl.M2 * sizeof(float);
  if (pl.off_part + per_split > cap) return FCFS_EUNSUPPORTED;
  const long long smax = (long long)((cap - pl.off_part) / per_split);
  const long long nchunks = (pl.V + pl.chunk - 1) / pl.chunk;
  const long long per = (nchunks + smax - 1) / smax;
  pl.split_len = per * pl.chunk;
  pl.splits = (int)((pl.V + pl.split_len - 1) / pl.split_len);
  pl.total = pl.off_part + align_up((size_t)pl.splits * per_split, kWsAlign);
  return pl.total <= cap ? FCFS_OK : FCFS_EUNSUPPORTED;
}

}  // namespace
}  // namespace fcfs

using namespace fcfs;

extern "C" fcfs_status fcfs_forward_noalloc(const int32_t* x, const int32_t* y, const int8_t* s, int64_t V,
                                            int32_t T, int32_t K, int32_t prec, uint32_t flags, float* F_out,
                                            int64_t* area_out, void* stream) {
  if (!F_out || !area_out || flags != 0) return FCFS_EINVAL;
  const auto aligned16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (V > 0 && (!x || !y || !s || !aligned16(x) || !aligned16(y) || !aligned16(s))) return FCFS_EINVAL;
  Plan pl;
  fcfs_status r = make_plan_ex(V, T, K, prec, true, pl);
  if (r != FCFS_OK) return r;
  if ((r = fit_plan(pl, FCFS_NOALLOC_SCRATCH_BYTES)) != FCFS_OK) return r;
  void* ws = nullptr;
  if ((r = scratch_on_current_device(&ws)) != FCFS_OK) return r;
  VertexMaps mp{};
  pl.vx = x;
  pl.vy = y;
  pl.vsg = s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (launch_prep(pl, ws, false, st) != cudaSuccess) return FCFS_ECUDA;
  if (launch_axis(pl, x, y, s, ws, false, st) != cudaSuccess) return FCFS_ECUDA;
  const cudaError_t e = prec == FCFS_PREC_SPLIT_F16 ? launch_gemm_tc(pl, mp, ws, st)
                                                     : launch_gemm_simt(pl, x, y, s, ws, st);
  if (e != cudaSuccess) return FCFS_ECUDA;
  if (launch_reduce(pl, ws, F_out, area_out, false, st) != cudaSuccess) return FCFS_ECUDA;
  return FCFS_OK;
}
