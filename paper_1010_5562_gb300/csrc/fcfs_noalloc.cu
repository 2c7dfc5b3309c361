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

#include <cudaTypedefs.h>

#include "fcfs_common.cuh"

namespace fcfs {

fcfs_status make_plan_ex(int64_t V, int32_t T, int32_t K, int32_t prec, bool single, Plan& pl);

// The scratch array.  In host code its name is only a stand-in for the symbol,
// not a device address: the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FCFS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
struct ScratchSlot {
  unsigned long long ctx_id;   // driver context the address belongs to (0: none yet)
  void* ptr;
};
std::mutex g_scratch_mu;
ScratchSlot g_scratch[kMaxDevices] = {};

PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;
PFN_cuCtxGetId_v12000 g_ctx_id = nullptr;
std::once_flag g_ctx_once;

// Unique id of the context current on this thread (0 if none or unknown).
// Context ids are never reused within a process, unlike context handles.
unsigned long long current_context_id() {
  std::call_once(g_ctx_once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f);
  });
  if (!g_ctx_current || !g_ctx_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (g_ctx_current(&c) != CUDA_SUCCESS || c == nullptr) return 0;
  if (g_ctx_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array on the current device.  The address is
// looked up (cudaGetSymbolAddress, which allocates nothing) on the first call
// on a device and again whenever the device's context has changed since (after
// cudaDeviceReset the module is loaded anew and the old address is invalid).
fcfs_status scratch_on_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FCFS_ECUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  ScratchSlot& sl = g_scratch[dev];
  unsigned long long id = current_context_id();
  if (sl.ptr == nullptr || id == 0 || id != sl.ctx_id) {
    void* p = nullptr;
    // also makes the device's primary context current if none is
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return FCFS_ECUDA;
    sl.ptr = p;
    sl.ctx_id = id ? id : current_context_id();
  }
  *out = sl.ptr;
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

// Status word of the last call on this device: waits for `stream`, then reads
// the status the kernels wrote into the scratch array (a bounded wait that gave
// up, FCFS_ETIMEOUT; otherwise FCFS_OK).
extern "C" fcfs_status fcfs_noalloc_status(void* stream) {
  void* ws = nullptr;
  fcfs_status r = scratch_on_current_device(&ws);
  if (r != FCFS_OK) return r;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return FCFS_ECUDA;
  Status h{0, 0};
  if (cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return FCFS_ECUDA;
  return static_cast<fcfs_status>(h.code);
}
