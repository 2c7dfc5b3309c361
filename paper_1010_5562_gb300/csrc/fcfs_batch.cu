// Batch of clips sharing T and K in one pass of the forward kernels.
//
// Tiles of a layout are independent (Sec. III-A), so a batch is a list of
// units (clip, output tile, vertex split): clip c of V_c corners contributes
// tiles * ceil(V_c / U) units of at most U corners.  The list is built on the
// device from the device offsets (one block scans the per-clip unit counts),
// so the call needs no host synchronisation and can be captured in a CUDA
// graph.  One launch of the contraction kernel covers every unit (its grid is
// the host-side bound on the unit count; blocks past the actual count exit at
// once), the axis kernel keeps per-clip integer sums, and the reduce kernel
// sums each clip's splits.  U is tunable (fcfs_set_batch_unit_chunks).
#include <algorithm>

#include "fcfs_common.cuh"
#include "fcfs_group.cuh"

namespace fcfs {

fcfs_status make_plan(int64_t V, int32_t T, int32_t K, int32_t prec, Plan& pl);

fcfs_status check_ws(const Plan& pl, void* ws, size_t ws_bytes);

static int g_unit_chunks = 0;   // 0: default (4096 corners per unit)

static fcfs_status make_batch_plan(int64_t V, int32_t n, int32_t T, int32_t K, int32_t prec, const int64_t* offsets,
                                   Plan& pl) {
  if (n < 1) return FCFS_EINVAL;
  fcfs_status r = make_plan(V, T, K, prec, pl);
  if (r != FCFS_OK) return r;
  pl.batch = 1;
  pl.n_clips = n;
  pl.offsets = offsets;
  size_t o = pl.off_axis;       // tables stay where the single-clip plan put them
  o = align_up(o + (size_t)n * (4 * K + 1) * sizeof(long long), kWsAlign);
  pl.off_bins = o;
  o = align_up(o + (size_t)n * bins_bytes(T), kWsAlign);
  pl.off_hist = o;
  // Grouped batch (corners of each clip grouped by y, every clip contracted
  // over its T + 1 values of y on CTA pairs): split FP16, 2K >= 256; taken
  // automatically with on average 8 corners or more per value of y and
  // K >= 256 (the single-clip rule)
  const int mode = hybrid_mode();
  if (prec == FCFS_PREC_SPLIT_F16 && pl.M2 >= 256 && pl.logT <= 16 && V > 0 && n <= 65535 &&
      (mode == 2 || (mode == 1 && V >= 8LL * n * (T + 1) && K >= 256))) {
    pl.hyb = 1;
    pl.pair = 1;
    pl.bn = 256;
    pl.tiles_n = (pl.M2 + 255) / 256;
    pl.tiles_m = 2 * pl.tiles_n;
    pl.ny_pad = (T + 1 + 63) / 64 * 64;
    const long long nchunks = pl.ny_pad / 64;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long ctas1 = (long long)n * pl.tiles_m * pl.tiles_n;   // CTAs of one y split
    const long long s = std::min<long long>(nchunks, std::max<long long>(1, (2LL * sms + ctas1 - 1) / ctas1));
    const long long per = (nchunks + s - 1) / s;
    pl.split_len = per * 64;
    pl.splits = (int)((nchunks + per - 1) / per);
    pl.off_part = o;
    o = align_up(o + (size_t)n * pl.splits * pl.M2 * pl.M2 * sizeof(float), kWsAlign);
    pl.off_ycnt = o;
    o = align_up(o + batch_group_bytes(V, n, T, pl.ny_pad), kWsAlign);
    pl.off_h = o;
    o = align_up(o + (size_t)n * 2 * pl.M2 * pl.ny_pad * 2, kWsAlign);
    pl.total = o;
    return FCFS_OK;
  }
  const Knobs* kn = current_knobs();
  const int uc = kn && kn->unit_chunks > 0 ? kn->unit_chunks : g_unit_chunks;
  const int chunks = uc > 0 ? uc : 4096 / pl.chunk;
  pl.unit_vertices = (int64_t)chunks * pl.chunk;
  // split FP16 with 2K >= 256: units on CTA pairs (256 x 256 tiles, 2-SM MMA)
  if (prec == FCFS_PREC_SPLIT_F16 && pl.M2 >= 256 && pair_enabled()) {
    pl.pair = 1;
    pl.bn = 256;
    pl.tiles_n = (pl.M2 + 255) / 256;
    pl.tiles_m = 2 * pl.tiles_n;
  }
  const long long tiles = pl.pair ? (long long)pl.tiles_n * pl.tiles_n : (long long)pl.tiles_m * pl.tiles_n;
  const long long units_max = tiles * ((V + pl.unit_vertices - 1) / pl.unit_vertices + n);
  if (units_max >= (1LL << 30)) return FCFS_EUNSUPPORTED;
  pl.splits = (int)units_max;   // unit slots of the contraction kernel (CTA pairs: 2 CTAs each)
  pl.off_units = o;
  o = align_up(o + (size_t)(n + 1) * sizeof(int), kWsAlign);
  pl.off_part = o;
  o = align_up(o + (size_t)units_max * (pl.pair ? 2 : 1) * pl.bm * pl.bn * sizeof(float), kWsAlign);
  pl.total = o;
  return FCFS_OK;
}

// unit_start[c] = sum over clips c' < c of tiles * ceil(V_c' / U); unit_start[n] = total
__global__ void __launch_bounds__(1024) batch_units_kernel(Plan pl, uint8_t* ws) {
  int* ustart = reinterpret_cast<int*>(ws + pl.off_units);
  const int n = pl.n_clips, tiles = pl.pair ? pl.tiles_n * pl.tiles_n : pl.tiles_m * pl.tiles_n;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int c0 = min(n, (int)threadIdx.x * per), c1 = min(n, c0 + per);
  auto units = [&](int c) {
    const long long vc = pl.offsets[c + 1] - pl.offsets[c];
    return tiles * (int)((vc + pl.unit_vertices - 1) / pl.unit_vertices);
  };
  int local = 0;
  for (int c = c0; c < c1; ++c) local += units(c);
  __shared__ int scan[1024];
  scan[threadIdx.x] = local;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {   // inclusive scan
    const int v = threadIdx.x >= (unsigned)off ? scan[threadIdx.x - off] : 0;
    __syncthreads();
    scan[threadIdx.x] += v;
    __syncthreads();
  }
  int run = scan[threadIdx.x] - local;
  for (int c = c0; c < c1; ++c) {
    ustart[c] = run;
    run += units(c);
  }
  if (threadIdx.x == blockDim.x - 1) ustart[n] = scan[threadIdx.x];
}

fcfs_status batch_impl(const int32_t* x, const int32_t* y, const int8_t* s, const int64_t* offsets,
                              int32_t n, int64_t V, int32_t T, int32_t K, int32_t prec, uint32_t flags, float* F,
                              int64_t* area, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (!F || !area || !offsets || n < 1) return FCFS_EINVAL;
  if (flags != 0) return FCFS_EUNSUPPORTED;   // device validation is offered for single clips
  const auto aligned16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (V > 0 && (!x || !y || !s || !aligned16(x) || !aligned16(y) || !aligned16(s))) return FCFS_EINVAL;
  Plan pl;
  fcfs_status r = make_batch_plan(V, n, T, K, prec, offsets, pl);
  if (r != FCFS_OK) return r;
  if ((r = check_ws(pl, ws, ws_bytes)) != FCFS_OK) return r;
  VertexMaps mp{};
  pl.vx = x;
  pl.vy = y;
  pl.vsg = s;
  if (launch_prep(pl, ws, false, st) != cudaSuccess) return FCFS_ECUDA;
  if (pl.hyb) {   // grouped: grouping, H, contraction over y; binning, axis DFT, reduce
    pl.bin_in_gemm = 0;
    if (launch_hybrid(pl, ws, st) != cudaSuccess) return FCFS_ECUDA;
    if (launch_axis(pl, x, y, s, ws, false, st) != cudaSuccess) return FCFS_ECUDA;
    if (launch_reduce(pl, ws, F, area, false, st) != cudaSuccess) return FCFS_ECUDA;
    return FCFS_OK;
  }
  batch_units_kernel<<<1, 1024, 0, st>>>(pl, static_cast<uint8_t*>(ws));
  count_launch(1);
  if (cudaGetLastError() != cudaSuccess) return FCFS_ECUDA;
  pl.bin_in_gemm = 1;   // the contraction bins the corners; the axis DFT follows it
  if (V > 0) {
    const cudaError_t e = prec == FCFS_PREC_SPLIT_F16 ? launch_gemm_tc(pl, mp, ws, st)
                                                       : launch_gemm_simt(pl, x, y, s, ws, st);
    if (e != cudaSuccess) return FCFS_ECUDA;
  }
  if (launch_axis(pl, x, y, s, ws, false, st) != cudaSuccess) return FCFS_ECUDA;
  if (launch_reduce(pl, ws, F, area, false, st) != cudaSuccess) return FCFS_ECUDA;
  return FCFS_OK;
}

// Whether a batch is grouped by y, its chunks per unit and its tile shape under
// the current knobs.
fcfs_status batch_plan_info(int64_t V, int32_t n, int32_t T, int32_t K, int32_t prec, int* grouped,
                            int* unit_chunks, int* pair) {
  Plan pl;
  const fcfs_status r = make_batch_plan(V, n, T, K, prec, nullptr, pl);
  if (r != FCFS_OK) return r;
  *grouped = pl.hyb;
  *unit_chunks = pl.hyb ? 0 : (int)(pl.unit_vertices / pl.chunk);
  *pair = pl.pair;
  return FCFS_OK;
}

}  // namespace fcfs

using namespace fcfs;

extern "C" {

size_t fcfs_batch_workspace_size(int64_t V_total, int32_t n_clips, int32_t T, int32_t K, int32_t prec) {
  Plan pl;
  if (make_batch_plan(V_total, n_clips, T, K, prec, nullptr, pl) != FCFS_OK) return 0;
  return pl.total;
}

fcfs_status fcfs_batch(const int32_t* x, const int32_t* y, const int8_t* s, const int64_t* offsets, int32_t n_clips,
                       int64_t V_total, int32_t T, int32_t K, int32_t prec, uint32_t flags, float* F_out,
                       int64_t* area_out, void* workspace, size_t ws_bytes, void* stream) {
  return batch_impl(x, y, s, offsets, n_clips, V_total, T, K, prec, flags, F_out, area_out, workspace, ws_bytes,
                    static_cast<cudaStream_t>(stream));
}

void fcfs_set_batch_unit_chunks(int32_t n) { g_unit_chunks = n > 0 ? n : 0; }

}  // extern "C"
