// C ABI of the FCFS library: argument checks, the launch plan (tiles, vertex
// splits, workspace layout) and the kernel sequence of each entry point.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include <math_constants.h>

#include "fcfs_common.cuh"
#include "fcfs_group.cuh"

namespace fcfs {

static std::atomic<uint64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// Stage timing: when enabled, every stage of a call is bracketed by CUDA events
// recorded on the caller's stream (prep, axis, contraction, reduce).
constexpr int kProfStages = 4;
static bool g_prof = false;
static cudaEvent_t g_ev[2 * kProfStages];
static bool g_ev_made = false;
static void prof_mark(int i, cudaStream_t st) {
  if (!g_prof) return;
  if (!g_ev_made) {
    for (auto& e : g_ev) cudaEventCreate(&e);
    g_ev_made = true;
  }
  cudaEventRecord(g_ev[i], st);
}

size_t tc_smem_for(int bn, int T, int full);

// Kernel timing records: name and a pair of events each, up to kKtMax per
// enable; one stage is open at a time.
constexpr int kKtMax = 64;
static bool g_kt = false;
static bool g_kt_made = false;
static cudaEvent_t g_kt_ev[2 * kKtMax];
static const char* g_kt_name[kKtMax];
static int g_kt_n = 0, g_kt_open = -1;
void kt_begin(const char* name, cudaStream_t st) {
  if (!g_kt || g_kt_n >= kKtMax) return;
  g_kt_name[g_kt_n] = name;
  cudaEventRecord(g_kt_ev[2 * g_kt_n], st);
  g_kt_open = g_kt_n;
}
void kt_end(cudaStream_t st) {
  if (!g_kt || g_kt_open < 0) return;
  cudaEventRecord(g_kt_ev[2 * g_kt_open + 1], st);
  g_kt_n = g_kt_open + 1;
  g_kt_open = -1;
}

static std::atomic<int> g_overlap{-1};   // -1: not yet read from the environment
SideStream* side_stream() {
  int on = g_overlap.load(std::memory_order_relaxed);
  if (on < 0) {
    on = (getenv("FCFS_OVERLAP") && atoi(getenv("FCFS_OVERLAP")) == 0) ? 0 : 1;
    int expect = -1;
    g_overlap.compare_exchange_strong(expect, on);
    on = g_overlap.load(std::memory_order_relaxed);
  }
  if (!on) return nullptr;
  constexpr int kDevMax = 64;
  thread_local SideStream tab[kDevMax] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevMax) return nullptr;
  SideStream& ss = tab[dev];
  if (!ss.s) {
    cudaStream_t s = nullptr;
    cudaEvent_t f = nullptr, j = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    if (cudaEventCreateWithFlags(&f, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess) {
      if (f) cudaEventDestroy(f);
      cudaStreamDestroy(s);
      return nullptr;
    }
    ss = SideStream{s, f, j};
  }
  return &ss;
}
cudaError_t side_fork(SideStream* ss, cudaStream_t st) {
  const cudaError_t e = cudaEventRecord(ss->fork, st);
  return e != cudaSuccess ? e : cudaStreamWaitEvent(ss->s, ss->fork, 0);
}
cudaError_t side_join(SideStream* ss, cudaStream_t st) {
  const cudaError_t e = cudaEventRecord(ss->join, ss->s);
  return e != cudaSuccess ? e : cudaStreamWaitEvent(st, ss->join, 0);
}

static int ceil_log2(long long v) {
  int r = 0;
  while ((1LL << r) < v) ++r;
  return r;
}

static int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 148;
  return n;
}

// Number of vertex splits: the smallest count whose CTAs fill the machine's
// waves to >= 90% while every split keeps >= min_chunks chunks; otherwise the
// best wave efficiency found.
static int choose_splits(long long tiles, long long nchunks, long long slots, long long min_chunks) {
  if (nchunks <= 0) return 0;
  long long smax = std::max(1LL, nchunks / std::max(1LL, min_chunks));
  smax = std::min(smax, 4096LL);
  long long best = 1;
  double best_eff = -1.0;
  for (long long s = 1; s <= smax; ++s) {
    long long ctas = tiles * s;
    long long waves = (ctas + slots - 1) / slots;
    double eff = (double)ctas / (double)(waves * slots);
    if (eff >= 0.9) return (int)s;
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = s;
    }
  }
  return (int)best;
}

static int g_split_override = 0;   // testing/autotuning hook, 0 = automatic
static int g_fuse = 1;             // testing hook: 0 keeps the axis and reduce kernels separate
static int g_pair = 1;             // testing hook: 0 keeps single clips on one-CTA tiles
static int g_barrier_extra = 0;    // testing hook: see fcfs_debug_set_barrier_extra
static int g_hybrid = 1;           // 0: never group by y, 1: automatic, 2: grouped tc, 3: grouped FFT

static thread_local const Knobs* t_knobs = nullptr;
const Knobs* current_knobs() { return t_knobs; }
KnobScope::KnobScope(const Knobs* k) : prev(t_knobs) { t_knobs = k; }
KnobScope::~KnobScope() { t_knobs = prev; }
int knob_splits() { return t_knobs && t_knobs->splits > 0 ? t_knobs->splits : g_split_override; }
static int knob_pair() { return t_knobs && t_knobs->pair >= 0 ? t_knobs->pair : g_pair; }
static int knob_hybrid() { return t_knobs && t_knobs->hybrid >= 0 ? t_knobs->hybrid : g_hybrid; }

// Tag of the cached tables: their kind, period, fixed-point scale and offsets.
static uint64_t table_tag(const Plan& pl) {
  uint64_t h = 0xCBF29CE484222325ull;   // FNV-1a over the fields that fix the table bytes
  const uint64_t f[6] = {4u /* layout version */, (uint64_t)pl.T, (uint64_t)pl.fixq, (uint64_t)pl.full,
                         (uint64_t)pl.off_tab_f32, (uint64_t)pl.off_tab_fix};
  for (uint64_t v : f)
    for (int b = 0; b < 8; ++b) {
      h ^= (v >> (8 * b)) & 0xFFu;
      h *= 0x100000001B3ull;
    }
  return h | 1u;   // never 0, so zeroed memory is never mistaken for a tag
}

// single: a one-clip forward call, whose tensor-core contraction may run on
// CTA pairs; batches and the adjoint use one-CTA tiles.  cosine: the cosine
// series of a clip of period T / 2 (K sine rows, tensor cores always on pairs).
static fcfs_status plan_impl(int64_t V, int32_t T, int32_t K, int32_t prec, bool single, bool cosine, Plan& pl) {
  memset(&pl, 0, sizeof(pl));
  if (T < 4 || T > 65536 || (T & (T - 1)) != 0) return FCFS_EUNSUPPORTED;
  if (K < 1 || K > 4096) return FCFS_EUNSUPPORTED;
  if (V < 0 || V >= (1LL << 31)) return FCFS_EINVAL;
  if (prec != FCFS_PREC_FP32 && prec != FCFS_PREC_SPLIT_F16) return FCFS_EINVAL;
  pl.V = V;
  pl.T = T;
  pl.K = K;
  pl.prec = prec;
  pl.logT = ceil_log2(T);
  const bool tc = prec == FCFS_PREC_SPLIT_F16;
  pl.full = T <= (tc ? kTcFullTableMaxT : kFullTableMaxT) ? 1 : 0;
  pl.fixq = min(30, 62 - ceil_log2(std::max<long long>(V, 1)) - pl.logT);
  pl.cosine = cosine ? 1 : 0;
  pl.M2 = cosine ? K : 2 * K;
  pl.quad_scale = (float)((double)T * (double)T / (4.0 * CUDART_PI * CUDART_PI));
  if (tc) {
    pl.bm = 128;
    pl.bn = (pl.full && pl.M2 > 128) ? 256 : 128;
    pl.chunk = 64;
  } else {
    pl.bm = pl.bn = 128;
    pl.chunk = 32;
  }
  pl.tiles_m = (pl.M2 + pl.bm - 1) / pl.bm;
  pl.tiles_n = (pl.M2 + pl.bn - 1) / pl.bn;
  if (tc && single && (cosine || (knob_pair() && pl.M2 >= 256))) {
    // 256 x 256 tiles on CTA pairs: tile row pair (2 tm', 2 tm' + 1), one per CTA
    pl.pair = 1;
    pl.bn = 256;
    pl.tiles_n = (pl.M2 + 255) / 256;
    pl.tiles_m = 2 * pl.tiles_n;
  }
  const long long nchunks = (V + pl.chunk - 1) / pl.chunk;
  const long long slots = (long long)sm_count() * (tc ? 1 : 2);
  int s = knob_splits() > 0 ? (int)std::min<long long>(knob_splits(), nchunks)
                               : choose_splits((long long)pl.tiles_m * pl.tiles_n, nchunks, slots, 4);
  if (s > 0) {
    const long long per = (nchunks + s - 1) / s;
    pl.split_len = per * pl.chunk;
    pl.splits = (int)((V + pl.split_len - 1) / pl.split_len);
  }
  size_t o = 0;
  pl.off_status = o;
  o = align_up(o + sizeof(Status), kWsAlign);
  pl.off_tab_f32 = o;
  o = align_up(o + tab_f32_bytes(T, pl.full), kWsAlign);
  pl.off_tab_fix = o;
  o = align_up(o + tab_fix_bytes(T, pl.full), kWsAlign);
  pl.off_axis = o;
  o = align_up(o + axis_bytes(K), kWsAlign);
  pl.off_bins = o;
  o = align_up(o + bins_bytes(T), kWsAlign);
  pl.off_hist = o;
  o = align_up(o + (size_t)2 * (T + 1) * sizeof(int), kWsAlign);
  if (single && !cosine && T >= kAxisFftMinT) {
    // before the partials: the grouped forms lay their regions out from off_part
    pl.axfft = 1;
    pl.off_axfft = o;
    o = align_up(o + axis_fft_bytes(T, K), kWsAlign);
  }
  pl.off_part = o;
  o = align_up(o + (size_t)pl.splits * pl.M2 * pl.M2 * sizeof(float), kWsAlign);
  pl.total = o;
  pl.tag = table_tag(pl);
  return FCFS_OK;
}

fcfs_status make_plan_ex(int64_t V, int32_t T, int32_t K, int32_t prec, bool single, Plan& pl) {
  return plan_impl(V, T, K, prec, single, false, pl);
}

fcfs_status make_plan(int64_t V, int32_t T, int32_t K, int32_t prec, Plan& pl) {
  return make_plan_ex(V, T, K, prec, false, pl);
}

// The cosine series of a clip of period T works on sines of period 2T.
fcfs_status make_plan_cosine(int64_t V, int32_t T, int32_t K, int32_t prec, Plan& pl) {
  if (T < 4 || T > 32768 || (T & (T - 1)) != 0) {
    memset(&pl, 0, sizeof(pl));
    return FCFS_EUNSUPPORTED;
  }
  return plan_impl(V, 2 * T, K, prec, true, true, pl);
}

int hybrid_mode() { return knob_hybrid() == 3 ? 1 : knob_hybrid(); }
int hybrid_knob() { return knob_hybrid(); }
bool pair_enabled() { return knob_pair() != 0; }

// The contraction of a single-clip call (fcfs_forward_grouped reports it):
//   kDirect      over the V corners (tensor cores, or the plain FP32 kernel);
//   kGroupedTc   corners grouped by y, split-FP16 contraction over the T + 1
//                values of y (split-FP16 calls on CTA pairs);
//   kGroupedFft  corners grouped by y, pruned FFT along y in FP32 (any precision:
//                its error is below the plain FP32 path's).
// The automatic choice takes the cheapest estimate (ms) among the forms the call
// may take; the estimates are fitted to GB300 measurements of each form's stages
// (T = 2048 .. 65536, K = 128 .. 1024, V / (T + 1) = 0.8 .. 49):
//   direct, tensor cores   0.028 + 1.5e-11 V K^2          ((2K)^2 tensor MACs per corner)
//   direct, plain FP32     0.02 + 1.7e-10 V K^2
//   grouped, tensor cores  g + 4.3e-10 V K p1 + 5.4e-9 T K   (H in FP16 rows, one CTA per SM)
//                          + 1.35e-11 (T + 1) K^2             (contraction over y)
//                          + 3.6e-9 K T + 3.5e-8 K^2          (axis lines, split-K sum)
//   grouped, FFT           g + 3.8e-10 V K p2 + 1.24e-8 K T   (H in polyphase order, the FFT
//                                                             along y and the axis lines)
//   g = 0.055 + 6e-8 V (prep, grouping, launches); p1, p2 = the H kernel's CTA slots
//   (one or two per SM) over its T / 64 items of 64 rows, at least 1.
enum { kDirect = 0, kGroupedTc = 1, kGroupedFft = 2 };

static int forward_form(const Plan& pl, bool validate) {
  const int hy = knob_hybrid();
  if (hy == 0 || validate || pl.V <= 0 || pl.logT > 16 || pl.cosine) return kDirect;
  const bool tc_ok = pl.pair && pl.prec == FCFS_PREC_SPLIT_F16;
  const bool fft_ok = pl.K <= 4096;
  if (hy == 2) return tc_ok ? kGroupedTc : kDirect;
  if (hy == 3) return fft_ok ? kGroupedFft : kDirect;
  const double v = (double)pl.V, k = (double)pl.K, t = (double)pl.T;
  const double items = std::max(1.0, t / 64.0), sms = (double)sm_count();
  const double g = 0.055 + 6e-8 * v;
  double best = pl.prec == FCFS_PREC_SPLIT_F16 ? 0.028 + 1.5e-11 * v * k * k : 0.02 + 1.7e-10 * v * k * k;
  int form = kDirect;
  if (tc_ok) {
    const double c = g + 4.3e-10 * v * k * std::max(1.0, sms / items) + 5.4e-9 * t * k +
                     1.35e-11 * (t + 1.0) * k * k + 3.6e-9 * k * t + 3.5e-8 * k * k;
    if (c < best) {
      best = c;
      form = kGroupedTc;
    }
  }
  if (fft_ok) {
    const double c = g + 3.8e-10 * v * k * std::max(1.0, 2.0 * sms / items) + 1.24e-8 * k * t;
    if (c < best) {
      best = c;
      form = kGroupedFft;
    }
  }
  return form;
}

// Turn a single-clip pair plan into the row-binned one: splits over 64-y
// chunks and the grouping, permutation and H regions after the partials.
static void plan_hybrid(Plan& pl) {
  pl.hyb = 1;
  pl.ny_pad = (pl.T + 1 + 63) / 64 * 64;
  const long long nchunks = pl.ny_pad / 64;
  const int s = knob_splits() > 0 ? (int)std::min<long long>(knob_splits(), nchunks)
                                     : choose_splits((long long)pl.tiles_m * pl.tiles_n, nchunks, sm_count(), 4);
  const long long per = (nchunks + s - 1) / s;
  pl.split_len = per * 64;
  pl.splits = (int)((nchunks + per - 1) / per);
  size_t o = align_up(pl.off_part + (size_t)pl.splits * pl.M2 * pl.M2 * sizeof(float), kWsAlign);
  pl.total = hybrid_extra_bytes(pl.V, pl.T, pl.M2, pl.ny_pad, pl.off_ycnt, pl.off_h, o);
}

// The grouped form with the pruned FFT along y: no partial planes; the grouping
// and the polyphase conj(H) (K T complex values) after the shared regions.
static void plan_fft(Plan& pl) {
  pl.hyb = 1;
  pl.yfft = 1;
  pl.ny_pad = (pl.T + 1 + 63) / 64 * 64;
  pl.splits = 0;
  pl.split_len = 0;
  pl.fft_logL = fft_log_len(pl.T, pl.K);
  size_t o = align_up(pl.off_part, kWsAlign);
  pl.off_ycnt = o;
  o = align_up(o + group_bytes(pl.V, pl.T, pl.ny_pad), kWsAlign);
  pl.off_poly = o;
  o = align_up(o + (size_t)pl.K * pl.T * 8, kWsAlign);
  pl.off_fftab = o;
  o = align_up(o + fft_tables_bytes(pl.T, pl.fft_logL), kWsAlign);
  pl.total = o;
}

static void plan_form(Plan& pl, int form) {
  if (form == kGroupedTc) plan_hybrid(pl);
  else if (form == kGroupedFft) plan_fft(pl);
}

// ---------------------------------------------------------------------------
// Tensor maps for the 1-D TMA vertex loads
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return g_encode;
}


cudaError_t ensure_smem(const void* fn, size_t bytes) {
  struct Entry {
    const void* fn;
    int dev;
    size_t bytes;
  };
  static std::mutex mu;
  static Entry tab[256];
  static int n = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  int i = 0;
  for (; i < n; ++i)
    if (tab[i].fn == fn && tab[i].dev == dev) break;
  if (i < n && tab[i].bytes >= bytes) return cudaSuccess;
  if (bytes > 0 && (e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)) !=
                       cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess) return e;
  if (i == n) {
    if (n == 256) return cudaSuccess;   // table full: attributes set, just not remembered
    tab[n++] = Entry{fn, dev, bytes};
  } else {
    tab[i].bytes = bytes;
  }
  return cudaSuccess;
}

// The first `parts` FP32 partials of a single clip as a 3-D tensor
// [part][row][col] of M2 x M2 x parts floats; one box is the cos and sin rows
// of one k, 64 floats (32 l values) wide, over every part (read by the fused tail).
bool make_part_map(const Plan& pl, void* ws, int parts, CUtensorMap* map) {
  if (!encode_fn() || parts < 1 || parts > 256 || (pl.M2 * 4) % 16 != 0) return false;
  thread_local struct {
    const void* base = nullptr;
    int M2 = -1, S = -1;
    CUtensorMap m;
  } last;
  const void* base = static_cast<uint8_t*>(ws) + pl.off_part;
  if (last.base == base && last.M2 == pl.M2 && last.S == parts) {
    *map = last.m;
    return true;
  }
  cuuint64_t dims[3] = {(cuuint64_t)pl.M2, (cuuint64_t)pl.M2, (cuuint64_t)parts};
  cuuint64_t strides[2] = {(cuuint64_t)pl.M2 * 4, (cuuint64_t)pl.M2 * pl.M2 * 4};
  cuuint32_t box[3] = {64, 2, (cuuint32_t)parts};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return false;
  last.base = base;
  last.M2 = pl.M2;
  last.S = parts;
  last.m = *map;
  return true;
}

bool encode_f16_2d_sw128(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_cols,
                         uint32_t box_rows) {
  if (!encode_fn() || (reinterpret_cast<uintptr_t>(base) & 15u) != 0 || (cols * 2) % 16 != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estr[2] = {1, 1};
  return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

fcfs_status check_ws(const Plan& pl, void* ws, size_t ws_bytes) {
  if (!ws || (reinterpret_cast<uintptr_t>(ws) % kWsAlign) != 0 || ws_bytes < pl.total) return FCFS_EWORKSPACE;
  return FCFS_OK;
}

#define FCFS_CU(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) {                            \
      if (getenv("FCFS_LOG"))                           \
        fprintf(stderr, "fcfs: %s: %s\n", #call, cudaGetErrorString(e_)); \
      return FCFS_ECUDA;                                \
    }                                                   \
  } while (0)

fcfs_status forward_impl(const int32_t* x, const int32_t* y, const int8_t* s, int64_t V, int32_t T, int32_t K,
                         int32_t prec, uint32_t flags, float* F, int64_t* area, void* ws, size_t ws_bytes,
                         cudaStream_t st) {
  if (!F || !area) return FCFS_EINVAL;
  if (V > 0 && (!x || !y || !s || !aligned16(x) || !aligned16(y) || !aligned16(s))) return FCFS_EINVAL;
  if (flags & ~(uint32_t)FCFS_FLAG_VALIDATE) return FCFS_EINVAL;
  Plan pl;
  fcfs_status r = make_plan_ex(V, T, K, prec, true, pl);
  if (r != FCFS_OK) return r;
  const bool validate = (flags & FCFS_FLAG_VALIDATE) != 0;
  plan_form(pl, forward_form(pl, validate));
  if ((r = check_ws(pl, ws, ws_bytes)) != FCFS_OK) return r;
  VertexMaps mp{};
  pl.vx = x;
  pl.vy = y;
  pl.vsg = s;
  prof_mark(0, st);
  {
    KtScope ks("prep", st);
    FCFS_CU(launch_prep(pl, ws, validate, st));
  }
  prof_mark(1, st);
  // the contraction also bins the corners for the axis lines (Steps 2-3), so
  // the axis DFT follows it; device validation keeps its own binning pass
  pl.bin_in_gemm = (validate || pl.hyb) ? 0 : 1;
  // one resident wave of tensor-core CTAs: they also sum the splits, take the
  // axis DFT and write the output behind a grid barrier (two launches per call)
  const int cluster =
      (prec == FCFS_PREC_SPLIT_F16 && !validate && !pl.hyb && g_fuse && V > 0) ? gemm_tc_fuse_cluster(pl) : 0;
  if (cluster > 0 && make_part_map(pl, ws, pl.splits / cluster, &mp.part)) {
    pl.fused = 1;
    pl.cluster = cluster;
    pl.barrier_extra = g_barrier_extra;
    pl.F = reinterpret_cast<float2*>(F);
    pl.area_out = reinterpret_cast<long long*>(area);
  }
  prof_mark(4, st);
  if (pl.yfft || pl.hyb) {
    // grouping, H, the contraction or the FFT along y; beside them (they need only
    // the bins) the exact axis lines on the side stream; then the output
    SideStream* ss = side_stream();
    if (ss) {
      FCFS_CU(side_fork(ss, st));
      KtScope ks("axis_lines", ss->s);
      FCFS_CU(launch_axis(pl, x, y, s, ws, false, ss->s));
    }
    FCFS_CU(pl.yfft ? launch_grouped_fft(pl, ws, F, st) : launch_hybrid(pl, ws, st));
    prof_mark(5, st);
    prof_mark(2, st);
    if (ss) {
      FCFS_CU(side_join(ss, st));
    } else {
      KtScope ks("axis_lines", st);
      FCFS_CU(launch_axis(pl, x, y, s, ws, false, st));
    }
    prof_mark(3, st);
    prof_mark(6, st);
    if (pl.hyb && !pl.yfft) {
      KtScope ks("reduce", st);
      FCFS_CU(launch_reduce(pl, ws, F, area, validate, st));
      prof_mark(7, st);
      return FCFS_OK;
    }
    {
      KtScope ks("axis_out", st);
      FCFS_CU(launch_axis_out(pl, ws, F, area, st));
    }
    prof_mark(7, st);
    return FCFS_OK;
  }
  if (prec == FCFS_PREC_SPLIT_F16) {
    KtScope ks(pl.fused ? "gemm_tc_fused" : "gemm_tc", st);
    FCFS_CU(launch_gemm_tc(pl, mp, ws, st));
  } else {
    KtScope ks("gemm_fp32", st);
    FCFS_CU(launch_gemm_simt(pl, x, y, s, ws, st));
  }
  prof_mark(5, st);
  if (pl.fused) {
    for (int i = 2; i <= 3; ++i) prof_mark(i, st);
    for (int i = 6; i <= 7; ++i) prof_mark(i, st);
    return FCFS_OK;
  }
  prof_mark(2, st);
  {
    KtScope ks("axis_lines", st);
    FCFS_CU(launch_axis(pl, x, y, s, ws, validate, st));
  }
  prof_mark(3, st);
  prof_mark(6, st);
  {
    KtScope ks("reduce", st);
    FCFS_CU(launch_reduce(pl, ws, F, area, validate, st));
  }
  prof_mark(7, st);
  return FCFS_OK;
}

// The form, split count and tile shape a single-clip forward call takes under
// the current knobs.
fcfs_status forward_plan_info(int64_t V, int32_t T, int32_t K, int32_t prec, int* form, int* splits, int* pair) {
  Plan pl;
  const fcfs_status r = make_plan_ex(V, T, K, prec, true, pl);
  if (r != FCFS_OK) return r;
  const int f = forward_form(pl, false);
  plan_form(pl, f);
  *form = f;
  *splits = pl.splits;
  *pair = pl.pair;
  return FCFS_OK;
}

}  // namespace fcfs

using namespace fcfs;

extern "C" {

int fcfs_version(void) { return 100; }

const char* fcfs_status_string(fcfs_status st) {
  switch (st) {
    case FCFS_OK: return "ok";
    case FCFS_EINVAL: return "invalid argument";
    case FCFS_EINVAL_DATA: return "invalid vertex data";
    case FCFS_EWORKSPACE: return "workspace missing, misaligned or too small";
    case FCFS_ECUDA: return "CUDA error";
    case FCFS_ETIMEOUT: return "device wait timed out";
    case FCFS_EUNSUPPORTED: return "unsupported size or precision";
  }
  return "unknown status";
}

uint64_t fcfs_launch_count(void) { return g_launches.load(); }

size_t fcfs_workspace_size(int64_t V, int32_t T, int32_t K, int32_t prec) {
  Plan pl;
  if (make_plan_ex(V, T, K, prec, true, pl) != FCFS_OK) return 0;
  size_t total = pl.total;   // covers calls with device validation, which never group by y
  plan_form(pl, forward_form(pl, false));
  return std::max(total, pl.total);
}

fcfs_status fcfs_forward(const int32_t* x, const int32_t* y, const int8_t* s, int64_t V, int32_t T, int32_t K,
                         int32_t prec, uint32_t flags, float* F_out, int64_t* area_out, void* workspace,
                         size_t ws_bytes, void* stream) {
  return forward_impl(x, y, s, V, T, K, prec, flags, F_out, area_out, workspace, ws_bytes,
                      static_cast<cudaStream_t>(stream));
}

fcfs_status fcfs_get_status(const void* workspace, void* stream) {
  if (!workspace) return FCFS_EWORKSPACE;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return FCFS_ECUDA;
  Status h{0, 0};
  if (cudaMemcpy(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return FCFS_ECUDA;
  return static_cast<fcfs_status>(h.code);
}

// Test hook: force the number of vertex splits (0 restores the automatic choice).
void fcfs_debug_set_splits(int32_t s) { g_split_override = s; }
void fcfs_debug_set_fuse(int32_t on) { g_fuse = on ? 1 : 0; }
void fcfs_debug_set_pair(int32_t on) { g_pair = on ? 1 : 0; }
void fcfs_debug_set_barrier_extra(int32_t n) { g_barrier_extra = n > 0 ? n : 0; }
void fcfs_debug_set_hybrid(int32_t mode) { g_hybrid = mode < 0 ? 0 : (mode > 3 ? 3 : mode); }
void fcfs_debug_set_overlap(int32_t on) { g_overlap.store(on ? 1 : 0, std::memory_order_relaxed); }

int32_t fcfs_forward_grouped(int64_t V, int32_t T, int32_t K, int32_t prec) {
  Plan pl;
  if (make_plan_ex(V, T, K, prec, true, pl) != FCFS_OK) return -1;
  return forward_form(pl, false);
}

void fcfs_profile_enable(int32_t on) { g_prof = on != 0; }

void fcfs_kernel_timing_enable(int32_t on) {
  if (on && !g_kt_made) {
    for (auto& e : g_kt_ev) cudaEventCreate(&e);
    g_kt_made = true;
  }
  g_kt = on != 0;
  g_kt_n = 0;
  g_kt_open = -1;
}

int32_t fcfs_kernel_timing_count(void) {
  if (!g_kt_made || g_kt_n == 0) return 0;
  if (cudaEventSynchronize(g_kt_ev[2 * g_kt_n - 1]) != cudaSuccess) return 0;
  return g_kt_n;
}

const char* fcfs_kernel_timing_name(int32_t i) { return (i >= 0 && i < g_kt_n) ? g_kt_name[i] : ""; }

float fcfs_kernel_timing_ms(int32_t i) {
  float ms = -1.f;
  if (i < 0 || i >= g_kt_n || cudaEventElapsedTime(&ms, g_kt_ev[2 * i], g_kt_ev[2 * i + 1]) != cudaSuccess)
    return -1.f;
  return ms;
}

int32_t fcfs_profile_read(float* ms, int32_t n) {
  if (!g_ev_made || !ms) return 0;
  if (cudaEventSynchronize(g_ev[2 * kProfStages - 1]) != cudaSuccess) return 0;
  int k = 0;
  for (; k < n && k < kProfStages; ++k)
    if (cudaEventElapsedTime(&ms[k], g_ev[2 * k], g_ev[2 * k + 1]) != cudaSuccess) ms[k] = -1.f;
  return k;
}

}  // extern "C"
