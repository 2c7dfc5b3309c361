// Row-binned contraction for clips with many more corners than y values.
//
// The quarter-plane product of the contraction (see fcfs_tc.cu),
//   P[m, n] = sum_v s_v A[m, x_v] B[n, y_v],
// regrouped by the corners' y -- the binning of Steps 2-3 applied to the
// off-axis block, as in the sparse-image form of Step 4 --
//   P[m, n] = sum_{y=0..T} H[m, y] B[n, y],   H[m, y] = sum_{v: y_v = y} s_v A[m, x_v],
// contracts over the T + 1 values of y instead of the V corners.  Stages:
//   1. group the corners by y: count per y, exclusive scan, scatter of the
//      corner indices (the order inside a group is free: stage 2 is exact);
//   2. H in 64-bit fixed point from the integer sincos table (the phase k x mod T
//      read from the decimated quarter-wave levels, as in the axis DFT): exact
//      integer sums, hence independent of the order; then FP32, scaled by a
//      power of two 2^-e_y per y where a group is large (no FP16 overflow),
//      and split into FP16 hi = rn(h), lo = rn(h - hi);
//   3. the contraction on CTA pairs: H tiles by TMA, B generated on chip from
//      the exact phase l y mod T (two-level sincos table, angle addition over
//      runs of 8 frequencies) times 2^e_y, three split products into two TMEM
//      accumulators, FP32 partial tiles per y split for the compensated split-K
//      sum of the reduce kernel.
#include <algorithm>

#include "fcfs_epilogue.cuh"
#include "fcfs_fft.cuh"
#include "fcfs_group.cuh"
#include "fcfs_launch.cuh"

namespace fcfs {

namespace {

// ---------------------------------------------------------------------------
// Stage 1: grouping (fcfs_group.cuh); blockIdx.y selects the coordinate
// ---------------------------------------------------------------------------
__global__ void group_count_kernel(const int32_t* __restrict__ c0, const int32_t* __restrict__ c1, long long V,
                                   int T, int ny_pad, uint8_t* base, int key_logP) {
  griddep_wait();   // may be launched behind the previous kernel (programmatic dependent launch)
  const int32_t* c = blockIdx.y ? c1 : c0;
  const Groups g = groups_at(base + blockIdx.y * group_bytes(V, T, ny_pad), T, ny_pad);
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const int y = __ldg(c + v);
    if (y >= 0 && y <= T) atomicAdd(&g.cnt[group_key(y, T, key_logP)], 1);
  }
}

// One CTA: exclusive scan of the T + 1 counts of g into start (and the
// cursors), plus `first`; start[T + 1] = first + the number of grouped corners;
// the exponents e of the large groups.  The counts are read as 4-vectors in
// rounds of one vector per thread (round j, thread t: vector j kScanThreads + t,
// coalesced), every round's loads in flight together: a first pass sums each
// vector, scans the sums within the warps and then over the warps and the
// rounds; a second pass reloads the vectors and writes the running sums and the
// exponents.  R (a template parameter: the fewest rounds that cover the counts)
// bounds the registers, so that a small scan's CTA fits beside the kernel before
// it.
constexpr int kScanThreads = 1024;
constexpr int kScanRounds = 17;   // 4 kScanRounds kScanThreads >= group_stride(65536)
__device__ __forceinline__ int8_t group_exponent(int c) {   // ceil(log2 c) - 14, within [0, 15]
  if (c <= (1 << 14)) return 0;
  const int l = 32 - __clz(c - 1);
  return (int8_t)min(15, l - 14);
}
// Rounds of vectors that cover the counts of coordinates in [0, T].
__host__ __device__ inline int scan_rounds(int T) { return (group_stride(T) / 4 + kScanThreads - 1) / kScanThreads; }

template <int R>
__device__ void scan_groups(const Groups& g, int T, int ny_pad, int first) {
  constexpr int kW = kScanThreads / 32;
  static_assert(kW == 32 && R <= 32, "one lane per warp and per round");
  const int n = T + 1, S = group_stride(T), nvec = S >> 2;
  const int rounds = min(R, (nvec + kScanThreads - 1) / kScanThreads);   // rounds that hold counts (block-uniform)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ int wpre[R][kW];   // per round: the warps' exclusive prefix
  __shared__ int rtot[R], rpre[R], total;
  auto counts = [&](int v) {   // vector v of the counts (inside the padded array); past n: 0
    const int i = 4 * v;
    int4 c = v < nvec ? *reinterpret_cast<const int4*>(g.cnt + i) : make_int4(0, 0, 0, 0);
    if (i >= n) c.x = 0;
    if (i + 1 >= n) c.y = 0;
    if (i + 2 >= n) c.z = 0;
    if (i + 3 >= n) c.w = 0;
    return c;
  };
  int pre[R];   // first the vectors' sums, then their exclusive prefix within the warp
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int4 c = counts(j * kScanThreads + tid);
    pre[j] = c.x + c.y + c.z + c.w;
  }
#pragma unroll
  for (int j = 0; j < R; ++j) {
    if (j >= rounds) break;
    int x = pre[j];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    pre[j] = x - pre[j];
    if (lane == 31) wpre[j][warp] = x;
  }
  __syncthreads();
  if (warp < rounds) {   // warp j: the warps' totals of round j
    const int w = wpre[warp][lane];
    int x = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    wpre[warp][lane] = x - w;
    if (lane == 31) rtot[warp] = x;
  }
  __syncthreads();
  if (warp == 0) {   // the rounds' totals
    const int r = lane < rounds ? rtot[lane] : 0;
    int x = r;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    if (lane < rounds) rpre[lane] = x - r;
    if (lane == 31) total = x;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < R; ++j) {
    if (j >= rounds) break;
    const int v = j * kScanThreads + tid;
    if (v < nvec) {
      const int4 c = counts(v);
      const int run = first + rpre[j] + wpre[j][warp] + pre[j];
      const int i = 4 * v;
      const int4 st4 = make_int4(run, run + c.x, run + c.x + c.y, run + c.x + c.y + c.z);
      if (i < n) {   // start and cursors of the n groups (whole vectors stay inside the padded arrays)
        *reinterpret_cast<int4*>(g.start + i) = st4;
        *reinterpret_cast<int4*>(g.cur + i) = st4;
      }
      if (i < ny_pad) {   // the exponents of these four groups (0 past n), one 4-byte store
        const uint32_t e = (uint32_t)(uint8_t)group_exponent(c.x) | ((uint32_t)(uint8_t)group_exponent(c.y) << 8) |
                           ((uint32_t)(uint8_t)group_exponent(c.z) << 16) |
                           ((uint32_t)(uint8_t)group_exponent(c.w) << 24);
        *reinterpret_cast<uint32_t*>(g.ey + i) = e;
      }
    }
  }
  // exponents past the counts array (ny_pad > S): zero
  for (int i = S + 4 * (int)threadIdx.x; i < ny_pad; i += 4 * kScanThreads) *reinterpret_cast<uint32_t*>(g.ey + i) = 0u;
  __syncthreads();   // start[n] after the vector stores that may cover it
  if (threadIdx.x == 0) g.start[n] = first + total;
}

// One CTA per coordinate.
template <int R>
__global__ void __launch_bounds__(kScanThreads) group_scan_kernel(long long V, int T, int ny_pad, uint8_t* base) {
  griddep_wait();
  scan_groups<R>(groups_at(base + blockIdx.x * group_bytes(V, T, ny_pad), T, ny_pad), T, ny_pad, 0);
}

// Batch: clip c = blockIdx.y groups its corners [offsets[c], offsets[c + 1])
// by y into its own count/start/cursor rows; start values are positions in
// the shared perm (the clip's corners fill [offsets[c], offsets[c + 1])).
__global__ void batch_group_count_kernel(const int32_t* __restrict__ y, const int64_t* __restrict__ offsets, int n,
                                         int T, int ny_pad, long long V, uint8_t* base) {
  const int c = blockIdx.y;
  const Groups g = groups_clip(base, T, ny_pad, n, c, V);
  const long long v0 = offsets[c], v1 = offsets[c + 1];
  for (long long v = v0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; v < v1; v += (long long)gridDim.x * blockDim.x) {
    const int yv = __ldg(y + v);
    if (yv >= 0 && yv <= T) atomicAdd(&g.cnt[yv], 1);
  }
}
template <int R>
__global__ void __launch_bounds__(kScanThreads) batch_group_scan_kernel(const int64_t* __restrict__ offsets, int n,
                                                                        int T, int ny_pad, long long V,
                                                                        uint8_t* base) {
  const int c = blockIdx.x;
  scan_groups<R>(groups_clip(base, T, ny_pad, n, c, V), T, ny_pad, (int)offsets[c]);
}
__global__ void batch_group_scatter_kernel(const int32_t* __restrict__ y, const int64_t* __restrict__ offsets, int n,
                                           int T, int ny_pad, long long V, uint8_t* base) {
  const int c = blockIdx.y;
  const Groups g = groups_clip(base, T, ny_pad, n, c, V);
  const long long v0 = offsets[c], v1 = offsets[c + 1];
  for (long long v = v0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; v < v1; v += (long long)gridDim.x * blockDim.x) {
    const int yv = __ldg(y + v);
    if (yv >= 0 && yv <= T) g.perm[atomicAdd(&g.cur[yv], 1)] = (int)v;
  }
}

__global__ void group_scatter_kernel(const int32_t* __restrict__ c0, const int32_t* __restrict__ c1, long long V,
                                     int T, int ny_pad, uint8_t* base, int key_logP) {
  griddep_wait();
  const int32_t* c = blockIdx.y ? c1 : c0;
  const Groups g = groups_at(base + blockIdx.y * group_bytes(V, T, ny_pad), T, ny_pad);
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const int y = __ldg(c + v);
    if (y >= 0 && y <= T) g.perm[atomicAdd(&g.cur[group_key(y, T, key_logP)], 1)] = (int)v;
  }
}

// FP16 split of two values: hi = rn(v), lo = rn(v - hi)
__device__ __forceinline__ void split2h(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(v0, v1);
  const float2 hf = __half22float2(h);
  memcpy(&hi, &h, 4);
  const __half2 l = __floats2half2_rn(v0 - hf.x, v1 - hf.y);
  memcpy(&lo, &l, 4);
}

// ---------------------------------------------------------------------------
// Stage 2: H[k, y] = sum over the corners of row y of s_v exp(+j 2 pi k x_v / T)
// ---------------------------------------------------------------------------
// Fast path (an item's corners fit in shared memory): the corners of the item's
// rows are sorted by (row, x, sign) and consecutive corners of a row are paired
// (for a set of disjoint polygons these are exactly the row's horizontal edges).
// A pair a < b contributes
//     s_a e^{j k x_a} (1 - e^{j k w})   (opposite signs, w = x_b - x_a),
//     s_a e^{j k x_a} (2 - (1 - e^{j k w}))   (equal signs), or s_a e^{j k x_a} (alone),
// so an edge's two corners cancel in the factor D_k = 1 - e^{j k w} before any
// rounding, and D_k is carried with a relative error of a few ulp however small it
// is (versine tables; D_{k+32} = D_k + D_32 - D_k D_32 stays free of cancellation).
// A lane owns the 8 frequencies k0 + 32 i (the 32 lanes of a warp cover 256
// consecutive frequencies, so their table reads fall on distinct banks): the
// anchors at k0 come from two-level tables at the exact integer phase, the
// next 7 by angle addition (A_{k+32} = A_k e^{j 32 x_a}) and the D recurrence;
// the pair's steps e^{j 32 x_a} and D_32 are formed once per item.  Rows are
// summed in FP32 in the sorted order, so repeated calls are bit-identical.
// Output formats:
//   kHRowsFp16: FP16 hi/lo rows 2(k-1) (Re) and 2(k-1)+1 (Im), columns y (the
//               tensor-core contraction over y); a pass covers 256 frequencies
//               of the item's 64 rows in a shared-memory tile, written out
//               coalesced (512 threads, one CTA per SM);
//   kHPolyF32:  conj(H) as complex FP32 in polyphase order [k-1][a][b],
//               y = a + P b (the pruned FFT along y), row T folded onto row 0
//               (e^{-j 2 pi l T / T} = 1); each lane stores its row's values
//               directly (the item's rows fill whole 32-byte sectors of each
//               (k, a) run in L2), so work units (row, pass) need no barrier
//               (256 threads, two CTAs per SM).
// Items with more corners than the sort holds fall back to exact 64-bit
// fixed-point sums from the integer quarter-wave table (order-free, exact up to
// the table's rounding), written in the same formats.
constexpr int kHY = 64;                 // rows per item
constexpr int kHPassF = 256;            // frequencies per pass (8 per lane)
constexpr int kHCap = 4096;             // corners sorted in shared memory (fast path)
constexpr int kHPairMax = kHCap / 2 + kHY;   // pairs of an item: sum of ceil(n_row / 2)
constexpr int kHLd = kHPassF + 2;       // tile row stride (float2; rows stay 16-byte aligned)
constexpr int kHTabMax = 256;           // two-level table entries per level (T <= 2^16)
constexpr int kHCacheFB = 2048;         // fallback: corners staged in shared memory
constexpr int kHRowsFp16 = 0, kHPolyF32 = 1;
constexpr int kHRankMax = 128;          // items whose rows hold at most this many corners are sorted by rank

template <int FMT>
struct HCfg {
  static constexpr int threads = FMT == kHRowsFp16 ? 512 : 256;
  static constexpr int min_blocks = FMT == kHRowsFp16 ? 1 : 2;
  static constexpr size_t tile = FMT == kHRowsFp16 ? (size_t)kHY * kHLd * 8 : (size_t)kHCap * 4;   // tile | keys
  static constexpr size_t meta = tile;                                  // uint2 [kHPairMax]
  static constexpr size_t cst = meta + (size_t)kHPairMax * 8;           // float4 [kHPairMax]
  static constexpr size_t cst2 = cst + (size_t)kHPairMax * 16;          // float4 [kHPairMax] (kHPolyF32)
  static constexpr size_t tabs = cst2 + (FMT == kHPolyF32 ? (size_t)kHPairMax * 16 : 0);   // float2 [4][kHTabMax]
  static constexpr size_t rows = tabs + (size_t)4 * kHTabMax * 8;       // int [2][kHY + 2]
  static constexpr size_t total = rows + (size_t)2 * (kHY + 2) * 4 + 16;
};

size_t hyb_h_smem(int fmt) { return fmt == kHRowsFp16 ? HCfg<kHRowsFp16>::total : HCfg<kHPolyF32>::total; }

// Two-level tables of e^{j 2 pi p / T} (W) and of the versine D(p) = 1 - e^{j 2 pi p / T}:
// p = u 2^f + v, W(p) = Wc[u] Wf[v].  D uses D(T - q) = conj D(q) to take q <= T/2,
// then D(q) = Dc[i] + Wc[i] Df[b] (q = i 2^f + b): both terms turn by at most a
// right angle from each other, so the sum has no cancellation.
struct HTabs {
  const float2 *Wc, *Wf, *Dc, *Df;
  uint32_t f, fm, T, half;
};
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -(a.y * b.y)), fmaf(a.y, b.x, a.x * b.y));
}
__device__ __forceinline__ float2 tab_w(const HTabs& t, uint32_t p) { return cmul(t.Wc[p >> t.f], t.Wf[p & t.fm]); }
__device__ __forceinline__ float2 tab_d(const HTabs& t, uint32_t p) {
  const bool neg = p > t.half;
  const uint32_t q = neg ? t.T - p : p;
  const float2 c = t.Dc[q >> t.f], w = t.Wc[q >> t.f], d = t.Df[q & t.fm];
  const float im = c.y + fmaf(w.y, d.x, w.x * d.y);
  return make_float2(c.x + fmaf(w.x, d.x, -(w.y * d.y)), neg ? -im : im);
}
// 1 - e^{j theta} from cos and sin: 1 - cos as sin^2 / (1 + cos) where cos >= 0
__device__ __forceinline__ float2 versine(float2 cs) {
  const float re = cs.x >= 0.f ? (cs.y * cs.y) / (1.f + cs.x) : 1.f - cs.x;
  return make_float2(re, -cs.y);
}

// A staged corner of the fallback: the phase k x mod T of every frequency k is
// read at index k u (mod 4 Q) of the level that starts at lbase (quarter period
// Q = 2^lq); sflip = 1 for s = -1.  With decimated levels in shared memory
// (DEC), x = 2^e u reads level e, which keeps the 32 consecutive frequencies of
// a warp on distinct banks; without them every corner reads level 0.
template <bool DEC>
__device__ __forceinline__ int4 stage_corner(uint32_t xm, int sgn, int logQ) {
  int e = 0;
  uint32_t u = xm;
  if (DEC) {
    e = xm ? __ffs(xm) - 1 : 0;
    u = xm >> e;
    if (e > logQ - 1) {   // x a multiple of T/4 (or 0): level 0 reads at most 4 entries
      e = 0;
      u = xm;
    }
  }
  const int lq = logQ - e;
  return make_int4((int)u, level_offset(e, logQ), lq | ((sgn < 0 ? 1 : 0) << 8), 1 << lq);
}

struct HOut {
  __half* hi;       // kHRowsFp16: [clips][2K][ny_pad] hi, then lo
  __half* lo;
  float2* poly;     // kHPolyF32: [K][P][L]
  int logP, L;
};

// Item rows: kHRowsFp16 covers rows y0 .. y0 + 63 of [0, T] (row T its own);
// kHPolyF32 rows y0 .. of [0, T), the corners of row T staged into row 0.
template <int FMT>
__device__ __forceinline__ int item_rows(int y0, int T) {
  return FMT == kHRowsFp16 ? min(kHY, T + 1 - y0) : min(kHY, T - y0);
}

// The corner range(s) of an item in the grouping: [a, b) and, for the
// polyphase item holding row 0, row T's corners [fa, fa + nf) after it.
struct HRange {
  int a, b, fa, nf;
  __device__ __forceinline__ int count() const { return (b - a) + nf; }
  __device__ __forceinline__ int corner(const int* perm, int i) const {
    return i < b - a ? perm[a + i] : perm[fa + i - (b - a)];
  }
};
template <int FMT>
__device__ __forceinline__ HRange item_range(const Groups& g, int y0, int T) {
  HRange r;
  r.a = g.start[min(y0, T + 1)];
  r.b = g.start[min(y0 + kHY, T + 1)];
  r.fa = 0;
  r.nf = 0;
  if (FMT == kHPolyF32 && y0 == 0 && T >= kHY) {   // below one item, row T is already in [a, b)
    r.fa = g.start[T];
    r.nf = g.start[T + 1] - g.start[T];
  }
  return r;
}

// Fallback for an item with more than kHCap corners: exact fixed-point sums,
// thread (group q, frequency t of 128) over the item's y octets q, q + G, ...
// (G = blockDim / 128).  DEC: the decimated levels are in shared memory (lv);
// otherwise level 0 is read from the workspace's fixed-point table.
template <int FMT, bool DEC>
__device__ void h_item_exact(const Plan& pl, const Groups& g, int clip, int y0, const int* lv, int4* vc,
                             int* soff, const HOut& out) {
  const int T = pl.T, K = pl.K, logQ = pl.logT - 2;
  const uint32_t mask = (uint32_t)T - 1u;
  const float inv_q = ldexpf(1.f, -pl.fixq);
  const int small_group = (1 << (31 - pl.fixq)) - 1;   // |sum| < 2^31 in int32
  const int* perm = g.perm;
  const int nrows = item_rows<FMT>(y0, T);
  const HRange rg = item_range<FMT>(g, y0, T);
  const int n = rg.count();
  const bool cached = n <= kHCacheFB;
  for (int i = threadIdx.x; i <= kHY; i += blockDim.x) soff[i] = g.start[min(y0 + i, T + 1)] - rg.a;
  if (cached)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int v = rg.corner(perm, i);
      vc[i] = stage_corner<DEC>((uint32_t)__ldg(pl.vx + v) & mask, (int)__ldg(pl.vsg + v), logQ);
    }
  __syncthreads();
  // row T onto row 0 (polyphase): staged after the item's range, or inside it below one item
  const bool fold = FMT == kHPolyF32 && y0 == 0;
  const int f0 = fold ? (rg.nf ? rg.b - rg.a : soff[min(T, kHY)]) : 0;
  const int f1 = fold ? (rg.nf ? n : soff[min(T + 1, kHY)]) : 0;
  const int G = blockDim.x / 128;
  const int q = threadIdx.x / 128, t = threadIdx.x % 128;
  for (int pass = 0; pass < (K + 127) / 128; ++pass) {
    const int k = pass * 128 + 1 + t;
    if (k > K) continue;
    for (int oc = q; oc < kHY / 8; oc += G) {
      float fcv[8], fsv[8];
#pragma unroll
      for (int yy = 0; yy < 8; ++yy) {
        const int y = oc * 8 + yy;
        auto term = [&](int i, auto& ac_, auto& as_) {
          int4 cn;
          if (cached) {
            cn = vc[i];
          } else {
            const int v = rg.corner(perm, i);
            cn = stage_corner<DEC>((uint32_t)__ldg(pl.vx + v) & mask, (int)__ldg(pl.vsg + v), logQ);
          }
          const int lq = cn.z & 0xFF, Q = cn.w;
          const uint32_t sf = (uint32_t)cn.z >> 8;
          const uint32_t p = ((uint32_t)k * (uint32_t)cn.x) & (4u * (uint32_t)Q - 1u);
          const uint32_t qd = p >> lq, r = p & (uint32_t)(Q - 1);
          const bool odd = qd & 1u;
          const int* L = lv + cn.y;
          const int c = DEC ? L[odd ? Q - r : r] : __ldg(L + (odd ? Q - r : r));
          const int sn = DEC ? L[odd ? r : Q - r] : __ldg(L + (odd ? r : Q - r));
          // cos < 0 in quadrants 1, 2; sin < 0 in quadrants 2, 3; s = -1 flips both
          ac_ += ((((qd + 1u) >> 1) & 1u) ^ sf) ? -c : c;
          as_ += ((qd >> 1) ^ sf) ? -sn : sn;
        };
        int i0 = soff[y], i1 = soff[y + 1], j0 = 0, j1 = 0;
        if (y >= nrows) i1 = i0;
        if (fold && y == 0) {
          j0 = f0;
          j1 = f1;
        }
        long long ac = 0, as = 0;
        if ((i1 - i0) + (j1 - j0) <= small_group) {   // warp-uniform
          int ac32 = 0, as32 = 0;
          for (int i = i0; i < i1; ++i) term(i, ac32, as32);
          for (int i = j0; i < j1; ++i) term(i, ac32, as32);
          ac = ac32;
          as = as32;
        } else {
          for (int i = i0; i < i1; ++i) term(i, ac, as);
          for (int i = j0; i < j1; ++i) term(i, ac, as);
        }
        const float sc = FMT == kHRowsFp16 ? ldexpf(inv_q, -(int)g.ey[y0 + y]) : inv_q;
        fcv[yy] = __ll2float_rn(ac) * sc;
        fsv[yy] = __ll2float_rn(as) * sc;
      }
      if (FMT == kHRowsFp16) {
        uint32_t hc[4], hs[4], lc[4], ls[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          split2h(fcv[2 * qq], fcv[2 * qq + 1], hc[qq], lc[qq]);
          split2h(fsv[2 * qq], fsv[2 * qq + 1], hs[qq], ls[qq]);
        }
        const size_t rc = ((size_t)clip * pl.M2 + 2 * (k - 1)) * pl.ny_pad + y0 + 8 * oc, rs = rc + pl.ny_pad;
        *reinterpret_cast<uint4*>(out.hi + rc) = make_uint4(hc[0], hc[1], hc[2], hc[3]);
        *reinterpret_cast<uint4*>(out.hi + rs) = make_uint4(hs[0], hs[1], hs[2], hs[3]);
        *reinterpret_cast<uint4*>(out.lo + rc) = make_uint4(lc[0], lc[1], lc[2], lc[3]);
        *reinterpret_cast<uint4*>(out.lo + rs) = make_uint4(ls[0], ls[1], ls[2], ls[3]);
      } else {
        const int P = 1 << out.logP;
        for (int yy = 0; yy < 8; ++yy) {
          const int y = y0 + oc * 8 + yy;
          if (oc * 8 + yy >= nrows) break;
          out.poly[((size_t)(k - 1) * P + (y & (P - 1))) * out.L + (y >> out.logP)] = make_float2(fcv[yy], -fsv[yy]);
        }
      }
    }
  }
}

// Fast-path staging of an item: sort keys (row << 17 | x << 1 | sign) (a
// counting sort by row, then ranks within the rows; a bitonic sort of the item
// when a row holds more than kHRankMax corners), the first sorted corner of each
// row (rowc), the first pair of each row (rowp), and
// per pair meta {x_a | kind << 20 | sign_a << 22, w} (kind 0: opposite signs, 1:
// equal, 2: alone) and steps {e^{j 32 x_a}, D_32} (kHPolyF32 also {e^{j 64 x_a},
// D_64} in cst2).
template <int FMT>
__device__ void h_stage(const Plan& pl, const Groups& g, int y0, const HRange& rg, uint32_t* keys, uint32_t* tmp,
                        uint2* meta, float4* cst, float4* cst2, int* rowc, int* rowp, const HTabs& tb) {
  const int T = pl.T, n = rg.count(), tid = threadIdx.x, nt = blockDim.x;
  const uint32_t mask = (uint32_t)T - 1u;
  __shared__ int s_rank;
  // the keys in item order, and the corners per row
  for (int r = tid; r < kHY + 2; r += nt) rowc[r] = 0;
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    const int v = rg.corner(g.perm, i);
    const int yv = __ldg(pl.vy + v);
    const int yl = (FMT == kHPolyF32 && yv == T) ? 0 : yv - y0;
    const uint32_t xm = (uint32_t)__ldg(pl.vx + v) & mask;
    const uint32_t key = ((uint32_t)yl << 17) | (xm << 1) | (__ldg(pl.vsg + v) < 0 ? 1u : 0u);
    tmp[i] = key;
    atomicAdd(&rowc[yl], 1);
  }
  __syncthreads();
  if (tid < 32) {   // rowc = the rows' first sorted positions (two rows a lane), rowp their cursors
    const int c0 = rowc[2 * tid], c1 = rowc[2 * tid + 1];
    int incl = c0 + c1, mx = max(c0, c1);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t2 = __shfl_up_sync(0xffffffffu, incl, o);
      if (tid >= o) incl += t2;
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int ex = incl - c0 - c1;
    rowc[2 * tid] = rowp[2 * tid] = ex;
    rowc[2 * tid + 1] = rowp[2 * tid + 1] = ex + c0;
    if (tid == 31) rowc[kHY] = incl;
    if (tid == 0) s_rank = mx <= kHRankMax ? 1 : 0;
  }
  __syncthreads();
  if (s_rank) {
    // a counting sort by row, then each corner placed at its rank among its row's
    // keys (equal keys are equal corners: their order does not matter)
    for (int i = tid; i < n; i += nt) {
      const uint32_t key = tmp[i];
      keys[atomicAdd(&rowp[key >> 17], 1)] = key;
    }
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
      const uint32_t key = keys[i];
      const int r = (int)(key >> 17), b = rowc[r], e = rowc[r + 1];
      int rank = 0;
      for (int j = b; j < e; ++j) {
        const uint32_t kj = keys[j];
        rank += (kj < key || (kj == key && j < i)) ? 1 : 0;
      }
      tmp[b + rank] = key;
    }
    __syncthreads();
    for (int i = tid; i < n; i += nt) keys[i] = tmp[i];
  } else {
    // rows of many corners: a bitonic sort of the whole item
    int npad = 1;
    while (npad < n) npad <<= 1;
    for (int i = tid; i < npad; i += nt) keys[i] = i < n ? tmp[i] : 0xFFFFFFFFu;
    __syncthreads();
    for (int kk = 2; kk <= npad; kk <<= 1)
      for (int j = kk >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < npad; i += nt) {
          const int ixj = i ^ j;
          if (ixj > i) {
            const uint32_t u = keys[i], w = keys[ixj];
            if ((u > w) == ((i & kk) == 0)) {
              keys[i] = w;
              keys[ixj] = u;
            }
          }
        }
        __syncthreads();
      }
  }
  __syncthreads();
  if (tid < 32) {   // rowp = exclusive scan of ceil(n_row / 2) over the 64 rows
    const int c0 = (rowc[2 * tid + 1] - rowc[2 * tid] + 1) >> 1;
    const int c1 = (rowc[2 * tid + 2] - rowc[2 * tid + 1] + 1) >> 1;
    int incl = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t2 = __shfl_up_sync(0xffffffffu, incl, o);
      if (tid >= o) incl += t2;
    }
    rowp[2 * tid] = incl - c0 - c1;
    rowp[2 * tid + 1] = incl - c1;
    if (tid == 31) rowp[kHY] = incl;
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    const uint32_t ka = keys[i];
    const int r = (int)(ka >> 17), pos = i - rowc[r];
    if (pos & 1) continue;
    const uint32_t xa = (ka >> 1) & 0xFFFFu, sa = ka & 1u;
    uint32_t kind = 2u, w = 0u;
    if (i + 1 < rowc[r + 1]) {
      const uint32_t kb2 = keys[i + 1];
      w = ((kb2 >> 1) & 0xFFFFu) - xa;
      kind = (kb2 & 1u) == sa ? 1u : 0u;
    }
    const int p = rowp[r] + (pos >> 1);
    meta[p] = make_uint2(xa | (kind << 20) | (sa << 22), w);
    const float2 S = tab_w(tb, (32u * xa) & mask), D = tab_d(tb, (32u * w) & mask);
    cst[p] = make_float4(S.x, S.y, D.x, D.y);
    if (FMT == kHPolyF32) {
      const float2 S2 = tab_w(tb, (64u * xa) & mask), D2 = tab_d(tb, (64u * w) & mask);
      cst2[p] = make_float4(S2.x, S2.y, D2.x, D2.y);
    }
  }
  __syncthreads();   // the keys are dead from here on
}

// The 8 sums of one row for frequencies k0 + 32 i (acc zeroed by the caller).
__device__ __forceinline__ void row_sums(const uint2* __restrict__ meta, const float4* __restrict__ cst, int p0,
                                         int p1, uint32_t k0, uint32_t mask, const HTabs& tb, float2 (&acc)[8]) {
  for (int p = p0; p < p1; ++p) {
    const uint2 pr = meta[p];
    const float4 c = cst[p];
    const uint32_t xa = pr.x & 0xFFFFFu, kind = (pr.x >> 20) & 3u, w = pr.y;
    const float2 S = make_float2(c.x, c.y);
    float2 A = tab_w(tb, (k0 * xa) & mask);
    if (pr.x >> 22) A = make_float2(-A.x, -A.y);
    if (kind == 2u) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        acc[j].x += A.x;
        acc[j].y += A.y;
        A = cmul(A, S);
      }
    } else {
      // D_{k+32} = D_k + D_32 - D_k D_32 = D_32 + D_k C, C = 1 - D_32 = e^{j 32 w}
      // (four FMAs); kind is uniform over the warp (one row, one pair at a time)
      const float2 D1 = make_float2(c.z, c.w), C = make_float2(1.f - c.z, -c.w);
      float2 D = tab_d(tb, (k0 * w) & mask);
      if (kind == 0u) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          acc[j].x = fmaf(A.x, D.x, fmaf(-A.y, D.y, acc[j].x));
          acc[j].y = fmaf(A.x, D.y, fmaf(A.y, D.x, acc[j].y));
          A = cmul(A, S);
          D = make_float2(fmaf(D.x, C.x, fmaf(-D.y, C.y, D1.x)), fmaf(D.x, C.y, fmaf(D.y, C.x, D1.y)));
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float2 E = make_float2(2.f - D.x, -D.y);
          acc[j].x = fmaf(A.x, E.x, fmaf(-A.y, E.y, acc[j].x));
          acc[j].y = fmaf(A.x, E.y, fmaf(A.y, E.x, acc[j].y));
          A = cmul(A, S);
          D = make_float2(fmaf(D.x, C.x, fmaf(-D.y, C.y, D1.x)), fmaf(D.x, C.y, fmaf(D.y, C.x, D1.y)));
        }
      }
    }
  }
}

// Packed FP32 pairs: ffma2 / fmul2 (fcfs_fft.cuh); dup broadcasts a value to both halves.
__device__ __forceinline__ float2 dup(float v) { return make_float2(v, v); }

// The 8 sums of one row as in row_sums, the lane's frequencies taken two at a
// time, k0 + 32 j and k0 + 32 (j + 1) for j = 0, 2, 4, 6, in the halves of packed
// f32x2 operations: re[j / 2] = (Re_j, Re_{j+1}), im[j / 2] likewise (zeroed by
// the caller).  Both chains start from the table anchor at k0 and its exact-step
// successor at k0 + 32 (A_{k+32} = A_k e^{j 32 x_a}, D_{k+32} = D_32 + D_k e^{j 32 w})
// and step by 64 frequencies: A_{k+64} = A_k S^2 and D_{k+64} = D_64 + D_k C^2,
// with S^2 = e^{j 64 x_a} and D_64 from the tables (staged per pair) and
// C^2 = e^{j 64 w} = 1 - D_64: half the steps of the scalar chains.  The
// opposite-sign product Re(A D) = A_x D_x - A_y D_y has its negative part summed
// on its own (q) and taken off at the end of the row; the rare equal-sign pairs
// take scalar FMAs on the halves.
__device__ __forceinline__ void row_sums_x2(const uint2* __restrict__ meta, const float4* __restrict__ cst,
                                            const float4* __restrict__ cst2, int p0, int p1, uint32_t k0,
                                            uint32_t mask, const HTabs& tb, float2 (&re)[4], float2 (&im)[4]) {
  float2 q[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) q[j] = make_float2(0.f, 0.f);
  for (int p = p0; p < p1; ++p) {
    const uint2 pr = meta[p];
    const float4 c = cst[p];
    const float4 c2 = cst2[p];
    const uint32_t xa = pr.x & 0xFFFFFu, kind = (pr.x >> 20) & 3u, w = pr.y;
    const float2 S = make_float2(c.x, c.y);
    float2 A0 = tab_w(tb, (k0 * xa) & mask);
    if (pr.x >> 22) A0 = make_float2(-A0.x, -A0.y);
    const float2 A1 = cmul(A0, S);
    float2 ax = make_float2(A0.x, A1.x), ay = make_float2(A0.y, A1.y);
    const float2 s2x = dup(c2.x), s2y = dup(c2.y), ns2y = dup(-c2.y);
    if (kind == 2u) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        re[j] = ffma2(ax, dup(1.f), re[j]);
        im[j] = ffma2(ay, dup(1.f), im[j]);
        if (j < 3) {
          const float2 nx = ffma2(ay, ns2y, fmul2(ax, s2x));
          ay = ffma2(ay, s2x, fmul2(ax, s2y));
          ax = nx;
        }
      }
      continue;
    }
    const float2 D32 = make_float2(c.z, c.w), C = make_float2(1.f - c.z, -c.w);
    const float2 D0 = tab_d(tb, (k0 * w) & mask);
    const float2 D1 = make_float2(fmaf(D0.x, C.x, fmaf(-D0.y, C.y, D32.x)), fmaf(D0.x, C.y, fmaf(D0.y, C.x, D32.y)));
    const float2 c2x = dup(1.f - c2.z), c2y = dup(-c2.w), nc2y = dup(c2.w);
    const float2 d64x = dup(c2.z), d64y = dup(c2.w);
    float2 dx = make_float2(D0.x, D1.x), dy = make_float2(D0.y, D1.y);
    // kind is uniform over the warp (one row, one pair at a time)
    if (kind == 0u) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        re[j] = ffma2(ax, dx, re[j]);
        q[j] = ffma2(ay, dy, q[j]);
        im[j] = ffma2(ax, dy, ffma2(ay, dx, im[j]));
        if (j < 3) {
          const float2 nx = ffma2(ay, ns2y, fmul2(ax, s2x));
          ay = ffma2(ay, s2x, fmul2(ax, s2y));
          ax = nx;
          const float2 ex = ffma2(dy, nc2y, ffma2(dx, c2x, d64x));
          dy = ffma2(dy, c2x, ffma2(dx, c2y, d64y));
          dx = ex;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        // A (2 - D) on each half
        const float ex0 = 2.f - dx.x, ey0 = -dy.x, ex1 = 2.f - dx.y, ey1 = -dy.y;
        re[j].x = fmaf(ax.x, ex0, fmaf(-ay.x, ey0, re[j].x));
        im[j].x = fmaf(ax.x, ey0, fmaf(ay.x, ex0, im[j].x));
        re[j].y = fmaf(ax.y, ex1, fmaf(-ay.y, ey1, re[j].y));
        im[j].y = fmaf(ax.y, ey1, fmaf(ay.y, ex1, im[j].y));
        if (j < 3) {
          const float2 nx = ffma2(ay, ns2y, fmul2(ax, s2x));
          ay = ffma2(ay, s2x, fmul2(ax, s2y));
          ax = nx;
          const float2 ex = ffma2(dy, nc2y, ffma2(dx, c2x, d64x));
          dy = ffma2(dy, c2x, ffma2(dx, c2y, d64y));
          dx = ex;
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) re[j] = ffma2(q[j], dup(-1.f), re[j]);
}

// kHRowsFp16 fast path: passes of 256 frequencies over the item's 64 rows into
// the tile, written out as FP16 hi/lo row segments.
__device__ void h_rows_fp16(const Plan& pl, int clip, int y0, float2* tile, const uint2* meta, const float4* cst,
                            const int* rowp, int* s_row, const HTabs& tb, const HOut& out) {
  const int T = pl.T, K = pl.K, tid = threadIdx.x, lane = tid & 31;
  const uint32_t mask = (uint32_t)T - 1u;
  const int nrows = item_rows<kHRowsFp16>(y0, T);
  const int npass = (K + kHPassF - 1) / kHPassF;
  for (int pass = 0; pass < npass; ++pass) {
    const int kb = pass * kHPassF + 1;
    if (tid == 0) *s_row = 0;
    __syncthreads();
    const uint32_t k0 = (uint32_t)(kb + lane);
    for (;;) {
      int r = 0;
      if (lane == 0) r = atomicAdd(s_row, 1);
      r = __shfl_sync(0xffffffffu, r, 0);
      if (r >= kHY) break;
      float2 acc[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = make_float2(0.f, 0.f);
      if ((int)k0 <= K && r < nrows) row_sums(meta, cst, rowp[r], rowp[r + 1], k0, mask, tb, acc);
      float2* row = tile + (size_t)r * kHLd + lane;
#pragma unroll
      for (int j = 0; j < 8; ++j) row[32 * j] = acc[j];
    }
    __syncthreads();
    for (int e = tid; e < kHPassF * (kHY / 8); e += blockDim.x) {
      const int kl = e % kHPassF, oc = e / kHPassF, k = kb + kl;
      if (k > K) continue;
      float fcv[8], fsv[8];
#pragma unroll
      for (int yy = 0; yy < 8; ++yy) {
        const float2 v = tile[(size_t)(oc * 8 + yy) * kHLd + kl];
        fcv[yy] = v.x;
        fsv[yy] = v.y;
      }
      uint32_t hc[4], hs[4], lc[4], ls[4];
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) {
        split2h(fcv[2 * qq], fcv[2 * qq + 1], hc[qq], lc[qq]);
        split2h(fsv[2 * qq], fsv[2 * qq + 1], hs[qq], ls[qq]);
      }
      const size_t rc = ((size_t)clip * pl.M2 + 2 * (k - 1)) * pl.ny_pad + y0 + 8 * oc, rs = rc + pl.ny_pad;
      *reinterpret_cast<uint4*>(out.hi + rc) = make_uint4(hc[0], hc[1], hc[2], hc[3]);
      *reinterpret_cast<uint4*>(out.hi + rs) = make_uint4(hs[0], hs[1], hs[2], hs[3]);
      *reinterpret_cast<uint4*>(out.lo + rc) = make_uint4(lc[0], lc[1], lc[2], lc[3]);
      *reinterpret_cast<uint4*>(out.lo + rs) = make_uint4(ls[0], ls[1], ls[2], ls[3]);
    }
    __syncthreads();
  }
}

// kHPolyF32 fast path: work units (residue a, group of 4 b, pass) from a
// counter.  A warp sums the unit's 4 rows y = a + P b (consecutive b), so each
// lane ends with 4 consecutive b of each of its 8 frequencies: one 32-byte
// sector of conj(H)[k-1][a][.] per frequency, stored directly.
__device__ void h_poly_direct(const Plan& pl, int y0, const uint2* meta, const float4* cst, const float4* cst2,
                              const int* rowp, int* s_row, const HTabs& tb, const HOut& out) {
  const int T = pl.T, K = pl.K, lane = threadIdx.x & 31;
  const uint32_t mask = (uint32_t)T - 1u;
  const int nrows = item_rows<kHPolyF32>(y0, T);
  const int npass = (K + kHPassF - 1) / kHPassF;
  const int logP = out.logP, P = 1 << logP;
  const int nb = nrows >> logP;            // b values of each residue in this item
  const int ngrp = (nb + 3) >> 2;
  const int nunit = P * ngrp;              // per pass
  const size_t b0 = (size_t)(y0 >> logP);
  if (threadIdx.x == 0) *s_row = 0;
  __syncthreads();
  for (;;) {
    int u = 0;
    if (lane == 0) u = atomicAdd(s_row, 1);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= nunit * npass) break;
    const int pass = u / nunit, w = u % nunit, a = w % P, grp = w / P;
    const uint32_t k0 = (uint32_t)(pass * kHPassF + 1 + lane);
    if ((int)k0 > K) continue;   // lanes past K (last pass) idle; nothing below is warp-collective
    float2 re[4][4], im[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) re[i][j] = im[i][j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int bl = 4 * grp + i;
      if (bl < nb) {
        const int r = a + (bl << logP);
        row_sums_x2(meta, cst, cst2, rowp[r], rowp[r + 1], k0, mask, tb, re[i], im[i]);
      }
    }
    // frequency k0 + 32 j of row i: (re, im)[i][j / 2], half j mod 2
    float2 acc[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[i][2 * j] = make_float2(re[i][j].x, im[i][j].x);
        acc[i][2 * j + 1] = make_float2(re[i][j].y, im[i][j].y);
      }
    const size_t kstride = (size_t)32 * T;   // 32 frequencies further on
    float2* dst = out.poly + ((size_t)(k0 - 1) * P + a) * out.L + b0 + 4 * grp;
    if (4 * grp + 4 <= nb) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if ((int)k0 + 32 * j > K) break;
        float4* d4 = reinterpret_cast<float4*>(dst + j * kstride);
        d4[0] = make_float4(acc[0][j].x, -acc[0][j].y, acc[1][j].x, -acc[1][j].y);
        d4[1] = make_float4(acc[2][j].x, -acc[2][j].y, acc[3][j].x, -acc[3][j].y);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if ((int)k0 + 32 * j > K) break;
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (4 * grp + i < nb) dst[j * kstride + i] = make_float2(acc[i][j].x, -acc[i][j].y);
      }
    }
  }
}

// Items (clip, 64-row chunk) are taken from a work counter (clips differ in
// size by orders of magnitude, so a static split leaves CTAs idle).
template <int FMT>
__global__ void __launch_bounds__(HCfg<FMT>::threads, HCfg<FMT>::min_blocks)
    hyb_h_kernel(Plan pl, uint8_t* ws, HOut out) {
  using C = HCfg<FMT>;
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ int s_item, s_row;
  const int T = pl.T, logT = pl.logT;
  uint32_t* keys = reinterpret_cast<uint32_t*>(sm);
  float2* tile = reinterpret_cast<float2*>(sm);
  uint2* meta = reinterpret_cast<uint2*>(sm + C::meta);
  float4* cst = reinterpret_cast<float4*>(sm + C::cst);
  float4* cst2 = reinterpret_cast<float4*>(sm + C::cst2);
  // the staging's second key array: behind the keys in the tile (kHRowsFp16), the
  // second step array (kHPolyF32); both are written only after the staging
  uint32_t* tmp = reinterpret_cast<uint32_t*>(sm + (FMT == kHRowsFp16 ? (size_t)kHCap * 4 : C::cst2));
  float2* tabs = reinterpret_cast<float2*>(sm + C::tabs);
  int* rowc = reinterpret_cast<int*>(sm + C::rows);
  int* rowp = rowc + kHY + 2;
  const int nclips = pl.batch ? pl.n_clips : 1;
  unsigned* counter = reinterpret_cast<unsigned*>(ws + kSyncOffset) + 2;   // zeroed by the prep kernel

  // two-level W and D tables from the FP32 sincos table
  const uint32_t f = ((uint32_t)logT + 1u) / 2u, nf = 1u << f, nc = (uint32_t)T >> f;
  float2 *Wc = tabs, *Wf = tabs + kHTabMax, *Dc = tabs + 2 * kHTabMax, *Df = tabs + 3 * kHTabMax;
  {
    const float* gt = reinterpret_cast<const float*>(ws + pl.off_tab_f32);
    const uint32_t logQ = (uint32_t)logT - 2u;
    for (uint32_t i = threadIdx.x; i < nc + nf; i += blockDim.x) {
      const bool coarse = i < nc;
      const uint32_t u = coarse ? i : i - nc;
      const uint32_t p = coarse ? u << f : u;
      const float2 w = pl.full ? f32_lookup<true>(gt, p, logQ) : f32_lookup<false>(gt, p, logQ);
      (coarse ? Wc : Wf)[u] = w;
      (coarse ? Dc : Df)[u] = versine(w);
    }
  }
  const HTabs tb{Wc, Wf, Dc, Df, f, nf - 1u, (uint32_t)T, (uint32_t)T / 2u};
  const int nchunk = FMT == kHRowsFp16 ? pl.ny_pad / kHY : max(1, T / kHY);
  const long long nitems = (long long)nclips * nchunk;
  bool levels = false;   // the fallback's decimated levels are in shared memory
  for (;;) {
    __syncthreads();   // the previous item's readers are done (and the tables are built)
    if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int cu = s_item;   // (clip, chunk)
    if (cu >= nitems) break;
    const int clip = cu / nchunk, chunk = cu % nchunk;
    const int y0 = chunk * kHY;
    const Groups g = pl.batch ? groups_clip(ws + pl.off_ycnt, T, pl.ny_pad, nclips, clip, pl.V)
                              : groups_at(ws + pl.off_ycnt, T, pl.ny_pad);
    const HRange rg = item_range<FMT>(g, y0, T);
    if (rg.count() <= kHCap) {
      levels = false;   // the fast path overwrites them
      h_stage<FMT>(pl, g, y0, rg, keys, tmp, meta, cst, cst2, rowc, rowp, tb);
      if (FMT == kHRowsFp16)
        h_rows_fp16(pl, clip, y0, tile, meta, cst, rowp, &s_row, tb, out);
      else
        h_poly_direct(pl, y0, meta, cst, cst2, rowp, &s_row, tb, out);
    } else if (FMT == kHRowsFp16) {
      // level 0 = the fixed-point quarter-wave table, then the decimated levels
      int* lv = reinterpret_cast<int*>(sm);
      int4* vc = reinterpret_cast<int4*>(sm + align_up(axis_levels_ints(T) * 4, 16));
      if (!levels) {
        const int* tq = reinterpret_cast<const int*>(ws + pl.off_tab_fix);
        for (int i = threadIdx.x; i <= T / 4; i += blockDim.x) lv[i] = tq[i];
        __syncthreads();
        axis_build_levels(lv, T, logT);
        __syncthreads();
        levels = true;
      }
      h_item_exact<FMT, true>(pl, g, clip, y0, lv, vc, rowc, out);
    } else {
      h_item_exact<FMT, false>(pl, g, clip, y0, reinterpret_cast<const int*>(ws + pl.off_tab_fix),
                               reinterpret_cast<int4*>(sm), rowc, out);
    }
  }
}

// ---------------------------------------------------------------------------
// Stage 3: the contraction over y on CTA pairs
// ---------------------------------------------------------------------------
constexpr int kGS = 3;                   // stages
constexpr int kGGroup = 64;              // generator threads per chunk: 8 y octets x 8 runs of 8 frequencies
constexpr int kGGen = kGS * kGGroup;     // group g fills the chunks of stage g
constexpr int kGThreads = kGGen + 64;    // + MMA warp + TMA warp
constexpr int kGTile = 128 * 128;        // one 128-row FP16 tile of a chunk (hi or lo), bytes
constexpr int kGStage = 4 * kGTile;      // H hi, H lo (TMA), B hi, B lo (generated)
constexpr int kGOps = kGS * kGStage;
constexpr int kTlMax = 512;              // two-level table entries for T <= 2^16
constexpr size_t kGSmem = 1024 + kGOps + kTlMax * 8 + 256;

__device__ __forceinline__ void st_shared_v4h(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ void ld_shared_v4h(uint32_t addr, uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d) {
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(a), "=r"(b), "=r"(c), "=r"(d) : "r"(addr) : "memory");
}
__device__ __forceinline__ void tma_load_2dh(void* dst, const CUtensorMap* map, int32_t c0, int32_t c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}
// (cos, sin)(2 pi p / T) = coarse[p >> f] * fine[p mod 2^f] (correctly rounded FP32 factors)
struct TwoLevelH {
  const float2* t;
  uint32_t f, fmask, nc;
};
__device__ __forceinline__ float2 tl_lookup_h(const TwoLevelH& tl, uint32_t p) {
  const float2 c = tl.t[p >> tl.f], d = tl.t[tl.nc + (p & tl.fmask)];
  return make_float2(fmaf(c.x, d.x, -(c.y * d.y)), fmaf(c.y, d.x, c.x * d.y));
}

// blockIdx.x = 2 (pair tile) + rank, blockIdx.y = y split.  Rank r holds H
// rows [128 tm, 128 tm + 128) (tm = 2 (pair tile / tiles_n) + r) and the B
// rows of frequencies l in tn 128 + 64 r + [1, 64].
__global__ void __launch_bounds__(kGThreads, 1)
    hyb_gemm_kernel(const __grid_constant__ CUtensorMap hhi, const __grid_constant__ CUtensorMap hlo, Plan pl,
                    uint8_t* ws) {
  constexpr int GW = kGGen / 32;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint8_t* ops = sm;
  float2* tlt = reinterpret_cast<float2*>(sm + kGOps);
  uint64_t* ofull = reinterpret_cast<uint64_t*>(tlt + kTlMax);   // [kGS] rank 0: chunk ready in both CTAs
  uint64_t* tfull = ofull + kGS;                                 // [kGS] this CTA's H tiles landed
  uint64_t* empty = tfull + kGS;                                 // [kGS] the chunk's MMAs completed
  uint64_t* accfull = empty + kGS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accfull + 1);

  Status* st = reinterpret_cast<Status*>(ws + pl.off_status);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_ctarank();
  const int ptile = blockIdx.x >> 1;
  const int tm = 2 * (ptile / pl.tiles_n) + (int)rank, tn = ptile % pl.tiles_n;
  const int y0 = blockIdx.y * (int)pl.split_len;
  const int y1 = min(pl.ny_pad, y0 + (int)pl.split_len);
  const int nch = max(0, (y1 - y0) / 64);
  const int clip = blockIdx.z;   // batch: the clip; 0 for a single clip

  if (tid == kGGen + 32) {
    for (int i = 0; i < kGS; ++i) {
      mbar_init(&ofull[i], 2 * (kGGroup / 32) + 1);   // one group's warps in both CTAs, rank 1's forwarder
      mbar_init(&tfull[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(accfull, 1);
    fence_mbar_init();
  }
  if (warp == GW) {   // collective with the peer's MMA warp: D1 at 0, D2 at 256
    tmem_alloc_pair(tmem_slot, 512);
    tmem_relinquish_pair();
  }
  const uint32_t logT = (uint32_t)pl.logT, f = (logT + 1u) / 2u, nc = 1u << (logT - f);
  const TwoLevelH tl{tlt, f, (1u << f) - 1u, nc};
  if (tid < kGGen) {
    const float* gt = reinterpret_cast<const float*>(ws + pl.off_tab_f32);
    const uint32_t logQ = logT - 2u;
    for (uint32_t i = tid; i < nc + (1u << f); i += kGGen) {
      const uint32_t p = i < nc ? i << f : i - nc;
      tlt[i] = pl.full ? f32_lookup<true>(gt, p, logQ) : f32_lookup<false>(gt, p, logQ);
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == GW + 1) {
    // ---------------- H tiles (TMA) ----------------
    if (lane == 0) {
      prefetch_tensormap(&hhi);
      prefetch_tensormap(&hlo);
      int j = 0;
      for (; j < nch; ++j) {
        const int s = j % kGS;
        const uint32_t ph = (uint32_t)(j / kGS) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, st, 60)) break;
        uint8_t* at = ops + (size_t)s * kGStage;
        mbar_arrive_expect_tx(&tfull[s], 2u * kGTile);
        // rows past the last clip's 2K read as zeros; a tile's rows past 2K of
        // another clip only feed partial rows that are never stored
        tma_load_2dh(at, &hhi, y0 + j * 64, clip * pl.M2 + tm * 128, &tfull[s]);
        tma_load_2dh(at + kGTile, &hlo, y0 + j * 64, clip * pl.M2 + tm * 128, &tfull[s]);
      }
      for (int q = max(0, j - kGS); q < j; ++q) mbar_wait(&tfull[q % kGS], (uint32_t)(q / kGS) & 1u, st, 61);
    }
  } else if (warp == GW) {
    if (lane == 0 && rank == 0) {
      // ---------------- MMA issuer (rank 0 for the pair) ----------------
      constexpr uint32_t idesc = idesc_f16_f32(256, 256);
      const uint32_t ops_a = smem_u32(ops);
      for (int j = 0; j < nch; ++j) {
        const int s = j % kGS;
        const uint32_t ph = (uint32_t)(j / kGS) & 1u;
        if (!mbar_wait_cluster(&ofull[s], ph, st, 62) || !mbar_wait(&tfull[s], ph, st, 63)) break;
        tc_fence_after();
        const uint32_t ahi = ops_a + s * kGStage, alo = ahi + kGTile, bhi = alo + kGTile, blo = bhi + kGTile;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t o = ks * 32;
          const uint64_t dah = sdesc_sw128(ahi + o), dal = sdesc_sw128(alo + o);
          const uint64_t dbh = sdesc_sw128(bhi + o), dbl = sdesc_sw128(blo + o);
          tc_mma_f16_pair(tmem, dah, dbh, idesc, (j | ks) != 0);
          tc_mma_f16_pair(tmem + 256, dah, dbl, idesc, (j | ks) != 0);
          tc_mma_f16_pair(tmem + 256, dal, dbh, idesc, 1);
        }
        tc_commit_pair(&empty[s]);
      }
      tc_commit_pair(accfull);
    } else if (lane == 0) {
      // rank 1: each chunk's H tiles have landed here -> count it on rank 0's barrier
      for (int j = 0; j < nch; ++j) {
        const int s = j % kGS;
        if (!mbar_wait(&tfull[s], (uint32_t)(j / kGS) & 1u, st, 64)) break;
        mbar_arrive_cluster(&ofull[s], 0);
      }
    }
  } else {
    // ---------------- generators: B rows of this CTA ----------------
    const int group = tid / kGGroup, gtid = tid % kGGroup;
    const int oct = gtid & 7, run = gtid >> 3;
    const int i0 = 8 * run;   // first row pair of the run in this CTA's B tile
    const uint32_t f0 = (uint32_t)(tn * 128 + (int)rank * 64 + 1 + i0);
    const uint32_t mask = (uint32_t)pl.T - 1u;
    const uint32_t ops_a = smem_u32(ops);
    const Groups yg = pl.batch ? groups_clip(ws + pl.off_ycnt, pl.T, pl.ny_pad, pl.n_clips, clip, pl.V)
                               : groups_at(ws + pl.off_ycnt, pl.T, pl.ny_pad);
    uint32_t xo[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) xo[c] = (uint32_t)((oct ^ c) << 4);
    for (int j = group; j < nch; j += kGS) {
      const int s = j % kGS;
      const uint32_t ph = (uint32_t)(j / kGS) & 1u;
      const int yb = y0 + j * 64 + oct * 8;   // this thread's 8 consecutive y
      const uint2 ex = __ldg(reinterpret_cast<const uint2*>(yg.ey + yb));
      float c[8], sn[8], wc[8], wsn[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const uint32_t yv = (uint32_t)(yb + t);
        const float2 an = tl_lookup_h(tl, (f0 * yv) & mask);
        const float2 w = tl_lookup_h(tl, yv & mask);
        const int e = (int)(int8_t)(((t < 4 ? ex.x : ex.y) >> (8 * (t & 3))) & 0xFFu);
        const float sc = ldexpf(1.f, e);   // undoes H's 2^-e_y exactly
        c[t] = an.x * sc;
        sn[t] = an.y * sc;
        wc[t] = w.x;
        wsn[t] = w.y;
      }
      if (!__all_sync(0xffffffffu, mbar_wait(&empty[s], ph ^ 1u, st, 65) ? 1 : 0)) break;
      const uint32_t tile_hi = ops_a + s * kGStage + 2u * kGTile + 256u * (uint32_t)i0;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        if (r) {
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const float ncs = fmaf(c[t], wc[t], -(sn[t] * wsn[t]));
            const float nsn = fmaf(sn[t], wc[t], c[t] * wsn[t]);
            c[t] = ncs;
            sn[t] = nsn;
          }
        }
        uint32_t ch[4], cl[4], sh[4], sl[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          split2h(c[2 * qq], c[2 * qq + 1], ch[qq], cl[qq]);
          split2h(sn[2 * qq], sn[2 * qq + 1], sh[qq], sl[qq]);
        }
        // cos row 2(i0 + r) and sin row 2(i0 + r) + 1 of the hi and lo tiles
        const uint32_t rc = tile_hi + 256u * r + xo[(2 * r) & 7];
        const uint32_t rs = tile_hi + 256u * r + 128u + xo[(2 * r + 1) & 7];
        st_shared_v4h(rc, ch[0], ch[1], ch[2], ch[3]);
        st_shared_v4h(rs, sh[0], sh[1], sh[2], sh[3]);
        st_shared_v4h(rc + kGTile, cl[0], cl[1], cl[2], cl[3]);
        st_shared_v4h(rs + kGTile, sl[0], sl[1], sl[2], sl[3]);
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(&ofull[s], 0);
    }

    // ---------------- epilogue: TMEM -> FP32 partial tile (warps 0-3) ----------------
    // Warp w drains TMEM lanes 32 w .. (tile rows) over the 256 columns; each
    // 32 x 32 block goes through a padded shared-memory transpose (row stride
    // 36 floats) so that the global stores cover whole 128-byte rows.  The
    // operand stages are free: the last MMA has completed.
    if (warp < 4) {
      const bool acc_ok = __all_sync(0xffffffffu, mbar_wait(accfull, 0, st, 66) ? 1 : 0) != 0;
      tc_fence_after();
      const int M2 = pl.M2;
      const int row0 = warp * 32;
      const uint32_t tr = smem_u32(ops) + (uint32_t)warp * (32u * 36u * 4u);
      float* P = reinterpret_cast<float*>(ws + pl.off_part) + ((size_t)clip * pl.splits + blockIdx.y) * M2 * M2;
#pragma unroll 1
      for (int cb = 0; cb < 8; ++cb) {
        const int n0 = tn * 256 + cb * 32;
        if (n0 >= M2) break;   // warp-uniform
        uint32_t r[32];
        if (acc_ok && nch > 0) {
          uint32_t r2[32];
          tmem_ld32(tmem + ((uint32_t)row0 << 16) + (uint32_t)(cb * 32), r);
          tmem_ld32(tmem + ((uint32_t)row0 << 16) + (uint32_t)(256 + cb * 32), r2);
          tmem_wait_ld();
#pragma unroll
          for (int qq = 0; qq < 32; ++qq) r[qq] = __float_as_uint(__uint_as_float(r[qq]) + __uint_as_float(r2[qq]));
        } else {
#pragma unroll
          for (int qq = 0; qq < 32; ++qq) r[qq] = 0u;
        }
#pragma unroll
        for (int qq = 0; qq < 8; ++qq)
          st_shared_v4h(tr + (uint32_t)(lane * 36 + 4 * qq) * 4u, r[4 * qq], r[4 * qq + 1], r[4 * qq + 2],
                        r[4 * qq + 3]);
        __syncwarp();
        const int c4 = lane & 7;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int rr = 4 * i + (lane >> 3);
          const int m = tm * 128 + row0 + rr, n = n0 + 4 * c4;
          uint32_t v0, v1, v2, v3;
          ld_shared_v4h(tr + (uint32_t)(rr * 36 + 4 * c4) * 4u, v0, v1, v2, v3);
          if (m < M2 && n < M2) {
            float* dst = P + (size_t)m * M2 + n;
            if (n + 4 <= M2 && (M2 & 3) == 0) {   // 16-byte aligned rows only when 2K is a multiple of 4
              *reinterpret_cast<float4*>(dst) =
                  make_float4(__uint_as_float(v0), __uint_as_float(v1), __uint_as_float(v2), __uint_as_float(v3));
            } else {
              const uint32_t vv[4] = {v0, v1, v2, v3};
              for (int t = 0; t < 4 && n + t < M2; ++t) dst[t] = __uint_as_float(vv[t]);
            }
          }
        }
        __syncwarp();
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  if (warp == GW) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc_pair(tmem, 512);
  }
}

}  // namespace

size_t hybrid_extra_bytes(int64_t V, int T, int M2, int ny_pad, size_t& off_ycnt, size_t& off_h, size_t base) {
  size_t o = base;
  off_ycnt = o;
  o = align_up(o + group_bytes(V, T, ny_pad), kWsAlign);
  off_h = o;
  o = align_up(o + (size_t)2 * M2 * ny_pad * 2, kWsAlign);
  return o;
}

cudaError_t launch_grouping(const int32_t* c0, const int32_t* c1, int64_t V, int T, int ny_pad, uint8_t* base,
                            cudaStream_t st, int key_logP) {
  const int nc = c1 ? 2 : 1;
  const size_t gb = group_bytes(V, T, ny_pad);
  for (int i = 0; i < nc; ++i) {
    const cudaError_t e = cudaMemsetAsync(base + i * gb, 0, (size_t)group_stride(T) * 4, st);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int vblocks = (int)std::max<long long>(1, std::min<long long>((V + 255) / 256, 8LL * sms));
  cudaError_t e;
  if ((e = launch_after(group_count_kernel, dim3(vblocks, nc), dim3(256), 0, st, c0, c1, (long long)V, T, ny_pad,
                        base, key_logP)) != cudaSuccess)
    return e;
  const int rounds = scan_rounds(T);
  auto scan = rounds <= 1 ? group_scan_kernel<1> : rounds <= 4 ? group_scan_kernel<4> : group_scan_kernel<kScanRounds>;
  if ((e = launch_after(scan, dim3(nc), dim3(kScanThreads), 0, st, (long long)V, T, ny_pad, base)) != cudaSuccess)
    return e;
  return launch_after(group_scatter_kernel, dim3(vblocks, nc), dim3(256), 0, st, c0, c1, (long long)V, T, ny_pad,
                      base, key_logP);
}

// Group the corners of a single clip or of every clip of a batch by y.
static cudaError_t group_rows(const Plan& pl, uint8_t* ws, cudaStream_t st) {
  cudaError_t e;
  const int nclips = pl.batch ? pl.n_clips : 1;
  if (pl.batch) {
    // per clip: counts, scan (one CTA per clip), scatter
    if ((e = cudaMemsetAsync(ws + pl.off_ycnt, 0, (size_t)nclips * group_stride(pl.T) * 4, st)) != cudaSuccess)
      return e;
    const long long per_clip = (pl.V + nclips - 1) / nclips;
    const int bx = (int)std::max<long long>(1, std::min<long long>((per_clip + 255) / 256, 64));
    batch_group_count_kernel<<<dim3(bx, nclips), 256, 0, st>>>(pl.vy, pl.offsets, nclips, pl.T, pl.ny_pad, pl.V,
                                                              ws + pl.off_ycnt);
    const int rounds = scan_rounds(pl.T);
    auto scan = rounds <= 1   ? batch_group_scan_kernel<1>
                : rounds <= 4 ? batch_group_scan_kernel<4>
                              : batch_group_scan_kernel<kScanRounds>;
    scan<<<nclips, kScanThreads, 0, st>>>(pl.offsets, nclips, pl.T, pl.ny_pad, pl.V, ws + pl.off_ycnt);
    batch_group_scatter_kernel<<<dim3(bx, nclips), 256, 0, st>>>(pl.vy, pl.offsets, nclips, pl.T, pl.ny_pad, pl.V,
                                                                ws + pl.off_ycnt);
    count_launch(3);
    return cudaGetLastError();
  }
  return launch_grouping(pl.vy, nullptr, pl.V, pl.T, pl.ny_pad, ws + pl.off_ycnt, st);
}

// The H kernel in output format fmt (kHRowsFp16 or kHPolyF32).
static cudaError_t launch_h(const Plan& pl, uint8_t* ws, int fmt, cudaStream_t st) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int nclips = pl.batch ? pl.n_clips : 1;
  HOut out{};
  long long items;
  if (fmt == kHRowsFp16) {
    out.hi = reinterpret_cast<__half*>(ws + pl.off_h);
    out.lo = out.hi + (size_t)nclips * pl.M2 * pl.ny_pad;
    items = (long long)nclips * (pl.ny_pad / kHY);
  } else {
    out.poly = reinterpret_cast<float2*>(ws + pl.off_poly);
    out.logP = pl.logT - pl.fft_logL;
    out.L = 1 << pl.fft_logL;
    items = std::max(1, pl.T / kHY);
  }
  const size_t hs = hyb_h_smem(fmt);
  auto kern = fmt == kHRowsFp16 ? hyb_h_kernel<kHRowsFp16> : hyb_h_kernel<kHPolyF32>;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kern), hs);
  if (e != cudaSuccess) return e;
  const int threads = fmt == kHRowsFp16 ? HCfg<kHRowsFp16>::threads : HCfg<kHPolyF32>::threads;
  const int per_sm = fmt == kHRowsFp16 ? HCfg<kHRowsFp16>::min_blocks : HCfg<kHPolyF32>::min_blocks;
  kern<<<(int)std::min<long long>(items, (long long)per_sm * sms), threads, hs, st>>>(pl, ws, out);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_grouped_fft(const Plan& pl, void* ws_, float* F, cudaStream_t st) {
  uint8_t* ws = static_cast<uint8_t*>(ws_);
  if (!pl.hyb || !pl.yfft || pl.batch || pl.logT > 16) return cudaErrorInvalidValue;
  cudaError_t e;
  {
    KtScope ks("group_rows", st);
    if ((e = group_rows(pl, ws, st)) != cudaSuccess) return e;
  }
  {
    KtScope ks("h_poly", st);
    if ((e = launch_h(pl, ws, kHPolyF32, st)) != cudaSuccess) return e;
  }
  KtScope ks("fft_y", st);
  return launch_fft_y(pl, ws, F, st);
}

cudaError_t launch_hybrid(const Plan& pl, void* ws_, cudaStream_t st) {
  uint8_t* ws = static_cast<uint8_t*>(ws_);
  if (!pl.hyb || !pl.pair || pl.logT > 16) return cudaErrorInvalidValue;
  const int nclips = pl.batch ? pl.n_clips : 1;
  cudaError_t e;
  {
    KtScope ks("group_rows", st);
    if ((e = group_rows(pl, ws, st)) != cudaSuccess) return e;
  }
  {
    KtScope ks("h_rows", st);
    if ((e = launch_h(pl, ws, kHRowsFp16, st)) != cudaSuccess) return e;
  }
  KtScope ks("gemm_y", st);

  const __half* h = reinterpret_cast<const __half*>(ws + pl.off_h);
  CUtensorMap mhi, mlo;
  const uint64_t hrows = (uint64_t)nclips * pl.M2;   // clips stacked: row clip 2K + r
  if (!encode_f16_2d_sw128(&mhi, h, pl.ny_pad, hrows, 64, 128) ||
      !encode_f16_2d_sw128(&mlo, h + (size_t)hrows * pl.ny_pad, pl.ny_pad, hrows, 64, 128))
    return cudaErrorInvalidValue;
  if ((e = ensure_smem(reinterpret_cast<const void*>(hyb_gemm_kernel), kGSmem)) != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(pl.tiles_m * pl.tiles_n), (unsigned)pl.splits, (unsigned)nclips);
  cfg.blockDim = dim3(kGThreads);
  cfg.dynamicSmemBytes = kGSmem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, hyb_gemm_kernel, mhi, mlo, pl, ws);
  count_launch(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace fcfs
