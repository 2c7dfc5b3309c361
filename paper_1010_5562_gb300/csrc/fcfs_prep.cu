// Table fill, exact area and axis lines, and the compensated split-K reduction
// with the quarter-plane butterfly and the Prop. CFT scale factors.
#include <algorithm>

#include <math_constants.h>

#include "fcfs_epilogue.cuh"
#include "fcfs_launch.cuh"

namespace fcfs {

// ---------------------------------------------------------------------------
// Prep: zero the status word and the integer accumulators; build the tables
// unless the workspace already holds them (its tag matches the plan's).
//
// Base values are C[r] = cos(2 pi r / T), r in [0, T/4], from the FP64 cospi
// (correctly reduced because 2r/T is exact for a power-of-two T).  Every other
// entry is an exact sign/swap of a base value, so the tables keep the symmetries
// cos(th + pi) = -cos(th) etc. bit for bit.
//  - F32 table: float2 {cos, sin} per phase (full) or float C[r] (quarter).
//  - Fixed table (axis lines): int32 round(c * 2^q), int2 (full) or int (quarter).
// The tag is written by the last kernel of a call, once every kernel that reads
// the tables has been enqueued behind this one.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double base_cos(int r, int T) { return cospi(2.0 * (double)r / (double)T); }

__global__ void prep_kernel(Plan pl, uint8_t* ws, int validate) {
  // the contraction kernel behind this one may start its prologue now
  griddep_launch_dependents();
  const int T = pl.T;
  const int logQ = pl.logT - 2;
  const int Q = T / 4;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gsz = (long long)gridDim.x * blockDim.x;
  if (gid == 0) {
    Status* st = reinterpret_cast<Status*>(ws + pl.off_status);
    st->code = 0;
    st->detail = 0;
    unsigned* sync = reinterpret_cast<unsigned*>(ws + kSyncOffset);
    sync[0] = 0;
    sync[1] = 0;
    sync[2] = 0;   // work counter of the grouped contraction's H kernel
  }
  long long* acc = reinterpret_cast<long long*>(ws + pl.off_axis);
  const long long nclips = pl.batch ? pl.n_clips : 1;
  const long long nacc = (4LL * pl.K + 1) * nclips;
  for (long long i = gid; i < nacc; i += gsz) acc[i] = 0;
  long long* bins = reinterpret_cast<long long*>(ws + pl.off_bins);
  for (long long i = gid; i < 2LL * (T + 1) * nclips; i += gsz) bins[i] = 0;
  if (validate) {
    int* hist = reinterpret_cast<int*>(ws + pl.off_hist);
    for (long long i = gid; i < 2LL * (T + 1); i += gsz) hist[i] = 0;
  }
  if (*reinterpret_cast<volatile const unsigned long long*>(ws + kTagOffset) == pl.tag) return;
  // The tables are about to change: drop the old tag first, so that a call that
  // fails after this kernel cannot leave a tag that vouches for the tables of
  // another period (every CTA that sees a mismatch rebuilds, so the cleared tag
  // never makes one skip).
  if (threadIdx.x == 0) *reinterpret_cast<volatile unsigned long long*>(ws + kTagOffset) = 0ull;
  const double scale = ldexp(1.0, pl.fixq);
  if (pl.full) {
    for (long long p = gid; p < T; p += gsz) {
      Quad qd = quad_split((uint32_t)p, (uint32_t)logQ);
      double c = base_cos((int)qd.i1, T), s = base_cos((int)qd.i2, T);
      if (qd.cneg) c = -c;
      if (qd.sneg) s = -s;
      reinterpret_cast<float2*>(ws + pl.off_tab_f32)[p] = make_float2((float)c, (float)s);
    }
    for (long long r = gid; r <= Q; r += gsz)
      reinterpret_cast<int*>(ws + pl.off_tab_fix)[r] = (int)llrint(base_cos((int)r, T) * scale);
  } else {
    for (long long r = gid; r <= Q; r += gsz) {
      const double c = base_cos((int)r, T);
      reinterpret_cast<float*>(ws + pl.off_tab_f32)[r] = (float)c;
      reinterpret_cast<int*>(ws + pl.off_tab_fix)[r] = (int)llrint(c * scale);
    }
  }
}

// ---------------------------------------------------------------------------
// Area and axis lines, exact in 64-bit integers (Eqs. Fdc, Fk0, F0l; Steps 1-3).
//
// Steps 2 and 3 of FCFS: bin the weights by coordinate, then take a 1-D DFT
// of the bins.  bin_x[n] = sum over corners with x = n of s y (the signed
// vertical-edge lengths at x = n), bin_y[n] = sum over y = n of s x, n in [0, T]:
//   Sx(k) = sum_n bin_x[n] exp(-j 2 pi k n / T),  F(k,0) = j T/(2 pi k) Sx(k),
//   Sy(l) = sum_n bin_y[n] exp(-j 2 pi l n / T),  F(0,l) = j T/(2 pi l) Sy(l),
//   area  = sum_n n bin_x[n]                      (Step 1, Eq. Fdc).
// Bins are int64 integer atomics (exact, order-free); the DFT multiplies them
// by fixed-point twiddles round(cos * 2^q) in int64, with q chosen on the host
// so that V * T * 2^q < 2^62 (no partial sum can overflow).  The only error is
// the 2^-(q+1) rounding of each twiddle.  Balance is not assumed.  Work is
// O(V) for the bins and O(T K) for the DFT instead of O(V K).
// ---------------------------------------------------------------------------
constexpr int kAxisThreads = 256;

template <bool BATCH>
__global__ void bin_kernel(Plan pl, const int32_t* __restrict__ x, const int32_t* __restrict__ y,
                           const int8_t* __restrict__ s, uint8_t* ws, int validate) {
  griddep_wait();   // launched behind the previous kernel (programmatic dependent launch)
  const int T = pl.T;
  long long* bins = reinterpret_cast<long long*>(ws + pl.off_bins);
  Status* st = reinterpret_cast<Status*>(ws + pl.off_status);
  int* hist = reinterpret_cast<int*>(ws + pl.off_hist);
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < pl.V;
       v += (long long)gridDim.x * blockDim.x) {
    const int xv = x[v], yv = y[v], sgn = s[v];
    const bool ok = xv >= 0 && xv <= T && yv >= 0 && yv <= T && (sgn == 1 || sgn == -1);
    if (validate) {
      if (!ok) {
        set_status(st, FCFS_EINVAL_DATA, (unsigned)v);
      } else {
        atomicAdd(&hist[xv], sgn);
        atomicAdd(&hist[T + 1 + yv], sgn);
      }
    }
    if (!ok) continue;   // out-of-range corners are never binned
    int c = 0;
    if (BATCH) {   // last clip whose first vertex is <= v
      int lo = 0, hi = pl.n_clips;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pl.offsets[mid] <= v) lo = mid; else hi = mid;
      }
      c = lo;
    }
    long long* b = bins + (size_t)c * 2 * (T + 1);
    atomicAdd(reinterpret_cast<unsigned long long*>(&b[xv]), (unsigned long long)((long long)sgn * yv));
    atomicAdd(reinterpret_cast<unsigned long long*>(&b[T + 1 + yv]), (unsigned long long)((long long)sgn * xv));
  }
}

size_t axis_smem_bytes(int T, int full) {
  (void)full;
  return align_up(axis_levels_ints(T) * sizeof(int), 16);
}

// Block (frequency block, bin slice, clip): thread (group q, kt) takes
// frequency k = 128 blockIdx.x + kt + 1 over the bins of the slice with index
// q mod G (G groups of kAxisThreads threads, so that the large-period blocks,
// one per SM for their 128 KB of levels, still keep 16 warps busy); the groups'
// sums are added in shared memory and then, exactly, into the clip's totals.
constexpr int kAxisGroupsMax = 4;
template <bool BATCH>
__global__ void __launch_bounds__(kAxisThreads * kAxisGroupsMax) axis_dft_kernel(Plan pl, uint8_t* ws, int nper) {
  griddep_wait();   // launched behind the previous kernel (programmatic dependent launch)
  extern __shared__ __align__(128) uint8_t sm[];
  int* lv = reinterpret_cast<int*>(sm);
  const int T = pl.T, logT = pl.logT, logQ = logT - 2;
  const size_t tb = tab_fix_bytes(T, 0);
  // after the levels: staged bins (one per thread) and, for several groups,
  // their partial sums [group][5][kAxisThreads]
  long long* sbx = reinterpret_cast<long long*>(sm + align_up(axis_levels_ints(T) * sizeof(int), 16));
  long long* sby = sbx + blockDim.x;
  long long* red = sby + blockDim.x;
  __shared__ uint64_t tbar;
  Status* st = reinterpret_cast<Status*>(ws + pl.off_status);
  if (threadIdx.x == 0) {
    mbar_init(&tbar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&tbar, (uint32_t)tb);
    bulk_load(lv, ws + pl.off_tab_fix, (uint32_t)tb, &tbar);
  }
  __syncthreads();
  mbar_wait(&tbar, 0, st, 20);
  axis_build_levels(lv, T, logT);
  __syncthreads();

  const int G = blockDim.x / kAxisThreads;
  const int grp = threadIdx.x / kAxisThreads, kt = threadIdx.x % kAxisThreads;
  const int clip = blockIdx.z;
  const long long* bx = reinterpret_cast<const long long*>(ws + pl.off_bins) + (size_t)clip * 2 * (T + 1);
  const long long* by = bx + (T + 1);
  const int k = blockIdx.x * kAxisThreads + kt + 1;
  const int n0 = blockIdx.y * nper, n1 = min(T + 1, n0 + nper);
  long long a0 = 0, a1 = 0, a2 = 0, a3 = 0, area = 0;
  // bins are staged through shared memory in coalesced slices (a dependent
  // global load per bin would leave the loop latency-bound)
  for (int b0 = n0; b0 < n1; b0 += blockDim.x) {
    const int cnt = min((int)blockDim.x, n1 - b0);
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      sbx[threadIdx.x] = bx[b0 + threadIdx.x];
      sby[threadIdx.x] = by[b0 + threadIdx.x];
    }
    __syncthreads();
    for (int i = grp; i < cnt; i += G) {
      const int n = b0 + i;
      const long long wx = sbx[i], wy = sby[i];   // same address across the group: broadcast
      if (wx == 0 && wy == 0) continue;          // group-uniform
      if (blockIdx.x == 0 && kt == 0) area += (long long)n * wx;
      if (k > pl.K) continue;
      if (fits_i32(wx) && fits_i32(wy))   // group-uniform
        axis_bin_add<true>(lv, T, logQ, k, n, wx, wy, a0, a1, a2, a3);
      else
        axis_bin_add(lv, T, logQ, k, n, wx, wy, a0, a1, a2, a3);
    }
  }
  if (G > 1) {   // add the groups' sums (integers: exact in any order)
    long long* r = red + (size_t)grp * 5 * kAxisThreads + kt;
    r[0] = a0;
    r[kAxisThreads] = a1;
    r[2 * kAxisThreads] = a2;
    r[3 * kAxisThreads] = a3;
    r[4 * kAxisThreads] = area;
    __syncthreads();
    if (grp == 0)
      for (int q = 1; q < G; ++q) {
        const long long* rq = red + (size_t)q * 5 * kAxisThreads + kt;
        a0 += rq[0];
        a1 += rq[kAxisThreads];
        a2 += rq[2 * kAxisThreads];
        a3 += rq[3 * kAxisThreads];
        area += rq[4 * kAxisThreads];
      }
  }
  if (grp != 0) return;
  long long* acc = reinterpret_cast<long long*>(ws + pl.off_axis) + (size_t)clip * (4 * pl.K + 1);
  if (k <= pl.K) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&acc[k - 1]), (unsigned long long)a0);
    atomicAdd(reinterpret_cast<unsigned long long*>(&acc[pl.K + k - 1]), (unsigned long long)a1);
    atomicAdd(reinterpret_cast<unsigned long long*>(&acc[2 * pl.K + k - 1]), (unsigned long long)a2);
    atomicAdd(reinterpret_cast<unsigned long long*>(&acc[3 * pl.K + k - 1]), (unsigned long long)a3);
  }
  if (blockIdx.x == 0 && kt == 0 && area != 0)
    atomicAdd(reinterpret_cast<unsigned long long*>(&acc[4 * pl.K]), (unsigned long long)area);
}

// ---------------------------------------------------------------------------
// Reduce + epilogue.  One thread per (k, l) in [0, K]^2.
//  - (0,0): the exact area (and F(0,0) = its nearest float).
//  - (k,0), (0,l): axis lines from the integer sums, F(k,0) = (T / 2 pi k)(S + jC)
//    where sum s y exp(-j w k x) = C - jS; F(-k,0) = conj F(k,0).
//  - k,l >= 1: sum over splits, in split order, of the FP32 quarter-plane
//    partials CC, CS, SC, SS (rows 2(k-1)+{cos,sin}, columns 2(l-1)+{cos,sin}),
//    compensated: every addition is an error-free TwoSum (Knuth) and the
//    rounding errors are carried in a second float, so the sum is as accurate
//    as an FP64 one while it runs on the FP32 pipe;
//    G(k,l) = CC - SS - j(SC + CS), G(k,-l) = CC + SS - j(SC - CS);
//    F(k,l) = -T^2/(4 pi^2 k l) G(k,l), F(k,-l) = +T^2/(4 pi^2 k l) G(k,-l) (Eq. Fkl);
//    F(-k,-l) = conj F(k,l), F(-k,l) = conj F(k,-l) (real image).
// The last thread to finish writes the table tag of the workspace.
// ---------------------------------------------------------------------------
__global__ void reduce_kernel(Plan pl, uint8_t* ws, float2* __restrict__ F, long long* __restrict__ area_out,
                              int validate) {
  griddep_wait();   // launched behind the previous kernel (programmatic dependent launch)
  const int K = pl.K;
  const long long n1 = (long long)K + 1;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long W = 2LL * K + 1;
  if (validate && blockIdx.x == 0) {
    const int* hist = reinterpret_cast<const int*>(ws + pl.off_hist);
    Status* st = reinterpret_cast<Status*>(ws + pl.off_status);
    for (int i = threadIdx.x; i < 2 * (pl.T + 1); i += blockDim.x)
      if (hist[i] != 0) set_status(st, FCFS_EINVAL_DATA, 0x80000000u | (unsigned)i);
  }
  if (idx == 0 && blockIdx.y == 0) *reinterpret_cast<unsigned long long*>(ws + kTagOffset) = pl.tag;
  if (idx >= n1 * n1) return;
  const int clip = blockIdx.y;   // 0 for a single clip
  F += (size_t)clip * W * W;
  area_out += clip;
  const int k = (int)(idx / n1), l = (int)(idx % n1);
  const long long* acc = reinterpret_cast<const long long*>(ws + pl.off_axis) + (size_t)clip * (4 * K + 1);
  if (k == 0 || l == 0) {
    axis_entry(pl, acc, F, area_out, k == 0 ? (l == 0 ? 0 : K + l) : k);
    return;
  }
  const int M2 = pl.M2;
  const float* P = reinterpret_cast<const float*>(ws + pl.off_part);
  // where split sp of entry (k, l) lives: single clip, P[sp][m][n]; grouped
  // batch, P[clip][sp][m][n]; batch, the unit's own bm x bn tile
  const int m = 2 * (k - 1), n = 2 * (l - 1);
  size_t base, stride, ld;
  int S;
  if (!pl.batch || pl.hyb) {
    S = pl.splits;
    base = ((size_t)clip * S * M2 + m) * M2 + n;
    stride = (size_t)M2 * M2;
    ld = M2;
  } else {
    const int* ustart = reinterpret_cast<const int*>(ws + pl.off_units);
    const long long vc = pl.offsets[clip + 1] - pl.offsets[clip];
    S = (int)((vc + pl.unit_vertices - 1) / pl.unit_vertices);
    const int bmu = pl.pair ? 2 * pl.bm : pl.bm;   // a unit's tile: one CTA's, or a pair's
    const int tm = m / bmu, tn = n / pl.bn;
    const size_t u0 = (size_t)ustart[clip] + (size_t)(tm * pl.tiles_n + tn) * S;
    base = u0 * bmu * pl.bn + (size_t)(m - tm * bmu) * pl.bn + (n - tn * pl.bn);
    stride = (size_t)bmu * pl.bn;
    ld = pl.bn;
  }
  quad_entry<false>(pl, P, base, stride, ld, S, F, k, l);
}

// ---------------------------------------------------------------------------
// Host launch wrappers
// ---------------------------------------------------------------------------
cudaError_t launch_prep(const Plan& pl, void* ws, bool validate, cudaStream_t st) {
  // one thread per table entry on a cold workspace (the FP64 cospi is the cost)
  long long work = pl.full ? pl.T : pl.T / 4 + 1;
  work = max(work, (4LL * pl.K + 1 + 2LL * (pl.T + 1)) * (pl.batch ? pl.n_clips : 1));
  if (validate) work = max(work, 2LL * (pl.T + 1));
  int blocks = (int)min((work + 63) / 64, 2048LL);
  // every kernel of a call asks for the largest shared-memory carveout, so the
  // SMs never repartition L1/shared memory between the kernels of a call
  ensure_smem(reinterpret_cast<const void*>(prep_kernel), 0);
  prep_kernel<<<blocks, 64, 0, st>>>(pl, static_cast<uint8_t*>(ws), validate ? 1 : 0);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_axis(const Plan& pl, const int32_t* x, const int32_t* y, const int8_t* s, void* ws,
                        bool validate, cudaStream_t st) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (pl.V > 0 && !pl.bin_in_gemm) {
    const int blocks = (int)std::min<long long>((pl.V + 255) / 256, 8LL * sms);
    const cudaError_t e = launch_after(pl.batch ? bin_kernel<true> : bin_kernel<false>, dim3(blocks), dim3(256), 0,
                                       st, pl, x, y, s, static_cast<uint8_t*>(ws), validate ? 1 : 0);
    if (e != cudaSuccess) return e;
  }
  if (pl.axfft) return launch_axis_fft(pl, ws, st);   // large single clips: pruned FFT of the bins
  const int kblocks = (pl.K + kAxisThreads - 1) / kAxisThreads;
  const int clips = pl.batch ? pl.n_clips : 1;
  // blocks per SM to aim for: many when the level tables are small (each
  // block builds its own), two for the 128 KB tables of large periods
  const long long per_sm = pl.T <= 8192 ? 16 : 2;
  const long long want = std::max(1LL, per_sm * sms / ((long long)kblocks * clips));
  const int nper = (int)std::max(64LL, (pl.T + 1 + want - 1) / want);
  const int nblocks = (pl.T + 1 + nper - 1) / nper;
  const int groups = pl.T > 8192 ? kAxisGroupsMax : 1;   // large periods: one block per SM
  const int threads = kAxisThreads * groups;
  const size_t smem = axis_smem_bytes(pl.T, pl.full) + (size_t)2 * threads * sizeof(long long) +
                      (groups > 1 ? (size_t)groups * 5 * kAxisThreads * sizeof(long long) : 0);
  auto kern = pl.batch ? axis_dft_kernel<true> : axis_dft_kernel<false>;
  ensure_smem(reinterpret_cast<const void*>(kern), smem);
  return launch_after(kern, dim3(kblocks, nblocks, clips), dim3(threads), smem, st, pl, static_cast<uint8_t*>(ws),
                      nper);
}

cudaError_t launch_reduce(const Plan& pl, void* ws, float* F, int64_t* area, bool validate, cudaStream_t st) {
  const long long n = (long long)(pl.K + 1) * (pl.K + 1);
  const dim3 blocks((unsigned)((n + 255) / 256), pl.batch ? pl.n_clips : 1);
  ensure_smem(reinterpret_cast<const void*>(reduce_kernel), 0);
  return launch_after(reduce_kernel, blocks, dim3(256), 0, st, pl, static_cast<uint8_t*>(ws),
                      reinterpret_cast<float2*>(F), reinterpret_cast<long long*>(area), validate ? 1 : 0);
}

}  // namespace fcfs
