// Device pieces of the last stages of a forward call, shared by the standalone
// axis/reduce kernels and by the fused tail of the contraction kernel:
//  - the binned axis-line DFT (Steps 2-3) on decimated quarter-wave levels,
//  - the compensated split-K sum + quarter-plane butterfly of one (k, l),
//  - the axis lines, F(0,0) and the exact area from the integer sums,
//  - a bounded grid-wide barrier for kernels launched cooperatively.
#pragma once

#include <math_constants.h>

#include "fcfs_common.cuh"

namespace fcfs {

// Grid-barrier and completion counters (uint32 each) in the workspace header,
// zeroed by the prep kernel of every call.
constexpr size_t kSyncOffset = 16;

// ---------------------------------------------------------------------------
// Axis lines (Eqs. Fdc, Fk0, F0l; Steps 1-3)
//   Sx(k) = sum_n bin_x[n] exp(-j 2 pi k n / T),  F(k,0) = j T/(2 pi k) Sx(k),
//   Sy(l) = sum_n bin_y[n] exp(-j 2 pi l n / T),  F(0,l) = j T/(2 pi l) Sy(l),
//   area  = sum_n n bin_x[n].
// Fixed-point twiddles round(cos * 2^q) in int64 (exact sums).
// ---------------------------------------------------------------------------

// Decimated quarter-wave levels of the fixed-point table in shared memory:
// level e holds C[m 2^e] for m in [0, Q >> e], so the phases k n mod T of 32
// consecutive k (a stride-n access) are read at stride n >> ctz(n) in level
// ctz(n), which is conflict-free.
__host__ __device__ __forceinline__ int level_offset(int e, int logQ) {
  // sum over e' < e of ((1 << (logQ - e')) + 1)
  return ((1 << (logQ + 1)) - (1 << (logQ + 1 - e))) + e;
}

// int32 entries of all levels
__host__ __device__ inline size_t axis_levels_ints(int T) { return (size_t)2 * (T / 4) + 32; }

// Build levels 1.. from level 0 (already in lv[0 .. Q]); block-wide, the caller syncs after.
__device__ __forceinline__ void axis_build_levels(int* lv, int T, int logT) {
  const int logQ = logT - 2, Q = T / 4;
  for (int e = 1; e <= logQ; ++e) {
    const int off = level_offset(e, logQ), n = (Q >> e) + 1;
    for (int m = threadIdx.x; m < n; m += blockDim.x) lv[off + m] = lv[m << e];
  }
}

// Add bin n (weights wx = bin_x[n], wy = bin_y[n]) to the four sums of frequency k.
// W32: both weights fit in int32, so each product is one 32 x 32 -> 64-bit multiply.
template <bool W32 = false>
__device__ __forceinline__ void axis_bin_add(const int* lv, int T, int logQ, int k, int n, long long wx,
                                             long long wy, long long& a0, long long& a1, long long& a2,
                                             long long& a3) {
  // phase k n mod T in the decimated level of n
  const uint32_t nm = (uint32_t)n & (uint32_t)(T - 1);
  int e = nm ? __ffs(nm) - 1 : 0;
  uint32_t u = nm >> e;
  if (e > logQ - 1) {   // n a multiple of T/4 (or 0): the level-0 lookup reads at most 4 entries
    e = 0;
    u = nm;
  }
  const int lq = logQ - e;   // log2 of this level's quarter period
  const uint32_t p = ((uint32_t)k * u) & ((4u << lq) - 1u);
  const Quad qd = quad_split(p, (uint32_t)lq);
  const int* L = lv + level_offset(e, logQ);
  int c = L[qd.i1], sn = L[qd.i2];
  if (qd.cneg) c = -c;
  if (qd.sneg) sn = -sn;
  if (W32) {
    const int x32 = (int)wx, y32 = (int)wy;
    a0 += (long long)c * x32;
    a1 += (long long)sn * x32;
    a2 += (long long)c * y32;
    a3 += (long long)sn * y32;
  } else {
    a0 += (long long)c * wx;
    a1 += (long long)sn * wx;
    a2 += (long long)c * wy;
    a3 += (long long)sn * wy;
  }
}
__device__ __forceinline__ bool fits_i32(long long w) { return w == (long long)(int)w; }

// F(+-f, 0) (row) or F(0, +-f) (column) from the fixed-point sums
// Cq = sum w cos * 2^q, Sq = sum w sin * 2^q: F = (T / 2 pi f)(S + jC).
__device__ __forceinline__ void axis_write(const Plan& pl, float2* F, int f, bool row, long long Cq, long long Sq) {
  const int K = pl.K;
  const long long W = 2LL * K + 1;
  const double inv = ldexp(1.0, -pl.fixq);
  const double C = (double)Cq * inv, S = (double)Sq * inv;
  const double g = (double)pl.T / (2.0 * CUDART_PI * f);
  const float re = (float)(g * S), im = (float)(g * C);
  if (row) {
    F[(K + f) * W + K] = make_float2(re, im);
    F[(K - f) * W + K] = make_float2(re, -im);
  } else {
    F[K * W + K + f] = make_float2(re, im);
    F[K * W + K - f] = make_float2(re, -im);
  }
}

// Axis entry i of a clip: i = 0 the centre (and the area), i in [1, K] F(+-i, 0),
// i in [K+1, 2K] F(0, +-(i-K)).  acc = the clip's integer sums, F its W x W block.
__device__ __forceinline__ void axis_entry(const Plan& pl, const long long* acc, float2* F, long long* area_out,
                                           int i) {
  const int K = pl.K;
  const long long W = 2LL * K + 1;
  if (i == 0) {
    const long long a = __ldcg(&acc[4 * K]);
    *area_out = a;
    F[K * W + K] = make_float2((float)a, 0.f);
    return;
  }
  const bool row = i <= K;
  const int f = row ? i : i - K;   // the nonzero frequency
  const int base = row ? 0 : 2 * K;
  axis_write(pl, F, f, row, __ldcg(&acc[base + f - 1]), __ldcg(&acc[base + K + f - 1]));
}

// ---------------------------------------------------------------------------
// Compensated split-K sum + butterfly of one quarter-plane entry (k, l >= 1):
// sum over splits, in split order, of the FP32 partials CC, CS, SC, SS (rows
// 2(k-1)+{cos,sin}, columns 2(l-1)+{cos,sin}); every addition is an error-free
// TwoSum (Knuth) with the rounding errors carried in a second float;
//   G(k,l) = CC - SS - j(SC + CS), G(k,-l) = CC + SS - j(SC - CS);
//   F(k,l) = -T^2/(4 pi^2 k l) G(k,l), F(k,-l) = +T^2/(4 pi^2 k l) G(k,-l) (Eq. Fkl);
//   F(-k,-l) = conj F(k,l), F(-k,l) = conj F(k,-l) (real image).
// P + base is the CC entry of split 0, stride the distance between splits, ld
// the row stride of a partial tile.
// ---------------------------------------------------------------------------
struct CSum {
  float hi, lo;
};
__device__ __forceinline__ void csum_add(CSum& a, float b) {
  const float s = a.hi + b;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b - bb);
  a.hi = s;
  a.lo += e;
}

template <bool SMEM>   // partials in global memory (streamed) or staged in shared memory
__device__ __forceinline__ void quad_entry(const Plan& pl, const float* __restrict__ P, size_t base, size_t stride,
                                           size_t ld, int S, float2* F, int k, int l) {
  const int K = pl.K;
  const long long W = 2LL * K + 1;
  CSum cc{0.f, 0.f}, cs{0.f, 0.f}, sc{0.f, 0.f}, ss{0.f, 0.f};
  // issue a whole batch of split loads before the dependent sums (latency bound otherwise)
  constexpr int kBatch = 8;
  for (int sp0 = 0; sp0 < S; sp0 += kBatch) {
    float2 r0[kBatch], r1[kBatch];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      if (sp0 + b < S) {
        const float2* q0 = reinterpret_cast<const float2*>(P + base + (size_t)(sp0 + b) * stride);
        const float2* q1 = reinterpret_cast<const float2*>(P + base + (size_t)(sp0 + b) * stride + ld);
        r0[b] = SMEM ? *q0 : __ldcs(q0);
        r1[b] = SMEM ? *q1 : __ldcs(q1);
      }
    }
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      if (sp0 + b < S) {
        csum_add(cc, r0[b].x);
        csum_add(cs, r0[b].y);
        csum_add(sc, r1[b].x);
        csum_add(ss, r1[b].y);
      }
    }
  }
  // combine hi and lo parts; the cancellations below are exact or relative to
  // the result, and the result is rounded to FP32 anyway
  const float a = pl.quad_scale / ((float)k * (float)l);   // T^2 / (4 pi^2 k l)
  const float gr_p = (cc.hi - ss.hi) + (cc.lo - ss.lo);    // Re G(k,l)
  const float gi_p = -((sc.hi + cs.hi) + (sc.lo + cs.lo)); // Im G(k,l)
  const float gr_m = (cc.hi + ss.hi) + (cc.lo + ss.lo);    // Re G(k,-l)
  const float gi_m = -((sc.hi - cs.hi) + (sc.lo - cs.lo)); // Im G(k,-l)
  const float pr = -a * gr_p, pi = -a * gi_p;   // F(k,l)  = -a G(k,l)
  const float mr = a * gr_m, mi = a * gi_m;     // F(k,-l) = +a G(k,-l)
  F[(K + k) * W + (K + l)] = make_float2(pr, pi);
  F[(K - k) * W + (K - l)] = make_float2(pr, -pi);
  F[(K + k) * W + (K - l)] = make_float2(mr, mi);
  F[(K - k) * W + (K + l)] = make_float2(mr, -mi);
}

// ---------------------------------------------------------------------------
// Grid barrier for a cooperative launch (every CTA resident).  Thread 0 of each
// CTA releases the CTA's writes (the bar.sync before the fence makes them part
// of its release), counts itself in, and spins with acquire loads until all
// CTAs have arrived.  The spin is bounded (about a second); on time-out the
// status word gets FCFS_ETIMEOUT and every thread of the CTA sees false.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// sflag: one int of shared memory for the CTA's verdict.
__device__ inline bool grid_barrier(unsigned* count, unsigned expected, Status* st, unsigned where, int* sflag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1u);
    const long long t0 = clock64();
    int good = 1;
    while (ld_acquire_gpu(count) < expected) {
      if (clock64() - t0 > 2000000000LL) {
        set_status(st, FCFS_ETIMEOUT, where);
        good = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    *sflag = good;
  }
  __syncthreads();
  return *sflag != 0;
}

// ---------------------------------------------------------------------------
// Fused tail of a single-clip forward, run by every CTA of a cooperatively
// launched contraction kernel after its FP32 partial tile is written and the
// corners of its vertex range are binned:
//  1. grid barrier: all partials and bins are complete;
//  2. one thread issues the CTA's copies: the bins and the fixed-point table
//     (bulk copies, one mbarrier), then one tiled TMA load per unit of the
//     CTA's share of the quarter plane -- the cos and sin rows of one k, 32
//     consecutive l, every partial: one box of the 3-D partials tensor map --
//     on a second mbarrier;
//  3. the axis-line DFT of the CTA's share of the frequencies over all bins
//     (in-CTA integer sums), while the partials land; CTA 0 also writes the
//     area and F(0,0);
//  4. the compensated split-K sum + butterfly of its units from shared memory.
// No CTA waits for another after the barrier.
// ---------------------------------------------------------------------------
constexpr int kQuadUnit = 32;   // l values per unit (256 bytes of a partial row)

__host__ __device__ inline int quad_units_per_row(int K) { return (K + kQuadUnit - 1) / kQuadUnit; }

struct TailSmem {   // byte offsets in the tail's shared memory
  size_t bins, lv0, lvk, red, total;
};
__host__ __device__ inline TailSmem tail_smem(int T, int K, int S, long long ctas, int threads) {
  TailSmem t;
  const long long NU = (long long)K * quad_units_per_row(K);
  t.bins = (size_t)((NU + ctas - 1) / ctas) * S * 2 * (kQuadUnit * 8);   // partial staging first
  t.lv0 = t.bins + (size_t)16 * (T + 1);                                  // bin_x, bin_y (int64)
  t.lvk = t.lv0 + tab_fix_bytes(T, 0);                                    // level 0 = the quarter table
  t.red = t.lvk + 2 * align_up((size_t)((T / 8) + 1) * 4, 16);            // two decimated levels
  t.total = t.red + (size_t)(8 + (threads / 32) * 8) * 8;
  return t;
}

// v[0..7] summed over the CTA; the sums are left in red[0..7].  All threads call.
__device__ __forceinline__ void block_sum8(long long (&v)[8], long long* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int o = 16; o; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 8; ++q) red[8 + warp * 8 + q] = v[q];
  __syncthreads();
  if (threadIdx.x < 8) {
    long long t = 0;
    for (int w = 0; w < nw; ++w) t += red[8 + w * 8 + threadIdx.x];
    red[threadIdx.x] = t;
  }
  __syncthreads();
}

// Decimated level of frequency k: the table of C[m 2^e] (e = ctz(k mod T),
// capped as in axis_bin_add) and the odd factor u, so that the phase k n mod T
// of bin n is read at index u n in that level: consecutive bins hit distinct
// banks.
struct KLevel {
  const int* L;
  int lq;        // log2 of the level's quarter period
  uint32_t u;
};
__device__ __forceinline__ KLevel k_level(int k, int T, int logQ, const int* lv0, int* buf) {
  const uint32_t km = (uint32_t)k & (uint32_t)(T - 1);
  int e = km ? __ffs(km) - 1 : 0;
  uint32_t u = km >> e;
  if (e > logQ - 1) {
    e = 0;
    u = km;
  }
  KLevel r;
  r.lq = logQ - e;
  r.u = u;
  if (e == 0) {
    r.L = lv0;
  } else {
    const int n = ((T / 4) >> e) + 1;
    for (int m = threadIdx.x; m < n; m += blockDim.x) buf[m] = lv0[m << e];
    r.L = buf;
  }
  return r;
}

__device__ __forceinline__ void k_bin_add(const KLevel& kl, int n, long long wx, long long wy, long long& a0,
                                          long long& a1, long long& a2, long long& a3) {
  const uint32_t p = ((uint32_t)n * kl.u) & ((4u << kl.lq) - 1u);
  const Quad qd = quad_split(p, (uint32_t)kl.lq);
  int c = kl.L[qd.i1], sn = kl.L[qd.i2];
  if (qd.cneg) c = -c;
  if (qd.sneg) sn = -sn;
  a0 += (long long)c * wx;
  a1 += (long long)sn * wx;
  a2 += (long long)c * wy;
  a3 += (long long)sn * wy;
}

__device__ inline void fused_tail(const Plan& pl, uint8_t* ws, uint8_t* smem, int* sflag, uint64_t* bar_axis,
                                  uint64_t* bar_part, const CUtensorMap* part_map) {
  Status* st = reinterpret_cast<Status*>(ws + pl.off_status);
  unsigned* sync = reinterpret_cast<unsigned*>(ws + kSyncOffset);
  const unsigned nblk = gridDim.x * gridDim.y;
  const unsigned b = blockIdx.y * gridDim.x + blockIdx.x;
  if (!grid_barrier(&sync[0], nblk + (unsigned)pl.barrier_extra, st, 0x7000u, sflag)) return;
  // partials left after the in-cluster sums: one per cluster of splits
  const int K = pl.K, T = pl.T, logQ = pl.logT - 2, S = pl.splits / pl.cluster;
  float2* F = pl.F;
  const TailSmem ts = tail_smem(T, K, S, nblk, blockDim.x);
  uint8_t* stage = smem;
  long long* sbins = reinterpret_cast<long long*>(smem + ts.bins);
  int* lv0 = reinterpret_cast<int*>(smem + ts.lv0);
  int* lvk = reinterpret_cast<int*>(smem + ts.lvk);
  long long* red = reinterpret_cast<long long*>(smem + ts.red);
  const int JB = quad_units_per_row(K);
  const long long NU = (long long)K * JB;
  const int u0 = (int)(NU * b / nblk), u1 = (int)(NU * (b + 1) / nblk), nu = u1 - u0;
  const int k0 = (int)((long long)K * b / nblk) + 1, k1 = (int)((long long)K * (b + 1) / nblk) + 1;
  const bool area_cta = b == 0;
  const bool do_axis = k1 > k0 || area_cta;   // CTA-uniform

  // (2) copies
  if (threadIdx.x == 0) {
    // the bins and partials are generic-proxy writes of other CTAs (acquired
    // at the barrier); order them before this thread's async-proxy reads
    asm volatile("fence.proxy.async.global;" ::: "memory");
    if (do_axis) {
      const uint32_t bb = 16u * (uint32_t)(T + 1), tb = (uint32_t)tab_fix_bytes(T, 0);
      mbar_arrive_expect_tx(bar_axis, bb + tb);
      bulk_load(sbins, ws + pl.off_bins, bb, bar_axis);
      bulk_load(lv0, ws + pl.off_tab_fix, tb, bar_axis);
    }
    if (nu > 0) {
      mbar_arrive_expect_tx(bar_part, (uint32_t)nu * S * 2 * (kQuadUnit * 8));
      for (int i = 0; i < nu; ++i) {
        const int u = u0 + i, k = u / JB + 1, j = u % JB;
        tma_load_3d(stage + (size_t)i * S * 2 * (kQuadUnit * 8), part_map, 2 * kQuadUnit * j, 2 * (k - 1), 0,
                    bar_part);
      }
    }
  }

  // (3) axis lines of frequencies [k0, k1), two per pass (the area rides along
  // in CTA 0's first pass)
  if (do_axis) {
    if (!mbar_wait(bar_axis, 0, st, 0x7002u)) return;
    const long long* sbx = sbins;
    const long long* sby = sbins + (T + 1);
    const size_t lvk_ints = align_up((size_t)((T / 8) + 1) * 4, 16) / 4;
    for (int kg = k0; kg < k1 || (kg == k0 && area_cta); kg += 2) {
      const int nk = min(2, k1 - kg);
      KLevel la{}, lb{};
      if (nk > 0) la = k_level(kg, T, logQ, lv0, lvk);
      if (nk > 1) lb = k_level(kg + 1, T, logQ, lv0, lvk + lvk_ints);
      __syncthreads();
      long long v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      long long area = 0;
#pragma unroll 4
      for (int n = threadIdx.x; n <= T; n += blockDim.x) {
        const long long wx = sbx[n], wy = sby[n];
        if ((wx | wy) == 0) continue;
        if (area_cta && kg == k0) area += (long long)n * wx;
        if (nk > 0) k_bin_add(la, n, wx, wy, v[0], v[1], v[2], v[3]);
        if (nk > 1) k_bin_add(lb, n, wx, wy, v[4], v[5], v[6], v[7]);
      }
      block_sum8(v, red);
      if (threadIdx.x < 2 * nk) {
        const int kk = threadIdx.x >> 1;
        const bool row = (threadIdx.x & 1) == 0;   // row (k,0): x-bins; column (0,k): y-bins
        axis_write(pl, F, kg + kk, row, red[4 * kk + (row ? 0 : 2)], red[4 * kk + (row ? 1 : 3)]);
      }
      if (area_cta && kg == k0) {
        long long av[8] = {area, 0, 0, 0, 0, 0, 0, 0};
        block_sum8(av, red);
        if (threadIdx.x == 0) {
          const long long W = 2LL * K + 1;
          *pl.area_out = red[0];
          F[K * W + K] = make_float2((float)red[0], 0.f);
          *reinterpret_cast<unsigned long long*>(ws + kTagOffset) = pl.tag;
        }
      }
      if (nk <= 0) break;
    }
  }

  // (4) split-K sum + butterfly of the staged units
  if (nu > 0) {
    if (!mbar_wait(bar_part, 0, st, 0x7001u)) return;
    const float* stg = reinterpret_cast<const float*>(stage);
    for (int t = threadIdx.x; t < nu * kQuadUnit; t += blockDim.x) {
      const int i = t / kQuadUnit, e = t % kQuadUnit;
      const int u = u0 + i, k = u / JB + 1, l = kQuadUnit * (u % JB) + e + 1;
      if (l > K) continue;
      // split sp, row r of unit i at float offset ((i S + sp) 2 + r) 2 kQuadUnit
      quad_entry<true>(pl, stg, (size_t)i * S * 4 * kQuadUnit + 2 * e, 4 * kQuadUnit, 2 * kQuadUnit, S, F, k, l);
    }
  }
}

}  // namespace fcfs
