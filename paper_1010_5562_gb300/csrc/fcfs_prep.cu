// Table fill, exact area and axis lines, and the compensated split-K reduction
// with the quarter-plane butterfly and the Prop. CFT scale factors.
#include <math_constants.h>

#include "fcfs_common.cuh"

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
  const int T = pl.T;
  const int logQ = pl.logT - 2;
  const int Q = T / 4;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gsz = (long long)gridDim.x * blockDim.x;
  if (gid == 0) {
    Status* st = reinterpret_cast<Status*>(ws + pl.off_status);
    st->code = 0;
    st->detail = 0;
  }
  long long* acc = reinterpret_cast<long long*>(ws + pl.off_axis);
  const long long nacc = (4LL * pl.K + 1) * (pl.batch ? pl.n_clips : 1);
  for (long long i = gid; i < nacc; i += gsz) acc[i] = 0;
  if (validate) {
    int* hist = reinterpret_cast<int*>(ws + pl.off_hist);
    for (long long i = gid; i < 2LL * (T + 1); i += gsz) hist[i] = 0;
  }
  if (*reinterpret_cast<volatile const unsigned long long*>(ws + kTagOffset) == pl.tag) return;
  const double scale = ldexp(1.0, pl.fixq);
  if (pl.full) {
    for (long long p = gid; p < T; p += gsz) {
      Quad qd = quad_split((uint32_t)p, (uint32_t)logQ);
      double c = base_cos((int)qd.i1, T), s = base_cos((int)qd.i2, T);
      if (qd.cneg) c = -c;
      if (qd.sneg) s = -s;
      reinterpret_cast<float2*>(ws + pl.off_tab_f32)[p] = make_float2((float)c, (float)s);
      reinterpret_cast<int2*>(ws + pl.off_tab_fix)[p] =
          make_int2((int)llrint(c * scale), (int)llrint(s * scale));
    }
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
//   area        = sum_v s_v x_v y_v                      (int64, exact)
//   Sx(k)       = sum_v s_v y_v exp(-j 2 pi k x_v / T)   (F(k,0) = j T/(2 pi k) Sx(k))
//   Sy(l)       = sum_v s_v x_v exp(-j 2 pi l y_v / T)   (F(0,l) = j T/(2 pi l) Sy(l))
//
// The twiddles are fixed-point integers round(cos * 2^q); products and sums
// are exact int64, so the only error is the 2^-(q+1) rounding of each twiddle.
// q is chosen on the host so that V * T * 2^q < 2^62: the final sums then fit,
// and modular int64 addition makes the order of the partial sums irrelevant
// (the result is bit-identical run to run).  Balance is not assumed.
//
// Block: 256 threads = 256 consecutive k; blockIdx.x picks a vertex range.
// The 32 lanes of a warp read the table at phases k a mod T for consecutive k,
// i.e. at stride a.  With a = 2^e u (u odd) that stride hits the same banks
// 2^e times over, so full-period tables are expanded in shared memory into
// decimated levels: level e holds the entries at multiples of 2^e and is read
// at (k u) mod (T / 2^e), a unit stride in k, which is conflict-free.
// ---------------------------------------------------------------------------
constexpr int kAxisThreads = 256;
constexpr int kAxisStage = 256;

template <bool FULL>
__device__ __forceinline__ int2 fix_lookup(const void* tab, uint32_t p, uint32_t logQ) {
  if (FULL) return reinterpret_cast<const int2*>(tab)[p];
  const int* t = reinterpret_cast<const int*>(tab);
  Quad qd = quad_split(p, logQ);
  int c = t[qd.i1], s = t[qd.i2];
  return make_int2(qd.cneg ? -c : c, qd.sneg ? -s : s);
}

// level of coordinate a in the decimated full-period table: (first entry, odd factor, index mask)
__device__ __forceinline__ int3 decimate(int a, int T, int logT) {
  const uint32_t am = (uint32_t)a & (uint32_t)(T - 1);
  if (am == 0) return make_int3(0, 0, 0);           // phase 0 for every k
  const int e = __ffs(am) - 1;
  const int size = T >> e;
  return make_int3(2 * T - 2 * size, (int)(am >> e), size - 1);
}

size_t axis_smem_bytes(int T, int full) {
  return (full ? (size_t)2 * T * 8 : tab_fix_bytes(T, 0)) + 9 * kAxisStage * sizeof(int) +
         kAxisStage * sizeof(long long);
}

template <bool FULL, bool BATCH>
__global__ void __launch_bounds__(kAxisThreads) axis_kernel(Plan pl, const int32_t* __restrict__ x,
                                                          const int32_t* __restrict__ y,
                                                          const int8_t* __restrict__ s, uint8_t* ws, int vper,
                                                          int validate) {
  extern __shared__ __align__(128) uint8_t sm[];
  const int T = pl.T;
  const size_t tb = tab_fix_bytes(T, FULL);
  const size_t tall = FULL ? (size_t)2 * T * 8 : tb;
  int* sv = reinterpret_cast<int*>(sm + tall);   // per staged vertex: 8 ints
  int* sclip = sv + 8 * kAxisStage;              // per staged vertex: clip index
  long long* sarea = reinterpret_cast<long long*>(sclip + kAxisStage);   // s x y
  __shared__ uint64_t tbar;
  Status* st = reinterpret_cast<Status*>(ws + pl.off_status);
  if (threadIdx.x == 0) {
    mbar_init(&tbar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&tbar, (uint32_t)tb);
    bulk_load(sm, ws + pl.off_tab_fix, (uint32_t)tb, &tbar);
  }
  __syncthreads();   // barrier initialised before anyone waits on it
  mbar_wait(&tbar, 0, st, 20);
  if (FULL) {
    // decimated levels e = 1 .. logT-1 from level 0
    int2* t2 = reinterpret_cast<int2*>(sm);
    for (int e = 1; e < pl.logT; ++e) {
      const int size = T >> e, off = 2 * T - 2 * size;
      for (int m = threadIdx.x; m < size; m += blockDim.x) t2[off + m] = t2[m << e];
    }
    __syncthreads();
  }
  const uint32_t mask = (uint32_t)T - 1u;
  const uint32_t logQ = (uint32_t)pl.logT - 2u;
  const int k = blockIdx.y * kAxisThreads + threadIdx.x + 1;
  const long long v0 = (long long)blockIdx.x * vper;
  const long long v1 = min((long long)pl.V, v0 + vper);
  long long a0 = 0, a1 = 0, a2 = 0, a3 = 0, area = 0;
  int* hist = reinterpret_cast<int*>(ws + pl.off_hist);
  long long* acc = reinterpret_cast<long long*>(ws + pl.off_axis);
  const int A = 4 * pl.K + 1;   // accumulators per clip
  int cur = -1;                 // clip of the running sums
  auto flush = [&](int c) {
    long long* ac = acc + (size_t)c * A;
    if (k <= pl.K) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&ac[k - 1]), (unsigned long long)a0);
      atomicAdd(reinterpret_cast<unsigned long long*>(&ac[pl.K + k - 1]), (unsigned long long)a1);
      atomicAdd(reinterpret_cast<unsigned long long*>(&ac[2 * pl.K + k - 1]), (unsigned long long)a2);
      atomicAdd(reinterpret_cast<unsigned long long*>(&ac[3 * pl.K + k - 1]), (unsigned long long)a3);
    }
    if (blockIdx.y == 0 && threadIdx.x == 0 && area != 0)
      atomicAdd(reinterpret_cast<unsigned long long*>(&ac[4 * pl.K]), (unsigned long long)area);
    a0 = a1 = a2 = a3 = area = 0;
  };
  for (long long b = v0; b < v1; b += kAxisStage) {
    const int n = (int)min((long long)kAxisStage, v1 - b);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int xv = x[b + i], yv = y[b + i], sgn = s[b + i];
      int* e = sv + 8 * i;
      int c = 0;
      if (BATCH) {   // last clip whose first vertex is <= b + i
        int lo = 0, hi = pl.n_clips;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (pl.offsets[mid] <= b + i) lo = mid; else hi = mid;
        }
        c = lo;
      }
      if (BATCH) {
        sclip[i] = c;
        sarea[i] = (long long)sgn * xv * (long long)yv;
      } else if (blockIdx.y == 0) {
        area += (long long)sgn * xv * (long long)yv;
      }
      if (FULL) {
        const int3 dx = decimate(xv, T, pl.logT), dy = decimate(yv, T, pl.logT);
        e[0] = dx.x; e[1] = dx.y; e[2] = dx.z; e[3] = sgn * yv;
        e[4] = dy.x; e[5] = dy.y; e[6] = dy.z; e[7] = sgn * xv;
      } else {
        e[0] = xv; e[1] = sgn * yv; e[4] = yv; e[5] = sgn * xv;
      }
      if (blockIdx.y == 0) {
        if (validate) {
          const bool ok = xv >= 0 && xv <= T && yv >= 0 && yv <= T && (sgn == 1 || sgn == -1);
          if (!ok) {
            set_status(st, FCFS_EINVAL_DATA, (unsigned)(b + i));
          } else {
            atomicAdd(&hist[xv], sgn);
            atomicAdd(&hist[T + 1 + yv], sgn);
          }
        }
      }
    }
    __syncthreads();
    {
      const int2* t2 = reinterpret_cast<const int2*>(sm);
      const bool act = k <= pl.K;
#pragma unroll 4
      if (!BATCH) cur = 0;
      for (int i = 0; i < n; ++i) {
        if (BATCH && sclip[i] != cur) {   // block-uniform: the clips of the staged vertices
          if (cur >= 0) flush(cur);
          cur = sclip[i];
        }
        if (!act) continue;
        const int4 ex = reinterpret_cast<const int4*>(sv + 8 * i)[0];
        const int4 ey = reinterpret_cast<const int4*>(sv + 8 * i)[1];
        int2 tx, ty;
        int wy, wx;
        if (FULL) {
          tx = t2[ex.x + (int)(((uint32_t)k * (uint32_t)ex.y) & (uint32_t)ex.z)];
          ty = t2[ey.x + (int)(((uint32_t)k * (uint32_t)ey.y) & (uint32_t)ey.z)];
          wy = ex.w;
          wx = ey.w;
        } else {
          tx = fix_lookup<false>(sm, ((uint32_t)k * (uint32_t)ex.x) & mask, logQ);
          ty = fix_lookup<false>(sm, ((uint32_t)k * (uint32_t)ey.x) & mask, logQ);
          wy = ex.y;
          wx = ey.y;
        }
        a0 += (long long)tx.x * wy;
        a1 += (long long)tx.y * wy;
        a2 += (long long)ty.x * wx;
        a3 += (long long)ty.y * wx;
        // batch: the area sum_v s x y rides on thread 0 of the first k-block
        if (BATCH && threadIdx.x == 0 && blockIdx.y == 0) area += sarea[i];
      }
    }
  }
  if (!BATCH && blockIdx.y == 0) {   // single clip: the staging threads hold the area
    for (int o = 16; o > 0; o >>= 1) area += __shfl_xor_sync(0xffffffffu, area, o);
    if ((threadIdx.x & 31) != 0) area = 0;
    __shared__ long long warea[kAxisThreads / 32];
    if ((threadIdx.x & 31) == 0) warea[threadIdx.x >> 5] = area;
    __syncthreads();
    area = 0;
    if (threadIdx.x == 0)
      for (int w = 0; w < kAxisThreads / 32; ++w) area += warea[w];
  }
  if (cur >= 0) flush(cur);
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

__global__ void reduce_kernel(Plan pl, uint8_t* ws, float2* __restrict__ F, long long* __restrict__ area_out,
                              int validate) {
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
  const double T = (double)pl.T;
  const long long* acc = reinterpret_cast<const long long*>(ws + pl.off_axis) + (size_t)clip * (4 * K + 1);
  const double inv = ldexp(1.0, -pl.fixq);
  if (k == 0 && l == 0) {
    const long long a = acc[4 * K];
    area_out[0] = a;
    F[K * W + K] = make_float2((float)a, 0.f);
    return;
  }
  if (l == 0 || k == 0) {
    const int f = k + l;   // the nonzero one
    const int base = (l == 0) ? 0 : 2 * K;
    const double C = (double)acc[base + f - 1] * inv;
    const double S = (double)acc[base + K + f - 1] * inv;
    const double g = T / (2.0 * CUDART_PI * f);
    const float re = (float)(g * S), im = (float)(g * C);
    if (l == 0) {
      F[(K + k) * W + K] = make_float2(re, im);
      F[(K - k) * W + K] = make_float2(re, -im);
    } else {
      F[K * W + K + l] = make_float2(re, im);
      F[K * W + K - l] = make_float2(re, -im);
    }
    return;
  }
  const int M2 = pl.M2;
  const float* P = reinterpret_cast<const float*>(ws + pl.off_part);
  // where split sp of entry (k, l) lives: single clip, P[sp][m][n]; batch,
  // the unit's own bm x bn tile
  const int m = 2 * (k - 1), n = 2 * (l - 1);
  size_t base, stride, ld;
  int S;
  if (!pl.batch) {
    S = pl.splits;
    base = (size_t)m * M2 + n;
    stride = (size_t)M2 * M2;
    ld = M2;
  } else {
    const int* ustart = reinterpret_cast<const int*>(ws + pl.off_units);
    const long long vc = pl.offsets[clip + 1] - pl.offsets[clip];
    S = (int)((vc + pl.unit_vertices - 1) / pl.unit_vertices);
    const int tm = m / pl.bm, tn = n / pl.bn;
    const size_t u0 = (size_t)ustart[clip] + (size_t)(tm * pl.tiles_n + tn) * S;
    base = u0 * pl.bm * pl.bn + (size_t)(m - tm * pl.bm) * pl.bn + (n - tn * pl.bn);
    stride = (size_t)pl.bm * pl.bn;
    ld = pl.bn;
  }
  CSum cc{0.f, 0.f}, cs{0.f, 0.f}, sc{0.f, 0.f}, ss{0.f, 0.f};
  // issue a whole batch of split loads before the dependent sums (latency bound otherwise)
  constexpr int kBatch = 8;
  for (int sp0 = 0; sp0 < S; sp0 += kBatch) {
    float2 r0[kBatch], r1[kBatch];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      if (sp0 + b < S) {
        r0[b] = __ldcs(reinterpret_cast<const float2*>(P + base + (size_t)(sp0 + b) * stride));
        r1[b] = __ldcs(reinterpret_cast<const float2*>(P + base + (size_t)(sp0 + b) * stride + ld));
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
  const float a = (float)(T * T / (4.0 * CUDART_PI * CUDART_PI)) / ((float)k * (float)l);
  const float gr_p = (cc.hi - ss.hi) + (cc.lo - ss.lo);   // Re G(k,l)
  const float gi_p = -((sc.hi + cs.hi) + (sc.lo + cs.lo)); // Im G(k,l)
  const float gr_m = (cc.hi + ss.hi) + (cc.lo + ss.lo);   // Re G(k,-l)
  const float gi_m = -((sc.hi - cs.hi) + (sc.lo - cs.lo)); // Im G(k,-l)
  const float pr = -a * gr_p, pi = -a * gi_p;   // F(k,l)  = -a G(k,l)
  const float mr = a * gr_m, mi = a * gi_m;     // F(k,-l) = +a G(k,-l)
  F[(K + k) * W + (K + l)] = make_float2(pr, pi);
  F[(K - k) * W + (K - l)] = make_float2(pr, -pi);
  F[(K + k) * W + (K - l)] = make_float2(mr, mi);
  F[(K - k) * W + (K + l)] = make_float2(mr, -mi);
}

// ---------------------------------------------------------------------------
// Host launch wrappers
// ---------------------------------------------------------------------------
cudaError_t launch_prep(const Plan& pl, void* ws, bool validate, cudaStream_t st) {
  // one thread per table entry on a cold workspace (the FP64 cospi is the cost)
  long long work = pl.full ? pl.T : pl.T / 4 + 1;
  work = max(work, (4LL * pl.K + 1) * (pl.batch ? pl.n_clips : 1));
  if (validate) work = max(work, 2LL * (pl.T + 1));
  int blocks = (int)min((work + 63) / 64, 2048LL);
  // every kernel of a call asks for the largest shared-memory carveout, so the
  // SMs never repartition L1/shared memory between the kernels of a call
  cudaFuncSetAttribute(prep_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  prep_kernel<<<blocks, 64, 0, st>>>(pl, static_cast<uint8_t*>(ws), validate ? 1 : 0);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_axis(const Plan& pl, const int32_t* x, const int32_t* y, const int8_t* s, void* ws,
                        bool validate, cudaStream_t st) {
  if (pl.V == 0) return cudaSuccess;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int kblocks = (pl.K + kAxisThreads - 1) / kAxisThreads;
  // equal vertex ranges, one block per SM and k-block
  const long long target = max(1LL, (long long)sms / kblocks);
  long long vper = max(8LL, (pl.V + target - 1) / target);
  const int vblocks = (int)((pl.V + vper - 1) / vper);
  const size_t smem = axis_smem_bytes(pl.T, pl.full);
  dim3 grid(vblocks, kblocks);
  auto kern = pl.full ? (pl.batch ? axis_kernel<true, true> : axis_kernel<true, false>)
                      : (pl.batch ? axis_kernel<false, true> : axis_kernel<false, false>);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  kern<<<grid, kAxisThreads, smem, st>>>(pl, x, y, s, static_cast<uint8_t*>(ws), (int)vper, validate ? 1 : 0);
  count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const Plan& pl, void* ws, float* F, int64_t* area, bool validate, cudaStream_t st) {
  const long long n = (long long)(pl.K + 1) * (pl.K + 1);
  const dim3 blocks((unsigned)((n + 255) / 256), pl.batch ? pl.n_clips : 1);
  cudaFuncSetAttribute(reduce_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  reduce_kernel<<<blocks, 256, 0, st>>>(pl, static_cast<uint8_t*>(ws), reinterpret_cast<float2*>(F),
                                        reinterpret_cast<long long*>(area), validate ? 1 : 0);
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace fcfs
