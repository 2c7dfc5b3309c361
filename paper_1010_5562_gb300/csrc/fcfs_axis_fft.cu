// Axis lines of a large clip by a pruned FFT of the integer bins (Steps 2-3).
//
// The axis lines need, for k = 1..K, the sums (Eqs. Fk0, F0l)
//     Sx(k) = sum_{n=0}^{T} bin_x[n] e^{-j 2 pi k n / T}   (and Sy with bin_y),
// a DFT of length T of an integer sequence (bin T folds onto bin 0) wanted at
// its first K frequencies.  With T = P L (L the smallest power of two > K, at
// most T) and n = a + P b,
//     Sx(k) = sum_{a<P} e^{-j 2 pi k a / T} D_a(k mod L),   D_a(m) = sum_{b<L} bin_x[a + P b] e^{-j 2 pi m b / L}:
// P FFTs of length L per axis (O(T log L)) instead of the K T products of the
// direct sum.  The bins are exact integers below 2^53, so they are exact in
// FP64; the FFTs and the twiddled sums run in FP64 (twiddles from sincospi at
// exact rational arguments), whose rounding (~1e-15 of the sums) is far below
// the fixed-point rounding of the direct sum.  The results are stored in the
// same int64 fixed-point form (sum * 2^fixq, nearest) as the direct sum's, so
// every output stage reads them unchanged; the area sum n bin_x[n] stays an
// exact int64 sum.
//
// axis_fft_kernel: one CTA per (residue a, axis): the residue's L bins in
// bit-reversed order, an in-place radix-2 FFT in shared memory, then
// D_a(k mod L) e^{-j 2 pi k a / T} for k = 1..K to the workspace (and the
// residue's part of the area).  axis_fft_sum_kernel: per (k, axis) the sum over
// the residues in residue order (deterministic) and the fixed-point rounding.
#include <math_constants.h>

#include "fcfs_epilogue.cuh"
#include "fcfs_launch.cuh"

namespace fcfs {

namespace {

constexpr int kAxFftThreads = 256;

__device__ __forceinline__ double2 dmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x));
}

// e^{-j 2 pi p / q} for integers 0 <= p < q (q a power of two, so 2 p / q is exact)
__device__ __forceinline__ double2 dtw(long long p, long long q) {
  double s, c;
  sincospi(2.0 * (double)p / (double)q, &s, &c);
  return make_double2(c, -s);
}

__global__ void __launch_bounds__(kAxFftThreads) axis_fft_kernel(Plan pl, uint8_t* ws, int logL) {
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ long long red[kAxFftThreads / 32];
  const int T = pl.T, K = pl.K, L = 1 << logL, P = T >> logL;
  const int a = blockIdx.x, axis = blockIdx.y;
  double2* buf = reinterpret_cast<double2*>(sm);   // L points, in place
  double2* tw = buf + L;                           // e^{-j 2 pi e / L}, e < L / 2
  griddep_wait();   // the bins
  const long long* bins = reinterpret_cast<const long long*>(ws + pl.off_bins) + (size_t)axis * (T + 1);
  long long area = 0;
  for (int b = threadIdx.x; b < L; b += blockDim.x) {
    const int n = a + P * b;
    long long w = __ldg(bins + n);
    if (axis == 0) area += (long long)n * w;
    if (n == 0) {   // bin T has the phase of bin 0
      const long long wT = __ldg(bins + T);
      w += wT;
      if (axis == 0) area += (long long)T * wT;
    }
    const int rb = logL ? (int)(__brev((unsigned)b) >> (32 - logL)) : 0;
    buf[rb] = make_double2((double)w, 0.0);
  }
  for (int e = threadIdx.x; e < L / 2; e += blockDim.x) tw[e] = dtw(e, L);
  __syncthreads();
  // radix-2 decimation in time, natural order out
  for (int lh = 0; lh < logL; ++lh) {
    const int half = 1 << lh;
    for (int i = threadIdx.x; i < L / 2; i += blockDim.x) {
      const int pos = i & (half - 1);
      const int i0 = ((i >> lh) << (lh + 1)) + pos, i1 = i0 + half;
      const double2 t = dmul(buf[i1], tw[pos << (logL - 1 - lh)]);
      const double2 u = buf[i0];
      buf[i0] = make_double2(u.x + t.x, u.y + t.y);
      buf[i1] = make_double2(u.x - t.x, u.y - t.y);
    }
    __syncthreads();
  }
  // D_a(k mod L) e^{-j 2 pi k a / T}: the twiddle of the thread's first k exact,
  // the next ones (k + blockDim.x, ...) by the exact step (a few FP64 products)
  double2* out = reinterpret_cast<double2*>(ws + pl.off_axfft) + ((size_t)axis * P + a) * K;
  const int k0 = 1 + (int)threadIdx.x;
  double2 w = dtw(((long long)k0 * a) & (T - 1), T);
  const double2 step = dtw(((long long)blockDim.x * a) & (T - 1), T);
  for (int k = k0; k <= K; k += blockDim.x) {
    out[k - 1] = dmul(buf[k & (L - 1)], w);
    w = dmul(w, step);
  }
  // the residue's part of the area (x axis)
  if (axis == 0) {
#pragma unroll
    for (int o = 16; o; o >>= 1) area += __shfl_down_sync(0xffffffffu, area, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = area;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long t = 0;
      for (int i = 0; i < kAxFftThreads / 32; ++i) t += red[i];
      reinterpret_cast<long long*>(ws + pl.off_axfft + (size_t)2 * P * K * sizeof(double2))[a] = t;
    }
  }
}

// Thread (axis, k): S(k) = sum over the residues; C = Re S, S' = -Im S, stored
// as round(C 2^q), round(S' 2^q) in the direct sum's slots; thread 0 the area.
__global__ void axis_fft_sum_kernel(Plan pl, uint8_t* ws, int logL) {
  griddep_wait();
  const int K = pl.K, P = pl.T >> logL;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  long long* acc = reinterpret_cast<long long*>(ws + pl.off_axis);
  const double2* part = reinterpret_cast<const double2*>(ws + pl.off_axfft);
  if (t == 0) {
    const long long* ar = reinterpret_cast<const long long*>(ws + pl.off_axfft + (size_t)2 * P * K * sizeof(double2));
    long long s = 0;
    for (int a = 0; a < P; ++a) s += ar[a];
    acc[4 * K] = s;
  }
  if (t >= 2 * K) return;
  const int axis = t / K, k = t % K + 1;
  double re = 0.0, im = 0.0;
  for (int a = 0; a < P; ++a) {
    const double2 v = part[((size_t)axis * P + a) * K + (k - 1)];
    re += v.x;
    im += v.y;
  }
  const double sc = ldexp(1.0, pl.fixq);
  const int base = axis * 2 * K;
  acc[base + k - 1] = __double2ll_rn(re * sc);
  acc[base + K + k - 1] = __double2ll_rn(-im * sc);
}

}  // namespace

// FFT length of the axis lines: the smallest power of two > K, at most T.
int axis_fft_log_len(int T, int K) {
  int lg = 0;
  while ((1 << lg) <= K) ++lg;
  int logT = 0;
  while ((1 << logT) < T) ++logT;
  return lg < logT ? lg : logT;
}

size_t axis_fft_bytes(int T, int K) {
  const int P = T >> axis_fft_log_len(T, K);
  return (size_t)2 * P * K * sizeof(double2) + (size_t)P * sizeof(long long);
}

cudaError_t launch_axis_fft(const Plan& pl, void* ws, cudaStream_t st) {
  const int logL = axis_fft_log_len(pl.T, pl.K);
  const int L = 1 << logL, P = pl.T >> logL;
  const size_t smem = (size_t)(L + L / 2) * sizeof(double2);
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(axis_fft_kernel), smem);
  if (e != cudaSuccess) return e;
  if ((e = launch_after(axis_fft_kernel, dim3(P, 2), dim3(kAxFftThreads), smem, st, pl, static_cast<uint8_t*>(ws),
                        logL)) != cudaSuccess)
    return e;
  return launch_after(axis_fft_sum_kernel, dim3((2 * pl.K + 255) / 256), dim3(256), 0, st, pl,
                      static_cast<uint8_t*>(ws), logL);
}

}  // namespace fcfs
