// Pruned-FFT adjoint: the adjoint's sums over the grouped coordinate as one
// input-pruned FFT per frequency k (the paper's pruned FFT of Step 4, run on
// the adjoint), then one dot per corner.
//
// For matrix m (0: gx, contracted coordinate b = y, epilogue coordinate a = x;
// 1: gy, b = x, a = y) and D the conjugate of the cotangent (D(k,l) = conj dF(k,l),
// transposed for m = 1), the derivative of F = sum_v s_v X_k(x_v) X_l(y_v) is
//   g_v = -s_v Re sum_{k=-K}^{K} E_k(a_v) U_k(b_v),   U_k(b) = sum_l D(k,l) X_l(b),
// E_k(a) = e^{-j 2 pi k a / T}, X_l(b) = jT/(2 pi l) (1 - E_l(b)), X_0(b) = T - b
// (Lemma polyip with the tail primitive).  E_{-k} = conj E_k folds +-k:
//   g_v = -s_v sum_{k=0}^{K} Re(E_k(a_v) V_k(b_v)),   V_0 = U_0,  V_k = U_k + conj U_{-k},
//   V_k(b) = sum_{l != 0} c_{k,l} e^{-j 2 pi l b / T} + const_k + lin_k b,
//   Dv(k,l) = D(k,l) + [k > 0] conj D(-k,-l),   c_{k,l} = -j T/(2 pi l) Dv(k,l),
//   const_k = -sum_l c_{k,l} + T Dv(k,0),   lin_k = -Dv(k,0).
// The trigonometric part of V_k is a DFT of length T with 2K nonzero inputs,
// wanted at every b.  With T = P L (L a power of two >= 2K) and b = p + P m,
//   V_k(p + P m) = sum_{r<L} u_p[r] e^{-j 2 pi r m / L},
//   u_p[r] = sum_{l = r mod L} c_{k,l} e^{-j 2 pi l p / T}:
// P FFTs of length L per k, O(T log L) instead of the 2K T of the contraction
// over b.  l = +-K share the residue K when L = 2K; their terms add, since the
// kernel e^{-j 2 pi r m / L} depends on l only through r.
//
// adj_tables_kernel writes the FFTs' and dots' twiddle tables and the
// transposed cotangent, so that both matrices read D(k, .) along rows.
// adj_fft_kernel, one CTA per (k, m): c_{k,.}, const_k and lin_k from the
// cotangent (the constant's sum compensated, T Dv(k,0) added in FP64), then the
// residues p two at a time (4096 points per buffer): inputs at exact integer
// phases, mixed-radix Stockham passes, and V_k(b) written in a tiled
// polyphase order, b' = p L + m = 16 t + i -> Z[m][t][k][i], so that the 16
// values of a tile take 128 bytes per k and a tile's values for every k are one
// contiguous range.
// adj_dot_kernel, one CTA per (tile, m): the corners whose b' falls in the tile
// (grouped by b', fcfs_group.cuh) each accumulate Re(E_k(a) V_k(b)) over k while
// the tile's Z streams through shared memory in chunks of 64 frequencies (bulk
// copies, a ring of mbarriers).  E_k(a) comes from a two-level table at the
// exact phase k a mod T every 8 frequencies and by angle addition between.  A
// corner at b = T takes V_k(0) + lin_k T (the periodic part repeats).
// Arithmetic is FP32 throughout; every twiddle is a correctly rounded FP32
// value (or a product of two) at an exact integer phase.
#include <algorithm>

#include <math_constants.h>

#include "fcfs_epilogue.cuh"
#include "fcfs_fft.cuh"
#include "fcfs_group.cuh"
#include "fcfs_launch.cuh"

namespace fcfs {

namespace {

constexpr int kABufPts = 4096;     // complex points per FFT buffer (several residues when L < 4096)
constexpr int kATab = 256;         // two-level table entries per level (T <= 2^16)
constexpr int kAFTab = 256;        // first-pass twiddle factors F (R0 P entries)
constexpr int kAFftThreads = 256;
constexpr int kDotThreads = 128;
constexpr int kDotTile = 16;       // polyphase positions b' per dot tile (128 bytes per k)
constexpr int kDotRows = 64;       // frequencies per streamed chunk (8 KiB)
constexpr int kDotStages = 4;

__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }

// e^{+j 2 pi p / T} from the two-level table (wc: p >> f, wf: p mod 2^f)
__device__ __forceinline__ float2 tab_w(const float2* wc, const float2* wf, uint32_t f, uint32_t p) {
  return c_mul(wc[p >> f], wf[p & ((1u << f) - 1u)]);
}


// Shared-memory layout of the FFT kernel: two padded buffers, the
// coefficients c_{k,l} (l = -K..K), the two-level table, the pass twiddles,
// the first pass's twiddle factors.
struct FftSmem {
  int bufpts, ncoef, nlev;
  __host__ __device__ static FftSmem of(int K, int logL) {
    FftSmem s;
    s.bufpts = ((kABufPts + (kABufPts >> 4)) + 2) & ~1;   // L <= kABufPts (K <= 2048)
    s.ncoef = (2 * K + 1 + 1) & ~1;
    s.nlev = 0;
    for (int lm = first_log_radix(logL) + 4; lm <= logL; lm += 4) s.nlev += tw_level_entries(lm);
    return s;
  }
  __host__ __device__ size_t bytes() const { return (size_t)(2 * bufpts + ncoef + 2 * kATab + nlev + kAFTab) * 8; }
};

// Tables of the FFTs and the dots, written once per call (float2, fixed slots):
//   [0, 256)           wc: e^{+j 2 pi (i << f) / T}, i < T >> f   (two-level table,
//   [256, 512)         wf: e^{+j 2 pi i / T}, i < 2^f               f = ceil(log2 T / 2))
//   [512, 512 + n2)    twiddles e^{-j 2 pi e / M} of the second pass (M = 2^LM2)
//   [.., + n3)         twiddles of the third pass (M = 2^LM3; two-level above 2^11)
//   [.., + kAFTab)     first-pass factors F[m] = e^{+j 2 pi m PER1 / T}, m < R0 P
// each FFT CTA takes them with one bulk copy, each dot CTA its first 512 entries.
struct TabLayout {
  int n2, n3, total;
  __host__ __device__ static TabLayout of(int logL) {
    TabLayout t;
    const int f0 = first_log_radix(logL);
    t.n2 = f0 + 4 <= logL ? tw_level_entries(f0 + 4) : 0;
    t.n3 = f0 + 8 <= logL ? tw_level_entries(f0 + 8) : 0;
    t.total = 2 * kATab + t.n2 + t.n3 + kAFTab;
    return t;
  }
};

// The transposed cotangent dFt(l, k) = dF(k, l): 32 x 32 tiles through shared
// memory, rows read and written whole (blocks past the tables' own).
constexpr int kTrTile = 32;
__device__ __forceinline__ void transpose_tile(const float2* __restrict__ dF, float2* __restrict__ dFt, int W, int t) {
  __shared__ float2 tile[kTrTile][kTrTile + 1];
  const int nt = (W + kTrTile - 1) / kTrTile;
  const int c0 = (t % nt) * kTrTile, r0 = (t / nt) * kTrTile;
  const int tx = threadIdx.x & (kTrTile - 1), ty = threadIdx.x / kTrTile;
#pragma unroll
  for (int i = ty; i < kTrTile; i += 8)
    if (r0 + i < W && c0 + tx < W) tile[i][tx] = __ldg(dF + (size_t)(r0 + i) * W + c0 + tx);
  __syncthreads();
#pragma unroll
  for (int i = ty; i < kTrTile; i += 8)
    if (c0 + i < W && r0 + tx < W) dFt[(size_t)(c0 + i) * W + r0 + tx] = tile[tx][i];
}

// 256 threads: blocks [0, ntab) the tables, the next ones a tile of the
// transposed cotangent each.
__global__ void __launch_bounds__(256) adj_tables_kernel(AdjFftArgs ar, uint8_t* ws, int ntab) {
  griddep_wait();   // the prep kernel's FP32 table (and, before it, the caller's cotangent)
  if ((int)blockIdx.x >= ntab) {
    transpose_tile(ar.dF, reinterpret_cast<float2*>(ws + ar.off_dft), 2 * ar.pl.K + 1, (int)blockIdx.x - ntab);
    return;
  }
  const Plan& pl = ar.pl;
  const int T = pl.T, logT = pl.logT, logL = ar.logL;
  const TabLayout lay = TabLayout::of(logL);
  const int f0 = first_log_radix(logL);
  const uint32_t logQ = (uint32_t)logT - 2u, mask = (uint32_t)T - 1u;
  const uint32_t f = ((uint32_t)logT + 1u) / 2u, nc = (uint32_t)T >> f;
  const float* gt = reinterpret_cast<const float*>(ws + pl.off_tab_f32);
  float2* out = reinterpret_cast<float2*>(ws + ar.off_tabs);
  auto W = [&](uint32_t p) { return pl.full ? f32_lookup<true>(gt, p, logQ) : f32_lookup<false>(gt, p, logQ); };
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= lay.total) return;
  float2 v = make_float2(0.f, 0.f);
  if (i < kATab) {
    if ((uint32_t)i < nc) v = W((uint32_t)i << f);
  } else if (i < 2 * kATab) {
    if ((uint32_t)(i - kATab) < (1u << f)) v = W((uint32_t)(i - kATab));
  } else if (i < 2 * kATab + lay.n2 + lay.n3) {
    const bool second = i < 2 * kATab + lay.n2;
    const int lm = second ? f0 + 4 : f0 + 8, e0 = second ? i - 2 * kATab : i - 2 * kATab - lay.n2;
    // direct level: entry e0; two-level: coarse entries e0 < 2^(lm-6) are 64 e0, fine entries the first 64
    const int e = lm <= 11 ? e0 : (e0 < (1 << (lm - 6)) ? 64 * e0 : e0 - (1 << (lm - 6)));
    v = conj2(W(((uint32_t)e << (logT - lm)) & mask));   // e^{-j 2 pi e / M} = conj W(e T / M)
  } else {
    const int m = i - (2 * kATab + lay.n2 + lay.n3);
    const int R0 = 1 << f0, PER1 = (1 << logL) / R0, RP = R0 * (T >> logL);
    if (PER1 >= 16 && m < RP && RP <= kAFTab) {
      // the product the FFT kernel's inputs use: wc[p >> f] wf[p mod 2^f]
      const uint32_t p = ((uint32_t)m * (uint32_t)PER1) & mask;
      v = c_mul(W((p >> f) << f), W(p & ((1u << f) - 1u)));
    }
  }
  out[i] = v;
}

// One CTA per (k, m): blockIdx.x = k in [0, K], blockIdx.y = m; L = 2^LOGL.
template <int LOGL>
__global__ void __launch_bounds__(kAFftThreads, 2) adj_fft_kernel(AdjFftArgs ar, uint8_t* ws) {
  constexpr int L = 1 << LOGL, F0 = first_log_radix(LOGL), R0 = 1 << F0;
  constexpr int LM2 = F0 + 4, LM3 = F0 + 8;   // levels of the radix-16 passes (when <= LOGL)
  extern __shared__ __align__(128) uint8_t sm[];
  __shared__ float red[4][kAFftThreads / 32];
  __shared__ float4 s_side;
  const Plan& pl = ar.pl;
  const int T = pl.T, K = pl.K, logT = pl.logT, W = 2 * K + 1;
  const int logP = ar.logP, P = 1 << logP;
  const int nfft = min(P, kABufPts >> LOGL);   // residues per round
  const FftSmem lay = FftSmem::of(K, LOGL);
  float2* bufA = reinterpret_cast<float2*>(sm);
  float2* bufB = bufA + lay.bufpts;
  float2* coef = bufB + lay.bufpts;   // c_{k,l} at coef[l + K]
  float2* wc = coef + lay.ncoef;      // e^{+j 2 pi p / T} = wc[p >> f] wf[p mod 2^f]
  float2* wf = wc + kATab;
  float2* lev2 = wf + kATab;          // twiddles of the radix-16 passes
  float2* lev3 = lev2 + (LM2 <= LOGL ? tw_level_entries(LM2) : 0);
  const int k = blockIdx.x, mat = blockIdx.y;
  const uint32_t mask = (uint32_t)T - 1u;
  const uint32_t f = ((uint32_t)logT + 1u) / 2u;

  __shared__ __align__(8) uint64_t tab_bar;
  Status* st = reinterpret_cast<Status*>(ws + pl.off_status);
  griddep_wait();   // the tables kernel (and before it the prep kernel)
  const uint32_t tab_bytes = (uint32_t)TabLayout::of(LOGL).total * 8u;
  if (threadIdx.x == 0) {
    mbar_init(&tab_bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&tab_bar, tab_bytes);
    bulk_load(wc, ws + ar.off_tabs, tab_bytes, &tab_bar);   // wc, wf, lev2, lev3, ft are contiguous
  }

  // c_{k,l} = -j T/(2 pi l) Dv(k,l) and the compensated sum of the c_{k,l}
  // gy reads the rows of the transposed cotangent: both matrices read D(k, .) as a row
  const float2* Dsrc = mat == 0 ? ar.dF : reinterpret_cast<const float2*>(ws + ar.off_dft);
  auto D = [&](int kk, int ll) -> float2 { return conj2(__ldg(Dsrc + (size_t)(kk + K) * W + (ll + K))); };
  const float t2pi = (float)((double)T / (2.0 * CUDART_PI));
  CSum sr{0.f, 0.f}, si{0.f, 0.f};
  // four values of l per thread at a time: their loads are issued together
  constexpr int kB = 4;
  for (int l0 = -K + (int)threadIdx.x; l0 <= K; l0 += kB * kAFftThreads) {
    float2 dk[kB], dm[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int l = l0 + u * kAFftThreads;
      dk[u] = dm[u] = make_float2(0.f, 0.f);
      if (l <= K) {
        dk[u] = D(k, l);
        if (k > 0) dm[u] = D(-k, -l);
      }
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int l = l0 + u * kAFftThreads;
      if (l > K) break;
      float2 c = make_float2(0.f, 0.f);
      if (l != 0) {
        const float a = t2pi / (float)l;
        const float2 d = make_float2(dk[u].x + dm[u].x, dk[u].y - dm[u].y);   // Dv(k,l) = D(k,l) + conj D(-k,-l)
        c = make_float2(a * d.y, -(a * d.x));
        csum_add(sr, c.x);
        csum_add(si, c.y);
      }
      coef[l + K] = c;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float h0 = __shfl_down_sync(0xffffffffu, sr.hi, o), l0 = __shfl_down_sync(0xffffffffu, sr.lo, o);
    const float h1 = __shfl_down_sync(0xffffffffu, si.hi, o), l1 = __shfl_down_sync(0xffffffffu, si.lo, o);
    csum_add(sr, h0);
    sr.lo += l0;
    csum_add(si, h1);
    si.lo += l1;
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][warp] = sr.hi;
    red[1][warp] = sr.lo;
    red[2][warp] = si.hi;
    red[3][warp] = si.lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    CSum tr{0.f, 0.f}, ti{0.f, 0.f};
    for (int w = 0; w < kAFftThreads / 32; ++w) {
      csum_add(tr, red[0][w]);
      tr.lo += red[1][w];
      csum_add(ti, red[2][w]);
      ti.lo += red[3][w];
    }
    float2 d0 = D(k, 0);
    if (k > 0) {
      const float2 e = D(-k, 0);   // + conj D(-k, 0)
      d0.x += e.x;
      d0.y -= e.y;
    }
    const double cr = -((double)tr.hi + (double)tr.lo) + (double)T * (double)d0.x;
    const double ci = -((double)ti.hi + (double)ti.lo) + (double)T * (double)d0.y;
    s_side = make_float4((float)cr, (float)ci, -d0.x, -d0.y);
    reinterpret_cast<float4*>(ws + ar.off_side)[(size_t)mat * (K + 1) + k] = s_side;
  }
  // the tables have landed (the wait is bounded; a copy that never lands records
  // FCFS_ETIMEOUT and leaves the block's values unwritten)
  const bool tabs_ok = __syncthreads_and(mbar_wait(&tab_bar, 0, st, 63) ? 1 : 0) != 0;
  if (!tabs_ok) {
    if (threadIdx.x == 0) mbar_wait(&tab_bar, 0, st, 64);   // let a late copy land before the CTA exits
    return;
  }
  const float4 sd = s_side;
  float2* Zm = reinterpret_cast<float2*>(ws + ar.off_z) + (size_t)mat * T * (K + 1);

  // the FFT of the residues p = a0 .. a0 + nfft - 1, point e = q L + r (p = a0 + q):
  // inputs u_p[r] formed in the first pass (l = r for r <= K, l = r - L for
  // r >= L - K), outputs V_k(b) = X + const_k + lin_k b at b = p + P m written by
  // the last pass at b' = p L + m
  constexpr int NPASS = 1 + (LM2 <= LOGL ? 1 : 0) + (LM3 <= LOGL ? 1 : 0);
  constexpr int PER1 = L / R0;            // stride of the first pass's inputs
  constexpr int NSL = (NPASS == 1) ? 1 : L / 16;   // stride of the last pass's outputs
  // first-pass twiddles e^{-j 2 pi (j + PER1 s) p / T} = conj(w(j p) F[s p mod R0 P]),
  // F[m] = e^{+j 2 pi m PER1 / T}, when the first pass has a stride and R0 P fits the table
  const int RP = R0 * P;
  const bool fact = PER1 >= 16 && RP <= kAFTab;
  float2* ft = lev3 + (LM3 <= LOGL ? tw_level_entries(LM3) : 0);
  const size_t zstride = (size_t)(K + 1) * kDotTile;   // float2 between consecutive tiles of b'
  const size_t zstep = (size_t)(NSL / kDotTile > 0 ? NSL / kDotTile : 0) * zstride;   // output q -> q + 1
  const float bstep = (float)NSL * (float)P;                                          // b of output q -> q + 1
  for (int a0 = 0, round = 0; a0 < P; a0 += nfft, ++round) {
    auto in_u = [&](int e0, int s) -> float2 {
      const int q = e0 >> LOGL, j = e0 & (L - 1), r = j + s * PER1;
      const uint32_t p = (uint32_t)(a0 + q);
      if (fact) {
        // t = sum of c_l conj(F[...]) over the terms, then u = t conj(w(j p))
        float2 t = make_float2(0.f, 0.f);
        if (r >= 1 && r <= K) t = c_mul(coef[r + K], conj2(ft[((uint32_t)s * p) & (uint32_t)(RP - 1)]));
        if (r - L >= -K)
          t = c_add(t, c_mul(coef[r - L + K], conj2(ft[((uint32_t)(s - R0) * p) & (uint32_t)(RP - 1)])));
        return c_mul(t, conj2(tab_w(wc, wf, f, ((uint32_t)j * p) & mask)));
      }
      float2 u = make_float2(0.f, 0.f);
      if (r >= 1 && r <= K) u = c_mul(coef[r + K], conj2(tab_w(wc, wf, f, ((uint32_t)r * p) & mask)));
      const int l2 = r - L;
      if (l2 >= -K) u = c_add(u, c_mul(coef[l2 + K], conj2(tab_w(wc, wf, f, ((uint32_t)l2 * p) & mask))));
      return u;
    };
    auto out_z = [&](int b0, int qq, float2 v) {
      // point b0 + qq NSL: residue p = a0 + (b0 >> LOGL), m = (b0 & (L - 1)) + qq NSL;
      // the parts from b0 are common to the butterfly's outputs, qq adds constant steps
      const int p = a0 + (b0 >> LOGL), m0 = b0 & (L - 1);
      const float b = (float)(p + (m0 << logP)) + (float)qq * bstep;
      const int bp0 = (p << LOGL) | m0;
      size_t idx;
      if constexpr (NSL % kDotTile == 0)
        idx = (size_t)(bp0 >> 4) * zstride + (size_t)k * kDotTile + (bp0 & 15) + (size_t)qq * zstep;
      else {
        const int bp = bp0 + qq * NSL;
        idx = (size_t)(bp >> 4) * zstride + (size_t)k * kDotTile + (bp & 15);
      }
      Zm[idx] = make_float2(v.x + fmaf(sd.z, b, sd.x), v.y + fmaf(sd.w, b, sd.y));
    };
    // two buffers alternate over the rounds when there are two passes, so one
    // barrier per round suffices
    float2* B1 = (NPASS == 2 && (round & 1)) ? bufA : bufB;
    constexpr int NS2 = 1 << F0;   // output stride of the second pass (and input stride PER of the passes: L/16)
    auto out_1 = [&](int b0, int qq, float2 v) { B1[pad16_step<1>(b0, qq)] = v; };
    auto in_2 = [&](int e0, int s) -> float2 { return B1[pad16_step<L / 16>(e0, s)]; };
    auto out_2 = [&](int b0, int qq, float2 v) { bufA[pad16_step<NS2>(b0, qq)] = v; };
    auto in_3 = [&](int e0, int s) -> float2 { return bufA[pad16_step<L / 16>(e0, s)]; };
    if constexpr (NPASS == 1) {
      stockham_pass_io<R0, LOGL, 0, false>(in_u, out_z, lev2, lev2, nfft);
    } else if constexpr (NPASS == 2) {
      stockham_pass_io<R0, LOGL, 0, false>(in_u, out_1, lev2, lev2, nfft);
      __syncthreads();
      stockham_pass_io<16, LOGL, F0, (LM2 > 11)>(in_2, out_z, lev2, lev2 + (1 << (LM2 > 6 ? LM2 - 6 : 0)), nfft);
    } else {
      // the first pass writes bufB, the second bufA: a buffer is rewritten only
      // after a barrier that follows its last read
      stockham_pass_io<R0, LOGL, 0, false>(in_u, out_1, lev2, lev2, nfft);
      __syncthreads();
      stockham_pass_io<16, LOGL, F0, (LM2 > 11)>(in_2, out_2, lev2, lev2 + (1 << (LM2 > 6 ? LM2 - 6 : 0)), nfft);
      __syncthreads();
      stockham_pass_io<16, LOGL, F0 + 4, (LM3 > 11)>(in_3, out_z, lev3, lev3 + (1 << (LM3 > 6 ? LM3 - 6 : 0)), nfft);
    }
  }
}

// Two corners of one polyphase position: epilogue coordinates a, the steps
// z = e^{-j 2 pi a / T} and z^8, and the running sums of Re(z^k V_k(b)).
struct DotPair {
  uint32_t a0, a1;
  float2 z0, z1, q0, q1;
  float acc0, acc1;
};

// Frequencies k0 .. k0 + n - 1 of a streamed chunk (n = kDotRows unless TAIL)
// for the pair at column j.  Re(E_k(a) V_k) = Re(z^k V_k) with z = e^{-j 2 pi a / T}:
// per block of 8 frequencies S = sum_t V_{k0+8m+t} z^t by Horner's rule (four
// FMAs per frequency), then Re(z^{k0+8m} S) with the block anchor z^{k0+8m}
// from an exact table value at k0 (phase k0 a mod T) and the exact step z^8.
// The sums run in three levels (the blocks, the chunk's 8 blocks, the chunks).
// The pair's two corners share each V_k load and advance together in packed
// FP32 pairs.
// The angle-addition alternative (E_k by one rotation per frequency, six FMAs
// with the accumulation) measured 0.59 ms on the T = 65536 clip; the
// three-term recurrence 2 cos(2 pi a / T) E_k - E_{k-1}, 9e-7 error.
template <bool TAIL>
__device__ __forceinline__ void dot_chunk(const float2* __restrict__ zc, int n, int k0, int j, DotPair& d,
                                          const TwoLevel& tl, uint32_t mask) {
  const int rows = TAIL ? n : kDotRows;
  float2 A0 = tl_lookup(tl, ((uint32_t)k0 * d.a0) & mask), A1 = tl_lookup(tl, ((uint32_t)k0 * d.a1) & mask);
  A0.y = -A0.y;   // z^{k0} = conj(e^{+j 2 pi k0 a / T})
  A1.y = -A1.y;
  // the two corners side by side in packed pairs (x of corner 0, x of corner 1), ...:
  // one f32x2 FMA advances both, each half rounded as its scalar FMA
  const float2 zx = make_float2(d.z0.x, d.z1.x), zy = make_float2(d.z0.y, d.z1.y);
  const float2 nzy = make_float2(-d.z0.y, -d.z1.y);
  float c0 = 0.f, c1 = 0.f;
#pragma unroll
  for (int kk = 0; kk < rows; kk += 8) {
    const int nb = TAIL ? min(8, rows - kk) : 8;
    const float2 top = zc[(kk + nb - 1) * kDotTile + j];
    float2 Sx = make_float2(top.x, top.x), Sy = make_float2(top.y, top.y);   // S of corners 0 and 1
#pragma unroll
    for (int t = 6; t >= 0; --t) {
      if (!TAIL || t < nb - 1) {
        const float2 v = zc[(kk + t) * kDotTile + j];
        // S <- S z + v:  Sx' = Sx zx - Sy zy + vx,  Sy' = Sx zy + Sy zx + vy
        const float2 nx = ffma2(Sx, zx, ffma2(Sy, nzy, make_float2(v.x, v.x)));
        const float2 ny = ffma2(Sx, zy, ffma2(Sy, zx, make_float2(v.y, v.y)));
        Sx = nx;
        Sy = ny;
      }
    }
    c0 += fmaf(A0.x, Sx.x, -(A0.y * Sy.x));   // Re(A S)
    c1 += fmaf(A1.x, Sx.y, -(A1.y * Sy.y));
    A0 = c_mul(A0, d.q0);
    A1 = c_mul(A1, d.q1);
  }
  d.acc0 += c0;
  d.acc1 += c1;
}

// One CTA per (tile, m): blockIdx.x = tile of 16 polyphase positions, blockIdx.y = m.
__global__ void __launch_bounds__(kDotThreads, 6) adj_dot_kernel(AdjFftArgs ar, uint8_t* ws) {
  extern __shared__ __align__(128) uint8_t sm[];
  __shared__ __align__(8) uint64_t full[kDotStages], empty[kDotStages], tab_bar;
  __shared__ int s_gs[kDotTile + 1], s_po[kDotTile + 1];   // group starts, pair offsets
  const Plan& pl = ar.pl;
  const int T = pl.T, K = pl.K, tile = blockIdx.x, mat = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int nrows = K + 1, nch = (nrows + kDotRows - 1) / kDotRows;
  float2* zs = reinterpret_cast<float2*>(sm);             // [kDotStages][kDotRows][kDotTile]
  float2* tlt = zs + kDotStages * kDotRows * kDotTile;     // two-level table: coarse, then fine
  Status* st = reinterpret_cast<Status*>(ws + pl.off_status);

  griddep_wait();   // the FFT kernel's V_k and the groups
  // last kernel of the call: the tables built by this call's prep are now valid
  if (tile == 0 && mat == 0 && threadIdx.x == 0) *reinterpret_cast<unsigned long long*>(ws + kTagOffset) = pl.tag;
  const Groups gr = groups_at(ws + ar.off_groups + (size_t)mat * group_bytes(pl.V, T, ar.ny_pad), T, ar.ny_pad);
  const int b0 = tile * kDotTile;
  if (gr.start[b0] >= gr.start[b0 + kDotTile]) return;   // no corner in the tile: its values are not read

  // pairs of corners of one position: ceil(n_i / 2) per position i of the tile
  if (threadIdx.x < 32) {
    const int i = lane;
    const int g0 = i <= kDotTile ? gr.start[b0 + min(i, kDotTile)] : 0;
    const int g1 = i < kDotTile ? gr.start[b0 + i + 1] : g0;
    int np = i < kDotTile ? (g1 - g0 + 1) >> 1 : 0, incl = np;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (i <= kDotTile) {
      s_gs[i] = g0;
      s_po[i] = incl - np;
    }
  }
  const uint32_t logT = (uint32_t)pl.logT, f = (logT + 1u) / 2u;
  const uint32_t mask = (uint32_t)T - 1u;
  // the two-level table (coarse entries in slots [0, 256), fine in [256, 512))
  // by one bulk copy from the tables kernel's output
  const TwoLevel tl{tlt, f, (1u << f) - 1u, (uint32_t)kATab};
  if (threadIdx.x == 0) {
    for (int s = 0; s < kDotStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kDotThreads / 32);
    }
    mbar_init(&tab_bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&tab_bar, 2u * kATab * 8u);
    bulk_load(tlt, ws + ar.off_tabs, 2u * kATab * 8u, &tab_bar);
  }
  __syncthreads();

  const float2* src =
      reinterpret_cast<const float2*>(ws + ar.off_z) + ((size_t)mat * (T / kDotTile) + tile) * nrows * kDotTile;
  const int npairs = s_po[kDotTile];
  const int npass = (npairs + kDotThreads - 1) / kDotThreads;
  const int total = npass * nch;   // chunks this CTA streams (the tile's values once per pass)
  auto issue = [&](int g) {
    const int c = g % nch, s = g % kDotStages;
    const uint32_t bytes = (uint32_t)min(kDotRows, nrows - c * kDotRows) * kDotTile * 8u;
    mbar_arrive_expect_tx(&full[s], bytes);
    bulk_load(zs + (size_t)s * kDotRows * kDotTile, src + (size_t)c * kDotRows * kDotTile, bytes, &full[s]);
  };
  int issued = 0;
  if (threadIdx.x == 0)
    for (; issued < min(total, kDotStages); ++issued) issue(issued);

  const int32_t* ca = mat == 0 ? pl.vx : pl.vy;
  const int32_t* cb = mat == 0 ? pl.vy : pl.vx;
  float* gout = mat == 0 ? ar.gx : ar.gy;
  bool ok = true;
  int g = 0;   // chunks consumed
  for (int pass = 0; pass < npass && ok; ++pass) {
    // this thread's pair: position j of the tile, corners c0 and c0 + 1 (if in the group)
    const int q = pass * kDotThreads + (int)threadIdx.x;
    int j = 0;
#pragma unroll
    for (int i = 1; i < kDotTile; ++i) j = s_po[i] <= q ? i : j;
    const bool live = q < npairs;
    const int c0 = s_gs[j] + 2 * (q - s_po[j]);
    const bool has1 = live && c0 + 1 < s_gs[j + 1];
    const int v0 = live ? gr.perm[c0] : -1, v1 = has1 ? gr.perm[c0 + 1] : -1;
    const int a0 = v0 >= 0 ? __ldg(ca + v0) : 0, a1 = v1 >= 0 ? __ldg(ca + v1) : a0;
    const bool t0 = v0 >= 0 && __ldg(cb + v0) == T, t1 = v1 >= 0 && __ldg(cb + v1) == T;
    if (pass == 0 && !__all_sync(0xffffffffu, mbar_wait(&tab_bar, 0, st, 65) ? 1 : 0)) {
      ok = false;   // the table copy did not land in time
      break;
    }
    DotPair d;
    d.a0 = (uint32_t)a0;
    d.a1 = (uint32_t)a1;
    d.z0 = tl_lookup(tl, d.a0 & mask);
    d.z1 = tl_lookup(tl, d.a1 & mask);
    d.q0 = tl_lookup(tl, (8u * d.a0) & mask);
    d.q1 = tl_lookup(tl, (8u * d.a1) & mask);
    d.z0.y = -d.z0.y;   // z = e^{-j 2 pi a / T}, z^8
    d.z1.y = -d.z1.y;
    d.q0.y = -d.q0.y;
    d.q1.y = -d.q1.y;
    d.acc0 = d.acc1 = 0.f;
    for (int ch = 0; ch < nch; ++ch, ++g) {
      const int s = g % kDotStages;
      const uint32_t ph = (uint32_t)(g / kDotStages) & 1u;
      if (!__all_sync(0xffffffffu, mbar_wait(&full[s], ph, st, 60) ? 1 : 0)) {
        ok = false;
        break;
      }
      const float2* zc = zs + (size_t)s * kDotRows * kDotTile;
      const int rows = min(kDotRows, nrows - ch * kDotRows), k0 = ch * kDotRows;
      if (rows == kDotRows) dot_chunk<false>(zc, rows, k0, j, d, tl, mask);
      else dot_chunk<true>(zc, rows, k0, j, d, tl, mask);
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      if (threadIdx.x == 0 && issued < total) {
        // every warp has read this stage: refill it with the chunk kDotStages further on
        if (mbar_wait(&empty[s], ph, st, 61)) issue(issued++);
      }
    }
    if (!ok) break;
    // b = T: V_k(T) = V_k(0) + lin_k T (the corner sits at position 0 of tile 0)
    auto border = [&](uint32_t a) {
      const float4* side = reinterpret_cast<const float4*>(ws + ar.off_side) + (size_t)mat * nrows;
      float ex = 0.f;
      for (int k = 0; k < nrows; ++k) {
        const float2 e = tl_lookup(tl, ((uint32_t)k * a) & mask);
        const float4 sd = side[k];
        ex = fmaf(e.x, sd.z, fmaf(e.y, sd.w, ex));
      }
      return (float)T * ex;
    };
    if (v0 >= 0) {
      float tot = d.acc0;
      if (t0) tot += border(d.a0);
      gout[v0] = -(float)pl.vsg[v0] * tot;
    }
    if (v1 >= 0) {
      float tot = d.acc1;
      if (t1) tot += border(d.a1);
      gout[v1] = -(float)pl.vsg[v1] * tot;
    }
  }
  if (!ok && threadIdx.x == 0) {
    // a wait ran out: let the copies in flight land before the CTA exits
    mbar_wait(&tab_bar, 0, st, 66);
    for (int q = g; q < issued; ++q) mbar_wait(&full[q % kDotStages], (uint32_t)(q / kDotStages) & 1u, st, 62);
  }
}

}  // namespace

size_t adj_fft_smem(int K, int logL) { return FftSmem::of(K, logL).bytes(); }

size_t adj_tables_bytes(int logL) { return (size_t)TabLayout::of(logL).total * 8; }

cudaError_t launch_adj_tables(const AdjFftArgs& ar, void* ws, cudaStream_t st) {
  const int ntab = (TabLayout::of(ar.logL).total + 255) / 256;
  const int nt = (2 * ar.pl.K + 1 + kTrTile - 1) / kTrTile;
  return launch_after(adj_tables_kernel, dim3(ntab + nt * nt), dim3(256), 0, st, ar, static_cast<uint8_t*>(ws),
                      ntab);
}

static size_t adj_dot_smem() { return (size_t)kDotStages * kDotRows * kDotTile * 8 + (size_t)2 * kATab * 8; }

cudaError_t launch_adj_fft(const AdjFftArgs& ar, void* ws, cudaStream_t st) {
  void (*kern)(AdjFftArgs, uint8_t*) = nullptr;
  switch (ar.logL) {
    case 1: kern = adj_fft_kernel<1>; break;
    case 2: kern = adj_fft_kernel<2>; break;
    case 3: kern = adj_fft_kernel<3>; break;
    case 4: kern = adj_fft_kernel<4>; break;
    case 5: kern = adj_fft_kernel<5>; break;
    case 6: kern = adj_fft_kernel<6>; break;
    case 7: kern = adj_fft_kernel<7>; break;
    case 8: kern = adj_fft_kernel<8>; break;
    case 9: kern = adj_fft_kernel<9>; break;
    case 10: kern = adj_fft_kernel<10>; break;
    case 11: kern = adj_fft_kernel<11>; break;
    case 12: kern = adj_fft_kernel<12>; break;
    default: return cudaErrorInvalidValue;
  }
  const size_t smem = adj_fft_smem(ar.pl.K, ar.logL);
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  return launch_after(kern, dim3(ar.pl.K + 1, 2), dim3(kAFftThreads), smem, st, ar, static_cast<uint8_t*>(ws));
}

cudaError_t launch_adj_dot(const AdjFftArgs& ar, void* ws, cudaStream_t st) {
  const size_t smem = adj_dot_smem();
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(adj_dot_kernel), smem);
  if (e != cudaSuccess) return e;
  return launch_after(adj_dot_kernel, dim3(ar.pl.T / kDotTile, 2), dim3(kDotThreads), smem, st, ar,
                      static_cast<uint8_t*>(ws));
}

}  // namespace fcfs
