// Pruned FFT along y for the grouped forward block (the sparse-image DFT of
// Step 4 with its output pruned to |l| <= K, as the paper's pruned FFT does).
//
// With the corners grouped by y, h_k[y] = sum over row y of s_v e^{-j 2 pi k x_v / T}
// (the conjugate of the grouped contraction's H, written by the H kernel), the
// off-axis block is
//     G(k, l) = sum_{y=0}^{T-1} h_k[y] e^{-j 2 pi l y / T},   F(k, l) = -T^2/(4 pi^2 k l) G(k, l)
// (Eq. Fkl; row y = T folded onto y = 0).  Only |l| <= K is wanted.  With
// T = P L (L a power of two >= 2K, P <= 16) and y = a + P b,
//     G(k, l) = sum_{a<P} e^{-j 2 pi l a / T} D_a(l mod L),   D_a(m) = sum_{b<L} h_k[a + P b] e^{-j 2 pi m b / L},
// so each k costs P FFTs of length L (O(T log L)) and (2K+1) P twiddled sums,
// instead of the contraction's 2 (2K) T MACs.  h_k arrives in polyphase order
// [k-1][a][b], so every FFT reads L consecutive complex values.
//
// One CTA per frequency k >= 1 (and its mirror -k): the FFTs run as mixed-radix
// Stockham passes (one radix-2/4/8/16 pass reading global memory, then radix-16
// passes in padded shared memory), each thread owning 2K+1 / blockDim outputs l
// whose twiddled sums it accumulates in registers over the P residues.
// Arithmetic is FP32 throughout; every twiddle is a correctly rounded FP32 table
// value at an exact integer phase.
#include <algorithm>

#include "fcfs_epilogue.cuh"
#include "fcfs_fft.cuh"
#include "fcfs_launch.cuh"

namespace fcfs {

namespace {

constexpr int kFBufPts = 4096;   // complex points per buffer (several FFTs when L < 4096)
constexpr int kFOwnMax = 9;      // outputs per thread (2K + 1 <= 9 blockDim)
constexpr int kFTab = 256;       // two-level table entries per level (T <= 2^16)

struct FftArgs {
  Plan pl;
  const uint8_t* ws;
  const float2* poly;   // [K][P][L] conj(H) in polyphase order
  int logL, logP;
  float2* F;            // (2K+1)^2 block
};

// blockIdx.x = k - 1; NT threads (256, or 1024 when 2K + 1 > 9 * 256).  The
// residues' inputs arrive by bulk copy into an unpadded buffer, the next range's
// copy overlapping this range's later passes and sums.
template <int NT>
__global__ void __launch_bounds__(NT) fft_y_kernel(FftArgs ar) {
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ __align__(8) uint64_t full_bar;
  const Plan& pl = ar.pl;
  const int T = pl.T, K = pl.K, logT = pl.logT;
  const int logL = ar.logL, L = 1 << logL, P = 1 << ar.logP;
  const int nfft = max(1, min(P, kFBufPts >> logL));   // FFTs per pass
  const int pts = nfft * L;
  const int bufpts = (pad16(pts) + 2) & ~1;            // keeps the next buffer 16-byte aligned
  float2* raw = reinterpret_cast<float2*>(sm);         // bulk-copy target, pts entries
  float2* bufA = raw + pts;
  float2* bufB = bufA + bufpts;
  float2* wc = bufB + bufpts;                          // e^{+j 2 pi p / T} = wc[p >> f] wf[p & fm]
  float2* wf = wc + kFTab;
  float2* lev = wf + kFTab;                            // twiddle levels of passes 1, 2, ...
  const int k = blockIdx.x + 1;
  const int f0 = first_log_radix(logL);
  Status* st = reinterpret_cast<Status*>(const_cast<uint8_t*>(ar.ws) + pl.off_status);
  const uint32_t bytes = (uint32_t)pts * 8u;
  const float2* src = ar.poly + (size_t)(k - 1) * P * L;

  // twiddle levels (the prep kernel wrote the table before the H kernel ran)
  const float* gt = reinterpret_cast<const float*>(ar.ws + pl.off_tab_f32);
  const uint32_t logQ = (uint32_t)logT - 2u, mask = (uint32_t)T - 1u;
  {
    int off = 0;
    for (int lm = f0 + 4; lm <= logL; lm += 4) {
      const int n = level_entries(lm);
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        // direct level: entry i; two-level: hi entries i < 2^(lm-6) are 64 i, lo entries the first 64
        const int e = lm <= 8 ? i : (i < (1 << (lm - 6)) ? 64 * i : i - (1 << (lm - 6)));
        const uint32_t p = ((uint32_t)e << (logT - lm)) & mask;   // e^{-j 2 pi e / M} = conj W(e T / M)
        const float2 w = pl.full ? f32_lookup<true>(gt, p, logQ) : f32_lookup<false>(gt, p, logQ);
        lev[off + i] = make_float2(w.x, -w.y);
      }
      off += n;
    }
  }
  const uint32_t f = ((uint32_t)logT + 1u) / 2u, nf = 1u << f, nc = (uint32_t)T >> f;
  for (uint32_t i = threadIdx.x; i < nc + nf; i += blockDim.x) {
    const uint32_t p = i < nc ? i << f : i - nc;
    const float2 w = pl.full ? f32_lookup<true>(gt, p, logQ) : f32_lookup<false>(gt, p, logQ);
    (i < nc ? wc[i] : wf[i - nc]) = w;
  }
  if (threadIdx.x == 0) {
    mbar_init(&full_bar, 1);
    fence_mbar_init();
  }
  griddep_wait();   // launched behind the H kernel (programmatic dependent launch)
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&full_bar, bytes);
    bulk_load(raw, src, bytes, &full_bar);
  }

  // outputs of this thread: l = -K + threadIdx.x + blockDim.x i
  float2 acc[kFOwnMax];
#pragma unroll
  for (int i = 0; i < kFOwnMax; ++i) acc[i] = make_float2(0.f, 0.f);
  uint32_t phase = 0;
  bool ok = true;
  for (int a0 = 0; a0 < P && ok; a0 += nfft) {
    // bounded wait, its outcome made block-uniform before the barriers below
    ok = __syncthreads_and(mbar_wait(&full_bar, phase, st, 90) ? 1 : 0) != 0;
    phase ^= 1u;
    if (!ok) break;   // FCFS_ETIMEOUT is recorded; the copy did not land
    float2 *X = bufA, *Y = bufB;
    const TwLevel none{lev, lev, 0};
    if (f0 == 1) stockham_pass<2, true>(raw, X, none, logL, nfft, 1);
    else if (f0 == 2) stockham_pass<4, true>(raw, X, none, logL, nfft, 1);
    else if (f0 == 3) stockham_pass<8, true>(raw, X, none, logL, nfft, 1);
    else stockham_pass<16, true>(raw, X, none, logL, nfft, 1);
    __syncthreads();   // raw is read: the next range's copy may land in it
    if (threadIdx.x == 0 && a0 + nfft < P) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&full_bar, bytes);
      bulk_load(raw, src + (size_t)(a0 + nfft) * L, bytes, &full_bar);
    }
    int off = 0;
    for (int lm = f0 + 4; lm <= logL; lm += 4) {
      const TwLevel tl{lev + off, lev + off + (lm <= 8 ? 0 : (1 << (lm - 6))), lm <= 8 ? 0 : 1};
      stockham_pass<16, false>(X, Y, tl, logL, nfft, 1 << (lm - 4));
      off += level_entries(lm);
      float2* t = X;
      X = Y;
      Y = t;
      __syncthreads();
    }
    // G(l) += e^{-j 2 pi l a / T} D_a(l mod L) over the residues of this range
    // (twiddles from the two-level table at the exact phase)
#pragma unroll
    for (int i = 0; i < kFOwnMax; ++i) {
      const int l = -K + (int)threadIdx.x + (int)blockDim.x * i;
      if (l > K) break;
      const int m = l & (L - 1);
      for (int q = 0; q < nfft; ++q) {
        const uint32_t ph = ((uint32_t)l * (uint32_t)(a0 + q)) & mask;
        const float2 w = c_mul(wc[ph >> f], wf[ph & (nf - 1u)]);   // e^{+j ...}
        const float2 d = X[pad16(q * L + m)];
        // acc += conj(w) d
        acc[i].x = fmaf(w.x, d.x, fmaf(w.y, d.y, acc[i].x));
        acc[i].y = fmaf(w.x, d.y, fmaf(-w.y, d.x, acc[i].y));
      }
    }
    __syncthreads();   // the sums have read X before the next range's passes overwrite it
  }
  if (!ok) {
    if (threadIdx.x == 0) mbar_wait(&full_bar, phase ^ 1u, st, 92);   // a late copy lands before the exit
    return;
  }
  // F(k, l) = -T^2 / (4 pi^2 k l) G(k, l) for l != 0 (the axis lines come from the
  // exact integer sums); F(-k, -l) = conj F(k, l)
  const long long W = 2LL * K + 1;
#pragma unroll
  for (int i = 0; i < kFOwnMax; ++i) {
    const int l = -K + (int)threadIdx.x + (int)blockDim.x * i;
    if (l > K) break;
    if (l == 0) continue;
    const float a = -pl.quad_scale / ((float)k * (float)l);
    const float2 v = make_float2(a * acc[i].x, a * acc[i].y);
    ar.F[(K + k) * W + (K + l)] = v;
    ar.F[(K - k) * W + (K - l)] = make_float2(v.x, -v.y);
  }
}

// ---------------------------------------------------------------------------
// L = 4096 (the T = 65536 clips, and K = 2048): one residue per round on
// L / 16 threads, the passes at compile-time sizes, and the last pass summing
// its outputs straight into each thread's outputs l (thread j owns the l with
// l mod L = j + q L / 16): no shared-memory round trip for the sums.
// Tables (float2, fixed slots), written once per call by fft_tables_kernel:
//   [0, 256) wc, [256, 512) wf      two-level e^{+j 2 pi p / T}
//   [512, + n2), [.., + n3)         twiddles of the second and third pass
//   [.., + 17 P)                    per residue a: e^{+j 2 pi q (L/16) a / T}, q < 16,
//                                   then e^{+j 2 pi L a / T}
// ---------------------------------------------------------------------------
constexpr int kFusedLogL = 12;

struct FusedTabs {
  int n2, n3, ng, total;
  __host__ __device__ static FusedTabs of(int P) {
    constexpr int f0 = first_log_radix(kFusedLogL);
    FusedTabs t;
    t.n2 = tw_level_entries(f0 + 4);
    t.n3 = tw_level_entries(f0 + 8);
    t.ng = 17 * P;
    t.total = 2 * kFTab + t.n2 + t.n3 + ((t.ng + 1) & ~1);
    return t;
  }
};

__global__ void fft_tables_kernel(Plan pl, uint8_t* ws, float2* out) {
  constexpr int LOGL = kFusedLogL, L = 1 << LOGL, f0 = first_log_radix(LOGL);
  const int T = pl.T, logT = pl.logT, P = T >> LOGL;
  const FusedTabs lay = FusedTabs::of(P);
  const uint32_t logQ = (uint32_t)logT - 2u, mask = (uint32_t)T - 1u;
  const uint32_t f = ((uint32_t)logT + 1u) / 2u, nc = (uint32_t)T >> f;
  const float* gt = reinterpret_cast<const float*>(ws + pl.off_tab_f32);
  griddep_wait();   // the prep kernel's FP32 table
  auto W = [&](uint32_t p) { return pl.full ? f32_lookup<true>(gt, p, logQ) : f32_lookup<false>(gt, p, logQ); };
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= lay.total) return;
  float2 v = make_float2(0.f, 0.f);
  if (i < kFTab) {
    if ((uint32_t)i < nc) v = W((uint32_t)i << f);
  } else if (i < 2 * kFTab) {
    if ((uint32_t)(i - kFTab) < (1u << f)) v = W((uint32_t)(i - kFTab));
  } else if (i < 2 * kFTab + lay.n2 + lay.n3) {
    const bool second = i < 2 * kFTab + lay.n2;
    const int lm = second ? f0 + 4 : f0 + 8, e0 = second ? i - 2 * kFTab : i - 2 * kFTab - lay.n2;
    const int e = lm <= 11 ? e0 : (e0 < (1 << (lm - 6)) ? 64 * e0 : e0 - (1 << (lm - 6)));
    const float2 w = W(((uint32_t)e << (logT - lm)) & mask);   // e^{-j 2 pi e / M} = conj W(e T / M)
    v = make_float2(w.x, -w.y);
  } else {
    const int g = i - (2 * kFTab + lay.n2 + lay.n3);
    if (g < lay.ng) {
      const int a = g / 17, q = g % 17;
      const uint32_t p = q < 16 ? ((uint32_t)(q * (L / 16)) * (uint32_t)a) & mask : ((uint32_t)L * (uint32_t)a) & mask;
      v = W(p);
    }
  }
  out[i] = v;
}

__global__ void __launch_bounds__(1 << (kFusedLogL - 4), 2) fft_y_fused_kernel(FftArgs ar, const float2* tabs) {
  constexpr int LOGL = kFusedLogL, L = 1 << LOGL, NS = L / 16, F0 = first_log_radix(LOGL), R0 = 1 << F0;
  constexpr int LM2 = F0 + 4, LM3 = F0 + 8;
  constexpr int BUF = ((L + (L >> 4)) + 2) & ~1;
  extern __shared__ __align__(16) uint8_t sm[];
  __shared__ __align__(8) uint64_t full_bar, tab_bar;
  const Plan& pl = ar.pl;
  const int T = pl.T, K = pl.K, logT = pl.logT, P = T >> LOGL;
  const FusedTabs lay = FusedTabs::of(P);
  float2* raw = reinterpret_cast<float2*>(sm);   // bulk-copy target, L entries
  float2* bufA = raw + L;
  float2* bufB = bufA + BUF;
  float2* wc = bufB + BUF;                       // the tables, one bulk copy
  float2* wf = wc + kFTab;
  float2* lev2 = wf + kFTab;
  float2* lev3 = lev2 + lay.n2;
  float2* gq = lev3 + lay.n3;                    // [a][17]
  const int k = blockIdx.x + 1, j = threadIdx.x;
  const uint32_t mask = (uint32_t)T - 1u, f = ((uint32_t)logT + 1u) / 2u;
  Status* st = reinterpret_cast<Status*>(const_cast<uint8_t*>(ar.ws) + pl.off_status);
  const float2* src = ar.poly + (size_t)(k - 1) * P * L;
  if (threadIdx.x == 0) {
    mbar_init(&full_bar, 1);
    mbar_init(&tab_bar, 1);
    fence_mbar_init();
  }
  griddep_wait();   // the H kernel's conj(H), the tables kernel's tables
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&tab_bar, (uint32_t)lay.total * 8u);
    bulk_load(wc, tabs, (uint32_t)lay.total * 8u, &tab_bar);
    mbar_arrive_expect_tx(&full_bar, (uint32_t)L * 8u);
    bulk_load(raw, src, (uint32_t)L * 8u, &full_bar);
  }
  // outputs of this thread: m = j + q NS, l = m (m <= K) or m - L (m >= L - K);
  // with L = 2K, m = K is both l = K and l = -K (the second in accK)
  float2 acc[16], accK = make_float2(0.f, 0.f);
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = make_float2(0.f, 0.f);
  // every wait is bounded and its outcome made block-uniform before any barrier
  bool ok = __syncthreads_and(mbar_wait(&tab_bar, 0, st, 91) ? 1 : 0) != 0;
  int a = 0;
  for (; a < P && ok; ++a) {
    ok = __syncthreads_and(mbar_wait(&full_bar, (uint32_t)a & 1u, st, 90) ? 1 : 0) != 0;
    if (!ok) break;   // FCFS_ETIMEOUT is recorded; the copy did not land
    auto in_raw = [&](int e0, int r) -> float2 { return raw[e0 + r * (L / R0)]; };
    auto out_b = [&](int b0, int q, float2 v) { bufB[pad16_step<1>(b0, q)] = v; };
    stockham_pass_io<R0, LOGL, 0, false>(in_raw, out_b, lev2, lev2, 1);
    __syncthreads();   // raw is read: the next residue may land in it
    if (threadIdx.x == 0 && a + 1 < P) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&full_bar, (uint32_t)L * 8u);
      bulk_load(raw, src + (size_t)(a + 1) * L, (uint32_t)L * 8u, &full_bar);
    }
    auto in_b = [&](int e0, int r) -> float2 { return bufB[pad16_step<NS>(e0, r)]; };
    auto out_a = [&](int b0, int q, float2 v) { bufA[pad16_step<(1 << F0)>(b0, q)] = v; };
    stockham_pass_io<16, LOGL, F0, (LM2 > 11)>(in_b, out_a, lev2, lev2 + (LM2 > 11 ? (1 << (LM2 - 6)) : 0), 1);
    __syncthreads();
    // last pass of butterfly j: D_a(j + q NS), then the twiddled sums
    float2 v[16], y[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = bufA[pad16_step<NS>(j, r)];
#pragma unroll
    for (int r = 1; r < 16; ++r) {
      const int i = (r * j) & (L - 1);
      v[r] = c_mul(v[r], (LM3 > 11) ? c_mul(lev3[i >> 6], lev3[(1 << (LM3 - 6)) + (i & 63)]) : lev3[i]);
    }
    Dft<16>::template sub<1, 0>(v, y);
    // G(k, l) += e^{-j 2 pi l a / T} D_a(l mod L): e^{+j 2 pi m a / T} = w(j a) gq[a][q],
    // and for l = m - L one more factor conj(gq[a][16])
    const float2 base = c_mul(wc[(((uint32_t)j * (uint32_t)a) & mask) >> f],
                              wf[((uint32_t)j * (uint32_t)a) & mask & ((1u << f) - 1u)]);
    const float2 hl = gq[a * 17 + 16];
    const float2* ga = gq + a * 17;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int m = j + q * NS;
      const bool pos = m <= K, neg = m >= L - K;
      if (pos || neg) {
        const float2 w = c_mul(base, ga[q]);   // e^{+j 2 pi m a / T}
        const float2 wn = c_mul(w, make_float2(hl.x, -hl.y));   // e^{+j 2 pi (m - L) a / T}
        const float2 ww = pos ? w : wn;
        acc[q].x = fmaf(ww.x, y[q].x, fmaf(ww.y, y[q].y, acc[q].x));   // acc += conj(ww) y
        acc[q].y = fmaf(ww.x, y[q].y, fmaf(-ww.y, y[q].x, acc[q].y));
        if (pos && neg) {
          accK.x = fmaf(wn.x, y[q].x, fmaf(wn.y, y[q].y, accK.x));
          accK.y = fmaf(wn.x, y[q].y, fmaf(-wn.y, y[q].x, accK.y));
        }
      }
    }
  }
  if (!ok) {
    if (threadIdx.x == 0) {   // let the copies in flight land before the CTA exits
      mbar_wait(&tab_bar, 0, st, 93);
      if (a < P) mbar_wait(&full_bar, (uint32_t)a & 1u, st, 92);
    }
    return;
  }
  // F(k, l) = -T^2 / (4 pi^2 k l) G(k, l) for l != 0; F(-k, -l) = conj F(k, l)
  const long long W = 2LL * K + 1;
  auto put = [&](int l, float2 g) {
    const float sc = -pl.quad_scale / ((float)k * (float)l);
    const float2 v = make_float2(sc * g.x, sc * g.y);
    ar.F[(K + k) * W + (K + l)] = v;
    ar.F[(K - k) * W + (K - l)] = make_float2(v.x, -v.y);
  };
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int m = j + q * NS;
    const bool pos = m <= K, neg = m >= L - K;
    if (pos && m != 0) put(m, acc[q]);
    else if (neg && !pos) put(m - L, acc[q]);
    if (pos && neg) put(-K, accK);
  }
}

// The axis lines and the centre of the block from the exact integer sums; the
// last kernel of the call, so it also writes the table tag.
__global__ void axis_out_kernel(Plan pl, uint8_t* ws, float2* __restrict__ F, long long* __restrict__ area_out) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *reinterpret_cast<unsigned long long*>(ws + kTagOffset) = pl.tag;
  if (i > 2 * pl.K) return;
  const long long* acc = reinterpret_cast<const long long*>(ws + pl.off_axis);
  axis_entry(pl, acc, F, area_out, i);
}

}  // namespace

// Shared memory of the FFT kernel for L points: the bulk-copy buffer, two
// padded buffers and the twiddle levels.
size_t fft_y_smem(int logL) {
  const size_t L = (size_t)1 << logL;
  const size_t pts = std::max<size_t>(L, kFBufPts);
  const size_t buf = (pts + (pts >> 4) + 2) & ~(size_t)1;
  size_t lev = 0;
  const int f0 = (logL & 3) ? (logL & 3) : 4;
  for (int lm = f0 + 4; lm <= logL; lm += 4) lev += (size_t)level_entries(lm);
  return (pts + 2 * buf + 2 * kFTab + lev) * 8;
}

// FFT length for a period T and cut-off K: a power of two >= 2K (no two wanted
// l share a residue but +-K), >= T / 16 (so P <= 16 and the H kernel writes
// whole 32-byte sectors), at most T.
int fft_log_len(int T, int K) {
  int lg = 1;
  while ((1 << lg) < 2 * K) ++lg;
  int logT = 0;
  while ((1 << logT) < T) ++logT;
  lg = std::max(lg, logT - 4);
  return std::min(lg, logT);
}

size_t fft_tables_bytes(int T, int logL) {
  return logL == kFusedLogL ? (size_t)FusedTabs::of(T >> kFusedLogL).total * 8 : 0;
}

cudaError_t launch_fft_y(const Plan& pl, void* ws, float* F, cudaStream_t st) {
  const int logL = pl.fft_logL;
  if (logL == kFusedLogL) {
    FftArgs ar;
    ar.pl = pl;
    ar.ws = static_cast<const uint8_t*>(ws);
    ar.poly = reinterpret_cast<const float2*>(static_cast<const uint8_t*>(ws) + pl.off_poly);
    ar.logL = logL;
    ar.logP = pl.logT - logL;
    ar.F = reinterpret_cast<float2*>(F);
    float2* tabs = reinterpret_cast<float2*>(static_cast<uint8_t*>(ws) + pl.off_fftab);
    const FusedTabs lay = FusedTabs::of(pl.T >> logL);
    cudaError_t e = launch_after(fft_tables_kernel, dim3((lay.total + 255) / 256), dim3(256), 0, st, pl,
                                 static_cast<uint8_t*>(ws), tabs);
    if (e != cudaSuccess) return e;
    constexpr int L = 1 << kFusedLogL, BUF = ((L + (L >> 4)) + 2) & ~1;
    const size_t smem = (size_t)(L + 2 * BUF + lay.total) * 8;
    if ((e = ensure_smem(reinterpret_cast<const void*>(fft_y_fused_kernel), smem)) != cudaSuccess) return e;
    return launch_after(fft_y_fused_kernel, dim3(pl.K), dim3(L / 16), smem, st, ar,
                        static_cast<const float2*>(tabs));
  }
  FftArgs ar;
  ar.pl = pl;
  ar.ws = static_cast<const uint8_t*>(ws);
  ar.poly = reinterpret_cast<const float2*>(static_cast<const uint8_t*>(ws) + pl.off_poly);
  ar.logL = logL;
  ar.logP = pl.logT - logL;
  ar.F = reinterpret_cast<float2*>(F);
  const bool small = 2 * pl.K + 1 <= kFOwnMax * 256;
  auto kern = small ? fft_y_kernel<256> : fft_y_kernel<1024>;
  const size_t smem = fft_y_smem(logL);
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  return launch_after(kern, dim3(pl.K), dim3(small ? 256 : 1024), smem, st, ar);
}

cudaError_t launch_axis_out(const Plan& pl, void* ws, float* F, int64_t* area, cudaStream_t st) {
  ensure_smem(reinterpret_cast<const void*>(axis_out_kernel), 0);
  return launch_after(axis_out_kernel, dim3((2 * pl.K + 1 + 255) / 256), dim3(256), 0, st, pl,
                      static_cast<uint8_t*>(ws), reinterpret_cast<float2*>(F), reinterpret_cast<long long*>(area));
}

}  // namespace fcfs
