// Building blocks of the pruned FFTs (forward along y, adjoint along the
// grouped coordinate) and of the adjoint's per-corner dots: complex
// arithmetic, in-register DFTs of 2..16 points, padded shared-memory buffers,
// twiddle levels, one Stockham pass, packed FP32 pair operations and the
// two-level sincos table.  Every twiddle is a correctly rounded FP32 value at
// an exact integer phase (a table entry, or the product of two entries of a
// two-level table).
#pragma once

#include "fcfs_common.cuh"

namespace fcfs {

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -(a.y * b.y)), fmaf(a.y, b.x, a.x * b.y));
}
// a * e^{-j 2 pi q / R} for the compile-time twiddles of the radix butterflies
template <int R, int Q>
__device__ __forceinline__ float2 rot(float2 a) {
  constexpr int q = Q % R;
  if constexpr (q == 0) {
    return a;
  } else if constexpr (4 * q == R) {   // -j
    return make_float2(a.y, -a.x);
  } else if constexpr (2 * q == R) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (4 * q == 3 * R) {   // +j
    return make_float2(-a.y, a.x);
  } else {
    // cos and sin of 2 pi q / R for R in {8, 16}
    constexpr double c8 = 0.70710678118654752440, c16 = 0.92387953251128675613, s16 = 0.38268343236508977173;
    constexpr int qq = R == 8 ? 2 * q : q;   // in sixteenths of a turn
    constexpr double cs = (qq == 1 || qq == 15) ? c16 : (qq == 2 || qq == 14) ? c8 : (qq == 3 || qq == 13) ? s16
                        : (qq == 5 || qq == 11) ? -s16 : (qq == 6 || qq == 10) ? -c8 : -c16;
    constexpr double sn = (qq == 1 || qq == 7) ? s16 : (qq == 2 || qq == 6) ? c8 : (qq == 3 || qq == 5) ? c16
                        : (qq == 9 || qq == 15) ? -s16 : (qq == 10 || qq == 14) ? -c8 : -c16;
    const float c = (float)cs, s = (float)sn;   // e^{-j t} = c - j s
    return make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -(a.x * s)));
  }
}

// In-register DFT of R points, forward sign, by halving (even/odd).
template <int R>
struct Dft {
  template <int S, int O>
  __device__ __forceinline__ static void sub(const float2* x, float2* y) {
    // y[q] = sum_r x[O + S r] e^{-j 2 pi q r / R}, q < R
    if constexpr (R == 1) {
      y[0] = x[O];
    } else {
      float2 e[R / 2], o[R / 2];
      Dft<R / 2>::template sub<2 * S, O>(x, e);
      Dft<R / 2>::template sub<2 * S, O + S>(x, o);
      apply<0>(e, o, y);
    }
  }
  template <int Q>
  __device__ __forceinline__ static void apply(const float2* e, const float2* o, float2* y) {
    if constexpr (Q < R / 2) {
      const float2 t = rot<R, Q>(o[Q]);
      y[Q] = c_add(e[Q], t);
      y[Q + R / 2] = c_sub(e[Q], t);
      apply<Q + 1>(e, o, y);
    }
  }
};

// Shared-memory buffers are padded by one element per 16 (index i at i + i/16),
// so the strided stores of the first passes fall on distinct banks.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// Twiddle level of a pass, e^{-j 2 pi i / M} for i < M: a table of M entries
// for M <= 256, else the product hi[i >> 6] lo[i & 63] of two correctly
// rounded tables (M / 64 and 64 entries).
struct TwLevel {
  const float2* hi;
  const float2* lo;
  int two;
};
__device__ __forceinline__ float2 tw_at(const TwLevel& t, int i) {
  return t.two ? c_mul(t.hi[i >> 6], t.lo[i & 63]) : t.hi[i];
}

// One Stockham pass of radix R over nfft FFTs of L points: X -> Y (Y padded; X
// padded, or unpadded for the first pass, which reads the buffer the bulk copy
// filled).
template <int R, bool RAW_IN>
__device__ __forceinline__ void stockham_pass(const float2* __restrict__ X, float2* __restrict__ Y,
                                              const TwLevel& twl, int logL, int nfft, int Ns) {
  const int L = 1 << logL, per = L / R, M = Ns * R;
  const int total = nfft * per;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int fo = (t / per) * L, j = t % per;
    const int kp = j & (Ns - 1);
    float2 v[R], y[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = RAW_IN ? X[fo + j + r * per] : X[pad16(fo + j + r * per)];
    if (kp != 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = c_mul(v[r], tw_at(twl, (r * kp) & (M - 1)));
    }
    Dft<R>::template sub<1, 0>(v, y);
    const int base = fo + (j - kp) * R + kp;
#pragma unroll
    for (int q = 0; q < R; ++q) Y[pad16(base + q * Ns)] = y[q];
  }
}

// Passes with the FFT length 2^LOGL, the radix and the stride 2^LOGNS known at
// compile time (shifts instead of divisions, unrolled indexing).  Twiddles
// e^{-j 2 pi i / M}, M = 2^LOGNS R, come from a direct table of M entries (tw)
// or, with TWO, from the product tw[i >> 6] lo[i & 63].  At kp = 0 the
// twiddles are 1 and the products exact, so every butterfly takes the same path.
template <int R>
struct LogRadix {
  static constexpr int v = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4;
};
// A compile-time pass whose inputs come from in(e0, r) (point e0 + r PER,
// PER = 2^LOGL / R) and whose outputs go to out(b0, q, value) (point
// b0 + q 2^LOGNS), the points counted over the nfft FFTs: the first pass can
// form its inputs on the fly and the last can store its outputs directly, and
// both see the per-butterfly base and the compile-time step separately.
template <int R, int LOGL, int LOGNS, bool TWO, class In, class Out>
__device__ __forceinline__ void stockham_pass_io(In in, Out out, const float2* __restrict__ tw,
                                                 const float2* __restrict__ lo, int nfft) {
  constexpr int LOGR = LogRadix<R>::v, LOGPER = LOGL - LOGR, PER = 1 << LOGPER;
  constexpr int NS = 1 << LOGNS, M = NS * R;
  const int total = nfft << LOGPER;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int fo = (t >> LOGPER) << LOGL, j = t & (PER - 1);
    const int kp = j & (NS - 1);
    float2 v[R], y[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in(fo + j, r);
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const int i = (r * kp) & (M - 1);
        v[r] = c_mul(v[r], TWO ? c_mul(tw[i >> 6], lo[i & 63]) : tw[i]);
      }
    }
    Dft<R>::template sub<1, 0>(v, y);
    const int base = fo + ((j >> LOGNS) << (LOGNS + LOGR)) + kp;
#pragma unroll
    for (int q = 0; q < R; ++q) out(base, q, y[q]);
  }
}

// Padded shared-memory buffer seen by a pass: point e0 + r STEP at
// pad16(e0) + r (STEP + STEP / 16) when STEP is a multiple of 16, and at
// pad16(e0) + r when STEP = 1 and e0 + r stays in e0's group of 16.
template <int STEP>
__device__ __forceinline__ int pad16_step(int e0, int r) {
  if constexpr (STEP % 16 == 0) return pad16(e0) + r * (STEP + STEP / 16);
  else if constexpr (STEP == 1) return pad16(e0) + r;
  else return pad16(e0 + r * STEP);
}

// Pass structure of an L = 2^logL point FFT: a first pass of radix 2^f0 (f0 =
// logL mod 4, or 4), then radix-16 passes.  Pass i >= 1 runs at Ns = 2^(f0 + 4(i-1))
// with twiddle level M_i = 2^(f0 + 4 i), stored after the levels before it.
__host__ __device__ constexpr int first_log_radix(int logL) { return (logL & 3) ? (logL & 3) : 4; }

// Entries of a twiddle level of size 2^lm in the compile-time passes: a direct
// table up to 2^11 entries, else 2^(lm-6) coarse and 64 fine entries.
__host__ __device__ constexpr int tw_level_entries(int lm) { return lm <= 11 ? 1 << lm : (1 << (lm - 6)) + 64; }

// Entries of the twiddle level of size 2^lm.
__host__ __device__ __forceinline__ int level_entries(int lm) { return lm <= 8 ? 1 << lm : (1 << (lm - 6)) + 64; }

// Packed FP32 pairs (Blackwell f32x2): d = a * b + c and d = a * b elementwise,
// each element rounded as its scalar counterpart.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
// One angle-addition step (c, s) -> (c w.x - s w.y, s w.x + c w.y) in two packed operations.
__device__ __forceinline__ float2 rot2(float2 v, float2 w) {
  return ffma2(make_float2(v.y, v.x), make_float2(-w.y, w.y), fmul2(v, make_float2(w.x, w.x)));
}

// Two-level sincos table: (cos, sin)(2 pi p / T) = coarse[p >> f] * fine[p mod 2^f],
// both factors correctly rounded FP32 values copied from the plan's table.
struct TwoLevel {
  const float2* t;   // coarse [nc], then fine [2^f]
  uint32_t f, fmask, nc;
};
__device__ __forceinline__ float2 tl_lookup(const TwoLevel& tl, uint32_t p) {
  const float2 c = tl.t[p >> tl.f], d = tl.t[tl.nc + (p & tl.fmask)];
  return make_float2(fmaf(c.x, d.x, -(c.y * d.y)), fmaf(c.y, d.x, c.x * d.y));
}

}  // namespace fcfs
