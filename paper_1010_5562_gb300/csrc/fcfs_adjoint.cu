// Adjoint of the block transform and edge chaining.
//
// For a real loss with cotangent G = dL/dRe F + j dL/dIm F and D = conj(G),
// differentiating F(k,l) = sum_v s_v X_k(x_v) X_l(y_v) (Lemma polyip with the
// tail primitive, dX_k(a)/da = -exp(-j 2 pi k a / T)) gives
//   gx_v = -s_v Re sum_k E_k(x_v) U_k(y_v),  U_k(y) = sum_l D(k,l) X_l(y),
// E_k(a) = exp(-j 2 pi k a / T).  With X_l(y) = a_l (1 - E_l(y)), a_l = jT/(2 pi l),
// and X_0(y) = T - y:
//   U_k(y) = C_k - D(k,0) y - sum_{l>0} [Hp(k,l) cos(2 pi l y/T) + Hm(k,l) sin(2 pi l y/T)],
//   H(k,l) = D(k,l) a_l,  Hp = H(k,l) + H(k,-l),  Hm = -j (H(k,l) - H(k,-l)),
//   C_k = sum_{l != 0} H(k,l) + T D(k,0).
// Folding +-k (cos even, sin odd) turns Re sum_k E_k(x) Z_k into sum_rows A'[row] Z'[row]
// with A' = (1, cos(2 pi k x/T), sin(2 pi k x/T))_k and Z'[0] = Re Z_0,
// Z'[(k,c)] = Re Z_k + Re Z_-k, Z'[(k,s)] = Im Z_k - Im Z_-k.  Hence
//   gx_v = -s_v sum_rows A'[row, v] (M' B')[row, v],
// a contraction of the real (2K+1) x (2K+2) coefficient matrix M' with the
// generated operand B' = (cos, sin of 2 pi l y_v / T for l = 1..K, 1, y_v) and a
// fused column dot with A'.  The full tail integrals are kept (their constant
// parts do not cancel per corner).  gy is the same with x and y swapped and D
// transposed.
#include <algorithm>

#include <cuda_fp16.h>
#include <math_constants.h>

#include "fcfs_common.cuh"
#include "fcfs_epilogue.cuh"
#include "fcfs_group.cuh"

namespace fcfs {

fcfs_status make_plan(int64_t V, int32_t T, int32_t K, int32_t prec, Plan& pl);
fcfs_status check_ws(const Plan& pl, void* ws, size_t ws_bytes);
static bool aligned16_ptr(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Workspace of an adjoint call: the forward plan's header and tables, then the
// two transposed coefficient matrices Mt[col][row] (rows padded to kAdjRowsPad)
// and the per-row-tile partial gradients.
struct AdjPlan {
  Plan p;
  int rows, cols, rows_pad, R, row_tiles;
  size_t off_m, off_part, total;
  // tensor-core contraction (split FP16): the frequency block packed as FP16
  // hi / lo [hi|lo][matrix][nrows_pad][kdim_pad], its row terms and the k = 0 row
  int tc, nrows_pad, kdim_pad;
  size_t off_mp, off_rows, off_m0;
  // form: 0 per corner, 1 grouped tensor-core contraction, 2 grouped pruned FFT;
  // the grouped forms group the corners by y (gx) and by x (gy)
  int form, grouped, ny_pad;
  size_t off_groups;
  // pruned FFT: T = P L, V_k at the polyphase positions, the side terms, the tables,
  // the transposed cotangent
  int fft_logL;
  size_t off_z, off_side, off_tabs, off_dft;
};
constexpr int kAdjThreads = 128;
constexpr size_t kAdjSmemBudget = 200 * 1024;

// Estimated time (ms) of each adjoint form, fitted to GB300 measurements of
// all of them on 17 clips (T = 1024 .. 65536, K = 64 .. 1024, V = 1.2e3 ..
// 9.5e5; within 16% of each measured time, 48% for the FP32 contraction):
//   per corner, tensor cores  0.037 + 1.97e-11 V K^2 + 5.76e-9 V K + 1.84e-7 K^2
//   per corner, plain FP32    0.045 + 7.5e-10 V K^2 + 1.14e-6 K^2
//   grouped, tensor cores     0.055 + 2.1e-6 T + 2.66e-11 (T + 1) K^2 + 9.74e-10 V K + 1.42e-7 K^2
//   grouped, pruned FFT       0.022 + 4.03e-5 2 (K + 1)                  (one CTA per k and matrix)
//                             + 3.58e-10 2 (K + 1) T log2 L + 3.43e-9 2 T (K + 1)   (FFTs; V_k
//                             written and read once) + 1.77e-7 V
// The pruned FFT measured fastest on every one of the 17 clips.
static double adj_cost(int form, bool tc, double v, double k, double t, double logL) {
  switch (form) {
    case 0:
      return tc ? 0.037 + 1.97e-11 * v * k * k + 5.76e-9 * v * k + 1.84e-7 * k * k
                : 0.045 + 7.5e-10 * v * k * k + 1.14e-6 * k * k;
    case 1: return 0.055 + 2.1e-6 * t + 2.66e-11 * (t + 1.0) * k * k + 9.74e-10 * v * k + 1.42e-7 * k * k;
    default:
      return 0.022 + 4.03e-5 * 2.0 * (k + 1.0) + 3.58e-10 * 2.0 * (k + 1.0) * t * logL +
             3.43e-9 * 2.0 * t * (k + 1.0) + 1.77e-7 * v;
  }
}

// FFT length of the pruned-FFT adjoint: the smallest power of two >= 2K (0 when
// the form does not apply: L > T, L > 4096, T < 16 or T > 2^16).
static int adj_fft_log_len(int T, int K) {
  int lg = 1;
  while ((1 << lg) < 2 * K) ++lg;
  if (T < 16 || T > 65536 || (1 << lg) > T || lg > 12) return 0;
  return lg;
}

static fcfs_status make_adj_plan(int64_t V, int32_t T, int32_t K, int32_t prec, AdjPlan& ap) {
  fcfs_status r = make_plan(V, T, K, FCFS_PREC_FP32, ap.p);
  if (r != FCFS_OK) return r;
  ap.tc = prec == FCFS_PREC_SPLIT_F16 ? 1 : 0;
  ap.form = 0;
  ap.grouped = 0;
  ap.ny_pad = (T + 1 + 63) / 64 * 64;
  ap.off_groups = 0;
  ap.fft_logL = adj_fft_log_len(T, K);
  ap.off_z = ap.off_side = ap.off_tabs = ap.off_dft = 0;
  ap.rows = 2 * K + 1;
  ap.cols = 2 * K + 2;
  const size_t tab = align_up(tab_f32_bytes(T, ap.p.full), 128);
  ap.R = 0;
  for (int R : {64, 32, 16, 8})
    if (!ap.R && tab + (size_t)ap.cols * R * sizeof(float) <= kAdjSmemBudget) ap.R = R;
  // the FP32 per-corner contraction needs a row tile in shared memory; the tensor cores do not
  const bool per_corner_ok = ap.tc || ap.R > 0;
  const bool tc_grouped_ok = ap.tc && V > 0;
  const bool fft_ok = ap.fft_logL > 0 && V > 0;
  if (!per_corner_ok && !fft_ok) return FCFS_EUNSUPPORTED;
  {
    const int mode = hybrid_knob();
    const double v = (double)V, k = (double)K, t = (double)T, lg = (double)ap.fft_logL;
    if (mode == 0 && per_corner_ok) ap.form = 0;
    else if (mode == 2 && tc_grouped_ok) ap.form = 1;
    else if (mode == 3 && fft_ok) ap.form = 2;
    else {
      double best = 1e300;
      const bool ok[3] = {per_corner_ok, tc_grouped_ok, fft_ok};
      for (int f = 0; f < 3; ++f) {
        if (!ok[f]) continue;
        const double c = adj_cost(f, ap.tc != 0, v, k, t, lg);
        if (c < best) {
          best = c;
          ap.form = f;
        }
      }
    }
  }
  if (!ap.R) ap.R = 8;
  ap.row_tiles = (ap.rows + ap.R - 1) / ap.R;
  ap.rows_pad = ap.row_tiles * ap.R;
  size_t o = ap.p.off_part;   // the forward's split partials are not needed here
  if (ap.form == 2) {
    // corners grouped by the polyphase position of b, V_k for every b < T, side terms
    ap.grouped = 1;
    ap.off_groups = o;
    o = align_up(o + 2 * group_bytes(V, T, ap.ny_pad), kWsAlign);
    ap.off_side = o;
    o = align_up(o + (size_t)2 * (K + 1) * sizeof(float4), kWsAlign);
    ap.off_tabs = o;
    o = align_up(o + adj_tables_bytes(ap.fft_logL), kWsAlign);
    ap.off_dft = o;
    o = align_up(o + (size_t)(2 * K + 1) * (2 * K + 1) * sizeof(float2), kWsAlign);
    ap.off_z = o;
    o = align_up(o + (size_t)2 * T * (K + 1) * sizeof(float2), kWsAlign);
    ap.off_m = ap.off_part = 0;
    ap.total = o;
    ap.p.total = o;
    return FCFS_OK;
  }
  ap.off_m = o;
  o = align_up(o + (size_t)2 * ap.cols * ap.rows_pad * sizeof(float), kWsAlign);
  if (ap.tc) {
    ap.row_tiles = (2 * K + kAdjPairRows - 1) / kAdjPairRows;
    ap.nrows_pad = ap.row_tiles * kAdjPairRows;
    ap.kdim_pad = (2 * K + 63) / 64 * 64;
    ap.off_mp = o;
    o = align_up(o + (size_t)2 * 2 * ap.nrows_pad * ap.kdim_pad * sizeof(__half), kWsAlign);
    ap.off_rows = o;
    o = align_up(o + (size_t)2 * ap.nrows_pad * sizeof(float4), kWsAlign);
    ap.off_m0 = o;
    o = align_up(o + (size_t)2 * (ap.kdim_pad + 4) * sizeof(float), kWsAlign);
    // grouped form: the MMA runs over the T + 1 values of b and the epilogue
    // over the corners grouped by b
    ap.grouped = ap.form == 1 ? 1 : 0;
    if (ap.grouped) {
      ap.off_groups = o;
      o = align_up(o + 2 * group_bytes(V, T, ap.ny_pad), kWsAlign);
    }
  }
  ap.off_part = o;
  o = align_up(o + (size_t)2 * ap.row_tiles * V * sizeof(float), kWsAlign);
  ap.total = o;
  ap.p.total = o;
  return FCFS_OK;
}

// Pack the coefficient matrices for the tensor-core contraction.  Block
// (packed row rp, matrix):
//  * rp < nrows_pad: frequency row rp (original row rp + 1: k = rp/2 + 1, cos
//    then sin; zeros past 2K) over the 2K frequency columns, scaled by a power
//    of two 2^-e that puts its largest magnitude in [2^14, 2^15) (no FP16
//    overflow, exact to undo) and split into FP16 hi = rn(v), lo = rn(v - hi);
//    its row terms (2^e, column-1 coefficient, column-b coefficient, 0) in FP32.
//  * rp = nrows_pad: the k = 0 row over the frequency columns (zeros past 2K),
//    then its column-1 and column-b coefficients, FP32.
__global__ void adj_pack_kernel(AdjPlan ap, uint8_t* ws) {
  const int rp = blockIdx.x, mat = blockIdx.y;
  const int nf = 2 * ap.p.K;
  const float* Mt = reinterpret_cast<const float*>(ws + ap.off_m) + (size_t)mat * ap.cols * ap.rows_pad;
  if (rp == ap.nrows_pad) {
    float* m0 = reinterpret_cast<float*>(ws + ap.off_m0) + (size_t)mat * (ap.kdim_pad + 4);
    for (int c = threadIdx.x; c < ap.kdim_pad + 4; c += blockDim.x) {
      const int src = c < nf ? c : (c == ap.kdim_pad ? nf : (c == ap.kdim_pad + 1 ? nf + 1 : -1));
      m0[c] = src < 0 ? 0.f : Mt[(size_t)src * ap.rows_pad];
    }
    return;
  }
  const int orig = rp < nf ? rp + 1 : -1;
  auto val = [&](int c) -> float { return orig < 0 || c >= nf ? 0.f : Mt[(size_t)c * ap.rows_pad + orig]; };
  __shared__ float red[256];
  float mx = 0.f;
  for (int c = threadIdx.x; c < nf; c += blockDim.x) mx = fmaxf(mx, fabsf(val(c)));
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  const float rmax = red[0];
  const int e = rmax > 0.f ? ilogbf(rmax) - 14 : 0;
  const float scale = ldexpf(1.f, -e);
  __half* hi = reinterpret_cast<__half*>(ws + ap.off_mp) + ((size_t)mat * ap.nrows_pad + rp) * ap.kdim_pad;
  __half* lo = hi + (size_t)2 * ap.nrows_pad * ap.kdim_pad;
  for (int c = threadIdx.x; c < ap.kdim_pad; c += blockDim.x) {
    const float v = val(c) * scale;
    const __half h = __float2half_rn(v);
    hi[c] = h;
    lo[c] = __float2half_rn(v - __half2float(h));
  }
  if (threadIdx.x == 0)
    reinterpret_cast<float4*>(ws + ap.off_rows)[(size_t)mat * ap.nrows_pad + rp] =
        orig < 0 ? make_float4(0.f, 0.f, 0.f, 0.f)
                 : make_float4(ldexpf(1.f, e), Mt[(size_t)nf * ap.rows_pad + orig],
                               Mt[(size_t)(nf + 1) * ap.rows_pad + orig], 0.f);
}

// Coefficient matrices.  Block (row, matrix): matrix 0 serves gx (D), matrix 1
// serves gy (D transposed).  With a_l = T / (2 pi l), H(k,l) = j a_l D(k,l) and
// H(k,-l) = -j a_l D(k,-l), so Hp(k,l) = j a_l (D(k,l) - D(k,-l)) and
// Hm(k,l) = a_l (D(k,l) + D(k,-l)); the folds over +-k are linear, so each
// stored coefficient is a_l times a signed sum of four cotangent entries
// (FP32).  The column-1 coefficient fold(C_k, C_-k) is minus the compensated
// sum of the row's cos-column coefficients plus T fold(D(k,0), D(-k,0)), the
// latter in FP64 (the k = 0 / l = 0 polynomial factor).
__global__ void adj_coef_kernel(AdjPlan ap, const float2* __restrict__ dF, uint8_t* ws) {
  const int K = ap.p.K, W = 2 * K + 1;
  const int row = blockIdx.x, mat = blockIdx.y;
  float* Mt = reinterpret_cast<float*>(ws + ap.off_m) + (size_t)mat * ap.cols * ap.rows_pad;
  const int k = (row + 1) / 2;
  const int kind = row == 0 ? 0 : (row & 1 ? 1 : 2);   // 0: k = 0, 1: cos row, 2: sin row
  // D(kk, ll) = conj(G) of this matrix
  auto D = [&](int kk, int ll) -> float2 {
    const float2 g = mat == 0 ? dF[(size_t)(kk + K) * W + (ll + K)] : dF[(size_t)(ll + K) * W + (kk + K)];
    return make_float2(g.x, -g.y);
  };
  const float t2pi = (float)((double)ap.p.T / (2.0 * CUDART_PI));
  CSum csum{0.f, 0.f};   // sum over l of the cos-column coefficients
  for (int l = 1 + threadIdx.x; l <= K; l += blockDim.x) {
    const float a = t2pi / (float)l;
    const float2 dkp = D(k, l), dkm = D(k, -l);
    float vc, vs;   // coefficients of columns 2(l-1) (cos) and 2(l-1)+1 (sin)
    if (kind == 0) {
      vc = a * (dkp.y - dkm.y);
      vs = -a * (dkp.x + dkm.x);
    } else {
      const float2 dmp = D(-k, l), dmm = D(-k, -l);
      if (kind == 1) {
        vc = a * ((dkp.y - dkm.y) + (dmp.y - dmm.y));
        vs = -a * ((dkp.x + dkm.x) + (dmp.x + dmm.x));
      } else {
        vc = -a * ((dkp.x - dkm.x) - (dmp.x - dmm.x));
        vs = -a * ((dkp.y + dkm.y) - (dmp.y + dmm.y));
      }
    }
    Mt[(size_t)(2 * (l - 1)) * ap.rows_pad + row] = vc;
    Mt[(size_t)(2 * (l - 1) + 1) * ap.rows_pad + row] = vs;
    csum_add(csum, vc);
  }
  // block sum of the (hi, lo) pairs in a fixed tree order
  __shared__ float red[2][kAdjThreads / 32];
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float h2 = __shfl_down_sync(0xffffffffu, csum.hi, o), l2 = __shfl_down_sync(0xffffffffu, csum.lo, o);
    csum_add(csum, h2);
    csum.lo += l2;
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = csum.hi;
    red[1][threadIdx.x >> 5] = csum.lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    CSum tot{0.f, 0.f};
    for (int w = 0; w < (int)blockDim.x / 32; ++w) {
      csum_add(tot, red[0][w]);
      tot.lo += red[1][w];
    }
    const float2 dk0 = D(k, 0), dmk0 = D(-k, 0);
    const double f0 = kind == 0 ? (double)dk0.x
                                : (kind == 1 ? (double)dk0.x + (double)dmk0.x : (double)dk0.y - (double)dmk0.y);
    Mt[(size_t)(2 * K) * ap.rows_pad + row] = (float)(-((double)tot.hi + (double)tot.lo) + (double)ap.p.T * f0);
    Mt[(size_t)(2 * K + 1) * ap.rows_pad + row] = (float)(-f0);
  }
  // padding rows of the last tile
  if (row == 0)
    for (int i = threadIdx.x; i < ap.cols * (ap.rows_pad - ap.rows); i += blockDim.x) {
      const int c = i / (ap.rows_pad - ap.rows), rr = ap.rows + i % (ap.rows_pad - ap.rows);
      Mt[(size_t)c * ap.rows_pad + rr] = 0.f;
    }
}

// Contraction with fused column dot.  Block (row tile, vertex range, matrix);
// each thread takes one corner at a time and accumulates R rows in registers.
template <int R, bool FULL>
__global__ void __launch_bounds__(kAdjThreads) adj_gemm_kernel(AdjPlan ap, const int32_t* __restrict__ x,
                                                             const int32_t* __restrict__ y, uint8_t* ws,
                                                             int vper) {
  extern __shared__ __align__(128) uint8_t sm[];
  const Plan& pl = ap.p;
  const size_t tb = tab_f32_bytes(pl.T, FULL);
  float* tab = reinterpret_cast<float*>(sm);
  float* Ms = reinterpret_cast<float*>(sm + align_up(tb, 128));   // [cols][R]
  const int tile = blockIdx.x, mat = blockIdx.z;
  const float* Mt = reinterpret_cast<const float*>(ws + ap.off_m) + (size_t)mat * ap.cols * ap.rows_pad;
  __shared__ uint64_t tbar;
  Status* st = reinterpret_cast<Status*>(ws + pl.off_status);
  if (threadIdx.x == 0) {
    mbar_init(&tbar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&tbar, (uint32_t)tb);
    bulk_load(tab, ws + pl.off_tab_f32, (uint32_t)tb, &tbar);
  }
  for (int i = threadIdx.x; i < ap.cols * R; i += blockDim.x) {
    const int c = i / R, r = i % R;
    Ms[i] = Mt[(size_t)c * ap.rows_pad + tile * R + r];
  }
  __syncthreads();
  mbar_wait(&tbar, 0, st, 30);
  const int K = pl.K;
  const uint32_t mask = (uint32_t)pl.T - 1u;
  const uint32_t logQ = (uint32_t)pl.logT - 2u;
  const int32_t* ca = mat == 0 ? x : y;   // coordinate of the epilogue operand A'
  const int32_t* cb = mat == 0 ? y : x;   // coordinate of the contraction operand B'
  float* part = reinterpret_cast<float*>(ws + ap.off_part) + ((size_t)mat * ap.row_tiles + tile) * pl.V;
  const long long v0 = (long long)blockIdx.y * vper;
  const long long v1 = min((long long)pl.V, v0 + vper);
  for (long long v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
    const int a = ca[v], b = cb[v];
    float acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.f;
    for (int l = 1; l <= K; ++l) {
      const float2 e = f32_lookup<FULL>(tab, ((uint32_t)l * (uint32_t)b) & mask, logQ);
      const float4* mc = reinterpret_cast<const float4*>(Ms + (size_t)(2 * (l - 1)) * R);
      const float4* ms = reinterpret_cast<const float4*>(Ms + (size_t)(2 * (l - 1) + 1) * R);
#pragma unroll
      for (int q = 0; q < R / 4; ++q) {
        const float4 c4 = mc[q], s4 = ms[q];
        acc[4 * q] = fmaf(c4.x, e.x, fmaf(s4.x, e.y, acc[4 * q]));
        acc[4 * q + 1] = fmaf(c4.y, e.x, fmaf(s4.y, e.y, acc[4 * q + 1]));
        acc[4 * q + 2] = fmaf(c4.z, e.x, fmaf(s4.z, e.y, acc[4 * q + 2]));
        acc[4 * q + 3] = fmaf(c4.w, e.x, fmaf(s4.w, e.y, acc[4 * q + 3]));
      }
    }
    {
      const float fb = (float)b;
      const float4* m1 = reinterpret_cast<const float4*>(Ms + (size_t)(2 * K) * R);
      const float4* mb = reinterpret_cast<const float4*>(Ms + (size_t)(2 * K + 1) * R);
#pragma unroll
      for (int q = 0; q < R / 4; ++q) {
        const float4 c4 = m1[q], b4 = mb[q];
        acc[4 * q] += fmaf(b4.x, fb, c4.x);
        acc[4 * q + 1] += fmaf(b4.y, fb, c4.y);
        acc[4 * q + 2] += fmaf(b4.z, fb, c4.z);
        acc[4 * q + 3] += fmaf(b4.w, fb, c4.w);
      }
    }
    // column dot with A' = (1 | cos, sin of 2 pi k a / T) over this tile's rows
    float out = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = tile * R + r;
      if (row >= ap.rows) break;
      float av;
      if (row == 0) {
        av = 1.f;
      } else {
        const int k = (row + 1) >> 1;
        const float2 e = f32_lookup<FULL>(tab, ((uint32_t)k * (uint32_t)a) & mask, logQ);
        av = (row & 1) ? e.x : e.y;
      }
      out = fmaf(av, acc[r], out);
    }
    part[v] = out;
  }
}

// gx_v = -s_v sum_tiles part[0][tile][v], gy likewise (compensated, tile order).
__global__ void adj_finalize_kernel(AdjPlan ap, const int8_t* __restrict__ s, uint8_t* ws,
                                    float* __restrict__ gx, float* __restrict__ gy) {
  const long long V = ap.p.V;
  // last kernel of the call: the tables built by this call's prep are now valid
  if (blockIdx.x == 0 && threadIdx.x == 0) *reinterpret_cast<unsigned long long*>(ws + kTagOffset) = ap.p.tag;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
    const float* part = reinterpret_cast<const float*>(ws + ap.off_part);
    float out[2];
    for (int m = 0; m < 2; ++m) {
      float hi = 0.f, lo = 0.f;
      for (int t = 0; t < ap.row_tiles; ++t) {
        const float b = part[((size_t)m * ap.row_tiles + t) * V + v];
        const float sum = hi + b, bb = sum - hi;
        lo += (hi - (sum - bb)) + (b - bb);
        hi = sum;
      }
      out[m] = -(float)s[v] * (hi + lo);
    }
    gx[v] = out[0];
    gy[v] = out[1];
  }
}

template <int R, bool FULL>
static cudaError_t launch_adj_gemm(const AdjPlan& ap, const int32_t* x, const int32_t* y, void* ws, cudaStream_t st) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long target = std::max(1LL, (long long)(2 * sms) / (2LL * ap.row_tiles));
  const long long vper = std::max(128LL, (ap.p.V + target - 1) / target);
  const int vb = (int)((ap.p.V + vper - 1) / vper);
  const size_t smem = align_up(tab_f32_bytes(ap.p.T, FULL), 128) + (size_t)ap.cols * R * sizeof(float);
  auto kern = adj_gemm_kernel<R, FULL>;
  ensure_smem(reinterpret_cast<const void*>(kern), smem);
  kern<<<dim3(ap.row_tiles, vb, 2), kAdjThreads, smem, st>>>(ap, x, y, static_cast<uint8_t*>(ws), (int)vper);
  count_launch(1);
  return cudaGetLastError();
}

template <bool FULL>
static cudaError_t launch_adj_gemm_r(const AdjPlan& ap, const int32_t* x, const int32_t* y, void* ws,
                                     cudaStream_t st) {
  switch (ap.R) {
    case 64: return launch_adj_gemm<64, FULL>(ap, x, y, ws, st);
    case 32: return launch_adj_gemm<32, FULL>(ap, x, y, ws, st);
    case 16: return launch_adj_gemm<16, FULL>(ap, x, y, ws, st);
    default: return launch_adj_gemm<8, FULL>(ap, x, y, ws, st);
  }
}

static fcfs_status adjoint_impl(const int32_t* x, const int32_t* y, const int8_t* s, int64_t V, int32_t T, int32_t K,
                                int32_t prec, const float* dF, float* gx, float* gy, void* ws, size_t ws_bytes,
                                cudaStream_t st) {
  if (prec != FCFS_PREC_FP32 && prec != FCFS_PREC_SPLIT_F16) return FCFS_EINVAL;
  if (!dF || (V > 0 && (!x || !y || !s || !gx || !gy))) return FCFS_EINVAL;
  AdjPlan ap;
  fcfs_status r = make_adj_plan(V, T, K, prec, ap);
  if (r != FCFS_OK) return r;
  if ((r = check_ws(ap.p, ws, ws_bytes)) != FCFS_OK) return r;
  if (V == 0) return FCFS_OK;
  if (ap.tc && ap.form != 2 && (!aligned16_ptr(x) || !aligned16_ptr(y))) return FCFS_EINVAL;
  if (ap.form == 2) {
    // pruned FFT along b for every k, then the per-corner dots
    AdjFftArgs ar;
    ar.pl = ap.p;
    ar.pl.vx = x;
    ar.pl.vy = y;
    ar.pl.vsg = s;
    ar.dF = reinterpret_cast<const float2*>(dF);
    ar.logL = ap.fft_logL;
    ar.logP = ap.p.logT - ap.fft_logL;
    ar.off_z = ap.off_z;
    ar.off_side = ap.off_side;
    ar.off_groups = ap.off_groups;
    ar.off_tabs = ap.off_tabs;
    ar.off_dft = ap.off_dft;
    ar.ny_pad = ap.ny_pad;
    ar.gx = gx;
    ar.gy = gy;
    // the grouping on the side stream beside the prep, tables and FFTs (only the
    // dots need it; it leaves out coordinates outside [0, T], so it need not
    // wait for the prep kernel's checks)
    SideStream* ss = side_stream();
    {
      const cudaStream_t gs = ss ? ss->s : st;
      if (ss && side_fork(ss, st) != cudaSuccess) return FCFS_ECUDA;
      KtScope ks("adj_group", gs);
      if (launch_grouping(y, x, V, T, ap.ny_pad, static_cast<uint8_t*>(ws) + ap.off_groups, gs, ar.logP) !=
          cudaSuccess)
        return FCFS_ECUDA;
    }
    {
      KtScope ks("adj_prep", st);
      if (launch_prep(ap.p, ws, false, st) != cudaSuccess) return FCFS_ECUDA;
    }
    {
      KtScope ks("adj_fft", st);
      if (launch_adj_tables(ar, ws, st) != cudaSuccess || launch_adj_fft(ar, ws, st) != cudaSuccess)
        return FCFS_ECUDA;
    }
    if (ss && side_join(ss, st) != cudaSuccess) return FCFS_ECUDA;
    KtScope ks("adj_dot", st);
    if (launch_adj_dot(ar, ws, st) != cudaSuccess) return FCFS_ECUDA;
    return FCFS_OK;
  }
  {
    KtScope ks("adj_prep", st);
    if (launch_prep(ap.p, ws, false, st) != cudaSuccess) return FCFS_ECUDA;
  }
  {
    KtScope ks("adj_coef", st);
    adj_coef_kernel<<<dim3(ap.rows, 2), kAdjThreads, 0, st>>>(ap, reinterpret_cast<const float2*>(dF),
                                                              static_cast<uint8_t*>(ws));
  }
  count_launch(1);
  if (cudaGetLastError() != cudaSuccess) return FCFS_ECUDA;
  if (ap.tc) {
    {
      KtScope ks("adj_pack", st);
      adj_pack_kernel<<<dim3(ap.nrows_pad + 1, 2), 256, 0, st>>>(ap, static_cast<uint8_t*>(ws));
    }
    count_launch(1);
    if (cudaGetLastError() != cudaSuccess) return FCFS_ECUDA;
    const __half* mp = reinterpret_cast<const __half*>(static_cast<uint8_t*>(ws) + ap.off_mp);
    CUtensorMap mhi, mlo;
    if (!encode_f16_2d_sw128(&mhi, mp, ap.kdim_pad, 2ull * ap.nrows_pad, 64, kAdjPairRows / 2) ||
        !encode_f16_2d_sw128(&mlo, mp + (size_t)2 * ap.nrows_pad * ap.kdim_pad, ap.kdim_pad, 2ull * ap.nrows_pad,
                             64, kAdjPairRows / 2))
      return FCFS_ECUDA;
    AdjTcArgs ar;
    ar.pl = ap.p;
    ar.pl.vx = x;
    ar.pl.vy = y;
    ar.pl.vsg = s;
    ar.nrows = 2 * K;
    ar.nrows_pad = ap.nrows_pad;
    ar.kdim_pad = ap.kdim_pad;
    ar.rtiles = ap.row_tiles;
    ar.off_rows = ap.off_rows;
    ar.off_m0 = ap.off_m0;
    ar.off_part = ap.off_part;
    ar.grouped = ap.grouped;
    ar.ny_pad = ap.ny_pad;
    ar.off_groups = ap.off_groups;
    // gx contracts over y, gy over x: group the corners by y and by x
    if (ap.grouped) {
      KtScope ks("adj_group", st);
      if (launch_grouping(y, x, V, T, ap.ny_pad, static_cast<uint8_t*>(ws) + ap.off_groups, st) != cudaSuccess)
        return FCFS_ECUDA;
    }
    KtScope ks(ap.grouped ? "adj_tc_grouped" : "adj_tc", st);
    if (launch_adj_tc(ar, mhi, mlo, ws, st) != cudaSuccess) return FCFS_ECUDA;
  } else {
    KtScope ks("adj_gemm_fp32", st);
    const cudaError_t e =
        ap.p.full ? launch_adj_gemm_r<true>(ap, x, y, ws, st) : launch_adj_gemm_r<false>(ap, x, y, ws, st);
    if (e != cudaSuccess) return FCFS_ECUDA;
  }
  const int blocks = (int)std::min<long long>((V + 255) / 256, 4096);
  KtScope ks("adj_finalize", st);
  adj_finalize_kernel<<<blocks, 256, 0, st>>>(ap, s, static_cast<uint8_t*>(ws), gx, gy);
  count_launch(1);
  if (cudaGetLastError() != cudaSuccess) return FCFS_ECUDA;
  return FCFS_OK;
}

// gE[e] = g_axis[ev0[e]] + g_axis[ev1[e]]: an edge moves both of its corners.
__global__ void edge_chain_kernel(const float* __restrict__ gx, const float* __restrict__ gy,
                                  const int32_t* __restrict__ ev0, const int32_t* __restrict__ ev1,
                                  const int8_t* __restrict__ eaxis, long long E, float* __restrict__ gE) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (long long)gridDim.x * blockDim.x) {
    const float* g = eaxis[e] == 0 ? gx : gy;
    gE[e] = g[ev0[e]] + g[ev1[e]];
  }
}

}  // namespace fcfs

using namespace fcfs;

extern "C" {

fcfs_status fcfs_edge_chain(const float* gx, const float* gy, const int32_t* ev0, const int32_t* ev1,
                            const int8_t* eaxis, int64_t E, float* gE, void* stream) {
  if (E < 0) return FCFS_EINVAL;
  if (E == 0) return FCFS_OK;
  if (!gx || !gy || !ev0 || !ev1 || !eaxis || !gE) return FCFS_EINVAL;
  const int blocks = (int)std::min<long long>((E + 255) / 256, 4096);
  edge_chain_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(gx, gy, ev0, ev1, eaxis, E, gE);
  count_launch(1);
  return cudaGetLastError() == cudaSuccess ? FCFS_OK : FCFS_ECUDA;
}

size_t fcfs_adjoint_workspace_size(int64_t V, int32_t T, int32_t K, int32_t prec) {
  if (prec != FCFS_PREC_FP32 && prec != FCFS_PREC_SPLIT_F16) return 0;
  AdjPlan ap;
  if (make_adj_plan(V, T, K, prec, ap) != FCFS_OK) return 0;
  return ap.total;
}

int32_t fcfs_adjoint_grouped(int64_t V, int32_t T, int32_t K, int32_t prec) {
  if (prec != FCFS_PREC_FP32 && prec != FCFS_PREC_SPLIT_F16) return -1;
  AdjPlan ap;
  if (make_adj_plan(V, T, K, prec, ap) != FCFS_OK) return -1;
  return ap.form;
}

fcfs_status fcfs_adjoint(const int32_t* x, const int32_t* y, const int8_t* s, int64_t V, int32_t T, int32_t K,
                         int32_t prec, const float* dF, float* gx, float* gy, void* workspace, size_t ws_bytes,
                         void* stream) {
  return adjoint_impl(x, y, s, V, T, K, prec, dF, gx, gy, workspace, ws_bytes, static_cast<cudaStream_t>(stream));
}


}  // extern "C"
