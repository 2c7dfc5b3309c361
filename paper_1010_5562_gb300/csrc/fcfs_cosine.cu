// Continuous cosine series of a clip (the cosine extension of FCFS named in
// the concluding section):
//
//   C(k, l) = integral over the image of cos(pi k x / T) cos(pi l y / T) dx dy,  0 <= k, l <= K.
//
// The tail primitive of Lemma polyip, now of the cosine, makes every polygon
// the signed sum of upper-right quadrants at its corners, so that
// C = Xc diag(s) Yc^T with Xc_0(a) = T - a and Xc_k(a) = -(T / (pi k)) sin(pi k a / T).
// For a balanced corner set (every vertical and horizontal line carries signs
// summing to zero) the constant parts of the tails cancel as they do in
// Prop. CFT, which leaves
//   C(0, 0) = the exact area (Eq. Fdc),
//   C(k, 0) = (T / (pi k)) sum_v s_v y_v sin(pi k x_v / T),   C(0, l) with x and y swapped,
//   C(k, l) = T^2 / (pi^2 k l) sum_v s_v sin(pi k x_v / T) sin(pi l y_v / T).
// Written with the period T2 = 2T, sin(pi k a / T) = sin(2 pi k a / T2): the axis
// lines are the sine halves of the axis-line DFT at period T2 (Steps 2-3), and
// the off-axis block is the quarter-plane contraction at period T2 with its
// sine rows only (M = N = K instead of 2K: a quarter of the Fourier block's
// terms).  One call: prep (tables at period T2), the contraction (tensor cores
// on CTA pairs, or the plain FP32 kernel), the axis DFT, and the reduction below.
#include "fcfs_epilogue.cuh"
#include "fcfs_launch.cuh"

namespace fcfs {

fcfs_status make_plan_cosine(int64_t V, int32_t T, int32_t K, int32_t prec, Plan& pl);
fcfs_status check_ws(const Plan& pl, void* ws, size_t ws_bytes);

// One thread per (k, l) of the (K + 1) x (K + 1) block; pl.T is T2 = 2T.
//  (0, 0): the exact area.
//  (k, 0): (T2 / (2 pi k)) Sx(k), Sx(k) = sum_n bin_x[n] sin(2 pi k n / T2) from the
//          fixed-point axis sums (exact integers times 2^-q); (0, l) from Sy.
//  k, l >= 1: T2^2 / (4 pi^2 k l) times the sum over the splits, in split order,
//          of the FP32 partials P[k - 1][l - 1], each addition an error-free
//          TwoSum with the rounding errors carried in a second float.
__global__ void cosine_reduce_kernel(Plan pl, uint8_t* ws, float* __restrict__ C,
                                     long long* __restrict__ area_out) {
  griddep_wait();   // launched behind the axis DFT (programmatic dependent launch)
  const int K = pl.K;
  const long long n1 = (long long)K + 1;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx == 0) *reinterpret_cast<unsigned long long*>(ws + kTagOffset) = pl.tag;
  if (idx >= n1 * n1) return;
  const int k = (int)(idx / n1), l = (int)(idx % n1);
  const long long* acc = reinterpret_cast<const long long*>(ws + pl.off_axis);
  if (k == 0 && l == 0) {
    const long long a = __ldcg(&acc[4 * K]);
    *area_out = a;
    C[0] = (float)a;
    return;
  }
  if (k == 0 || l == 0) {
    const int f = k ? k : l;
    const long long Sq = __ldcg(&acc[(k ? K : 3 * K) + f - 1]);   // the sine sum of the row or column line
    const double g = (double)pl.T / (2.0 * CUDART_PI * f);
    C[idx] = (float)(g * ldexp((double)Sq, -pl.fixq));
    return;
  }
  const int M2 = pl.M2;
  const float* P = reinterpret_cast<const float*>(ws + pl.off_part) + (size_t)(k - 1) * M2 + (l - 1);
  const size_t stride = (size_t)M2 * M2;
  const int S = pl.splits;
  CSum ss{0.f, 0.f};
  constexpr int kBatch = 8;   // a batch of independent loads ahead of the dependent sums
  for (int sp0 = 0; sp0 < S; sp0 += kBatch) {
    float r[kBatch];
#pragma unroll
    for (int b = 0; b < kBatch; ++b)
      if (sp0 + b < S) r[b] = __ldcs(P + (size_t)(sp0 + b) * stride);
#pragma unroll
    for (int b = 0; b < kBatch; ++b)
      if (sp0 + b < S) csum_add(ss, r[b]);
  }
  const float a = pl.quad_scale / ((float)k * (float)l);   // T2^2 / (4 pi^2 k l)
  C[idx] = a * (ss.hi + ss.lo);
}

static cudaError_t launch_cosine_reduce(const Plan& pl, void* ws, float* C, int64_t* area, cudaStream_t st) {
  const long long n = (long long)(pl.K + 1) * (pl.K + 1);
  ensure_smem(reinterpret_cast<const void*>(cosine_reduce_kernel), 0);
  return launch_after(cosine_reduce_kernel, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st, pl,
                      static_cast<uint8_t*>(ws), C, reinterpret_cast<long long*>(area));
}

}  // namespace fcfs

using namespace fcfs;

extern "C" {

size_t fcfs_cosine_workspace_size(int64_t V, int32_t T, int32_t K, int32_t prec) {
  Plan pl;
  if (make_plan_cosine(V, T, K, prec, pl) != FCFS_OK) return 0;
  return pl.total;
}

fcfs_status fcfs_cosine(const int32_t* x, const int32_t* y, const int8_t* s, int64_t V, int32_t T, int32_t K,
                        int32_t prec, uint32_t flags, float* C_out, int64_t* area_out, void* workspace,
                        size_t ws_bytes, void* stream) {
  auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (!C_out || !area_out || flags != 0) return FCFS_EINVAL;
  if (V > 0 && (!x || !y || !s || !a16(x) || !a16(y) || !a16(s))) return FCFS_EINVAL;
  Plan pl;
  fcfs_status r = make_plan_cosine(V, T, K, prec, pl);
  if (r != FCFS_OK) return r;
  if ((r = check_ws(pl, workspace, ws_bytes)) != FCFS_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  pl.vx = x;
  pl.vy = y;
  pl.vsg = s;
  pl.bin_in_gemm = 1;   // the contraction bins the corners for the axis lines
  if (launch_prep(pl, workspace, false, st) != cudaSuccess) return FCFS_ECUDA;
  const VertexMaps mp{};
  const cudaError_t e = prec == FCFS_PREC_SPLIT_F16 ? launch_gemm_tc(pl, mp, workspace, st)
                                                   : launch_gemm_simt(pl, x, y, s, workspace, st);
  if (e != cudaSuccess) return FCFS_ECUDA;
  if (launch_axis(pl, x, y, s, workspace, false, st) != cudaSuccess) return FCFS_ECUDA;
  if (launch_cosine_reduce(pl, workspace, C_out, area_out, st) != cudaSuccess) return FCFS_ECUDA;
  return FCFS_OK;
}

}  // extern "C"
