// Plain FP32 path: the quarter-plane contraction on CUDA cores, one FMA per
// vertex-coefficient term.
//
//   P[m, n] = sum_v A[m, v] B[n, v]   over the block's vertex range,
//   A[2i, v] = s_v cos(2 pi k_i x_v / T),  A[2i+1, v] = s_v sin(2 pi k_i x_v / T),
//   B[2j, v] =     cos(2 pi l_j y_v / T),  B[2j+1, v] =     sin(2 pi l_j y_v / T),
//
// with k_i = i + 1, l_j = j + 1.  The 2 x 2 blocks (CC, CS; SC, SS) of P give
// G(k, +-l) in the reduce kernel.  COS (continuous cosine series): row m holds
// s_v sin(2 pi (m + 1) x_v / T) alone (columns likewise with y), so the row pair
// (2i, 2i+1) of a tile takes the sines of frequencies 2i + 1 and 2i + 2.
// Operands are generated per 32-vertex chunk
// into shared memory from the FP32 table (exact integer phase), never stored
// to global memory.  Each 256-thread block owns a 128 x 128 tile of P and one
// vertex split; each thread accumulates an 8 x 8 register tile in FP32.
#include "fcfs_launch.cuh"

namespace fcfs {

constexpr int kSB = 128;       // tile rows = tile columns
constexpr int kSChunk = 32;    // vertices per chunk
constexpr int kSThreads = 256;

template <bool FULL, bool COS = false>
__global__ void __launch_bounds__(kSThreads, 2) gemm_simt_kernel(Plan pl, const int32_t* __restrict__ x,
                                                                const int32_t* __restrict__ y,
                                                                const int8_t* __restrict__ s, uint8_t* ws) {
  griddep_wait();   // launched behind the prep kernel (programmatic dependent launch)
  extern __shared__ __align__(128) uint8_t sm[];
  const size_t tb = tab_f32_bytes(pl.T, FULL);
  float* tab = reinterpret_cast<float*>(sm);
  float* As = reinterpret_cast<float*>(sm + tb);           // [kSChunk][kSB]
  float* Bs = As + kSChunk * kSB;                          // [kSChunk][kSB]
  int* vx = reinterpret_cast<int*>(Bs + kSChunk * kSB);    // [kSChunk]
  int* vy = vx + kSChunk;
  float* vs = reinterpret_cast<float*>(vy + kSChunk);

  const int tid = threadIdx.x;
  __shared__ uint64_t tbar;
  if (pl.batch && blockIdx.x >= reinterpret_cast<const int*>(ws + pl.off_units)[pl.n_clips]) return;
  Status* st = reinterpret_cast<Status*>(ws + pl.off_status);
  if (tid == 0) {   // the table arrives by one bulk copy
    mbar_init(&tbar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&tbar, (uint32_t)tb);
    bulk_load(tab, ws + pl.off_tab_f32, (uint32_t)tb, &tbar);
  }
  __syncthreads();
  mbar_wait(&tbar, 0, st, 21);
  const Unit U = unit_of_block(pl, ws, kSB, kSB);
  if (!U.live) return;
  const int tm = U.tm, tn = U.tn;
  const int kbase = tm * (kSB / 2) + 1;    // first k of the tile's rows
  const int lbase = tn * (kSB / 2) + 1;
  const long long v0 = U.v0, v1 = U.v1;
  const uint32_t mask = (uint32_t)pl.T - 1u;
  const uint32_t logQ = (uint32_t)pl.logT - 2u;

  const int tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  // generation mapping: row pair gp = tid & 63, vertices gv = (tid >> 6) + 4 t
  const int gp = tid & 63;
  const int gv = tid >> 6;
  const uint32_t kg = (uint32_t)(kbase + gp), lg = (uint32_t)(lbase + gp);

  for (long long b = v0; b < v1; b += kSChunk) {
    __syncthreads();
    if (tid < kSChunk) {
      const long long v = b + tid;
      const bool ok = v < v1;
      const int xv = ok ? x[v] : 0, yv = ok ? y[v] : 0, sv = ok ? s[v] : 0;
      vx[tid] = xv;
      vy[tid] = yv;
      vs[tid] = (float)sv;
      if (ok && pl.bin_in_gemm && tm == 0 && tn == 0) bin_corner(pl, ws, U.clip, xv, yv, sv);
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kSChunk / 4; ++t) {
      const int j = gv + 4 * t;
      const float sg = vs[j];
      if (COS) {
        const uint32_t kc = (uint32_t)(tm * kSB + 2 * gp + 1), lc = (uint32_t)(tn * kSB + 2 * gp + 1);
        const float a0 = f32_lookup<FULL>(tab, (kc * (uint32_t)vx[j]) & mask, logQ).y;
        const float a1 = f32_lookup<FULL>(tab, ((kc + 1u) * (uint32_t)vx[j]) & mask, logQ).y;
        const float b0 = f32_lookup<FULL>(tab, (lc * (uint32_t)vy[j]) & mask, logQ).y;
        const float b1 = f32_lookup<FULL>(tab, ((lc + 1u) * (uint32_t)vy[j]) & mask, logQ).y;
        reinterpret_cast<float2*>(As + j * kSB)[gp] = make_float2(sg * a0, sg * a1);
        reinterpret_cast<float2*>(Bs + j * kSB)[gp] = make_float2(b0, b1);
      } else {
        const float2 a = f32_lookup<FULL>(tab, (kg * (uint32_t)vx[j]) & mask, logQ);
        const float2 bb = f32_lookup<FULL>(tab, (lg * (uint32_t)vy[j]) & mask, logQ);
        reinterpret_cast<float2*>(As + j * kSB)[gp] = make_float2(sg * a.x, sg * a.y);
        reinterpret_cast<float2*>(Bs + j * kSB)[gp] = bb;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int j = 0; j < kSChunk; ++j) {
      const float4 a0 = reinterpret_cast<const float4*>(As + j * kSB)[ty];
      const float4 a1 = reinterpret_cast<const float4*>(As + j * kSB + 64)[ty];
      const float4 b0 = reinterpret_cast<const float4*>(Bs + j * kSB)[tx];
      const float4 b1 = reinterpret_cast<const float4*>(Bs + j * kSB + 64)[tx];
      const float ar[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float br[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(ar[r], br[c], acc[r][c]);
    }
  }

  // epilogue: rows ty*4 + r (r < 4) and 64 + ty*4 + r - 4; columns likewise with tx
  const int M2 = pl.M2;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int mr = r < 4 ? ty * 4 + r : 64 + ty * 4 + r - 4;
    const int m = tm * kSB + mr;
    if (m >= M2) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int nr = h * 64 + tx * 4;
      const int n = tn * kSB + nr;
      float* dst = U.P + (size_t)mr * U.ld + nr;
      if (n + 3 < M2 && (M2 & 3) == 0) {
        *reinterpret_cast<float4*>(dst) =
            make_float4(acc[r][4 * h], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
      } else {
        for (int c = 0; c < 4; ++c)
          if (n + c < M2) dst[c] = acc[r][4 * h + c];
      }
    }
  }
}

cudaError_t launch_gemm_simt(const Plan& pl, const int32_t* x, const int32_t* y, const int8_t* s, void* ws,
                             cudaStream_t st) {
  if (pl.splits == 0) return cudaSuccess;
  const size_t smem = tab_f32_bytes(pl.T, pl.full) + 2 * kSChunk * kSB * sizeof(float) + 3 * kSChunk * 4;
  dim3 grid = pl.batch ? dim3(pl.splits, 1) : dim3(pl.tiles_m * pl.tiles_n, pl.splits);
  auto kern = pl.cosine ? (pl.full ? gemm_simt_kernel<true, true> : gemm_simt_kernel<false, true>)
                        : (pl.full ? gemm_simt_kernel<true> : gemm_simt_kernel<false>);
  ensure_smem(reinterpret_cast<const void*>(kern), smem);
  return launch_after(kern, grid, dim3(kSThreads), smem, st, pl, x, y, s, static_cast<uint8_t*>(ws));
}

}  // namespace fcfs
