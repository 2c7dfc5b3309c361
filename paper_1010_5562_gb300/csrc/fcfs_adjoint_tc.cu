// Split-FP16 tensor-core adjoint: the contraction of the adjoint (see
// fcfs_adjoint.cu for the formulation) on tcgen05.
//
// For matrix m (0: gx, 1: gy) and corner v with contraction coordinate b
// (y for gx, x for gy) and epilogue coordinate a (x for gx, y for gy):
//   Z[r, v] = sum_c M'[r, c] B'[c, v],   part[m][tile][v] = sum_{r in tile} A'[r, v] Z[r, v],
// B'[., v] = (cos, sin of 2 pi l b / T for l = 1..K, 1, b / T, 0 ...),
// A'[., v] = (cos, sin of 2 pi k a / T for k = 1..K, 1): the rows are ordered
// (k=1 cos, k=1 sin, ..., k=K sin, k=0).
//
// The GEMM runs with the corners as the MMA's M dimension: a CTA holds 256
// corners (two M = 128 accumulators in TMEM, lane = corner) against BNR rows
// of M' (N), contracted over the columns c in chunks of 64.  M' is packed once
// per call as FP16 hi + lo with a power-of-two scale per row (so that no entry
// overflows FP16) and streamed by TMA in 128-byte swizzled K-major tiles; B' is
// generated on chip like the forward operands (integer phase, table anchor,
// angle addition over runs of 8 frequencies, hi = rn(v), lo = rn(v - hi)).
// Products hi*hi go to accumulator D1, hi*lo + lo*hi to D2.  The epilogue is a
// per-thread dot: the thread of TMEM lane v multiplies its row of D1 + D2 (one
// value per M' row) by A'[., v], generated along k the same way, and writes the
// partial of this row tile; the finalize kernel sums the row tiles.
#include <algorithm>

#include "fcfs_common.cuh"

namespace fcfs {

namespace {

constexpr int kVT = 256;         // corners per CTA (two M = 128 sub-tiles)
constexpr int kAC = 64;          // columns per chunk = one 128-byte swizzle row of FP16
constexpr int kGenThreadsA = 256;   // one generator thread per corner
constexpr int kThreadsA = kGenThreadsA + 64;

template <int BNR>
struct AdjTcLayout {
  static constexpr int kATile = 128 * 128;   // one M = 128 sub-tile, FP16 (hi or lo)
  static constexpr int kBTile = BNR * 128;
  // A0_hi, A0_lo, A1_hi, A1_lo, B_hi, B_lo
  static constexpr int kStage = 4 * kATile + 2 * kBTile;
  static constexpr int kStages = 2;
  static constexpr int kOps = kStages * kStage;
};

__device__ __forceinline__ void st_shared_v4a(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ uint32_t h2bits(__half2 h) {
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}
__device__ __forceinline__ void split_pair(float v0, float v1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(v0, v1);
  const float2 hf = __half22float2(h);
  hi = h2bits(h);
  lo = h2bits(__floats2half2_rn(v0 - hf.x, v1 - hf.y));
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int32_t c0, int32_t c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

template <int BNR, bool FULL>
__global__ void __launch_bounds__(kThreadsA, 1)
    adj_tc_kernel(const __grid_constant__ CUtensorMap mhi, const __grid_constant__ CUtensorMap mlo, AdjTcArgs ar,
                  uint8_t* ws) {
  using L = AdjTcLayout<BNR>;
  constexpr int GW = kGenThreadsA / 32;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* sm = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  const Plan& pl = ar.pl;
  const size_t tb = tab_f32_bytes(pl.T, FULL);
  uint8_t* ops = sm;
  float* tab = reinterpret_cast<float*>(sm + L::kOps);
  float* rscale = reinterpret_cast<float*>(sm + L::kOps + align_up(tb, 128));   // BNR row scales
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + L::kOps + align_up(tb, 128) + BNR * 4);
  uint64_t* full = bars;                 // [kStages]: generated A and loaded B of a chunk
  uint64_t* empty = full + L::kStages;   // [kStages]: the chunk's MMAs completed
  uint64_t* accfull = empty + L::kStages;
  uint64_t* tabbar = accfull + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tabbar + 1);

  Status* st = reinterpret_cast<Status*>(ws + pl.off_status);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int vt = blockIdx.x, rt = blockIdx.y, mat = blockIdx.z;
  const long long vbase = (long long)vt * kVT;
  const int nrows = ar.nrows;
  const int r0 = rt * BNR;
  const int nr = min(BNR, nrows - r0);
  const int nmma = (nr + 15) / 16 * 16;   // MMA N: this tile's rows rounded up to 16
  const int nch = ar.kdim_pad / kAC;

  if (tid == kGenThreadsA + 32) {
    for (int i = 0; i < L::kStages; ++i) {
      mbar_init(&full[i], kGenThreadsA + 1);   // every generator thread and the TMA thread
      mbar_init(&empty[i], 1);
    }
    mbar_init(accfull, 1);
    mbar_init(tabbar, 1);
    fence_mbar_init();
  }
  if (warp == GW) {
    tmem_alloc(tmem_slot, 4 * BNR);   // sub-tile s: D1 at 2 s BNR, D2 at 2 s BNR + BNR
    tmem_relinquish();
  }
  for (int i = tid; i < BNR; i += blockDim.x)
    rscale[i] = i < nr ? __ldg(reinterpret_cast<const float*>(ws + ar.off_scale) + (size_t)mat * nrows + r0 + i)
                       : 0.f;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t mask = (uint32_t)pl.T - 1u;
  const uint32_t logQ = (uint32_t)pl.logT - 2u;
  const int K = pl.K;

  if (warp == GW + 1) {
    // ---------------- table copy and M' tiles (TMA) ----------------
    if (lane == 0) {
      prefetch_tensormap(&mhi);
      prefetch_tensormap(&mlo);
      mbar_arrive_expect_tx(tabbar, (uint32_t)tb);
      bulk_load(tab, ws + pl.off_tab_f32, (uint32_t)tb, tabbar);
      int j = 0;
      for (; j < nch; ++j) {
        const int s = j % L::kStages;
        const uint32_t ph = (uint32_t)(j / L::kStages) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, st, 40)) break;
        uint8_t* stage = ops + (size_t)s * L::kStage;
        mbar_arrive_expect_tx(&full[s], 2u * L::kBTile);
        // rows past the matrix read as zeros; coordinate 2 selects (matrix)
        tma_load_2d(stage + 4 * L::kATile, &mhi, j * kAC, mat * ar.nrows_pad + r0, &full[s]);
        tma_load_2d(stage + 4 * L::kATile + L::kBTile, &mlo, j * kAC, mat * ar.nrows_pad + r0, &full[s]);
      }
      // drain: every issued copy has landed before the CTA may exit
      for (int q = max(0, j - L::kStages); q < j; ++q)
        mbar_wait(&full[q % L::kStages], (uint32_t)(q / L::kStages) & 1u, st, 41);
      mbar_wait(tabbar, 0, st, 42);
    }
  } else if (warp == GW) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_f16_f32(128, nmma);
      const uint32_t ops_a = smem_u32(ops);
      for (int j = 0; j < nch; ++j) {
        const int s = j % L::kStages;
        const uint32_t ph = (uint32_t)(j / L::kStages) & 1u;
        if (!mbar_wait(&full[s], ph, st, 43)) break;
        tc_fence_after();
        const uint32_t base = ops_a + s * L::kStage;
        const uint32_t bhi = base + 4 * L::kATile, blo = bhi + L::kBTile;
#pragma unroll
        for (int ks = 0; ks < kAC / 16; ++ks) {
          const uint32_t o = ks * 32;
          const uint64_t dbh = sdesc_sw128(bhi + o), dbl = sdesc_sw128(blo + o);
#pragma unroll
          for (int sub = 0; sub < 2; ++sub) {
            const uint32_t ahi = base + sub * 2 * L::kATile, alo = ahi + L::kATile;
            const uint64_t dah = sdesc_sw128(ahi + o), dal = sdesc_sw128(alo + o);
            const uint32_t d1 = tmem + (uint32_t)(sub * 2 * BNR), d2 = d1 + BNR;
            tc_mma_f16(d1, dah, dbh, idesc, (j | ks) != 0);
            tc_mma_f16(d2, dah, dbl, idesc, (j | ks) != 0);
            tc_mma_f16(d2, dal, dbh, idesc, 1);
          }
        }
        tc_commit(&empty[s]);
      }
      tc_commit(accfull);
    }
  } else {
    // ---------------- generators: one thread per corner ----------------
    // Corner i = tid of the CTA's 256 (sub-tile i / 128, row i % 128).  A chunk
    // of 64 columns holds l = 32 j + 1 .. 32 j + 32 as (cos, sin) pairs, the
    // last chunks also the columns 1 and b / T and zero padding.
    const int sub = tid >> 7, row = tid & 127;
    const long long v = vbase + tid;
    const bool live = v < pl.V;
    const int32_t* cbp = mat == 0 ? pl.vy : pl.vx;
    const uint32_t b = live ? (uint32_t)__ldg(cbp + v) : 0u;
    const uint32_t ops_a = smem_u32(ops);
    bool ok = mbar_wait(tabbar, 0, st, 44);
    const float2 w = f32_lookup<FULL>(tab, b & mask, logQ);   // step cos/sin(2 pi b / T)
    for (int j = 0; ok && j < nch; ++j) {
      const int s = j % L::kStages;
      const uint32_t ph = (uint32_t)(j / L::kStages) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u, st, 45)) break;
      const uint32_t hi_row = ops_a + s * L::kStage + sub * 2 * L::kATile + (uint32_t)row * 128u;
#pragma unroll
      for (int run = 0; run < 4; ++run) {   // 8 frequencies = 16 columns = two 16-byte chunks
        const int l0 = 32 * j + 8 * run + 1;   // first frequency of the run
        uint32_t hv[8], lv[8];
        if (l0 + 7 <= K) {
          const float2 an = f32_lookup<FULL>(tab, (uint32_t)l0 * b & mask, logQ);
          float c = an.x, sn = an.y;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            float c1 = fmaf(c, w.x, -(sn * w.y)), s1 = fmaf(sn, w.x, c * w.y);
            split_pair(c, sn, hv[2 * t], lv[2 * t]);
            c = c1;
            sn = s1;
            c1 = fmaf(c, w.x, -(sn * w.y));
            s1 = fmaf(sn, w.x, c * w.y);
            split_pair(c, sn, hv[2 * t + 1], lv[2 * t + 1]);
            c = c1;
            sn = s1;
          }
        } else {
          // the run crosses the end of the frequencies: direct lookups, then
          // the columns 1 and b / T, then zeros
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int l = l0 + t;
            float c = 0.f, sn = 0.f;
            if (l <= K) {
              const float2 e = f32_lookup<FULL>(tab, (uint32_t)l * b & mask, logQ);
              c = e.x;
              sn = e.y;
            } else if (l == K + 1) {
              c = live ? 1.f : 0.f;
              sn = (float)b * ar.inv_T;
            }
            split_pair(c, sn, hv[t], lv[t]);
          }
        }
        if (!live) {
#pragma unroll
          for (int t = 0; t < 8; ++t) hv[t] = lv[t] = 0u;
        }
        const uint32_t c0 = (uint32_t)(2 * run), c1 = c0 + 1;
        const uint32_t o0 = (c0 ^ (uint32_t)(row & 7)) << 4, o1 = (c1 ^ (uint32_t)(row & 7)) << 4;
        st_shared_v4a(hi_row + o0, hv[0], hv[1], hv[2], hv[3]);
        st_shared_v4a(hi_row + o1, hv[4], hv[5], hv[6], hv[7]);
        st_shared_v4a(hi_row + L::kATile + o0, lv[0], lv[1], lv[2], lv[3]);
        st_shared_v4a(hi_row + L::kATile + o1, lv[4], lv[5], lv[6], lv[7]);
      }
      fence_proxy_async_smem();
      mbar_arrive(&full[s]);
    }

    // ---------------- epilogue: per-corner dot with A' ----------------
    // warp w drains TMEM lanes 32 (w mod 4) .. of sub-tile w / 4: the thread
    // of lane row holds Z[r, corner] for this tile's rows r
    const bool acc_ok = __all_sync(0xffffffffu, mbar_wait(accfull, 0, st, 46) ? 1 : 0) != 0;
    tc_fence_after();
    const int32_t* cap = mat == 0 ? pl.vx : pl.vy;
    const uint32_t a = live ? (uint32_t)__ldg(cap + v) : 0u;
    const float2 wa = f32_lookup<FULL>(tab, a & mask, logQ);
    const uint32_t lane_base = ((uint32_t)(warp & 3) * 32u) << 16;
    float outv = 0.f;
    if (acc_ok) {
      for (int cb = 0; cb < nmma; cb += 32) {   // 32 rows = 16 frequencies (or the k = 0 row)
        uint32_t d1[32], d2[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(sub * 2 * BNR + cb), d1);
        tmem_ld32(tmem + lane_base + (uint32_t)(sub * 2 * BNR + BNR + cb), d2);
        tmem_wait_ld();
        // rows r0 + cb + 2 i (cos) and + 1 (sin) of frequency k = (r0 + cb) / 2 + 1 + i
        const int kb = (r0 + cb) / 2 + 1;
        float c = 0.f, sn = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int rr = cb + 2 * i;   // row within the tile
          if (i % 8 == 0) {            // anchor of a run of 8 frequencies
            const float2 an = f32_lookup<FULL>(tab, (uint32_t)(kb + i) * a & mask, logQ);
            c = an.x;
            sn = an.y;
          }
          const int rg = r0 + rr;      // global row
          if (rr < nr) {
            const float z0 = (__uint_as_float(d1[2 * i]) + __uint_as_float(d2[2 * i])) * rscale[rr];
            const float av0 = rg < 2 * K ? c : 1.f;   // the last row is k = 0
            outv = fmaf(av0, z0, outv);
          }
          if (rr + 1 < nr && rg + 1 < 2 * K) {
            const float z1 = (__uint_as_float(d1[2 * i + 1]) + __uint_as_float(d2[2 * i + 1])) * rscale[rr + 1];
            outv = fmaf(sn, z1, outv);
          }
          const float c1 = fmaf(c, wa.x, -(sn * wa.y)), s1 = fmaf(sn, wa.x, c * wa.y);
          c = c1;
          sn = s1;
        }
      }
    }
    if (live) reinterpret_cast<float*>(ws + ar.off_part)[((size_t)mat * ar.rtiles + rt) * pl.V + v] = outv;
  }

  tc_fence_before();
  __syncthreads();
  if (warp == GW) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 4 * BNR);
  }
}

template <int BNR, bool FULL>
cudaError_t launch_adj_tc_t(const AdjTcArgs& ar, const CUtensorMap& mhi, const CUtensorMap& mlo, void* ws,
                            cudaStream_t st) {
  using L = AdjTcLayout<BNR>;
  const size_t smem = 1024 + L::kOps + align_up(tab_f32_bytes(ar.pl.T, FULL), 128) + BNR * 4 + 256;
  auto kern = adj_tc_kernel<BNR, FULL>;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((ar.pl.V + kVT - 1) / kVT), (unsigned)ar.rtiles, 2);
  kern<<<grid, kThreadsA, smem, st>>>(mhi, mlo, ar, static_cast<uint8_t*>(ws));
  count_launch(1);
  return cudaGetLastError();
}

}  // namespace

int adj_tc_rows_per_tile(int full) { return full ? 128 : 64; }

cudaError_t launch_adj_tc(const AdjTcArgs& ar, const CUtensorMap& mhi, const CUtensorMap& mlo, void* ws,
                          cudaStream_t st) {
  if (ar.pl.full) return launch_adj_tc_t<128, true>(ar, mhi, mlo, ws, st);
  return launch_adj_tc_t<64, false>(ar, mhi, mlo, ws, st);
}

}  // namespace fcfs
